"""Batched segmented sorting: the 4096-array workload shape, capture of the
one-launch call into a CUDA graph, and the autotuner."""
import os

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import gpu_util  # noqa: E402
import paper_2401_00710_gb300 as dts  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = gpu_util.GpuSort(torch)
    yield g
    g.reset_options()
    g.ws = None
    g.close()


def c4_input(total, seed=1, nseg=4096, hi=1e6):
    off, fam = gen.segmented_layout(nseg=nseg, lo=100, hi=hi, seed=seed, total=total)
    n = int(off[-1])
    keys = np.empty(n, dtype=np.uint32)
    vals = np.empty(n, dtype=np.uint32)
    gen.fill_segmented_u32(keys.ctypes.data, vals.ctypes.data, off, fam, seed=seed)
    return keys, vals, off


def test_c4_shape_parity(G):
    # 4096 arrays, log-uniform sizes, each uniform or Zipf(1.0): scaled to
    # 2*10^7 records so that the oracle finishes in seconds
    keys, vals, off = c4_input(2e7)
    gk, gv = G.sort(keys, vals, off)
    ek, ev = oracle.stable_sort_segmented(keys, vals, off)
    gpu_util.assert_same(gk, gv, ek, ev)


def test_c4_key_only_and_u64(G):
    keys, vals, off = c4_input(3e6, seed=2, nseg=700)
    gk, _ = G.sort(keys, None, off)
    ek, _ = oracle.stable_sort_segmented(keys, None, off)
    gpu_util.assert_same(gk, None, ek, None)
    k64 = (keys.astype(np.uint64) << np.uint64(20)) ^ gen.family("uniform", len(keys),
                                                                 np.uint64, seed=3)
    v64 = vals.astype(np.uint64)
    gk, gv = G.sort(k64, v64, off)
    ek, ev = oracle.stable_sort_segmented(k64, v64, off)
    gpu_util.assert_same(gk, gv, ek, ev)


def test_graph_capture_and_replay(G):
    # the segmented call is one memset + one cooperative launch with no host
    # synchronisation, so it can be captured once and replayed
    keys, vals, off = c4_input(4e6, seed=5, nseg=1024)
    n = len(keys)
    pk = gpu_util.to_dev(keys, torch, G.dev)
    pv = gpu_util.to_dev(vals, torch, G.dev)
    k = pk.clone()
    v = pv.clone()
    o = torch.from_numpy(off).to(G.dev)
    G.workspace(dts.DTSORT_OP_U32_KV, n, len(off) - 1)  # allocate before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = G.launch(k, v, n, dts.DTSORT_OP_U32_KV, o, len(off) - 1)
    assert st == dts.DTSORT_OK
    ek, ev = oracle.stable_sort_segmented(keys, vals, off)
    for _ in range(2):
        k.copy_(pk)
        v.copy_(pv)
        graph.replay()
        torch.cuda.synchronize()
        assert G.device_status() == dts.DTSORT_OK
        gpu_util.assert_same(gpu_util.from_dev(k, np.uint32), gpu_util.from_dev(v, np.uint32),
                             ek, ev)


def test_autotune_picks_a_setting_and_keeps_output(G, tmp_path, monkeypatch):
    cache = tmp_path / "tune.tsv"
    monkeypatch.setenv("DTSORT_AUTOTUNE_CACHE", str(cache))
    keys, vals, off = c4_input(3e6, seed=7, nseg=512)
    n = len(keys)
    k = gpu_util.to_dev(keys, torch, G.dev)
    v = gpu_util.to_dev(vals, torch, G.dev)
    o = torch.from_numpy(off).to(G.dev)
    op = dts.DTSORT_OP_U32_KV
    sb = dts.dtsort_autotune_scratch_bytes(G.h, op, n, len(off) - 1)
    scratch = torch.empty(sb, dtype=torch.uint8, device=G.dev)
    s = torch.cuda.current_stream(G.dev).cuda_stream
    st, best = dts.dtsort_autotune(G.h, op, k.data_ptr(), v.data_ptr(), o.data_ptr(),
                                   len(off) - 1, n, scratch.data_ptr(), sb, s)
    assert st == dts.DTSORT_OK, dts.status_string(st)
    assert best.gamma_max in (7, 8, 9) and best.block_tiles in (4, 8)
    # the caller's arrays were only read
    np.testing.assert_array_equal(gpu_util.from_dev(k, np.uint32), keys)
    text = cache.read_text()
    assert len(text.strip().splitlines()) == 1
    # a sort that consults the cache gives the same output
    G.set_options(autotune=1)
    gk, gv = G.sort(keys, vals, off)
    ek, ev = oracle.stable_sort_segmented(keys, vals, off)
    gpu_util.assert_same(gk, gv, ek, ev)
    G.reset_options()


def test_block_tiles_option(G):
    keys = gen.family("zipf1.0", 2_000_003, np.uint32, seed=8)
    vals = gen.iota(len(keys), np.uint32)
    ek, ev = oracle.stable_sort(keys, vals)
    for bt in (1, 3, 8):
        G.set_options(block_tiles=bt)
        gk, gv = G.sort(keys, vals)
        gpu_util.assert_same(gk, gv, ek, ev)
    G.reset_options()
