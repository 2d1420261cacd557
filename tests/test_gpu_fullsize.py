"""Parity at the benchmark's full size (10^9 records, and the 2*10^9 point of
the size sweep), in the launch sequence bench.py times (the default options:
the predicted levels as one launch per phase, then the persistent kernel).
The oracle cannot sort 10^9 records in seconds, so each output is checked
against the definition of the stable sort (oracle.check_stable: (key,
original index) strictly increasing, the indices a permutation, every key the
input's key at its index — exactly one output passes) and 16 sampled records
against the oracle's own position formula.  Key-only outputs are checked
against the key-only definition (oracle.check_sorted_keys: non-decreasing,
and every key value exactly as often as in the input)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

import gpu_util  # noqa: E402
import paper_2401_00710_gb300 as dts  # noqa: E402

N = 1_000_000_000


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = gpu_util.GpuSort(torch)
    yield g
    g.ws = None
    g.close()
    torch.cuda.empty_cache()


def check_full(G, name, dtype, bucketing=None):
    keys = gen.family(name, N, dtype, seed=1)  # the benchmark's stream
    vals = gen.iota(N, dtype)
    if bucketing is not None:
        G.set_options(bucketing=bucketing)
    gk, gv = G.sort(keys, vals)
    st = G.stats()
    G.reset_options()
    assert st["status"] == 0
    assert oracle.check_stable(keys, gk, gv) == -1
    js = np.random.RandomState(5).randint(0, N, size=16).astype(np.int64)
    pos = oracle.stable_positions(keys, js)
    np.testing.assert_array_equal(gv[pos], js.astype(dtype))
    np.testing.assert_array_equal(gk[pos], keys[js])
    G.ws = None
    return st


@pytest.mark.parametrize("name", ["uniform", "zipf0.8", "zipf1.0", "zipf1.2", "zipf1.5",
                                  "zipf1.2hash", "exp", "bitexp", "distinct10", "bexp30",
                                  "unif1e3", "edges"])
def test_full_u32_kv(G, name):
    st = check_full(G, name, np.uint32)
    if name == "uniform":
        assert st["levels"] == 2 and st["heavy_keys"][0] == 0


@pytest.mark.parametrize("name", ["uniform", "zipf1.2hash", "heavymix"])
def test_full_u64_kv(G, name):
    check_full(G, name, np.uint64)


def test_full_learned_mixture(G):
    # the learned-bucketing workload, the model forced (the fallback test
    # lives with the learned tests)
    st = check_full(G, "skewmix", np.uint64, bucketing=dts.DTSORT_BUCKETING_LEARNED_ALWAYS)
    assert st["learned_zones_used"] == 1


@pytest.mark.parametrize("dtype,name", [(np.uint32, "uniform"), (np.uint32, "zipf1.2"),
                                        (np.uint64, "uniform"), (np.uint64, "heavymix")])
def test_full_key_only(G, dtype, name):
    # key-only sorts have their own base case (64-bit keys: 6144 records per
    # bucket) and scatter counters; bench.py --op u32 / u64 times these
    keys = gen.family(name, N, dtype, seed=1)
    gk, _ = G.sort(keys)
    st = G.stats()
    assert st["status"] == 0
    assert oracle.check_sorted_keys(keys, gk) == -1
    if name == "uniform":
        assert st["levels"] == 2
    G.ws = None


def test_size_sweep_top_point_2e9(G):
    # the largest point of the size sweep: 2*10^9 u32 key/value pairs need a
    # third distribution level; values = original index, made on the device
    n = 2 * N
    keys = gen.family("uniform", n, np.uint32, seed=1)
    k = gpu_util.to_dev(keys, torch, G.dev)
    v = torch.arange(n, dtype=torch.int64, device=G.dev).to(torch.int32)
    st = G.launch(k, v, n, dts.DTSORT_OP_U32_KV)
    assert st == dts.DTSORT_OK
    assert G.device_status() == dts.DTSORT_OK
    stats = G.stats()
    assert stats["levels"] == 3
    G.ws = None
    gk = gpu_util.from_dev(k, np.uint32)
    del k
    gv = gpu_util.from_dev(v, np.uint32)
    del v
    torch.cuda.empty_cache()
    assert oracle.check_stable(keys, gk, gv) == -1
    js = np.random.RandomState(6).randint(0, n, size=16).astype(np.int64)
    pos = oracle.stable_positions(keys, js)
    np.testing.assert_array_equal(gv[pos], js.astype(np.uint32))
