"""GPU parity: the CUDA sort through the C-ABI against the CPU oracle, bit for
bit (a stable sort's output is unique, so there is no tolerance)."""
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


@pytest.fixture(autouse=True)
def _defaults(G):
    G.reset_options()
    yield
    G.reset_options()


def check(G, keys, vals=None, offsets=None):
    gk, gv = G.sort(keys, vals, offsets)
    if offsets is None:
        ek, ev = oracle.stable_sort(keys, vals)
    else:
        ek, ev = oracle.stable_sort_segmented(keys, vals, offsets)
    gpu_util.assert_same(gk, gv, ek, ev)
    return G.stats()


# ------------------------------------------------------------ configurations
def test_config_small_uniform_u32_kv(G):
    # 10^6 uint32 keys uniform, values = original index
    n = 1_000_000
    keys = gen.family("uniform", n, np.uint32, seed=1)
    vals = gen.iota(n, np.uint32)
    st = check(G, keys, vals)
    assert st["status"] == 0
    assert st["heavy_keys"][0] == 0


U32_NAMES = sorted(gen.U32_FAMILIES)


@pytest.mark.parametrize("name", U32_NAMES)
def test_u32_kv_families(G, name):
    n = 3_000_017
    keys = gen.family(name, n, np.uint32, seed=2)
    vals = gen.iota(n, np.uint32)
    check(G, keys, vals)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_queued_levels_beyond_the_recursion(G, dtype):
    # narrow digits make the host queue three levels of phase launches for a
    # uniform input of this size, while two distinct keys are both heavy at
    # level 0: the queued levels 1 and 2 must find no subproblems
    n = 3_000_017
    keys = gen.keys(n, gen.DISTINCT, dtype, seed=6, p1=2)
    vals = gen.iota(n, dtype)
    G.set_options(gamma_max=4)
    st = check(G, keys, vals)
    assert st["status"] == 0
    assert st["levels"] == 1


def test_graph_transpose_edges(G):
    # a power-law edge list ordered by source, sorted stably by destination
    # (the transpose): each destination's sources stay in increasing order
    n = 4_000_037
    dst = gen.family("edges", n, np.uint32, seed=5)
    src = gen.edge_src(n, np.uint32)
    check(G, dst, src)


@pytest.mark.parametrize("name", ["uniform", "zipf1.2", "distinct10", "bitexp"])
def test_u32_key_only(G, name):
    n = 2_500_001
    keys = gen.family(name, n, np.uint32, seed=3)
    check(G, keys)


@pytest.mark.parametrize("name", sorted(gen.U64_FAMILIES))
def test_u64_kv_families(G, name):
    n = 1_500_007
    keys = gen.family(name, n, np.uint64, seed=4)
    vals = gen.iota(n, np.uint64)
    check(G, keys, vals)


@pytest.mark.parametrize("name", ["uniform", "heavymix", "zipf1.2hash"])
def test_u64_key_only(G, name):
    n = 1_200_003
    keys = gen.family(name, n, np.uint64, seed=5)
    check(G, keys)


# -------------------------------------------------------------- edge cases
EDGE_N = [1, 2, 3, 31, 32, 33, 511, 513, 3071, 3072, 3073, 4095, 4096, 4097,
          4607, 4608, 4609, 6143, 6144, 6145, 8191, 8192, 8193, 12288, 12289, 16391,
          100_003]


@pytest.mark.parametrize("n", EDGE_N)
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_edge_sizes_kv(G, n, dtype):
    keys = gen.family("uniform", n, dtype, seed=n)
    keys[: n // 3] = keys[0]  # a run of duplicates as well
    vals = gen.iota(n, dtype)
    check(G, keys, vals)


@pytest.mark.parametrize("mult", [2, 5, 16, 17, 40])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_base_case_ties(G, mult, dtype):
    # keys repeated `mult` times in shuffled order: equal keys share a bin of
    # the one-pass base case and must come out in input order (more than 16
    # in a bin takes the LSD passes instead)
    rs = np.random.RandomState(mult)
    for n in (4800, 250_000):
        distinct = gen.family("uniform", n // mult + 1, dtype, seed=mult)
        keys = np.repeat(distinct, mult)[:n]
        keys = keys[rs.permutation(n)].copy()
        vals = gen.iota(n, dtype)
        check(G, keys, vals)
        G.set_options(heavy_detection=-1)
        check(G, keys, vals)
        G.reset_options()
        check(G, keys, None)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_in_place_lsd_fallback(G, dtype):
    # a base case sorted in place (one sort below the capacity; segments of a
    # batch) whose tied keys overflow a bin, so that the LSD passes run and
    # gather the values by original index from the buffer they overwrite
    rs = np.random.RandomState(11)
    for n in (300, 3000, 4607):
        keys = gen.family("uniform", n, dtype, seed=n)
        keys[rs.permutation(n)[: n // 2]] = keys[0]
        vals = gen.iota(n, dtype)
        check(G, keys, vals)
        assert G.stats()["finisher_lsd_tasks"] >= 1
    sizes = [50 + (37 * s) % 4000 for s in range(64)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    keys = gen.family("uniform", int(off[-1]), dtype, seed=12)
    for s in range(64):
        a, b = off[s], off[s + 1]
        keys[a + rs.permutation(b - a)[: (b - a) // 2]] = keys[a]
    vals = gen.iota(len(keys), dtype)
    gk, gv = G.sort(keys, vals, off)
    ek, ev = oracle.stable_sort_segmented(keys, vals, off)
    gpu_util.assert_same(gk, gv, ek, ev)
    assert G.stats()["finisher_lsd_tasks"] >= 1


def test_n_zero_is_noop(G):
    keys = np.zeros(0, dtype=np.uint32)
    st = G.launch(None, None, 0, dts.DTSORT_OP_U32_KV)
    assert st == dts.DTSORT_OK
    assert G.device_status() == dts.DTSORT_OK


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_special_inputs(G, dtype):
    top = np.iinfo(dtype).max
    n = 200_000
    vals = gen.iota(n, dtype)
    for keys in (np.full(n, 7, dtype=dtype),                       # all equal
                 np.full(n, top, dtype=dtype),                     # all max
                 np.arange(n, dtype=dtype),                        # sorted
                 np.arange(n, dtype=dtype)[::-1].copy(),           # reversed
                 np.tile(np.array([top, 0, 1, top - 1], dtype=dtype), n // 4),
                 (np.arange(n, dtype=dtype) % 2) * top):           # two values
        check(G, keys, vals)


def test_narrow_key_ranges(G):
    # keys confined to a narrow range high up: exercises the overflow bucket
    # and the skipped leading bits
    n = 400_000
    base = np.uint32(0xF0000000)
    keys = (gen.family("uniform", n, np.uint32, seed=8) % 5000 + base).astype(np.uint32)
    check(G, keys, gen.iota(n, np.uint32))
    keys64 = (gen.family("uniform", n, np.uint64, seed=9) % 70000 +
              np.uint64(1 << 63)).astype(np.uint64)
    check(G, keys64, gen.iota(n, np.uint64))


def test_overflow_bucket_outliers(G):
    # small keys plus rare huge outliers that a sample can miss
    n = 600_000
    keys = (gen.family("uniform", n, np.uint32, seed=10) % 100_000).astype(np.uint32)
    keys[::99_991] = 0xFFFFFFF0
    check(G, keys, gen.iota(n, np.uint32))


# ---------------------------------------------------------------- options
@pytest.mark.parametrize("opts", [dict(heavy_detection=-1), dict(gamma_max=2),
                                  dict(gamma_max=5, finisher_capacity=700),
                                  dict(finisher_capacity=64),
                                  dict(seed=12345, sample_log_factor=3)])
def test_options_do_not_change_output(G, opts):
    n = 700_001
    for name in ("zipf1.2", "uniform", "bitexp"):
        keys = gen.family(name, n, np.uint32, seed=11)
        vals = gen.iota(n, np.uint32)
        G.set_options(**opts)
        check(G, keys, vals)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_generic_merge_matches(G, mode):
    # the merge ablation: merge-path merging of every heavy zone (key
    # comparisons) instead of dovetail merging gives the same stable order
    zones = {}
    for name, dtype, n, seed in (("zipf1.2", np.uint32, 3_000_000, 1),
                                 ("distinct10", np.uint32, 1_300_007, 16),
                                 ("exp", np.uint32, 1_300_007, 16),
                                 ("heavymix", np.uint64, 1_300_007, 16),
                                 ("zipf1.2hash", np.uint64, 1_300_007, 16)):
        keys = gen.family(name, n, dtype, seed=seed)
        vals = gen.iota(n, dtype)
        G.set_options(merge=dts.DTSORT_MERGE_GENERIC, launch_mode=mode)
        st = check(G, keys, vals)
        zones[name] = (st["merge_zones"], st["merge_records"])
        check(G, keys, None)
    assert zones["zipf1.2"][0] > 0 and zones["zipf1.2"][1] > 0, zones
    G.reset_options()
    o = dts.dtsort_default_options()
    o.merge = 2
    with pytest.raises(dts.DtsortError) as e:
        dts.dtsort_set_options(G.h, o)
    assert e.value.status == dts.DTSORT_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [1, 2])
def test_launch_modes_match(G, mode):
    # 1: one launch per phase, host-driven (profiling aid); 2: the persistent
    # kernel alone; the default (0) queues the predicted levels as phase
    # launches and hands the rest to the persistent kernel
    n = 1_500_000
    for name in ("zipf1.2", "uniform", "distinct10"):
        keys = gen.family(name, n, np.uint32, seed=14)
        vals = gen.iota(n, np.uint32)
        G.set_options(launch_mode=mode)
        st = check(G, keys, vals)
        assert st["levels"] >= 1
        if mode == 2:
            assert st["kernel_launches"] == 1
        else:
            assert st["kernel_launches"] > 7
    G.reset_options()


@pytest.mark.parametrize("name,dtype", [("uniform", np.uint32), ("zipf1.2", np.uint32),
                                        ("bitexp", np.uint64), ("distinct10", np.uint32)])
def test_queued_levels_capture_and_replay(G, name, dtype):
    # the default single-array launch sequence has no host synchronisation:
    # it is captured into a CUDA graph and replayed; inputs that need fewer
    # levels than predicted (10 keys) or more (skewed) come out right
    n = 3_000_017
    keys = gen.family(name, n, dtype, seed=21)
    vals = gen.iota(n, dtype)
    op = gpu_util.op_of(keys, vals)
    pk = gpu_util.to_dev(keys, torch, G.dev)
    pv = gpu_util.to_dev(vals, torch, G.dev)
    k, v = pk.clone(), pv.clone()
    G.workspace(op, n)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        assert G.launch(k, v, n, op) == dts.DTSORT_OK
    ek, ev = oracle.stable_sort(keys, vals)
    for _ in range(2):
        k.copy_(pk)
        v.copy_(pv)
        graph.replay()
        torch.cuda.synchronize()
        assert G.device_status() == dts.DTSORT_OK
        gpu_util.assert_same(gpu_util.from_dev(k, dtype), gpu_util.from_dev(v, dtype), ek, ev)


# --------------------------------------------------------------- segmented
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_segmented(G, dtype):
    rs = np.random.RandomState(12)
    sizes = np.concatenate([rs.randint(0, 3, 40), rs.randint(0, 5000, 100),
                            rs.randint(5000, 200_000, 12)])
    rs.shuffle(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    keys = gen.family("zipf1.2hash", n, dtype, seed=13)
    vals = np.zeros(n, dtype=dtype)
    for s in range(len(sizes)):
        vals[off[s]:off[s + 1]] = np.arange(sizes[s], dtype=dtype)
    check(G, keys, vals, off)
    check(G, keys, None, off)


def test_segmented_bad_offsets_reported(G):
    keys = gen.family("uniform", 1000, np.uint32, seed=1)
    off = np.array([0, 600, 400, 1000], dtype=np.int64)  # decreasing
    k = gpu_util.to_dev(keys, torch, G.dev)
    o = torch.from_numpy(off).to(G.dev)
    st = G.launch(k, None, 1000, dts.DTSORT_OP_U32, o, 3)
    assert st == dts.DTSORT_OK
    assert G.device_status() == dts.DTSORT_ERR_INVALID_ARG


# ----------------------------------------------------- method structure
def test_ten_distinct_keys_are_all_heavy_at_the_root(G):
    # Thm 3.5: with few distinct keys every key is heavy at the root, and
    # nothing is distributed again
    n = 4_000_000
    keys = gen.family("distinct10", n, np.uint32, seed=1)
    st = check(G, keys, gen.iota(n, np.uint32))
    assert st["heavy_keys"][0] == 10
    assert st["records"][1] == 0
    assert st["heavy_records"][0] == n


def test_uniform_has_no_heavy_keys_and_two_levels(G):
    n = 2_000_000
    keys = gen.family("uniform", n, np.uint32, seed=1)
    st = check(G, keys, gen.iota(n, np.uint32))
    assert sum(st["heavy_keys"]) == 0
    assert st["merge_zones"] == 0
    assert st["finisher_records"] == n


def test_zipf_heavy_keys_below_the_light_ones_need_no_merge(G):
    # Zipf ranks: the heavy keys are the smallest keys of their zone, so the
    # zone's buckets numbered [heavy][light] are already in key order (Alg. 3
    # would place every heavy run before the light bucket): no merge
    n = 3_000_000
    keys = gen.family("zipf1.2", n, np.uint32, seed=1)
    st = check(G, keys, gen.iota(n, np.uint32))
    assert st["heavy_keys"][0] > 0
    # a few deep zones of a handful of keys may still interleave
    assert st["merge_free_zones"] > st["merge_zones"]
    assert st["merge_records"] < n // 10


def test_hashed_zipf_heavy_keys_inside_the_zone_are_merged(G):
    # hashed Zipf ranks: a heavy key lies among its zone's light keys, so the
    # zone needs the dovetail merge
    n = 3_000_000
    keys = gen.family("zipf1.2hash", n, np.uint64, seed=1)
    st = check(G, keys, gen.iota(n, np.uint64))
    assert st["heavy_keys"][0] > 0
    assert st["merge_zones"] > 0 and st["merge_records"] > 0


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("side", ["below", "above"])
def test_unsampled_light_key_outside_the_layout_forces_the_merge(G, dtype, side):
    # keys in [0, 2^30): one heavy key (30% of the records) at the bottom (or
    # top) of its level-0 zone, whose other keys all lie above (below) it,
    # and one record on the other side, which the sample almost surely
    # misses: the layout [heavy][light] ([light][heavy]) chosen from the
    # sample is wrong for that record, the histogram sees it and the zone is
    # merged after all
    n = 3_000_000
    rng = np.random.default_rng(7)
    top = (1 << 30) - 1
    if side == "below":
        h, lone = 1000, 5
        keys = rng.integers(2000, top, size=n, endpoint=True).astype(dtype)
    else:
        h, lone = top - 1000, top
        keys = rng.integers(0, top - 2000, size=n, endpoint=True).astype(dtype)
    keys[rng.random(n) < 0.3] = h
    keys[n // 2] = lone
    vals = gen.iota(n, dtype)
    st = check(G, keys, vals)
    assert st["heavy_keys"][0] >= 1
    assert st["merge_zones"] >= 1
    check(G, keys, None)


def test_heavy_min_share(G):
    # one key holding 15% of the records among uniform ones: below the default
    # minimum share (250 thousandths of the sample) the root keeps no heavy
    # key and distributes it by its digit; -1 keeps any share (the paper's
    # rule), 1000 none.  At 40% the default keeps it.  The output is the same
    # stable order in every case.
    n = 3_000_000
    rng = np.random.default_rng(9)
    vals = gen.iota(n, np.uint32)
    for share, expect in ((0.15, {0: 0, -1: 1, 1000: 0}), (0.40, {0: 1, -1: 1, 1000: 0})):
        keys = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        keys[rng.random(n) < share] = 12345
        for hms, nh in expect.items():
            G.set_options(heavy_min_share=hms)
            st = check(G, keys, vals)
            assert st["heavy_keys"][0] == nh, (share, hms, st["heavy_keys"][:3])
    for bad in (-2, 1001):
        o = dts.dtsort_default_options()
        o.heavy_min_share = bad
        with pytest.raises(dts.DtsortError) as e:
            dts.dtsort_set_options(G.h, o)
        assert e.value.status == dts.DTSORT_ERR_INVALID_ARG


def test_deterministic(G):
    n = 1_000_000
    keys = gen.family("zipf1.0", n, np.uint32, seed=21)
    vals = gen.iota(n, np.uint32)
    G.sort(keys, vals)
    a = G.stats()
    G.sort(keys, vals)
    b = G.stats()
    for k in ("levels", "segments", "records", "heavy_keys", "heavy_records",
              "overflow_records", "finisher_tasks", "merge_zones", "merge_records"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_sampler_matches_oracle(G, dtype):
    n = 2_000_000
    keys = gen.family("zipf1.2" if dtype == np.uint32 else "heavymix", n, dtype, seed=3)
    keys[1000:300_000] = keys[5]
    d = gpu_util.to_dev(keys, torch, G.dev)
    heavy = torch.zeros(8192, dtype=torch.int64, device=G.dev)
    nh = torch.zeros(1, dtype=torch.int64, device=G.dev)
    mx = torch.zeros(1, dtype=torch.int64, device=G.dev)
    s = torch.cuda.current_stream(G.dev).cuda_stream
    for (start, size, hi, seed, count, L) in [(0, n, 8 * keys.itemsize, 1, 7680, 21),
                                              (12345, 999_999, 20, 77, 8192, 17),
                                              (5, 300_000, 3, 2, 1000, 3),
                                              (0, 10, 32, 9, 4096, 1)]:
        st = dts.dtsort_debug_sample(G.h, d.data_ptr(), keys.itemsize, start, size, hi,
                                     seed, count, L, heavy.data_ptr(), nh.data_ptr(),
                                     mx.data_ptr(), s)
        assert st == dts.DTSORT_OK
        torch.cuda.synchronize()
        got_n = int(nh.item())
        got = heavy[:got_n].cpu().numpy().view(np.uint64)
        exp, exp_max = oracle.sample_heavy(keys, seed, start, size, hi, count, L)
        np.testing.assert_array_equal(got, exp)
        assert int(mx.cpu().numpy().view(np.uint64)[0]) == exp_max


# ------------------------------------------------------------ error paths
def test_argument_checks(G):
    n = 1000
    k = torch.zeros(n, dtype=torch.int32, device=G.dev)
    ws = G.workspace(dts.DTSORT_OP_U32, n)
    s = torch.cuda.current_stream(G.dev).cuda_stream
    assert dts.dtsort_u32(G.h, k.data_ptr(), -1, ws.data_ptr(), ws.numel(), s) == \
        dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_u32(G.h, None, n, ws.data_ptr(), ws.numel(), s) == \
        dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_u32_kv(G.h, k.data_ptr(), None, n, ws.data_ptr(), ws.numel(), s) == \
        dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_u32(G.h, k.data_ptr(), n, ws.data_ptr(), 100, s) == \
        dts.DTSORT_ERR_WORKSPACE_TOO_SMALL
    assert dts.dtsort_u32(G.h, k.data_ptr() + 1, n, ws.data_ptr(), ws.numel(), s) == \
        dts.DTSORT_ERR_INVALID_ARG


def test_bounded_wait_expires_without_hanging(G):
    # a look-back chunk that never publishes its status: the successors'
    # waits run out, the sort latches DEVICE_TIMEOUT and the context stays
    # usable (6M records = 3 chunks of 32 rows of 64K-record blocks in the
    # level-0 count matrix: chunk 2 waits on the muted chunk 1)
    n = 6_000_000
    keys = gen.family("uniform", n, np.uint32, seed=4)
    vals = gen.iota(n, np.uint32)
    G.set_options(debug_fault=1, wait_limit_ms=50)
    k = gpu_util.to_dev(keys, torch, G.dev)
    v = gpu_util.to_dev(vals, torch, G.dev)
    assert G.launch(k, v, n, dts.DTSORT_OP_U32_KV) == dts.DTSORT_OK
    assert G.device_status() == dts.DTSORT_ERR_DEVICE_TIMEOUT
    G.reset_options()
    check(G, keys, vals)


@pytest.mark.parametrize("dtype,kv", [(np.uint32, True), (np.uint64, True), (np.uint32, False)])
def test_sort_from_host_buffers(G, dtype, kv):
    # dtsort_sort_host: pinned host arrays in, sorted host arrays out, through
    # the caller's device buffers and workspace
    n = 1_234_567
    keys = gen.family("zipf1.2hash" if dtype == np.uint64 else "zipf1.0", n, dtype, seed=41)
    vals = gen.iota(n, dtype) if kv else None
    tdt = torch.int32 if dtype == np.uint32 else torch.int64
    hk = torch.from_numpy(keys.view(np.int32 if dtype == np.uint32 else np.int64)).pin_memory()
    hv = (torch.from_numpy(vals.view(np.int32 if dtype == np.uint32 else np.int64)).pin_memory()
          if kv else None)
    dk = torch.empty(n, dtype=tdt, device=G.dev)
    dv = torch.empty(n, dtype=tdt, device=G.dev) if kv else None
    op = gpu_util.op_of(keys, vals)
    ws = G.workspace(op, n)
    s = torch.cuda.current_stream(G.dev).cuda_stream
    st = dts.dtsort_sort_host(G.h, op, hk.data_ptr(), hv.data_ptr() if kv else None, n,
                              dk.data_ptr(), dv.data_ptr() if kv else None, ws.data_ptr(),
                              ws.numel(), s)
    assert st == dts.DTSORT_OK
    torch.cuda.synchronize()
    assert G.device_status() == dts.DTSORT_OK
    ek, ev = oracle.stable_sort(keys, vals)
    gk = hk.numpy().view(dtype)
    gv = hv.numpy().view(dtype) if kv else None
    gpu_util.assert_same(gk, gv, ek, ev)
    # a key-only op must not be given values, a key/value op must be
    bad_op = dts.DTSORT_OP_U32 if dtype == np.uint32 else dts.DTSORT_OP_U64
    if kv:
        assert dts.dtsort_sort_host(G.h, bad_op, hk.data_ptr(), hv.data_ptr(), n, dk.data_ptr(),
                                    dv.data_ptr(), ws.data_ptr(), ws.numel(),
                                    s) == dts.DTSORT_ERR_INVALID_ARG
