"""The sharded (one-exchange, multi-GPU) sort on CPU ranks.

What needs no GPU is tested here: the oracle's definition of the rank-local
partition (against the stable sort it must compose to), the library's host
routine that picks the splitters, and the whole exchange of
paper_2401_00710_gb300.sharded.sharded_sort on 2 and 4 gloo ranks, with CPU
stand-ins for the three device steps (sample, partition, local sort).  The
assembled output must equal the oracle's stable sort of the whole array,
including a heavily duplicated key that straddles a splitter and an empty
shard.  The device steps themselves are tested in test_gpu_sharded.py.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import gen
import oracle
from oracle import sharded as osh

torch = pytest.importorskip("torch")

import paper_2401_00710_gb300 as dts  # noqa: E402
from paper_2401_00710_gb300 import sharded  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    dts.build()
    return dts.lib()


# ------------------------------------------------------ the partition oracle
def _composites(keys, gidx):
    return [(int(k), int(g)) for k, g in zip(keys, gidx)]


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_partition_oracle_composes_to_the_stable_sort(dtype):
    # ranges of the whole array, each sorted stably and concatenated in
    # order, give the stable sort; shards partitioned on their own and
    # concatenated in shard order give the same ranges
    rs = np.random.RandomState(3)
    for n, parts in [(1, 1), (7, 3), (200, 2), (1000, 5), (5000, 8)]:
        keys = rs.randint(0, 12, size=n).astype(dtype)
        keys[rs.rand(n) < 0.4] = dtype(5)  # a heavy key
        if dtype == np.uint64:
            keys[rs.rand(n) < 0.1] = np.iinfo(np.uint64).max
        vals = np.arange(n, dtype=dtype)
        gidx = np.arange(n, dtype=np.int64)
        pick = np.sort(rs.randint(0, n, size=parts - 1))
        order = sorted(range(n), key=lambda i: (int(keys[i]), i))
        sk = np.array([keys[order[j]] for j in pick], dtype=np.uint64)
        sg = np.array([order[j] for j in pick], dtype=np.int64)
        pk, pv, cnt = osh.partition(keys, vals, 0, sk, sg, parts)
        assert cnt.sum() == n
        ek, ev = oracle.stable_sort(keys, vals)
        got_k, got_v, a = [], [], 0
        comp = _composites(pk, pv.astype(np.int64))
        for p in range(parts):
            seg = comp[a:a + cnt[p]]
            assert seg == sorted(seg, key=lambda c: c[1])  # index order inside
            if p + 1 < parts and cnt[p] and cnt[p + 1]:
                assert max(seg) < min(comp[a + cnt[p]:a + cnt[p] + cnt[p + 1]])
            k_, v_ = oracle.stable_sort(pk[a:a + cnt[p]], pv[a:a + cnt[p]])
            got_k.append(k_)
            got_v.append(v_)
            a += cnt[p]
        np.testing.assert_array_equal(np.concatenate(got_k), ek)
        np.testing.assert_array_equal(np.concatenate(got_v), ev)
        # shards: the same ranges, shard by shard
        cut = sorted(rs.randint(0, n + 1, size=2))
        bounds = [0, cut[0], cut[1], n]
        parts_by_shard = [osh.partition(keys[bounds[q]:bounds[q + 1]],
                                        vals[bounds[q]:bounds[q + 1]], bounds[q], sk, sg,
                                        parts) for q in range(3)]
        for p in range(parts):
            want = pk[np.cumsum(cnt)[p] - cnt[p]:np.cumsum(cnt)[p]]
            got = np.concatenate([b[0][np.cumsum(b[2])[p] - b[2][p]:np.cumsum(b[2])[p]]
                                  for b in parts_by_shard])
            np.testing.assert_array_equal(got, want)
    # gidx alone decides within a key: a splitter inside a run of equal keys
    r = osh.range_of(np.array([9, 9, 9, 9], dtype=np.uint32), np.arange(4),
                     np.array([9], dtype=np.uint64), np.array([2]))
    np.testing.assert_array_equal(r, [0, 0, 1, 1])


# --------------------------------------------- the library's host splitters
def test_splitters_pick_sample_ranks(lib):
    rs = np.random.RandomState(4)
    m = 1001
    sk = rs.randint(0, 50, size=m).astype(np.uint64)
    sg = rs.permutation(m).astype(np.int64)
    order = sorted(range(m), key=lambda i: (int(sk[i]), int(sg[i])))
    for parts in (1, 2, 3, 8, 64):
        k, g = sharded.pick_splitters(sk, sg, parts)
        assert len(k) == parts - 1 == len(g)
        for j in range(1, parts):
            i = order[j * m // parts]
            assert (int(k[j - 1]), int(g[j - 1])) == (int(sk[i]), int(sg[i]))
    # no sample: every record falls into range 0
    k, g = sharded.pick_splitters(np.zeros(0, np.uint64), np.zeros(0, np.int64), 4)
    assert (k == np.iinfo(np.uint64).max).all() and (g == np.iinfo(np.int64).max).all()
    out = np.zeros(70, dtype=np.uint64)
    og = np.zeros(70, dtype=np.int64)
    for bad in (0, 65):
        assert dts.dtsort_shard_splitters(sk.ctypes.data, sg.ctypes.data, m, bad,
                                          out.ctypes.data, og.ctypes.data) == \
            dts.DTSORT_ERR_INVALID_ARG


def test_partition_workspace_and_argument_checks(lib):
    assert dts.dtsort_shard_partition_workspace_bytes(0, 4) == 256
    assert dts.dtsort_shard_partition_workspace_bytes(10 ** 9, 8) <= 256 + 8 * 8 * 4097
    with pytest.raises(dts.DtsortError):
        dts.dtsort_shard_partition_workspace_bytes(10, 65)
    # host-detectable errors return before anything touches a device
    assert dts.dtsort_shard_partition(None, None, 3, 10, 0, None, None, 2, None, None, None,
                                      None, 0) == dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_shard_sample(None, 4, 10, 0, 1, -1, None, None) == \
        dts.DTSORT_ERR_INVALID_ARG
    assert dts.dtsort_shard_sample(None, 4, 0, 0, 1, 0, None, None) == dts.DTSORT_OK


# ------------------------------------------------- the exchange, gloo ranks
class CpuShardOps:
    """CPU stand-ins for the device steps: a seeded sample, the oracle's
    partition and stable sort; the splitters come from the library's host
    routine, as on GPUs."""

    def sample(self, keys, gidx0, count, seed):
        k = keys.numpy()
        pos = np.random.RandomState((seed * 7919 + gidx0) % (2 ** 31)).randint(
            0, max(len(k), 1), size=count)
        sk = k[pos].astype(np.uint64) if k.dtype == np.int64 else \
            k.view(np.uint32)[pos].astype(np.uint64)
        return (torch.from_numpy(sk.view(np.int64).copy()),
                torch.from_numpy((gidx0 + pos).astype(np.int64)))

    def splitters(self, sample_keys, sample_gidx, parts):
        return sharded.pick_splitters(sample_keys, sample_gidx, parts)

    def partition(self, keys, values, gidx0, split_keys, split_gidx, parts):
        udt = np.uint32 if keys.dtype == torch.int32 else np.uint64
        k = keys.numpy().view(udt)
        v = None if values is None else values.numpy().view(udt)
        pk, pv, cnt = osh.partition(k, v, gidx0, split_keys, split_gidx, parts)
        sdt = keys.numpy().dtype
        return (torch.from_numpy(pk.view(sdt).copy()),
                None if pv is None else torch.from_numpy(pv.view(sdt).copy()),
                [int(c) for c in cnt])

    def sort(self, keys, values):
        udt = np.uint32 if keys.dtype == torch.int32 else np.uint64
        sdt = keys.numpy().dtype
        k, v = oracle.stable_sort(keys.numpy().view(udt),
                                  None if values is None else values.numpy().view(udt))
        return (torch.from_numpy(k.view(sdt).copy()),
                None if v is None else torch.from_numpy(v.view(sdt).copy()))


CASES = {
    # name: (key dtype, n, shard cuts as fractions, with values)
    "uniform_u32_kv": (np.uint32, 40_000, (0.25, 0.5, 0.75), True),
    # 60% of the records share one key: it straddles the splitters
    "heavy_u32_kv": (np.uint32, 40_000, (0.1, 0.5, 0.9), True),
    # an empty shard, 64-bit keys without values
    "empty_shard_u64": (np.uint64, 30_001, (0.0, 0.3, 0.6), False),
    "all_equal_u64_kv": (np.uint64, 20_000, (0.25, 0.5, 0.75), True),
}


def case_input(name):
    dtype, n, cuts, has_v = CASES[name]
    if name.startswith("uniform"):
        keys = gen.family("uniform", n, dtype, seed=11)
    elif name.startswith("heavy"):
        keys = gen.family("zipf1.0", n, dtype, seed=12)
        keys[np.random.RandomState(1).rand(n) < 0.6] = dtype(123456)
    elif name.startswith("empty"):
        keys = gen.family("heavymix", n, dtype, seed=13)
    else:
        keys = np.full(n, 77, dtype=dtype)
    vals = np.arange(n, dtype=dtype) if has_v else None
    return keys, vals, cuts


def _worker(rank, world, port, name, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, vals, cuts = case_input(name)
        n = len(keys)
        fr = [0.0] + list(cuts[:world - 1]) + [1.0] if world == 4 else [0.0, cuts[1], 1.0]
        a, b = int(fr[rank] * n), int(fr[rank + 1] * n)
        sdt = np.int32 if keys.dtype == np.uint32 else np.int64
        k = torch.from_numpy(keys[a:b].view(sdt).copy())
        v = None if vals is None else torch.from_numpy(vals[a:b].view(sdt).copy())
        res = sharded.sharded_sort(k, v, CpuShardOps(), seed=5, samples_per_part=256)
        np.savez(os.path.join(outdir, "r%d.npz" % rank), keys=res["keys"].numpy(),
                 values=np.zeros(0) if res["values"] is None else res["values"].numpy(),
                 offset=res["offset"], sizes=np.array(res["sizes"]), sent=np.array(res["sent"]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("name", sorted(CASES))
def test_sharded_sort_on_gloo_ranks(lib, world, name):
    import torch.multiprocessing as mp
    keys, vals, _ = case_input(name)
    n = len(keys)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), name, d), nprocs=world, join=True)
        parts = [np.load(os.path.join(d, "r%d.npz" % r)) for r in range(world)]
    udt = keys.dtype
    offs = [int(p["offset"]) for p in parts]
    assert offs == sorted(offs) and offs[0] == 0
    gk = np.concatenate([p["keys"].view(udt) for p in parts])
    ek, ev = oracle.stable_sort(keys, vals)
    np.testing.assert_array_equal(gk, ek)
    if vals is not None:
        gv = np.concatenate([p["values"].view(udt) for p in parts])
        np.testing.assert_array_equal(gv, ev)
    sizes = parts[0]["sizes"]
    assert sizes.sum() == n
    if name.startswith(("heavy", "all_equal")):
        # the duplicated key is split by global index: parts stay balanced
        assert sizes.max() <= 1.25 * n / world
