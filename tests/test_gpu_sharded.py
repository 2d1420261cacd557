"""The device steps of the sharded sort, through the C-ABI: the sampler and
the stable partition kernel against the oracle's definitions, and the whole
P-rank pipeline with P shards on this one GPU (the exchange done by slicing;
the collectives themselves are tested on gloo ranks in test_sharded_cpu.py).
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import sharded as osh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2401_00710_gb300 as dts  # noqa: E402
from paper_2401_00710_gb300 import sharded  # noqa: E402

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dts.build()
    return torch.device("cuda", 0)


def _t(a, dev):
    sdt = np.int32 if a.dtype == np.uint32 else np.int64
    return torch.from_numpy(np.ascontiguousarray(a).view(sdt)).to(dev)


def _np(t, udt):
    return t.cpu().numpy().view(udt)


def fmix64(x):
    # SplitMix64's finaliser: output 0 of the sequence whose state is x - gamma
    return oracle.splitmix64_at((x - GOLDEN_GAMMA) & M64, 0)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_sample_kernel_follows_its_definition(dev, dtype):
    n, gidx0, seed, count = 100_003, 12345, 99, 4000
    keys = gen.family("uniform", n, dtype, seed=4)
    ops = sharded.GpuShardOps(dev)
    sk, sg = ops.sample(_t(keys, dev), gidx0, count, seed)
    sk, sg = _np(sk, np.uint64), sg.cpu().numpy()
    state = seed ^ fmix64((gidx0 + GOLDEN_GAMMA) & M64)
    pos = np.array([oracle.splitmix64_at(state, i) % n for i in range(count)], dtype=np.int64)
    np.testing.assert_array_equal(sg, gidx0 + pos)
    np.testing.assert_array_equal(sk, keys[pos].astype(np.uint64))


def _splitters_from(keys, gidx0, parts, rs):
    """Splitters drawn from the shard's own (key, global index) pairs."""
    n = len(keys)
    if parts == 1 or n == 0:
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    pick = rs.randint(0, n, size=4 * parts)
    return sharded.pick_splitters(keys[pick].astype(np.uint64), gidx0 + pick, parts)


@pytest.mark.parametrize("dtype,has_v", [(np.uint32, True), (np.uint32, False),
                                         (np.uint64, True), (np.uint64, False)])
def test_partition_kernel_matches_oracle(dev, dtype, has_v):
    rs = np.random.RandomState(6)
    ops = sharded.GpuShardOps(dev)
    for n, parts in [(0, 3), (1, 1), (1000, 2), (4097, 64), (300_001, 3),
                     (5_000_000, 8), (20_000_017, 5)]:
        keys = gen.family("zipf1.0" if dtype == np.uint32 else "zipf1.2hash", n, dtype,
                          seed=n % 97)
        if n:
            keys[rs.rand(n) < 0.3] = dtype(42)  # a key across the splitters
        vals = np.arange(n, dtype=dtype) if has_v else None
        gidx0 = 7_000_000 if n else 0
        sk, sg = _splitters_from(keys, gidx0, parts, rs)
        gk, gv, cnt = ops.partition(_t(keys, dev), None if vals is None else _t(vals, dev),
                                    gidx0, sk, sg, parts)
        ek, ev, ecnt = osh.partition(keys, vals, gidx0, sk, sg, parts)
        assert cnt == [int(c) for c in ecnt], (n, parts)
        np.testing.assert_array_equal(_np(gk, dtype), ek)
        if has_v:
            np.testing.assert_array_equal(_np(gv, dtype), ev)


@pytest.mark.parametrize("dtype,name", [(np.uint32, "zipf1.2"), (np.uint64, "heavymix")])
def test_sharded_pipeline_on_one_gpu(dev, dtype, name):
    # P shards of one array on this GPU: every device step of the sharded
    # sort, the exchange done by slicing; the parts concatenated in rank
    # order are the oracle's stable sort
    P, n = 4, 6_000_000
    keys = gen.family(name, n, dtype, seed=21)
    vals = np.arange(n, dtype=dtype)
    ops = sharded.GpuShardOps(dev)
    cuts = [0, n // 7, n // 2, n // 2, n]  # uneven shards, one empty
    shards = [(_t(keys[cuts[r]:cuts[r + 1]], dev), _t(vals[cuts[r]:cuts[r + 1]], dev))
              for r in range(P)]
    samples = [ops.sample(k, cuts[r], 2048 if k.numel() else 0, 3)
               for r, (k, _) in enumerate(shards)]
    all_k = np.concatenate([_np(s[0], np.uint64) for s in samples])
    all_g = np.concatenate([s[1].cpu().numpy() for s in samples])
    sk, sg = ops.splitters(all_k, all_g, P)
    parts = [ops.partition(k, v, cuts[r], sk, sg, P) for r, (k, v) in enumerate(shards)]
    got_k, got_v, sizes = [], [], []
    for p in range(P):
        rk, rv = [], []
        for q in range(P):
            a = sum(parts[q][2][:p])
            rk.append(parts[q][0][a:a + parts[q][2][p]])
            rv.append(parts[q][1][a:a + parts[q][2][p]])
        k = torch.cat(rk).contiguous()
        v = torch.cat(rv).contiguous()
        k, v = ops.sort(k, v)
        got_k.append(_np(k, dtype))
        got_v.append(_np(v, dtype))
        sizes.append(k.numel())
    ek, ev = oracle.stable_sort(keys, vals)
    np.testing.assert_array_equal(np.concatenate(got_k), ek)
    np.testing.assert_array_equal(np.concatenate(got_v), ev)
    assert max(sizes) <= 1.2 * n / P
