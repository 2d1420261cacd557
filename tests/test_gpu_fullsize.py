"""Parity at the benchmark's full size (10^9 records), in the launch sequence
bench.py times (the default options: the predicted levels as one launch per
phase, then the persistent kernel).  The oracle cannot sort 10^9 records in
seconds, so each output is checked against the definition of the stable sort
(oracle.check_stable: (key, original index) strictly increasing, the indices a
permutation, every key the input's key at its index — exactly one output
passes) and 16 sampled records against the oracle's own position formula."""
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


@pytest.mark.parametrize("name", ["uniform", "zipf1.2", "exp", "bitexp", "distinct10"])
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
