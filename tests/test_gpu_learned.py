"""Learned CDF bucketing on the GPU: the model's own forward / backward /
Adam kernels against the fp64 oracle, the learned sort's output against the
stable-sort oracle, and what the trained model gains over digit zones."""
import numpy as np
import pytest

import gen
import oracle
from oracle import learned as OL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import gpu_util  # noqa: E402
import paper_2401_00710_gb300 as dts  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dts.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def G(dev):
    g = gpu_util.GpuSort(torch)
    yield g
    g.reset_options()
    g.ws = None
    g.close()


def f32(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


def cdf_data(n, seed=0):
    # features of sorted lognormal keys and their empirical CDF
    rs = np.random.RandomState(seed)
    keys = np.sort(np.floor(np.exp(rs.normal(30.0, 2.0, n)))).astype(np.uint64)
    x = (np.log2(keys.astype(np.float64) + 1.0) / 64.0).astype(np.float32)
    t = ((np.arange(n) + 0.5) / n).astype(np.float32)
    return x, t


def params(seed, scale=0.5):
    return (np.random.RandomState(seed).randn(OL.NPARAM) * scale).astype(np.float32)


def test_forward_matches_oracle(dev):
    p = params(1)
    x = np.random.RandomState(2).rand(10_007).astype(np.float32)
    y = torch.empty(len(x), dtype=torch.float32, device=dev)
    assert dts.dtsort_mlp_forward(f32(p, dev).data_ptr(), f32(x, dev).data_ptr(), len(x),
                                  y.data_ptr()) == dts.DTSORT_OK
    torch.cuda.synchronize()
    ref, _ = OL.forward(p.astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("n", [256, 1000, 4096, 65_537])
def test_gradients_match_oracle(dev, n):
    # fp32 GPU gradient vs fp64 oracle: every parameter group within a relative
    # 1e-3 (norm of the difference over the norm of the reference)
    x, t = cdf_data(n, seed=n)
    p = params(3)
    part = torch.empty(((n + 255) // 256) * 322, dtype=torch.float32, device=dev)
    g = torch.empty(322, dtype=torch.float32, device=dev)
    assert dts.dtsort_mlp_grad(f32(p, dev).data_ptr(), f32(x, dev).data_ptr(),
                               f32(t, dev).data_ptr(), n, part.data_ptr(),
                               g.data_ptr()) == dts.DTSORT_OK
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.float64)
    ref = OL.backward(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    groups = {"W1": slice(0, 16), "b1": slice(16, 32), "W2": slice(32, 288),
              "b2": slice(288, 304), "W3": slice(304, 320), "b3": slice(320, 321)}
    for name, sl in groups.items():
        err = np.linalg.norm(got[sl] - ref[sl]) / max(np.linalg.norm(ref[sl]), 1e-12)
        assert err < 1e-3, (name, err)
    loss = OL.loss(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(got[321] - loss) <= 1e-4 * max(loss, 1e-6)


def test_adam_step_matches_oracle(dev):
    p = params(4)
    g = np.random.RandomState(5).randn(322).astype(np.float32)
    m = np.random.RandomState(6).randn(OL.NPARAM).astype(np.float32) * 0.1
    v = np.abs(np.random.RandomState(7).randn(OL.NPARAM)).astype(np.float32) * 0.01
    P, M, V = f32(p, dev), f32(m, dev), f32(v, dev)
    assert dts.dtsort_mlp_adam(P.data_ptr(), M.data_ptr(), V.data_ptr(), f32(g, dev).data_ptr(),
                               3, 0.01) == dts.DTSORT_OK
    torch.cuda.synchronize()
    rp, rm, rv = OL.adam_step(p.astype(np.float64), g[:321].astype(np.float64),
                              m.astype(np.float64), v.astype(np.float64), 3, lr=0.01)
    # fp32 arithmetic on inputs of magnitude <= ~3: a few units of 2^-24 of
    # the operands, i.e. about 1e-6 absolute
    np.testing.assert_allclose(P.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(M.cpu().numpy(), rm, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(V.cpu().numpy(), rv, rtol=1e-5, atol=1e-7)


def test_training_tracks_oracle(dev):
    # the same init, data and batch schedule on both sides: the GPU loss curve
    # stays with the fp64 one and the loss falls
    n, batch, steps = 32_768, 2048, 60
    x, t = cdf_data(n, seed=11)
    p0 = params(8, 0.3)
    P = f32(p0, dev)
    M = torch.zeros(OL.NPARAM, dtype=torch.float32, device=dev)
    V = torch.zeros(OL.NPARAM, dtype=torch.float32, device=dev)
    part = torch.empty((batch // 256) * 322, dtype=torch.float32, device=dev)
    assert dts.dtsort_mlp_train(P.data_ptr(), M.data_ptr(), V.data_ptr(), f32(x, dev).data_ptr(),
                                f32(t, dev).data_ptr(), n, steps, batch, 0.01,
                                part.data_ptr()) == dts.DTSORT_OK
    torch.cuda.synchronize()
    # oracle with the GPU's schedule: batch k uses (k-1) mod S + i*S
    S = n // batch
    p = p0.astype(np.float64)
    m = np.zeros(OL.NPARAM)
    v = np.zeros(OL.NPARAM)
    xs, ts = x.astype(np.float64), t.astype(np.float64)
    for k in range(1, steps + 1):
        idx = ((k - 1) % S) + np.arange(batch) * S
        g = OL.backward(p, xs[idx], ts[idx])
        p, m, v = OL.adam_step(p, g, m, v, k, lr=0.01)
    lg = OL.loss(P.cpu().numpy().astype(np.float64), xs, ts)
    lr_ = OL.loss(p, xs, ts)
    l0 = OL.loss(p0.astype(np.float64), xs, ts)
    assert lg < 0.5 * l0
    assert abs(lg - lr_) <= 0.05 * lr_ + 1e-6


@pytest.mark.parametrize("name,dtype", [("skewmix", np.uint64), ("zipf1.0", np.uint32),
                                        ("uniform", np.uint64)])
def test_learned_sort_matches_oracle(G, name, dtype):
    n = 2_000_003
    keys = gen.family(name, n, dtype, seed=12)
    vals = gen.iota(n, dtype)
    G.set_options(bucketing=dts.DTSORT_BUCKETING_LEARNED_ALWAYS, learned_train_steps=100)
    gk, gv = G.sort(keys, vals)
    ek, ev = oracle.stable_sort(keys, vals)
    gpu_util.assert_same(gk, gv, ek, ev)
    st = G.stats()
    assert st["status"] == 0 and st["learned_zones_used"] == 1
    G.reset_options()


def test_learned_zones_balance_the_skewed_mixture(G):
    # the skewed 64-bit mixture (30% Zipf heavy part, 70% lognormal light
    # part): learned zones spread the light keys far more evenly than the top
    # key bits do, which is what the trained model buys
    n = 8_000_000
    keys = gen.family("skewmix", n, np.uint64, seed=13)
    vals = gen.iota(n, np.uint64)
    G.set_options(bucketing=dts.DTSORT_BUCKETING_DIGIT)
    G.sort(keys, vals)
    digit = G.stats()
    G.set_options(bucketing=dts.DTSORT_BUCKETING_LEARNED_ALWAYS)
    gk, gv = G.sort(keys, vals)
    lrn = G.stats()
    G.reset_options()
    ek, ev = oracle.stable_sort(keys, vals)
    gpu_util.assert_same(gk, gv, ek, ev)
    assert lrn["learned_bucket_cv"] < 0.5 * digit["learned_bucket_cv"], (lrn, digit)
    assert lrn["learned_bucket_max_over_mean"] < digit["learned_bucket_max_over_mean"]
    # most keys need no fix-up step beyond the model's prediction
    assert lrn["learned_fixup_records"] < 0.5 * n


def test_learned_bucketing_is_used_only_when_it_pays(G):
    # bucketing LEARNED estimates, from the sorted model sample, the
    # distribution passes below level 0 with digit zones and with the model's
    # zones (+ their extra cost) and keeps the cheaper.  Uniform keys: every
    # digit zone already needs the fewest levels, so the digit zones stay.
    # Bit-exponential keys (roughly log-uniform; most fall into the lowest
    # top-bit zone): whichever the estimate picks, the output is the oracle's
    n = 8_000_000
    G.set_options(bucketing=dts.DTSORT_BUCKETING_LEARNED, learned_train_steps=60)
    used = {}
    for name in ("uniform", "bitexp"):
        keys = gen.family(name, n, np.uint64, seed=31)
        vals = gen.iota(n, np.uint64)
        gk, gv = G.sort(keys, vals)
        ek, ev = oracle.stable_sort(keys, vals)
        gpu_util.assert_same(gk, gv, ek, ev)
        st = G.stats()
        digit_cost, learned_cost = st["learned_estimate"]
        assert digit_cost > 0 and learned_cost > 0
        assert st["learned_zones_used"] == (1 if digit_cost > learned_cost else 0)
        used[name] = (st["learned_zones_used"], digit_cost, learned_cost)
    G.reset_options()
    assert used["uniform"][0] == 0, used
