"""Pins for the fp64 learned-bucketing oracle (no GPU).

Gradients are pinned by central finite differences; Adam by its closed form at
step 1; the piecewise-linear knots by brute-force quantiles; bucket membership
by a direct count of splitters.
"""
import numpy as np
import pytest

from oracle import learned as L


def _params(seed, scale=0.7):
    rs = np.random.RandomState(seed)
    return rs.randn(L.NPARAM) * scale


def test_parameter_count_and_layout():
    assert L.NPARAM == 321
    p = np.arange(L.NPARAM, dtype=np.float64)
    np.testing.assert_array_equal(L.pack(*L.unpack(p)), p)
    W1, b1, W2, b2, W3, b3 = L.unpack(p)
    assert W1.shape == (16, 1) and W2.shape == (16, 16) and W3.shape == (1, 16)
    assert W2[0, 1] == 33  # row-major, after W1 (16) and b1 (16)


def test_forward_closed_form_small_cases():
    # zero weights: y = b3
    p = np.zeros(L.NPARAM)
    p[-1] = 0.25
    y, _ = L.forward(p, np.array([0.0, 0.5, 1.0]))
    np.testing.assert_allclose(y, 0.25)
    # one path: W1[0]=a, W2[0,0]=c, W3[0,0]=e -> y = e*tanh(c*tanh(a x))
    p = np.zeros(L.NPARAM)
    W1, b1, W2, b2, W3, b3 = L.unpack(p)
    a, c, e = 1.3, -0.7, 2.0
    q = p.copy()
    q[0] = a
    q[32 + 0] = c          # W2[0,0]
    q[32 + 256 + 16] = e   # W3[0,0]
    x = np.linspace(-1, 1, 7)
    y, _ = L.forward(q, x)
    np.testing.assert_allclose(y, e * np.tanh(c * np.tanh(a * x)), rtol=1e-14)


def test_gradients_match_central_differences():
    rs = np.random.RandomState(3)
    for seed in range(3):
        p = _params(seed)
        x = rs.rand(37)
        t = np.sort(rs.rand(37))
        g = L.backward(p, x, t)
        h = 1e-6
        for i in range(L.NPARAM):
            e = np.zeros(L.NPARAM)
            e[i] = h
            fd = (L.loss(p + e, x, t) - L.loss(p - e, x, t)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_gradient_of_output_bias_closed_form():
    rs = np.random.RandomState(4)
    p = _params(5)
    x, t = rs.rand(50), rs.rand(50)
    y, _ = L.forward(p, x)
    g = L.backward(p, x, t)
    assert abs(g[-1] - 2.0 * np.mean(y - t)) < 1e-12


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    p1, m1, v1 = L.adam_step(p, g, m, v, 1, lr=0.01, eps=1e-8)
    # m_hat = g, v_hat = g^2 at t = 1: update = -lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_reduces_loss_on_a_cdf():
    rs = np.random.RandomState(6)
    s = np.sort(rs.lognormal(0, 1, 4000))
    x = np.log2(1 + s) / 8
    t = (np.arange(4000) + 0.5) / 4000
    p0 = _params(1, 0.3)
    p, losses = L.train(p0, x, t, steps=300, batch=256, lr=1e-2)
    assert L.loss(p, x, t) < 0.2 * L.loss(p0, x, t)


def test_pl_knots_are_exact_quantiles():
    rs = np.random.RandomState(7)
    for m, P in [(10, 4), (1000, 16), (997, 1024), (5000, 1024)]:
        s = np.sort(rs.randint(0, 50, size=m)).astype(np.uint64)
        k = L.pl_knots(s, P)
        for j in range(P + 1):
            # smallest value v in s such that #(s < v) ... brute force: the
            # value at the first rank r with r >= j*m/P
            r = next(r for r in range(m) if r * P >= j * m) if j * m <= (m - 1) * P else m - 1
            assert k[j] == s[r]
        assert np.all(np.diff(k.astype(np.int64)) >= 0)


def test_bucket_of_counts_splitters():
    rs = np.random.RandomState(8)
    spl = np.sort(rs.randint(0, 1000, size=31)).astype(np.uint64)
    keys = rs.randint(0, 1100, size=5000).astype(np.uint64)
    b = L.bucket_of(keys, spl)
    for i in range(0, 5000, 97):
        assert b[i] == sum(int(s) <= int(keys[i]) for s in spl)
