"""fp64 oracle for the learned CDF bucketing (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this follows the configuration that adds
one to the method: a small CDF model fit on the sample the method already
draws (Alg. 2 step 1) proposes bucket boundaries in place of fixed digits.
Bucket membership itself stays an exact integer comparison with the
boundaries, so the sort's output is unchanged.

Model (1 -> 16 -> 16 -> 1, tanh hidden layers, linear output):
    z1 = W1 x + b1,  h1 = tanh(z1)
    z2 = W2 h1 + b2, h2 = tanh(z2)
    y  = W3 h2 + b3
Loss over a batch of B pairs (x_i, t_i):  L = (1/B) sum_i (y_i - t_i)^2.
Parameters are flattened in the order W1[16,1], b1[16], W2[16,16] (row-major,
W2[j,k] multiplies h1[k]), b2[16], W3[1,16], b3[1]: 321 values.

Adam (Kingma & Ba 2015):  m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
    p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Piecewise-linear CDF: knot k (k = 0..P) sits at the exact empirical
k/P-quantile of the sorted sample.
"""
import numpy as np

H = 16
NPARAM = H + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H].reshape(H, 1); o += H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H].reshape(1, H); o += H
    b3 = p[o:o + 1]; o += 1
    assert o == NPARAM
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2),
                           np.ravel(b2), np.ravel(W3), np.ravel(b3)])


def forward(p, x):
    """y for a batch x (shape [B]); also returns the activations."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x[:, None] * W1[:, 0][None, :] + b1[None, :]
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2[None, :]
    h2 = np.tanh(z2)
    y = h2 @ W3[0] + b3[0]
    return y, (x, h1, h2)


def loss(p, x, t):
    y, _ = forward(p, x)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def backward(p, x, t):
    """Gradient of the mean squared error with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (x, h1, h2) = forward(p, x)
    B = len(x)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B          # [B]
    dW3 = (dy[:, None] * h2).sum(axis=0)[None, :]                   # [1,H]
    db3 = np.array([dy.sum()])
    dh2 = dy[:, None] * W3[0][None, :]                              # [B,H]
    dz2 = dh2 * (1.0 - h2 * h2)
    dW2 = dz2.T @ h1                                                # [H,H]
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2                                                  # [B,H]
    dz1 = dh1 * (1.0 - h1 * h1)
    dW1 = (dz1 * x[:, None]).sum(axis=0)[:, None]                   # [H,1]
    db1 = dz1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(p, g, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train(p0, x, t, steps, batch, lr=1e-2):
    """Adam on consecutive mini-batches x[(s*batch) % len : ...] (wrapping)."""
    p = np.array(p0, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    n = len(x)
    losses = []
    for s in range(steps):
        lo = (s * batch) % n
        idx = (lo + np.arange(batch)) % n
        g = backward(p, x[idx], t[idx])
        losses.append(loss(p, x[idx], t[idx]))
        p, m, v = adam_step(p, g, m, v, s + 1, lr=lr)
    return p, losses


def pl_knots(sorted_sample, P):
    """Knot k = smallest sample value whose rank r (0-based) has r >= k*m/P,
    i.e. the exact empirical k/P quantile; knot P is the largest sample."""
    s = np.asarray(sorted_sample)
    m = len(s)
    ks = []
    for k in range(P + 1):
        r = min(m - 1, (k * m + P - 1) // P)   # ceil(k*m/P), clamped
        ks.append(s[r])
    return np.array(ks, dtype=s.dtype)


def bucket_of(keys, splitters):
    """Exact bucket of every key for increasing splitters s_1..s_{B-1}:
    the number of splitters <= key (bucket j holds [s_j, s_{j+1}))."""
    return np.searchsorted(np.asarray(splitters), np.asarray(keys), side="right")
