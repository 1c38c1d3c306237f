"""Oracle of the learned proposal's network (TEST INFRASTRUCTURE ONLY: only
tests/, the smoke check and the benchmark's CPU leg may use it; the product
path never does).

Plain float64 NumPy restatement of the per-edge MLP 16 -> 64 -> 64 -> 1
(ReLU, ReLU, logistic), its mean weighted binary cross-entropy
    L = mean_s -(pw y_s log p_s + (1 - y_s) log(1 - p_s)),
the gradient of L by backpropagation, and one Adam step (Kingma & Ba,
"Adam: a method for stochastic optimization", 2015: m <- b1 m + (1-b1) g,
v <- b2 v + (1-b2) g^2, p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)).

Parameter layout (flat): W1 [16][64] at 0, b1 [64] at 1024, W2 [64][64] at
1088, b2 [64] at 5184, W3 [64] at 5248, b3 at 5312; W[i][j] maps input i to
output j.  The paper has no learned component; this network is the
proposal of the build's design (deferring predicted rejects of Section 5.3).
"""
import numpy as np

IN, H = 16, 64
O_W1, O_B1 = 0, IN * H
O_W2 = O_B1 + H
O_B2 = O_W2 + H * H
O_W3 = O_B2 + H
O_B3 = O_W3 + H
N_PARAMS = O_B3 + 1


def unpack(p):
    p = np.asarray(p, np.float64)
    return (p[O_W1:O_B1].reshape(IN, H), p[O_B1:O_W2], p[O_W2:O_B2].reshape(H, H),
            p[O_B2:O_W3], p[O_W3:O_B3], p[O_B3])


def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest even), returned as
    float32: the precision the network's weights are used in."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def forward(p, X, mu=None, sd=None):
    """Logits z, and the hidden activations, of rows X [n, 16] (standardised
    first as (X - mu) / sd when mu and sd are given)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    if mu is not None:
        X = (X - np.asarray(mu, np.float64)) / np.asarray(sd, np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    z = a2 @ W3 + b3
    return z, (X, z1, h1, z2, a2)


def prob(p, X, mu=None, sd=None):
    z, _ = forward(p, X, mu, sd)
    return 1.0 / (1.0 + np.exp(-z))


def loss_grad(p, X, y, pos_weight=1.0):
    """(L, dL/dp) of the mean weighted binary cross-entropy."""
    y = np.asarray(y, np.float64)
    n = len(y)
    z, (Xd, z1, h1, z2, a2) = forward(p, X)
    W1, b1, W2, b2, W3, b3 = unpack(p)
    # log p = -softplus(-z), log(1 - p) = -softplus(z)
    sp = lambda t: np.logaddexp(0.0, t)  # noqa: E731
    L = np.mean(pos_weight * y * sp(-z) + (1.0 - y) * sp(z))
    pz = 1.0 / (1.0 + np.exp(-z))
    d3 = (pos_weight * y * (pz - 1.0) + (1.0 - y) * pz) / n      # dL/dz
    g = np.zeros(N_PARAMS)
    g[O_W3:O_B3] = a2.T @ d3
    g[O_B3] = d3.sum()
    d2 = np.outer(d3, W3) * (z2 > 0)                                # dL/dz2
    g[O_W2:O_B2] = (h1.T @ d2).ravel()
    g[O_B2:O_W3] = d2.sum(0)
    d1 = (d2 @ W2.T) * (z1 > 0)                                     # dL/dz1
    g[O_W1:O_B1] = (Xd.T @ d1).ravel()
    g[O_B1:O_W2] = d1.sum(0)
    return L, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
