"""Pins for the oracle of the learned proposal's network (oracle/mlp.py).

The network is the build's own design (the paper has no learned component), so
the pins come from calculus and from the published Adam update: the gradient
must match central finite differences of the loss; with every weight zero the
network is the constant sigmoid(b3); with pass-through hidden layers it is
logistic regression; Adam's first step from a zero state moves every
parameter by lr * g / (|g| + eps).
"""
import numpy as np

from oracle import mlp


def _rand_params(rng, scale=0.5):
    return rng.normal(0.0, scale, mlp.N_PARAMS)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _rand_params(rng)
    X = rng.normal(size=(40, mlp.IN))
    y = (rng.random(40) < 0.3).astype(float)
    for pw in (1.0, 3.5):
        L, g = mlp.loss_grad(p, X, y, pw)
        idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
        idx = np.concatenate([idx, [mlp.O_B3, mlp.O_W3, mlp.O_B2, mlp.O_B1, 0]])
        h = 1e-6
        for i in idx:
            e = np.zeros(mlp.N_PARAMS)
            e[i] = h
            fd = (mlp.loss_grad(p + e, X, y, pw)[0] - mlp.loss_grad(p - e, X, y, pw)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_zero_network_is_a_constant():
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.O_B3] = 0.7
    X = np.random.default_rng(1).normal(size=(10, mlp.IN))
    assert np.allclose(mlp.prob(p, X), 1 / (1 + np.exp(-0.7)))
    y = np.array([1, 0] * 5, float)
    L, g = mlp.loss_grad(p, X, y, 2.0)
    pz = 1 / (1 + np.exp(-0.7))
    # only b3 has a gradient: mean of pw y (p - 1) + (1 - y) p
    assert np.isclose(g[mlp.O_B3], np.mean(2.0 * y * (pz - 1) + (1 - y) * pz))
    assert np.count_nonzero(g) == 1
    assert np.isclose(L, np.mean(-2.0 * y * np.log(pz) - (1 - y) * np.log(1 - pz)))


def test_pass_through_network_is_logistic_regression():
    # W1 = [I | 0], W2 = [I | 0] on positive inputs: z = w . x + b
    rng = np.random.default_rng(2)
    w = rng.normal(size=mlp.IN)
    p = np.zeros(mlp.N_PARAMS)
    W1 = np.zeros((mlp.IN, mlp.H)); W1[:, :mlp.IN] = np.eye(mlp.IN)
    W2 = np.zeros((mlp.H, mlp.H)); W2[:mlp.IN, :mlp.IN] = np.eye(mlp.IN)
    W3 = np.zeros(mlp.H); W3[:mlp.IN] = w
    p[mlp.O_W1:mlp.O_B1] = W1.ravel()
    p[mlp.O_W2:mlp.O_B2] = W2.ravel()
    p[mlp.O_W3:mlp.O_B3] = W3
    p[mlp.O_B3] = -0.3
    X = rng.random((25, mlp.IN))
    assert np.allclose(mlp.forward(p, X)[0], X @ w - 0.3)


def test_adam_first_step_is_a_sign_step():
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    q, m, v = mlp.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=1e-8)
    assert np.allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8))


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3e-39], np.float32)
    r = mlp.bf16_round(x)
    # 8 stored mantissa bits; ties to even
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 ** -6 and r[4] == -2.5
    assert (r.view(np.uint32) & 0xFFFF == 0).all()
