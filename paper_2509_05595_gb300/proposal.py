"""Learned proposal (no counterpart in the paper): a per-edge network that
predicts which collapses the exact intersection check (Section 5.2) would
undo (Section 5.3), so that the simplification defers them for a round
instead of collapsing, checking and undoing them.  Every committed collapse
still passes the exact check; the plain method stays the fallback (a round
after one that committed nothing defers nothing).

Training data are the accept / reject labels the plain method produces: the
16 features of every winner of a round (pamo_ctx_winner_features) and
whether its collapse stood after the undo loop.  The network is trained by
the library's own kernels (pamo_mlp_grad, pamo_mlp_adam_step); this module
only orders the calls and prepares minibatches.
"""
from __future__ import annotations

import numpy as np

from . import MLP, MLP_IN, MLP_PARAMS, Ctx, Options

H = 64
O_W1, O_B1 = 0, MLP_IN * H
O_W2 = O_B1 + H
O_B2 = O_W2 + H * H
O_W3 = O_B2 + H
O_B3 = O_W3 + H


def he_init(seed=0):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(MLP_PARAMS, np.float32)
    p[O_W1:O_B1] = rng.normal(0.0, np.sqrt(2.0 / MLP_IN), MLP_IN * H)
    p[O_W2:O_B2] = rng.normal(0.0, np.sqrt(2.0 / H), H * H)
    p[O_W3:O_B3] = rng.normal(0.0, np.sqrt(1.0 / H), H)
    return p


def log_winners(V, F, target, options: Options | None = None, max_rounds=400):
    """Simplify with the plain method, round by round, and return (X, y):
    the features of every winner (torch CUDA, [n, 16]) and 1.0 where its
    collapse was undone by the intersection check."""
    import torch
    c = Ctx(V, F, options or Options())
    Xs, ys = [], []
    nF, idle = len(F), 0
    try:
        for _ in range(max_rounds):
            if nF <= target:
                break
            c.round_cost()
            nW = c.round_select()
            X = c.winner_features(nW).clone() if nW else None
            c.round_collapse()
            c.round_check_undo()
            if nW:
                s = c.winner_standing(nW)
                Xs.append(X)
                ys.append((1 - s.to(torch.float32)))
            nF = c.round_commit()
            idle = idle + 1 if nW == 0 else 0
            if idle >= 3:
                break
    finally:
        c.close()
    if not Xs:
        return (torch.empty((0, MLP_IN), device="cuda"), torch.empty(0, device="cuda"))
    return torch.cat(Xs), torch.cat(ys)


def train(X, y, steps=2000, batch=8192, lr=2e-3, seed=0, pos_weight=None, log_every=0):
    """Train a network on (X, y) with weighted binary cross-entropy and Adam,
    all in the library's kernels; returns (MLP taking raw features, losses)."""
    import torch
    X = X.contiguous()
    y = y.to(torch.float32).contiguous()
    npos = float(y.sum().item())
    nneg = float(len(y) - npos)
    pw = pos_weight if pos_weight is not None else max(1.0, nneg / max(npos, 1.0))
    m = MLP(he_init(seed))
    m.fit_input_norm(X)  # mean / sd on the device; applied in the kernels (FP32)
    rng = np.random.default_rng(seed + 1)
    n = len(y)
    losses = []
    perm = torch.as_tensor(rng.permutation(n), device=X.device)
    pos = 0
    for step in range(steps):
        if pos + batch > n:
            perm = torch.as_tensor(rng.permutation(n), device=X.device)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        loss = m.grad(X.index_select(0, idx), y.index_select(0, idx), pw)
        m.adam_step(lr)
        if log_every and step % log_every == 0:
            losses.append(loss)
    return m, dict(losses=losses, pos_weight=pw, positives=int(npos), samples=n)
