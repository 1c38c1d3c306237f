"""The learned proposal on the GPU: the network's forward pass, gradient and
Adam step against the float64 oracle (oracle/mlp.py, with the same BF16
weights), the exported edge features, training by the library's kernels, and
a simplification with deferral that must stay closed, manifold and free of
self-intersections (every committed collapse still passes the exact check).
"""
import numpy as np
import pytest

import meshgen
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2509_05595_gb300 as pamo  # noqa: E402
from paper_2509_05595_gb300 import proposal  # noqa: E402
from tests.meshcheck import euler, is_closed_manifold  # noqa: E402


def _model(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, omlp.N_PARAMS).astype(np.float32)
    return pamo.MLP(p), omlp.bf16_round(p).astype(np.float64)


def test_forward_matches_oracle():
    m, pb = _model(1)
    _, bits = m.get_params()
    assert np.array_equal(bits.astype(np.uint32) << 16,
                          omlp.bf16_round(m.get_params()[0]).view(np.uint32))
    X = np.random.default_rng(2).normal(size=(5000, 16)).astype(np.float32)
    got = m.forward(torch.from_numpy(X)).cpu().numpy()
    want = omlp.prob(pb, X)
    assert np.max(np.abs(got - want)) < 2e-5


def test_input_standardisation_matches_oracle():
    m, pb = _model(7)
    rng = np.random.default_rng(8)
    mu = rng.normal(0, 3, 16).astype(np.float32)
    sd = rng.uniform(0.1, 5, 16).astype(np.float32)
    m.set_input_norm(mu, sd)
    X = (mu + sd * rng.normal(size=(4000, 16))).astype(np.float32)
    got = m.forward(torch.from_numpy(X)).cpu().numpy()
    # the kernel multiplies by the float32 reciprocal of sd
    inv = (np.float32(1.0) / sd).astype(np.float64)
    want = omlp.prob(pb, X, mu.astype(np.float64), 1.0 / inv)
    assert np.max(np.abs(got - want)) < 2e-5


def test_gradient_matches_oracle_and_is_deterministic():
    m, pb = _model(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(7777, 16)).astype(np.float32)   # several chunks and a ragged tail
    y = (rng.random(7777) < 0.2).astype(np.float32)
    loss = m.grad(torch.from_numpy(X), torch.from_numpy(y), 3.0)
    g = m.get_grad()
    L, gw = omlp.loss_grad(pb, X, y, 3.0)
    assert abs(loss - L) <= 1e-5 * abs(L)
    assert np.max(np.abs(g - gw)) <= 1e-4 * np.max(np.abs(gw))
    m.grad(torch.from_numpy(X), torch.from_numpy(y), 3.0)
    assert np.array_equal(m.get_grad(), g)  # fixed reduction order


def test_adam_step_matches_oracle():
    m, pb = _model(5)
    p0, _ = m.get_params()
    rng = np.random.default_rng(6)
    X = rng.normal(size=(3000, 16)).astype(np.float32)
    y = (rng.random(3000) < 0.5).astype(np.float32)
    mm = np.zeros(omlp.N_PARAMS)
    vv = np.zeros(omlp.N_PARAMS)
    p = p0.astype(np.float64)
    for t in (1, 2):
        m.grad(torch.from_numpy(X), torch.from_numpy(y), 1.0)
        g = m.get_grad().astype(np.float64)
        m.adam_step(1e-3)
        p, mm, vv = omlp.adam_step(p, g, mm, vv, t, 1e-3)
    got, bits = m.get_params()
    assert np.max(np.abs(got - p)) < 1e-6
    assert np.array_equal(bits.astype(np.uint32) << 16, omlp.bf16_round(got).view(np.uint32))


def test_winner_features_are_consistent():
    V, F = meshgen.nested_shells(4, check=False)
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F))
    c.round_cost()
    nW = c.round_select()
    X = c.winner_features(nW).cpu().numpy()
    c.close()
    assert X.shape == (nW, 16) and np.isfinite(X).all()
    val = np.bincount(F.ravel(), minlength=len(V))
    # valences / 6 and produced triangles = valence(a) + valence(b) - 4
    assert np.allclose(X[:, 5] * 6, X[:, 3] * 6 + X[:, 4] * 6 - 4, atol=1e-5)
    assert (X[:, 11] >= -10).all() and (X[:, 11] <= 10).all()
    assert set(np.round(X[:, 3] * 6).astype(int)) <= set(val.tolist())
    assert np.isin(X[:, 15], [0, 1]).all()
    # before the first check no clearance is known; nothing survived a collapse
    assert (X[:, 14] == 10).all() and (X[:, 15] == 0).all()
    assert (X[:, 2] >= 0).all() and (X[:, 9] <= 1.0 + 1e-6).all()


def test_training_and_deferral_keep_the_output_valid():
    # labels from the plain method on a few near-contact meshes
    Xs, ys = [], []
    for seed in range(4):
        V, F = meshgen.nested_shells_seeded(4, 1000 + seed)
        X, y = proposal.log_winners(V, F, len(F) // 20)
        Xs.append(X)
        ys.append(y)
    X, y = torch.cat(Xs), torch.cat(ys)
    assert 0 < y.sum().item() < len(y)
    m, info = proposal.train(X, y, steps=300, batch=2048, lr=3e-3, log_every=50)
    assert info["losses"][-1] < info["losses"][0]
    # deferral on a held-out mesh: still closed, manifold, intersection-free
    V, F = meshgen.nested_shells_seeded(4, 2000)
    assert pamo.pamo_check_self_intersections(V, F)[0] == 0
    Vo, Fo, st, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F),
                                            len(F) // 20, proposal=m, proposal_threshold=0.5)
    Fo_h = Fo.cpu().numpy()
    assert is_closed_manifold(Fo_h, len(Vo)) and euler(Fo_h, len(Vo)) == euler(F, len(V))
    n_pairs, _ = pamo.pamo_check_self_intersections(Vo, Fo)
    assert n_pairs == 0
    assert st["deferred"] > 0
