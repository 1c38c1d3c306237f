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


def _plain_run_with_rounds(V, F, target):
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F), record_rounds=1)
    st, status = c.run(target)
    n, _ = c.rounds()
    rounds = []
    for r in range(n):
        d = c.round_info(r)
        d["committed_pairs"] = c.round_pairs(r, 1)
        d["undone_pairs"] = c.round_pairs(r, 2)
        rounds.append(d)
    Vo, Fo = c.export()
    c.close()
    return Vo.cpu().numpy(), Fo.cpu().numpy(), st, status, rounds


def test_perfect_deferral_replays_the_plain_run_without_undo_iterations():
    """The bound on the learned proposal: deferring, in every round, exactly
    the winners the plain run's check undid (pamo_ctx_set_deferrals) gives the
    plain run's output and per-round committed / undone sets, with a single
    clean check per round -- all the undo work a predictor could save."""
    V, F = meshgen.nested_shells(5, check=False)
    target = len(F) // 60
    Vp, Fp, stp, sp, rp = _plain_run_with_rounds(V, F, target)
    undone = [d["undone_pairs"] for d in rp]
    assert sum(len(u) for u in undone) > 50 and stp["undo_iters_hist"][0] < stp["rounds"]
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F), record_rounds=1)
    c.set_deferrals(undone)
    st, status = c.run(target)
    n, _ = c.rounds()
    assert status == sp and n == len(rp)
    for r in range(n):
        d = c.round_info(r)
        assert d["undo_iters"] == 0 and d["pairs_found"] == 0, r
        assert d["winners"] == rp[r]["winners"] and d["committed"] == rp[r]["committed"], r
        assert np.array_equal(c.round_pairs(r, 1), rp[r]["committed_pairs"]), r
        assert np.array_equal(c.round_pairs(r, 2), rp[r]["undone_pairs"]), r
    Vo, Fo = c.export()
    c.close()
    assert np.array_equal(Fo.cpu().numpy(), Fp)
    assert np.array_equal(Vo.cpu().numpy().view(np.uint32), Vp.view(np.uint32))
    assert st["deferred"] == sum(len(u) for u in undone)
    assert st["undo_iters_hist"][0] == st["rounds"]


def test_deferral_schedule_arguments():
    V, F = meshgen.nested_shells(3, check=False)
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F))
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        c.set_deferrals([np.array([[5, 3]])])          # a > b
    c.round_cost()
    with pytest.raises(pamo.PamoError, match="EINVAL"):  # after the first round began
        c.set_deferrals([np.zeros((0, 2))])
    c.close()


def _features_cpu(V, F, ab, vbar, cost, scale):
    """The 16 winner features restated in float32 numpy from their definition
    (round 0: no clearance known yet, no survivor of an earlier round)."""
    f32 = np.float32
    P = V.astype(f32)
    out = np.zeros((len(ab), 16), f32)
    faces_of = [[] for _ in range(len(V))]
    for fi, t in enumerate(F):
        for x in t:
            faces_of[x].append(fi)
    for i, (a, b) in enumerate(ab):
        pa, pb, v = P[a], P[b], vbar[i].astype(f32)
        l = max(f32(np.linalg.norm(pb - pa)), f32(1e-30))
        mincos, sumcos, minq, sumskin, aold, anew, dmax = f32(1), f32(0), f32(1), f32(0), f32(0), f32(0), f32(0)
        ntri, nab = 0, []
        seen = set()
        for x in (a, b):
            for fi in faces_of[x]:
                if fi in seen:
                    continue
                seen.add(fi)
                t = F[fi]
                q = P[t]
                n_old = np.cross(q[1] - q[0], q[2] - q[0]).astype(f32)
                lo = f32(np.linalg.norm(n_old))
                aold += f32(0.5) * lo
                if lo > 0:
                    dmax = max(dmax, f32(abs(np.dot(n_old, v - q[0])) / lo))
                if a in t and b in t:
                    nab.append(n_old)
                    continue
                r = np.array([v if c in (a, b) else P[c] for c in t], f32)
                u, w = r[1] - r[0], r[2] - r[0]
                n_new = np.cross(u, w).astype(f32)
                ln = f32(np.linalg.norm(n_new))
                c = f32(np.dot(n_new, n_old) / (ln * lo)) if ln > 0 and lo > 0 else f32(-1)
                mincos = min(mincos, c)
                sumcos += c
                den = f32(np.dot(u, u) + np.dot(w, w) + np.dot(w - u, w - u))
                qq = f32(3.4641016) * ln / den if den > 0 else f32(0)
                minq = min(minq, qq)
                sumskin += f32(1) - qq
                anew += f32(0.5) * ln
                ntri += 1
        dih = f32(1)
        if len(nab) == 2:
            l0, l1 = np.linalg.norm(nab[0]), np.linalg.norm(nab[1])
            dih = f32(np.dot(nab[0], nab[1]) / (l0 * l1)) if l0 > 0 and l1 > 0 else f32(-1)
        va, vb = len(faces_of[a]), len(faces_of[b])
        nt = f32(max(ntri, 1))
        mid = f32(0.5) * (pa + pb)
        gap = f32(np.inf)
        out[i] = [np.log10(max(cost[i], 1e-12)), np.log2(max(scale * l, 1e-12)),
                  np.linalg.norm(v - mid) / l, va / 6, vb / 6, (va + vb - 4) / 6, dih,
                  mincos, sumcos / nt, minq, sumskin / nt,
                  min(max(np.log2(max(dmax, 1e-30) / gap) if np.isfinite(gap) else -np.inf, -10), 10),
                  np.log2(max(aold / (l * l), 1e-12)), anew / aold if aold > 0 else 0,
                  min(max(np.log2(gap / l) if np.isfinite(gap) else np.inf, -10), 10), 0]
    return out


def test_winner_features_match_a_cpu_restatement():
    """Every one of the 16 features of the round-0 winners, restated in float32
    numpy from the definitions (the winners, their placements and costs from
    the oracle), element by element."""
    import oracle
    V, F = meshgen.nested_shells(4, check=False)
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F))
    c.round_cost()
    nW = c.round_select()
    X = c.winner_features(nW).cpu().numpy()
    c.close()
    ref = oracle.simplify(V, F, len(F) // 4, max_rounds=1)
    pairs = ref.rounds[0]["winner_pairs"]   # edge order, as the GPU lists winners
    assert len(pairs) == nW > 100
    T = oracle.edge_table(V, F)
    row = {tuple(p): i for i, p in enumerate(T["ab"].tolist())}
    idx = np.array([row[tuple(p)] for p in pairs.tolist()])
    cost = (T["key"][idx] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    scale = 1.0 / (V.astype(np.float64).max(0) - V.astype(np.float64).min(0)).max()
    want = _features_cpu(V, F, pairs, T["vbar"][idx], cost, np.float32(scale))
    assert np.allclose(X, want, rtol=2e-5, atol=2e-5), np.abs(X - want).max(0)


def test_fitted_input_norm_matches_numpy_statistics():
    """pamo_mlp_fit_input_norm (device, float64, fixed order) against numpy's
    mean and population standard deviation: the fitted model and one given
    numpy's statistics predict the same probabilities."""
    rng = np.random.default_rng(9)
    X = (rng.normal(size=(100003, 16)) * rng.uniform(0.01, 50, 16)
         + rng.uniform(-100, 100, 16)).astype(np.float32)
    X[:, 7] = 3.0  # a constant feature: sd taken as 1
    p = proposal.he_init(4)
    a, b = pamo.MLP(p), pamo.MLP(p)
    a.fit_input_norm(torch.from_numpy(X))
    Xd = X.astype(np.float64)
    sd = Xd.std(0)
    sd[sd < 1e-6] = 1.0
    b.set_input_norm(Xd.mean(0).astype(np.float32), sd.astype(np.float32))
    Q = torch.from_numpy(X[:5000])
    assert torch.allclose(a.forward(Q), b.forward(Q), rtol=1e-5, atol=1e-6)


def test_learned_against_plain_on_held_out_meshes(capsys):
    """The trained network against the plain method on held-out near-contact
    meshes: the time ratio and undo work are reported; every output must be
    closed, manifold and free of exact self-intersections, with a one-sided
    Hausdorff distance to the input within 1.05x of the plain output's, on
    average and on every mesh."""
    from bench import one_sided_hausdorff
    Xs, ys = [], []
    for seed in range(12):
        V, F = meshgen.nested_shells_seeded(5, 1000 + seed)
        X, y = proposal.log_winners(V, F, len(F) // 100)
        Xs.append(X)
        ys.append(y)
    X, y = torch.cat(Xs), torch.cat(ys)
    m, _ = proposal.train(X, y, steps=400, batch=4096, lr=2e-3, pos_weight=1.0)
    ratios, t_plain, t_learned, undo = [], 0.0, 0.0, [0, 0]
    for seed in range(2000, 2004):
        V, F = meshgen.nested_shells_seeded(5, seed)
        Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
        out = {}
        for name, kw in (("plain", {}), ("learned", dict(proposal=m, proposal_threshold=0.9))):
            for _ in range(2):  # the second run is timed
                c = pamo.Ctx(Vd, Fd, **kw)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                st, status = c.run(len(F) // 100)
                e1.record()
                e1.synchronize()
                Vo, Fo = c.export()
                c.close()
            Vh, Fh = Vo.cpu().numpy(), Fo.cpu().numpy()
            # a near-contact mesh may stop above 1 % (a valid output, Section 5.3)
            assert status in ("PAMO_OK", "PAMO_ESTALL") and is_closed_manifold(Fh, len(Vh))
            assert euler(Fh, len(Vh)) == euler(F, len(V))
            assert pamo.pamo_check_self_intersections(Vo, Fo)[0] == 0
            out[name] = (e0.elapsed_time(e1), one_sided_hausdorff(Vh, Fh, V, F), st)
        t_plain += out["plain"][0]
        t_learned += out["learned"][0]
        undo[0] += sum(i * n for i, n in enumerate(out["plain"][2]["undo_iters_hist"]))
        undo[1] += sum(i * n for i, n in enumerate(out["learned"][2]["undo_iters_hist"]))
        ratios.append(out["learned"][1] / out["plain"][1])
    with capsys.disabled():
        print(f"\nlearned vs plain on 4 held-out level-5 shells: time x{t_learned / t_plain:.3f}, "
              f"undo iterations {undo[1]} vs {undo[0]}, Hausdorff ratio mean "
              f"{np.mean(ratios):.3f} max {np.max(ratios):.3f}")
    assert np.mean(ratios) <= 1.05 and np.max(ratios) <= 1.05
