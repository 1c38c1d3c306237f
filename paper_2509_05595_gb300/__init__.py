"""Python binding of libpamo.so: the GB300 (sm_103a) parallel intersection-free
edge-collapse simplifier (the simplification stage of PaMO, arXiv 2509.05595:
Algorithm 1, Eq. 1, Sections 5.1-5.3, Algorithm 3).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors; the current torch stream is
passed to the library.  There is no CPU fallback: if the shared library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpamo.so")
_lib = None

STATUS = {0: "PAMO_OK", 1: "PAMO_EINVAL", 2: "PAMO_ENOMEM", 3: "PAMO_ECUDA",
          4: "PAMO_ESTALL", 5: "PAMO_ETIMEOUT", 6: "PAMO_ENOTMANIFOLD",
          7: "PAMO_EINTERNAL", 8: "PAMO_EINTERSECT"}
PAMO_OK, PAMO_ESTALL = 0, 4

KERNEL_CLASSES = ("adjacency", "cost", "select", "collapse", "bvh", "query", "commit", "other")

ROUND_FIELDS = ("nV", "nF", "nE", "link_rejects", "flagged", "eligible",
                "winners", "committed", "undone", "undo_iters", "pairs_found", "us")


class PamoError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().pamo_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")


class _Options(ctypes.Structure):
    _fields_ = [("w_e", ctypes.c_double), ("w_s", ctypes.c_double),
                ("tolerance", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("stall_limit", ctypes.c_int32), ("validate_input", ctypes.c_int32),
                ("check_mode", ctypes.c_int32), ("record_rounds", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("exact_target", ctypes.c_int32),
                ("max_cost", ctypes.c_double), ("grid_blocks_per_sm", ctypes.c_int32),
                ("resort_percent", ctypes.c_int32), ("proposal", ctypes.c_void_p),
                ("proposal_threshold", ctypes.c_float),
                ("check_input_intersections", ctypes.c_int32),
                ("recompute_quadrics", ctypes.c_int32), ("device_loop", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("undo_iters_hist", ctypes.c_int32 * 8),
                ("committed", ctypes.c_int64), ("undone", ctypes.c_int64),
                ("link_rejects", ctypes.c_int64), ("winners", ctypes.c_int64),
                ("nV_out", ctypes.c_int64), ("nF_out", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("bytes_model", ctypes.c_double),
                ("launches", ctypes.c_int64), ("class_ms", ctypes.c_double * 8),
                ("class_launches", ctypes.c_int64 * 8), ("class_bytes", ctypes.c_double * 8),
                ("class_flops", ctypes.c_double * 8), ("deferred", ctypes.c_int64),
                ("cost_edges", ctypes.c_int64), ("cost_f64", ctypes.c_int64)]


@dataclass
class Options:
    """pamo_options (defaults = the paper's: Eq. 1 weights, tolerance 4)."""
    w_e: float = 0.001
    w_s: float = 0.005
    tolerance: int = 4
    max_rounds: int = 100000
    stall_limit: int = 12
    validate_input: int = 1
    check_mode: int = 0
    record_rounds: int = 0
    profile: int = 0
    exact_target: int = 0
    max_cost: float = float("inf")
    grid_blocks_per_sm: int = 0
    resort_percent: int = 0
    proposal: object = None        # an MLP (learned proposal) or None
    proposal_threshold: float = 0.5
    check_input_intersections: int = 0
    recompute_quadrics: int = 0
    device_loop: int = 0           # 1: all rounds in one graph launch (conditional nodes)

    def c(self):
        d = {f.name: getattr(self, f.name) for f in fields(self)}
        p = d.pop("proposal")
        o = _Options(**d)
        o.proposal = p.handle.value if isinstance(p, MLP) else p
        return o


MLP_IN, MLP_HIDDEN, MLP_PARAMS = 16, 64, 5313


class MLP:
    """The learned proposal's network (pamo_mlp): 16 -> 64 -> 64 -> 1, BF16
    weights over FP32 master weights, trained with the library's kernels."""

    def __init__(self, params=None):
        self.handle = ctypes.c_void_p()
        _check(lib().pamo_mlp_create(ctypes.byref(self.handle)), "pamo_mlp_create")
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        if p.shape != (MLP_PARAMS,):
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        _check(lib().pamo_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)),
               "pamo_mlp_set_params")

    def set_input_norm(self, mu, sd):
        """Standardise inputs as (x - mu) / sd before the first layer."""
        mu = np.ascontiguousarray(mu, np.float32)
        sd = np.ascontiguousarray(sd, np.float32)
        _check(lib().pamo_mlp_set_input_norm(self.handle, mu.ctypes.data_as(ctypes.c_void_p),
                                             sd.ctypes.data_as(ctypes.c_void_p)),
               "pamo_mlp_set_input_norm")

    def fit_input_norm(self, X):
        """Standardise inputs by the per-feature mean and standard deviation of
        the rows of X (computed by the library on the device)."""
        import torch
        X = _dev(X, torch.float32, MLP_IN)
        _check(lib().pamo_mlp_fit_input_norm(self.handle, _ptr(X), X.shape[0], _stream()),
               "pamo_mlp_fit_input_norm")

    def get_params(self):
        """(fp32 master parameters, bf16 copy as uint16 bit patterns)."""
        p = np.zeros(MLP_PARAMS, np.float32)
        b = np.zeros(MLP_PARAMS, np.uint16)
        _check(lib().pamo_mlp_get_params(self.handle, p.ctypes.data_as(ctypes.c_void_p),
                                         b.ctypes.data_as(ctypes.c_void_p)), "pamo_mlp_get_params")
        return p, b

    def forward(self, X):
        import torch
        X = _dev(X, torch.float32, MLP_IN)
        out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        _check(lib().pamo_mlp_forward(self.handle, _ptr(X), X.shape[0], _ptr(out), _stream()),
               "pamo_mlp_forward")
        return out

    def grad(self, X, y, pos_weight=1.0):
        """Loss (and the gradient, kept in the model) of the weighted BCE."""
        import torch
        X = _dev(X, torch.float32, MLP_IN)
        y = _dev(y, torch.float32)
        loss = ctypes.c_float()
        _check(lib().pamo_mlp_grad(self.handle, _ptr(X), _ptr(y), X.shape[0],
                                   ctypes.c_float(pos_weight), _stream(), ctypes.byref(loss)),
               "pamo_mlp_grad")
        return loss.value

    def get_grad(self):
        g = np.zeros(MLP_PARAMS, np.float32)
        _check(lib().pamo_mlp_get_grad(self.handle, g.ctypes.data_as(ctypes.c_void_p)),
               "pamo_mlp_get_grad")
        return g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().pamo_mlp_adam_step(self.handle, ctypes.c_float(lr), ctypes.c_float(beta1),
                                        ctypes.c_float(beta2), ctypes.c_float(eps), _stream()),
               "pamo_mlp_adam_step")

    def close(self):
        if self.handle:
            lib().pamo_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lib():
    """Load libpamo.so (built by paper_2509_05595_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        pi64 = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "pamo_default_options": (None, [P]),
            "pamo_simplify": (ctypes.c_int, [P, i64, P, i64, i64, P, P, P, pi64, P, pi64, P]),
            "pamo_simplify_host": (ctypes.c_int, [P, i64, P, i64, i64, P, P, P, pi64, P, pi64, P]),
            "pamo_simplify_batch": (ctypes.c_int, [i32, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                                   P]),
            "pamo_autotune_batch": (ctypes.c_int, [i32, P, P, P, P, P, P, P, P, P, P]),
            "pamo_ctx_winner_features": (ctypes.c_int, [P, P]),
            "pamo_ctx_winner_standing": (ctypes.c_int, [P, P]),
            "pamo_ctx_set_deferrals": (ctypes.c_int, [P, P, i64, P]),
            "pamo_mlp_create": (ctypes.c_int, [ctypes.POINTER(P)]),
            "pamo_mlp_destroy": (None, [P]),
            "pamo_mlp_set_params": (ctypes.c_int, [P, P]),
            "pamo_mlp_set_input_norm": (ctypes.c_int, [P, P, P]),
            "pamo_mlp_fit_input_norm": (ctypes.c_int, [P, P, i64, P]),
            "pamo_mlp_get_params": (ctypes.c_int, [P, P, P]),
            "pamo_mlp_forward": (ctypes.c_int, [P, P, i64, P, P]),
            "pamo_mlp_grad": (ctypes.c_int, [P, P, P, i64, ctypes.c_float, P, P]),
            "pamo_mlp_get_grad": (ctypes.c_int, [P, P]),
            "pamo_mlp_adam_step": (ctypes.c_int, [P, ctypes.c_float, ctypes.c_float,
                                                  ctypes.c_float, ctypes.c_float, P]),
            "pamo_ctx_create": (ctypes.c_int, [P, i64, P, i64, P, P, ctypes.POINTER(P)]),
            "pamo_round_cost": (ctypes.c_int, [P]),
            "pamo_round_select": (ctypes.c_int, [P, pi64]),
            "pamo_round_collapse": (ctypes.c_int, [P]),
            "pamo_round_check_undo": (ctypes.c_int, [P, ctypes.POINTER(i32)]),
            "pamo_round_commit": (ctypes.c_int, [P, pi64]),
            "pamo_ctx_sizes": (ctypes.c_int, [P, pi64, pi64, pi64]),
            "pamo_ctx_export": (ctypes.c_int, [P, P, P, P, P]),
            "pamo_ctx_round_info": (ctypes.c_int, [P, i64, P]),
            "pamo_ctx_round_pairs": (ctypes.c_int, [P, i64, i32, P, i64, pi64]),
            "pamo_ctx_rounds": (ctypes.c_int, [P, pi64]),
            "pamo_ctx_run": (ctypes.c_int, [P, i64, P]),
            "pamo_ctx_destroy": (None, [P]),
            "pamo_check_self_intersections": (ctypes.c_int, [P, i64, P, i64, P, pi64, P, i64]),
            "pamo_check_self_intersections_noalloc": (ctypes.c_int,
                                                      [P, i64, P, i64, P, pi64, P, i64]),
            "pamo_tri_intersect_batch": (ctypes.c_int, [P, P, i64, P, P]),
            "pamo_orient3d_batch": (ctypes.c_int, [P, i64, P, P]),
            "pamo_orient2d_batch": (ctypes.c_int, [P, i64, P, P]),
            "pamo_last_error": (ctypes.c_char_p, []),
            "pamo_release_cached_memory": (ctypes.c_int, []),
            "pamo_measure_fp64": (ctypes.c_int, [P, P]),
            "pamo_skinny_terms": (ctypes.c_int, [P, i64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, cols=None):
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    t = t.to(device="cuda", dtype=dtype).contiguous()
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"expected [n, {cols}] array, got {tuple(t.shape)}")
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check(code, where, ok=(PAMO_OK,)):
    if code not in ok:
        raise PamoError(code, where)
    return code


def _stats_dict(s: _Stats):
    return dict(rounds=s.rounds, undo_iters_hist=list(s.undo_iters_hist),
                committed=s.committed, undone=s.undone, link_rejects=s.link_rejects,
                winners=s.winners, nV_out=s.nV_out, nF_out=s.nF_out,
                ms_total=s.ms_total, bytes_model=s.bytes_model, launches=s.launches,
                class_ms=list(s.class_ms), class_launches=list(s.class_launches),
                class_bytes=list(s.class_bytes), class_flops=list(s.class_flops),
                deferred=s.deferred, cost_edges=s.cost_edges, cost_f64=s.cost_f64)


def pamo_simplify(V, F, target_faces, options: Options | None = None, **kw):
    """Simplify a closed manifold mesh on the GPU until |F| <= target_faces.

    V: [nV,3] float32, F: [nF,3] int32 (torch CUDA tensors or array-likes).
    Returns (V', F', stats, status) with V', F' CUDA tensors; status is
    "PAMO_OK" or "PAMO_ESTALL" (valid output above the target)."""
    import torch
    o = options or Options(**kw)
    V = _dev(V, torch.float32, 3)
    F = _dev(F, torch.int32, 3)
    Vo = torch.empty_like(V)
    Fo = torch.empty_like(F)
    nv, nf = ctypes.c_int64(), ctypes.c_int64()
    st = _Stats()
    opt = o.c()
    code = lib().pamo_simplify(_ptr(V), V.shape[0], _ptr(F), F.shape[0], int(target_faces),
                               ctypes.byref(opt), _stream(), _ptr(Vo), ctypes.byref(nv),
                               _ptr(Fo), ctypes.byref(nf), ctypes.byref(st))
    _check(code, "pamo_simplify", ok=(PAMO_OK, PAMO_ESTALL))
    return Vo[: nv.value], Fo[: nf.value], _stats_dict(st), STATUS[code]


def concat_meshes(meshes):
    """Concatenate [(V, F), ...] (each F indexing its own V from 0) into the
    batch layout: V [sum nV, 3], vertex offsets, F [sum nF, 3], face offsets."""
    Vs = [np.ascontiguousarray(v, np.float32) for v, _ in meshes]
    Fs = [np.ascontiguousarray(f, np.int32) for _, f in meshes]
    voff = np.concatenate([[0], np.cumsum([len(v) for v in Vs])]).astype(np.int64)
    foff = np.concatenate([[0], np.cumsum([len(f) for f in Fs])]).astype(np.int64)
    return np.concatenate(Vs), voff, np.concatenate(Fs), foff


def pamo_simplify_batch(V, voff, F, foff, targets, options: Options | None = None, **kw):
    """Simplify many closed manifold meshes in one pass: every round runs once
    over the whole batch and each mesh keeps its own normalisation, target,
    flags and termination (each output equals that mesh simplified alone).

    V: [sum nV, 3] float32 and F: [sum nF, 3] int32 concatenated (torch CUDA
    tensors or array-likes; each mesh's faces index its own vertices from 0);
    voff, foff: the M + 1 vertex / face offsets (host); targets: M face
    targets.  Returns (V', voff', F', foff', status[M], rounds[M], stats)."""
    import torch
    o = options or Options(**kw)
    V = _dev(V, torch.float32, 3)
    F = _dev(F, torch.int32, 3)
    voff = np.ascontiguousarray(voff, np.int64)
    foff = np.ascontiguousarray(foff, np.int64)
    M = len(voff) - 1
    tg = np.ascontiguousarray(targets, np.int64)
    if len(foff) != M + 1 or len(tg) != M:
        raise ValueError("offsets need M + 1 entries and targets M")
    Vo = torch.empty_like(V)
    Fo = torch.empty_like(F)
    vo = np.zeros(M + 1, np.int64)
    fo = np.zeros(M + 1, np.int64)
    status = np.zeros(M, np.int32)
    rounds = np.zeros(M, np.int32)
    st = _Stats()
    opt = o.c()
    code = lib().pamo_simplify_batch(
        M, _ptr(V), voff.ctypes.data_as(ctypes.c_void_p), _ptr(F),
        foff.ctypes.data_as(ctypes.c_void_p), tg.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(opt), _stream(), _ptr(Vo), vo.ctypes.data_as(ctypes.c_void_p), _ptr(Fo),
        fo.ctypes.data_as(ctypes.c_void_p), status.ctypes.data_as(ctypes.c_void_p),
        rounds.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
    _check(code, "pamo_simplify_batch", ok=(PAMO_OK, PAMO_ESTALL))
    return (Vo[: vo[-1]], vo, Fo[: fo[-1]], fo, [STATUS[int(x)] for x in status], rounds,
            _stats_dict(st))


def pamo_autotune_batch(V, voff, F, foff, targets, options: Options | None = None, **kw):
    """Choose the speed-only knobs (grid_blocks_per_sm, resort_percent) for a
    batch by timing candidate runs on it.  Returns (Options, trial_ms)."""
    import torch
    o = options or Options(**kw)
    V = _dev(V, torch.float32, 3)
    F = _dev(F, torch.int32, 3)
    voff = np.ascontiguousarray(voff, np.int64)
    foff = np.ascontiguousarray(foff, np.int64)
    tg = np.ascontiguousarray(targets, np.int64)
    best = _Options()
    ms = np.zeros(8, np.float64)
    nt = ctypes.c_int32()
    base = o.c()
    code = lib().pamo_autotune_batch(
        len(voff) - 1, _ptr(V), voff.ctypes.data_as(ctypes.c_void_p), _ptr(F),
        foff.ctypes.data_as(ctypes.c_void_p), tg.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(base), _stream(), ctypes.byref(best), ms.ctypes.data_as(ctypes.c_void_p),
        ctypes.byref(nt))
    _check(code, "pamo_autotune_batch")
    chosen = Options(**{f.name: getattr(best, f.name) for f in fields(Options)})
    return chosen, ms[: nt.value].tolist()


def pamo_simplify_host(V, F, target_faces, options: Options | None = None, **kw):
    """pamo_simplify on host (numpy) arrays; copies in and out inside the call."""
    o = options or Options(**kw)
    V = np.ascontiguousarray(V, dtype=np.float32)
    F = np.ascontiguousarray(F, dtype=np.int32)
    Vo = np.empty_like(V)
    Fo = np.empty_like(F)
    nv, nf = ctypes.c_int64(), ctypes.c_int64()
    st = _Stats()
    opt = o.c()
    code = lib().pamo_simplify_host(V.ctypes.data_as(ctypes.c_void_p), V.shape[0],
                                    F.ctypes.data_as(ctypes.c_void_p), F.shape[0],
                                    int(target_faces), ctypes.byref(opt), _stream(),
                                    Vo.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nv),
                                    Fo.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf),
                                    ctypes.byref(st))
    _check(code, "pamo_simplify_host", ok=(PAMO_OK, PAMO_ESTALL))
    return Vo[: nv.value], Fo[: nf.value], _stats_dict(st), STATUS[code]


class Ctx:
    """A simplification context (pamo_ctx) for round-by-round control."""

    def __init__(self, V, F, options: Options | None = None, **kw):
        import torch
        o = options or Options(**kw)
        self._V = _dev(V, torch.float32, 3)
        self._F = _dev(F, torch.int32, 3)
        self._h = ctypes.c_void_p()
        opt = o.c()
        _check(lib().pamo_ctx_create(_ptr(self._V), self._V.shape[0], _ptr(self._F),
                                     self._F.shape[0], ctypes.byref(opt), _stream(),
                                     ctypes.byref(self._h)), "pamo_ctx_create")

    def round_cost(self):
        _check(lib().pamo_round_cost(self._h), "pamo_round_cost")

    def round_select(self):
        n = ctypes.c_int64()
        _check(lib().pamo_round_select(self._h, ctypes.byref(n)), "pamo_round_select")
        return n.value

    def round_collapse(self):
        _check(lib().pamo_round_collapse(self._h), "pamo_round_collapse")

    def round_check_undo(self):
        n = ctypes.c_int32()
        _check(lib().pamo_round_check_undo(self._h, ctypes.byref(n)), "pamo_round_check_undo")
        return n.value

    def round_commit(self):
        n = ctypes.c_int64()
        _check(lib().pamo_round_commit(self._h, ctypes.byref(n)), "pamo_round_commit")
        return n.value

    def sizes(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pamo_ctx_sizes(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "pamo_ctx_sizes")
        return a.value, b.value, c.value

    def export(self, keys=False):
        """Current mesh (and, with keys=True, edge keys and endpoints)."""
        import torch
        nv, nf, ne = self.sizes()
        V = torch.empty((nv, 3), dtype=torch.float32, device="cuda")
        F = torch.empty((nf, 3), dtype=torch.int32, device="cuda")
        K = E = None
        if keys:
            K = torch.empty(ne, dtype=torch.int64, device="cuda")
            E = torch.empty((ne, 2), dtype=torch.int32, device="cuda")
        _check(lib().pamo_ctx_export(self._h, _ptr(V), _ptr(F), _ptr(K) if keys else None,
                                     _ptr(E) if keys else None), "pamo_ctx_export")
        return (V, F, K, E) if keys else (V, F)

    def rounds(self):
        n = ctypes.c_int64()
        code = lib().pamo_ctx_rounds(self._h, ctypes.byref(n))
        return n.value, STATUS[code]

    def round_info(self, r):
        out = np.zeros(12, np.int64)
        _check(lib().pamo_ctx_round_info(self._h, r, out.ctypes.data_as(ctypes.c_void_p)),
               "pamo_ctx_round_info")
        return dict(zip(ROUND_FIELDS, (int(x) for x in out)))

    def round_pairs(self, r, kind):
        n = ctypes.c_int64()
        _check(lib().pamo_ctx_round_pairs(self._h, r, kind, None, 0, ctypes.byref(n)),
               "pamo_ctx_round_pairs")
        out = np.zeros((max(n.value, 1), 2), np.int32)
        _check(lib().pamo_ctx_round_pairs(self._h, r, kind, out.ctypes.data_as(ctypes.c_void_p),
                                          n.value, ctypes.byref(n)), "pamo_ctx_round_pairs")
        return out[: n.value]

    def winner_features(self, n_winners):
        """[n_winners, 16] float32 features of this round's winners (after
        round_select): the learned proposal's inputs."""
        import torch
        X = torch.empty((max(n_winners, 1), MLP_IN), dtype=torch.float32, device="cuda")
        _check(lib().pamo_ctx_winner_features(self._h, _ptr(X)), "pamo_ctx_winner_features")
        return X[:n_winners]

    def winner_standing(self, n_winners):
        """[n_winners] uint8: 1 where the collapse stands after the undo loop."""
        import torch
        s = torch.empty(max(n_winners, 1), dtype=torch.uint8, device="cuda")
        _check(lib().pamo_ctx_winner_standing(self._h, _ptr(s)), "pamo_ctx_winner_standing")
        return s[:n_winners]

    def set_deferrals(self, rounds):
        """Defer, in round r, the winners whose vertex pairs are rows of
        rounds[r] (int [n, 2], a < b, that round's numbering): they are not
        collapsed and count as undone.  Call before the first round."""
        arrs = [np.ascontiguousarray(np.asarray(p, np.int32).reshape(-1, 2)) for p in rounds]
        off = np.zeros(len(arrs) + 1, np.int64)
        off[1:] = np.cumsum([len(a) for a in arrs])
        pairs = (np.concatenate(arrs) if arrs and off[-1] else np.zeros((1, 2), np.int32))
        pairs = np.ascontiguousarray(pairs, np.int32)
        _check(lib().pamo_ctx_set_deferrals(self._h, off.ctypes.data_as(ctypes.c_void_p),
                                            len(arrs), pairs.ctypes.data_as(ctypes.c_void_p)),
               "pamo_ctx_set_deferrals")

    def run(self, target_faces):
        st = _Stats()
        code = lib().pamo_ctx_run(self._h, int(target_faces), ctypes.byref(st))
        _check(code, "pamo_ctx_run", ok=(PAMO_OK, PAMO_ESTALL))
        return _stats_dict(st), STATUS[code]

    def close(self):
        if self._h:
            lib().pamo_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pamo_check_self_intersections(V, F, cap=1 << 20):
    """All intersecting face pairs (Algorithm 3 over every face)."""
    import torch
    V = _dev(V, torch.float32, 3)
    F = _dev(F, torch.int32, 3)
    out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    n = ctypes.c_int64()
    _check(lib().pamo_check_self_intersections(_ptr(V), V.shape[0], _ptr(F), F.shape[0],
                                               _stream(), ctypes.byref(n), _ptr(out), cap),
           "pamo_check_self_intersections")
    return n.value, out[: min(n.value, cap)]


def _require(t, name, dtype, cols):
    """Check, without converting, that t is a contiguous CUDA tensor of dtype
    and shape [n, cols] on the current device."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor, got one on {t.device}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: expected a tensor on cuda:{torch.cuda.current_device()}, "
                         f"got {t.device}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.dim() != 2 or t.shape[1] != cols:
        raise ValueError(f"{name}: expected shape [n, {cols}], got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")


def pamo_check_self_intersections_noalloc(V, F, out):
    """pamo_check_self_intersections for callers that cannot allocate device
    memory during the call: the library uses its fixed internal scratch (at
    most 32,768 faces and vertices) and writes up to len(out) pairs into the
    caller's int32 CUDA tensor out [cap, 2].  V, F must already be contiguous
    CUDA tensors of the right dtype (float32 [nV,3], int32 [nF,3]) on the
    current device; nothing is converted or allocated here, and anything else
    raises ValueError.  Returns the number of intersecting pairs."""
    import torch
    _require(V, "V", torch.float32, 3)
    _require(F, "F", torch.int32, 3)
    _require(out, "out", torch.int32, 2)
    n = ctypes.c_int64()
    _check(lib().pamo_check_self_intersections_noalloc(
        _ptr(V), V.shape[0], _ptr(F), F.shape[0], _stream(), ctypes.byref(n), _ptr(out),
        out.shape[0]), "pamo_check_self_intersections_noalloc")
    return n.value


def pamo_tri_intersect_batch(P, idx):
    """The triangle-pair predicate: P [n,18] float32, idx [n,6] int32 -> bool [n]."""
    import torch
    P = _dev(P, torch.float32, 18)
    idx = _dev(idx, torch.int32, 6)
    out = torch.empty(P.shape[0], dtype=torch.uint8, device="cuda")
    _check(lib().pamo_tri_intersect_batch(_ptr(P), _ptr(idx), P.shape[0], _ptr(out), _stream()),
           "pamo_tri_intersect_batch")
    return out.bool()


def pamo_orient3d_batch(P):
    import torch
    P = _dev(P, torch.float32, 12)
    out = torch.empty(P.shape[0], dtype=torch.int8, device="cuda")
    _check(lib().pamo_orient3d_batch(_ptr(P), P.shape[0], _ptr(out), _stream()),
           "pamo_orient3d_batch")
    return out


def pamo_orient2d_batch(P):
    import torch
    P = _dev(P, torch.float32, 6)
    out = torch.empty(P.shape[0], dtype=torch.int8, device="cuda")
    _check(lib().pamo_orient2d_batch(_ptr(P), P.shape[0], _ptr(out), _stream()),
           "pamo_orient2d_batch")
    return out


def pamo_skinny_terms(T):
    """Both evaluations of the skinny term 1 - C_ijk (Eq. 1) of triangles T
    ([n, 9] float32: placement, then the other two corners): the float64 value
    the edge-cost kernel computes, and the float-float pair ([n, 2] float32)
    it certifies keys with (NaN outside the certified range)."""
    import torch
    T = _dev(T, torch.float32, 9)
    t64 = torch.empty(T.shape[0], dtype=torch.float64, device="cuda")
    tff = torch.empty((T.shape[0], 2), dtype=torch.float32, device="cuda")
    _check(lib().pamo_skinny_terms(_ptr(T), T.shape[0], _ptr(t64), _ptr(tff), _stream()),
           "pamo_skinny_terms")
    return t64, tff


def pamo_last_error():
    return lib().pamo_last_error().decode()


def pamo_measure_fp64():
    """Measured float64 rates of the current GPU: dict of fused multiply-adds,
    divisions and square roots per second."""
    out = np.zeros(3, np.float64)
    _check(lib().pamo_measure_fp64(_stream(), out.ctypes.data_as(ctypes.c_void_p)),
           "pamo_measure_fp64")
    return dict(fma_per_s=float(out[0]), div_per_s=float(out[1]), sqrt_per_s=float(out[2]))


def pamo_release_cached_memory():
    """Return the device and pinned host memory the library keeps between
    calls (and no live context uses) to the CUDA driver."""
    _check(lib().pamo_release_cached_memory(), "pamo_release_cached_memory")
