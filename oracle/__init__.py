"""CPU oracle for the simplification path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so`` (built from
``oracle.cpp`` by ``oracle/build.py``), a plain single-threaded restatement of
Algorithm 1, Eq. 1 and Sections 5.1-5.3 of the paper.  It shares no code with
the CUDA library.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

W_E, W_S = 0.001, 0.005          # Eq. 1 default weights (Section 5.1)
TOLERANCE = 4                    # Section 5.3 default tolerance

CHECK_GRID, CHECK_CHANGED_BRUTE, CHECK_ALL_PAIRS, CHECK_NONE = 0, 1, 2, 3

ROUND_FIELDS = ("nV", "nF", "nE", "link_rejects", "flagged", "eligible",
                "winners", "committed", "undone", "undo_iters", "pairs_found")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.or_orient3d.restype = ctypes.c_int
        L.or_orient3d_exact.restype = ctypes.c_int
        L.or_orient2d.restype = ctypes.c_int
        L.or_orient2d_exact.restype = ctypes.c_int
        L.or_tri_intersect.restype = ctypes.c_int
        L.or_edge_table.restype = i64
        L.or_edge_table.argtypes = [P, i64, P, i64, P, i64, P, P, P, P, P, P]
        L.or_vertex_quadrics.argtypes = [P, i64, P, i64, P]
        L.or_run.restype = P
        L.or_run.argtypes = [P, i64, P, i64, i64, P, P]
        for name in ("or_free",):
            getattr(L, name).argtypes = [P]
        for name in ("or_status",):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = ctypes.c_int
        for name in ("or_rounds", "or_nv", "or_nf"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = i64
        L.or_scale.argtypes = [P]
        L.or_scale.restype = ctypes.c_double
        L.or_mesh.argtypes = [P, P, P, P]
        L.or_round_info.argtypes = [P, i64, P]
        L.or_round_pairs.argtypes = [P, i64, ctypes.c_int, P, i64]
        L.or_round_pairs.restype = i64
        L.or_self_intersections.argtypes = [P, i64, P, i64, P, i64, ctypes.c_int]
        L.or_tri_quality.argtypes = [P]
        L.or_tri_quality.restype = ctypes.c_double
        L.or_set_plain_products.argtypes = [ctypes.c_int]
        L.or_self_intersections.restype = i64
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def orient3d(a, b, c, d, exact=False):
    p = _f32(np.concatenate([a, b, c, d]).ravel())
    f = lib().or_orient3d_exact if exact else lib().or_orient3d
    return int(f(_ptr(p)))


def orient2d(a, b, c, exact=False):
    p = _f32(np.concatenate([a, b, c]).ravel())
    f = lib().or_orient2d_exact if exact else lib().or_orient2d
    return int(f(_ptr(p)))


def tri_intersect(T, C, ti=(0, 1, 2), ci=(3, 4, 5)):
    """Exact self-intersection predicate for two mesh faces (Algorithm 3).

    T, C: 3x3 corner positions; ti, ci: their vertex indices (shared indices
    select the vertex-/edge-sharing cases)."""
    p = _f32(np.concatenate([np.asarray(T).ravel(), np.asarray(C).ravel()]))
    idx = _i32(np.concatenate([ti, ci]))
    return bool(lib().or_tri_intersect(_ptr(p), _ptr(idx)))


def vertex_quadrics(V, F):
    V, F = _f32(V), _i32(F)
    K = np.zeros((len(V), 10), np.float64)
    lib().or_vertex_quadrics(_ptr(V), len(V), _ptr(F), len(F), _ptr(K))
    return K


def edge_table(V, F, w_e=W_E, w_s=W_S, plain_products=False):
    """Round-0 edge table: dict of arrays (ab, key, vbar, Q, l, Cs, cost, link_ok,
    vsolve = the float64 placement before rounding, NaN where the fallback is taken).

    ``key`` is ~0 for ineligible edges.  plain_products=True evaluates every
    fused multiply-add of the cost as a multiply and an add (two roundings)
    instead of the fixed fma order of reading R13."""
    if plain_products:
        lib().or_set_plain_products(1)
        try:
            return edge_table(V, F, w_e, w_s)
        finally:
            lib().or_set_plain_products(0)
    V, F = _f32(V), _i32(F)
    cap = 3 * len(F)
    ab = np.zeros((cap, 2), np.int32)
    key = np.zeros(cap, np.uint64)
    vbar = np.zeros((cap, 3), np.float32)
    terms = np.zeros((cap, 4), np.float64)
    bits = np.zeros(cap, np.int32)
    vsolve = np.zeros((cap, 3), np.float64)
    w = np.array([w_e, w_s], np.float64)
    n = lib().or_edge_table(_ptr(V), len(V), _ptr(F), len(F), _ptr(w), cap,
                            _ptr(ab), _ptr(key), _ptr(vbar), _ptr(terms), _ptr(bits),
                            _ptr(vsolve))
    return dict(ab=ab[:n], key=key[:n], vbar=vbar[:n], Q=terms[:n, 0],
                l=terms[:n, 1], Cs=terms[:n, 2], cost=terms[:n, 3],
                link_ok=bits[:n].astype(bool), vsolve=vsolve[:n])


class Result:
    """Outcome of one oracle run: mesh, status and per-round logs."""

    def __init__(self, V, F, K, status, rounds, scale):
        self.V, self.F, self.K = V, F, K
        self.status = status
        self.rounds = rounds
        self.scale = scale


def simplify(V, F, target, w_e=W_E, w_s=W_S, tolerance=TOLERANCE,
             max_rounds=100000, stall_limit=12, check_mode=CHECK_GRID,
             keep_pairs=True, exact_target=0, max_cost=float("inf"), recompute_quadrics=0):
    """Algorithm 1 on the CPU.  exact_target / max_cost: the two termination
    refinements of Section 5.1 (keep only the lowest-key winners needed to
    reach N_t; edges costing more than max_cost are not eligible)."""
    V, F = _f32(V), _i32(F)
    L = lib()
    w = np.array([w_e, w_s, max_cost], np.float64)
    iopt = np.array([tolerance, max_rounds, stall_limit, check_mode, exact_target,
                     recompute_quadrics], np.int32)
    h = L.or_run(_ptr(V), len(V), _ptr(F), len(F), int(target), _ptr(w), _ptr(iopt))
    try:
        nv, nf = L.or_nv(h), L.or_nf(h)
        Vo = np.zeros((nv, 3), np.float32)
        Fo = np.zeros((nf, 3), np.int32)
        Ko = np.zeros((nv, 10), np.float64)
        L.or_mesh(h, _ptr(Vo), _ptr(Fo), _ptr(Ko))
        rounds = []
        info = np.zeros(11, np.int64)
        for r in range(L.or_rounds(h)):
            L.or_round_info(h, r, _ptr(info))
            d = dict(zip(ROUND_FIELDS, (int(x) for x in info)))
            if keep_pairs:
                for kind, name in ((0, "winner_pairs"), (1, "committed_pairs"),
                                   (2, "undone_pairs")):
                    n = L.or_round_pairs(h, r, kind, None, 0)
                    buf = np.zeros((max(n, 1), 2), np.int32)
                    L.or_round_pairs(h, r, kind, _ptr(buf), n)
                    d[name] = buf[:n]
            rounds.append(d)
        return Result(Vo, Fo, Ko, L.or_status(h), rounds, L.or_scale(h))
    finally:
        L.or_free(h)


def self_intersections(V, F, cap=1 << 20, brute=False):
    """All intersecting face pairs (exact predicate).

    brute=True tests every face pair (O(F^2)); otherwise box-overlap
    candidates from a uniform cell grid."""
    V, F = _f32(V), _i32(F)
    out = np.zeros((cap, 2), np.int32)
    n = lib().or_self_intersections(_ptr(V), len(V), _ptr(F), len(F), _ptr(out),
                                    cap, 1 if brute else 0)
    return out[:min(n, cap)], int(n)


def tri_quality(q0, q1, q2):
    """C_ijk of Eq. 1 for one triangle given in float64."""
    q = np.ascontiguousarray(np.concatenate([q0, q1, q2]), dtype=np.float64)
    return float(lib().or_tri_quality(_ptr(q)))
