"""Topology checks for closed triangle meshes (numpy, test helper)."""
import numpy as np


def edges_of(F):
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]).astype(np.int64)
    return e


def is_closed_manifold(F, nV):
    """Every directed edge once, every reverse edge present (closed, oriented,
    edge-manifold), no repeated corners, and every vertex link one cycle."""
    F = np.asarray(F, np.int64)
    if len(F) == 0:
        return False
    if ((F[:, 0] == F[:, 1]) | (F[:, 1] == F[:, 2]) | (F[:, 2] == F[:, 0])).any():
        return False
    e = edges_of(F)
    k = e[:, 0] * nV + e[:, 1]
    kr = e[:, 1] * nV + e[:, 0]
    if len(np.unique(k)) != len(k):
        return False
    if not np.isin(kr, k).all():
        return False
    # vertex links: map x -> y for each face (v, x, y) around v
    nxt = {}
    for f in F:
        for c in range(3):
            v, x, y = f[c], f[(c + 1) % 3], f[(c + 2) % 3]
            nxt.setdefault(int(v), {})[int(x)] = int(y)
    for v, m in nxt.items():
        start = next(iter(m))
        cur, n = start, 0
        while True:
            cur = m[cur]
            n += 1
            if cur == start or n > len(m):
                break
        if n != len(m):
            return False
    used = np.unique(F)
    return len(used) == nV


def euler(F, nV):
    e = edges_of(np.asarray(F, np.int64))
    und = np.unique(np.sort(e, 1), axis=0)
    return nV - len(und) + len(F)


def components(F, nV):
    parent = list(range(nV))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for f in np.asarray(F):
        for c in range(3):
            a, b = find(int(f[c])), find(int(f[(c + 1) % 3]))
            if a != b:
                parent[a] = b
    return len({find(v) for v in range(nV)})
