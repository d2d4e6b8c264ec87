"""Conforming recovery of free segments in the oracle. TEST INFRASTRUCTURE
ONLY: used by the tests, the smoke check and the benchmark's CPU legs; the
CUDA path has its own implementation and shares no code with this one.

The paper takes a CDT of the PLC as its input (Sec. 1) and does not say how
it is built. Reading used here: the initial mesh is the Delaunay mesh of the
input points plus midpoints on the free segments. In passes, every subsegment
that is not an edge of the Delaunay mesh of the current points is split at its
midpoint (all of a pass's missing subsegments together, in segment order, then
along each segment from its first end); the new points are inserted, and the
next pass checks again. When no subsegment is missing, every segment is a
chain of Delaunay edges, and the Delaunay mesh is a CDT of the segments.
"""
from __future__ import annotations

import numpy as np


def _edge_keys(tets):
    t = np.asarray(tets, dtype=np.int64)
    e = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    e.sort(axis=1)
    return np.unique((e[:, 0] << 32) | e[:, 1])


def recover_segments(pts, segs, max_passes=64):
    """Returns (mesh, coordinates, chains, passes): the oracle's box Delaunay
    mesh of the points and the recovery's midpoints (appended after the input
    points, in the order they were made), and each segment's vertex chain."""
    from . import Mesh, midpoint
    X = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    m = Mesh.box_delaunay(X)
    if m.skipped:
        raise ValueError("duplicate input points")
    chains = [[int(a), int(b)] for a, b in np.asarray(segs)]
    for npass in range(max_passes):
        E = _edge_keys(m.export()["tets"])
        miss = []
        for s, ch in enumerate(chains):
            c = np.asarray(ch, dtype=np.int64)
            lo_, hi_ = np.minimum(c[:-1], c[1:]), np.maximum(c[:-1], c[1:])
            k = (lo_ << 32) | hi_
            pos = np.searchsorted(E, k)
            ok = (pos < len(E)) & (E[np.minimum(pos, len(E) - 1)] == k)
            for j in np.nonzero(~ok)[0]:
                miss.append((s, int(j)))
        if not miss:
            return m, X, chains, npass
        new = np.array([midpoint(X[chains[s][j]], X[chains[s][j + 1]]) for s, j in miss])
        ids = len(X) + np.arange(len(miss))
        X = np.ascontiguousarray(np.concatenate([X, new]))
        by_seg = {}
        for (s, j), v in zip(miss, ids):
            by_seg.setdefault(s, []).append((j, int(v)))
        for s, lst in by_seg.items():
            for j, v in sorted(lst, reverse=True):
                chains[s].insert(j + 1, v)
        if m.insert_points(new) != 0:
            raise ValueError("a midpoint coincides with a point")
    raise RuntimeError("segment recovery did not finish in %d passes" % max_passes)


# ------------------------------------------------------------------ facets
# Reading used for triangles (facets) that are not unions of faces of the
# points' Delaunay mesh (Sec. 1 asks that every polygon of the PLC appear as a
# union of triangles of the mesh): the same passes, segments first. Once every
# subsegment is an edge, each facet's points (the vertices of the chains of
# its three edges and the points already inserted on it) are triangulated in
# the facet's plane by the Delaunay rule, with the in-facet circle test of a
# subface (the lifted insphere against the facet's reference point q_f,
# reading c7); triangles whose three vertices lie on one edge's chain lie
# outside the facet and are left out. The lexicographically first of these
# triangles that is not a face of the mesh is split: at its circumcentre,
# unless that point lies strictly inside the diametral sphere of one of the
# facet's subsegments, which are then split at their midpoints instead. A
# pass first inserts every midpoint (in segment order, then along each
# segment), then the facets' circumcentres (in facet order). When nothing is
# missing, each facet is the union of its triangles, all faces of the mesh.


def facet_reference(X, a, b, c, s):
    """q_f of facet (a, b, c): a moved by s along the axis of the largest
    component of (b - a) x (c - a), ties to the lower axis (reading c7)."""
    A, Bp, C = X[a], X[b], X[c]
    ux, uy, uz = float(Bp[0] - A[0]), float(Bp[1] - A[1]), float(Bp[2] - A[2])
    vx, vy, vz = float(C[0] - A[0]), float(C[1] - A[1]), float(C[2] - A[2])
    n = [uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx]
    k = 0
    for j in (1, 2):
        if abs(n[j]) > abs(n[k]):
            k = j
    q = [float(A[0]), float(A[1]), float(A[2])]
    q[k] = q[k] + s
    return np.array(q)


def reference_shift(X):
    """The smallest power of two at least 4 x the largest bounding-box extent."""
    ex = float(np.max(np.max(X, axis=0) - np.min(X, axis=0)))
    s = 1.0
    while s < 4.0 * ex:
        s *= 2.0
    while s * 0.5 >= 4.0 * ex and s > 1e-300:
        s *= 0.5
    return s


def facet_delaunay(X, V, q, chains):
    """Triangles of the facet's points V by the in-facet Delaunay rule (no
    point strictly inside a triangle's circle), each as sorted ids, skipping
    triangles whose vertices all lie on one of `chains` (vertex sets)."""
    from . import insphere, orient3d
    V = sorted(int(v) for v in V)
    out = []
    for x in range(len(V)):
        for y in range(x + 1, len(V)):
            for z in range(y + 1, len(V)):
                i, j, k = V[x], V[y], V[z]
                if any(i in c and j in c and k in c for c in chains):
                    continue
                o = orient3d(X[i], X[j], X[k], q)
                if o == 0:
                    continue
                t = (i, j, k) if o > 0 else (i, k, j)
                if all(insphere(X[t[0]], X[t[1]], X[t[2]], q, X[p]) <= 0
                       for p in V if p not in (i, j, k)):
                    out.append((i, j, k))
    return out


def _face_keys(tets):
    t = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    f = np.concatenate([t[:, [1, 2, 3]], t[:, [0, 2, 3]], t[:, [0, 1, 3]], t[:, [0, 1, 2]]])
    return set(map(tuple, np.unique(f, axis=0).tolist()))


def recover_plc(pts, segs, tris, tri_segs, max_passes=400):
    """Conforming recovery of free segments and triangle facets.

    pts: input points (8 box corners first); segs: (m, 2) segments between
    input points, among them every triangle edge once; tris: (t, 3) facets;
    tri_segs: (t, 3) the segment of each facet's edges (a, b), (b, c), (c, a).
    Returns a dict: mesh (the oracle's box Delaunay mesh of all points), xyz,
    chains (each segment's vertex ids from its first end), facet_points (the
    points inserted on each facet), subfaces (per facet, its triangles as
    sorted ids), facetq (q_f per facet), passes."""
    from . import Mesh, midpoint, tri_circumcenter, diametral
    X = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    n_in = len(X)
    s_ref = reference_shift(X)
    tris = [tuple(int(v) for v in t) for t in np.asarray(tris).reshape(-1, 3)]
    tri_segs = [tuple(int(v) for v in t) for t in np.asarray(tri_segs).reshape(-1, 3)]
    Q = [facet_reference(X, a, b, c, s_ref) for a, b, c in tris]
    m = Mesh.box_delaunay(X)
    if m.skipped:
        raise ValueError("duplicate input points")
    chains = [[int(a), int(b)] for a, b in np.asarray(segs).reshape(-1, 2)]
    fpts = [[] for _ in tris]
    for npass in range(max_passes):
        tets = m.export()["tets"]
        E = _edge_keys(tets)
        split = []
        for s, ch in enumerate(chains):
            c = np.asarray(ch, dtype=np.int64)
            k = (np.minimum(c[:-1], c[1:]) << 32) | np.maximum(c[:-1], c[1:])
            pos = np.searchsorted(E, k)
            ok = (pos < len(E)) & (E[np.minimum(pos, len(E) - 1)] == k)
            split += [(s, int(j)) for j in np.nonzero(~ok)[0]]
        new_f = []
        facets = None
        if not split:
            F = _face_keys(tets)
            facets = []
            enc = set()
            for f, (a, b, c) in enumerate(tris):
                cs = [chains[s] for s in tri_segs[f]]
                V = set(fpts[f])
                for ch in cs:
                    V.update(ch)
                T = facet_delaunay(X, V, Q[f], [set(ch) for ch in cs])
                facets.append(T)
                miss = sorted(t for t in T if t not in F)
                if not miss:
                    continue
                t = miss[0]
                p, ok = tri_circumcenter(X[t[0]], X[t[1]], X[t[2]])
                if not ok:
                    raise RuntimeError("degenerate facet triangle %s" % (t,))
                hit = [(s, j) for s in tri_segs[f] for j in range(len(chains[s]) - 1)
                       if diametral(X[chains[s][j]], X[chains[s][j + 1]], p) < 0]
                if hit:
                    enc.update(hit)
                else:
                    new_f.append((f, p))
            split = sorted(enc)
        if not split and not new_f:
            return dict(mesh=m, xyz=X, chains=chains, facet_points=fpts, subfaces=facets,
                        facetq=np.array(Q).reshape(-1, 3), passes=npass, n_in=n_in)
        mids = [midpoint(X[chains[s][j]], X[chains[s][j + 1]]) for s, j in split]
        new = mids + [p for _, p in new_f]
        ids = len(X) + np.arange(len(new))
        X = np.ascontiguousarray(np.concatenate([X, np.array(new).reshape(-1, 3)]))
        by_seg = {}
        for (s, j), v in zip(split, ids[: len(split)]):
            by_seg.setdefault(s, []).append((j, int(v)))
        for s, lst in by_seg.items():
            for j, v in sorted(lst, reverse=True):
                chains[s].insert(j + 1, v)
        for (f, _), v in zip(new_f, ids[len(split):]):
            fpts[f].append(int(v))
        if m.insert_points(np.array(new).reshape(-1, 3)) != 0:
            raise ValueError("a recovery point coincides with a point")
    raise RuntimeError("recovery did not finish in %d passes" % max_passes)
