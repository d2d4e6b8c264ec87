"""Recovery of free segments for the initial mesh, on the GPU.

The refinement takes a constrained Delaunay mesh of the PLC as its input
(Sec. 1). When a PLC's segments are not all edges of its points' Delaunay
mesh, this builds one: in passes, the Delaunay mesh of the current points is
built on the device (cdr_delaunay_box, the library's point-insertion rounds),
every subsegment that is not one of its edges is split at its midpoint
(computed on the device by the library's midpoint formula, all of a pass's
missing subsegments together, in segment order, then along each segment from
its first end), and the midpoints join the points. When nothing is missing,
every segment is a chain of Delaunay edges and the last mesh is a CDT of the
segments. Untimed set-up for the benchmark and the tests.
"""
from __future__ import annotations

import itertools

import numpy as np


def _edges(tets):
    t = np.asarray(tets, dtype=np.int64)
    e = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    e.sort(axis=1)
    return np.unique((e[:, 0] << 32) | e[:, 1])


def _has(E, u, v):
    k = (np.minimum(u, v) << 32) | np.maximum(u, v)
    pos = np.searchsorted(E, k)
    return (pos < len(E)) & (E[np.minimum(pos, len(E) - 1)] == k)


def recover_segments(pts, segs, cdr, stream=None, max_passes=64):
    """Returns (xyz, tets, chains, passes): the points followed by the
    midpoints in the order they were made, their Delaunay mesh, and each
    segment's vertex chain."""
    xyz = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    chains = [np.asarray(s, dtype=np.int64) for s in np.asarray(segs)]
    for npass in range(max_passes):
        dt = cdr.Handle.delaunay_box(xyz, stream=stream)
        if dt.skipped:
            dt.close()
            raise ValueError("a point coincides with another")
        tets = dt.export()["tets"]
        dt.close()
        E = _edges(tets)
        where = [np.nonzero(~_has(E, c[:-1], c[1:]))[0] for c in chains]
        todo = [(s, int(j)) for s, w in enumerate(where) for j in w]
        if not todo:
            return xyz, tets, [c.tolist() for c in chains], npass
        items = np.zeros((len(todo), 16))
        for r, (s, j) in enumerate(todo):
            items[r, 0:3] = xyz[chains[s][j]]
            items[r, 3:6] = xyz[chains[s][j + 1]]
        _, mid = cdr.eval_predicates("midpoint", items, stream=stream)
        first = len(xyz)
        xyz = np.ascontiguousarray(np.concatenate([xyz, mid]))
        r = 0
        for s, w in enumerate(where):
            if len(w):
                ids = first + r + np.arange(len(w))
                chains[s] = np.insert(chains[s], w + 1, ids)
                r += len(w)
    raise RuntimeError("segment recovery did not finish in %d passes" % max_passes)


# ------------------------------------------------------------------ facets
# Triangles (facets) that are not unions of faces of the points' Delaunay mesh
# are recovered in the same passes, after the segments (Sec. 1: every polygon
# of the PLC must appear as a union of triangles of the mesh). Once every
# subsegment is an edge, a facet's points (its edges' chains and the points
# inserted on it) are triangulated in its plane by the Delaunay rule, using
# the in-facet circle test of the refinement (the lifted insphere against the
# facet's reference point q_f), every predicate evaluated on the device in one
# batch per pass; triangles with all three vertices on one edge's chain lie
# outside the facet and are dropped. Per facet and pass, the first triangle
# (by sorted vertex ids) that is not a face of the mesh is split at its
# circumcentre, or, if that point is strictly inside the diametral sphere of
# some of the facet's subsegments, those are split at their midpoints. A pass
# inserts the midpoints (by segment, then along it), then the circumcentres
# (by facet). Untimed set-up, like the segment recovery.

def _refs(xyz, tris):
    """q_f of each facet (a, b, c): a moved along the axis of the largest
    |component| of (b - a) x (c - a) (lower axis on ties) by the smallest power
    of two >= 4 x the largest extent of the points' bounding box."""
    ext = float((xyz.max(axis=0) - xyz.min(axis=0)).max())
    s = 1.0
    while s < 4.0 * ext:
        s *= 2.0
    while s * 0.5 >= 4.0 * ext and s > 1e-300:
        s *= 0.5
    out = np.empty((len(tris), 3))
    for f, (a, b, c) in enumerate(tris):
        p0, p1, p2 = xyz[a], xyz[b], xyz[c]
        u = [float(p1[k] - p0[k]) for k in range(3)]
        v = [float(p2[k] - p0[k]) for k in range(3)]
        n = (abs(u[1] * v[2] - u[2] * v[1]), abs(u[2] * v[0] - u[0] * v[2]),
             abs(u[0] * v[1] - u[1] * v[0]))
        axis = 0
        if n[1] > n[axis]:
            axis = 1
        if n[2] > n[axis]:
            axis = 2
        out[f] = p0
        out[f, axis] = float(p0[axis]) + s
    return out


def box_facet_refs(xyz, lab):
    """Reference points of every facet of labels `lab` (box facets 0..5 from
    their first triangle, the library's default rule)."""
    first = {}
    for t, f in zip(lab["tris"], lab["facet_id"]):
        first.setdefault(int(f), tuple(int(v) for v in t))
    return _refs(np.asarray(xyz), [first[f] for f in range(6)])


def _items(*pts):
    """(n, 16) predicate items from up to five (n, 3) point arrays."""
    n = len(pts[0])
    it = np.zeros((n, 16))
    for k, p in enumerate(pts):
        it[:, 3 * k:3 * k + 3] = p
    return it


_TRIPLES = {}


def _triples(k):
    """Index triples (a < b < c) of range(k), lexicographic, cached per k."""
    t = _TRIPLES.get(k)
    if t is None:
        t = np.asarray(list(itertools.combinations(range(k), 3)), dtype=np.int64).reshape(-1, 3)
        _TRIPLES[k] = t
    return t


def _facet_triangles(xyz, verts, chain_sets, q, ev):
    """Per facet: its Delaunay triangles (sorted id triples, sorted), from the
    device's orient3d and insphere signs, each kind in one batch."""
    cand, owner, vsets = [], [], []
    for f, V in enumerate(verts):
        V = np.asarray(sorted(V), dtype=np.int64)
        vsets.append(V)
        if len(V) < 3:
            continue
        tr = _triples(len(V))
        on = np.stack([np.isin(V, np.fromiter(c, dtype=np.int64)) for c in chain_sets[f]],
                      axis=1)  # (k, chains): vertex on chain
        one = (on[tr[:, 0]] & on[tr[:, 1]] & on[tr[:, 2]]).any(axis=1)
        cand.append(V[tr[~one]])
        owner.append(np.full(int((~one).sum()), f, dtype=np.int64))
    out = [[] for _ in verts]
    if not cand:
        return out
    T = np.concatenate(cand)
    own = np.concatenate(owner)
    if not len(T):
        return out
    o, _ = ev("orient", _items(xyz[T[:, 0]], xyz[T[:, 1]], xyz[T[:, 2]], q[own]))
    keep = np.nonzero(o != 0)[0]
    P = T[keep].copy()
    neg = o[keep] < 0
    P[neg, 1], P[neg, 2] = T[keep][neg, 2], T[keep][neg, 1]  # positively oriented
    # every other point of the facet against each kept triangle
    rows, pts_ = [], []
    ko = own[keep]
    for f in np.unique(ko):
        r = np.nonzero(ko == f)[0]
        V = vsets[f]
        other = ~((V[None, :] == T[keep][r][:, :1]) | (V[None, :] == T[keep][r][:, 1:2]) |
                  (V[None, :] == T[keep][r][:, 2:3]))
        rr, cc = np.nonzero(other)
        rows.append(r[rr])
        pts_.append(V[cc])
    rows = np.concatenate(rows)
    inside = np.zeros(len(keep), dtype=bool)
    if len(rows):
        pp = np.concatenate(pts_)
        s, _ = ev("insphere", _items(xyz[P[rows, 0]], xyz[P[rows, 1]], xyz[P[rows, 2]],
                                     q[own[keep][rows]], xyz[pp]))
        np.logical_or.at(inside, rows, s > 0)
    for r in np.nonzero(~inside)[0]:
        out[int(ko[r])].append(tuple(int(v) for v in T[keep[r]]))
    return [sorted(x) for x in out]


def recover_plc(pts, segs, tris, tri_segs, cdr, stream=None, max_passes=400, evaluate=None,
                delaunay=None):
    """Recovery of free segments and triangle facets on the device.

    pts: the input points (8 box corners first); segs: (m, 2) segments between
    them, every triangle edge among them once; tris: (t, 3) facets; tri_segs:
    (t, 3) the segment of each facet's edges (a, b), (b, c), (c, a). Returns a
    dict: xyz (the points, then the recovery's points in the order made), tets
    (their Delaunay mesh), chains (each segment's vertex ids from its first
    end), facet_points (the points made on each facet), subfaces (each facet's
    triangles, sorted id triples, all faces of tets), facetq (q_f per facet),
    passes. evaluate(kind, items) and delaunay(xyz) -> tets replace the
    device calls (cdr_eval_predicates, cdr_delaunay_box) where a test drives
    the pass logic with other primitives."""
    ev = evaluate or (lambda kind, items: cdr.eval_predicates(kind, items, stream=stream))

    def build(x):
        if delaunay is not None:
            return delaunay(x)
        dt = cdr.Handle.delaunay_box(x, stream=stream)
        try:
            if dt.skipped:
                raise ValueError("a point coincides with another")
            return dt.export()["tets"]
        finally:
            dt.close()

    xyz = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    facets = [tuple(int(v) for v in t) for t in np.asarray(tris).reshape(-1, 3)]
    fsegs = [tuple(int(v) for v in t) for t in np.asarray(tri_segs).reshape(-1, 3)]
    q = _refs(xyz, facets)
    chains = [np.asarray(s, dtype=np.int64) for s in np.asarray(segs).reshape(-1, 2)]
    fpts = [[] for _ in facets]
    for npass in range(max_passes):
        tets = build(xyz)
        E = _edges(tets)
        todo = [(s, int(j)) for s, c in enumerate(chains)
                for j in np.nonzero(~_has(E, c[:-1], c[1:]))[0]]
        on_facet = []  # (facet, circumcentre)
        subfaces = None
        if not todo:
            t4 = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
            fk = np.concatenate([t4[:, [1, 2, 3]], t4[:, [0, 2, 3]], t4[:, [0, 1, 3]],
                                 t4[:, [0, 1, 2]]])
            F = np.unique((fk[:, 0] << 42) | (fk[:, 1] << 21) | fk[:, 2])
            sets = [[set(chains[s].tolist()) for s in fsegs[f]] for f in range(len(facets))]
            verts = []
            for f in range(len(facets)):
                V = set(fpts[f])
                for c in sets[f]:
                    V |= c
                verts.append(V)
            subfaces = _facet_triangles(xyz, verts, sets, q, ev)
            first = []  # (facet, triangle) of each facet's first missing triangle
            for f, Tf in enumerate(subfaces):
                if not Tf:
                    continue
                A = np.asarray(Tf, dtype=np.int64)
                k = (A[:, 0] << 42) | (A[:, 1] << 21) | A[:, 2]
                pos = np.searchsorted(F, k)
                miss = ~((pos < len(F)) & (F[np.minimum(pos, len(F) - 1)] == k))
                if miss.any():
                    first.append((f, Tf[int(np.nonzero(miss)[0][0])]))
            if first:
                tt = np.asarray([t for _, t in first], dtype=np.int64)
                ok, cc = ev("tri_cc", _items(xyz[tt[:, 0]], xyz[tt[:, 1]], xyz[tt[:, 2]]))
                if not ok.all():
                    raise RuntimeError("a degenerate facet triangle")
                rows, subs = [], []
                for r, (f, _) in enumerate(first):
                    for s in fsegs[f]:
                        for j in range(len(chains[s]) - 1):
                            rows.append(r)
                            subs.append((s, j))
                a = np.asarray([chains[s][j] for s, j in subs], dtype=np.int64)
                b = np.asarray([chains[s][j + 1] for s, j in subs], dtype=np.int64)
                d, _ = ev("diametral", _items(xyz[a], xyz[b], cc[np.asarray(rows)]))
                hit = np.zeros(len(first), dtype=bool)
                enc = set()
                for r, sj, sg in zip(rows, subs, d):
                    if sg < 0:
                        hit[r] = True
                        enc.add(sj)
                todo = sorted(enc)
                on_facet = [(f, cc[r]) for r, (f, _) in enumerate(first) if not hit[r]]
        if not todo and not on_facet:
            return dict(xyz=xyz, tets=tets, chains=[c.tolist() for c in chains],
                        facet_points=fpts, subfaces=subfaces, facetq=q, passes=npass)
        new = []
        if todo:
            a = np.asarray([chains[s][j] for s, j in todo], dtype=np.int64)
            b = np.asarray([chains[s][j + 1] for s, j in todo], dtype=np.int64)
            _, mid = ev("midpoint", _items(xyz[a], xyz[b]))
            new.append(mid)
        if on_facet:
            new.append(np.asarray([p for _, p in on_facet]).reshape(-1, 3))
        first_id = len(xyz)
        xyz = np.ascontiguousarray(np.concatenate([xyz] + new))
        for r in sorted(range(len(todo)), key=lambda r: (todo[r][0], -todo[r][1])):
            s, j = todo[r]
            chains[s] = np.insert(chains[s], j + 1, first_id + r)
        for r, (f, _) in enumerate(on_facet):
            fpts[f].append(first_id + len(todo) + r)
    raise RuntimeError("recovery did not finish in %d passes" % max_passes)
