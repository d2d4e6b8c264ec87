"""Seeded synthetic inputs for the refinement step.

This module only draws random points and picks constraint edges and faces out
of a given Delaunay mesh; it holds none of the refinement method's arithmetic.
Both the CUDA path (tests, benchmark) and the CPU oracle (tests, CPU baseline)
take their inputs from here.

Recipes (all coordinates FP64):

* ``cube``      -- the unit-cube PLC: 8 corners, 12 edges, 6 square facets, plus
                   ``n`` points uniform in [0.05, 0.95]^3 (2,000 points, seed 0,
                   B = 2.0 in the small configuration).
* ``uniform``   -- ``n`` points uniform in [0, 1000]^3 plus the 8 box corners
                   (100,000 points, seed 1, B = 1.4 in the benchmark
                   configuration), with ``n_seg`` segments and ``n_tri``
                   triangles inside the box.
* ``clustered`` -- ``n`` points from an equal-weight mixture of 3 isotropic
                   Gaussians (sigma 50, centres uniform in the box), samples
                   outside the box redrawn.

Constraint recipe (the paper's own generator is unpublished): segments are
Delaunay edges of the point set and triangles are Delaunay faces, chosen
uniformly at random, with no two constraints sharing a vertex and no constraint
touching a box corner. Triangles must have every angle >= ``min_angle`` degrees
(45 by default). Since they are edges and faces of the Delaunay mesh and share no
vertex, the constraints never cross one another and the Delaunay mesh is already
a constrained Delaunay triangulation of the PLC. Every triangle edge is also a
segment, as a PLC polygon's boundary edges belong to E.

Facet ids: 0..5 are the box faces (x=lo, x=hi, y=lo, y=hi, z=lo, z=hi), then one
per triangle. Segment ids: 0..11 are the box edges, then the free segments, then
three per triangle.

Recovered recipe (``free_segments`` + ``plc_with_chains``, the single-mesh
workloads): the free segments join two input points drawn at random, the
second among the first's 16 nearest neighbours. A segment is rejected if it
shares a point with an earlier one or passes within a quarter of the shorter
length of an earlier one (in 3D two random segments never meet exactly, so
"crossing" is read as coming that close). Such segments are in general not
edges of the points' Delaunay mesh: the caller recovers them by inserting
midpoints (each segment becomes a chain of subsegments). The triangles are
then drawn among the faces of the recovered Delaunay mesh whose three corners
are input points touching no other constraint (every angle >= 45 degrees);
after each triangle, with probability 1/4, a second triangle sharing one of
its edges is added as a facet of its own when the two meet at a dihedral
angle of at least 70 degrees, so some interior facets share a segment.

Facet-recovered recipe (``free_segments`` + ``free_triangles``, for the
recovery of r18 and its tests): triangles between input points, a seed point
and two of its nearest neighbours, kept when their grown bounding balls meet
no other constraint's; each triangle edge becomes a segment, and some
triangles get an edge-sharing partner. Neither segments nor triangles need be
in the points' Delaunay mesh; the recovery makes them so. ``plc_recovered``
labels the result.
"""
from __future__ import annotations

import numpy as np

# recipe "delaunay": constraints among the Delaunay edges and faces
# (plc_from_delaunay); "recovered": free segments recovered by midpoints, then
# triangles among the recovered mesh's faces (free_segments, plc_with_chains)
CONFIGS = {
    "cube2k": dict(kind="cube", n=2000, seed=0, B=2.0, n_seg=0, n_tri=0, recipe="delaunay"),
    "uniform100k": dict(kind="uniform", n=100_000, seed=1, B=1.4, n_seg=1000, n_tri=1000,
                        recipe="recovered"),
    "clustered500k": dict(kind="clustered", n=500_000, seed=2, B=1.4, n_seg=5000, n_tri=5000,
                          recipe="recovered"),
}


def box_points(kind: str, n: int, seed: int) -> tuple[np.ndarray, float, float]:
    """Points with the 8 box corners first. Returns (points, lo, hi)."""
    rng = np.random.default_rng(seed)
    if kind == "cube":
        lo, hi = 0.0, 1.0
        inner = rng.uniform(0.05, 0.95, size=(n, 3))
    elif kind == "uniform":
        lo, hi = 0.0, 1000.0
        inner = rng.uniform(lo, hi, size=(n, 3))
    elif kind == "clustered":
        lo, hi = 0.0, 1000.0
        centres = rng.uniform(lo, hi, size=(3, 3))
        out = np.empty((0, 3))
        while len(out) < n:
            m = n - len(out)
            comp = rng.integers(0, 3, size=m)
            x = centres[comp] + rng.normal(0.0, 50.0, size=(m, 3))
            ok = np.all((x > lo) & (x < hi), axis=1)
            out = np.concatenate([out, x[ok]])
        inner = out[:n]
    elif kind == "ball":
        # uniform in the ball of radius 450 about the box centre
        lo, hi = 0.0, 1000.0
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        inner = 500.0 + 450.0 * d * rng.uniform(0.0, 1.0, size=(n, 1)) ** (1.0 / 3.0)
    else:
        raise ValueError(kind)
    corners = np.array([[hi if (c >> k) & 1 else lo for k in range(3)] for c in range(8)],
                       dtype=np.float64)
    # drop interior samples that landed exactly on the box surface (measure zero)
    on = np.any((inner == lo) | (inner == hi), axis=1)
    inner = inner[~on]
    return np.ascontiguousarray(np.concatenate([corners, inner])), lo, hi


def _faces_edges(tets: np.ndarray):
    t = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    faces = np.concatenate([t[:, [1, 2, 3]], t[:, [0, 2, 3]], t[:, [0, 1, 3]], t[:, [0, 1, 2]]])
    fk = (faces[:, 0] << 42) | (faces[:, 1] << 21) | faces[:, 2]
    uk, cnt = np.unique(fk, return_counts=True)
    uf = np.stack([uk >> 42, (uk >> 21) & 0x1FFFFF, uk & 0x1FFFFF], axis=1)
    edges = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    ek = np.unique((edges[:, 0] << 32) | edges[:, 1])
    ue = np.stack([ek >> 32, ek & 0xFFFFFFFF], axis=1)
    return uf, cnt, ue


def _box_labels(pts, faces, cnt):
    """Box facets (hull faces grouped by box face) and the 12 box edges."""
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    hull = faces[cnt == 1]
    tris, fids = [], []
    for f in hull:
        P = pts[f]
        fid = -1
        for k in range(3):
            if np.all(P[:, k] == lo[k]):
                fid = 2 * k
            elif np.all(P[:, k] == hi[k]):
                fid = 2 * k + 1
        if fid < 0:
            raise ValueError("hull face not on the box")
        tris.append(f)
        fids.append(fid)
    # box edges: corner pairs that differ in one coordinate
    segs, sids = [], []
    for c in range(8):
        for k in range(3):
            if not (c >> k) & 1:
                segs.append((c, c | (1 << k)))
                sids.append(len(sids))
    return tris, fids, segs, sids


def _angles_ok(P, cosmax):
    for j in range(3):
        u = P[(j + 1) % 3] - P[j]
        v = P[(j + 2) % 3] - P[j]
        c = np.dot(u, v) / np.sqrt(np.dot(u, u) * np.dot(v, v))
        if c > cosmax:
            return False
    return True


def _labels(tris, fids, segs, sids, nf):
    return dict(segs=np.asarray(segs, dtype=np.int32).reshape(-1, 2),
                seg_id=np.asarray(sids, dtype=np.int32),
                tris=np.asarray(tris, dtype=np.int32).reshape(-1, 3),
                facet_id=np.asarray(fids, dtype=np.int32),
                nfacets=nf)


def plc_from_delaunay(pts: np.ndarray, tets: np.ndarray, n_seg: int, n_tri: int, seed: int,
                      min_angle: float = 45.0) -> dict:
    """Constraint labels for a box PLC whose initial CDT is the Delaunay mesh
    ``tets`` of ``pts`` (8 box corners first)."""
    pts = np.asarray(pts, dtype=np.float64)
    if len(pts) >= (1 << 21):
        raise ValueError("too many points for the face packing")
    rng = np.random.default_rng(seed + 7919)
    faces, cnt, edges = _faces_edges(tets)
    tris, fids, segs, sids = _box_labels(pts, faces, cnt)
    used = np.zeros(len(pts), dtype=bool)
    used[:8] = True

    # free segments
    order = rng.permutation(len(edges))
    got = 0
    for i in order:
        if got >= n_seg:
            break
        a, b = edges[i]
        if used[a] or used[b]:
            continue
        used[a] = used[b] = True
        segs.append((int(a), int(b)))
        sids.append(len(sids))
        got += 1
    if got < n_seg:
        raise ValueError("not enough free edges")
    # triangles (inner faces only)
    inner = faces[cnt == 2]
    order = rng.permutation(len(inner))
    cosmax = np.cos(np.radians(min_angle))
    got = 0
    nf = 6
    for i in order:
        if got >= n_tri:
            break
        f = inner[i]
        if used[f].any():
            continue
        if not _angles_ok(pts[f], cosmax):
            continue
        used[f] = True
        tris.append(f)
        fids.append(nf)
        for j in range(3):
            segs.append((int(f[j]), int(f[(j + 1) % 3])))
            sids.append(len(sids))
        nf += 1
        got += 1
    if got < n_tri:
        raise ValueError("not enough well-shaped faces")
    return _labels(tris, fids, segs, sids, nf)


def _seg_dist(p0, p1, Q0, Q1):
    """Closest distance between segment p0p1 and each segment Q0[i]Q1[i]."""
    d1 = p1 - p0
    D2 = Q1 - Q0
    r = p0 - Q0
    a = np.dot(d1, d1)
    e = np.einsum("ij,ij->i", D2, D2)
    f = np.einsum("ij,ij->i", D2, r)
    c = r @ d1
    b = D2 @ d1
    den = a * e - b * b
    s = np.where(den > 1e-300, np.clip((b * f - c * e) / np.where(den > 1e-300, den, 1.0), 0, 1),
                 0.0)
    t = (b * s + f) / np.where(e > 0, e, 1.0)
    s = np.where(t < 0, np.clip(-c / a, 0, 1), np.where(t > 1, np.clip((b - c) / a, 0, 1), s))
    t = np.clip(t, 0, 1)
    diff = (p0 + s[:, None] * d1) - (Q0 + t[:, None] * D2)
    return np.sqrt(np.einsum("ij,ij->i", diff, diff))


def free_segments(pts: np.ndarray, n_seg: int, seed: int, knn: int = 16,
                  gap: float = 0.25) -> np.ndarray:
    """n_seg segments between input points (the recovered recipe above):
    the first end uniform among the non-corner points, the second among its
    knn nearest neighbours; rejected if it shares a point with, or passes
    within gap x the shorter length of, an earlier segment."""
    from scipy.spatial import cKDTree
    pts = np.asarray(pts, dtype=np.float64)
    rng = np.random.default_rng(seed + 104729)
    tree = cKDTree(pts)
    used = np.zeros(len(pts), dtype=bool)
    used[:8] = True
    A, Bq, L = [], [], []
    tries = 0
    while len(A) < n_seg:
        tries += 1
        if tries > 50 * n_seg + 1000:
            raise ValueError("not enough free segments")
        a = int(rng.integers(8, len(pts)))
        if used[a]:
            continue
        _, nb = tree.query(pts[a], k=knn + 1)
        b = int(nb[1 + rng.integers(0, knn)])
        if used[b] or b < 8:
            continue
        la = float(np.linalg.norm(pts[b] - pts[a]))
        if A:
            P0, P1 = pts[np.asarray(A)], pts[np.asarray(Bq)]
            d = _seg_dist(pts[a], pts[b], P0, P1)
            if np.any(d < gap * np.minimum(la, np.asarray(L))):
                continue
        used[a] = used[b] = True
        A.append(a)
        Bq.append(b)
        L.append(la)
    return np.stack([np.asarray(A, dtype=np.int32), np.asarray(Bq, dtype=np.int32)], axis=1)


def _dihedral_deg(P, Q, e0, e1):
    """Angle at edge (e0, e1) between the half-planes through P and Q."""
    u = e1 - e0
    u = u / np.linalg.norm(u)
    a = P - e0
    b = Q - e0
    a = a - np.dot(a, u) * u
    b = b - np.dot(b, u) * u
    c = np.dot(a, b) / np.sqrt(np.dot(a, a) * np.dot(b, b))
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def plc_with_chains(xyz: np.ndarray, tets: np.ndarray, chains, n_in: int, n_tri: int, seed: int,
                    min_angle: float = 45.0, pair_prob: float = 0.25,
                    min_dihedral: float = 70.0) -> dict:
    """Constraint labels for the recovered recipe: ``xyz`` holds the n_in input
    points (8 box corners first) followed by the recovery's midpoints, ``tets``
    is their Delaunay mesh and ``chains[s]`` the vertex ids along free segment
    s (each consecutive pair an edge of ``tets``). Adds the box facets and
    edges, one segment per chain (its subsegments), and n_tri triangles drawn
    among the faces (some in edge-sharing pairs, see the module notes)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    if len(xyz) >= (1 << 21):
        raise ValueError("too many points for the face packing")
    rng = np.random.default_rng(seed + 7919)
    faces, cnt, edges = _faces_edges(tets)
    tris, fids, segs, sids = _box_labels(xyz, faces, cnt)
    used = np.zeros(len(xyz), dtype=bool)
    used[:8] = True
    used[n_in:] = True  # recovery midpoints lie on their segments
    nseg = 12
    for ch in chains:
        for k in range(len(ch) - 1):
            segs.append((int(ch[k]), int(ch[k + 1])))
            sids.append(nseg)
        used[np.asarray(ch)] = True
        nseg += 1
    inner = faces[cnt == 2]
    # (edge, apex) of every inner face, sorted by edge key, for the pairs
    ek = np.concatenate([(inner[:, 0] << 21) | inner[:, 1], (inner[:, 0] << 21) | inner[:, 2],
                         (inner[:, 1] << 21) | inner[:, 2]])
    ap = np.concatenate([inner[:, 2], inner[:, 1], inner[:, 0]])
    srt = np.argsort(ek, kind="stable")
    ek, ap = ek[srt], ap[srt]

    def apexes(u, v):
        k = (min(u, v) << 21) | max(u, v)
        lo_, hi_ = np.searchsorted(ek, k, "left"), np.searchsorted(ek, k, "right")
        return sorted(int(x) for x in ap[lo_:hi_])

    order = rng.permutation(len(inner))
    cosmax = np.cos(np.radians(min_angle))
    got = 0
    nf = 6
    for i in order:
        if got >= n_tri:
            break
        f = [int(v) for v in inner[i]]
        if used[f].any() or not _angles_ok(xyz[f], cosmax):
            continue
        used[f] = True
        tris.append(f)
        fids.append(nf)
        nf += 1
        got += 1
        for j in range(3):
            segs.append((f[j], f[(j + 1) % 3]))
            sids.append(nseg)
            nseg += 1
        if got >= n_tri or rng.random() >= pair_prob:
            continue
        # a second triangle on one of the edges, a facet of its own: its other
        # two edges are new segments, the shared edge stays one segment
        j0 = int(rng.integers(0, 3))
        for dj in range(3):
            e0, e1 = f[(j0 + dj) % 3], f[(j0 + dj + 1) % 3]
            opp = f[(j0 + dj + 2) % 3]
            g = None
            for v in apexes(e0, e1):
                if v == opp or used[v]:
                    continue
                if (_angles_ok(xyz[[e0, e1, v]], cosmax) and
                        _dihedral_deg(xyz[opp], xyz[v], xyz[e0], xyz[e1]) >= min_dihedral):
                    g = [e0, e1, v]
                    break
            if g is None:
                continue
            used[g[2]] = True
            tris.append(g)
            fids.append(nf)
            nf += 1
            got += 1
            for p_, q_ in ((e1, g[2]), (g[2], e0)):
                segs.append((p_, q_))
                sids.append(nseg)
                nseg += 1
            break
    if got < n_tri:
        raise ValueError("not enough well-shaped faces")
    return _labels(tris, fids, segs, sids, nf)


def free_triangles(pts: np.ndarray, segs: np.ndarray, n_tri: int, seed: int, knn: int = 8,
                   min_angle: float = 30.0, gap: float = 0.25, pair_prob: float = 0.25,
                   min_dihedral: float = 70.0) -> dict:
    """n_tri triangles between input points for the facet-recovered recipe:
    a seed point uniform among the unused non-corner points and two of its knn
    nearest neighbours, every angle >= min_angle. A triangle is kept when its
    ball (centred at its centroid, through its farthest corner), grown by the
    factor 1 + gap, meets no grown ball of an earlier constraint (the given
    segments, centred at their midpoints, and earlier triangles), so that no
    two constraints meet. With probability pair_prob, a kept triangle gets a
    partner on one of its edges (a facet of its own, sharing that segment):
    the apex among the knn nearest unused points of the edge's midpoint, with
    every angle >= min_angle, a dihedral angle of at least min_dihedral with
    the first, and a ball that meets no other constraint's.
    Returns dict(segs=(m, 2) the given segments followed by every triangle
    edge once, tris=(t, 3), tri_segs=(t, 3) the segment of each triangle's
    edges (a, b), (b, c), (c, a))."""
    from scipy.spatial import cKDTree
    pts = np.asarray(pts, dtype=np.float64)
    segs = np.asarray(segs, dtype=np.int64).reshape(-1, 2)
    rng = np.random.default_rng(seed + 15485863)
    tree = cKDTree(pts)
    used = np.zeros(len(pts), dtype=bool)
    used[:8] = True
    used[segs.ravel()] = True
    centres = [0.5 * (pts[a] + pts[b]) for a, b in segs]
    radii = [0.5 * float(np.linalg.norm(pts[b] - pts[a])) for a, b in segs]
    cosmax = np.cos(np.radians(min_angle))
    out_segs = [tuple(int(v) for v in e) for e in segs]
    tris, tri_segs = [], []

    def ball(P):
        c = P.mean(axis=0)
        return c, float(np.max(np.linalg.norm(P - c, axis=1)))

    def clear(c, r, skip=()):
        for k, (c2, r2) in enumerate(zip(centres, radii)):
            if k in skip:
                continue
            if np.linalg.norm(c - c2) <= (1.0 + gap) * (r + r2):
                return False
        return True

    def add(t, edge_ids):
        tris.append(tuple(int(v) for v in t))
        tri_segs.append(tuple(edge_ids))
        c, r = ball(pts[list(t)])
        centres.append(c)
        radii.append(r)
        used[list(t)] = True

    tries = 0
    while len(tris) < n_tri:
        tries += 1
        if tries > 200 * n_tri + 1000:
            raise ValueError("not enough room for %d triangles" % n_tri)
        a = int(rng.integers(8, len(pts)))
        if used[a]:
            continue
        _, nb = tree.query(pts[a], k=knn + 1)
        pick = rng.choice(knn, size=2, replace=False) + 1
        b, c = int(nb[pick[0]]), int(nb[pick[1]])
        if used[b] or used[c] or b < 8 or c < 8:
            continue
        P = pts[[a, b, c]]
        if not _angles_ok(P, cosmax):
            continue
        cb, rb = ball(P)
        if not clear(cb, rb):
            continue
        e0 = len(out_segs)
        out_segs += [(a, b), (b, c), (c, a)]
        add((a, b, c), (e0, e0 + 1, e0 + 2))
        me = len(centres) - 1
        if len(tris) >= n_tri or rng.random() >= pair_prob:
            continue
        j0 = int(rng.integers(0, 3))
        f = (a, b, c)
        for dj in range(3):
            j = (j0 + dj) % 3
            u, v, opp = f[j], f[(j + 1) % 3], f[(j + 2) % 3]
            _, nb2 = tree.query(0.5 * (pts[u] + pts[v]), k=knn)
            g = None
            for x in (int(y) for y in nb2):
                if used[x] or x < 8:
                    continue
                Q = pts[[u, v, x]]
                if not _angles_ok(Q, cosmax):
                    continue
                if _dihedral_deg(pts[opp], pts[x], pts[u], pts[v]) < min_dihedral:
                    continue
                cq, rq = ball(Q)
                if not clear(cq, rq, skip=(me,)):
                    continue
                g = x
                break
            if g is None:
                continue
            e1 = len(out_segs)
            out_segs += [(v, g), (g, u)]
            add((u, v, g), (e0 + j, e1, e1 + 1))
            break
    return dict(segs=np.asarray(out_segs, dtype=np.int32).reshape(-1, 2),
                tris=np.asarray(tris, dtype=np.int32).reshape(-1, 3),
                tri_segs=np.asarray(tri_segs, dtype=np.int32).reshape(-1, 3))


def plc_recovered(xyz: np.ndarray, tets: np.ndarray, chains, subfaces) -> dict:
    """Labels of a mesh whose segments and triangle facets were recovered:
    box facets and edges, then one segment per chain (its subsegments) and one
    facet per recovered triangle (its subfaces, facet ids from 6 on)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    if len(xyz) >= (1 << 21):
        raise ValueError("too many points for the face packing")
    faces, cnt, _ = _faces_edges(tets)
    tris, fids, segs, sids = _box_labels(xyz, faces, cnt)
    nseg = 12
    for ch in chains:
        for k in range(len(ch) - 1):
            segs.append((int(ch[k]), int(ch[k + 1])))
            sids.append(nseg)
        nseg += 1
    nf = 6
    for T in subfaces:
        for t in T:
            tris.append(tuple(int(v) for v in t))
            fids.append(nf)
        nf += 1
    return _labels(tris, fids, segs, sids, nf)


def rectangles(pts: np.ndarray, count: int, seed: int, tries: int = 50) -> np.ndarray:
    """count rectangles for a Table-1-like PLC (the paper's polygons are
    "mainly rectangles"): near random input points, parallel to a random pair
    of axes, with sides of 0.3 to 0.6 times the distance from the point to its
    nearest neighbour. A rectangle is kept when no point (input or corner of an
    earlier rectangle) lies within 1.05 times its circumradius of its centre,
    and none of its corners lies that close to an earlier rectangle's centre,
    so that its four corners, which lie on one circle, span faces of the
    Delaunay mesh. Returns the corners, (count, 4, 3), in order around the
    rectangle."""
    from scipy.spatial import cKDTree
    pts = np.asarray(pts, dtype=np.float64)
    rng = np.random.default_rng(seed + 65537)
    tree = cKDTree(pts)
    dnn, _ = tree.query(pts, k=2)
    out, centres, radii = [], [], []
    old_corners = old_centres = None  # trees of the rectangles before `recent`
    recent = 0  # rectangles accepted since the trees were built
    rmax = 0.0
    attempts = 0
    while len(out) < count:
        attempts += 1
        if attempts > tries * count + 1000:
            raise ValueError("not enough room for %d rectangles" % count)
        i = int(rng.integers(8, len(pts)))
        s0 = dnn[i, 1]
        a_, b_ = rng.uniform(0.3, 0.6, size=2) * s0
        c = pts[i] + 0.5 * s0 * rng.normal(size=3) / np.sqrt(3.0)
        # axis-parallel, so that the corners share coordinates exactly: they are
        # exactly coplanar and exactly on one circle
        k = int(rng.integers(0, 3))
        k1, k2 = (k + 1) % 3, (k + 2) % 3
        q = np.empty((4, 3))
        q[:, k] = c[k]
        q[:, k1] = [c[k1] - a_ / 2, c[k1] + a_ / 2, c[k1] + a_ / 2, c[k1] - a_ / 2]
        q[:, k2] = [c[k2] - b_ / 2, c[k2] - b_ / 2, c[k2] + b_ / 2, c[k2] + b_ / 2]
        if np.any(q <= 0.0) or np.any(q >= 1000.0):
            continue
        c = q.mean(axis=0)
        R = 0.5 * np.linalg.norm(q[2] - q[0])
        if tree.query_ball_point(c, 1.05 * R):
            continue
        n_old = len(out) - recent
        if old_corners is not None and old_corners.query_ball_point(c, 1.05 * R):
            continue
        if recent and np.any(np.linalg.norm(np.concatenate(out[n_old:]) - c, axis=1) < 1.05 * R):
            continue
        # no corner inside an earlier rectangle's sphere
        bad = False
        if old_centres is not None:
            for j in set(sum(old_centres.query_ball_point(q, 1.05 * rmax), [])):
                if np.any(np.linalg.norm(q - centres[j], axis=1) < 1.05 * radii[j]):
                    bad = True
                    break
        for j in range(n_old, len(out)):
            if bad:
                break
            bad = np.any(np.linalg.norm(q - centres[j], axis=1) < 1.05 * radii[j])
        if bad:
            continue
        out.append(q)
        centres.append(c)
        radii.append(R)
        rmax = max(rmax, R)
        recent += 1
        if recent == 256:
            old_corners = cKDTree(np.concatenate(out))
            old_centres = cKDTree(np.asarray(centres))
            recent = 0
    return np.asarray(out)


def plc_rectangles(xyz: np.ndarray, tets: np.ndarray, n_in: int, n_rect: int) -> dict:
    """Labels for the box PLC plus rectangles whose corners are xyz[n_in:]
    (four per rectangle, in order): each rectangle is a facet made of the two
    faces of ``tets`` on its corners (whichever diagonal the Delaunay mesh of
    the cocircular corners has; the diagonal is not a segment), and its four
    sides are segments."""
    xyz = np.asarray(xyz, dtype=np.float64)
    faces, cnt, edges = _faces_edges(tets)
    tris, fids, segs, sids = _box_labels(xyz, faces, cnt)
    inner = faces[cnt == 2]
    key = (inner[:, 0] << 42) | (inner[:, 1] << 21) | inner[:, 2]
    srt = np.sort(key)
    nf = 6
    for r in range(n_rect):
        c = [n_in + 4 * r + k for k in range(4)]
        found = []
        for tri in ((c[0], c[1], c[2]), (c[0], c[2], c[3]), (c[0], c[1], c[3]), (c[1], c[2], c[3])):
            t = sorted(tri)
            k = (t[0] << 42) | (t[1] << 21) | t[2]
            j = np.searchsorted(srt, k)
            if j < len(srt) and srt[j] == k:
                found.append(t)
        if len(found) != 2:
            raise ValueError("rectangle %d is not two faces of the mesh" % r)
        for t in found:
            tris.append(t)
            fids.append(nf)
        for k in range(4):
            segs.append((c[k], c[(k + 1) % 4]))
            sids.append(len(sids))
        nf += 1
    return _labels(tris, fids, segs, sids, nf)

