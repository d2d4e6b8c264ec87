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
"""
from __future__ import annotations

import numpy as np

CONFIGS = {
    "cube2k": dict(kind="cube", n=2000, seed=0, B=2.0, n_seg=0, n_tri=0),
    "uniform100k": dict(kind="uniform", n=100_000, seed=1, B=1.4, n_seg=1000, n_tri=1000),
    "clustered500k": dict(kind="clustered", n=500_000, seed=2, B=1.4, n_seg=5000, n_tri=5000),
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


def plc_from_delaunay(pts: np.ndarray, tets: np.ndarray, n_seg: int, n_tri: int, seed: int,
                      min_angle: float = 45.0) -> dict:
    """Constraint labels for a box PLC whose initial CDT is the Delaunay mesh
    ``tets`` of ``pts`` (8 box corners first)."""
    pts = np.asarray(pts, dtype=np.float64)
    if len(pts) >= (1 << 21):
        raise ValueError("too many points for the face packing")
    rng = np.random.default_rng(seed + 7919)
    lo, hi = pts.min(axis=0), pts.max(axis=0)
    faces, cnt, edges = _faces_edges(tets)

    # box facets: the hull faces, grouped by the box face they lie on
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
        P = pts[f]
        ok = True
        for j in range(3):
            u = P[(j + 1) % 3] - P[j]
            v = P[(j + 2) % 3] - P[j]
            c = np.dot(u, v) / np.sqrt(np.dot(u, u) * np.dot(v, v))
            if c > cosmax:
                ok = False
        if not ok:
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
    return dict(segs=np.asarray(segs, dtype=np.int32).reshape(-1, 2),
                seg_id=np.asarray(sids, dtype=np.int32),
                tris=np.asarray(tris, dtype=np.int32).reshape(-1, 3),
                facet_id=np.asarray(fids, dtype=np.int32),
                nfacets=nf)
