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
