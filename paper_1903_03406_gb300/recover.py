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
