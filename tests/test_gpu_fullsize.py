"""Full-size refinements in the benchmark's launch configuration (needs a GPU).

uniform100k (the benchmark workload: 100,000 points, 1,000 segments, 1,000
triangles, B = 1.4) and clustered500k (500,000 clustered points, 5,000 segments,
5,000 triangles, B = 1.4) are refined by the library with the tuned launch
setting, as bench.py runs them. The oracle cannot refine meshes this large
within a test, so:
* its exact predicates check sampled outputs one by one: orientation, local
  Delaunay across interior faces, no encroached subsegment or subface, and the
  quality of the tetrahedra not given up;
* properties that hold at any size are checked on the whole mesh: the summed
  volume equals the box's, the Euler characteristic is 1, every input segment
  is a chain of subsegments, and every subface bounds one or two tetrahedra;
* the splitting points of full-size rounds are bit-identical to the oracle's
  formulas, candidate by candidate;
* the final Steiner count and fraction of bad tetrahedra left stay within
  1.15x of the oracle's sequential refinement of the same input run to the end
  (its counts stored in tests/golden/oracle_counts.json by
  tests/golden/make_oracle_counts.py, which calls only the oracle).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1903_03406_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    name: dict(kind=w["kind"], n=w["n"], seed=w["seed"], B=w["B"], ns=w["n_seg"], nt=w["n_tri"],
               recipe=w["recipe"])
    for name, w in inputs.CONFIGS.items() if name in ("uniform100k", "clustered500k")
}
NSAMPLE = 2000


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


def _workload(cdr, w):
    """The benchmark's initial mesh, built on the GPU as bench.py builds it."""
    pts, lo, hi = inputs.box_points(w["kind"], w["n"], w["seed"])
    if w["recipe"] == "recovered":
        from paper_1903_03406_gb300 import recover
        segs = inputs.free_segments(pts, w["ns"], w["seed"])
        xyz, tets, chains, _ = recover.recover_segments(pts, segs, cdr)
        plc = inputs.plc_with_chains(xyz, tets, chains, len(pts), w["nt"], w["seed"])
        return {"xyz": xyz, "tets": tets}, plc, lo, hi
    dt = cdr.Handle.delaunay_box(pts)
    ex = dt.export()
    dt.close()
    plc = inputs.plc_from_delaunay(pts, ex["tets"], w["ns"], w["nt"], w["seed"])
    return ex, plc, lo, hi


# round kind per workload: the benchmark's (subsegments and subfaces together)
# on the clustered one, one class per round on the uniform one
MIXED = {"clustered500k": 2, "uniform100k": 0}


def _handle(cdr, ex, plc, mixed=0):
    from paper_1903_03406_gb300 import autotune
    h = cdr.Handle.create(ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"], mixed_rounds=mixed)
    autotune.apply(h, autotune.load(kind="plain"))
    return h


class Incidence:
    """Tetrahedra around each vertex (CSR), to find the tets holding an edge or face."""

    def __init__(self, tets):
        flat = tets.ravel()
        order = np.argsort(flat, kind="stable")
        self.tet_of = (order // 4).astype(np.int64)
        self.start = np.searchsorted(flat[order], np.arange(flat.max() + 2))

    def around(self, v):
        return self.tet_of[self.start[v]:self.start[v + 1]]

    def holding(self, vs):
        s = set(self.around(vs[0]).tolist())
        for v in vs[1:]:
            s &= set(self.around(v).tolist())
        return sorted(s)


def _check(ex, plc, B, lo, hi, rng):
    xyz, T, tflag = ex["xyz"], ex["tets"], ex["tflag"]
    sf, ss = ex["sf"], ex["ss"]
    inc = Incidence(T)
    # orientation (sampled, exact)
    for t in rng.choice(len(T), size=min(NSAMPLE, len(T)), replace=False):
        assert oracle.orient3d(*xyz[T[t]]) > 0, t
    # volume: the tetrahedra fill the box exactly
    a, b, c, d = (xyz[T[:, k]] for k in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a)) / 6.0
    assert abs(math.fsum(vol) - (hi - lo) ** 3) <= 1e-12 * (hi - lo) ** 3
    # Euler characteristic V - E + F - T = 1 (a ball). Faces: every interior
    # face bounds two tetrahedra and the hull faces are the subfaces of the six
    # box facets (ids 0..5), so F = (4 T + hull) / 2.
    n = np.int64(len(xyz))
    ed = np.sort(T[:, [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]]].reshape(-1, 2), axis=1)
    E = len(np.unique(ed[:, 0].astype(np.int64) * n + ed[:, 1]))
    hull = int(np.count_nonzero(sf[:, 3] < 6))
    assert (4 * len(T) + hull) % 2 == 0
    F = (4 * len(T) + hull) // 2
    used = int(np.count_nonzero(np.bincount(T.ravel(), minlength=len(xyz))))
    assert used - E + F - len(T) == 1
    # local Delaunay across sampled interior non-subface faces (exact insphere)
    sfset = {tuple(x) for x in np.sort(sf[:, :3], axis=1)}
    checked = 0
    for t in rng.choice(len(T), size=min(NSAMPLE, len(T)), replace=False):
        f = int(rng.integers(0, 4))
        face = [int(T[t, k]) for k in range(4) if k != f]
        if tuple(sorted(face)) in sfset:
            continue
        other = [u for u in inc.holding(face) if u != t]
        if not other:
            continue  # hull face
        assert len(other) == 1
        apex = [v for v in T[other[0]] if v not in face][0]
        assert oracle.insphere(*xyz[T[t]], xyz[apex]) <= 0, (t, other[0])
        checked += 1
    assert checked > NSAMPLE // 2
    # subfaces: one or two tetrahedra each, neither apex strictly inside the
    # equatorial sphere (sampled)
    for s in rng.choice(len(sf), size=min(NSAMPLE, len(sf)), replace=False):
        tri = [int(v) for v in sf[s, :3]]
        holders = inc.holding(tri)
        assert 1 <= len(holders) <= 2
        if ex["sfflag"][s] & 2:
            continue  # given up (unsplittable): may stay encroached
        for u in holders:
            apex = [v for v in T[u] if v not in tri][0]
            assert oracle.equatorial(*xyz[tri], xyz[apex]) >= 0
    # subsegments: no vertex of the edge's ring strictly inside the diametral sphere
    for g in rng.choice(len(ss), size=min(NSAMPLE, len(ss)), replace=False):
        e = [int(ss[g, 0]), int(ss[g, 1])]
        ring = {int(v) for u in inc.holding(e) for v in T[u]} - set(e)
        assert ring
        if ex["ssflag"][g] & 2:
            continue  # given up (unsplittable): may stay encroached
        for v in ring:
            assert oracle.diametral(xyz[e[0]], xyz[e[1]], xyz[v]) >= 0
    # every input segment is a chain of subsegments between its endpoints (the
    # ends of the chain it had in the initial mesh)
    segs, sid = plc["segs"], plc["seg_id"]

    def chain_ends(parts):
        deg = {}
        for p, q in parts:
            deg[int(p)] = deg.get(int(p), 0) + 1
            deg[int(q)] = deg.get(int(q), 0) + 1
        assert all(c in (1, 2) for c in deg.values())
        return sorted(v for v, c in deg.items() if c == 1)

    for k in rng.choice(np.unique(sid), size=min(300, len(np.unique(sid))), replace=False):
        ends = chain_ends(ss[ss[:, 2] == k][:, :2])
        assert len(ends) == 2 and ends == chain_ends(segs[sid == k])
    # quality: the tetrahedra that were not given up are not bad (sampled)
    ok = np.nonzero((tflag & 2) == 0)[0]
    for t in rng.choice(ok, size=min(NSAMPLE, len(ok)), replace=False):
        assert not oracle.tet_bad(*xyz[np.sort(T[t])], B)


@pytest.mark.parametrize("name", sorted(CASES))
def test_full_size_refinement_properties(cdr, name):
    w = CASES[name]
    ex0, plc, lo, hi = _workload(cdr, w)
    h = _handle(cdr, ex0, plc, MIXED[name])
    st = h.refine(w["B"])
    assert st["status"] == 0 and st["steiner_inserted"] > w["n"]
    ex = h.export()
    h.close()
    # the quality band against the oracle's sequential refinement to the end
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.json")) as f:
        ref = json.load(f)[name]
    assert ref["contract_ok"] and ref["mesh_verts_in"] == len(ex0["xyz"])
    assert st["steiner_inserted"] <= 1.15 * ref["steiner"]
    assert st["n_bad_left"] / len(ex["tets"]) <= 1.15 * ref["bad_frac"]
    _check(ex, plc, w["B"], lo, hi, np.random.default_rng(7))


def test_full_size_splitting_points_match_oracle(cdr):
    """Rounds on the full benchmark mesh: sampled splitting points of a
    subsegment round and of a subface round are bit-identical to the oracle's
    formulas on the candidates' vertices."""
    w = CASES["uniform100k"]
    ex0, plc, _, _ = _workload(cdr, w)
    h = _handle(cdr, ex0, plc)
    seen = set()
    rng = np.random.default_rng(11)
    for _ in range(300):
        g = h.round(w["B"])
        if g["cls"] < 0 or g["cls"] in seen:
            if seen >= {0, 1}:
                break
            continue
        rep = h.round_report()
        xyz = h.export()["xyz"]
        keys, pts = rep["keys"], rep["pts"]
        ok = np.nonzero(rep["outcome"] != 2)[0]  # points that were computed
        for i in rng.choice(ok, size=min(500, len(ok)), replace=False):
            k = keys[i][keys[i] >= 0]
            if g["cls"] == 0:
                ref, good = oracle.midpoint(xyz[k[0]], xyz[k[1]]), True
            else:
                ref, good = oracle.tri_circumcenter(*xyz[k])
            assert good and np.array_equal(pts[i], ref), (g["cls"], i)
        seen.add(g["cls"])
    h.close()
    assert seen >= {0, 1}
