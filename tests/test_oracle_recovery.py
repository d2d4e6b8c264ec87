"""Pins for the oracle's recovery of free segments (the initial CDT of a PLC
whose segments are not all Delaunay edges) and for the recovered recipe's
labels, checked against brute force and closed forms rather than against the
oracle's own code:

* every subsegment of a recovered chain is an edge of the final mesh, found by
  brute force over its tetrahedra, and the final mesh is Delaunay (empty
  circumspheres by brute force on a small case);
* the chains are midpoint subdivisions: every inserted vertex is the exact
  rational midpoint of the two vertices it split, rounded to FP64, and the
  vertices come in increasing order along the segment;
* a segment that is not an edge of the points' Delaunay mesh is split; a
  segment whose closed diametral ball holds no other point (a Gabriel edge,
  hence an edge of every Delaunay mesh of these points) is not;
* the labelled mesh meets the CDT contract and refines (both orders) within
  the quality band; some interior facets share a segment.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.recover import recover_segments
from paper_1903_03406_gb300 import inputs


def _edge_set(tets):
    out = set()
    for t in np.asarray(tets):
        t = sorted(int(v) for v in t)
        for a in range(4):
            for b in range(a + 1, 4):
                out.add((t[a], t[b]))
    return out


def _case(kind, n, ns, seed):
    pts, _, _ = inputs.box_points(kind, n, seed)
    segs = inputs.free_segments(pts, ns, seed)
    m, xyz, chains, passes = recover_segments(pts, segs)
    return pts, segs, m, xyz, chains, passes


@pytest.mark.parametrize("kind,n,ns,seed", [("uniform", 3000, 60, 3), ("clustered", 3000, 60, 4)])
def test_recovered_chains_are_midpoint_subdivisions_and_mesh_edges(kind, n, ns, seed):
    pts, segs, m, xyz, chains, passes = _case(kind, n, ns, seed)
    assert passes >= 1 and len(xyz) > len(pts)
    assert np.array_equal(xyz[: len(pts)], pts)
    E = _edge_set(m.export()["tets"])
    split = 0
    for (a, b), ch in zip(segs, chains):
        assert ch[0] == a and ch[-1] == b and len(set(ch)) == len(ch)
        for u, v in zip(ch[:-1], ch[1:]):
            assert (min(u, v), max(u, v)) in E
        split += len(ch) > 2
        # rebuild the subdivision tree from the chain and check each midpoint
        # exactly (one FP64 rounding per coordinate of the exact midpoint of
        # the two vertices it split)
        stack = [(0, len(ch) - 1)]
        while stack:
            i, j = stack.pop()
            if j - i < 2:
                continue
            # the vertex made when (ch[i], ch[j]) was split: the one with the
            # smallest id between them
            mid = min(range(i + 1, j), key=lambda q: ch[q])
            assert ch[mid] >= len(pts)
            exact = [(Fraction(float(xyz[ch[i]][c])) + Fraction(float(xyz[ch[j]][c]))) / 2
                     for c in range(3)]
            assert all(float(exact[c]) == xyz[ch[mid]][c] for c in range(3))
            stack += [(i, mid), (mid, j)]
        # vertices in order along the segment
        d = np.asarray(xyz[b]) - np.asarray(xyz[a])
        t = [(np.asarray(xyz[v]) - np.asarray(xyz[a])) @ d / (d @ d) for v in ch]
        assert all(t1 < t2 for t1, t2 in zip(t[:-1], t[1:]))
    assert split > 0


def test_split_exactly_where_needed():
    """Segments not in the Delaunay mesh of the points are split; Gabriel
    segments (closed diametral ball empty) are not."""
    pts, segs, m, xyz, chains, passes = _case("uniform", 3000, 80, 7)
    E0 = _edge_set(oracle.Mesh.box_delaunay(pts).export()["tets"])
    gabriel = missing = 0
    for (a, b), ch in zip(segs, chains):
        a, b = int(a), int(b)
        if (min(a, b), max(a, b)) not in E0:
            assert len(ch) > 2
            missing += 1
        # Gabriel by brute force with the exact diametral sign (>= 0: not
        # strictly inside; ties count as inside here, so 0 is excluded too)
        near = np.nonzero(np.linalg.norm(pts - (pts[a] + pts[b]) / 2, axis=1) <=
                          0.51 * np.linalg.norm(pts[b] - pts[a]))[0]
        if all(oracle.diametral(pts[a], pts[b], pts[v]) > 0 for v in near if v not in (a, b)):
            assert len(ch) == 2
            gabriel += 1
    assert missing > 0 and gabriel > 0


def test_recovered_mesh_is_delaunay_by_brute_force():
    pts, segs, m, xyz, chains, passes = _case("uniform", 300, 12, 11)
    assert len(xyz) > len(pts)
    assert m.check_brute() == 0


def test_recovered_recipe_meets_the_contract_and_refines_within_the_band():
    B = 1.4
    pts, _, _ = inputs.box_points("uniform", 900, 5)
    segs = inputs.free_segments(pts, 10, 5)
    runs = []
    for mode in ("R", "S"):
        m, xyz, chains, _ = recover_segments(pts, segs)
        e = m.export()
        plc = inputs.plc_with_chains(xyz, e["tets"], chains, len(pts), 10, 5)
        assert m.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                                 plc["nfacets"]) == 0
        c = m.check(B)
        for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
                  "hull_not_subface", "seg_chain_bad"):
            assert c[k] == 0, k
        assert c["euler"] == 1 and abs(c["vol_rel_err"]) < 1e-12
        # some interior facets share a segment
        fid = plc["facet_id"]
        owners = {}
        for t, f in zip(plc["tris"], fid):
            if f < 6:
                continue
            for j in range(3):
                e_ = tuple(sorted((int(t[j]), int(t[(j + 1) % 3]))))
                owners.setdefault(e_, set()).add(int(f))
        assert any(len(v) >= 2 for v in owners.values())
        st = m.refine_R(B) if mode == "R" else m.refine_S(B)
        c = m.check(B)
        for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
                  "seg_chain_bad", "enc_subsegs", "enc_subfaces", "bad_tets"):
            assert c[k] == 0, (mode, k)
        assert abs(c["vol_rel_err"]) < 1e-12 and c["euler"] == 1
        runs.append(st["inserted"])
    assert runs[0] <= 1.15 * runs[1] and runs[1] <= 1.15 * runs[0]
