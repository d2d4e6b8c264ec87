"""Pins for the mesh-quality report (paper_1903_03406_gb300/quality.py) and the
quality comparison of parallel rounds with sequential refinement.

Sec. 3 judges outputs by their size, their bad tetrahedra and the
distribution of their dihedral angles (Fig. 2), and finds the GPU's
distribution like the sequential program's. Here the oracle's round-emulating
refinement (mode R, which the GPU path equals bit for bit) is compared with its
sequential refinement (mode S) on the same input.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1903_03406_gb300 import inputs, quality


def test_right_corner_tetrahedron_closed_forms():
    # three faces on the coordinate planes meet at right angles along the axes;
    # the slanted face x+y+z=1 meets each of them at arccos(1/sqrt(3))
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    ang = quality.dihedral_angles(xyz, [[0, 1, 2, 3]])[0]
    slant = math.degrees(math.acos(1 / math.sqrt(3)))
    assert np.allclose(ang, [90, 90, 90, slant, slant, slant], atol=1e-12)
    # circumcentre (1/2, 1/2, 1/2): R = sqrt(3)/2, shortest edge 1
    assert quality.radius_edge(xyz, [[0, 1, 2, 3]])[0] == pytest.approx(math.sqrt(3) / 2,
                                                                       rel=1e-14)


def test_regular_tetrahedron_closed_forms():
    xyz = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    ang = quality.dihedral_angles(xyz, [[0, 1, 2, 3]])[0]
    assert np.allclose(ang, math.degrees(math.acos(1 / 3)), atol=1e-12)
    # R = a sqrt(6) / 4 for edge a
    assert quality.radius_edge(xyz, [[0, 1, 2, 3]])[0] == pytest.approx(math.sqrt(6) / 4,
                                                                       rel=1e-14)


def _solid_angle(a, b, c, d):
    """Solid angle at a subtended by triangle bcd (Van Oosterom and Strackee, 1983)."""
    u, v, w = b - a, c - a, d - a
    lu, lv, lw = (np.linalg.norm(x) for x in (u, v, w))
    num = abs(np.dot(u, np.cross(v, w)))
    den = lu * lv * lw + np.dot(u, v) * lw + np.dot(u, w) * lv + np.dot(v, w) * lu
    om = 2 * math.atan2(num, den)
    return om if om >= 0 else om + 2 * math.pi


def test_gram_euler_relation_on_random_tetrahedra():
    # for every tetrahedron: sum of vertex solid angles = 2 sum of dihedral angles - 4 pi
    rng = np.random.default_rng(11)
    P = rng.normal(size=(200, 4, 3))
    xyz = P.reshape(-1, 3)
    tets = np.arange(800).reshape(200, 4)
    ang = np.radians(quality.dihedral_angles(xyz, tets))
    for t in range(200):
        p = P[t]
        omega = sum(_solid_angle(p[i], *[p[j] for j in range(4) if j != i]) for i in range(4))
        assert omega == pytest.approx(2 * ang[t].sum() - 4 * math.pi, abs=1e-9)


def test_angles_follow_the_vertices_under_relabelling():
    rng = np.random.default_rng(12)
    xyz = rng.uniform(size=(4, 3))
    base = quality.dihedral_angles(xyz, [[0, 1, 2, 3]])[0]
    at = {frozenset(e): base[k] for k, e in enumerate(quality.EDGES)}
    for perm in ([1, 0, 2, 3], [3, 2, 1, 0], [2, 3, 0, 1], [0, 2, 3, 1]):
        ang = quality.dihedral_angles(xyz, [perm])[0]
        for k, (i, j) in enumerate(quality.EDGES):
            assert ang[k] == pytest.approx(at[frozenset((perm[i], perm[j]))], abs=1e-12)


def test_radius_edge_matches_the_oracles_circumcentre():
    rng = np.random.default_rng(13)
    P = rng.uniform(size=(50, 4, 3))
    rho = quality.radius_edge(P.reshape(-1, 3), np.arange(200).reshape(50, 4))
    for t in range(50):
        a, b, c, d = P[t]
        cc, ok = oracle.tet_circumcenter(a, b, c, d)
        assert ok
        lmin = min(np.linalg.norm(P[t, i] - P[t, j]) for i, j in quality.EDGES)
        assert rho[t] == pytest.approx(np.linalg.norm(cc - a) / lmin, rel=1e-9)


def test_report_histogram_is_a_distribution():
    rng = np.random.default_rng(14)
    P = rng.uniform(size=(30, 4, 3))
    r = quality.report(P.reshape(-1, 3), np.arange(120).reshape(30, 4), B=2.0)
    assert r["tets"] == 30 and len(r["dihedral_hist"]) == 18
    assert sum(r["dihedral_hist"]) == pytest.approx(1.0)
    assert 0 < r["dihedral_min_deg"] <= r["dihedral_max_deg"] < 180
    assert quality.hist_distance(r["dihedral_hist"], r["dihedral_hist"]) == 0.0


def test_rounds_and_sequential_refinement_give_the_same_quality():
    n, ns, B, seed = 600, 6, 1.5, 7
    pts, _, _ = inputs.box_points("uniform", n, seed)
    mS = oracle.Mesh.box_delaunay(pts)
    e = mS.export()
    plc = inputs.plc_from_delaunay(pts, e["tets"], ns, ns, seed)
    lab = (plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    mS.set_constraints(*lab)
    mR = oracle.Mesh.create(e["xyz"], e["tets"])
    mR.set_constraints(*lab)
    q0 = quality.report(e["xyz"], e["tets"], B)
    mS.refine_S(B)
    mR.refine_R(B)
    eS, eR = mS.export(), mR.export()
    qS = quality.report(eS["xyz"], eS["tets"], B)
    qR = quality.report(eR["xyz"], eR["tets"], B)
    # the report's bad fraction counts what the oracle's exact check leaves as
    # unsplittable (nothing else is above B after refinement)
    for m, q in ((mS, qS), (mR, qR)):
        c = m.check(B)
        assert c["bad_tets"] == 0
        assert round(q["frac_above_B"] * q["tets"]) == c["bad_tets_unspl"]
        assert q["frac_above_B"] < 0.01
    # refinement reshapes the angle distribution; the two orders end alike
    d_orders = quality.hist_distance(qS["dihedral_hist"], qR["dihedral_hist"])
    d_refined = quality.hist_distance(q0["dihedral_hist"], qS["dihedral_hist"])
    assert d_orders < 0.02
    assert d_refined > 5 * d_orders


def test_radius_edge_histogram():
    # the regular tetrahedron has the smallest ratio, sqrt(6)/4 = 0.612: first bin;
    # a flat-ish one with a huge ratio lands in the last, open-ended bin
    xyz = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1],
                    [0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, 1e-3]], dtype=float)
    r = quality.report(xyz, [[0, 1, 2, 3], [4, 5, 6, 7]], B=2.0)
    h = r["radius_edge_hist"]
    assert len(h) == len(r["radius_edge_bins"]) - 1
    assert h[0] == 0.5 and h[-1] == 0.5 and sum(h) == 1.0
    assert r["frac_above_B"] == 0.5
