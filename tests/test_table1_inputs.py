"""The Table-1-like workload (paper Table 1: points of a ball distribution plus
polygons, mainly rectangles): its rectangles are exact, their two triangles
are faces of the Delaunay mesh, and the oracle refines the PLC to the
contract in both orders, within the quality band of each other."""
import numpy as np

import oracle
from paper_1903_03406_gb300 import inputs


def _case(n, n_rect, seed):
    pts, _, _ = inputs.box_points("ball", n, seed)
    rect = inputs.rectangles(pts, n_rect, seed)
    xyz = np.concatenate([pts, rect.reshape(-1, 3)])
    return pts, rect, xyz


def test_ball_points_and_exact_rectangles():
    pts, rect, xyz = _case(3000, 150, 3)
    r = np.linalg.norm(pts[8:] - 500.0, axis=1)
    assert r.max() <= 450.0 and len(pts) == 3008
    for q in rect:
        # one coordinate shared by all four corners, two values on each other axis
        shared = [k for k in range(3) if len(set(q[:, k])) == 1]
        assert len(shared) == 1
        for k in range(3):
            if k != shared[0]:
                assert len(set(q[:, k])) == 2
        c = q.mean(axis=0)
        R = np.linalg.norm(q - c, axis=1)
        assert np.allclose(R, R[0], rtol=1e-12)
        # no other point within its circumsphere (the generator keeps a 5%
        # margin, so a floating-point distance test decides)
        d = np.linalg.norm(xyz - c, axis=1)
        inside = np.nonzero(d < R[0] * 1.0001)[0]
        assert len(inside) == 4


def test_rectangles_are_mesh_faces_and_refine_to_the_contract():
    pts, rect, xyz = _case(1200, 40, 5)
    B = 1.6
    ins = []
    for mode in ("R", "S"):
        m = oracle.Mesh.box_delaunay(xyz)
        e = m.export()
        plc = inputs.plc_rectangles(e["xyz"], e["tets"], len(pts), len(rect))
        assert len(plc["tris"]) == 12 + 2 * len(rect) and plc["nfacets"] == 6 + len(rect)
        assert m.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                                 plc["nfacets"]) == 0
        st = m.refine_R(B) if mode == "R" else m.refine_S(B)
        c = m.check(B)
        for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
                  "seg_chain_bad", "enc_subsegs", "enc_subfaces", "bad_tets"):
            assert c[k] == 0, (mode, k)
        assert abs(c["vol_rel_err"]) < 1e-12 and c["euler"] == 1
        assert c["facet_area_rel_err"] < 1e-12
        ins.append(st["inserted"])
    assert ins[0] <= 1.15 * ins[1] and ins[1] <= 1.15 * ins[0]
