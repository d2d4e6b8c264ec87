"""Segment and facet recovery on the GPU against the oracle's (needs a GPU).

The GPU recovery (Delaunay meshes built by the library's point-insertion
rounds, midpoints, circumcentres and predicate signs from its device
formulas) must give the oracle's recovery bit for bit on small inputs: the
same points in the same order, the same chains, facet points and subfaces,
and the same tetrahedra. PLCs built on recovered meshes (segments only, and
segments with triangle facets) are then refined in lockstep with the oracle's
mode R, round by round, to the end; so is a PLC of the Table-1-like recipe (a
ball of points with rectangles).
"""
import numpy as np
import pytest

from _meshes import assert_same_mesh, compare_reports

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


def _canon_tets(t):
    t = np.sort(np.asarray(t), axis=1)
    return t[np.lexsort(t.T[::-1])]


@pytest.mark.parametrize("kind,n,ns,seed", [("uniform", 3000, 60, 3), ("clustered", 4000, 80, 4),
                                            ("uniform", 20000, 300, 8)])
def test_gpu_recovery_equals_oracle(cdr, kind, n, ns, seed):
    from oracle.recover import recover_segments as oracle_recover
    from paper_1903_03406_gb300 import inputs, recover
    pts, _, _ = inputs.box_points(kind, n, seed)
    segs = inputs.free_segments(pts, ns, seed)
    xyz, tets, chains, passes = recover.recover_segments(pts, segs, cdr)
    om, oxyz, ochains, opasses = oracle_recover(pts, segs)
    assert passes == opasses and passes >= 1
    assert np.array_equal(xyz, oxyz)
    assert chains == ochains
    assert np.array_equal(_canon_tets(tets), _canon_tets(om.export()["tets"]))


def test_rounds_lockstep_on_recovered_segments(cdr):
    """Free segments recovered by midpoints and triangles sharing segments:
    every round of the GPU equals mode R's, to the end."""
    from _meshes import oracle_case
    om, e, plc = oracle_case("uniform", 900, 10, 10, 5, recovered=True)
    h = cdr.Handle.create(e["xyz"], e["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"])
    classes = []
    for r in range(3000):
        g = h.round(1.4)
        o = om.round(1.4)
        assert g["cls"] == o["cls"], r
        if g["cls"] < 0:
            break
        classes.append(g["cls"])
        compare_reports(h.round_report(), om.report(), "recovered round %d" % r)
        assert g["steiner_inserted"] == o["inserted"]
        assert_same_mesh(h.export(), om.export(), "recovered round %d" % r)
    assert set(classes) == {0, 1, 2}
    h.close()


def test_rounds_lockstep_ball_with_rectangles(cdr):
    """The Table-1-like recipe (points in a ball, axis-parallel rectangles whose
    corners lie on one circle): the initial Delaunay mesh built on the GPU is a
    valid Delaunay mesh of the same points (four cocircular, coplanar corners
    have two Delaunay triangulations, so it need not be the oracle's), and from
    the oracle's mesh every round equals mode R's, to the end."""
    import oracle
    from paper_1903_03406_gb300 import inputs
    pts, _, _ = inputs.box_points("ball", 1500, 6)
    rect = inputs.rectangles(pts, 50, 6)
    xyz = np.concatenate([pts, rect.reshape(-1, 3)])
    om = oracle.Mesh.box_delaunay(xyz)
    e = om.export()
    dt = cdr.Handle.delaunay_box(xyz)
    ge = dt.export()
    dt.close()
    assert dt.skipped == 0 and np.array_equal(ge["xyz"], xyz)
    c = oracle.Mesh.create(ge["xyz"], ge["tets"]).check(1.6)
    assert c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0 and c["euler"] == 1
    assert abs(c["vol_rel_err"]) < 1e-12
    plc = inputs.plc_rectangles(e["xyz"], e["tets"], len(pts), len(rect))
    assert om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                              plc["nfacets"]) == 0
    h = cdr.Handle.create(e["xyz"], e["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"])
    classes = []
    for r in range(3000):
        g = h.round(1.6)
        o = om.round(1.6)
        assert g["cls"] == o["cls"], r
        if g["cls"] < 0:
            break
        classes.append(g["cls"])
        compare_reports(h.round_report(), om.report(), "rectangles round %d" % r)
        assert g["steiner_inserted"] == o["inserted"]
        assert_same_mesh(h.export(), om.export(), "rectangles round %d" % r)
    assert set(classes) == {0, 1, 2}
    h.close()


def _free_plc_case(n, ns, nt, seed, knn):
    from paper_1903_03406_gb300 import inputs
    pts, _, _ = inputs.box_points("uniform", n, seed)
    segs = inputs.free_segments(pts, ns, seed)
    return pts, inputs.free_triangles(pts, segs, nt, seed, knn=knn)


def test_gpu_facet_recovery_equals_oracle(cdr):
    """Triangles that are not unions of Delaunay faces: the GPU recovery (device
    predicates in batches, device Delaunay meshes) makes the oracle's points,
    chains, facet points and subfaces, bit for bit, and the same mesh."""
    from oracle.recover import recover_plc as oracle_recover
    from paper_1903_03406_gb300 import recover
    pts, plc = _free_plc_case(2000, 6, 6, 5, 150)
    g = recover.recover_plc(pts, plc["segs"], plc["tris"], plc["tri_segs"], cdr)
    o = oracle_recover(pts, plc["segs"], plc["tris"], plc["tri_segs"])
    assert g["passes"] == o["passes"] and sum(map(len, o["facet_points"])) > 0
    assert np.array_equal(g["xyz"], o["xyz"])
    assert g["chains"] == o["chains"] and g["facet_points"] == o["facet_points"]
    assert [list(map(tuple, s)) for s in g["subfaces"]] == o["subfaces"]
    assert np.array_equal(g["facetq"], o["facetq"])
    assert np.array_equal(_canon_tets(g["tets"]), _canon_tets(o["mesh"].export()["tets"]))


def test_rounds_lockstep_on_recovered_facets(cdr):
    """A PLC with recovered segments and facets, each side labelled from its
    own recovery: every GPU round equals mode R's, to the end."""
    from oracle.recover import facet_reference, recover_plc as oracle_recover, reference_shift
    from paper_1903_03406_gb300 import inputs, recover
    pts, plc = _free_plc_case(900, 4, 5, 11, 80)
    o = oracle_recover(pts, plc["segs"], plc["tris"], plc["tri_segs"])
    om = o["mesh"]
    e = om.export()
    olab = inputs.plc_recovered(o["xyz"], e["tets"], o["chains"], o["subfaces"])
    first = {}
    for t, f in zip(olab["tris"], olab["facet_id"]):
        first.setdefault(int(f), t)
    oq = np.zeros((olab["nfacets"], 3))
    s = reference_shift(o["xyz"])
    for f in range(6):
        oq[f] = facet_reference(o["xyz"], int(first[f][0]), int(first[f][1]), int(first[f][2]), s)
    oq[6:] = o["facetq"]
    assert om.set_constraints(olab["segs"], olab["seg_id"], olab["tris"], olab["facet_id"],
                              olab["nfacets"], facetq=oq) == 0
    g = recover.recover_plc(pts, plc["segs"], plc["tris"], plc["tri_segs"], cdr)
    glab = inputs.plc_recovered(g["xyz"], g["tets"], g["chains"], g["subfaces"])
    gq = np.concatenate([recover.box_facet_refs(g["xyz"], glab), g["facetq"]])
    h = cdr.Handle.create(g["xyz"], g["tets"], glab["segs"], glab["seg_id"], glab["tris"],
                          glab["facet_id"], glab["nfacets"], facet_ref=gq)
    classes = []
    for r in range(3000):
        gr = h.round(1.5)
        orr = om.round(1.5)
        assert gr["cls"] == orr["cls"], r
        if gr["cls"] < 0:
            break
        classes.append(gr["cls"])
        compare_reports(h.round_report(), om.report(), "facets round %d" % r)
        assert gr["steiner_inserted"] == orr["inserted"]
        assert_same_mesh(h.export(), om.export(), "facets round %d" % r)
    assert 2 in classes
    h.close()
