"""Shared helpers for the tests: seeded workloads, canonical mesh forms."""
import numpy as np

import oracle
from paper_1903_03406_gb300 import inputs

# reasons whose cavity is complete (reported by both implementations)
FULL_REASONS = {0, 9, 8, 12}


def oracle_case(kind, n, n_seg, n_tri, seed, recovered=False):
    """Oracle Delaunay mesh of a seeded point set with constraint labels; with
    recovered=True, free segments recovered by midpoints (inputs.py's
    recovered recipe)."""
    pts, _, _ = inputs.box_points(kind, n, seed)
    if recovered:
        from oracle.recover import recover_segments
        segs = inputs.free_segments(pts, n_seg, seed)
        om, xyz, chains, _ = recover_segments(pts, segs)
        e = om.export()
        plc = inputs.plc_with_chains(xyz, e["tets"], chains, len(pts), n_tri, seed)
        bad = om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                                 plc["nfacets"])
        assert bad == 0
        return om, e, plc
    om = oracle.Mesh.box_delaunay(pts)
    e = om.export()
    plc = inputs.plc_from_delaunay(pts, e["tets"], n_seg, n_tri, seed)
    bad = om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                             plc["nfacets"])
    assert bad == 0
    return om, e, plc


def oracle_from_export(ex, nfacets):
    """An oracle mesh holding an exported mesh (GPU or oracle), flags included."""
    om = oracle.Mesh.create(ex["xyz"], ex["tets"])
    sf, ss = ex["sf"], ex["ss"]
    bad = om.set_constraints(ss[:, :2], ss[:, 2], sf[:, :3], sf[:, 3], nfacets,
                             facetq=ex["facetq"])
    assert bad == 0
    om.set_flags(ex["tflag"], ex["sfflag"], ex["ssflag"])
    return om


def canon(ex):
    """Storage-independent form of an exported mesh."""
    t = np.sort(ex["tets"], axis=1)
    kt = np.lexsort(t.T[::-1])
    sf = np.concatenate([np.sort(ex["sf"][:, :3], axis=1), ex["sf"][:, 3:4]], axis=1)
    ks = np.lexsort(sf.T[::-1])
    ss = np.concatenate([np.sort(ex["ss"][:, :2], axis=1), ex["ss"][:, 2:3]], axis=1)
    kg = np.lexsort(ss.T[::-1])
    return dict(xyz=ex["xyz"], tets=t[kt], tflag=ex["tflag"][kt], sf=sf[ks],
                sfflag=ex["sfflag"][ks], ss=ss[kg], ssflag=ex["ssflag"][kg])


def assert_same_mesh(a, b, what=""):
    ca, cb = canon(a), canon(b)
    assert ca["xyz"].shape == cb["xyz"].shape, what
    assert np.array_equal(ca["xyz"], cb["xyz"]), what + ": vertex coordinates differ"
    for k in ("tets", "tflag", "sf", "sfflag", "ss", "ssflag"):
        assert ca[k].shape == cb[k].shape, "%s: %s sizes %s vs %s" % (what, k, ca[k].shape,
                                                                     cb[k].shape)
        assert np.array_equal(ca[k], cb[k]), "%s: %s differ" % (what, k)


def compare_reports(g, o, what=""):
    """Round reports of the GPU (g) and the oracle (o): candidate order, points,
    outcomes and, for complete cavities, the cavity sets."""
    assert np.array_equal(g["keys"], o["keys"]), what + ": candidate order"
    n = len(g["keys"])
    # splitting points: bit-exact (and so within 1e-12 relative)
    np.testing.assert_array_equal(g["pts"], o["pts"], err_msg=what + ": splitting points")
    assert np.array_equal(g["outcome"], o["outcome"]), what + ": outcomes"
    assert np.array_equal(g["reason"], o["reason"]), what + ": reasons"
    assert np.array_equal(g["surv"], o["surv"]), what + ": survivors"
    full = np.array([(o["outcome"][i] in (0, 1) and o["reason"][i] in FULL_REASONS) or
                     o["reason"][i] in (8, 12) for i in range(n)], dtype=bool)
    assert np.array_equal(g["ncav"][full], o["ncav"][full]), what + ": cavity sizes"
    assert np.array_equal(g["nbnd"][full], o["nbnd"][full]), what + ": boundary sizes"
    assert np.array_equal(g["nfcav"][full], o["nfcav"][full]), what + ": facet cavity sizes"
    ooff = np.concatenate([[0], np.cumsum(o["ncav"])])
    goff = np.concatenate([[0], np.cumsum(g["ncav"])])
    for i in np.nonzero(o["outcome"] == 0)[0]:
        oc = o["cav"][ooff[i]:ooff[i + 1]]
        gc = g["cav"][goff[i]:goff[i + 1]]
        gc = gc[np.lexsort(gc.T[::-1])]
        assert np.array_equal(oc, gc), what + ": cavity of candidate %d" % i
