"""Pins for the oracle's recovery of triangle facets (the initial CDT of a PLC
whose polygons are not unions of faces of the points' Delaunay mesh, Sec. 1),
checked against brute force and closed forms rather than the oracle's own
code, and the product's pass logic driven with the oracle's primitives:

* every facet ends as a triangulated disk of mesh faces: each subface is a
  face of the mesh (brute force over its tetrahedra), each subsegment of the
  facet's three edges borders exactly one subface and every other subface
  edge exactly two, V - E + F = 1, and the subfaces' areas add up to the
  facet's area;
* every point made on a facet lies in the facet's plane and inside the
  triangle, and the final mesh is Delaunay (empty circumspheres, brute force);
* a facet that is already a union of Delaunay faces gets no point; a large
  one gets points;
* the labelled mesh meets the CDT contract and refines to the end;
* the product's recovery (paper_1903_03406_gb300.recover.recover_plc), given
  the oracle's predicates and Delaunay meshes in place of the device calls,
  makes the same points, chains and subfaces: the two share only the pass
  order, and on the GPU the device primitives are compared with the oracle's
  elsewhere.
"""
import numpy as np
import pytest

import oracle
from oracle.recover import facet_reference, recover_plc, reference_shift
from paper_1903_03406_gb300 import inputs


def _case(n, ns, nt, seed, knn):
    pts, _, _ = inputs.box_points("uniform", n, seed)
    segs = inputs.free_segments(pts, ns, seed)
    plc = inputs.free_triangles(pts, segs, nt, seed, knn=knn)
    return pts, plc, recover_plc(pts, plc["segs"], plc["tris"], plc["tri_segs"])


@pytest.fixture(scope="module")
def big():
    return _case(2000, 6, 6, 5, 150)


def _face_set(tets):
    out = set()
    for t in np.asarray(tets):
        t = sorted(int(v) for v in t)
        for k in range(4):
            out.add(tuple(t[:k] + t[k + 1:]))
    return out


def _area(P):
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def test_facets_end_as_disks_of_mesh_faces(big):
    pts, plc, r = big
    X = r["xyz"]
    F = _face_set(r["mesh"].export()["tets"])
    made = 0
    for f, (tri, fs) in enumerate(zip(plc["tris"], plc["tri_segs"])):
        T = r["subfaces"][f]
        assert T and all(t in F for t in T)
        chains = [r["chains"][s] for s in fs]
        # the chains close the facet's boundary: (a, b), (b, c), (c, a)
        a, b, c = (int(v) for v in tri)
        ends = [(ch[0], ch[-1]) for ch in chains]
        assert [tuple(sorted(e)) for e in ends] == [tuple(sorted(e)) for e in
                                                    ((a, b), (b, c), (c, a))]
        bnd = {tuple(sorted((u, v))) for ch in chains for u, v in zip(ch[:-1], ch[1:])}
        count = {}
        for t in T:
            for e in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2])):
                count[e] = count.get(e, 0) + 1
        for e, k in count.items():
            assert k == (1 if e in bnd else 2), (f, e, k)
        assert bnd <= set(count)
        V = {v for t in T for v in t}
        assert len(V) - len(count) + len(T) == 1
        whole = _area(X[[a, b, c]])
        parts = sum(_area(X[list(t)]) for t in T)
        assert abs(parts - whole) <= 1e-9 * whole
        made += len(r["facet_points"][f])
    assert made > 0


def test_facet_points_lie_on_their_facets(big):
    pts, plc, r = big
    X = r["xyz"]
    for f, tri in enumerate(plc["tris"]):
        P = X[list(tri)]
        nrm = np.cross(P[1] - P[0], P[2] - P[0])
        nrm /= np.linalg.norm(nrm)
        diam = max(np.linalg.norm(P[i] - P[j]) for i in range(3) for j in range(3))
        for v in r["facet_points"][f]:
            x = X[v]
            assert abs((x - P[0]) @ nrm) <= 1e-12 * diam
            # barycentric coordinates in the facet's plane: all positive
            w = [np.cross(P[(k + 1) % 3] - x, P[(k + 2) % 3] - x) @ nrm for k in range(3)]
            assert min(w) > 0, (f, v, w)


def test_recovered_mesh_is_delaunay_by_brute_force():
    pts, plc, r = _case(300, 2, 3, 7, 60)
    assert len(r["xyz"]) > len(pts) and sum(map(len, r["facet_points"])) > 0
    assert r["mesh"].check_brute() == 0


def test_facets_split_exactly_where_needed():
    """A triangle that is a face of the points' Delaunay mesh and whose edges
    are Delaunay edges gets no point; the large facets of the other case do."""
    pts, _, _ = inputs.box_points("uniform", 500, 9)
    tets = oracle.Mesh.box_delaunay(pts).export()["tets"]
    F = sorted(t for t in _face_set(tets) if min(t) >= 8)
    tri = np.array([F[len(F) // 2]], dtype=np.int32)
    segs = np.array([[tri[0, 0], tri[0, 1]], [tri[0, 1], tri[0, 2]], [tri[0, 2], tri[0, 0]]])
    r = recover_plc(pts, segs, tri, np.array([[0, 1, 2]]))
    assert r["passes"] == 0 and r["facet_points"] == [[]]
    assert r["subfaces"] == [[tuple(sorted(int(v) for v in tri[0]))]]


def _oracle_labels(r):
    X = r["xyz"]
    e = r["mesh"].export()
    lab = inputs.plc_recovered(X, e["tets"], r["chains"], r["subfaces"])
    s = reference_shift(X)
    first = {}
    for t, f in zip(lab["tris"], lab["facet_id"]):
        first.setdefault(int(f), t)
    q = np.zeros((lab["nfacets"], 3))
    for f in range(6):
        t = first[f]
        q[f] = facet_reference(X, int(t[0]), int(t[1]), int(t[2]), s)
    q[6:] = r["facetq"]
    return e, lab, q


def test_recovered_facets_meet_the_contract_and_refine():
    B = 1.5
    pts, plc, r = _case(900, 4, 5, 11, 80)
    e, lab, q = _oracle_labels(r)
    m = r["mesh"]
    assert m.set_constraints(lab["segs"], lab["seg_id"], lab["tris"], lab["facet_id"],
                             lab["nfacets"], facetq=q) == 0
    c = m.check(B)
    for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
              "hull_not_subface", "seg_chain_bad"):
        assert c[k] == 0, k
    assert c["euler"] == 1 and abs(c["vol_rel_err"]) < 1e-12
    m.refine_R(B)
    c = m.check(B)
    for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
              "seg_chain_bad", "enc_subsegs", "enc_subfaces", "bad_tets"):
        assert c[k] == 0, k


def _oracle_evaluate(kind, items):
    n = len(items)
    sg = np.zeros(n, dtype=np.int32)
    out = np.zeros((n, 3))
    for r, it in enumerate(items):
        a, b, c, d, e = it[0:3], it[3:6], it[6:9], it[9:12], it[12:15]
        if kind == "orient":
            sg[r] = oracle.orient3d(a, b, c, d)
        elif kind == "insphere":
            sg[r] = oracle.insphere(a, b, c, d, e)
        elif kind == "diametral":
            sg[r] = oracle.diametral(a, b, c)
        elif kind == "tri_cc":
            p, ok = oracle.tri_circumcenter(a, b, c)
            out[r], sg[r] = p, int(ok)
        elif kind == "midpoint":
            out[r], sg[r] = oracle.midpoint(a, b), 1
        else:
            raise ValueError(kind)
    return sg, out


def _oracle_delaunay(x):
    m = oracle.Mesh.box_delaunay(x)
    assert m.skipped == 0
    return m.export()["tets"]


def test_product_pass_logic_equals_the_oracle_with_its_primitives(big):
    from paper_1903_03406_gb300 import recover
    pts, plc, r = big
    g = recover.recover_plc(pts, plc["segs"], plc["tris"], plc["tri_segs"], None,
                            evaluate=_oracle_evaluate, delaunay=_oracle_delaunay)
    assert g["passes"] == r["passes"]
    assert np.array_equal(g["xyz"], r["xyz"])
    assert g["chains"] == r["chains"] and g["facet_points"] == r["facet_points"]
    assert [list(map(tuple, s)) for s in g["subfaces"]] == r["subfaces"]
    assert np.array_equal(g["facetq"], r["facetq"])
