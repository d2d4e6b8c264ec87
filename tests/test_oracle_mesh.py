"""Pins for the oracle's meshes: Delaunay by brute force on tiny inputs, and the
output contract of the refinement problem (Sec. 1) on refined meshes."""
import numpy as np
import pytest

import oracle
from paper_1903_03406_gb300 import inputs


def cube_mesh(n, seed=0):
    pts, lo, hi = inputs.box_points("cube", n, seed)
    m = oracle.Mesh.box_delaunay(pts)
    e = m.export()
    plc = inputs.plc_from_delaunay(pts, e["tets"], 0, 0, seed)
    assert m.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                             plc["nfacets"]) == 0
    return m, pts, e, plc


def constrained_mesh(n, ns, nt, seed, kind="uniform"):
    pts, lo, hi = inputs.box_points(kind, n, seed)
    m = oracle.Mesh.box_delaunay(pts)
    e = m.export()
    plc = inputs.plc_from_delaunay(pts, e["tets"], ns, nt, seed)
    assert m.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                             plc["nfacets"]) == 0
    return m, pts, e, plc


def assert_contract(c, B, allow_unspl=True):
    assert c["bad_orient"] == 0
    assert c["nonlocal_delaunay"] == 0
    assert abs(c["vol_rel_err"]) < 1e-12
    assert c["euler"] == 1
    assert c["sf_not_face"] == 0 and c["ss_not_edge"] == 0
    assert c["hull_not_subface"] == 0
    assert c["seg_chain_bad"] == 0
    assert c["facet_area_rel_err"] < 1e-12
    assert c["enc_subsegs"] == 0 and c["enc_subfaces"] == 0
    assert c["bad_tets"] == 0
    if not allow_unspl:
        assert c["bad_tets_unspl"] == 0


@pytest.mark.parametrize("n", [20, 60, 150])
def test_box_delaunay_brute_force(n):
    m, pts, e, plc = cube_mesh(n, seed=n)
    assert m.check_brute() == 0
    c = m.check(2.0)
    assert c["bad_orient"] == 0 and abs(c["vol_rel_err"]) < 1e-12 and c["euler"] == 1
    assert c["verts_used"] == n + 8
    assert c["hull_not_subface"] == 0 and c["subfaces"] == 12 and c["subsegs"] == 12


def test_box_delaunay_degenerate_grid():
    # the corners of [0,4]^3 and the interior grid {1,2,3}^3: every unit cell
    # has 8 cospherical corners (the builder takes interior points only)
    g = [[x, y, z] for x in (0, 4) for y in (0, 4) for z in (0, 4)]
    g += [[x, y, z] for x in (1, 2, 3) for y in (1, 2, 3) for z in (1, 2, 3)]
    m = oracle.Mesh.box_delaunay(np.array(g, dtype=float))
    assert m.skipped == 0
    assert m.check_brute() == 0
    c = m.check(2.0)
    assert c["bad_orient"] == 0 and abs(c["vol_rel_err"]) < 1e-12 and c["euler"] == 1
    assert c["verts_used"] == 35


def test_refine_cube_mode_S_contract():
    m, *_ = cube_mesh(120, seed=3)
    st = m.refine_S(2.0)
    assert st["inserted"] > 0
    c = m.check(2.0)
    assert_contract(c, 2.0, allow_unspl=False)
    # only hull constraints: the refined mesh is Delaunay, checked by brute force
    assert m.check_brute() == 0


def test_refine_cube_mode_R_contract_and_band():
    mS, pts, e, plc = cube_mesh(200, seed=4)
    mR = oracle.Mesh.create(e["xyz"], e["tets"])
    mR.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    sS = mS.refine_S(2.0)
    sR = mR.refine_R(2.0)
    cS, cR = mS.check(2.0), mR.check(2.0)
    assert_contract(cS, 2.0, allow_unspl=False)
    assert_contract(cR, 2.0, allow_unspl=False)
    assert mR.check_brute() == 0
    # Steiner counts of the two insertion orders agree within 1.15x
    assert max(sS["inserted"], sR["inserted"]) <= 1.15 * min(sS["inserted"], sR["inserted"])


def test_refine_constrained_both_modes():
    mS, pts, e, plc = constrained_mesh(1500, 15, 15, seed=5)
    mR = oracle.Mesh.create(e["xyz"], e["tets"])
    mR.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    B = 1.4
    sS = mS.refine_S(B)
    sR = mR.refine_R(B)
    cS, cR = mS.check(B), mR.check(B)
    assert_contract(cS, B)
    assert_contract(cR, B)
    # the bad tetrahedra left (unsplittable) are a small fraction of the mesh
    assert cS["bad_tets_unspl"] <= 0.01 * cS["tets"]
    assert cR["bad_tets_unspl"] <= 0.01 * cR["tets"]
    assert max(sS["inserted"], sR["inserted"]) <= 1.15 * min(sS["inserted"], sR["inserted"])
    # rounds leave no larger a fraction of bad tetrahedra than sequential refinement, within 1.15x
    assert cR["bad_tets_unspl"] / cR["tets"] <= 1.15 * cS["bad_tets_unspl"] / cS["tets"]


def test_mixed_rounds_contract_band_and_fewer_rounds():
    """Mixed rounds (every flagged element a candidate, class first in the
    priority): a valid refinement within the 1.15x band of mode S, in fewer
    rounds than one class per round."""
    B = 1.4
    mS, pts, e, plc = constrained_mesh(600, 6, 6, seed=8)
    m1 = oracle.Mesh.create(e["xyz"], e["tets"])
    m1.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    mM = oracle.Mesh.create(e["xyz"], e["tets"])
    mM.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    mM.set_mixed(True)
    sS = mS.refine_S(B)
    s1 = m1.refine_R(B)
    sM = mM.refine_R(B)
    assert_contract(mM.check(B), B)
    assert max(sS["inserted"], sM["inserted"]) <= 1.15 * min(sS["inserted"], sM["inserted"])
    assert sM["rounds"] < s1["rounds"]
    # a mixed round serves several classes while they are all flagged
    mM2 = oracle.Mesh.create(e["xyz"], e["tets"])
    mM2.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    mM2.set_mixed(True)
    seen = set()
    while True:
        c = mM2.round(B)["cls"]
        if c < 0:
            break
        seen.add(c)
        if c == 3:
            rep = mM2.report()
            assert len(rep["keys"]) > 0
    assert 3 in seen


def test_mode_R_survivors_touch_disjoint_sets():
    m, *_ = constrained_mesh(800, 8, 8, seed=6)
    B = 1.4
    rounds = 0
    while rounds < 40:
        o = m.round(B)
        if o["cls"] < 0:
            break
        rep = m.report()
        off = np.concatenate([[0], np.cumsum(rep["ncav"])])
        seen = set()
        for i in np.nonzero(rep["surv"])[0]:
            cav = {tuple(t) for t in rep["cav"][off[i]:off[i + 1]]}
            assert not (cav & seen)
            seen |= cav
        # the kept candidates are exactly the round's insertions
        assert rep["surv"].sum() == o["inserted"]
        # the highest-priority eligible candidate always survives
        ok = np.nonzero(rep["outcome"] == oracle.OUT_OK)[0]
        if len(ok):
            assert rep["surv"][ok[0]] == 1
        rounds += 1
    c = m.check(B)
    assert c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0
    assert c["sf_not_face"] == 0 and c["ss_not_edge"] == 0


def test_planted_mistakes_are_caught():
    """Plant mistakes into copies of the oracle's data and check the checkers see
    them: an inverted tetrahedron, a dropped tetrahedron, a missing subface."""
    m, pts, e, plc = cube_mesh(60, seed=7)
    tets = e["tets"].copy()
    tets[0, [1, 2]] = tets[0, [2, 1]]
    bad = oracle.Mesh.create(e["xyz"], tets)
    bad.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    assert bad.check(2.0)["bad_orient"] == 1
    dropped = oracle.Mesh.create(e["xyz"], e["tets"][1:])
    c = dropped.check(2.0)
    assert c["euler"] != 1 or c["hull_not_subface"] > 0
    # a constraint label that is not a mesh face is reported
    tris = plc["tris"].copy()
    tris[0] = [0, 7, 3]
    mm = oracle.Mesh.create(e["xyz"], e["tets"])
    assert mm.set_constraints(plc["segs"], plc["seg_id"], tris, plc["facet_id"], plc["nfacets"]) >= 1


RS_OVERFLOW = 7  # the oracle's reason code for a cavity over the limit


def _run_rounds(m, B, max_rounds=3000):
    """Mode R rounds to the end; returns (largest survivor cavity, overflow count)."""
    biggest = overflows = 0
    for _ in range(max_rounds):
        if m.round(B)["cls"] < 0:
            break
        rep = m.report()
        if rep["surv"].any():
            biggest = max(biggest, int(rep["ncav"][rep["surv"] == 1].max()))
        overflows += int((rep["reason"] == RS_OVERFLOW).sum())
    return biggest, overflows


def test_cavity_limit_gives_points_up_and_keeps_the_mesh_valid():
    """A region whose cavity outgrows the limit is not inserted: its element is
    given up as unsplittable (reading r12), and the mesh stays a valid CDT."""
    B, limit = 1.6, 24
    m, *_ = constrained_mesh(300, 3, 3, seed=8)
    m.set_limits(cav_limit=limit)
    biggest, overflows = _run_rounds(m, B)
    assert overflows > 0
    assert biggest <= limit
    c = m.check(B)
    assert_contract(c, B)
    assert c["bad_tets_unspl"] > 0
    # the default limit never binds on this input
    m2, *_ = constrained_mesh(300, 3, 3, seed=8)
    _, overflows2 = _run_rounds(m2, B)
    assert overflows2 == 0


def _faces(t):
    a, b, c, d = t
    return [tuple(sorted(x)) for x in ((b, c, d), (a, c, d), (a, b, d), (a, b, c))]


def _check_cavities_by_brute_force(snap, rep):
    """Every eligible candidate's cavity, on a mesh whose only constraints are
    on the hull (so it stays Delaunay), is the Bowyer-Watson region of its
    point: the tetrahedra whose circumsphere strictly contains p, connected
    through shared faces to the tetrahedra that contain p. Tetrahedra with p
    on their circumsphere may join only through the star closure. Returns
    (candidates checked, cavities equal to the strict region)."""
    xyz, tets = snap["xyz"], snap["tets"]
    key = [tuple(sorted(t)) for t in tets]
    index = {k: i for i, k in enumerate(key)}
    f2t = {}
    for i, t in enumerate(key):
        for f in _faces(t):
            f2t.setdefault(f, []).append(i)
    off = np.concatenate([[0], np.cumsum(rep["ncav"])])
    n = same = 0
    for i in np.nonzero(rep["outcome"] == oracle.OUT_OK)[0]:
        p = rep["pts"][i]
        C = {index[tuple(t)] for t in rep["cav"][off[i]:off[i + 1]]}
        ins = np.array([oracle.insphere(*xyz[t], p) for t in tets])
        inside = set(np.nonzero(ins > 0)[0])
        holds = [j for j, t in enumerate(tets)
                 if all(oracle.orient3d(*[p if k == q else xyz[t[k]] for k in range(4)]) >= 0
                        for q in range(4))]
        assert holds and set(holds) <= C
        K = {j for j in holds if j in inside}
        stack = list(K)
        while stack:
            j = stack.pop()
            for f in _faces(key[j]):
                for nb in f2t[f]:
                    if nb in inside and nb not in K:
                        K.add(nb)
                        stack.append(nb)
        assert K <= C
        assert all(ins[j] >= 0 for j in C)
        n += 1
        same += K == C
    return n, same


def test_cavities_are_bowyer_watson_regions():
    """Sec. 2's Delaunay region of a splitting point, checked by brute force over
    every tetrahedron, for the first rounds of each class."""
    m, *_ = cube_mesh(150, seed=9)
    B = 2.0
    seen = {0: 0, 1: 0, 2: 0}
    n = same = 0
    for _ in range(2000):
        snap = m.export()
        cls = m.round(B)["cls"]
        if cls < 0:
            break
        if seen[cls] < 3:
            seen[cls] += 1
            a, b = _check_cavities_by_brute_force(snap, m.report())
            n += a
            same += b
    assert seen == {0: 3, 1: 3, 2: 3}
    assert n > 50 and same == n  # no cospherical ties here: every cavity is the strict region


def _global_encroached(ex):
    """Subsegments and subfaces to split, by brute force over every mesh vertex:
    those with a vertex strictly inside their diametral (equatorial) sphere, or
    flagged by a refused point; unsplittable ones excluded. Floating point only
    preselects the vertices near the sphere; the exact predicates decide."""
    xyz = ex["xyz"]
    used = np.unique(ex["tets"])
    V = xyz[used]
    s2 = np.abs(xyz).max() ** 2
    ng = ns = 0
    for (a, b, _), fl in zip(ex["ss"], ex["ssflag"]):
        if fl & 2:
            continue
        if fl & 1:
            ng += 1
            continue
        A, Bv = xyz[a], xyz[b]
        near = np.nonzero(np.einsum("ij,ij->i", A - V, Bv - V) < 1e-9 * s2)[0]
        ng += any(oracle.diametral(A, Bv, xyz[used[j]]) < 0
                  for j in near if used[j] not in (a, b))
    for (a, b, c, _), fl in zip(ex["sf"], ex["sfflag"]):
        if fl & 2:
            continue
        if fl & 1:
            ns += 1
            continue
        A, Bv, Cv = xyz[a], xyz[b], xyz[c]
        cc, _ok = oracle.tri_circumcenter(A, Bv, Cv)
        R2 = np.sum((A - cc) ** 2)
        near = np.nonzero(np.sum((V - cc) ** 2, axis=1) - R2 < 1e-9 * R2 + 1e-12 * s2)[0]
        ns += any(oracle.equatorial(A, Bv, Cv, xyz[used[j]]) < 0
                  for j in near if used[j] not in (a, b, c))
    return ng, ns


@pytest.mark.parametrize("case", ["cube", "constrained"])
def test_local_encroachment_equals_global_brute_force(case):
    """Reading c1/r1 tests encroachment locally (the apexes of the tetrahedra
    around the element). On a CDT that finds every encroaching vertex: the
    class queues equal a brute-force test over all vertices, round by round."""
    if case == "cube":
        m, *_ = cube_mesh(300, seed=21)
        B, rounds = 2.0, 400
    else:
        m, *_ = constrained_mesh(400, 4, 4, seed=22)
        B, rounds = 1.5, 25
    total = [0, 0]
    for _ in range(rounds):
        q = m.classify(B)
        g = _global_encroached(m.export())
        assert (q[0], q[1]) == g
        total[0] += g[0]
        total[1] += g[1]
        if m.round(B)["cls"] < 0:
            break
    assert total[0] > 20 and total[1] > 20


def test_every_round_leaves_a_cdt():
    """Sec. 2: the mesh is a CDT again at the end of every round (the survivors'
    regions and shells are disjoint, so their concurrent insertion is valid)."""
    m, *_ = constrained_mesh(500, 5, 5, seed=23)
    B = 1.5
    classes = set()
    for _ in range(1000):
        o = m.round(B)
        if o["cls"] < 0:
            break
        classes.add(o["cls"])
        c = m.check(B)
        assert c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0
        assert abs(c["vol_rel_err"]) < 1e-12 and c["euler"] == 1
        assert c["sf_not_face"] == 0 and c["ss_not_edge"] == 0 and c["hull_not_subface"] == 0
        assert c["seg_chain_bad"] == 0 and c["facet_area_rel_err"] < 1e-12
    assert classes == {0, 1, 2}


def _splitmix_chain(cls, words):
    """Reading r3's hash, restated: SplitMix64's finaliser chained over 64-bit words,
    seeded by the golden-ratio constant times (class + 1)."""
    M64 = (1 << 64) - 1
    h = (0x9E3779B97F4A7C15 * (cls + 1)) & M64
    for w in words:
        z = h ^ int(w)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        h = z ^ (z >> 31)
    return h


def test_candidates_follow_the_predetermined_priority():
    """Sec. 2's predetermined priorities (reading r3): a round's candidates come
    in the order of class << 62 | (h >> 2), h the hash of the element's vertex
    coordinates in ascending id order, ties broken by the sorted vertex ids."""
    m, *_ = constrained_mesh(300, 3, 3, seed=24)
    B = 1.5
    seen = set()
    for _ in range(400):
        snap = m.export()
        o = m.round(B)
        if o["cls"] < 0:
            break
        if o["cls"] in seen and len(seen) < 3:
            continue
        seen.add(o["cls"])
        rep = m.report()
        keys = [tuple(int(v) for v in k if v >= 0) for k in rep["keys"]]
        order = []
        for k in keys:
            words = snap["xyz"][list(k)].reshape(-1).view(np.uint64)
            h = _splitmix_chain(o["cls"], words)
            order.append(((o["cls"] << 62) | (h >> 2), k))
        assert order == sorted(order)
        assert len(keys) == o["ncand"]
        if seen == {0, 1, 2}:
            break
    assert seen == {0, 1, 2}
