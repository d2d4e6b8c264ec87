"""Brute-force pins for three round rules of the oracle's mode R that decide
which candidates a round inserts (Sec. 2, grow-and-blast), each checked from
the round report against a restatement of the rule over the snapshot the round
started from:

* start-claim blasting (reading r5): every candidate whose point was located
  claims its start tetrahedra; a candidate is stopped ("blasted") exactly when
  its cavity, or the shell of tetrahedra across its cavity's boundary faces,
  holds a start claimed by a located candidate of higher priority;
* the stall rule of subsegment rounds (reading r12): a round with subsegment
  candidates gives its refused subsegment candidates up exactly when it
  inserted nothing, gave nothing else up and flagged no subsegment outside its
  candidate set;
* the facet part of a cavity (reading r6/r7): the subfaces of the point's facet
  whose circumcircle strictly contains it, connected to its start subfaces
  without crossing a subsegment, computed by brute force over every subface
  with exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from _meshes import oracle_case

RS_WALK = {1, 2, 3, 4, 5}  # bad point, walk crossed a subface / subsegment, limit, hull
RS_OVERFLOW = 7
RS_STALL = 10


def _split(a, counts, width):
    off = np.concatenate([[0], np.cumsum(counts)])
    return [{tuple(int(v) for v in t) for t in a[off[i]:off[i + 1]]} for i in range(len(counts))]


def _ncls(keys):
    return (keys >= 0).sum(axis=1)  # 2 subsegment, 3 subface, 4 tetrahedron


# --------------------------------------------------------------- blasting
def _check_blasting(snap, rep):
    """Returns (candidates checked, blasted, blasted through the shell only)."""
    tets = np.sort(snap["tets"], axis=1)
    tset = {tuple(int(v) for v in t) for t in tets}
    v2t = {}  # vertex -> tetrahedra holding it (built on first use)
    xyz = snap["xyz"]
    n = len(rep["keys"])
    starts = _split(rep["starts"], rep["nstart"], 4)
    cav = _split(rep["cav"], rep["ncav"], 4)
    shell = _split(rep["shell"], rep["nshell"], 4)
    sf = {tuple(sorted(int(v) for v in f[:3])): int(f[3]) for f in snap["sf"]}
    ncls = _ncls(rep["keys"])
    claimed = {}  # start tetrahedron -> first (highest-priority) located claimant
    blasted = via_shell = 0
    for i in range(n):
        located = len(starts[i]) > 0
        # located exactly when the point was found in the mesh (no walk failure),
        # and then its region was grown
        assert located == (rep["reason"][i] not in RS_WALK and len(cav[i]) > 0), i
        if located:
            assert starts[i] <= tset and starts[i] <= cav[i], i
            key = tuple(int(v) for v in rep["keys"][i][:ncls[i]])
            p = rep["pts"][i]
            if ncls[i] == 2:  # the ring of tetrahedra around the subsegment
                if not v2t:
                    for t in tset:
                        for v in t:
                            v2t.setdefault(v, set()).add(t)
                ring = v2t.get(key[0], set()) & v2t.get(key[1], set())
                assert starts[i] == ring, i
            elif ncls[i] == 4:  # one tetrahedron that holds the point
                assert len(starts[i]) == 1, i
                (t,) = starts[i]
                for q in range(4):
                    c = [p if k == q else xyz[t[k]] for k in range(4)]
                    s = oracle.orient3d(*c)
                    # oriented tetrahedra were sorted: compare with the sorted tet's sign
                    assert s * oracle.orient3d(*xyz[list(t)]) >= 0, i
            else:  # both sides of one subface of the candidate's facet
                assert 1 <= len(starts[i]) <= 2, i
                common = set.intersection(*[set(t) for t in starts[i]])
                faces = [tuple(sorted(c)) for c in
                         ([common] if len(common) == 3 else
                          [[v for v in next(iter(starts[i])) if v != w]
                           for w in next(iter(starts[i]))])]
                assert any(f in sf and sf[f] == sf[key] for f in faces), i
        for t in starts[i] if located else ():
            claimed.setdefault(t, i)
        hit_cav = any(claimed.get(t, n) < i for t in cav[i])
        hit_shell = rep["reason"][i] != RS_OVERFLOW and any(claimed.get(t, n) < i
                                                            for t in shell[i])
        expect = located and (hit_cav or hit_shell)
        assert (rep["outcome"][i] == oracle.OUT_BLASTED) == expect, \
            "candidate %d: outcome %d, cavity hit %s, shell hit %s" % (
                i, rep["outcome"][i], hit_cav, hit_shell)
        blasted += expect
        via_shell += expect and not hit_cav
    return n, blasted, via_shell


@pytest.mark.parametrize("mixed", [0, 1])
def test_blasting_follows_start_claims(mixed):
    om, e, plc = oracle_case("uniform", 600, 8, 8, 21)
    om.set_mixed(mixed)
    n = b = sh = 0
    classes = set()
    want = {0, 1, 2} if mixed == 0 else {3}
    for _ in range(400):
        snap = om.export()
        r = om.round(1.4)
        if r["cls"] < 0:
            break
        classes.add(r["cls"])
        a, bb, s = _check_blasting(snap, om.report())
        n, b, sh = n + a, b + bb, sh + s
        if n > 3000 and classes >= want and sh > 0:
            break
    assert n > 3000 and b > 100 and sh > 0
    assert classes >= want


# ------------------------------------------------------------- stall rule
def test_stall_rule_fires_exactly_on_stalled_subsegment_rounds():
    """Inputs with dense free segments, where the rule fires and where a round
    without insertions still makes progress by giving an element up (so a rule
    that ignored give-ups would fire there too)."""
    fired = decided_by_give_up = 0
    for kind, n, ns, nt, seed, mixed in [("uniform", 800, 60, 4, 25, 0),
                                         ("uniform", 800, 60, 4, 2, 0),
                                         ("uniform", 800, 60, 4, 2, 1)]:
        om, e, plc = oracle_case(kind, n, ns, nt, seed)
        om.set_mixed(mixed)
        for rnd in range(150):
            r = om.round(1.4)
            if r["cls"] < 0:
                break
            rep = om.report()
            seg = _ncls(rep["keys"]) == 2
            if not seg.any():
                assert not (rep["reason"] == RS_STALL).any()
                continue
            cand_segs = {tuple(int(v) for v in k[:2]) for k in rep["keys"][seg]}
            flagged = {tuple(int(v) for v in g) for g in rep["flagG"]}
            gave_up = ((rep["outcome"] == oracle.OUT_UNSPL) & (rep["reason"] != RS_STALL)).any()
            inserted = rep["surv"].sum() > 0
            stalled = not inserted and not gave_up and flagged <= cand_segs
            fires = bool((rep["reason"] == RS_STALL).any())
            assert fires == stalled, "%s %d round %d: stall rule %s" % (kind, seed, rnd, fires)
            if fires:
                fired += 1
                # every refused subsegment candidate was given up, nothing else
                assert not (seg & (rep["outcome"] == oracle.OUT_REJECT)).any()
                assert (seg[rep["reason"] == RS_STALL]).all()
            elif (not inserted and gave_up and flagged <= cand_segs
                  and (seg & (rep["outcome"] == oracle.OUT_REJECT)).any()):
                decided_by_give_up += 1  # a refused candidate the rule left alone
    assert fired >= 3 and decided_by_give_up >= 1


# ------------------------------------------------------ facet part of a cavity
def _q(x):
    return Fraction(float(x))


def _orient2(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _incircle2(a, b, c, p):
    """> 0: p strictly inside the circumcircle of the counter-clockwise a, b, c."""
    rows = [(x[0] - p[0], x[1] - p[1]) for x in (a, b, c)]
    m = [(u, v, u * u + v * v) for u, v in rows]
    det = (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
           - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
           + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))
    return det


def _check_facet_cavities(snap, rep):
    """Axis-parallel facets only (every point on such a facet lies exactly in
    its plane: midpoints and in-facet circumcentres keep the shared
    coordinate). Returns (candidates checked, equal)."""
    xyz = snap["xyz"]
    sf = [tuple(sorted(int(v) for v in f[:3])) for f in snap["sf"]]
    fid = {k: int(f[3]) for k, f in zip(sf, snap["sf"])}
    axis_of = {}
    for k in sf:
        for ax in range(3):
            if xyz[k[0]][ax] == xyz[k[1]][ax] == xyz[k[2]][ax]:
                axis_of.setdefault(fid[k], ax)
    segs = {tuple(sorted(int(v) for v in g[:2])) for g in snap["ss"]}
    edge2sf = {}
    for k in sf:
        for e in ((k[0], k[1]), (k[0], k[2]), (k[1], k[2])):
            edge2sf.setdefault(e, []).append(k)
    fcav = _split(rep["fcav"], rep["nfcav"], 3)
    ncls = _ncls(rep["keys"])
    n = same = 0
    for i in np.nonzero(rep["outcome"] == oracle.OUT_OK)[0]:
        if ncls[i] == 4:
            continue
        key = tuple(int(v) for v in rep["keys"][i][:ncls[i]])
        p3 = rep["pts"][i]
        if ncls[i] == 3:
            facets = {fid[key]}
        else:
            facets = {fid[s] for s in edge2sf.get(key, [])}
        region = set()
        for F in facets:
            ax = axis_of[F]
            keep = [k for k in range(3) if k != ax]
            P = {}

            def pt(v):
                if v not in P:
                    P[v] = (_q(xyz[v][keep[0]]), _q(xyz[v][keep[1]]))
                return P[v]
            p = (_q(p3[keep[0]]), _q(p3[keep[1]]))
            mine = [k for k in sf if fid[k] == F]
            inside = set()
            holds = []
            for k in mine:
                a, b, c = (pt(v) for v in k)
                if _orient2(a, b, c) < 0:
                    b, c = c, b
                if _incircle2(a, b, c, p) > 0:
                    inside.add(k)
                if ncls[i] == 3 and min(_orient2(a, b, p), _orient2(b, c, p),
                                        _orient2(c, a, p)) >= 0:
                    holds.append(k)
            if ncls[i] == 2:
                holds = [k for k in edge2sf[key] if fid[k] == F]
            assert holds
            K = {k for k in holds if k in inside}
            stack = list(K)
            while stack:
                k = stack.pop()
                for e in ((k[0], k[1]), (k[0], k[2]), (k[1], k[2])):
                    if e in segs:
                        continue
                    for nb in edge2sf[e]:
                        if fid[nb] == F and nb in inside and nb not in K:
                            K.add(nb)
                            stack.append(nb)
            region |= K
            # nothing outside the closed circumcircle joins the facet part
            for k in fcav[i]:
                if fid[k] == F:
                    a, b, c = (pt(v) for v in k)
                    if _orient2(a, b, c) < 0:
                        b, c = c, b
                    assert _incircle2(a, b, c, p) >= 0, (i, k)
        assert region <= fcav[i], i
        assert {fid[k] for k in fcav[i]} <= facets, i
        n += 1
        same += region == fcav[i]
    return n, same


def test_facet_cavities_are_bowyer_watson_regions():
    """Sec. 2's Delaunay region inside a facet, for subface and subsegment
    candidates on the box facets of a refined cube."""
    from test_oracle_mesh import cube_mesh
    m, *_ = cube_mesh(150, seed=9)
    n = same = 0
    seen = {0: 0, 1: 0}
    for _ in range(3000):
        snap = m.export()
        cls = m.round(2.0)["cls"]
        if cls < 0:
            break
        if cls in seen and seen[cls] < 6:
            seen[cls] += 1
            a, b = _check_facet_cavities(snap, m.report())
            n += a
            same += b
    assert seen == {0: 6, 1: 6}
    assert n > 40 and same == n


def _quad_case():
    """The unit cube and a quad facet in the plane z = 0.5 given as two
    triangles, with its diagonal declared a segment (a segment inside a
    facet, as a PLC allows). Cloud points are kept off the two triangles'
    equatorial balls so that both triangles are faces of the Delaunay mesh."""
    corners = np.array([[float((c >> k) & 1) for k in range(3)] for c in range(8)])
    quad = np.array([[0.2, 0.2, 0.5], [0.8, 0.25, 0.5], [0.75, 0.8, 0.5], [0.25, 0.7, 0.5]])
    rng = np.random.default_rng(3)
    cloud = rng.uniform(0.02, 0.98, size=(1500, 3))
    for tri in ([0, 1, 3], [1, 2, 3]):
        c, ok = oracle.tri_circumcenter(*quad[tri])
        r = np.linalg.norm(quad[tri[0]] - c)
        cloud = cloud[np.linalg.norm(cloud - c, axis=1) > 1.1 * r]
    pts = np.concatenate([corners, quad, cloud])
    m = oracle.Mesh.box_delaunay(pts)
    e = m.export()
    from paper_1903_03406_gb300 import inputs
    faces, cnt, _ = inputs._faces_edges(e["tets"])
    tris, fids, segs, sids = inputs._box_labels(pts, faces, cnt)
    a, b, c, d = 8, 9, 10, 11
    tris += [[a, b, d], [b, c, d]]
    fids += [6, 6]
    for u, v in ((a, b), (b, c), (c, d), (d, a), (b, d)):  # (b, d) lies inside the facet
        segs.append((u, v))
        sids.append(len(sids))
    assert m.set_constraints(np.array(segs), np.array(sids), np.array(tris), np.array(fids),
                             7) == 0
    return m


def test_facet_cavities_do_not_cross_a_segment_inside_the_facet():
    """A facet region is grown across the facet's edges but never across a
    subsegment, here the diagonal segment inside a quad facet: by brute force,
    the same facet parts as the oracle's, on the first subface and subsegment
    rounds of the refinement."""
    m = _quad_case()
    n = same = checked = 0
    for _ in range(400):
        snap = m.export()
        cls = m.round(2.0)["cls"]
        if cls < 0 or checked >= 12:
            break
        if cls in (0, 1):
            a, b = _check_facet_cavities(snap, m.report())
            n += a
            same += b
            checked += 1
    assert n > 20 and same == n

