"""Parity of the CUDA path with the oracle, through the C-ABI (needs a GPU).

* predicates and splitting-point formulas: signs bit-exact against the oracle's
  exact evaluation on random and degenerate inputs; points bit-identical;
* create -> export round-trips the mesh;
* rounds in lockstep from a shared snapshot: same class, same candidate order,
  bit-identical splitting points, same outcomes, survivors and cavities, and the
  same mesh after every round (vertex coordinates bit-exact).
"""
import numpy as np
import pytest

import oracle
from _meshes import assert_same_mesh, compare_reports, oracle_case, oracle_from_export

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


def gpu_handle(cdr, e, plc, **kw):
    return cdr.Handle.create(e["xyz"], e["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                             plc["facet_id"], plc["nfacets"], **kw)


# ------------------------------------------------------------------ predicates
def _families(rng, n):
    out = []
    for i in range(n):
        k = i % 6
        if k == 0:
            P = rng.uniform(-1, 1, size=(5, 3))
        elif k == 1:
            P = rng.integers(-2, 3, size=(5, 3)).astype(np.float64)
        elif k == 2:
            S = np.array([[1, 2, 2], [2, 1, 2], [2, 2, 1], [-1, 2, 2], [2, -1, 2], [2, 2, -1],
                          [1, -2, 2], [3, 0, 0], [0, 3, 0], [0, 0, 3], [0, 0, -3], [-2, -2, 1]],
                         dtype=np.float64)
            P = S[rng.choice(len(S), size=5, replace=False)] * 0.37 + 1000.0
        elif k == 3:
            P = rng.integers(-2, 3, size=(5, 3)).astype(np.float64) * 0.1 + 0.3
            j, c = rng.integers(0, 5), rng.integers(0, 3)
            P[j, c] = np.nextafter(P[j, c], np.inf if rng.random() < 0.5 else -np.inf)
        elif k == 4:
            # nearly cospherical, relative noise 1e-9..1e-5: the FP32 stage's bound
            # must make it defer, never decide wrongly
            d = rng.normal(size=(5, 3))
            P = 500.0 + 37.0 * d / np.linalg.norm(d, axis=1, keepdims=True)
            P *= 1.0 + 10.0 ** rng.uniform(-9, -5) * rng.normal(size=(5, 3))
        else:
            # nearly coplanar (for orient3d), same noise
            u, v = rng.normal(size=3), rng.normal(size=3)
            P = 250.0 + rng.normal(size=(5, 1)) * u * 40 + rng.normal(size=(5, 1)) * v * 40
            P *= 1.0 + 10.0 ** rng.uniform(-9, -5) * rng.normal(size=(5, 3))
        out.append(P)
    return out


def _items(Ps, B=None):
    it = np.zeros((len(Ps), 16))
    for i, P in enumerate(Ps):
        it[i, :15] = P.reshape(-1)[:15]
        if B is not None:
            it[i, 12] = B
    return it


def test_predicate_signs_match_oracle(cdr):
    rng = np.random.default_rng(101)
    Ps = _families(rng, 4000)
    it = _items(Ps)
    s_or, _ = cdr.eval_predicates("orient", it)
    s_or_x, _ = cdr.eval_predicates("orient_exact", it)
    s_in, _ = cdr.eval_predicates("insphere", it)
    s_in_x, _ = cdr.eval_predicates("insphere_exact", it)
    s_di, _ = cdr.eval_predicates("diametral", it)
    s_eq, _ = cdr.eval_predicates("equatorial", it)
    s_eq_x, _ = cdr.eval_predicates("equatorial_exact", it)
    zeros = 0
    for i, P in enumerate(Ps):
        a, b, c, d, e = P
        o = oracle.orient3d(a, b, c, d)
        assert s_or[i] == o and s_or_x[i] == o, i
        zeros += o == 0
        # insphere is defined for positively oriented (a,b,c,d); the sign of the
        # lifted determinant flips with orientation, the same on both sides
        assert s_in[i] == oracle.insphere(a, b, c, d, e), i
        assert s_in_x[i] == s_in[i], i
        assert s_di[i] == oracle.diametral(a, b, c), i
        if np.linalg.norm(np.cross(b - a, c - a)) > 0:
            eq = oracle.equatorial(a, b, c, d)
            assert s_eq[i] == eq and s_eq_x[i] == eq, i
    assert zeros > 100


def test_splitting_points_bit_identical(cdr):
    rng = np.random.default_rng(102)
    Ps = [rng.uniform(0, 1000, size=(5, 3)) for _ in range(2000)]
    Ps += [rng.uniform(0, 1, size=(5, 3)) * 1e-3 + 500.0 for _ in range(500)]
    it = _items(Ps, B=1.4)
    ok4, c4 = cdr.eval_predicates("tet_cc", it)
    ok3, c3 = cdr.eval_predicates("tri_cc", it)
    _, m2 = cdr.eval_predicates("midpoint", it)
    bad, _ = cdr.eval_predicates("tet_bad", it)
    for i, P in enumerate(Ps):
        cc, ok = oracle.tet_circumcenter(*P[:4])
        assert ok4[i] == ok and np.array_equal(c4[i], cc), i
        cc, ok = oracle.tri_circumcenter(*P[:3])
        assert ok3[i] == ok and np.array_equal(c3[i], cc), i
        assert np.array_equal(m2[i], oracle.midpoint(P[0], P[1])), i
        assert bad[i] == oracle.tet_bad(*P[:4], 1.4), i


# ------------------------------------------------------------------- meshes
def test_create_export_roundtrip(cdr):
    om, e, plc = oracle_case("uniform", 600, 6, 6, 3)
    h = gpu_handle(cdr, e, plc)
    assert_same_mesh(h.export(), om.export(), "create/export")


def test_create_rejects_bad_labels(cdr):
    om, e, plc = oracle_case("cube", 50, 0, 0, 4)
    tris = plc["tris"].copy()
    tris[0] = [0, 7, 3]  # not a face of the mesh
    with pytest.raises(cdr.CdrError):
        cdr.Handle.create(e["xyz"], e["tets"], plc["segs"], plc["seg_id"], tris,
                          plc["facet_id"], plc["nfacets"])
    tets = e["tets"].copy()
    tets[0, [1, 2]] = tets[0, [2, 1]]  # inverted
    with pytest.raises(cdr.CdrError):
        cdr.Handle.create(e["xyz"], tets, plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"])


def _lockstep(cdr, om, h, B, max_rounds, what):
    classes = []
    for r in range(max_rounds):
        g = h.round(B)
        o = om.round(B)
        assert g["cls"] == o["cls"], "%s round %d: class %d vs %d" % (what, r, g["cls"], o["cls"])
        if g["cls"] < 0:
            break
        classes.append(g["cls"])
        compare_reports(h.round_report(), om.report(), "%s round %d" % (what, r))
        assert g["steiner_inserted"] == o["inserted"]
        assert_same_mesh(h.export(), om.export(), "%s round %d" % (what, r))
    return classes


def test_rounds_lockstep_cube(cdr):
    om, e, plc = oracle_case("cube", 300, 0, 0, 0)
    h = gpu_handle(cdr, e, plc)
    classes = _lockstep(cdr, om, h, 2.0, 400, "cube300")
    assert set(classes) == {0, 1, 2}


def test_rounds_lockstep_constrained(cdr):
    # segments and triangles inside the box: every class, every round, to the end
    om, e, plc = oracle_case("uniform", 700, 7, 7, 5)
    h = gpu_handle(cdr, e, plc)
    classes = _lockstep(cdr, om, h, 1.4, 3000, "uniform700")
    assert set(classes) == {0, 1, 2}
    assert h.round(1.4)["cls"] == -1


def test_rounds_lockstep_mixed(cdr):
    """Mixed rounds (every flagged element is a candidate; the class decides
    priority first): same classes, candidates, outcomes and meshes as the
    oracle's mixed mode R, round by round, to the end."""
    om, e, plc = oracle_case("uniform", 700, 7, 7, 5)
    om.set_mixed(True)
    h = gpu_handle(cdr, e, plc, mixed_rounds=True)
    classes = _lockstep(cdr, om, h, 1.4, 3000, "mixed700")
    assert 3 in classes
    assert h.round(1.4)["cls"] == -1


def test_rounds_lockstep_boundary_mixed(cdr):
    """Subsegments and subfaces together, tetrahedra once both are done:
    lockstep with the oracle's mode R to the end."""
    om, e, plc = oracle_case("uniform", 700, 7, 7, 5)
    om.set_mixed(2)
    h = gpu_handle(cdr, e, plc, mixed_rounds=2)
    classes = _lockstep(cdr, om, h, 1.4, 3000, "boundary-mixed700")
    assert 3 in classes and 2 in classes
    assert h.round(1.4)["cls"] == -1


@pytest.mark.parametrize("fused", [-1, 0, 512])
def test_rounds_lockstep_tier2_growth(cdr, fused):
    """Tier-1 workspaces shrunk to 8 cavity tetrahedra and 24 boundary faces, so
    that most regions are re-grown in tier 2 (the separate k_grow2 launch, or
    the fused round's own tier 2, where at fused_max 512 a warp takes several
    candidates and several tier-2 regions in turn): lockstep with mode R to
    the end."""
    om, e, plc = oracle_case("uniform", 700, 7, 7, 5)
    h = gpu_handle(cdr, e, plc)
    h.tune(fused_max=fused, tier1_cavity=8, tier1_boundary=24)
    h.profile(enable=1, reset=True)
    classes = _lockstep(cdr, om, h, 1.4, 3000, "tier2-700")
    assert set(classes) == {0, 1, 2}
    prof = h.profile(enable=0)
    assert prof["counters"]["retried"] > 100
    if fused >= 0:
        assert prof["calls"]["fused"] > 0
    else:
        assert prof["calls"]["grow2"] > 0 and prof["calls"]["fused"] == 0


def test_rounds_lockstep_mixed_stall(cdr):
    """Mixed rounds with dense free segments: the stall rule applies per round
    to the subsegment candidates, identically on both sides."""
    om, e, plc = oracle_case("uniform", 2000, 120, 10, 1)
    om.set_mixed(True)
    h = gpu_handle(cdr, e, plc, mixed_rounds=True)
    _lockstep(cdr, om, h, 1.4, 40, "mixed-stall2000")


def test_results_do_not_depend_on_tuning(cdr):
    """Launch tuning changes speed only: with or without the fused small-round
    kernel, and with other growth grids and tier-2 warp counts, the refined
    mesh is the same."""
    om, e, plc = oracle_case("uniform", 1500, 12, 12, 9)
    ref = None
    for t in [dict(), dict(fused_max=-1), dict(fused_max=16), dict(fused_max=512),
              dict(grow1_blocks_per_sm=2), dict(tier2_warps=2, fused_max=-1)]:
        h = gpu_handle(cdr, e, plc)
        h.tune(**t)
        st = h.refine(1.4)
        ex = h.export()
        h.close()
        if ref is None:
            ref = (ex, st)
        else:
            assert_same_mesh(ex, ref[0], "tuning %s" % t)
            assert st["steiner_inserted"] == ref[1]["steiner_inserted"]
            assert st["rounds"] == ref[1]["rounds"]


def test_rounds_lockstep_subsegment_stall(cdr):
    """Dense free segments: two nearby segments whose midpoints encroach one
    another stall a subsegment round (round 46 here); both implementations give
    the refused candidates up the same way and carry on."""
    om, e, plc = oracle_case("uniform", 2000, 120, 10, 1)
    h = gpu_handle(cdr, e, plc)
    _lockstep(cdr, om, h, 1.4, 60, "stall2000")
    rep = om.report()
    ex = om.export()
    assert (ex["ssflag"] & 2).any()  # some subsegments were given up


def test_refine_cube2k_equals_round_oracle(cdr):
    """The unit-cube workload (2,000 points, B = 2.0) refined to the end on the
    GPU equals the oracle's round-by-round result, and meets the contract."""
    om, e, plc = oracle_case("cube", 2000, 0, 0, 0)
    h = gpu_handle(cdr, e, plc)
    # compact the tetrahedron arrays whenever a tenth of the slots is dead, so
    # that compaction runs (and is checked) inside this refinement
    h.tune(compact_min_tets=1, compact_dead_pct=10)
    h.profile(reset=True)
    st = h.refine(2.0)
    assert st["status"] == 0 and st["n_bad_left"] == 0
    assert h.profile()["counters"]["compactions"] > 0
    so = om.refine_R(2.0)
    assert st["rounds"] == so["rounds"] and st["steiner_inserted"] == so["inserted"]
    ex = h.export()
    assert_same_mesh(ex, om.export(), "cube2k final")
    c = oracle_from_export(ex, plc["nfacets"]).check(2.0)
    for k in ("bad_orient", "nonlocal_delaunay", "sf_not_face", "ss_not_edge",
              "hull_not_subface", "seg_chain_bad", "enc_subsegs", "enc_subfaces", "bad_tets",
              "bad_tets_unspl"):
        assert c[k] == 0, k
    assert abs(c["vol_rel_err"]) < 1e-12 and c["facet_area_rel_err"] < 1e-12 and c["euler"] == 1


def test_delaunay_box_equals_oracle(cdr):
    from paper_1903_03406_gb300 import inputs
    pts, _, _ = inputs.box_points("uniform", 3000, 9)
    h = cdr.Handle.delaunay_box(pts)
    assert h.skipped == 0
    ex = h.export()
    om = oracle.Mesh.box_delaunay(pts)
    oe = om.export()
    a = np.sort(ex["tets"], axis=1)
    b = np.sort(oe["tets"], axis=1)
    assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
    g = oracle.Mesh.create(ex["xyz"], ex["tets"])
    c = g.check(2.0)
    assert c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0 and c["euler"] == 1


def test_checkpoint_restore_replays(cdr):
    om, e, plc = oracle_case("uniform", 600, 6, 6, 11)
    h = gpu_handle(cdr, e, plc)
    for _ in range(20):
        h.round(1.4)
    h.checkpoint()
    h.refine(1.4)
    first = h.export()
    h.restore()
    h.refine(1.4)
    assert_same_mesh(first, h.export(), "restore")


def test_torch_allocator_and_stream(cdr):
    import torch
    om, e, plc = oracle_case("cube", 400, 0, 0, 12)
    s = torch.cuda.Stream()
    al = cdr.TorchAllocator()
    h1 = gpu_handle(cdr, e, plc, allocator=al, stream=s)
    h1.refine(2.0)
    h2 = gpu_handle(cdr, e, plc)
    h2.refine(2.0)
    assert_same_mesh(h1.export(), h2.export(), "torch allocator")


def test_resume_from_exported_mesh_equals_uninterrupted(cdr):
    """A mesh exported between rounds, element flags included, and created
    again (Handle.from_export, cdr_mesh_in's flag arrays) refines to the mesh
    of the uninterrupted run. The stops are chosen where the mode-R run holds
    a must-split subsegment (50 rounds), must-split subfaces and an
    unsplittable tetrahedron (150, 200)."""
    B = 1.5
    om, e, plc = oracle_case("uniform", 150, 3, 3, 41)
    h = gpu_handle(cdr, e, plc)
    h.refine(B)
    final = h.export()
    h.close()
    om.refine_R(B)
    assert_same_mesh(final, om.export(), "uninterrupted")
    seen = np.zeros(3, dtype=bool)
    for k in (50, 150, 200):
        hp = gpu_handle(cdr, e, plc)
        assert hp.refine(B, max_rounds=k)["rounds"] == k
        ex = hp.export()
        hp.close()
        seen |= [bool(ex["tflag"].any()), bool(ex["sfflag"].any()), bool(ex["ssflag"].any())]
        hr = cdr.Handle.from_export(ex)
        hr.refine(B)
        assert_same_mesh(hr.export(), final, "resumed after %d rounds" % k)
        hr.close()
    assert seen.all()
