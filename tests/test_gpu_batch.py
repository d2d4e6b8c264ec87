"""Batched refinement (cdr_batch_*): each instance's result is the same alone and
in the mix (needs a GPU).

Instances of different sizes, constraint counts and bounds B are refined alone
(cdr_create + cdr_refine) and together in one batch. The batch must give every
instance the identical mesh: same vertex coordinates in the same order, same
tetrahedra, subfaces and subsegments with the same flags (the tolerance is zero).
That holds whether an instance joins at the start or after other instances
have run rounds, and when it takes the slot of a removed instance. Every
instance's batched result is also compared with the oracle's round-by-round
refinement (mode R) of the same input, so a fault shared by the batched and
the one-mesh paths cannot pass.
"""
import numpy as np
import pytest

from _meshes import assert_same_mesh, oracle_case

pytestmark = pytest.mark.gpu

CASES = [  # (kind, points, segments, triangles, seed, B)
    ("uniform", 400, 4, 4, 11, 1.6),
    ("cube", 250, 0, 0, 12, 2.0),
    ("uniform", 900, 8, 6, 13, 1.4),
    ("clustered", 600, 5, 5, 14, 1.6),
    ("uniform", 300, 3, 3, 15, 2.0),
]


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


@pytest.fixture(scope="module")
def cases():
    out = []
    for kind, n, ns, nt, seed, B in CASES:
        _, e, plc = oracle_case(kind, n, ns, nt, seed)
        out.append((e, plc, B))
    return out


def _oracle_refined(i, mixed=0):
    kind, n, ns, nt, seed, B = CASES[i]
    om, _, _ = oracle_case(kind, n, ns, nt, seed)
    om.set_mixed(mixed)
    so = om.refine_R(B)
    return om.export(), so


@pytest.fixture(scope="module")
def oracle_results():
    return [_oracle_refined(i) for i in range(len(CASES))]


def _args(e, plc):
    return (e["xyz"], e["tets"], plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
            plc["nfacets"])


@pytest.fixture(scope="module")
def alone(cdr, cases):
    res = []
    for e, plc, B in cases:
        h = cdr.Handle.create(*_args(e, plc))
        st = h.refine(B)
        assert st["status"] == 0
        res.append((h.export(), st))
        h.close()
    return res


def test_batch_equals_alone(cdr, cases, alone, oracle_results):
    b = cdr.Batch()
    slots = [b.add(B, *_args(e, plc)) for e, plc, B in cases]
    assert slots == list(range(len(cases)))
    rounds = b.refine()
    assert rounds == max(a[1]["rounds"] for a in alone)
    for k, (ex, st), (oe, so) in zip(slots, alone, oracle_results):
        assert_same_mesh(b.export(k), ex, "instance %d" % k)
        assert_same_mesh(b.export(k), oe, "instance %d against the oracle" % k)
        assert st["steiner_inserted"] == so["inserted"] and st["rounds"] == so["rounds"]
        s = b.stats(k)
        assert s["state"] == "done"
        assert s["steiner_inserted"] == st["steiner_inserted"]
        assert s["rounds"] == st["rounds"]
        assert s["rounds_by_class"] == st["rounds_by_class"]
        assert s["n_bad_left"] == st["n_bad_left"]
        assert s["n_tets"] == len(ex["tets"])
    b.close()


def test_batch_equals_alone_mixed_rounds(cdr, cases):
    """Mixed rounds: every instance takes all its flagged elements each round;
    still the same mesh alone and in the batch."""
    res = []
    for e, plc, B in cases[:3]:
        h = cdr.Handle.create(*_args(e, plc), mixed_rounds=True)
        st = h.refine(B)
        res.append((h.export(), st))
        h.close()
    b = cdr.Batch(mixed_rounds=True)
    slots = [b.add(B, *_args(e, plc)) for e, plc, B in cases[:3]]
    b.refine()
    for k, (ex, st) in zip(slots, res):
        assert_same_mesh(b.export(k), ex, "mixed instance %d" % k)
        oe, so = _oracle_refined(k, mixed=1)
        assert_same_mesh(b.export(k), oe, "mixed instance %d against the oracle" % k)
        assert so["inserted"] == st["steiner_inserted"]
        assert b.stats(k)["steiner_inserted"] == st["steiner_inserted"]
        assert b.stats(k)["rounds"] == st["rounds"]
    b.close()


def test_late_admission_and_slot_reuse(cdr, cases, alone, oracle_results):
    b = cdr.Batch()
    s0 = b.add(cases[0][2], *_args(*cases[0][:2]))
    s1 = b.add(cases[1][2], *_args(*cases[1][:2]))
    for _ in range(7):
        b.round()
    s2 = b.add(cases[2][2], *_args(*cases[2][:2]))  # joins while the others refine
    for _ in range(5):
        b.round()
    b.remove(s1)  # leaves mid-refinement; its slot is reused
    s3 = b.add(cases[3][2], *_args(*cases[3][:2]))
    assert s3 == s1
    b.refine()
    assert_same_mesh(b.export(s0), alone[0][0], "first")
    assert_same_mesh(b.export(s2), alone[2][0], "late")
    assert_same_mesh(b.export(s3), alone[3][0], "reused slot")
    assert_same_mesh(b.export(s2), oracle_results[2][0], "late, against the oracle")
    assert_same_mesh(b.export(s3), oracle_results[3][0], "reused slot, against the oracle")
    assert b.stats(s3)["steiner_inserted"] == alone[3][1]["steiner_inserted"]
    b.close()


def test_batch_rejects_plain_calls_and_bad_slots(cdr, cases):
    b = cdr.Batch()
    e, plc, B = cases[4]
    k = b.add(B, *_args(e, plc))
    with pytest.raises(cdr.CdrError):
        b.export(k + 7)
    with pytest.raises(cdr.CdrError):
        b.add(-1.0, *_args(e, plc))
    # the plain refinement entry point refuses a batch handle
    st = cdr.lib().cdr_refine(b.ptr, 1.6, 10, None)
    assert st == -1
    b.close()
