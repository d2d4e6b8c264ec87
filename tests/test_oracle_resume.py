"""Checkpoint and resume through the exported mesh, on the oracle.

The state of a refinement between rounds is the mesh itself: vertices,
tetrahedra, constraint labels, the per-facet reference points and the element
flags (must split, unsplittable). A mesh exported after k rounds and loaded
into a fresh instance, flags included, refines to the same final mesh as the
uninterrupted run. The GPU tests rely on the same loading (oracle_from_export)
to put a GPU snapshot into the oracle.
"""
import pytest

from _meshes import assert_same_mesh, oracle_from_export, oracle_case

B = 1.5
CASE = ("uniform", 150, 3, 3, 41)


@pytest.fixture(scope="module")
def whole():
    m, _, plc = oracle_case(*CASE[:4], seed=CASE[4])
    m.refine_R(B)
    return m.export(), plc["nfacets"]


@pytest.mark.parametrize("k", [1, 100, 250])
def test_resume_from_export_equals_uninterrupted(whole, k):
    final, nfacets = whole
    part, _, _ = oracle_case(*CASE[:4], seed=CASE[4])
    assert part.refine_R(B, max_rounds=k)["rounds"] == k
    resumed = oracle_from_export(part.export(), nfacets)
    resumed.refine_R(B)
    assert_same_mesh(resumed.export(), final, "resumed after %d rounds" % k)


def test_dropping_the_flags_changes_the_result(whole):
    """The flags are part of the state: resumed without them, the run differs."""
    final, nfacets = whole
    part, _, _ = oracle_case(*CASE[:4], seed=CASE[4])
    for _ in range(10):
        part.refine_R(B, max_rounds=25)
        ex = part.export()
        if ex["sfflag"].any() or ex["ssflag"].any() or ex["tflag"].any():
            break
    else:
        pytest.fail("no flagged element to drop")
    for key in ("tflag", "sfflag", "ssflag"):
        ex[key] = ex[key] * 0
    resumed = oracle_from_export(ex, nfacets)
    resumed.refine_R(B)
    with pytest.raises(AssertionError):
        assert_same_mesh(resumed.export(), final)
