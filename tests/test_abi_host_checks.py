"""Host-side argument checks of the C-ABI (include/cdr.h, "Errors").

Malformed calls are refused with CDR_ERR_INVALID_INPUT, and oversized
fixed-capacity calls with CDR_ERR_TOO_LARGE, before the library touches the
device, so every case here runs without a GPU. Each malformed input below
changes one thing in a well-formed mesh: the unit cube split
into six tetrahedra around its main diagonal, with its 12 edges as segments and
its 6 square facets as 12 labelled triangles (the input of Sec. 1: a CDT of a
PLC). The binding raises when the library is missing: there is no fallback.
"""
import ctypes

import numpy as np
import pytest

INVALID, TOO_LARGE = -1, -6


@pytest.fixture(scope="module")
def cdr():
    from paper_1903_03406_gb300 import build
    try:
        build.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")
    from paper_1903_03406_gb300 import cdr as binding
    binding.lib()
    return binding


def _cube():
    """The unit cube as a CDT: vertex id = x + 2y + 4z; six tetrahedra around
    the diagonal 0-7, each positively oriented; 12 edges; 6 facets x 2 triangles."""
    xyz = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.float64)
    tets = []
    for p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        b1 = 1 << p[0]
        b2 = b1 | (1 << p[1])
        t = [0, b1, b2, 7]
        u, v, w = (xyz[t[1]] - xyz[t[0]], xyz[t[2]] - xyz[t[0]], xyz[t[3]] - xyz[t[0]])
        if np.dot(u, np.cross(v, w)) < 0:
            t[1], t[2] = t[2], t[1]
        tets.append(t)
    segs = [(a, b) for a in range(8) for b in range(a + 1, 8) if bin(a ^ b).count("1") == 1]
    tris, fid = [], []
    for axis in range(3):
        for side in (0, 1):
            q = sorted(i for i in range(8) if ((i >> axis) & 1) == side)
            tris += [(q[0], q[1], q[3]), (q[0], q[3], q[2])]
            fid += [len(fid) // 2] * 2
    return dict(xyz=xyz, tets=np.array(tets, dtype=np.int32),
                segs=np.array(segs, dtype=np.int32), seg_id=np.arange(12, dtype=np.int32),
                tris=np.array(tris, dtype=np.int32), facet_id=np.array(fid, dtype=np.int32),
                n_facets=6)


def test_cube_fixture_is_a_valid_cdt():
    m = _cube()
    vol = 0.0
    for t in m["tets"]:
        a, b, c, d = m["xyz"][t]
        det = np.dot(b - a, np.cross(c - a, d - a))
        assert det > 0
        vol += det / 6
    assert vol == pytest.approx(1.0, rel=1e-15)
    assert m["segs"].shape == (12, 2) and m["tris"].shape == (12, 3)
    assert sorted(np.bincount(m["facet_id"])) == [2] * 6


def _malformed():
    """(name, mesh) pairs, each failing a host check of cdr_create."""
    out = []

    def variant(name, **change):
        m = _cube()
        for k, v in change.items():
            m[k] = v(m[k]) if callable(v) else v
        out.append((name, m))

    def poke(arr, idx, val):
        arr = arr.copy()
        arr[idx] = val
        return arr

    variant("tet index past the last vertex", tets=lambda t: poke(t, (2, 1), 8))
    variant("negative tet index", tets=lambda t: poke(t, (0, 0), -1))
    variant("segment end past the last vertex", segs=lambda s: poke(s, (5, 1), 99))
    variant("triangle vertex negative", tris=lambda s: poke(s, (3, 2), -4))
    variant("facet label past n_facets", facet_id=lambda f: poke(f, 7, 6))
    variant("negative facet label", facet_id=lambda f: poke(f, 0, -1))
    variant("NaN coordinate", xyz=lambda x: poke(x, (3, 1), np.nan))
    variant("infinite coordinate", xyz=lambda x: poke(x, (6, 2), np.inf))
    variant("fewer than four vertices", xyz=lambda x: x[:3],
            tets=np.zeros((1, 4), dtype=np.int32))
    variant("no tetrahedra", tets=np.zeros((0, 4), dtype=np.int32))
    return out


@pytest.mark.parametrize("name,mesh", _malformed(), ids=[n for n, _ in _malformed()])
def test_create_refuses_malformed_mesh_on_the_host(cdr, name, mesh):
    with pytest.raises(cdr.CdrError) as e:
        cdr.Handle.create(mesh["xyz"], mesh["tets"], mesh["segs"], mesh["seg_id"],
                          mesh["tris"], mesh["facet_id"], mesh["n_facets"])
    assert e.value.status == INVALID, name


@pytest.mark.parametrize("name,flags", [
    ("tetrahedron flag with the must-split bit", (np.array([0, 0, 1, 0, 0, 0], np.uint8), None,
                                                   None)),
    ("tetrahedron flag past bit1", (np.array([0, 4, 0, 0, 0, 0], np.uint8), None, None)),
    ("subface flag past bit1", (None, np.eye(1, 12, 5, dtype=np.uint8).ravel() * 8, None)),
    ("subsegment flag past bit1", (None, None, np.full(12, 0x80, np.uint8))),
])
def test_create_refuses_unknown_element_flags_on_the_host(cdr, name, flags):
    """Element flags (a mesh exported between rounds) carry only the export's
    bits: tetrahedra bit1, subfaces and subsegments bits 0 and 1."""
    m = _cube()
    with pytest.raises(cdr.CdrError) as e:
        cdr.Handle.create(m["xyz"], m["tets"], m["segs"], m["seg_id"], m["tris"],
                          m["facet_id"], m["n_facets"], flags=flags)
    assert e.value.status == INVALID, name


def test_from_export_passes_labels_references_and_flags(cdr):
    """Handle.from_export reads an export()-shaped dict: subsegments (a, b, id),
    subfaces (a, b, c, facet), facet references and the three flag arrays; a
    flag bit the export never writes is refused on the host, so the flags do
    reach cdr_create."""
    m = _cube()
    ex = dict(xyz=m["xyz"], tets=m["tets"], tflag=np.zeros(6, np.uint8),
              sf=np.concatenate([m["tris"], m["facet_id"][:, None]], axis=1),
              sfflag=np.zeros(12, np.uint8),
              ss=np.concatenate([m["segs"], m["seg_id"][:, None]], axis=1),
              ssflag=np.zeros(12, np.uint8), facetq=np.zeros((6, 3)))
    for key, n in (("tflag", 6), ("sfflag", 12), ("ssflag", 12)):
        bad = dict(ex)
        bad[key] = np.full(n, 0x10, np.uint8)
        with pytest.raises(cdr.CdrError) as e:
            cdr.Handle.from_export(bad)
        assert e.value.status == INVALID, key


def test_flag_arrays_must_match_their_elements(cdr):
    m = _cube()
    with pytest.raises(ValueError):
        cdr.Handle.create(m["xyz"], m["tets"], m["segs"], m["seg_id"], m["tris"],
                          m["facet_id"], m["n_facets"], flags=(np.zeros(5, np.uint8), None, None))


def _box_points(extra):
    corners = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.float64)
    return np.vstack([corners, np.asarray(extra, dtype=np.float64).reshape(-1, 3)])


@pytest.mark.parametrize("name,xyz", [
    ("fewer than eight points", _box_points([])[:7]),
    ("a non-corner point on a box face", _box_points([[0.5, 0.5, 1.0]])),
    ("a missing corner", np.vstack([_box_points([])[:7], [[0.5, 0.5, 0.5]]])),
    ("NaN coordinate", _box_points([[0.25, np.nan, 0.5]])),
])
def test_delaunay_box_refuses_bad_point_sets_on_the_host(cdr, name, xyz):
    with pytest.raises(cdr.CdrError) as e:
        cdr.Handle.delaunay_box(xyz)
    assert e.value.status == INVALID, name


def test_predicate_batches_check_kind_and_size_on_the_host(cdr):
    L = cdr.lib()
    buf = np.zeros(16)
    sign = np.zeros(1, dtype=np.int32)
    dp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ip = sign.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for call in (L.cdr_eval_predicates, L.cdr_eval_predicates_noalloc):
        assert call(12, dp, 1, ip, None, None) == INVALID
        assert call(-1, dp, 1, ip, None, None) == INVALID
        assert call(0, dp, -1, ip, None, None) == INVALID
        assert call(0, None, 1, ip, None, None) == INVALID
        assert call(0, dp, 1, None, None, None) == INVALID
        assert call(0, dp, 0, ip, None, None) == 0  # empty batch: no device work
    # one item over the fixed array's capacity is refused before any copy
    with pytest.raises(cdr.CdrError) as e:
        cdr.eval_predicates_noalloc("orient", np.zeros((cdr.EVAL_NOALLOC_MAX_ITEMS + 1, 16)))
    assert e.value.status == TOO_LARGE


def test_calls_on_a_null_handle_are_refused(cdr):
    L = cdr.lib()
    s = cdr.Stats()
    c = ctypes.c_int32(0)
    assert L.cdr_refine(None, 2.0, 10, ctypes.byref(s)) == INVALID
    assert L.cdr_round(None, 2.0, ctypes.byref(c), ctypes.byref(s)) == INVALID
    assert L.cdr_export_sizes(None, ctypes.byref(cdr.Sizes())) == INVALID
    assert L.cdr_checkpoint(None) == INVALID
    assert L.cdr_restore(None) == INVALID
    assert L.cdr_batch_round(None, ctypes.byref(c)) == INVALID
    assert L.cdr_batch_refine(None, 10, ctypes.byref(c)) == INVALID
    assert L.cdr_batch_remove(None, 0) == INVALID
    assert L.cdr_set_tuning(None, ctypes.byref(cdr.Tuning(0, 0, 0))) == INVALID
    L.cdr_destroy(None)  # ignored


def test_binding_raises_when_the_library_is_missing(cdr, monkeypatch, tmp_path):
    monkeypatch.setattr(cdr, "_lib", None)
    monkeypatch.setattr(cdr, "LIB_PATH", str(tmp_path / "libcdr.so"))
    with pytest.raises(RuntimeError, match="not built"):
        cdr.lib()
    with pytest.raises(RuntimeError):
        cdr.Handle.create(*[_cube()[k] for k in ("xyz", "tets", "segs", "seg_id", "tris",
                                                 "facet_id", "n_facets")])


class _RefusingAllocator:
    """A cdr_allocator whose alloc always fails (returns NULL); counts calls."""

    def __init__(self, cdr):
        self.allocs = 0
        self.frees = 0
        self._a = cdr.ALLOC_FN(self._alloc)
        self._f = cdr.FREE_FN(self._free)
        self.struct = cdr.Allocator(self._a, self._f, None)

    def _alloc(self, nbytes, ctx, stream):
        self.allocs += 1
        return None

    def _free(self, ptr, nbytes, ctx, stream):
        self.frees += 1


def test_failing_allocator_gives_out_of_memory(cdr):
    """A caller's allocator that has no memory left: creation stops at the first
    request with CDR_ERR_OOM, frees nothing it did not get and leaves no handle
    (the device is never reached, so this runs without a GPU)."""
    m = _cube()
    al = _RefusingAllocator(cdr)
    with pytest.raises(cdr.CdrError) as e:
        cdr.Handle.create(m["xyz"], m["tets"], m["segs"], m["seg_id"], m["tris"],
                          m["facet_id"], m["n_facets"], allocator=al)
    assert e.value.status == -2
    assert al.allocs == 1 and al.frees == 0
    al2 = _RefusingAllocator(cdr)
    with pytest.raises(cdr.CdrError) as e:
        cdr.Batch(allocator=al2)
    assert e.value.status == -2
    assert al2.allocs == 1 and al2.frees == 0
