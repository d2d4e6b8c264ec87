"""Python binding of the C-ABI in include/cdr.h (argument marshalling only).

Every step of the refinement runs inside libcdr.so on the GPU. There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.

Names follow the C calls: Handle.create (cdr_create), Handle.refine
(cdr_refine), Handle.round (cdr_round), Handle.export (cdr_export_sizes +
cdr_export), Handle.round_report (cdr_round_report), Handle.checkpoint /
restore, Handle.delaunay_box (cdr_delaunay_box).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdr.so")
_lock = threading.Lock()
_lib = None

CDR_OK, CDR_ROUND_LIMIT = 0, 1


class CdrError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, status_string(status), status))


class MeshIn(ctypes.Structure):
    _fields_ = [("xyz", ctypes.POINTER(ctypes.c_double)), ("n_verts", ctypes.c_int32),
                ("tets", ctypes.POINTER(ctypes.c_int32)), ("n_tets", ctypes.c_int32),
                ("segs", ctypes.POINTER(ctypes.c_int32)), ("seg_id", ctypes.POINTER(ctypes.c_int32)),
                ("n_segs", ctypes.c_int32), ("tris", ctypes.POINTER(ctypes.c_int32)),
                ("facet_id", ctypes.POINTER(ctypes.c_int32)), ("n_tris", ctypes.c_int32),
                ("n_facets", ctypes.c_int32), ("facet_ref", ctypes.POINTER(ctypes.c_double)),
                ("tet_flag", ctypes.POINTER(ctypes.c_uint8)),
                ("subface_flag", ctypes.POINTER(ctypes.c_uint8)),
                ("subseg_flag", ctypes.POINTER(ctypes.c_uint8))]


class Options(ctypes.Structure):
    _fields_ = [("guard2", ctypes.c_double), ("walk_limit", ctypes.c_int32),
                ("reserve_factor", ctypes.c_int32), ("mixed_rounds", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("rounds_by_class", ctypes.c_int32 * 3),
                ("candidates", ctypes.c_int64), ("steiner_inserted", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("blasted", ctypes.c_int64),
                ("unsplittable", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("n_tets", ctypes.c_int64), ("n_subfaces", ctypes.c_int64),
                ("n_subsegs", ctypes.c_int64), ("n_bad_left", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["rounds_by_class"] = list(self.rounds_by_class)
        return d


class Tuning(ctypes.Structure):
    _fields_ = [("fused_max", ctypes.c_int32), ("grow1_blocks_per_sm", ctypes.c_int32),
                ("tier2_warps", ctypes.c_int32), ("tier1_cavity", ctypes.c_int32),
                ("tier1_boundary", ctypes.c_int32), ("compact_min_tets", ctypes.c_int32),
                ("compact_dead_pct", ctypes.c_int32)]


class Sizes(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int32), ("n_tets", ctypes.c_int32),
                ("n_subfaces", ctypes.c_int32), ("n_subsegs", ctypes.c_int32),
                ("n_facets", ctypes.c_int32)]


class MeshOut(ctypes.Structure):
    _fields_ = [("xyz", ctypes.POINTER(ctypes.c_double)), ("tets", ctypes.POINTER(ctypes.c_int32)),
                ("tet_flag", ctypes.POINTER(ctypes.c_uint8)),
                ("subfaces", ctypes.POINTER(ctypes.c_int32)),
                ("subface_flag", ctypes.POINTER(ctypes.c_uint8)),
                ("subsegs", ctypes.POINTER(ctypes.c_int32)),
                ("subseg_flag", ctypes.POINTER(ctypes.c_uint8)),
                ("facet_ref", ctypes.POINTER(ctypes.c_double))]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


def lib():
    """Load libcdr.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libcdr.so is not built; run "
                                   "python -c 'import __graft_entry__ as g; g.build()'")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.c_void_p
            pp = ctypes.POINTER(ctypes.c_void_p)
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.cdr_create.argtypes = [ctypes.POINTER(MeshIn), ctypes.POINTER(Options),
                                     ctypes.POINTER(Allocator), P, pp]
            L.cdr_refine.argtypes = [P, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(Stats)]
            L.cdr_round.argtypes = [P, ctypes.c_double, i32p, ctypes.POINTER(Stats)]
            L.cdr_export_sizes.argtypes = [P, ctypes.POINTER(Sizes)]
            L.cdr_export.argtypes = [P, ctypes.POINTER(MeshOut)]
            L.cdr_round_report.argtypes = [P, i32p, ctypes.POINTER(ctypes.c_int64), i32p,
                                           ctypes.POINTER(ctypes.c_double), i32p, i32p, i32p,
                                           i32p, i32p, i32p, i32p]
            L.cdr_checkpoint.argtypes = [P]
            L.cdr_restore.argtypes = [P]
            L.cdr_destroy.argtypes = [P]
            L.cdr_destroy.restype = None
            L.cdr_delaunay_box.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                           ctypes.POINTER(Options), ctypes.POINTER(Allocator), P,
                                           pp, i32p, i32p]
            L.cdr_status_string.argtypes = [ctypes.c_int]
            L.cdr_status_string.restype = ctypes.c_char_p
            L.cdr_device_arch.restype = ctypes.c_int
            L.cdr_profile.argtypes = [P, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]
            L.cdr_eval_predicates.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_int32, i32p,
                                              ctypes.POINTER(ctypes.c_double), P]
            L.cdr_eval_predicates_noalloc.argtypes = L.cdr_eval_predicates.argtypes
            L.cdr_batch_create.argtypes = [ctypes.POINTER(Options), ctypes.POINTER(Allocator), P,
                                           pp]
            L.cdr_batch_add.argtypes = [P, ctypes.POINTER(MeshIn), ctypes.c_double, i32p]
            L.cdr_batch_round.argtypes = [P, i32p]
            L.cdr_batch_refine.argtypes = [P, ctypes.c_int32, i32p]
            L.cdr_batch_stats.argtypes = [P, ctypes.c_int32, ctypes.POINTER(Stats), i32p]
            L.cdr_batch_export_sizes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(Sizes)]
            L.cdr_batch_export.argtypes = [P, ctypes.c_int32, ctypes.POINTER(MeshOut)]
            L.cdr_batch_remove.argtypes = [P, ctypes.c_int32]
            L.cdr_batch_finished.argtypes = [P, i32p, ctypes.c_int32, i32p]
            L.cdr_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
            _lib = L
    return _lib


def status_string(s):
    try:
        return lib().cdr_status_string(int(s)).decode()
    except Exception:  # the library itself is missing
        return "status %d" % s


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def _check(st, what, ok=(0,)):
    if st not in ok:
        raise CdrError(st, what)
    return st


class TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)
        self.struct = Allocator(self._alloc, self._free, None)

    def _a(self, nbytes, ctx, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
        except Exception:
            return None

    def _f(self, ptr, nbytes, ctx, stream):
        try:
            self.torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def set_tuning(ptr, fused_max=0, grow1_blocks_per_sm=0, tier2_warps=0, tier1_cavity=0,
               tier1_boundary=0, compact_min_tets=0, compact_dead_pct=0):
    """Launch tuning of a handle or batch (cdr_set_tuning); results do not depend on it."""
    t = Tuning(int(fused_max), int(grow1_blocks_per_sm), int(tier2_warps), int(tier1_cavity),
               int(tier1_boundary), int(compact_min_tets), int(compact_dead_pct))
    _check(lib().cdr_set_tuning(ptr, ctypes.byref(t)), "cdr_set_tuning")


def _mesh_in(xyz, tets, segs, seg_id, tris, facet_id, n_facets, facet_ref=None, flags=None):
    """A cdr_mesh_in over contiguous copies (returned too, to keep them alive).
    flags: optional (tet_flag, subface_flag, subseg_flag), any entry None."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    segs = np.ascontiguousarray(segs, dtype=np.int32).reshape(-1, 2)
    seg_id = np.ascontiguousarray(seg_id, dtype=np.int32).reshape(-1)
    tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    facet_id = np.ascontiguousarray(facet_id, dtype=np.int32).reshape(-1)
    fr = None
    if facet_ref is not None:
        fr = np.ascontiguousarray(facet_ref, dtype=np.float64).reshape(-1, 3)
    fl = [None if f is None else np.ascontiguousarray(f, dtype=np.uint8).reshape(-1)
          for f in (flags or (None, None, None))]
    for f, n in zip(fl, (len(tets), len(tris), len(segs))):
        if f is not None and len(f) != n:
            raise ValueError("a flag array does not match its elements")
    mi = MeshIn(_p(xyz, ctypes.c_double), len(xyz), _p(tets, ctypes.c_int32), len(tets),
                _p(segs, ctypes.c_int32), _p(seg_id, ctypes.c_int32), len(segs),
                _p(tris, ctypes.c_int32), _p(facet_id, ctypes.c_int32), len(tris),
                int(n_facets), _p(fr, ctypes.c_double), *[_p(f, ctypes.c_uint8) for f in fl])
    return mi, (xyz, tets, segs, seg_id, tris, facet_id, fr) + tuple(fl)


def _export(s, call, what):
    """Buffers sized from s, filled by call(cdr_mesh_out)."""
    xyz = np.zeros((s["nv"], 3))
    tets = np.zeros((s["nt"], 4), dtype=np.int32)
    tflag = np.zeros(s["nt"], dtype=np.uint8)
    sf = np.zeros((s["ns"], 4), dtype=np.int32)
    sfflag = np.zeros(s["ns"], dtype=np.uint8)
    ss = np.zeros((s["ng"], 3), dtype=np.int32)
    ssflag = np.zeros(s["ng"], dtype=np.uint8)
    fq = np.zeros((max(s["nfacets"], 1), 3))
    mo = MeshOut(_p(xyz, ctypes.c_double), _p(tets, ctypes.c_int32), _p(tflag, ctypes.c_uint8),
                 _p(sf, ctypes.c_int32), _p(sfflag, ctypes.c_uint8), _p(ss, ctypes.c_int32),
                 _p(ssflag, ctypes.c_uint8), _p(fq, ctypes.c_double))
    _check(call(mo), what)
    return dict(xyz=xyz, tets=tets, tflag=tflag, sf=sf, sfflag=sfflag, ss=ss, ssflag=ssflag,
                facetq=fq[: s["nfacets"]])


class Handle:
    """A refinement handle (cdr_handle) owning its device mesh."""

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        p = getattr(self, "ptr", None)
        if p:
            lib().cdr_destroy(p)
            self.ptr = None

    # -------------------------------------------------------------- creation
    @classmethod
    def create(cls, xyz, tets, segs, seg_id, tris, facet_id, n_facets, facet_ref=None,
               guard2=0.0, walk_limit=0, reserve_factor=0, mixed_rounds=False, allocator=None,
               stream=None, flags=None):
        mi, _arrays = _mesh_in(xyz, tets, segs, seg_id, tris, facet_id, n_facets, facet_ref,
                               flags)
        opt = Options(float(guard2), int(walk_limit), int(reserve_factor), int(mixed_rounds))
        out = ctypes.c_void_p()
        al = ctypes.byref(allocator.struct) if allocator is not None else None
        st = lib().cdr_create(ctypes.byref(mi), ctypes.byref(opt), al, _stream_handle(stream),
                              ctypes.byref(out))
        _check(st, "cdr_create")
        return cls(out, keep=(allocator,))

    @classmethod
    def from_export(cls, ex, **kw):
        """A handle from a mesh exported between rounds (export()'s dict): its
        labels, facet reference points and element flags, so that the
        refinement goes on as if it had not been interrupted (a host-side
        checkpoint). Keyword arguments as for create."""
        sf, ss = ex["sf"], ex["ss"]
        return cls.create(ex["xyz"], ex["tets"], ss[:, :2], ss[:, 2], sf[:, :3], sf[:, 3],
                          len(ex["facetq"]), facet_ref=ex["facetq"],
                          flags=(ex["tflag"], ex["sfflag"], ex["ssflag"]), **kw)

    @classmethod
    def delaunay_box(cls, xyz, walk_limit=0, allocator=None, stream=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        opt = Options(0.0, int(walk_limit), 0, 0)
        out = ctypes.c_void_p()
        sk, rd = ctypes.c_int32(0), ctypes.c_int32(0)
        al = ctypes.byref(allocator.struct) if allocator is not None else None
        st = lib().cdr_delaunay_box(_p(xyz, ctypes.c_double), len(xyz), ctypes.byref(opt), al,
                                    _stream_handle(stream), ctypes.byref(out), ctypes.byref(sk),
                                    ctypes.byref(rd))
        _check(st, "cdr_delaunay_box")
        h = cls(out, keep=(allocator,))
        h.skipped = sk.value
        h.dt_rounds = rd.value
        return h

    # ------------------------------------------------------------ refinement
    def refine(self, B, max_rounds=1 << 30):
        s = Stats()
        st = lib().cdr_refine(self.ptr, float(B), int(min(max_rounds, 2**31 - 1)), ctypes.byref(s))
        _check(st, "cdr_refine", ok=(CDR_OK, CDR_ROUND_LIMIT))
        d = s.as_dict()
        d["status"] = st
        return d

    def round(self, B):
        s = Stats()
        cls_ = ctypes.c_int32(-1)
        st = lib().cdr_round(self.ptr, float(B), ctypes.byref(cls_), ctypes.byref(s))
        _check(st, "cdr_round")
        d = s.as_dict()
        d["cls"] = cls_.value
        return d

    GROUPS = ["classify", "order", "split", "locate", "grow1", "grow2", "select", "scan",
              "insert", "compact", "fused"]
    COUNTERS = ["refused", "unsplittable", "blasted", "inserted", "retried", "invariant",
                "tested", "cavity", "boundary", "new_tets", "new_candidates", "blasted_early",
                "dead_tets", "compactions", "c14", "launches", "fused_tested", "fused_cavity",
                "fused_boundary"]

    def profile(self, enable=-1, reset=False):
        ms = np.zeros(32)
        calls = np.zeros(32, dtype=np.int64)
        ctr = np.zeros(32, dtype=np.int64)
        _check(lib().cdr_profile(self.ptr, int(enable), int(bool(reset)), _p(ms, ctypes.c_double),
                                 _p(calls, ctypes.c_int64), _p(ctr, ctypes.c_int64)),
               "cdr_profile")
        return dict(ms={g: float(ms[i]) for i, g in enumerate(self.GROUPS)},
                    calls={g: int(calls[i]) for i, g in enumerate(self.GROUPS)},
                    counters={c: int(ctr[i]) for i, c in enumerate(self.COUNTERS)})

    def tune(self, **kw):
        set_tuning(self.ptr, **kw)

    def checkpoint(self):
        _check(lib().cdr_checkpoint(self.ptr), "cdr_checkpoint")

    def restore(self):
        _check(lib().cdr_restore(self.ptr), "cdr_restore")

    # ---------------------------------------------------------------- export
    def sizes(self):
        s = Sizes()
        _check(lib().cdr_export_sizes(self.ptr, ctypes.byref(s)), "cdr_export_sizes")
        return dict(nv=s.n_verts, nt=s.n_tets, ns=s.n_subfaces, ng=s.n_subsegs,
                    nfacets=s.n_facets)

    def export(self):
        return _export(self.sizes(), lambda mo: lib().cdr_export(self.ptr, ctypes.byref(mo)),
                       "cdr_export")

    def round_report(self):
        n = ctypes.c_int32(0)
        tot = ctypes.c_int64(0)
        L = lib()
        _check(L.cdr_round_report(self.ptr, ctypes.byref(n), ctypes.byref(tot), None, None, None,
                                  None, None, None, None, None, None), "cdr_round_report")
        n = n.value
        keys = np.zeros((n, 4), dtype=np.int32)
        pts = np.zeros((n, 3))
        outcome, reason, surv, ncav, nbnd, nfcav = (np.zeros(n, dtype=np.int32) for _ in range(6))
        cav = np.zeros((max(tot.value, 1), 4), dtype=np.int32)
        n2 = ctypes.c_int32(0)
        _check(L.cdr_round_report(self.ptr, ctypes.byref(n2), ctypes.byref(tot),
                                  _p(keys, ctypes.c_int32), _p(pts, ctypes.c_double),
                                  _p(outcome, ctypes.c_int32), _p(reason, ctypes.c_int32),
                                  _p(surv, ctypes.c_int32), _p(ncav, ctypes.c_int32),
                                  _p(nbnd, ctypes.c_int32), _p(nfcav, ctypes.c_int32),
                                  _p(cav, ctypes.c_int32)), "cdr_round_report")
        return dict(keys=keys, pts=pts, outcome=outcome, reason=reason, surv=surv, ncav=ncav,
                    nbnd=nbnd, nfcav=nfcav, cav=cav[: tot.value])


class Batch:
    """Many instances refined together in one device-resident mesh
    (cdr_batch_*): every round runs each kernel once over all instances."""

    STATE = {0: "free", 1: "refining", 2: "done"}

    def __init__(self, guard2=0.0, walk_limit=0, mixed_rounds=False, allocator=None, stream=None):
        opt = Options(float(guard2), int(walk_limit), 0, int(mixed_rounds))
        out = ctypes.c_void_p()
        al = ctypes.byref(allocator.struct) if allocator is not None else None
        _check(lib().cdr_batch_create(ctypes.byref(opt), al, _stream_handle(stream),
                                      ctypes.byref(out)), "cdr_batch_create")
        self.ptr = out
        self._keep = (allocator,)

    def __del__(self):
        self.close()

    def close(self):
        p = getattr(self, "ptr", None)
        if p:
            lib().cdr_destroy(p)
            self.ptr = None

    def add(self, B, xyz, tets, segs, seg_id, tris, facet_id, n_facets, facet_ref=None):
        mi, _arrays = _mesh_in(xyz, tets, segs, seg_id, tris, facet_id, n_facets, facet_ref)
        slot = ctypes.c_int32(-1)
        _check(lib().cdr_batch_add(self.ptr, ctypes.byref(mi), float(B), ctypes.byref(slot)),
               "cdr_batch_add")
        return slot.value

    def round(self):
        n = ctypes.c_int32(0)
        _check(lib().cdr_batch_round(self.ptr, ctypes.byref(n)), "cdr_batch_round")
        return n.value

    def refine(self, max_rounds=1 << 30):
        r = ctypes.c_int32(0)
        st = lib().cdr_batch_refine(self.ptr, int(min(max_rounds, 2**31 - 1)), ctypes.byref(r))
        _check(st, "cdr_batch_refine", ok=(CDR_OK, CDR_ROUND_LIMIT))
        return r.value

    def stats(self, slot):
        s = Stats()
        state = ctypes.c_int32(0)
        _check(lib().cdr_batch_stats(self.ptr, int(slot), ctypes.byref(s), ctypes.byref(state)),
               "cdr_batch_stats")
        d = s.as_dict()
        d["state"] = self.STATE.get(state.value, state.value)
        return d

    def sizes(self, slot):
        s = Sizes()
        _check(lib().cdr_batch_export_sizes(self.ptr, int(slot), ctypes.byref(s)),
               "cdr_batch_export_sizes")
        return dict(nv=s.n_verts, nt=s.n_tets, ns=s.n_subfaces, ng=s.n_subsegs,
                    nfacets=s.n_facets)

    def export(self, slot):
        return _export(self.sizes(slot),
                       lambda mo: lib().cdr_batch_export(self.ptr, int(slot), ctypes.byref(mo)),
                       "cdr_batch_export")

    def remove(self, slot):
        _check(lib().cdr_batch_remove(self.ptr, int(slot)), "cdr_batch_remove")

    def tune(self, **kw):
        set_tuning(self.ptr, **kw)

    def finished(self):
        """Slots whose instance has finished refining."""
        n = ctypes.c_int32(0)
        _check(lib().cdr_batch_finished(self.ptr, None, 0, ctypes.byref(n)), "cdr_batch_finished")
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        _check(lib().cdr_batch_finished(self.ptr, _p(out, ctypes.c_int32), len(out),
                                        ctypes.byref(n)), "cdr_batch_finished")
        return [int(x) for x in out[: n.value]]


def device_arch():
    return lib().cdr_device_arch()


PRED = dict(orient=0, insphere=1, diametral=2, equatorial=3, tet_cc=4, tri_cc=5, midpoint=6,
            tet_bad=7, orient_exact=8, insphere_exact=9, equatorial_exact=10, diametral_exact=11)


def eval_predicates(kind, items, stream=None):
    """items: (n, 16) float64 (see cdr_eval_predicates). Returns (sign, points)."""
    items = np.ascontiguousarray(items, dtype=np.float64).reshape(-1, 16)
    n = len(items)
    sign = np.zeros(n, dtype=np.int32)
    out = np.zeros((n, 3))
    k = PRED[kind] if isinstance(kind, str) else int(kind)
    _check(lib().cdr_eval_predicates(k, _p(items, ctypes.c_double), n, _p(sign, ctypes.c_int32),
                                     _p(out, ctypes.c_double), _stream_handle(stream)),
           "cdr_eval_predicates")
    return sign, out


# largest batch of eval_predicates_noalloc (CDR_EVAL_NOALLOC_MAX_ITEMS in cdr.h)
EVAL_NOALLOC_MAX_ITEMS = 16384


def eval_predicates_noalloc(kind, items, stream=None):
    """eval_predicates without device allocation (cdr_eval_predicates_noalloc).

    For callers that cannot allocate device memory: code that keeps kernels
    running on other streams (cudaFree would wait for the whole device) and
    processes whose device memory is held by a caching allocator (cudaMalloc can
    fail there). The device copies live in a fixed array of the library, so at
    most EVAL_NOALLOC_MAX_ITEMS items go in one call, and calls whose device work
    overlaps (other streams or threads) race. Each call looks that array up on
    the current device and synchronises its stream, so it cannot run on a
    stream under graph capture. Host buffers only (numpy).
    """
    items = np.ascontiguousarray(items, dtype=np.float64).reshape(-1, 16)
    n = len(items)
    sign = np.zeros(n, dtype=np.int32)
    out = np.zeros((n, 3))
    k = PRED[kind] if isinstance(kind, str) else int(kind)
    st = lib().cdr_eval_predicates_noalloc(k, _p(items, ctypes.c_double), n,
                                           _p(sign, ctypes.c_int32), _p(out, ctypes.c_double),
                                           _stream_handle(stream))
    if st == -6:
        raise CdrError(st, "cdr_eval_predicates_noalloc: %d items, at most %d fit its fixed "
                       "device scratch" % (n, EVAL_NOALLOC_MAX_ITEMS))
    _check(st, "cdr_eval_predicates_noalloc")
    return sign, out
