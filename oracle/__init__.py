"""CPU oracle for the refinement step: a plain, slow, sequential restatement of the
method, used ONLY by the test suite, the smoke check and the benchmark's CPU
baseline leg. The product path (the CUDA library and its binding) never imports
this package.

The C++ sources in this directory share no code with the CUDA library. They are
built with ``-ffp-contract=off`` so that every FP64 formula is evaluated with one
IEEE rounding per operation, in the order written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["refine.cpp", "capi.cpp"]
_HEADERS = ["geom.hpp", "mesh.hpp", "oracle.hpp"]
_lock = threading.Lock()
_lib = None

CLS_SUBSEG, CLS_SUBFACE, CLS_TET, CLS_POINT = 0, 1, 2, 3
OUT_OK, OUT_REJECT, OUT_UNSPL, OUT_BLASTED = 0, 1, 2, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (g++, C++17, -O3, no FP contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, h) for h in _HEADERS]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_long)
            u8 = ctypes.POINTER(ctypes.c_uint8)
            for n in ["orc_orient3d", "orc_orient3d_exact", "orc_diametral"]:
                pass
            L.orc_orient3d.argtypes = [dp] * 4
            L.orc_orient3d_exact.argtypes = [dp] * 4
            L.orc_insphere.argtypes = [dp] * 5
            L.orc_insphere_exact.argtypes = [dp] * 5
            L.orc_diametral.argtypes = [dp] * 3
            L.orc_equatorial.argtypes = [dp] * 4
            L.orc_tet_cc.argtypes = [dp] * 5
            L.orc_tri_cc.argtypes = [dp] * 4
            L.orc_midpoint.argtypes = [dp] * 3
            L.orc_midpoint.restype = None
            L.orc_tet_bad.argtypes = [dp] * 4 + [ctypes.c_double]
            L.orc_prio_hash.argtypes = [ctypes.c_int, ip, ctypes.c_int]
            L.orc_prio_hash.restype = ctypes.c_uint64
            L.orc_prio_hash_xyz.argtypes = [ctypes.c_int, dp, ctypes.c_int]
            L.orc_set_mixed.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_set_mixed.restype = None
            L.orc_prio_hash_xyz.restype = ctypes.c_uint64
            L.orc_box_delaunay.argtypes = [dp, ctypes.c_int, ip]
            L.orc_box_delaunay.restype = P
            L.orc_insert_points.argtypes = [P, dp, ctypes.c_int]
            L.orc_insert_points.restype = ctypes.c_int
            L.orc_create.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int]
            L.orc_create.restype = P
            L.orc_free.argtypes = [P]
            L.orc_free.restype = None
            L.orc_set_constraints.argtypes = [P, ip, ip, ctypes.c_int, ip, ip, ctypes.c_int, dp,
                                              ctypes.c_int, ctypes.c_double]
            L.orc_set_limits.argtypes = [P, ctypes.c_int, ctypes.c_int]
            L.orc_set_limits.restype = None
            L.orc_set_flags.argtypes = [P, u8, u8, u8]
            L.orc_set_flags.restype = None
            L.orc_round.argtypes = [P, ctypes.c_double, ip]
            L.orc_refine_R.argtypes = [P, ctypes.c_double, ctypes.c_int, lp]
            L.orc_refine_S.argtypes = [P, ctypes.c_double, ctypes.c_long, lp]
            L.orc_refine_S.restype = ctypes.c_long
            L.orc_sizes.argtypes = [P, ip]
            L.orc_sizes.restype = None
            L.orc_export.argtypes = [P, dp, ip, u8, ip, u8, ip, u8, dp]
            L.orc_export.restype = None
            L.orc_guard2.argtypes = [P]
            L.orc_guard2.restype = ctypes.c_double
            L.orc_report_sizes.argtypes = [P, ip]
            L.orc_report_sizes.restype = None
            L.orc_report.argtypes = [P, ip, dp, ip, ip, ip, ip, ip, ip, ip, ip, ip, ip, ip, ip]
            L.orc_report.restype = None
            L.orc_report_claim_sizes.argtypes = [P, ip]
            L.orc_report_claim_sizes.restype = None
            L.orc_report_claims.argtypes = [P, ip, ip, ip, ip]
            L.orc_report_claims.restype = None
            L.orc_classify.argtypes = [P, ctypes.c_double, ip]
            L.orc_classify.restype = None
            L.orc_check.argtypes = [P, ctypes.c_double, dp]
            L.orc_check.restype = None
            L.orc_check_brute.argtypes = [P]
            L.orc_check_brute.restype = ctypes.c_long
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


# ------------------------------------------------------------------ predicates
def orient3d(a, b, c, d, exact=False):
    f = lib().orc_orient3d_exact if exact else lib().orc_orient3d
    a, b, c, d = map(_vec, (a, b, c, d))
    return f(_d(a), _d(b), _d(c), _d(d))


def insphere(a, b, c, d, e, exact=False):
    f = lib().orc_insphere_exact if exact else lib().orc_insphere
    a, b, c, d, e = map(_vec, (a, b, c, d, e))
    return f(_d(a), _d(b), _d(c), _d(d), _d(e))


def diametral(a, b, p):
    a, b, p = map(_vec, (a, b, p))
    return lib().orc_diametral(_d(a), _d(b), _d(p))


def equatorial(a, b, c, p):
    a, b, c, p = map(_vec, (a, b, c, p))
    return lib().orc_equatorial(_d(a), _d(b), _d(c), _d(p))


def tet_circumcenter(a, b, c, d):
    a, b, c, d = map(_vec, (a, b, c, d))
    out = np.zeros(3)
    ok = lib().orc_tet_cc(_d(a), _d(b), _d(c), _d(d), _d(out))
    return out, bool(ok)


def tri_circumcenter(a, b, c):
    a, b, c = map(_vec, (a, b, c))
    out = np.zeros(3)
    ok = lib().orc_tri_cc(_d(a), _d(b), _d(c), _d(out))
    return out, bool(ok)


def midpoint(a, b):
    a, b = map(_vec, (a, b))
    out = np.zeros(3)
    lib().orc_midpoint(_d(a), _d(b), _d(out))
    return out


def tet_bad(a, b, c, d, B):
    a, b, c, d = map(_vec, (a, b, c, d))
    return bool(lib().orc_tet_bad(_d(a), _d(b), _d(c), _d(d), float(B)))


def prio_hash(cls, ids):
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    return int(lib().orc_prio_hash(int(cls), _i(ids), len(ids)))


def prio_hash_xyz(cls, xyz):
    """Priority of an element from its vertices' coordinates, (n, 3), vertices in
    ascending id order."""
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    return int(lib().orc_prio_hash_xyz(int(cls), _d(xyz), len(xyz)))


# ---------------------------------------------------------------------- meshes
class Mesh:
    """A constrained mesh held by the oracle."""

    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle mesh construction failed")
        self.h = handle

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_free(h)
            self.h = None

    @classmethod
    def box_delaunay(cls, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        sk = ctypes.c_int(0)
        h = lib().orc_box_delaunay(_d(pts), len(pts), ctypes.byref(sk))
        m = cls(h)
        m.skipped = sk.value
        return m

    def insert_points(self, pts):
        """More points into a box Delaunay mesh (before set_constraints): the
        sequential Bowyer-Watson step, in Morton order. Returns the duplicates
        skipped."""
        pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
        r = lib().orc_insert_points(self.h, _d(pts), len(pts))
        if r < 0:
            raise ValueError("a point lies outside the box")
        return r

    @classmethod
    def create(cls, xyz, tets):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        return cls(lib().orc_create(_d(xyz), len(xyz), _i(tets), len(tets)))

    def set_constraints(self, segs, seg_id, tris, facet_id, nfacets, facetq=None, guard2=-1.0):
        segs = np.ascontiguousarray(np.asarray(segs, dtype=np.int32).reshape(-1, 2))
        seg_id = np.ascontiguousarray(np.asarray(seg_id, dtype=np.int32))
        tris = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
        facet_id = np.ascontiguousarray(np.asarray(facet_id, dtype=np.int32))
        fq = None
        if facetq is not None:
            fq = np.ascontiguousarray(np.asarray(facetq, dtype=np.float64).reshape(-1, 3))
        bad = lib().orc_set_constraints(
            self.h, _i(segs), _i(seg_id), len(segs), _i(tris), _i(facet_id), len(tris),
            _d(fq) if fq is not None else None, int(nfacets), float(guard2))
        return bad

    def set_limits(self, walk_limit=100000, cav_limit=4096):
        lib().orc_set_limits(self.h, int(walk_limit), int(cav_limit))

    def set_flags(self, tflag=None, sfflag=None, ssflag=None):
        a = [np.ascontiguousarray(x, dtype=np.uint8) if x is not None else None
             for x in (tflag, sfflag, ssflag)]
        lib().orc_set_flags(self.h, *[(_u8(x) if x is not None else None) for x in a])

    def sizes(self):
        out = np.zeros(5, dtype=np.int32)
        lib().orc_sizes(self.h, _i(out))
        return dict(nv=int(out[0]), nt=int(out[1]), ns=int(out[2]), ng=int(out[3]),
                    nfacets=int(out[4]))

    def export(self):
        s = self.sizes()
        xyz = np.zeros((s["nv"], 3))
        tets = np.zeros((s["nt"], 4), dtype=np.int32)
        tflag = np.zeros(s["nt"], dtype=np.uint8)
        sf = np.zeros((s["ns"], 4), dtype=np.int32)
        sfflag = np.zeros(s["ns"], dtype=np.uint8)
        ss = np.zeros((s["ng"], 3), dtype=np.int32)
        ssflag = np.zeros(s["ng"], dtype=np.uint8)
        fq = np.zeros((s["nfacets"], 3))
        lib().orc_export(self.h, _d(xyz), _i(tets), _u8(tflag), _i(sf), _u8(sfflag), _i(ss),
                         _u8(ssflag), _d(fq))
        return dict(xyz=xyz, tets=tets, tflag=tflag, sf=sf, sfflag=sfflag, ss=ss,
                    ssflag=ssflag, facetq=fq)

    @property
    def guard2(self):
        return lib().orc_guard2(self.h)

    def classify(self, B):
        out = np.zeros(3, dtype=np.int32)
        lib().orc_classify(self.h, float(B), _i(out))
        return [int(x) for x in out]

    def round(self, B):
        out = np.zeros(3, dtype=np.int32)
        lib().orc_round(self.h, float(B), _i(out))
        return dict(cls=int(out[0]), ncand=int(out[1]), inserted=int(out[2]))

    def report(self):
        L = lib()
        sz = np.zeros(7, dtype=np.int32)
        L.orc_report_sizes(self.h, _i(sz))
        n = int(sz[1])
        keys = np.zeros((n, 4), dtype=np.int32)
        pts = np.zeros((n, 3))
        outcome, reason, surv, ncav, nbnd, nfcav, nfs, nfg = (
            np.zeros(n, dtype=np.int32) for _ in range(8))
        cav = np.zeros(max(int(sz[2]), 1), dtype=np.int32)
        fcav = np.zeros(max(int(sz[3]), 1), dtype=np.int32)
        fls = np.zeros(max(int(sz[4]), 1), dtype=np.int32)
        flg = np.zeros(max(int(sz[5]), 1), dtype=np.int32)
        L.orc_report(self.h, _i(keys), _d(pts), _i(outcome), _i(reason), _i(surv), _i(ncav),
                     _i(nbnd), _i(nfcav), _i(cav), _i(fcav), _i(nfs), _i(nfg), _i(fls), _i(flg))
        cs = np.zeros(2, dtype=np.int32)
        L.orc_report_claim_sizes(self.h, _i(cs))
        nst, nsh = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
        st = np.zeros(max(4 * int(cs[0]), 1), dtype=np.int32)
        sh = np.zeros(max(4 * int(cs[1]), 1), dtype=np.int32)
        L.orc_report_claims(self.h, _i(nst), _i(st), _i(nsh), _i(sh))
        return dict(nstart=nst, starts=st[: 4 * cs[0]].reshape(-1, 4), nshell=nsh,
                    shell=sh[: 4 * cs[1]].reshape(-1, 4),
                    cls=int(sz[0]), keys=keys, pts=pts, outcome=outcome, reason=reason,
                    surv=surv, ncav=ncav, nbnd=nbnd, nfcav=nfcav,
                    cav=cav[: sz[2]].reshape(-1, 4), fcav=fcav[: sz[3]].reshape(-1, 3),
                    nflagS=nfs, nflagG=nfg, flagS=fls[: sz[4]].reshape(-1, 3),
                    flagG=flg[: sz[5]].reshape(-1, 2), inserted=int(sz[6]))

    def set_mixed(self, mixed):
        """Round kind: 0/False one class, 1/True every class, 2 subsegments and
        subfaces together (class-first priorities)."""
        lib().orc_set_mixed(self.h, int(mixed))

    def refine_R(self, B, max_rounds=1 << 30):
        out = (ctypes.c_long * 2)()
        lib().orc_refine_R(self.h, float(B), int(max_rounds), out)
        return dict(rounds=int(out[0]), inserted=int(out[1]))

    def refine_S(self, B, max_steps=1 << 62):
        out = (ctypes.c_long * 5)()
        lib().orc_refine_S(self.h, float(B), int(max_steps), out)
        return dict(steps=int(out[0]), evaluated=int(out[1]), inserted=int(out[2]),
                    rejected=int(out[3]), unsplittable=int(out[4]))

    CHECK_NAMES = ["tets", "verts_used", "bad_orient", "nonlocal_delaunay", "vol_rel_err",
                   "euler", "sf_not_face", "sf_bad_count", "hull_not_subface",
                   "ss_not_edge", "seg_chain_bad", "facet_area_rel_err", "enc_subsegs",
                   "enc_subfaces", "bad_tets", "bad_tets_unspl", "unspl_subsegs",
                   "unspl_subfaces", "subfaces", "subsegs", "verts"]

    def check(self, B):
        out = np.zeros(21)
        lib().orc_check(self.h, float(B), _d(out))
        return dict(zip(self.CHECK_NAMES, [float(x) for x in out]))

    def check_brute(self):
        return int(lib().orc_check_brute(self.h))
