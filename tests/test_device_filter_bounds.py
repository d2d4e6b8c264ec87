"""Soundness of the device predicates' floating-point stages, emulated on the CPU.

The CUDA orient3d and insphere first decide in FP32: coordinate differences
formed in FP64 and rounded once to FP32, the determinant and its permanent
evaluated in FP32 along a fixed straight-line program, and a sign returned only
when |det| exceeds 32 (orient3d) or 64 (insphere) times 2^-24 times the
permanent, plus 2^-40, and every nonzero difference lies in [2^-20, 2^24].
This file restates that program in numpy float32 (IEEE round to nearest, one
rounding per operation; where the device compiler fuses a multiply and an add,
it rounds once for both, and the same error bound covers it) and checks, on nearly
coplanar and nearly cospherical inputs, that every sign the stage decides is
the exact sign (the oracle's exact predicates, themselves pinned against
rational arithmetic). A bound 64 times smaller does give wrong signs on the
same inputs, so they do reach the edge of the bound.
"""
import numpy as np
import pytest

import oracle

U = np.float32(2.0 ** -24)
ABS = np.float32(2.0 ** -40)
LO, HI = np.float32(2.0 ** -20), np.float32(2.0 ** 24)
f32 = np.float32


def _in_range(*vs):
    ok = np.ones(vs[0].shape, dtype=bool)
    for v in vs:
        a = np.abs(v)
        ok &= (a == 0) | ((a >= LO) & (a <= HI))
    return ok


def _det3(ax, ay, az, bx, by, bz, cx, cy, cz):
    m1 = by * cz - bz * cy
    m2 = bz * cx - bx * cz
    m3 = bx * cy - by * cx
    perm = (np.abs(ax) * (np.abs(by * cz) + np.abs(bz * cy)) +
            np.abs(ay) * (np.abs(bz * cx) + np.abs(bx * cz)) +
            np.abs(az) * (np.abs(bx * cy) + np.abs(by * cx)))
    return ax * m1 + ay * m2 + az * m3, perm


def orient_stage(a, b, c, d, shrink=1):
    """(decided, sign) of the FP32 stage of orient3d for (n, 3) float64 arrays."""
    u, v, w = ((p - a).astype(f32) for p in (b, c, d))
    det, perm = _det3(u[:, 0], u[:, 1], u[:, 2], v[:, 0], v[:, 1], v[:, 2],
                      w[:, 0], w[:, 1], w[:, 2])
    bound = f32(32) * U / f32(shrink) * perm + ABS
    ok = _in_range(*u.T, *v.T, *w.T)
    dec = ok & ((det > bound) | (-det > bound))
    return dec, np.sign(det).astype(int)


def insphere_stage(a, b, c, d, e, shrink=1):
    """(decided, sign) of the FP32 stage of insphere (> 0: e strictly inside)."""
    A, Bq, C, D = ((p - e).astype(f32) for p in (a, b, c, d))
    al, bl, cl, dl = ((q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]) + q[:, 2] * q[:, 2]
                      for q in (A, Bq, C, D))
    m1, p1 = _det3(*A.T, *Bq.T, *C.T)
    m2, p2 = _det3(*A.T, *Bq.T, *D.T)
    m3, p3 = _det3(*A.T, *C.T, *D.T)
    m4, p4 = _det3(*Bq.T, *C.T, *D.T)
    det = -(((dl * m1 - cl * m2) + bl * m3) - al * m4)
    perm = ((dl * p1 + cl * p2) + bl * p3) + al * p4
    bound = f32(64) * U / f32(shrink) * perm + ABS
    ok = _in_range(*A.T, *Bq.T, *C.T, *D.T)
    dec = ok & ((det > bound) | (-det > bound))
    return dec, np.sign(det).astype(int)


def _near_coplanar(rng, n, scale, noise):
    a, b, c = (rng.uniform(0, scale, size=(n, 3)) for _ in range(3))
    s, t = rng.uniform(-1, 2, size=(2, n, 1))
    d = a + s * (b - a) + t * (c - a)
    d += rng.normal(size=(n, 3)) * noise * scale
    return a, b, c, d


def _near_cospherical(rng, n, scale, noise):
    ctr = rng.uniform(0, scale, size=(n, 1, 3))
    r = rng.uniform(0.01, 0.3, size=(n, 1, 1)) * scale
    dirs = rng.normal(size=(n, 5, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    P = ctr + r * dirs
    P[:, 4] += rng.normal(size=(n, 3)) * noise * scale
    a, b, c, d, e = (P[:, k].copy() for k in range(5))
    # positively oriented a, b, c, d (swap a and b where needed)
    neg = np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a)) < 0
    a[neg], b[neg] = b[neg].copy(), a[neg].copy()
    return a, b, c, d, e


def _wrong(dec, sign, exact_fn, args):
    idx = np.nonzero(dec)[0]
    return sum(sign[i] != exact_fn(*[x[i] for x in args]) for i in idx), len(idx)


@pytest.mark.parametrize("scale", [1.0, 1000.0])
def test_orient_fp32_stage_never_decides_a_wrong_sign(scale):
    rng = np.random.default_rng(31 + int(scale))
    wrong = decided = wrong_small = 0
    for noise in (1e-9, 1e-7, 1e-6, 1e-5):
        args = _near_coplanar(rng, 3000, scale, noise)
        ex = lambda a, b, c, d: oracle.orient3d(a, b, c, d, exact=True)
        w, n = _wrong(*orient_stage(*args), ex, args)
        wrong += w
        decided += n
        wrong_small += _wrong(*orient_stage(*args, shrink=64), ex, args)[0]
    assert wrong == 0
    assert decided > 2000          # the stage decides many of these near-degenerate calls
    assert wrong_small > 0         # and a smaller bound would not be safe on them


@pytest.mark.parametrize("scale", [1.0, 1000.0])
def test_insphere_fp32_stage_never_decides_a_wrong_sign(scale):
    rng = np.random.default_rng(41 + int(scale))
    wrong = decided = wrong_small = 0
    for noise in (1e-8, 1e-6, 1e-5, 1e-4):
        args = _near_cospherical(rng, 2000, scale, noise)
        ex = lambda a, b, c, d, e: oracle.insphere(a, b, c, d, e, exact=True)
        w, n = _wrong(*insphere_stage(*args), ex, args)
        wrong += w
        decided += n
        wrong_small += _wrong(*insphere_stage(*args, shrink=64), ex, args)[0]
    assert wrong == 0
    assert decided > 1000
    assert wrong_small > 0


# ----------------------------------------------------------- FP64 filters
# The second stage: the same polynomials in FP64 from FP64 differences, with
# bounds 16u (orient3d), 40u (insphere), 12u (diametral), 48u (equatorial)
# times the permanent, u = 2^-53, and a sign only when the permanent exceeds
# 1e-250. Restated here in numpy float64 like the FP32 stage above.
EPS = 2.0 ** -53
TINY = 1e-250


def _decide64(val, perm, k):
    bound = k * EPS * perm
    dec = (perm > TINY) & ((val > bound) | (-val > bound))
    return dec, np.sign(val).astype(int)


def orient_fp64(a, b, c, d, shrink=1):
    u, v, w = b - a, c - a, d - a
    det, perm = _det3(*u.T, *v.T, *w.T)
    return _decide64(det, perm, 16 / shrink)


def insphere_fp64(a, b, c, d, e, shrink=1):
    A, Bq, C, D = (p - e for p in (a, b, c, d))
    al, bl, cl, dl = ((q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]) + q[:, 2] * q[:, 2]
                      for q in (A, Bq, C, D))
    m1, p1 = _det3(*A.T, *Bq.T, *C.T)
    m2, p2 = _det3(*A.T, *Bq.T, *D.T)
    m3, p3 = _det3(*A.T, *C.T, *D.T)
    m4, p4 = _det3(*Bq.T, *C.T, *D.T)
    det = -(((dl * m1 - cl * m2) + bl * m3) - al * m4)
    perm = ((dl * p1 + cl * p2) + bl * p3) + al * p4
    return _decide64(det, perm, 40 / shrink)


def diametral_fp64(a, b, p, shrink=1):
    A, Bq = a - p, b - p
    v = (A[:, 0] * Bq[:, 0] + A[:, 1] * Bq[:, 1]) + A[:, 2] * Bq[:, 2]
    perm = (np.abs(A[:, 0] * Bq[:, 0]) + np.abs(A[:, 1] * Bq[:, 1])) + np.abs(A[:, 2] * Bq[:, 2])
    return _decide64(v, perm, 12 / shrink)


def equatorial_fp64(a, b, c, p, shrink=1):
    ux, uy, uz = (b - a).T
    vx, vy, vz = (c - a).T
    wx, wy, wz = (p - a).T
    ab = np.abs
    nx, ny, nz = uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx
    Nx, Ny, Nz = (ab(uy * vz) + ab(uz * vy), ab(uz * vx) + ab(ux * vz),
                  ab(ux * vy) + ab(uy * vx))
    lu = (ux * ux + uy * uy) + uz * uz
    lv = (vx * vx + vy * vy) + vz * vz
    lw = (wx * wx + wy * wy) + wz * wz
    ln = (nx * nx + ny * ny) + nz * nz
    Ln = (Nx * Nx + Ny * Ny) + Nz * Nz
    vnx, vny, vnz = vy * nz - vz * ny, vz * nx - vx * nz, vx * ny - vy * nx
    VNx, VNy, VNz = ab(vy) * Nz + ab(vz) * Ny, ab(vz) * Nx + ab(vx) * Nz, ab(vx) * Ny + ab(vy) * Nx
    nux, nuy, nuz = ny * uz - nz * uy, nz * ux - nx * uz, nx * uy - ny * ux
    NUx, NUy, NUz = Ny * ab(uz) + Nz * ab(uy), Nz * ab(ux) + Nx * ab(uz), Nx * ab(uy) + Ny * ab(ux)
    mx, my, mz = lu * vnx + lv * nux, lu * vny + lv * nuy, lu * vnz + lv * nuz
    Mx, My, Mz = lu * VNx + lv * NUx, lu * VNy + lv * NUy, lu * VNz + lv * NUz
    D = lw * ln - ((wx * mx + wy * my) + wz * mz)
    perm = lw * Ln + ((ab(wx) * Mx + ab(wy) * My) + ab(wz) * Mz)
    return _decide64(D, perm, 48 / shrink)


def _near_diametral(rng, n, scale, noise):
    a, b = (rng.uniform(0, scale, size=(n, 3)) for _ in range(2))
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    p = (a + b) / 2 + dirs * np.linalg.norm(b - a, axis=1, keepdims=True) / 2
    return a, b, p + rng.normal(size=(n, 3)) * noise * scale


def _near_equatorial(rng, n, scale, noise):
    a, b, c = (rng.uniform(0, scale, size=(n, 3)) for _ in range(3))
    u, v = b - a, c - a
    nrm = np.cross(u, v)
    cc = a + (np.einsum("ij,ij->i", u, u)[:, None] * np.cross(v, nrm) +
              np.einsum("ij,ij->i", v, v)[:, None] * np.cross(nrm, u)) / \
        (2 * np.einsum("ij,ij->i", nrm, nrm)[:, None])
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    p = cc + dirs * np.linalg.norm(a - cc, axis=1, keepdims=True)
    return a, b, c, p + rng.normal(size=(n, 3)) * noise * scale


FP64_CASES = [
    ("orient", lambda r, n, s, z: _near_coplanar(r, n, s, z), orient_fp64,
     lambda a, b, c, d: oracle.orient3d(a, b, c, d, exact=True)),
    ("insphere", lambda r, n, s, z: _near_cospherical(r, n, s, z), insphere_fp64,
     lambda a, b, c, d, e: oracle.insphere(a, b, c, d, e, exact=True)),
    ("diametral", _near_diametral, diametral_fp64, oracle.diametral),
    ("equatorial", _near_equatorial, equatorial_fp64, oracle.equatorial),
]


@pytest.mark.parametrize("name,gen,stage,exact", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_filters_never_decide_a_wrong_sign(name, gen, stage, exact):
    rng = np.random.default_rng(sum(map(ord, name)))
    wrong = decided = wrong_small = 0
    for scale in (1.0, 1000.0):
        for noise in (1e-16, 1e-15, 1e-14, 1e-12):
            args = gen(rng, 1500, scale, noise)
            w, n = _wrong(*stage(*args), exact, args)
            wrong += w
            decided += n
            wrong_small += _wrong(*stage(*args, shrink=256), exact, args)[0]
    assert wrong == 0
    assert decided > 1000
    assert wrong_small > 0
