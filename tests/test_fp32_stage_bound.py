"""Soundness of the device predicates' FP32 first stage, emulated on the CPU.

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
