"""Pins for the oracle's geometry against exact rational arithmetic.

Every reference here uses a formulation different from the oracle's: signs come
from exact rational circumcentres (solved by Gaussian elimination over
fractions.Fraction, which is exact for FP64 inputs) or from the 4x4 homogeneous
determinant, never from the oracle's own polynomials.
"""
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------ exact references
def det(m):
    m = [list(r) for r in m]
    n = len(m)
    s = F(1)
    for c in range(n):
        piv = next((r for r in range(c, n) if m[r][c] != 0), None)
        if piv is None:
            return F(0)
        if piv != c:
            m[c], m[piv] = m[piv], m[c]
            s = -s
        for r in range(c + 1, n):
            f = m[r][c] / m[c][c]
            for k in range(c, n):
                m[r][k] -= f * m[c][k]
        s *= m[c][c]
    return s


def solve(A, b):
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] != 0), None)
        if piv is None:
            return None
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                for k in range(c, n + 1):
                    M[r][k] -= f * M[c][k]
    return [M[i][n] / M[i][i] for i in range(n)]


def fr(p):
    return [F(float(x)) for x in p]


def sub(a, b):
    return [x - y for x, y in zip(a, b)]


def dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def sgn(x):
    return (x > 0) - (x < 0)


def ref_orient(a, b, c, d):
    # homogeneous 4x4 determinant; the unit tetrahedron (origin, e1, e2, e3) is
    # the positive orientation by the library's convention, which is -det4.
    rows = [fr(p) + [F(1)] for p in (a, b, c, d)]
    return sgn(-det(rows))


def ref_circumcentre(pts):
    P = [fr(p) for p in pts]
    A = [[2 * x for x in sub(P[i], P[0])] for i in range(1, 4)]
    b = [dot(P[i], P[i]) - dot(P[0], P[0]) for i in range(1, 4)]
    return solve(A, b)


def ref_insphere(a, b, c, d, e):
    cc = ref_circumcentre([a, b, c, d])
    if cc is None:
        return None
    A, E = fr(a), fr(e)
    r2 = dot(sub(A, cc), sub(A, cc))
    d2 = dot(sub(E, cc), sub(E, cc))
    return sgn(r2 - d2)


def ref_tri_circumcentre(a, b, c):
    A, B, C = fr(a), fr(b), fr(c)
    u, v = sub(B, A), sub(C, A)
    st = solve([[dot(u, u), dot(u, v)], [dot(u, v), dot(v, v)]],
               [dot(u, u) / 2, dot(v, v) / 2])
    if st is None:
        return None
    return [A[k] + st[0] * u[k] + st[1] * v[k] for k in range(3)]


def ref_equatorial(a, b, c, p):
    cc = ref_tri_circumcentre(a, b, c)
    A, P = fr(a), fr(p)
    return sgn(dot(sub(P, cc), sub(P, cc)) - dot(sub(A, cc), sub(A, cc)))


def ref_diametral(a, b, p):
    A, B, P = fr(a), fr(b), fr(p)
    m = [(x + y) / 2 for x, y in zip(A, B)]
    return sgn(dot(sub(P, m), sub(P, m)) - dot(sub(A, B), sub(A, B)) / 4)


# ------------------------------------------------------------ input families
def families(rng, n):
    """Random, integer-grid (degenerate) and 1-ulp-perturbed degenerate points."""
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            out.append(rng.uniform(-1, 1, size=(5, 3)))
        elif kind == 1:
            out.append(rng.integers(-2, 3, size=(5, 3)).astype(np.float64))
        elif kind == 2:
            # integer points on the sphere x^2+y^2+z^2 = 9 (exactly cospherical)
            S = np.array([[1, 2, 2], [2, 1, 2], [2, 2, 1], [-1, 2, 2], [2, -1, 2], [2, 2, -1],
                          [1, -2, 2], [3, 0, 0], [0, 3, 0], [0, 0, 3], [0, 0, -3], [-2, -2, 1]],
                         dtype=np.float64)
            out.append(S[rng.choice(len(S), size=5, replace=False)] + 1000.0)
        else:
            base = rng.integers(-2, 3, size=(5, 3)).astype(np.float64) * 0.1 + 0.3
            j = rng.integers(0, 5)
            k = rng.integers(0, 3)
            base[j, k] = np.nextafter(base[j, k], np.inf if rng.random() < 0.5 else -np.inf)
            out.append(base)
    return out


def test_orient3d_matches_exact():
    rng = np.random.default_rng(11)
    nz = 0
    for P in families(rng, 1200):
        a, b, c, d = P[:4]
        r = ref_orient(a, b, c, d)
        assert oracle.orient3d(a, b, c, d) == r
        assert oracle.orient3d(a, b, c, d, exact=True) == r
        nz += r == 0
    assert nz > 50  # the degenerate families really are degenerate


def test_insphere_matches_exact():
    rng = np.random.default_rng(12)
    zeros = 0
    checked = 0
    for P in families(rng, 1200):
        a, b, c, d, e = P
        o = ref_orient(a, b, c, d)
        if o == 0:
            continue
        if o < 0:
            a, b = b, a
        r = ref_insphere(a, b, c, d, e)
        assert oracle.insphere(a, b, c, d, e) == r
        assert oracle.insphere(a, b, c, d, e, exact=True) == r
        zeros += r == 0
        checked += 1
    assert checked > 600 and zeros > 20


def test_insphere_sign_convention():
    a, b, c, d = [0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]
    assert oracle.orient3d(a, b, c, d) == 1
    assert oracle.insphere(a, b, c, d, [0.25, 0.25, 0.25]) == 1
    assert oracle.insphere(a, b, c, d, [2, 2, 2]) == -1
    assert oracle.insphere(a, b, c, d, [1, 1, 1]) == 0  # a cube corner: cospherical


def test_diametral_equatorial_match_exact():
    rng = np.random.default_rng(13)
    nzd = nze = 0
    for P in families(rng, 1200):
        a, b, c, p = P[:4]
        if not np.array_equal(a, b):
            r = ref_diametral(a, b, p)
            assert oracle.diametral(a, b, p) == r
            nzd += r == 0
        if ref_orient(a, b, c, a + np.array([0.37, 0.71, 0.19])) != 0 or \
                np.linalg.norm(np.cross(b - a, c - a)) > 0:
            if ref_tri_circumcentre(a, b, c) is None:
                continue
            r = ref_equatorial(a, b, c, p)
            assert oracle.equatorial(a, b, c, p) == r
            nze += r == 0
    assert nzd > 5 and nze > 5


def _read_golden():
    rows = []
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, verts, exp = [x.strip() for x in line.split("|")]
            V = [np.array([float(t) for t in v.split()]) for v in verts.split(";")]
            rows.append((kind, V, np.array([float(t) for t in exp.split()])))
    return rows


@pytest.mark.parametrize("row", _read_golden(), ids=lambda r: r[0])
def test_closed_form_splitting_points(row):
    kind, V, exp = row
    if kind == "tet":
        got, ok = oracle.tet_circumcenter(*V)
        assert ok
    elif kind == "tri":
        got, ok = oracle.tri_circumcenter(*V)
        assert ok
    else:
        got = oracle.midpoint(*V)
    np.testing.assert_allclose(got, exp, rtol=0, atol=1e-15 * max(1.0, np.abs(exp).max()))


def test_circumcentres_near_exact():
    """FP64 circumcentres are within 1e-12 R of the exact rational circumcentre."""
    rng = np.random.default_rng(14)
    for _ in range(300):
        P = rng.uniform(0, 1000, size=(4, 3))
        if abs(np.linalg.det(P[1:] - P[0])) < 1e3:
            continue
        got, ok = oracle.tet_circumcenter(*P)
        cc = ref_circumcentre(P)
        R = float(np.sqrt(float(dot(sub(fr(P[0]), cc), sub(fr(P[0]), cc)))))
        err = np.linalg.norm(got - np.array([float(x) for x in cc]))
        assert ok and err <= 1e-12 * R
        T = P[:3]
        got, ok = oracle.tri_circumcenter(*T)
        cc = ref_tri_circumcentre(*T)
        R = float(np.sqrt(float(dot(sub(fr(T[0]), cc), sub(fr(T[0]), cc)))))
        err = np.linalg.norm(got - np.array([float(x) for x in cc]))
        assert ok and err <= 1e-12 * R


def test_bad_tet_matches_exact_ratio():
    """rho^2 = R^2 / l_min^2 > B^2 against the exact rational ratio (Sec. 1)."""
    rng = np.random.default_rng(15)
    n = 0
    for _ in range(400):
        P = rng.uniform(0, 1, size=(4, 3))
        if abs(np.linalg.det(P[1:] - P[0])) < 1e-4:
            continue
        cc = ref_circumcentre(P)
        A = fr(P[0])
        R2 = dot(sub(A, cc), sub(A, cc))
        Q = [fr(p) for p in P]
        l2 = min(dot(sub(Q[i], Q[j]), sub(Q[i], Q[j])) for i in range(4) for j in range(i + 1, 4))
        for B in (1.4, 2.0):
            exact = R2 / l2 - F(B) ** 2
            if abs(float(exact)) < 1e-9 * B * B:
                continue
            assert oracle.tet_bad(*P, B) == (exact > 0)
            n += 1
    assert n > 500


def test_priority_hash_is_splitmix64():
    # SplitMix64 (Steele, Lea, Flood 2014): from state 0 the first output is
    # mix(0x9E3779B97F4A7C15) = 0xE220A8397B1DCDAF (the generator's reference value).
    assert oracle.prio_hash(0, [0]) == 0xE220A8397B1DCDAF
    # chaining: h = mix(h ^ id) over the sorted ids, seeded by golden * (cls+1)
    def mix(z):
        M = (1 << 64) - 1
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)
    for cls, ids in [(2, [3, 17, 40, 99]), (1, [5, 6, 7]), (0, [123456, 999999])]:
        h = (0x9E3779B97F4A7C15 * (cls + 1)) & ((1 << 64) - 1)
        for i in ids:
            h = mix(h ^ i)
        assert oracle.prio_hash(cls, ids) == h
    # an element's priority chains the same finaliser over the bit patterns of
    # its vertex coordinates (x, y, z per vertex, ascending vertex id)
    P = np.array([[0.0, 1.5, -2.25], [1e-300, 3.0, 7.0], [5.0, -0.0, 1.0]])
    for cls in (0, 1, 2):
        h = (0x9E3779B97F4A7C15 * (cls + 1)) & ((1 << 64) - 1)
        for w in P.reshape(-1).view(np.uint64):
            h = mix(h ^ int(w))
        assert oracle.prio_hash_xyz(cls, P) == h
    # it depends on the geometry only, and -0.0 differs from 0.0 bitwise
    assert oracle.prio_hash_xyz(2, P) != oracle.prio_hash_xyz(2, P[::-1])
    Q = P.copy()
    Q[2, 1] = 0.0
    assert oracle.prio_hash_xyz(2, P) != oracle.prio_hash_xyz(2, Q)


def _facet_ref_point(a, b, c, s):
    """The per-facet reference point of the in-facet reading: the triangle's
    first vertex moved by s along its dominant normal axis (ties to the lowest)."""
    n = np.cross(b - a, c - a)
    k = int(np.argmax(np.abs(n)))  # argmax keeps the first of equal values
    q = a.copy()
    q[k] += s
    return q


def _ref_in_circumcircle(a, b, c, p):
    """Exact sign of (R^2 - |p - cc|^2) with cc the rational circumcentre of abc."""
    cc = ref_tri_circumcentre(a, b, c)
    A, P = fr(a), fr(p)
    return sgn(dot(sub(A, cc), sub(A, cc)) - dot(sub(P, cc), sub(P, cc)))


def test_in_facet_circle_reading_is_the_facet_incircle():
    """For a point in the facet's plane, the sphere through the subface and the
    facet's reference point q_f cuts that plane in the subface's circumcircle,
    so insphere(a, b, c, q_f, p) times the winding orient3d(a, b, c, q_f) is
    the in-circumcircle sign of p, whatever the plane and the vertex order."""
    rng = np.random.default_rng(17)
    circle = [(5, 0), (0, 5), (-5, 0), (0, -5), (3, 4), (4, 3), (-3, 4), (-4, -3), (3, -4)]
    planes = [  # maps from integer (u, v) to points exactly on a plane
        lambda u, v: np.array([u, v, 7.0]),                 # z = 7
        lambda u, v: np.array([u + 2.0, -3.0, v]),          # y = -3
        lambda u, v: np.array([u, v, -u - v + 1.0]),        # x + y + z = 1 (normal ties)
        lambda u, v: np.array([u, v, 2.0 * u - v + 3.0]),   # slanted, dominant axis z
    ]
    seen = {-1: 0, 0: 0, 1: 0}
    for trial in range(600):
        to3 = planes[trial % len(planes)]
        if trial % 3 == 0 and trial % len(planes) < 2:
            # cocircular quadruples on an axis-aligned plane: p on the circle
            idx = rng.choice(len(circle), size=4, replace=False)
            a, b, c, p = (to3(*map(float, circle[i])) for i in idx)
        else:
            uv = rng.integers(-6, 7, size=(4, 2)).astype(np.float64)
            a, b, c, p = (to3(*w) for w in uv)
        if np.linalg.norm(np.cross(b - a, c - a)) == 0:
            continue
        q = _facet_ref_point(a, b, c, 64.0)
        wind = oracle.orient3d(a, b, c, q)
        assert wind != 0
        got = oracle.insphere(a, b, c, q, p) * wind
        exp = _ref_in_circumcircle(a, b, c, p)
        assert got == exp, (a, b, c, p)
        # the reversed triangle reads the same circle
        assert oracle.insphere(b, a, c, q, p) * oracle.orient3d(b, a, c, q) == exp
        seen[exp] += 1
    assert min(seen.values()) > 20, seen
