// Oracle geometry: exact predicates and the fixed-order FP64 formulas.
//
// TEST INFRASTRUCTURE ONLY. This file belongs to the CPU oracle, a plain and slow
// restatement of the refinement method used to check the CUDA library. Only the
// test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
//
// Every predicate is written ONCE as a polynomial template and evaluated in two
// number types:
//   * Fe  -- an FP64 value carried with a running (a posteriori) bound on its
//            absolute error (Wilkinson-style running error analysis). If |value|
//            exceeds the bound, the sign is certain.
//   * Ex  -- an exact floating-point expansion (Priest / Shewchuk 1997 style
//            nonoverlapping expansions built only by Grow-Expansion), used when
//            the filter cannot decide. Its sign is the sign of its largest
//            component.
// Hence no predicate ever returns a wrong sign.
//
// Paper passages: bad tetrahedron = circumradius / shortest edge > B (Sec. 1);
// splitting points = subsegment midpoint, subface circumcentre, tetrahedron
// circumcentre (Sec. 2); Delaunay region membership = "circumcircle or
// circumsphere encloses p" (Sec. 2).
#pragma once
#include <cstring>
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

// ---------------------------------------------------------------- filter type
constexpr double kU = 1.1102230246251565e-16;  // unit roundoff 2^-53
constexpr double kTiny = 1e-300;               // covers underflow in any op

struct Fe {
  double v, e;
  Fe(double x = 0.0) : v(x), e(0.0) {}
  Fe(double x, double err) : v(x), e(err) {}
};
inline Fe operator+(Fe a, Fe b) {
  double s = a.v + b.v;
  return Fe(s, a.e + b.e + 2.0 * kU * std::fabs(s) + kTiny);
}
inline Fe operator-(Fe a, Fe b) {
  double s = a.v - b.v;
  return Fe(s, a.e + b.e + 2.0 * kU * std::fabs(s) + kTiny);
}
inline Fe operator-(Fe a) { return Fe(-a.v, a.e); }
inline Fe operator*(Fe a, Fe b) {
  double p = a.v * b.v;
  return Fe(p, std::fabs(a.v) * b.e + std::fabs(b.v) * a.e + a.e * b.e +
                   2.0 * kU * std::fabs(p) + kTiny);
}
// Sign if certain, else 2 ("undecided"). The bound itself was computed with
// rounding; the factor absorbs that relative error (a few hundred ulps at most).
inline int fe_sign(Fe a) {
  double bound = a.e * (1.0 + 1.0 / 1073741824.0);
  if (a.v > bound) return 1;
  if (-a.v > bound) return -1;
  return 2;
}

// ----------------------------------------------------------- exact expansions
inline void two_sum(double a, double b, double& s, double& err) {
  s = a + b;
  double bv = s - a;
  double av = s - bv;
  err = (a - av) + (b - bv);
}
inline void split27(double a, double& hi, double& lo) {
  double c = 134217729.0 * a;  // 2^27 + 1
  double big = c - a;
  hi = c - big;
  lo = a - hi;
}
inline void two_prod(double a, double b, double& p, double& err) {
  p = a * b;
  double ah, al, bh, bl;
  split27(a, ah, al);
  split27(b, bh, bl);
  double e1 = p - ah * bh;
  double e2 = e1 - al * bh;
  double e3 = e2 - ah * bl;
  err = al * bl - e3;
}

struct Ex {
  std::vector<double> c;  // nonoverlapping, increasing magnitude, no zeros
  Ex() {}
  Ex(double x) {
    if (x != 0.0) c.push_back(x);
  }
};
// Grow-Expansion with zero elimination: returns e + b exactly.
inline Ex ex_grow(const Ex& e, double b) {
  Ex h;
  h.c.reserve(e.c.size() + 1);
  double q = b;
  for (double ei : e.c) {
    double s, err;
    two_sum(q, ei, s, err);
    if (err != 0.0) h.c.push_back(err);
    q = s;
  }
  if (q != 0.0) h.c.push_back(q);
  return h;
}
inline Ex operator+(const Ex& a, const Ex& b) {
  Ex r = a;
  for (double x : b.c) r = ex_grow(r, x);
  return r;
}
inline Ex operator-(const Ex& a) {
  Ex r = a;
  for (double& x : r.c) x = -x;
  return r;
}
inline Ex operator-(const Ex& a, const Ex& b) { return a + (-b); }
inline Ex ex_scale(const Ex& a, double b) {
  Ex r;
  for (double x : a.c) {
    double p, err;
    two_prod(x, b, p, err);
    if (err != 0.0) r = ex_grow(r, err);
    if (p != 0.0) r = ex_grow(r, p);
  }
  return r;
}
inline Ex operator*(const Ex& a, const Ex& b) {
  Ex r;
  for (double x : b.c) r = r + ex_scale(a, x);
  return r;
}
inline int ex_sign(const Ex& a) {
  if (a.c.empty()) return 0;
  return a.c.back() > 0.0 ? 1 : -1;
}

// ------------------------------------------------------ predicate polynomials
// orient(a,b,c,d) = (b-a) . ((c-a) x (d-a)); tetrahedra are stored with orient > 0.
template <class N>
N poly_orient(const double* a, const double* b, const double* c, const double* d) {
  N ux = N(b[0]) - N(a[0]), uy = N(b[1]) - N(a[1]), uz = N(b[2]) - N(a[2]);
  N vx = N(c[0]) - N(a[0]), vy = N(c[1]) - N(a[1]), vz = N(c[2]) - N(a[2]);
  N wx = N(d[0]) - N(a[0]), wy = N(d[1]) - N(a[1]), wz = N(d[2]) - N(a[2]);
  return ux * (vy * wz - vz * wy) + uy * (vz * wx - vx * wz) + uz * (vx * wy - vy * wx);
}

template <class N>
N det3(const N& ax, const N& ay, const N& az, const N& bx, const N& by, const N& bz,
       const N& cx, const N& cy, const N& cz) {
  return ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
}

// The lifted 4x4 determinant with rows (x-e, |x-e|^2) for x = a,b,c,d, negated so
// that the result is positive iff e is strictly inside the circumsphere of a
// positively oriented (a,b,c,d).
template <class N>
N poly_insphere(const double* a, const double* b, const double* c, const double* d,
                const double* e) {
  N ax = N(a[0]) - N(e[0]), ay = N(a[1]) - N(e[1]), az = N(a[2]) - N(e[2]);
  N bx = N(b[0]) - N(e[0]), by = N(b[1]) - N(e[1]), bz = N(b[2]) - N(e[2]);
  N cx = N(c[0]) - N(e[0]), cy = N(c[1]) - N(e[1]), cz = N(c[2]) - N(e[2]);
  N dx = N(d[0]) - N(e[0]), dy = N(d[1]) - N(e[1]), dz = N(d[2]) - N(e[2]);
  N al = ax * ax + ay * ay + az * az;
  N bl = bx * bx + by * by + bz * bz;
  N cl = cx * cx + cy * cy + cz * cz;
  N dl = dx * dx + dy * dy + dz * dz;
  // cofactor expansion of the 4x4 determinant along the lift column
  N det4 = dl * det3(ax, ay, az, bx, by, bz, cx, cy, cz) -
           cl * det3(ax, ay, az, bx, by, bz, dx, dy, dz) +
           bl * det3(ax, ay, az, cx, cy, cz, dx, dy, dz) -
           al * det3(bx, by, bz, cx, cy, cz, dx, dy, dz);
  return -det4;
}

// (a-p).(b-p): negative iff p lies strictly inside the diametral sphere of ab.
template <class N>
N poly_diametral(const double* a, const double* b, const double* p) {
  N ax = N(a[0]) - N(p[0]), ay = N(a[1]) - N(p[1]), az = N(a[2]) - N(p[2]);
  N bx = N(b[0]) - N(p[0]), by = N(b[1]) - N(p[1]), bz = N(b[2]) - N(p[2]);
  return ax * bx + ay * by + az * bz;
}

// |w|^2 |n|^2 - w.m with u=b-a, v=c-a, w=p-a, n=u x v,
// m = |u|^2 (v x n) + |v|^2 (n x u). The circumcentre of abc is a + m/(2|n|^2),
// so the value is negative iff p is strictly inside the equatorial sphere.
template <class N>
N poly_equatorial(const double* a, const double* b, const double* c, const double* p) {
  N ux = N(b[0]) - N(a[0]), uy = N(b[1]) - N(a[1]), uz = N(b[2]) - N(a[2]);
  N vx = N(c[0]) - N(a[0]), vy = N(c[1]) - N(a[1]), vz = N(c[2]) - N(a[2]);
  N wx = N(p[0]) - N(a[0]), wy = N(p[1]) - N(a[1]), wz = N(p[2]) - N(a[2]);
  N nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  N lu = ux * ux + uy * uy + uz * uz;
  N lv = vx * vx + vy * vy + vz * vz;
  N lw = wx * wx + wy * wy + wz * wz;
  N ln = nx * nx + ny * ny + nz * nz;
  // v x n and n x u
  N vnx = vy * nz - vz * ny, vny = vz * nx - vx * nz, vnz = vx * ny - vy * nx;
  N nux = ny * uz - nz * uy, nuy = nz * ux - nx * uz, nuz = nx * uy - ny * ux;
  N mx = lu * vnx + lv * nux, my = lu * vny + lv * nuy, mz = lu * vnz + lv * nuz;
  return lw * ln - (wx * mx + wy * my + wz * mz);
}

inline int sgn_orient(const double* a, const double* b, const double* c, const double* d) {
  int s = fe_sign(poly_orient<Fe>(a, b, c, d));
  return s != 2 ? s : ex_sign(poly_orient<Ex>(a, b, c, d));
}
inline int sgn_insphere(const double* a, const double* b, const double* c, const double* d,
                        const double* e) {
  int s = fe_sign(poly_insphere<Fe>(a, b, c, d, e));
  return s != 2 ? s : ex_sign(poly_insphere<Ex>(a, b, c, d, e));
}
inline int sgn_diametral(const double* a, const double* b, const double* p) {
  int s = fe_sign(poly_diametral<Fe>(a, b, p));
  return s != 2 ? s : ex_sign(poly_diametral<Ex>(a, b, p));
}
inline int sgn_equatorial(const double* a, const double* b, const double* c, const double* p) {
  int s = fe_sign(poly_equatorial<Fe>(a, b, c, p));
  return s != 2 ? s : ex_sign(poly_equatorial<Ex>(a, b, c, p));
}

// Exact-only variants (used by tests to check that the filter never lies).
inline int sgn_orient_exact(const double* a, const double* b, const double* c, const double* d) {
  return ex_sign(poly_orient<Ex>(a, b, c, d));
}
inline int sgn_insphere_exact(const double* a, const double* b, const double* c,
                              const double* d, const double* e) {
  return ex_sign(poly_insphere<Ex>(a, b, c, d, e));
}

// ------------------------------------------------- fixed-order FP64 formulas
// These are evaluated left to right, one IEEE rounding per operation, with no
// contraction into fused multiply-adds (the oracle is built -ffp-contract=off).

// Subsegment splitting point: the midpoint (Sec. 2).
inline void midpoint(const double* a, const double* b, double* out) {
  for (int k = 0; k < 3; ++k) out[k] = (a[k] + b[k]) * 0.5;
}

// Tetrahedron circumcentre (Sec. 2): c = a + N / (2 u.(v x w)),
// N = |u|^2 (v x w) + |v|^2 (w x u) + |w|^2 (u x v), u,v,w = b-a, c-a, d-a.
// Returns the offset o = c - a through off (if non-null). Returns false if the
// FP64 denominator is zero or the result is not finite. Callers pass the
// vertices in ascending vertex-id order, so the result does not depend on how
// a tetrahedron happens to be stored.
inline bool tet_circumcenter(const double* a, const double* b, const double* c, const double* d,
                             double* out, double* off) {
  double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
  double vx = c[0] - a[0], vy = c[1] - a[1], vz = c[2] - a[2];
  double wx = d[0] - a[0], wy = d[1] - a[1], wz = d[2] - a[2];
  double lu = ux * ux + uy * uy + uz * uz;
  double lv = vx * vx + vy * vy + vz * vz;
  double lw = wx * wx + wy * wy + wz * wz;
  double vwx = vy * wz - vz * wy, vwy = vz * wx - vx * wz, vwz = vx * wy - vy * wx;
  double wux = wy * uz - wz * uy, wuy = wz * ux - wx * uz, wuz = wx * uy - wy * ux;
  double uvx = uy * vz - uz * vy, uvy = uz * vx - ux * vz, uvz = ux * vy - uy * vx;
  double det = ux * vwx + uy * vwy + uz * vwz;
  double den = 2.0 * det;
  double nx = lu * vwx + lv * wux + lw * uvx;
  double ny = lu * vwy + lv * wuy + lw * uvy;
  double nz = lu * vwz + lv * wuz + lw * uvz;
  double ox = nx / den, oy = ny / den, oz = nz / den;
  out[0] = a[0] + ox;
  out[1] = a[1] + oy;
  out[2] = a[2] + oz;
  if (off) {
    off[0] = ox;
    off[1] = oy;
    off[2] = oz;
  }
  return den != 0.0 && std::isfinite(out[0]) && std::isfinite(out[1]) && std::isfinite(out[2]);
}

// Subface circumcentre (Sec. 2): c = a + (|u|^2 (v x n) + |v|^2 (n x u)) / (2|n|^2).
inline bool tri_circumcenter(const double* a, const double* b, const double* c, double* out) {
  double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
  double vx = c[0] - a[0], vy = c[1] - a[1], vz = c[2] - a[2];
  double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  double lu = ux * ux + uy * uy + uz * uz;
  double lv = vx * vx + vy * vy + vz * vz;
  double ln = nx * nx + ny * ny + nz * nz;
  double vnx = vy * nz - vz * ny, vny = vz * nx - vx * nz, vnz = vx * ny - vy * nx;
  double nux = ny * uz - nz * uy, nuy = nz * ux - nx * uz, nuz = nx * uy - ny * ux;
  double mx = lu * vnx + lv * nux, my = lu * vny + lv * nuy, mz = lu * vnz + lv * nuz;
  double den = 2.0 * ln;
  out[0] = a[0] + mx / den;
  out[1] = a[1] + my / den;
  out[2] = a[2] + mz / den;
  return den != 0.0 && std::isfinite(out[0]) && std::isfinite(out[1]) && std::isfinite(out[2]);
}

inline double dist2(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return dx * dx + dy * dy + dz * dz;
}

// Bad-tetrahedron test (Sec. 1): rho^2 = R^2 / l_min^2 > B^2, with R^2 taken from
// the circumcentre offset of tet_circumcenter and l_min^2 the smallest squared
// edge length (edges ab, ac, ad, bc, bd, cd in that order). Vertices come in
// ascending id order. A tetrahedron whose FP64 circumcentre is degenerate counts
// as bad (its split is then refused as unsplittable).
inline bool tet_is_bad(const double* a, const double* b, const double* c, const double* d,
                       double B) {
  double cc[3], o[3];
  bool ok = tet_circumcenter(a, b, c, d, cc, o);
  if (!ok) return true;
  double r2 = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
  double l2 = dist2(b, a);
  double t;
  t = dist2(c, a); if (t < l2) l2 = t;
  t = dist2(d, a); if (t < l2) l2 = t;
  t = dist2(c, b); if (t < l2) l2 = t;
  t = dist2(d, b); if (t < l2) l2 = t;
  t = dist2(d, c); if (t < l2) l2 = t;
  return (r2 / l2) > (B * B);
}

// Priority hash for candidate ordering (the predetermined priorities of Sec. 2):
// the SplitMix64 finaliser (Steele, Lea and Flood 2014) chained over 64-bit words
// and seeded by the class. An element's words are the bit patterns of its
// vertices' coordinates (x, y, z per vertex, vertices in ascending id order), so
// its priority depends on its geometry and on the relative order of its vertex
// ids only: an instance refined alone or beside others in one mesh orders its
// candidates the same way. A plain point's word is its index.
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
inline uint64_t prio_hash(int cls, const int* ids, int n) {
  uint64_t h = 0x9E3779B97F4A7C15ULL * (uint64_t)(cls + 1);
  for (int i = 0; i < n; ++i) h = mix64(h ^ (uint64_t)(uint32_t)ids[i]);
  return h;
}
inline uint64_t prio_hash_xyz(int cls, const double* xyz, int nverts) {
  uint64_t h = 0x9E3779B97F4A7C15ULL * (uint64_t)(cls + 1);
  for (int i = 0; i < 3 * nverts; ++i) {
    uint64_t w;
    std::memcpy(&w, &xyz[i], 8);
    h = mix64(h ^ w);
  }
  return h;
}

}  // namespace orc
