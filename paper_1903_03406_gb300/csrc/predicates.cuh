// Device geometry for the refinement kernels: exact-sign predicates and the
// fixed-order FP64 formulas for splitting points and tetrahedron quality.
//
// Predicates evaluate an FP64 filter whose error bound comes from forward error
// analysis of the straight-line program (|fl(P) - P| <= gamma_k * |P|(|x|), with
// k the largest number of roundings on any path from an input to the result;
// Higham, "Accuracy and Stability of Numerical Algorithms", ch. 3). The bound is
// taken with a factor-of-two margin. When the filter cannot decide, the sign is
// computed exactly with floating-point expansions (Priest 1991; Shewchuk 1997:
// Two-Sum, Two-Product via FMA, Fast-Expansion-Sum and Scale-Expansion with zero
// elimination). No predicate ever returns a wrong sign.
//
// Paper passages: splitting points (Sec. 2: midpoint of a subsegment, circumcentre
// of a subface's circumcircle, circumcentre of a tetrahedron's circumsphere); bad
// tetrahedron: circumradius / shortest edge > B (Sec. 1); Delaunay region: the
// elements whose circumcircle / circumsphere encloses p (Sec. 2).
#pragma once
#include <cstdint>

namespace cdr {

#define CDR_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------ error bounds
// unit roundoff u = 2^-53
constexpr double kEps = 1.1102230246251565e-16;
constexpr double kOrientBound = 16.0 * kEps;    // k = 8 roundings per monomial
constexpr double kInsphereBound = 40.0 * kEps;  // k = 17
constexpr double kEquatBound = 48.0 * kEps;     // k = 20
constexpr double kDiamBound = 12.0 * kEps;      // k = 5
constexpr double kTinyPerm = 1e-250;            // below this, go exact (underflow)

// ------------------------------------------------------- expansion kernels
// Shewchuk's error-free transformations (round-to-nearest, no overflow).
__device__ __forceinline__ void ex_two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  y = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}
__device__ __forceinline__ void ex_fast_two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  y = __dsub_rn(b, __dsub_rn(x, a));
}
__device__ __forceinline__ void ex_two_diff(double a, double b, double& x, double& y) {
  x = __dsub_rn(a, b);
  double bv = __dsub_rn(a, x);
  double av = __dadd_rn(x, bv);
  y = __dadd_rn(__dsub_rn(a, av), __dsub_rn(bv, b));
}
__device__ __forceinline__ void ex_two_prod(double a, double b, double& x, double& y) {
  x = __dmul_rn(a, b);
  y = __fma_rn(a, b, -x);  // exact product error
}

// Fast-Expansion-Sum with zero elimination. e, f nonoverlapping, increasing
// magnitude; h must not alias e or f. Returns the length of h.
__device__ inline int ex_sum(int elen, const double* e, int flen, const double* f, double* h) {
  double Q, Qnew, hh, enow, fnow;
  int ei = 0, fi = 0, hi = 0;
  if (elen == 0) {
    for (int i = 0; i < flen; ++i) h[i] = f[i];
    return flen;
  }
  if (flen == 0) {
    for (int i = 0; i < elen; ++i) h[i] = e[i];
    return elen;
  }
  enow = e[0];
  fnow = f[0];
  if ((fnow > enow) == (fnow > -enow)) {
    Q = enow;
    enow = (++ei < elen) ? e[ei] : 0.0;
  } else {
    Q = fnow;
    fnow = (++fi < flen) ? f[fi] : 0.0;
  }
  if (ei < elen && fi < flen) {
    if ((fnow > enow) == (fnow > -enow)) {
      ex_fast_two_sum(enow, Q, Qnew, hh);
      enow = (++ei < elen) ? e[ei] : 0.0;
    } else {
      ex_fast_two_sum(fnow, Q, Qnew, hh);
      fnow = (++fi < flen) ? f[fi] : 0.0;
    }
    Q = Qnew;
    if (hh != 0.0) h[hi++] = hh;
    while (ei < elen && fi < flen) {
      if ((fnow > enow) == (fnow > -enow)) {
        ex_two_sum(Q, enow, Qnew, hh);
        enow = (++ei < elen) ? e[ei] : 0.0;
      } else {
        ex_two_sum(Q, fnow, Qnew, hh);
        fnow = (++fi < flen) ? f[fi] : 0.0;
      }
      Q = Qnew;
      if (hh != 0.0) h[hi++] = hh;
    }
  }
  while (ei < elen) {
    ex_two_sum(Q, enow, Qnew, hh);
    enow = (++ei < elen) ? e[ei] : 0.0;
    Q = Qnew;
    if (hh != 0.0) h[hi++] = hh;
  }
  while (fi < flen) {
    ex_two_sum(Q, fnow, Qnew, hh);
    fnow = (++fi < flen) ? f[fi] : 0.0;
    Q = Qnew;
    if (hh != 0.0) h[hi++] = hh;
  }
  if (Q != 0.0 || hi == 0) h[hi++] = Q;
  return hi;
}

// Scale-Expansion with zero elimination: h = e * b. h must not alias e.
__device__ inline int ex_scale(int elen, const double* e, double b, double* h) {
  if (elen == 0 || b == 0.0) return 0;
  double Q, sum, hh, p1, p0;
  int hi = 0;
  ex_two_prod(e[0], b, Q, hh);
  if (hh != 0.0) h[hi++] = hh;
  for (int i = 1; i < elen; ++i) {
    ex_two_prod(e[i], b, p1, p0);
    ex_two_sum(Q, p0, sum, hh);
    if (hh != 0.0) h[hi++] = hh;
    ex_fast_two_sum(p1, sum, Q, hh);
    if (hh != 0.0) h[hi++] = hh;
  }
  if (Q != 0.0 || hi == 0) h[hi++] = Q;
  return hi;
}

__device__ __forceinline__ int ex_negate(int n, double* e) {
  for (int i = 0; i < n; ++i) e[i] = -e[i];
  return n;
}
__device__ __forceinline__ int ex_sign(int n, const double* e) {
  for (int i = n - 1; i >= 0; --i)
    if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
  return 0;
}

// Compress (Shewchuk 1997): same value, fewer components, in place.
__device__ inline int ex_compress(int elen, double* e) {
  if (elen <= 1) return elen;
  double Q, q, Qnew;
  int bottom = elen - 1;
  Q = e[bottom];
  for (int i = elen - 2; i >= 0; --i) {
    ex_fast_two_sum(Q, e[i], Qnew, q);
    if (q != 0.0) {
      e[bottom--] = Qnew;
      Q = q;
    } else {
      Q = Qnew;
    }
  }
  int top = 0;
  for (int i = bottom + 1; i < elen; ++i) {
    ex_fast_two_sum(e[i], Q, Qnew, q);
    if (q != 0.0) e[top++] = q;
    Q = Qnew;
  }
  e[top++] = Q;
  return top;
}

// Exact arithmetic works in fixed buffers of kExCap doubles. Every operation
// checks its output bound first; a result that could exceed it sets
// g_exact_overflow (read by the host after each round, which then fails the
// call with CDR_ERR_INTERNAL) instead of returning a possibly wrong sign.
constexpr int kExCap = 256;
static __device__ int g_exact_overflow;

struct ExScratch {
  double t[kExCap], s[kExCap], u[kExCap];
};

// out = a + b, compressed. Returns -1 on capacity overflow.
__device__ inline int ex_add(int na, const double* a, int nb, const double* b, double* out) {
  if (na + nb > kExCap) return -1;
  int n = ex_sum(na, a, nb, b, out);
  return ex_compress(n, out);
}
// out = a * b, compressed. Returns -1 on capacity overflow.
__device__ inline int ex_mul(int na, const double* a, int nb, const double* b, double* out,
                             ExScratch& w) {
  if (na == 0 || nb == 0) return 0;
  if (2 * na * nb > kExCap) return -1;
  int n = 0;
  for (int j = 0; j < nb; ++j) {
    int m = ex_scale(na, a, b[j], w.t);
    int n2 = ex_sum(n, w.s, m, w.t, w.u);
    for (int q = 0; q < n2; ++q) w.s[q] = w.u[q];
    n = n2;
  }
  n = ex_compress(n, w.s);
  for (int q = 0; q < n; ++q) out[q] = w.s[q];
  return n;
}

// Exact difference a - b as an expansion (zero, one or two components).
struct Ex2 {
  double c[2];
  int n;
};
__device__ __forceinline__ Ex2 ex_diff(double a, double b) {
  Ex2 r;
  double x, y;
  ex_two_diff(a, b, x, y);
  if (y != 0.0) {
    r.c[0] = y;
    r.c[1] = x;
    r.n = 2;
  } else {
    r.c[0] = x;
    r.c[1] = 0.0;
    r.n = (x != 0.0) ? 1 : 0;
  }
  return r;
}

#define EX_TRY(expr)                    \
  do {                                  \
    if ((expr) < 0) {                   \
      atomicExch(&g_exact_overflow, 1); \
      return 0;                         \
    }                                   \
  } while (0)

// out = p*q - r*s
__device__ inline int ex_cross(const Ex2& p, const Ex2& q, const Ex2& r, const Ex2& s,
                               double* out, ExScratch& w) {
  double A[8], B[8];
  int na = ex_mul(p.n, p.c, q.n, q.c, A, w);
  int nb = ex_mul(r.n, r.c, s.n, s.c, B, w);
  if (na < 0 || nb < 0) return -1;
  ex_negate(nb, B);
  return ex_add(na, A, nb, B, out);
}

// exact 3x3 determinant with rows r0, r1, r2 of differences
__device__ inline int ex_det3(const Ex2* r0, const Ex2* r1, const Ex2* r2, double* out,
                              ExScratch& w) {
  double M[16], T[64], acc[kExCap], acc2[kExCap];
  int nacc = 0;
  const int I[3][2] = {{1, 2}, {2, 0}, {0, 1}};
  for (int k = 0; k < 3; ++k) {
    int i = I[k][0], j = I[k][1];
    int nm = ex_cross(r1[i], r2[j], r1[j], r2[i], M, w);
    if (nm < 0) return -1;
    int nt = ex_mul(r0[k].n, r0[k].c, nm, M, T, w);
    if (nt < 0) return -1;
    int n2 = ex_add(nacc, acc, nt, T, acc2);
    if (n2 < 0) return -1;
    for (int q = 0; q < n2; ++q) acc[q] = acc2[q];
    nacc = n2;
  }
  for (int q = 0; q < nacc; ++q) out[q] = acc[q];
  return nacc;
}

// exact |r|^2
__device__ inline int ex_len2(const Ex2* r, double* out, ExScratch& w) {
  double sq[8], acc[32], acc2[32];
  int nacc = 0;
  for (int k = 0; k < 3; ++k) {
    int n = ex_mul(r[k].n, r[k].c, r[k].n, r[k].c, sq, w);
    if (n < 0) return -1;
    int n2 = ex_add(nacc, acc, n, sq, acc2);
    if (n2 < 0) return -1;
    for (int q = 0; q < n2; ++q) acc[q] = acc2[q];
    nacc = n2;
  }
  for (int q = 0; q < nacc; ++q) out[q] = acc[q];
  return nacc;
}

// ---------------------------------------------------------- shared helpers
struct D3 {
  double x, y, z;
};

// ------------------------------------------------------ FP32 first stage
// GB300 runs FP32 far faster than FP64, so orient3d and insphere first decide
// in FP32. The coordinate differences are formed in FP64 and rounded once to
// FP32, so each equals the exact difference times (1 + eta) with
// |eta| <= 2^-24 + 2^-53; a degree-k monomial then moves by at most
// ((1+eta)^k - 1) of its magnitude. The determinant and its permanent (the
// same polynomial over absolute values) are evaluated in FP32 along the same
// straight-line program as the FP64 filter below, adding at most gamma_m(2^-24)
// times the permanent (m roundings on a path; Higham ch. 3). The bound is the
// sum of both terms with a factor-of-two margin:
//   orient3d  (k = 3, m = 8):  32 * 2^-24 * permanent
//   insphere  (k = 5, m = 17): 64 * 2^-24 * permanent
// The stage runs only when every nonzero difference lies in [2^-20, 2^24]: then
// no product overflows and a product can leave the normal range only after an
// exact (Sterbenz) cancellation; the absolute error such an underflow can
// carry, at most 2^-150 per operation times the remaining factors (< 2^100 in
// all), stays below the added absolute term 2^-40. Undecided cases fall
// through to the FP64 filter and then to exact arithmetic.
constexpr float kF32Unit = 5.9604644775390625e-08f;  // 2^-24
constexpr float kOrientBoundF = 32.0f * kF32Unit;
constexpr float kInsphereBoundF = 64.0f * kF32Unit;
constexpr float kF32Abs = 9.094947017729282e-13f;    // 2^-40
constexpr float kF32Lo = 9.5367431640625e-07f;       // 2^-20
constexpr float kF32Hi = 16777216.0f;                // 2^24
__device__ __forceinline__ bool f32_range(float v) {
  float a = fabsf(v);
  return a == 0.0f || (a >= kF32Lo && a <= kF32Hi);
}
CDR_HD D3 d3(double x, double y, double z) { return D3{x, y, z}; }

// ------------------------------------------------------------------ orient
// orient(a,b,c,d) = (b-a) . ((c-a) x (d-a)); stored tetrahedra have orient > 0.
__device__ __noinline__ int orient3d_exact(D3 a, D3 b, D3 c, D3 d) {
  ExScratch w;
  Ex2 r[3][3] = {{ex_diff(b.x, a.x), ex_diff(b.y, a.y), ex_diff(b.z, a.z)},
                 {ex_diff(c.x, a.x), ex_diff(c.y, a.y), ex_diff(c.z, a.z)},
                 {ex_diff(d.x, a.x), ex_diff(d.y, a.y), ex_diff(d.z, a.z)}};
  double out[kExCap];
  int n;
  EX_TRY(n = ex_det3(r[0], r[1], r[2], out, w));
  return ex_sign(n, out);
}

// FP64 filter, then exact arithmetic (out of line: the FP32 stage decides
// nearly every call, and one copy keeps the kernels' code small)
// The FP64 stages are kept out of line by default (smaller code at every call
// site); CDR_FP64_INLINE builds them inline (no call, no register save).
#ifdef CDR_FP64_INLINE
#define CDR_FP64_STAGE __device__ __forceinline__
#else
#define CDR_FP64_STAGE __device__ __noinline__
#endif
CDR_FP64_STAGE int orient3d_fp64(D3 a, D3 b, D3 c, D3 d) {
  double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
  double vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
  double wx = d.x - a.x, wy = d.y - a.y, wz = d.z - a.z;
  double m1 = vy * wz - vz * wy, m2 = vz * wx - vx * wz, m3 = vx * wy - vy * wx;
  double det = ux * m1 + uy * m2 + uz * m3;
  double perm = fabs(ux) * (fabs(vy * wz) + fabs(vz * wy)) +
                fabs(uy) * (fabs(vz * wx) + fabs(vx * wz)) +
                fabs(uz) * (fabs(vx * wy) + fabs(vy * wx));
  double bound = kOrientBound * perm;
  if (perm > kTinyPerm) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return orient3d_exact(a, b, c, d);
}

__device__ __forceinline__ int orient3d(D3 a, D3 b, D3 c, D3 d) {
  double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
  double vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
  double wx = d.x - a.x, wy = d.y - a.y, wz = d.z - a.z;
  {
    const float fux = __double2float_rn(ux), fuy = __double2float_rn(uy),
                fuz = __double2float_rn(uz), fvx = __double2float_rn(vx),
                fvy = __double2float_rn(vy), fvz = __double2float_rn(vz),
                fwx = __double2float_rn(wx), fwy = __double2float_rn(wy),
                fwz = __double2float_rn(wz);
    if (f32_range(fux) && f32_range(fuy) && f32_range(fuz) && f32_range(fvx) &&
        f32_range(fvy) && f32_range(fvz) && f32_range(fwx) && f32_range(fwy) &&
        f32_range(fwz)) {
      float m1 = fvy * fwz - fvz * fwy, m2 = fvz * fwx - fvx * fwz, m3 = fvx * fwy - fvy * fwx;
      float det = fux * m1 + fuy * m2 + fuz * m3;
      float perm = fabsf(fux) * (fabsf(fvy * fwz) + fabsf(fvz * fwy)) +
                   fabsf(fuy) * (fabsf(fvz * fwx) + fabsf(fvx * fwz)) +
                   fabsf(fuz) * (fabsf(fvx * fwy) + fabsf(fvy * fwx));
      float bound = kOrientBoundF * perm + kF32Abs;
      if (det > bound) return 1;
      if (-det > bound) return -1;
    }
  }
  return orient3d_fp64(a, b, c, d);
}

// ---------------------------------------------------------------- insphere
// > 0 iff e is strictly inside the circumsphere of positively oriented (a,b,c,d).
__device__ __noinline__ int insphere_exact(D3 a, D3 b, D3 c, D3 d, D3 e) {
  ExScratch w;
  const D3 P[4] = {a, b, c, d};
  Ex2 r[4][3];
  for (int i = 0; i < 4; ++i) {
    r[i][0] = ex_diff(P[i].x, e.x);
    r[i][1] = ex_diff(P[i].y, e.y);
    r[i][2] = ex_diff(P[i].z, e.z);
  }
  // -det4 = -(dl*M(a,b,c) - cl*M(a,b,d) + bl*M(a,c,d) - al*M(b,c,d))
  const int rows[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  const int liftRow[4] = {3, 2, 1, 0};
  const bool neg[4] = {true, false, true, false};
  double minor[kExCap], lift[32], prod[kExCap], total[kExCap], total2[kExCap];
  int nt = 0;
  for (int k = 0; k < 4; ++k) {
    int nm, nl, np, n2;
    EX_TRY(nm = ex_det3(r[rows[k][0]], r[rows[k][1]], r[rows[k][2]], minor, w));
    EX_TRY(nl = ex_len2(r[liftRow[k]], lift, w));
    EX_TRY(np = ex_mul(nm, minor, nl, lift, prod, w));
    if (neg[k]) ex_negate(np, prod);
    EX_TRY(n2 = ex_add(nt, total, np, prod, total2));
    for (int q = 0; q < n2; ++q) total[q] = total2[q];
    nt = n2;
  }
  return ex_sign(nt, total);
}

__device__ __forceinline__ double det3f(double ax, double ay, double az, double bx, double by,
                                        double bz, double cx, double cy, double cz,
                                        double& perm) {
  double m1 = by * cz - bz * cy, m2 = bz * cx - bx * cz, m3 = bx * cy - by * cx;
  perm = fabs(ax) * (fabs(by * cz) + fabs(bz * cy)) + fabs(ay) * (fabs(bz * cx) + fabs(bx * cz)) +
         fabs(az) * (fabs(bx * cy) + fabs(by * cx));
  return ax * m1 + ay * m2 + az * m3;
}

__device__ __forceinline__ float det3f32(float ax, float ay, float az, float bx, float by,
                                         float bz, float cx, float cy, float cz, float& perm) {
  float m1 = by * cz - bz * cy, m2 = bz * cx - bx * cz, m3 = bx * cy - by * cx;
  perm = fabsf(ax) * (fabsf(by * cz) + fabsf(bz * cy)) +
         fabsf(ay) * (fabsf(bz * cx) + fabsf(bx * cz)) +
         fabsf(az) * (fabsf(bx * cy) + fabsf(by * cx));
  return ax * m1 + ay * m2 + az * m3;
}

CDR_FP64_STAGE int insphere_fp64(D3 a, D3 b, D3 c, D3 d, D3 e) {
  double ax = a.x - e.x, ay = a.y - e.y, az = a.z - e.z;
  double bx = b.x - e.x, by = b.y - e.y, bz = b.z - e.z;
  double cx = c.x - e.x, cy = c.y - e.y, cz = c.z - e.z;
  double dx = d.x - e.x, dy = d.y - e.y, dz = d.z - e.z;
  double al = ax * ax + ay * ay + az * az;
  double bl = bx * bx + by * by + bz * bz;
  double cl = cx * cx + cy * cy + cz * cz;
  double dl = dx * dx + dy * dy + dz * dz;
  double p1, p2, p3, p4;
  double m1 = det3f(ax, ay, az, bx, by, bz, cx, cy, cz, p1);
  double m2 = det3f(ax, ay, az, bx, by, bz, dx, dy, dz, p2);
  double m3 = det3f(ax, ay, az, cx, cy, cz, dx, dy, dz, p3);
  double m4 = det3f(bx, by, bz, cx, cy, cz, dx, dy, dz, p4);
  // the lifted 4x4 determinant along its lift column, negated (inside > 0)
  double det = -(dl * m1 - cl * m2 + bl * m3 - al * m4);
  double perm = dl * p1 + cl * p2 + bl * p3 + al * p4;
  double bound = kInsphereBound * perm;
  if (perm > kTinyPerm) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return insphere_exact(a, b, c, d, e);
}

__device__ __forceinline__ int insphere(D3 a, D3 b, D3 c, D3 d, D3 e) {
  double ax = a.x - e.x, ay = a.y - e.y, az = a.z - e.z;
  double bx = b.x - e.x, by = b.y - e.y, bz = b.z - e.z;
  double cx = c.x - e.x, cy = c.y - e.y, cz = c.z - e.z;
  double dx = d.x - e.x, dy = d.y - e.y, dz = d.z - e.z;
  {
    const float fax = __double2float_rn(ax), fay = __double2float_rn(ay),
                faz = __double2float_rn(az), fbx = __double2float_rn(bx),
                fby = __double2float_rn(by), fbz = __double2float_rn(bz),
                fcx = __double2float_rn(cx), fcy = __double2float_rn(cy),
                fcz = __double2float_rn(cz), fdx = __double2float_rn(dx),
                fdy = __double2float_rn(dy), fdz = __double2float_rn(dz);
    if (f32_range(fax) && f32_range(fay) && f32_range(faz) && f32_range(fbx) &&
        f32_range(fby) && f32_range(fbz) && f32_range(fcx) && f32_range(fcy) &&
        f32_range(fcz) && f32_range(fdx) && f32_range(fdy) && f32_range(fdz)) {
      float al = fax * fax + fay * fay + faz * faz;
      float bl = fbx * fbx + fby * fby + fbz * fbz;
      float cl = fcx * fcx + fcy * fcy + fcz * fcz;
      float dl = fdx * fdx + fdy * fdy + fdz * fdz;
      float p1, p2, p3, p4;
      float m1 = det3f32(fax, fay, faz, fbx, fby, fbz, fcx, fcy, fcz, p1);
      float m2 = det3f32(fax, fay, faz, fbx, fby, fbz, fdx, fdy, fdz, p2);
      float m3 = det3f32(fax, fay, faz, fcx, fcy, fcz, fdx, fdy, fdz, p3);
      float m4 = det3f32(fbx, fby, fbz, fcx, fcy, fcz, fdx, fdy, fdz, p4);
      float det = -(dl * m1 - cl * m2 + bl * m3 - al * m4);
      float perm = dl * p1 + cl * p2 + bl * p3 + al * p4;
      float bound = kInsphereBoundF * perm + kF32Abs;
      if (det > bound) return 1;
      if (-det > bound) return -1;
    }
  }
  return insphere_fp64(a, b, c, d, e);
}

// --------------------------------------------------------------- diametral
// (a-p).(b-p): negative iff p is strictly inside the diametral sphere of ab.
__device__ __noinline__ int diametral_exact(D3 a, D3 b, D3 p) {
  ExScratch w;
  Ex2 ra[3] = {ex_diff(a.x, p.x), ex_diff(a.y, p.y), ex_diff(a.z, p.z)};
  Ex2 rb[3] = {ex_diff(b.x, p.x), ex_diff(b.y, p.y), ex_diff(b.z, p.z)};
  double acc[32], acc2[32], pr[8];
  int nacc = 0;
  for (int k = 0; k < 3; ++k) {
    int n, n2;
    EX_TRY(n = ex_mul(ra[k].n, ra[k].c, rb[k].n, rb[k].c, pr, w));
    EX_TRY(n2 = ex_add(nacc, acc, n, pr, acc2));
    for (int q = 0; q < n2; ++q) acc[q] = acc2[q];
    nacc = n2;
  }
  return ex_sign(nacc, acc);
}

__device__ __noinline__ int diametral(D3 a, D3 b, D3 p) {
  double ax = a.x - p.x, ay = a.y - p.y, az = a.z - p.z;
  double bx = b.x - p.x, by = b.y - p.y, bz = b.z - p.z;
  double v = ax * bx + ay * by + az * bz;
  double perm = fabs(ax * bx) + fabs(ay * by) + fabs(az * bz);
  double bound = kDiamBound * perm;
  if (perm > kTinyPerm) {
    if (v > bound) return 1;
    if (-v > bound) return -1;
  }
  return diametral_exact(a, b, p);
}

// -------------------------------------------------------------- equatorial
// |w|^2|n|^2 - w.m with u=b-a, v=c-a, w=p-a, n=u x v, m=|u|^2 (v x n)+|v|^2 (n x u).
// Negative iff p is strictly inside the equatorial sphere of triangle abc.
__device__ __noinline__ int equatorial_exact(D3 a, D3 b, D3 c, D3 p) {
  ExScratch w;
  Ex2 u[3] = {ex_diff(b.x, a.x), ex_diff(b.y, a.y), ex_diff(b.z, a.z)};
  Ex2 v[3] = {ex_diff(c.x, a.x), ex_diff(c.y, a.y), ex_diff(c.z, a.z)};
  Ex2 wv[3] = {ex_diff(p.x, a.x), ex_diff(p.y, a.y), ex_diff(p.z, a.z)};
  const int I[3][2] = {{1, 2}, {2, 0}, {0, 1}};
  double n[3][16];
  int nn[3];
  for (int k = 0; k < 3; ++k) {
    int i = I[k][0], j = I[k][1];
    EX_TRY(nn[k] = ex_cross(u[i], v[j], u[j], v[i], n[k], w));
  }
  double LU[32], LV[32], LW[32], LN[kExCap], t1[kExCap], t2[kExCap];
  int nlu, nlv, nlw, nln = 0;
  EX_TRY(nlu = ex_len2(u, LU, w));
  EX_TRY(nlv = ex_len2(v, LV, w));
  EX_TRY(nlw = ex_len2(wv, LW, w));
  for (int k = 0; k < 3; ++k) {
    int q, q2;
    EX_TRY(q = ex_mul(nn[k], n[k], nn[k], n[k], t1, w));
    EX_TRY(q2 = ex_add(nln, LN, q, t1, t2));
    for (int z = 0; z < q2; ++z) LN[z] = t2[z];
    nln = q2;
  }
  // D = LW*LN - sum_k w_k * (LU*(v x n)_k + LV*(n x u)_k)
  double D[kExCap], D2[kExCap], A[kExCap], Bv[kExCap], vn[kExCap], nu[kExCap], m[kExCap];
  int nD;
  EX_TRY(nD = ex_mul(nlw, LW, nln, LN, D, w));
  for (int k = 0; k < 3; ++k) {
    int i = I[k][0], j = I[k][1];
    int na, nb, nvn, nnu, nm, q, q2;
    // (v x n)_k = v_i n_j - v_j n_i
    EX_TRY(na = ex_mul(v[i].n, v[i].c, nn[j], n[j], A, w));
    EX_TRY(nb = ex_mul(v[j].n, v[j].c, nn[i], n[i], Bv, w));
    ex_negate(nb, Bv);
    EX_TRY(nvn = ex_add(na, A, nb, Bv, vn));
    // (n x u)_k = n_i u_j - n_j u_i
    EX_TRY(na = ex_mul(nn[i], n[i], u[j].n, u[j].c, A, w));
    EX_TRY(nb = ex_mul(nn[j], n[j], u[i].n, u[i].c, Bv, w));
    ex_negate(nb, Bv);
    EX_TRY(nnu = ex_add(na, A, nb, Bv, nu));
    EX_TRY(na = ex_mul(nlu, LU, nvn, vn, A, w));
    EX_TRY(nb = ex_mul(nlv, LV, nnu, nu, Bv, w));
    EX_TRY(nm = ex_add(na, A, nb, Bv, m));
    EX_TRY(q = ex_mul(wv[k].n, wv[k].c, nm, m, t1, w));
    ex_negate(q, t1);
    EX_TRY(q2 = ex_add(nD, D, q, t1, D2));
    for (int z = 0; z < q2; ++z) D[z] = D2[z];
    nD = q2;
  }
  return ex_sign(nD, D);
}

__device__ __noinline__ int equatorial(D3 a, D3 b, D3 c, D3 p) {
  double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
  double vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
  double wx = p.x - a.x, wy = p.y - a.y, wz = p.z - a.z;
  double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  double Nx = fabs(uy * vz) + fabs(uz * vy), Ny = fabs(uz * vx) + fabs(ux * vz),
         Nz = fabs(ux * vy) + fabs(uy * vx);
  double lu = ux * ux + uy * uy + uz * uz, lv = vx * vx + vy * vy + vz * vz;
  double lw = wx * wx + wy * wy + wz * wz, ln = nx * nx + ny * ny + nz * nz;
  double Ln = Nx * Nx + Ny * Ny + Nz * Nz;
  double vnx = vy * nz - vz * ny, vny = vz * nx - vx * nz, vnz = vx * ny - vy * nx;
  double VNx = fabs(vy) * Nz + fabs(vz) * Ny, VNy = fabs(vz) * Nx + fabs(vx) * Nz,
         VNz = fabs(vx) * Ny + fabs(vy) * Nx;
  double nux = ny * uz - nz * uy, nuy = nz * ux - nx * uz, nuz = nx * uy - ny * ux;
  double NUx = Ny * fabs(uz) + Nz * fabs(uy), NUy = Nz * fabs(ux) + Nx * fabs(uz),
         NUz = Nx * fabs(uy) + Ny * fabs(ux);
  double mx = lu * vnx + lv * nux, my = lu * vny + lv * nuy, mz = lu * vnz + lv * nuz;
  double Mx = lu * VNx + lv * NUx, My = lu * VNy + lv * NUy, Mz = lu * VNz + lv * NUz;
  double D = lw * ln - (wx * mx + wy * my + wz * mz);
  double perm = lw * Ln + (fabs(wx) * Mx + fabs(wy) * My + fabs(wz) * Mz);
  double bound = kEquatBound * perm;
  if (perm > kTinyPerm) {
    if (D > bound) return 1;
    if (-D > bound) return -1;
  }
  return equatorial_exact(a, b, c, p);
}

// --------------------------------------------------- fixed-order formulas
// Evaluated one IEEE rounding per operation, in the written order, with no
// fused multiply-add, so that the result is bit-identical on any IEEE machine.
__device__ __forceinline__ double mulr(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double subr(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double divr(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dot3r(double ax, double ay, double az, double bx, double by,
                                        double bz) {
  return addr(addr(mulr(ax, bx), mulr(ay, by)), mulr(az, bz));
}
__device__ __forceinline__ double crossr(double a1, double b2, double a2, double b1) {
  return subr(mulr(a1, b2), mulr(a2, b1));
}

// subsegment midpoint (a + b) * 0.5
__device__ __forceinline__ D3 midpoint_fixed(D3 a, D3 b) {
  return D3{mulr(addr(a.x, b.x), 0.5), mulr(addr(a.y, b.y), 0.5), mulr(addr(a.z, b.z), 0.5)};
}

// tetrahedron circumcentre c = a + N / (2 u.(v x w)), vertices in ascending id order;
// off receives c - a. Returns false if degenerate (zero denominator / not finite).
__device__ __forceinline__ bool tet_circumcenter_fixed(D3 a, D3 b, D3 c, D3 d, D3& out,
                                                       D3& off) {
  double ux = subr(b.x, a.x), uy = subr(b.y, a.y), uz = subr(b.z, a.z);
  double vx = subr(c.x, a.x), vy = subr(c.y, a.y), vz = subr(c.z, a.z);
  double wx = subr(d.x, a.x), wy = subr(d.y, a.y), wz = subr(d.z, a.z);
  double lu = dot3r(ux, uy, uz, ux, uy, uz);
  double lv = dot3r(vx, vy, vz, vx, vy, vz);
  double lw = dot3r(wx, wy, wz, wx, wy, wz);
  double vwx = crossr(vy, wz, vz, wy), vwy = crossr(vz, wx, vx, wz), vwz = crossr(vx, wy, vy, wx);
  double wux = crossr(wy, uz, wz, uy), wuy = crossr(wz, ux, wx, uz), wuz = crossr(wx, uy, wy, ux);
  double uvx = crossr(uy, vz, uz, vy), uvy = crossr(uz, vx, ux, vz), uvz = crossr(ux, vy, uy, vx);
  double det = dot3r(ux, uy, uz, vwx, vwy, vwz);
  double den = mulr(2.0, det);
  double nx = addr(addr(mulr(lu, vwx), mulr(lv, wux)), mulr(lw, uvx));
  double ny = addr(addr(mulr(lu, vwy), mulr(lv, wuy)), mulr(lw, uvy));
  double nz = addr(addr(mulr(lu, vwz), mulr(lv, wuz)), mulr(lw, uvz));
  off.x = divr(nx, den);
  off.y = divr(ny, den);
  off.z = divr(nz, den);
  out.x = addr(a.x, off.x);
  out.y = addr(a.y, off.y);
  out.z = addr(a.z, off.z);
  return den != 0.0 && isfinite(out.x) && isfinite(out.y) && isfinite(out.z);
}

// subface circumcentre c = a + (|u|^2 (v x n) + |v|^2 (n x u)) / (2 |n|^2)
__device__ __forceinline__ bool tri_circumcenter_fixed(D3 a, D3 b, D3 c, D3& out) {
  double ux = subr(b.x, a.x), uy = subr(b.y, a.y), uz = subr(b.z, a.z);
  double vx = subr(c.x, a.x), vy = subr(c.y, a.y), vz = subr(c.z, a.z);
  double nx = crossr(uy, vz, uz, vy), ny = crossr(uz, vx, ux, vz), nz = crossr(ux, vy, uy, vx);
  double lu = dot3r(ux, uy, uz, ux, uy, uz);
  double lv = dot3r(vx, vy, vz, vx, vy, vz);
  double ln = dot3r(nx, ny, nz, nx, ny, nz);
  double vnx = crossr(vy, nz, vz, ny), vny = crossr(vz, nx, vx, nz), vnz = crossr(vx, ny, vy, nx);
  double nux = crossr(ny, uz, nz, uy), nuy = crossr(nz, ux, nx, uz), nuz = crossr(nx, uy, ny, ux);
  double mx = addr(mulr(lu, vnx), mulr(lv, nux));
  double my = addr(mulr(lu, vny), mulr(lv, nuy));
  double mz = addr(mulr(lu, vnz), mulr(lv, nuz));
  double den = mulr(2.0, ln);
  out.x = addr(a.x, divr(mx, den));
  out.y = addr(a.y, divr(my, den));
  out.z = addr(a.z, divr(mz, den));
  return den != 0.0 && isfinite(out.x) && isfinite(out.y) && isfinite(out.z);
}

__device__ __forceinline__ double dist2_fixed(D3 a, D3 b) {
  double dx = subr(a.x, b.x), dy = subr(a.y, b.y), dz = subr(a.z, b.z);
  return dot3r(dx, dy, dz, dx, dy, dz);
}

// bad tetrahedron: R^2 / l_min^2 > B^2 (vertices in ascending id order; edges ab,
// ac, ad, bc, bd, cd). A degenerate circumcentre counts as bad.
__device__ __forceinline__ bool tet_bad_fixed(D3 a, D3 b, D3 c, D3 d, double B) {
  D3 cc, o;
  if (!tet_circumcenter_fixed(a, b, c, d, cc, o)) return true;
  double r2 = dot3r(o.x, o.y, o.z, o.x, o.y, o.z);
  double l2 = dist2_fixed(b, a), t;
  t = dist2_fixed(c, a); if (t < l2) l2 = t;
  t = dist2_fixed(d, a); if (t < l2) l2 = t;
  t = dist2_fixed(c, b); if (t < l2) l2 = t;
  t = dist2_fixed(d, b); if (t < l2) l2 = t;
  t = dist2_fixed(d, c); if (t < l2) l2 = t;
  return divr(r2, l2) > mulr(B, B);
}

// One item of the predicate batch probe: q holds the points a, b, c, d, e as
// (x, y, z) in doubles 0..14 (for kind 7 the bound B sits in double 12). Writes
// the sign or flag to *sg and the point of kinds 4..6 to *o (zero otherwise).
// Both batch entry points run their items through this one function.
__device__ __forceinline__ void eval_item(int kind, const double* q, int* sg, D3* o) {
  D3 a{q[0], q[1], q[2]}, b{q[3], q[4], q[5]}, c{q[6], q[7], q[8]}, d{q[9], q[10], q[11]},
      e{q[12], q[13], q[14]};
  int s = 0;
  D3 r{0, 0, 0};
  switch (kind) {
    case 0: s = orient3d(a, b, c, d); break;
    case 1: s = insphere(a, b, c, d, e); break;
    case 2: s = diametral(a, b, c); break;
    case 3: s = equatorial(a, b, c, d); break;
    case 4: {
      D3 off;
      s = tet_circumcenter_fixed(a, b, c, d, r, off) ? 1 : 0;
      break;
    }
    case 5: s = tri_circumcenter_fixed(a, b, c, r) ? 1 : 0; break;
    case 6: r = midpoint_fixed(a, b); s = 1; break;
    case 7: s = tet_bad_fixed(a, b, c, d, q[12]) ? 1 : 0; break;
    case 8: s = orient3d_exact(a, b, c, d); break;
    case 9: s = insphere_exact(a, b, c, d, e); break;
    case 10: s = equatorial_exact(a, b, c, d); break;
    case 11: s = diametral_exact(a, b, c); break;
  }
  *sg = s;
  *o = r;
}

// candidate priority: SplitMix64's output function chained over sorted ids
CDR_HD uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
CDR_HD uint64_t prio_hash(int cls, const int* ids, int n) {
  uint64_t h = 0x9E3779B97F4A7C15ULL * (uint64_t)(cls + 1);
  for (int i = 0; i < n; ++i) h = mix64(h ^ (uint64_t)(uint32_t)ids[i]);
  return h;
}
// An element's priority: the same chain over the bit patterns of its vertices'
// coordinates (x, y, z per vertex, ascending vertex id), so that it does not
// depend on the absolute ids (an instance orders its candidates alike whether
// it is refined alone or beside other instances in one mesh).
__device__ __forceinline__ uint64_t prio_hash_step(uint64_t h, double c) {
  return mix64(h ^ (uint64_t)__double_as_longlong(c));
}

}  // namespace cdr
