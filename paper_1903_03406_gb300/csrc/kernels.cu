// Refinement kernels for sm_103a.
//
// One round (Sec. 2 of Chen & Tan, I3D 2019) is: classify elements, order the
// candidates of the first non-empty class by predetermined priority, compute
// splitting points (k_split), locate them (k_locate), grow every point's
// Delaunay region with one warp per point and mark every touched element with
// atomicMin of the point's priority (k_grow1 / k_grow2: the "grow" step with
// work proportional to region size), keep the points that hold every mark
// (k_select: the "blast" step), and insert the kept points concurrently,
// re-linking the new stars to the rest of the mesh (k_insert).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "mesh.cuh"
#include "predicates.cuh"

namespace cdr {

#define FULLMASK 0xffffffffu

// grid for n items of `block` threads, at most 32 blocks per SM (152 SMs);
// kernels stride over the rest
static inline int grid_for(long n, int block) {
  long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

// Checked build (CDR_CHECKED): every mesh-array index is bounds-checked; a bad
// index is recorded (site = source line, index, bound) and replaced by 0 so
// that nothing is read or written out of bounds.
#ifdef CDR_CHECKED
static __device__ int g_chk[4];
__device__ __noinline__ int cdr_bad_index(int site, long long idx, int cap) {
  if (atomicCAS(&g_chk[0], 0, 1) == 0) {
    g_chk[1] = site;
    g_chk[2] = (int)idx;
    g_chk[3] = cap;
  }
  return 0;
}
#define CKI(idx, cap) (((unsigned long long)(long long)(idx) < (unsigned long long)(cap)) ? (idx) : cdr_bad_index(__LINE__, (long long)(idx), (cap)))
// a neighbour link (tet << 2 | face) or -1 whose tet is below `bound`
#define CKL(link, bound) do { int l_ = (link); if (l_ < -1 || (l_ >= 0 && (l_ >> 2) >= (bound))) cdr_bad_index(__LINE__, (long long)l_, (bound)); } while (0)
#else
#define CKI(idx, cap) (idx)
#define CKL(link, bound) do { } while (0)
#endif

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int geti(const int4& a, int k) {
  return k == 0 ? a.x : (k == 1 ? a.y : (k == 2 ? a.z : a.w));
}
__device__ __forceinline__ void seti(int4& a, int k, int v) {
  if (k == 0) a.x = v;
  else if (k == 1) a.y = v;
  else if (k == 2) a.z = v;
  else a.w = v;
}
__device__ __forceinline__ int vid(int x) { return x & kVidMask; }
__device__ __forceinline__ D3 vtx(const DevMesh& m, int v) {
  V4 q = m.V[CKI(v, m.capV)];
  return D3{q.x, q.y, q.z};
}
__device__ __forceinline__ TetRec ld_tet(const DevMesh& m, int t) { return m.T[CKI(t, m.capT)]; }
__device__ __forceinline__ int* tet_n_ptr(const DevMesh& m, int t) { return &m.T[CKI(t, m.capT)].n.x; }
__device__ __forceinline__ int* tet_v_ptr(const DevMesh& m, int t) { return &m.T[CKI(t, m.capT)].v.x; }
__device__ __forceinline__ int* ts_ptr(const DevMesh& m, int t) { return &m.TS[CKI(t, m.capT)].x; }
__device__ __forceinline__ int* sn_ptr(const DevMesh& m, int s) { return &m.SN[CKI(s, m.capS)].x; }

// edge e of a tetrahedron: 0:(0,1) 1:(0,2) 2:(0,3) 3:(1,2) 4:(1,3) 5:(2,3)
__device__ __forceinline__ int edge_i(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__device__ __forceinline__ int edge_j(int e) { return e < 3 ? e + 1 : (e < 5 ? e - 1 : 3); }
__device__ __forceinline__ int edge_of(int i, int j) {
  int a = min(i, j), b = max(i, j);
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}
__device__ __forceinline__ bool edge_bit(const int4& v, int e) {
  return (geti(v, e >> 1) >> (29 + (e & 1))) & 1;
}
__device__ __forceinline__ bool face_sub(const int4& v, int f) { return (geti(v, f) >> kSubBit) & 1; }

__device__ __forceinline__ void sort3(int& a, int& b, int& c) {
  int t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
}
__device__ __forceinline__ void sort4(int* s) {
  for (int i = 1; i < 4; ++i)
    for (int j = i; j > 0 && s[j - 1] > s[j]; --j) {
      int t = s[j];
      s[j] = s[j - 1];
      s[j - 1] = t;
    }
}
__device__ __forceinline__ bool lt3(int a0, int a1, int a2, int b0, int b1, int b2) {
  if (a0 != b0) return a0 < b0;
  if (a1 != b1) return a1 < b1;
  return a2 < b2;
}

// subsegment hash: key (min << 32 | max)
__device__ __forceinline__ unsigned long long ekey(int a, int b) {
  unsigned u = (unsigned)min(a, b), w = (unsigned)max(a, b);
  return ((unsigned long long)u << 32) | w;
}
__device__ int hash_lookup(const DevMesh& m, unsigned long long k) {
  unsigned h = (unsigned)mix64(k) & (unsigned)m.hmask;
  for (int it = 0; it <= m.hmask; ++it) {
    unsigned long long e = m.HK[h];
    if (e == k) return m.HV[h];
    if (e == ~0ULL) return -1;
    h = (h + 1) & (unsigned)m.hmask;
  }
  return -1;
}
__device__ void hash_insert(const DevMesh& m, unsigned long long k, int v) {
  unsigned h = (unsigned)mix64(k) & (unsigned)m.hmask;
  for (int it = 0; it <= m.hmask; ++it) {
    unsigned long long old = atomicCAS(&m.HK[h], ~0ULL, k);
    if (old == ~0ULL || old == k) {
      m.HV[h] = v;
      return;
    }
    h = (h + 1) & (unsigned)m.hmask;
  }
}

// orient of tetrahedron r with vertex f replaced by p, from its 4 vertices
__device__ __forceinline__ int orient_rep4(const D3* c, int f, D3 p) {
  return orient3d(f == 0 ? p : c[0], f == 1 ? p : c[1], f == 2 ? p : c[2], f == 3 ? p : c[3]);
}
__device__ __forceinline__ int orient_rep(const DevMesh& m, const TetRec& r, int f, D3 p) {
  D3 a = f == 0 ? p : vtx(m, vid(r.v.x));
  D3 b = f == 1 ? p : vtx(m, vid(r.v.y));
  D3 c = f == 2 ? p : vtx(m, vid(r.v.z));
  D3 d = f == 3 ? p : vtx(m, vid(r.v.w));
  return orient3d(a, b, c, d);
}
__device__ __forceinline__ bool tet_in_sphere(const DevMesh& m, const TetRec& r, D3 p) {
  return insphere(vtx(m, vid(r.v.x)), vtx(m, vid(r.v.y)), vtx(m, vid(r.v.z)), vtx(m, vid(r.v.w)),
                  p) > 0;
}
// subface winding seen from the facet reference point
__device__ __forceinline__ int sf_wind(const DevMesh& m, int4 S) {
  V4 q = m.FQ[S.w];
  return orient3d(vtx(m, S.x), vtx(m, S.y), vtx(m, S.z), D3{q.x, q.y, q.z});
}
__device__ __forceinline__ int sf_orient_rep(const DevMesh& m, int4 S, int k, D3 p) {
  V4 q = m.FQ[S.w];
  D3 a = k == 0 ? p : vtx(m, S.x);
  D3 b = k == 1 ? p : vtx(m, S.y);
  D3 c = k == 2 ? p : vtx(m, S.z);
  return orient3d(a, b, c, D3{q.x, q.y, q.z});
}
__device__ __forceinline__ bool sf_incircle(const DevMesh& m, int4 S, D3 p) {
  V4 q = m.FQ[S.w];
  D3 Q{q.x, q.y, q.z};
  int o = insphere(vtx(m, S.x), vtx(m, S.y), vtx(m, S.z), Q, p);
  return o * orient3d(vtx(m, S.x), vtx(m, S.y), vtx(m, S.z), Q) > 0;
}

__device__ __forceinline__ void set_status(const DevRound& r, int i, int outcome, int reason) {
  r.status[i] = outcome | (reason << 8);
}
// class and instance of candidate i; instance of vertex v; per-instance bound
// and shortest-edge guard
__device__ __forceinline__ int cls_of(const DevRound& r, int i) {
  return r.ccls ? (int)r.ccls[i] : r.cls;
}
__device__ __forceinline__ int inst_of(const DevRound& r, int i) {
  return r.cinst ? r.cinst[i] : 0;
}
__device__ __forceinline__ int vinst(const DevMesh& m, int v) { return m.Vinst ? m.Vinst[v] : 0; }
__device__ __forceinline__ double bound_of(const DevMesh& m, double B, int inst) {
  return m.instB ? m.instB[inst] : B;
}
__device__ __forceinline__ double guard2_of(const DevMesh& m, int inst) {
  return m.instG2 ? m.instG2[inst] : m.guard2;
}

// ================================================================= create
__global__ void k_init_tets(DevMesh m, const int4* tets, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    TetRec r;
    r.v = tets[i];
    r.n = make_int4(-1, -1, -1, -1);
    m.T[CKI(i, m.capT)] = r;
    m.TS[CKI(i, m.capT)] = make_int4(-1, -1, -1, -1);
    m.Tflag[CKI(i, m.capT)] = 0;
    m.Tmark[CKI(i, m.capT)] = ~0ULL;
    m.Tseed[CKI(i, m.capT)] = ~0ULL;
    m.Tfwd[CKI(i, m.capT)] = -1;
  }
}

__global__ void k_face_keys(DevMesh m, unsigned long long* hi, unsigned int* lo, int* val) {
  int n = m.nT * 4;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int t = i >> 2, f = i & 3;
    int4 v = m.T[CKI(t, m.capT)].v;
    int w[3], k = 0;
    for (int j = 0; j < 4; ++j)
      if (j != f) w[k++] = vid(geti(v, j));
    sort3(w[0], w[1], w[2]);
    hi[i] = ((unsigned long long)(unsigned)w[0] << 32) | (unsigned)w[1];
    lo[i] = (unsigned)w[2];
    if (val) val[i] = i;
  }
}

__global__ void k_pair_faces(DevMesh m, const unsigned long long* hi, const unsigned int* lo,
                             const int* val, int n, int* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool eqn = i + 1 < n && hi[i + 1] == hi[i] && lo[i + 1] == lo[i];
    bool eqp = i > 0 && hi[i - 1] == hi[i] && lo[i - 1] == lo[i];
    if (eqn && eqp) atomicOr(err, 1);  // a face shared by three tetrahedra
    if (eqn) {
      int a = val[i], b = val[i + 1];
      CKL(a, m.nT);
      CKL(b, m.nT);
      tet_n_ptr(m, a >> 2)[a & 3] = b;
      tet_n_ptr(m, b >> 2)[b & 3] = a;
    }
  }
}

__device__ int face_lower_bound(const unsigned long long* hi, const unsigned int* lo, int n,
                                unsigned long long h, unsigned l) {
  int a = 0, b = n;
  while (a < b) {
    int c = (a + b) >> 1;
    if (hi[c] < h || (hi[c] == h && lo[c] < l)) a = c + 1;
    else b = c;
  }
  return a;
}

__global__ void k_label_subfaces(DevMesh m, const int4* tris, int n, const unsigned long long* hi,
                                 const unsigned int* lo, const int* val, int nfaces, int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int4 S = tris[s];
    m.SV[CKI(s, m.capS)] = S;
    m.SN[CKI(s, m.capS)] = make_int4(-1, -1, -1, -1);
    m.Sflag[CKI(s, m.capS)] = 0;
    m.Smust[CKI(s, m.capS)] = 0;
    m.Smark[CKI(s, m.capS)] = ~0ULL;
    int a = S.x, b = S.y, c = S.z;
    if (a < 0 || b < 0 || c < 0 || a >= m.nV || b >= m.nV || c >= m.nV || S.w < 0 || S.w >= m.nF) {
      atomicOr(err, 8);
      continue;
    }
    sort3(a, b, c);
    unsigned long long h = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
    int j = face_lower_bound(hi, lo, nfaces, h, (unsigned)c);
    if (j >= nfaces || hi[j] != h || lo[j] != (unsigned)c) {
      atomicOr(err, 8);  // label is not a mesh face
      continue;
    }
    int first = val[j];
    m.SN[CKI(s, m.capS)].w = first;
    for (int q = j; q < nfaces && q < j + 2 && hi[q] == h && lo[q] == (unsigned)c; ++q) {
      int tf = val[q];
      ts_ptr(m, tf >> 2)[tf & 3] = s;
      atomicOr(&tet_v_ptr(m, tf >> 2)[tf & 3], 1 << kSubBit);
    }
  }
}

__global__ void k_subface_edge_keys(DevMesh m, unsigned long long* hi, unsigned int* lo, int* val) {
  int n = m.nS * 3;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int s = i / 3, k = i % 3;
    int4 S = m.SV[CKI(s, m.capS)];
    int u = geti(S, (k + 1) % 3), w = geti(S, (k + 2) % 3);
    if (u > w) { int t = u; u = w; w = t; }
    hi[i] = ((unsigned long long)(unsigned)u << 32) | (unsigned)w;
    lo[i] = (unsigned)S.w;
    if (val) val[i] = i;
  }
}

__global__ void k_pair_subface_edges(DevMesh m, const unsigned long long* hi,
                                     const unsigned int* lo, const int* val, int n, int* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool eqn = i + 1 < n && hi[i + 1] == hi[i] && lo[i + 1] == lo[i];
    bool eqp = i > 0 && hi[i - 1] == hi[i] && lo[i - 1] == lo[i];
    if (eqn && eqp) atomicOr(err, 16);  // three subfaces of one facet on an edge
    bool isseg = hash_lookup(m, hi[i]) >= 0;
    if (!eqn && !eqp && !isseg) atomicOr(err, 32);  // open facet edge that is not a segment
    if (eqn && !isseg) {
      int a = val[i], b = val[i + 1];  // subface * 3 + edge
      sn_ptr(m, a / 3)[a % 3] = b / 3;
      sn_ptr(m, b / 3)[b % 3] = a / 3;
    }
  }
}

__global__ void k_hash_clear(DevMesh m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= m.hmask; i += gridDim.x * blockDim.x) {
    m.HK[i] = ~0ULL;
    m.HV[i] = -1;
  }
}
__global__ void k_hash_insert_subsegs(DevMesh m, int g0, int g1) {
  for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += gridDim.x * blockDim.x) {
    if (m.Gflag[CKI(g, m.capG)] & F_DEAD) continue;
    int4 G = m.GV[CKI(g, m.capG)];
    hash_insert(m, ekey(G.x, G.y), g);
  }
}
__global__ void k_mark_edges(DevMesh m) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x) {
    if (m.Tflag[CKI(t, m.capT)] & F_DEAD) continue;
    int4 v = m.T[CKI(t, m.capT)].v;
    for (int e = 0; e < 6; ++e) {
      int a = vid(geti(v, edge_i(e))), b = vid(geti(v, edge_j(e)));
      int g = hash_lookup(m, ekey(a, b));
      if (g >= 0) {
        atomicOr(&tet_v_ptr(m, t)[e >> 1], 1 << (29 + (e & 1)));
        m.GV[CKI(g, m.capG)].w = t;
      }
    }
  }
}
__global__ void k_check_create(DevMesh m, int* err) {
  int n = m.nT + m.nG;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < m.nT) {
      TetRec r = m.T[CKI(i, m.capT)];
      int a = vid(r.v.x), b = vid(r.v.y), c = vid(r.v.z), d = vid(r.v.w);
      if (orient3d(vtx(m, a), vtx(m, b), vtx(m, c), vtx(m, d)) <= 0) atomicOr(err, 2);
      for (int f = 0; f < 4; ++f)
        if (geti(r.n, f) < 0 && !face_sub(r.v, f)) atomicOr(err, 4);  // hull face not a subface
    } else {
      int g = i - m.nT;
      if (m.GV[CKI(g, m.capG)].w < 0) atomicOr(err, 64);  // subsegment label is not a mesh edge
    }
  }
}
__global__ void k_recompute_bad(DevMesh m, double B) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x) {
    uint8_t f = m.Tflag[CKI(t, m.capT)];
    if (f & F_DEAD) continue;
    int4 v = m.T[CKI(t, m.capT)].v;
    int s[4] = {vid(v.x), vid(v.y), vid(v.z), vid(v.w)};
    sort4(s);
    const double Bt = bound_of(m, B, vinst(m, s[0]));
    bool bad = tet_bad_fixed(vtx(m, s[0]), vtx(m, s[1]), vtx(m, s[2]), vtx(m, s[3]), Bt);
    m.Tflag[CKI(t, m.capT)] = bad ? (f | F_BAD) : (f & ~F_BAD);
    m.candT[CKI(t, m.capT)] = (bad && !(f & F_UNSPL)) ? 1 : 0;
  }
}

// ============================================================ classification
// Ring of tetrahedra around a subsegment edge, starting from a live tet that
// contains it. Calls visit(tet record) for each tet. Returns false if the
// start tet is invalid or the ring is longer than the step limit.
template <class F>
__device__ bool edge_ring(const DevMesh& m, int t0, int a, int b, F visit) {
  if (t0 < 0 || t0 >= m.nT || (m.Tflag[CKI(t0, m.capT)] & F_DEAD)) return false;
  TetRec r0 = ld_tet(m, t0);
  int ia = -1, ib = -1;
  for (int k = 0; k < 4; ++k) {
    int x = vid(geti(r0.v, k));
    if (x == a) ia = k;
    if (x == b) ib = k;
  }
  if (ia < 0 || ib < 0) return false;
  int c = -1, d = -1;
  for (int k = 0; k < 4; ++k)
    if (k != ia && k != ib) (c < 0 ? c : d) = k;
  visit(t0, r0);
  // two directions: leave through the face opposite d (holding vertex c), then
  // opposite c (holding d) if the first direction hit the hull
  for (int dir = 0; dir < 2; ++dir) {
    int L = dir == 0 ? d : c;
    int z = vid(geti(r0.v, dir == 0 ? c : d));
    int cur = t0;
    TetRec rc = r0;
    for (int it = 0; it < 4096; ++it) {
      int n = geti(rc.n, L);
      if (n < 0) break;  // hull: try the other direction
      int nt = n >> 2;
      if (nt == t0) return true;  // closed ring
      rc = ld_tet(m, nt);
      int zpos = -1;
      for (int k = 0; k < 4; ++k)
        if (vid(geti(rc.v, k)) == z) zpos = k;
      if (zpos < 0) return false;
      visit(nt, rc);
      z = vid(geti(rc.v, n & 3));
      L = zpos;
      cur = nt;
    }
    if (dir == 1) return true;
  }
  return true;
}

// Classification (Sec. 2's split order: encroached subsegments, encroached
// subfaces, bad tetrahedra). Incremental: only subsegments and subfaces marked
// dirty (created or touched by the last round, or flagged since) are tested;
// tetrahedra get their flag when they are created or retired. full: test all.
// add: when not null, the element counts that the last round added on the
// device and the host has not read yet (x vertices, y tets, z subfaces, w
// subsegments)
__global__ void k_classify(DevMesh m, int full, int* err, const int4* add) {
  if (add) {
    const int4 a = *add;
    m.nV += a.x;
    m.nT += a.y;
    m.nS += a.z;
    m.nG += a.w;
  }
  unsigned char* candS = m.candS;
  unsigned char* candG = m.candG;
  unsigned char* candT = m.candT;
  long n = (long)m.nG + m.nS + (full ? m.nT : 0);
  for (long ii = (long)blockIdx.x * blockDim.x + threadIdx.x; ii < n;
       ii += (long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    if (i < m.nG) {
      int g = i;
      if (!full && !m.dirtyG[g]) continue;
      m.dirtyG[g] = 0;
      uint8_t f = m.Gflag[CKI(g, m.capG)];
      if (f & (F_DEAD | F_UNSPL)) {
        candG[g] = 0;
        continue;
      }
      if (m.Gmust[CKI(g, m.capG)]) {
        candG[g] = 1;
        continue;
      }
      int4 G = m.GV[CKI(g, m.capG)];
      D3 A = vtx(m, G.x), Bp = vtx(m, G.y);
      bool enc = false;
      bool ok = edge_ring(m, G.w, G.x, G.y, [&](int t, const TetRec& r) {
        for (int k = 0; k < 4; ++k) {
          int x = vid(geti(r.v, k));
          if (x == G.x || x == G.y) continue;
          if (!enc && diametral(A, Bp, vtx(m, x)) < 0) enc = true;
        }
      });
      if (!ok) atomicOr(err, 1);
      candG[g] = enc ? 1 : 0;
    } else if (i < m.nG + m.nS) {
      int s = i - m.nG;
      if (!full && !m.dirtyS[s]) continue;
      m.dirtyS[s] = 0;
      uint8_t f = m.Sflag[CKI(s, m.capS)];
      if (f & (F_DEAD | F_UNSPL)) {
        candS[s] = 0;
        continue;
      }
      if (m.Smust[CKI(s, m.capS)]) {
        candS[s] = 1;
        continue;
      }
      int4 S = m.SV[CKI(s, m.capS)];
      int w = m.SN[CKI(s, m.capS)].w;
      if (w < 0 || (w >> 2) >= m.nT) {
        atomicOr(err, 2);
        candS[s] = 0;
        continue;
      }
      TetRec r = ld_tet(m, w >> 2);
      D3 A = vtx(m, S.x), Bp = vtx(m, S.y), C = vtx(m, S.z);
      bool enc = equatorial(A, Bp, C, vtx(m, vid(geti(r.v, w & 3)))) < 0;
      int nb = geti(r.n, w & 3);
      if (!enc && nb >= 0) {
        TetRec r2 = ld_tet(m, nb >> 2);
        enc = equatorial(A, Bp, C, vtx(m, vid(geti(r2.v, nb & 3)))) < 0;
      }
      candS[s] = enc ? 1 : 0;
    } else {
      int t = i - m.nG - m.nS;
      uint8_t f = m.Tflag[CKI(t, m.capT)];
      candT[t] = ((f & (F_DEAD | F_UNSPL | F_BAD)) == F_BAD) ? 1 : 0;
    }
  }
}

__device__ int elem_key(const DevMesh& m, int cls, int e, int* ids) {
  if (cls == CLS_SUBSEG) {
    int4 G = m.GV[CKI(e, m.capG)];
    ids[0] = min(G.x, G.y);
    ids[1] = max(G.x, G.y);
    return 2;
  }
  if (cls == CLS_SUBFACE) {
    int4 S = m.SV[CKI(e, m.capS)];
    ids[0] = S.x;
    ids[1] = S.y;
    ids[2] = S.z;
    sort3(ids[0], ids[1], ids[2]);
    return 3;
  }
  if (cls == CLS_TET) {
    int4 v = m.T[CKI(e, m.capT)].v;
    ids[0] = vid(v.x);
    ids[1] = vid(v.y);
    ids[2] = vid(v.z);
    ids[3] = vid(v.w);
    sort4(ids);
    return 4;
  }
  ids[0] = e;
  return 1;
}

// Candidates of a round in which each instance serves its own class are listed
// by their index in the concatenation (subsegments | subfaces | tetrahedra).
__device__ __forceinline__ int decode_cand(const DevMesh& m, int idx, int& cls) {
  if (idx < m.nG) {
    cls = CLS_SUBSEG;
    return idx;
  }
  if (idx < m.nG + m.nS) {
    cls = CLS_SUBFACE;
    return idx - m.nG;
  }
  cls = CLS_TET;
  return idx - m.nG - m.nS;
}

// Priority key of element e of class c: class first (subsegments, subfaces,
// tetrahedra), then the top 62 bits of the hash of its vertex coordinates
__device__ unsigned long long prio_key(const DevMesh& m, int c, int e) {
  int ids[4];
  int k = elem_key(m, c, e, ids);
  uint64_t h;
  if (c == CLS_POINT) {
    h = prio_hash(c, ids, k);
  } else {
    h = 0x9E3779B97F4A7C15ULL * (uint64_t)(c + 1);
    for (int q = 0; q < k; ++q) {
      V4 v = m.V[CKI(ids[q], m.capV)];
      h = prio_hash_step(prio_hash_step(prio_hash_step(h, v.x), v.y), v.z);
    }
  }
  return ((uint64_t)c << 62) | (h >> 2);
}

// Priorities. cls >= 0: elems are element ids of that class; cls < 0: they are
// concatenated indices.
__global__ void k_prio(DevMesh m, int cls, const int* elems, int n, unsigned long long* keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = cls;
    int e = cls >= 0 ? elems[i] : decode_cand(m, elems[i], c);
    keys[i] = prio_key(m, c, e);
  }
}

// Equal priority hashes (practically never): order the run by class, then by
// the sorted vertex ids.
__global__ void k_tiefix(DevMesh m, int cls, const unsigned long long* keys, int* elems, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool start = (i == 0 || keys[i - 1] != keys[i]) && (i + 1 < n && keys[i + 1] == keys[i]);
    if (!start) continue;
    int j = i + 1;
    while (j < n && keys[j] == keys[i]) ++j;
    for (int a = i + 1; a < j; ++a)
      for (int b = a; b > i; --b) {
        int cx = cls, cy = cls;
        int ex = cls >= 0 ? elems[b - 1] : decode_cand(m, elems[b - 1], cx);
        int ey = cls >= 0 ? elems[b] : decode_cand(m, elems[b], cy);
        bool lt = false;
        if (cx != cy) {
          lt = cy < cx;
        } else {
          int x[4], y[4];
          int nk = elem_key(m, cx, ex, x);
          elem_key(m, cy, ey, y);
          bool eq = true;
          for (int q = 0; q < nk && eq; ++q)
            if (y[q] != x[q]) {
              lt = y[q] < x[q];
              eq = false;
            }
        }
        if (!lt) break;
        int t = elems[b];
        elems[b] = elems[b - 1];
        elems[b - 1] = t;
      }
  }
}

// concatenated indices (in priority order) -> element ids, classes, instances
__global__ void k_decode_cands(DevMesh m, int* cand, uint8_t* ccls, int* cinst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c;
    int e = decode_cand(m, cand[i], c);
    int v0 = c == CLS_SUBSEG ? m.GV[CKI(e, m.capG)].x
                             : (c == CLS_SUBFACE ? m.SV[CKI(e, m.capS)].x : vid(m.T[CKI(e, m.capT)].v.x));
    cand[i] = e;
    ccls[i] = (uint8_t)c;
    cinst[i] = vinst(m, v0);
  }
}

// Per-instance classification counts over the concatenated index space (lanes
// with the same instance and class add together).
__global__ void k_count_inst(DevMesh m, const uint8_t* candG, const uint8_t* candS,
                             const uint8_t* candT) {
  const long tot = (long)m.nG + m.nS + m.nT;
  const long stride = (long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long base = (long)blockIdx.x * blockDim.x; base < tot; base += stride) {
    long i = base + threadIdx.x;
    int key = -1;
    if (i < tot) {
      int c;
      int e = decode_cand(m, (int)i, c);
      bool f;
      int v0;
      if (c == CLS_SUBSEG) {
        f = candG[e] != 0;
        v0 = f ? m.GV[CKI(e, m.capG)].x : 0;
      } else if (c == CLS_SUBFACE) {
        f = candS[e] != 0;
        v0 = f ? m.SV[CKI(e, m.capS)].x : 0;
      } else {
        f = candT[e] != 0;
        v0 = f ? vid(m.T[CKI(e, m.capT)].v.x) : 0;
      }
      if (f) key = vinst(m, v0) * 3 + c;
    }
    unsigned grp = __match_any_sync(FULLMASK, key);
    if (key >= 0 && (__ffs(grp) - 1) == lane)
      atomicAdd(&m.instCnt[key], (unsigned long long)__popc(grp));
  }
}

// One instance: the candidates of each class are just the set flags. Sixteen
// flags per thread (uint4 loads; flag arrays are allocated in whole 16-byte
// units), one atomic per warp and class.
__global__ void k_count_single(const uint8_t* candG, int nG, const uint8_t* candS, int nS,
                               const uint8_t* candT, int nT, unsigned long long* cnt,
                               const int4* add) {
  const int lane = threadIdx.x & 31;
  if (add) {
    const int4 a = *add;
    nT += a.y;
    nS += a.z;
    nG += a.w;
  }
  const uint8_t* arr[3] = {candG, candS, candT};
  const int len[3] = {nG, nS, nT};
  for (int c = 0; c < 3; ++c) {
    const int nv = (len[c] + 15) / 16;
    unsigned tot = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
      uint4 q = reinterpret_cast<const uint4*>(arr[c])[v];
      unsigned w[4] = {q.x, q.y, q.z, q.w};
      const int base = v * 16;
      for (int k = 0; k < 4; ++k)
        for (int b = 0; b < 4; ++b)
          if (base + 4 * k + b < len[c] && ((w[k] >> (8 * b)) & 0xff)) ++tot;
    }
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULLMASK, tot, o);
    if (lane == 0 && tot) atomicAdd(&cnt[c], (unsigned long long)tot);
  }
}
void launch_count_single(const DevMesh& m, unsigned long long* cnt, cudaStream_t s,
                         const int4* add) {
  // with additions not yet known on the host the grid covers the capacities
  long nv = add ? ((long)std::max(m.capG, std::max(m.capS, m.capT)) + 15) / 16
                : ((long)std::max(m.nG, std::max(m.nS, m.nT)) + 15) / 16;
  k_count_single<<<grid_for(nv, 256), 256, 0, s>>>(m.candG, m.nG, m.candS, m.nS, m.candT, m.nT,
                                                      cnt, add);
}

// This round's candidates: flagged elements of the class their instance serves
// (of every class for an instance in mixed rounds).
__global__ void k_round_flags(DevMesh m, const uint8_t* candG, const uint8_t* candS,
                              const uint8_t* candT, uint8_t* out) {
  const long tot = (long)m.nG + m.nS + m.nT;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    int c;
    int e = decode_cand(m, (int)i, c);
    bool f;
    int v0 = 0;
    if (c == CLS_SUBSEG) {
      f = candG[e] != 0;
      if (f) v0 = m.GV[CKI(e, m.capG)].x;
    } else if (c == CLS_SUBFACE) {
      f = candS[e] != 0;
      if (f) v0 = m.SV[CKI(e, m.capS)].x;
    } else {
      f = candT[e] != 0;
      if (f) v0 = vid(m.T[CKI(e, m.capT)].v.x);
    }
    // sel: 0..2 one class, 3 every class, 4 subsegments and subfaces
    const int sel = f ? m.instCls[vinst(m, v0)] : -1;
    out[i] = (f && (sel == c || sel == 3 || (sel == 4 && c <= CLS_SUBFACE))) ? 1 : 0;
  }
}

// ============================================================ split + locate
// splitting point of candidate i (Sec. 2: midpoint, subface circumcentre,
// tetrahedron circumcentre)
__device__ void split_one(const DevMesh& m, const DevRound& r, int i) {
  int e = r.cand[i];
  const int cls = cls_of(r, i);
  D3 p{0, 0, 0};
  bool ok = true;
  if (cls == CLS_SUBSEG) {
    int4 G = m.GV[CKI(e, m.capG)];
    p = midpoint_fixed(vtx(m, min(G.x, G.y)), vtx(m, max(G.x, G.y)));
    ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
  } else if (cls == CLS_SUBFACE) {
    int ids[4];
    elem_key(m, CLS_SUBFACE, e, ids);
    ok = tri_circumcenter_fixed(vtx(m, ids[0]), vtx(m, ids[1]), vtx(m, ids[2]), p);
  } else if (cls == CLS_TET) {
    int ids[4];
    elem_key(m, CLS_TET, e, ids);
    D3 off;
    ok = tet_circumcenter_fixed(vtx(m, ids[0]), vtx(m, ids[1]), vtx(m, ids[2]),
                                vtx(m, ids[3]), p, off);
  } else {
    p = D3{r.given[3 * e], r.given[3 * e + 1], r.given[3 * e + 2]};
    ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
  }
  r.sp[i] = make_v4(p.x, p.y, p.z, 0.0);
  r.loc[i] = -1;
  set_status(r, i, ok ? OUT_OK : OUT_UNSPL, ok ? RS_NONE : RS_BADPOINT);
  r.slab2_of[i] = -1;
  if (r.ckey) {
    int ids[4] = {-1, -1, -1, -1};
    elem_key(m, cls, e, ids);
    r.ckey[i] = make_int4(ids[0], ids[1], ids[2], ids[3]);
  }
}

__global__ void k_split(DevMesh m, DevRound r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x) {
    split_one(m, r, i);
  }
}

// Visibility walk (exit through the face with the smallest sorted vertex triple
// among those p lies strictly beyond) and the facet walk (same rule on edges).
__device__ __forceinline__ void seed_claim(const DevMesh& m, const DevRound& r, int i);

// locate candidate i's point (and, in refinement rounds, claim its start
// tetrahedra)
__device__ void locate_one(const DevMesh& m, const DevRound& r, int* hint, int i) {
  if (r.status[i] != OUT_OK) return;
  int e = r.cand[i];
  const int cls = cls_of(r, i);
  V4 q = r.sp[i];
  D3 p{q.x, q.y, q.z};
  if (cls == CLS_TET || cls == CLS_POINT) {
    int t = cls == CLS_TET ? e : hint[e];
    bool done = false;
    for (int it = 0; it < m.walk_limit && !done; ++it) {
      TetRec rec = ld_tet(m, t);
      int vv[4] = {vid(rec.v.x), vid(rec.v.y), vid(rec.v.z), vid(rec.v.w)};
      D3 c[4] = {vtx(m, vv[0]), vtx(m, vv[1]), vtx(m, vv[2]), vtx(m, vv[3])};
      int best = -1, b0 = 0, b1 = 0, b2 = 0;
      for (int f = 0; f < 4; ++f) {
        if (orient_rep4(c, f, p) < 0) {
          int w[3], k = 0;
          for (int j = 0; j < 4; ++j)
            if (j != f) w[k++] = vv[j];
          sort3(w[0], w[1], w[2]);
          if (best < 0 || lt3(w[0], w[1], w[2], b0, b1, b2)) {
            best = f;
            b0 = w[0];
            b1 = w[1];
            b2 = w[2];
          }
        }
      }
      if (best < 0) {
        r.loc[i] = t;
        done = true;
        break;
      }
      if (face_sub(rec.v, best)) {
        int s = ts_ptr(m, t)[best];
        if (s < 0 || s >= m.nS) {
          atomicAdd(&r.stats[ST_ITER], 1ULL);
          set_status(r, i, OUT_UNSPL, RS_WALK_LIMIT);
          done = true;
          break;
        }
        if (m.Sflag[CKI(s, m.capS)] & F_UNSPL) {
          set_status(r, i, OUT_UNSPL, RS_ENCROACH_UNSPL);
        } else {
          set_status(r, i, OUT_REJECT, RS_WALK_SUBFACE);
        }
        m.Smust[CKI(s, m.capS)] = 1;
        m.dirtyS[CKI(s, m.capS)] = 1;
        done = true;
        break;
      }
      int n = geti(rec.n, best);
      if (n < 0) {
        set_status(r, i, OUT_UNSPL, RS_WALK_HULL);
        done = true;
        break;
      }
      t = n >> 2;
    }
    if (!done) set_status(r, i, OUT_UNSPL, RS_WALK_LIMIT);
  } else if (cls == CLS_SUBFACE) {
    int s = e;
    bool done = false;
    for (int it = 0; it < m.walk_limit && !done; ++it) {
      int4 S = m.SV[CKI(s, m.capS)];
      int w = sf_wind(m, S);
      int best = -1, b0 = 0, b1 = 0;
      for (int k = 0; k < 3; ++k) {
        if (sf_orient_rep(m, S, k, p) == -w) {
          int u = geti(S, (k + 1) % 3), x = geti(S, (k + 2) % 3);
          int e0 = min(u, x), e1 = max(u, x);
          if (best < 0 || e0 < b0 || (e0 == b0 && e1 < b1)) {
            best = k;
            b0 = e0;
            b1 = e1;
          }
        }
      }
      if (best < 0) {
        r.loc[i] = s;
        done = true;
        break;
      }
      int nb = geti(m.SN[CKI(s, m.capS)], best);
      if (nb < 0) {
        int g = hash_lookup(m, ekey(b0, b1));
        if (g < 0) {
          set_status(r, i, OUT_UNSPL, RS_WALK_LIMIT);
        } else {
          if (m.Gflag[CKI(g, m.capG)] & F_UNSPL) set_status(r, i, OUT_UNSPL, RS_ENCROACH_UNSPL);
          else set_status(r, i, OUT_REJECT, RS_WALK_SUBSEG);
          m.Gmust[CKI(g, m.capG)] = 1;
          m.dirtyG[CKI(g, m.capG)] = 1;
        }
        done = true;
        break;
      }
      s = nb;
    }
    if (!done) set_status(r, i, OUT_UNSPL, RS_WALK_LIMIT);
  } else {
    r.loc[i] = e;
  }
  // refinement rounds claim their start tetrahedra here (points do it in
  // k_seed, after their one-per-tetrahedron filter)
  if (r.cls != CLS_POINT && r.status[i] == OUT_OK) seed_claim(m, r, i);
}

__global__ void k_locate(DevMesh m, DevRound r, int* hint) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x) {
    locate_one(m, r, hint, i);
  }
}


// Start claims: every candidate whose point was located claims the tetrahedra
// its region starts from (the located tetrahedron; both sides of the located
// subface; the ring of the subsegment) with its priority rank.
__device__ __forceinline__ void seed_claim(const DevMesh& m, const DevRound& r, int i) {
  const unsigned long long mk = (r.seed_epoch << 32) | (unsigned long long)(unsigned)i;
  const int cls = cls_of(r, i);
  if (cls == CLS_TET || cls == CLS_POINT) {
    atomicMin(&m.Tseed[CKI(r.loc[i], m.capT)], mk);
  } else if (cls == CLS_SUBFACE) {
    int tf = m.SN[CKI(r.loc[i], m.capS)].w;
    if (tf < 0) return;
    atomicMin(&m.Tseed[CKI(tf >> 2, m.capT)], mk);
    int nb = tet_n_ptr(m, tf >> 2)[tf & 3];
    if (nb >= 0) atomicMin(&m.Tseed[CKI(nb >> 2, m.capT)], mk);
  } else {
    int4 G = m.GV[CKI(r.cand[i], m.capG)];
    edge_ring(m, G.w, G.x, G.y, [&](int t, const TetRec&) { atomicMin(&m.Tseed[CKI(t, m.capT)], mk); });
  }
}
__global__ void k_seed(DevMesh m, DevRound r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x)
    if (r.status[i] == OUT_OK) seed_claim(m, r, i);
}
#ifdef CDR_CHECKED
#define seed_blasts(m, r, t, i) seed_blasts_at(m, r, t, i, __LINE__)
__device__ __forceinline__ bool seed_blasts_at(const DevMesh& m, const DevRound& r, int t, int i,
                                               int site) {
  if ((unsigned)t >= (unsigned)m.nT) {
    cdr_bad_index(site * 10 + r.cls, (long long)t, m.nT);
    return false;
  }
  unsigned long long v = m.Tseed[t];
  return (v >> 32) == r.seed_epoch && (unsigned)(v & 0xffffffffu) < (unsigned)i;
}
#else
__device__ __forceinline__ bool seed_blasts(const DevMesh& m, const DevRound& r, int t, int i) {
  unsigned long long v = m.Tseed[t];
  return (v >> 32) == r.seed_epoch && (unsigned)(v & 0xffffffffu) < (unsigned)i;
}
#endif

// Diagnostic build (CDR_PHASES): cycles spent per phase of region growth,
// summed over regions (lane 0's clock), and the regions that reached each phase.
#ifdef CDR_PHASES
static __device__ unsigned long long g_phase[2][16];
#define PHASE(k)                                              \
  do {                                                        \
    if (lane == 0) {                                          \
      long long t_ = clock64();                               \
      atomicAdd(&g_phase[0][k], (unsigned long long)(t_ - ph_t)); \
      atomicAdd(&g_phase[1][k], 1ULL);                        \
      ph_t = t_;                                              \
    }                                                         \
  } while (0)
// why a tier-1 region moved to tier 2 (diagnostic build): 10 cavity cap, 11
// boundary-face cap, 12 facet caps, 13 a table filled up
#define RETRY_NOTE(k)                                       \
  do {                                                      \
    if (C::HCAP <= Tier1Big::HCAP && lane == 0) atomicAdd(&g_phase[0][k], 1ULL); \
  } while (0)
#else
#define PHASE(k) \
  do {           \
  } while (0)
#define RETRY_NOTE(k) \
  do {                \
  } while (0)
#endif

// =============================================================== growth
struct Ws {
  int* cav;   // cavity tets
  int* hset;  // (tet << 2 | state) open addressing, -1 empty; state 1 in, 2 out
  int* bin;   // boundary faces: tet << 2 | face
  int* bout;  // neighbour across (tet << 2 | face) or -1
  int* bv;    // the boundary face's 3 vertex ids
  int* fcav;  // facet part subfaces
  int* fbnd;  // facet boundary edges: subface << 2 | edge
  int* fbv;   // the edge's 2 vertex ids and the facet id
};

// Open addressing with linear probing and no deletions. A put gives up after
// kProbe slots (the caller then treats the table as full and grows the region
// again in a larger one), so every stored key sits within kProbe slots of its
// home slot, and a lookup can stop after kProbe slots too: a nearly full table
// never costs a scan of the whole table.
constexpr int kProbe = 64;
__device__ __forceinline__ unsigned hs_slot(int t, int cap) {
  return (unsigned)mix64((unsigned long long)(unsigned)t) & (unsigned)(cap - 1);
}
__device__ int hs_find(const int* hs, int cap, int t) {
  unsigned h = hs_slot(t, cap);
  const int np = min(cap, kProbe);
  for (int it = 0; it < np; ++it) {
    int e = hs[h];
    if (e == -1) return 0;
    if ((e >> 2) == t) return e & 3;
    h = (h + 1) & (unsigned)(cap - 1);
  }
  return 0;
}
// returns 1 inserted, 0 present (state overwritten when force), -1 full
__device__ int hs_put(int* hs, int cap, int t, int state, bool force) {
  unsigned h = hs_slot(t, cap);
  const int np = min(cap, kProbe);
  for (int it = 0; it < np; ++it) {
    int old = atomicCAS(&hs[h], -1, (t << 2) | state);
    if (old == -1) return 1;
    if ((old >> 2) == t) {
      if (force) hs[h] = (t << 2) | state;
      return 0;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
  return -1;
}
__device__ __forceinline__ bool in_list(const int* a, int n, int x) {
  for (int i = 0; i < n; ++i)
    if (a[i] == x) return true;
  return false;
}
// warp-uniform append of flagged lane values, in lane order; n is warp-uniform
__device__ __forceinline__ void wappend(int* list, int& n, int cap, bool pred, int val, int lane) {
  unsigned b = __ballot_sync(FULLMASK, pred);
  int pos = n + __popc(b & ((1u << lane) - 1));
  if (pred && pos < cap) list[pos] = val;
  n += __popc(b);
}

// Table of a region's boundary edges and vertices (open addressing in the
// storage of the tet hash set, which growth no longer needs). An entry e <
// 3 CAPB is the edge of boundary face e/3 opposite its vertex e%3 (each edge is
// entered once per face: twice on a closed boundary); e >= 3 CAPB is the
// vertex bv[e - 3 CAPB], entered once. Keys are (min, max) vertex pairs, (v, v)
// for a vertex.
__device__ __forceinline__ void bt_key(const int* bv, int e, int cap3, int& a, int& b) {
  if (e < cap3) {
    const int j = e / 3, q = e - 3 * j;
    const int u = bv[3 * j + (q + 1) % 3], x = bv[3 * j + (q + 2) % 3];
    a = min(u, x);
    b = max(u, x);
  } else {
    a = b = bv[e - cap3];
  }
}
__device__ __forceinline__ unsigned bt_slot(int a, int b, int cap) {
  return (unsigned)mix64(((unsigned long long)(unsigned)a << 32) | (unsigned)b) & (unsigned)(cap - 1);
}
// enter e (vertices: only if their key is absent); false if the table is full
__device__ bool bt_put(int* t, int cap, const int* bv, int cap3, int e, bool unique) {
  int a, b;
  bt_key(bv, e, cap3, a, b);
  unsigned h = bt_slot(a, b, cap);
  const int np = min(cap, kProbe);
  for (int it = 0; it < np; ++it) {
    int old = atomicCAS(&t[h], -1, e);
    if (old == -1) return true;
    if (unique) {
      int c, d;
      bt_key(bv, old, cap3, c, d);
      if (c == a && d == b) return true;
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
  return false;
}
// is key (a, b) in the table; with self >= 0: how many edge entries other
// than self have it (*other = one of them)
__device__ int bt_find(const int* t, int cap, const int* bv, int cap3, int a, int b, int self,
                       int* other) {
  unsigned h = bt_slot(a, b, cap);
  int cnt = 0;
  const int np = min(cap, kProbe);
  for (int it = 0; it < np; ++it) {
    const int e = t[h];
    if (e == -1) break;
    if (e != self) {
      int c, d;
      bt_key(bv, e, cap3, c, d);
      if (c == a && d == b) {
        if (self < 0) return 1;
        ++cnt;
        *other = e;
      }
    }
    h = (h + 1) & (unsigned)(cap - 1);
  }
  return cnt;
}

// work counters of one warp's regions, added to the round totals once per warp
struct GrowAcc {
  unsigned long long tested = 0, cav = 0, bnd = 0;
};
__device__ __forceinline__ void flush_acc(const DevRound& r, const GrowAcc& a, int lane) {
  if (lane == 0) {
    if (a.tested) atomicAdd(&r.stats[ST_TESTED], a.tested);
    if (a.cav) atomicAdd(&r.stats[ST_CAV], a.cav);
    if (a.bnd) atomicAdd(&r.stats[ST_BND], a.bnd);
  }
}

// kOnly >= 0: every candidate of the launch has that class (a one-class
// round), so the code of the other classes is compiled out. -1: any class.
// hcap: slots of the workspace's hash set / boundary table in use (a power of
// two, at most hcap; smaller tables are cleared faster). Returns true if a
// table filled up: the region was then left as OUT_RETRY and can be grown
// again with a larger table, with the same result.
template <class C, int kOnly = -1>
__device__ bool grow_one(const DevMesh& m, const DevRound& r, int i, const Ws& w, int* slab,
                         int lane, GrowAcc& acc, int hcap = C::HCAP) {
  using L = SlabLayout<C>;
  // Tier 1's cavity and boundary-face capacities can be lowered at run time
  // (a tuning setting; the arrays keep their compile-time size): a region that
  // outgrows them is re-run in tier 2, so the result does not change.
  constexpr bool kTier1 = C::HCAP <= Tier1Big::HCAP;  // Tier1 or Tier1Big
  const int capc = kTier1 && r.t1cav > 0 ? min(r.t1cav, C::CAPC) : C::CAPC;
  const int capb = kTier1 && r.t1bnd > 0 ? min(r.t1bnd, C::CAPB) : C::CAPB;
  // tetrahedra only: no facet part, no subsegment ring
  constexpr bool kFacets = kOnly != CLS_TET;
  const int cls = kOnly >= 0 ? kOnly : cls_of(r, i);
  int st = r.status[i];
  if (st != OUT_OK && st != OUT_RETRY) {
    if (lane == 0) {
      slab[0] = slab[1] = slab[2] = slab[3] = 0;
    }
    return false;
  }
  const int elem = r.cand[i];
  const V4 q4 = r.sp[i];
  const D3 p{q4.x, q4.y, q4.z};
  int sa = -1, sb = -1;
  if (cls == CLS_SUBSEG) {
    int4 G = m.GV[CKI(elem, m.capG)];
    sa = G.x;
    sb = G.y;
  }
  int ncav = 0, nf = 0, nbnd = 0, nfb = 0;
  int ntested = 0;  // per lane
  int outcome = OUT_OK, reason = RS_NONE;
  bool retry = false;  // tier-1 capacity exceeded
  bool blast = false;  // the region met a higher-priority start (warp-uniform)
  bool cfail = false;  // a closure failure was met (the growth goes on)
  bool hf = false;     // a hash set or table filled up (this lane)

#ifdef CDR_PHASES
  long long ph_t = clock64();
#endif
  for (int k = lane; k < hcap; k += 32) w.hset[k] = -1;
  __syncwarp();
  PHASE(0);

  // ---------------------------------------------------------- start sets
  if (cls == CLS_TET || cls == CLS_POINT) {
    if (lane == 0) {
      w.cav[0] = r.loc[i];
      hs_put(w.hset, hcap, r.loc[i], 1, false);
    }
    ncav = 1;
    if (seed_blasts(m, r, r.loc[i], i)) {
      blast = true;
      goto done;
    }
  } else if (cls == CLS_SUBFACE) {
    if (lane == 0) w.fcav[0] = r.loc[i];
    nf = 1;
  } else {  // subsegment: the ring of its edge, and the subfaces on the edge
    int nc = 0, nfl = 0, bad = 0;
    if (lane == 0) {
      int4 G = m.GV[CKI(elem, m.capG)];
      bool ok = edge_ring(m, G.w, sa, sb, [&](int t, const TetRec& rec) {
        if (nc < capc) w.cav[nc] = t;
        ++nc;
        if (seed_blasts(m, r, t, i)) bad |= 2;
        if (hs_put(w.hset, hcap, t, 1, false) < 0) bad |= 4;
        for (int f = 0; f < 4; ++f) {
          int x = vid(geti(rec.v, f));
          if (x == sa || x == sb) continue;
          if (face_sub(rec.v, f)) {
            int s = ts_ptr(m, t)[f];
            bool dup = false;
            for (int z = 0; z < min(nfl, C::CAPF); ++z) dup |= w.fcav[z] == s;
            if (!dup) {
              if (nfl < C::CAPF) w.fcav[nfl] = s;
              ++nfl;
            }
          }
        }
      });
      bad |= ok ? 0 : 1;
    }
    nc = __shfl_sync(FULLMASK, nc, 0);
    nfl = __shfl_sync(FULLMASK, nfl, 0);
    bad = __shfl_sync(FULLMASK, bad, 0);
    if (bad & 2) {
      blast = true;
      goto done;
    }
    if (bad & 4) {  // the ring did not fit the hash set
      hf = true;
      retry = true;
      goto done;
    }
    if (bad) {
      outcome = OUT_UNSPL;
      reason = RS_WALK_LIMIT;
      goto done;
    }
    if (nc > capc || nfl > C::CAPF) {
      RETRY_NOTE(nc > capc ? 10 : 12);
      retry = true;
      goto done;
    }
    ncav = nc;
    nf = nfl;
  }
  __syncwarp();

  PHASE(1);  // start sets
  // ---------------------------------------------------------- facet part
  if (kFacets && nf > 0) {
    int head = 0;
    for (;;) {
      while (head < nf) {
        int end = nf;
        int items = (end - head) * 3;
        for (int base = 0; base < items; base += 32) {
          int it = base + lane;
          int cand = -1;
          if (it < items) {
            int s = w.fcav[head + it / 3], k = it % 3;
            int4 S = m.SV[CKI(s, m.capS)];
            int u = geti(S, (k + 1) % 3), x = geti(S, (k + 2) % 3);
            bool split = sa >= 0 && ((u == sa && x == sb) || (u == sb && x == sa));
            int nb = geti(m.SN[CKI(s, m.capS)], k);
            if (!split && nb >= 0 && !in_list(w.fcav, min(nf, C::CAPF), nb)) cand = nb;
          }
          // one lane per distinct neighbour tests it
          unsigned grp = __match_any_sync(FULLMASK, cand);
          bool leader = cand >= 0 && (__ffs(grp) - 1) == lane;
          bool add = false;
          if (leader) add = sf_incircle(m, m.SV[CKI(cand, m.capS)], p);
          wappend(w.fcav, nf, C::CAPF, add, cand, lane);
          __syncwarp();
        }
        head = end;
        if (nf > C::CAPF) break;
      }
      if (nf > C::CAPF) {
        RETRY_NOTE(12);
        retry = true;
        goto done;
      }
      // closure: every boundary edge must see p strictly inside
      bool changed = false, fail = false;
      int items = nf * 3;
      for (int base = 0; base < items; base += 32) {
        int it = base + lane;
        int cand = -1;
        bool f_ = false;
        if (it < items) {
          int s = w.fcav[it / 3], k = it % 3;
          int4 S = m.SV[CKI(s, m.capS)];
          int u = geti(S, (k + 1) % 3), x = geti(S, (k + 2) % 3);
          bool split = sa >= 0 && ((u == sa && x == sb) || (u == sb && x == sa));
          int nb = geti(m.SN[CKI(s, m.capS)], k);
          if (!split && !(nb >= 0 && in_list(w.fcav, nf, nb))) {
            if (sf_orient_rep(m, S, k, p) != sf_wind(m, S)) {
              if (nb < 0) f_ = true;
              else cand = nb;
            }
          }
        }
        fail |= __any_sync(FULLMASK, f_);
        unsigned grp = __match_any_sync(FULLMASK, cand);
        bool leader = cand >= 0 && (__ffs(grp) - 1) == lane;
        // a neighbour may already have been appended in this pass by a lower chunk
        if (leader && in_list(w.fcav, nf, cand)) leader = false;
        __syncwarp();
        int before = nf;
        wappend(w.fcav, nf, C::CAPF, leader, cand, lane);
        changed |= nf != before;
        __syncwarp();
        if (nf > C::CAPF) break;
      }
      cfail |= fail;
      if (nf > C::CAPF) {
        retry = true;
        goto done;
      }
      if (!changed) break;
    }
    // boundary edges
    {
      int items = nf * 3;
      for (int base = 0; base < items; base += 32) {
        int it = base + lane;
        bool pred = false;
        int val = 0, eu = 0, ew = 0, fid = 0;
        if (it < items) {
          int s = w.fcav[it / 3], k = it % 3;
          int4 S = m.SV[CKI(s, m.capS)];
          eu = geti(S, (k + 1) % 3);
          ew = geti(S, (k + 2) % 3);
          fid = S.w;
          bool split = sa >= 0 && ((eu == sa && ew == sb) || (eu == sb && ew == sa));
          int nb = geti(m.SN[CKI(s, m.capS)], k);
          pred = !split && !(nb >= 0 && in_list(w.fcav, nf, nb));
          val = (s << 2) | k;
        }
        int b0 = nfb;
        unsigned bal = __ballot_sync(FULLMASK, pred);
        int pos = b0 + __popc(bal & ((1u << lane) - 1));
        if (pred && pos < C::CAPFB) {
          w.fbnd[pos] = val;
          w.fbv[3 * pos] = eu;
          w.fbv[3 * pos + 1] = ew;
          w.fbv[3 * pos + 2] = fid;
        }
        nfb += __popc(bal);
      }
      if (nfb > C::CAPFB) {
        RETRY_NOTE(12);
        retry = true;
        goto done;
      }
    }
    __syncwarp();
    // tets on both sides of every facet-part subface start the cavity
    {
      for (int base = 0; base < nf; base += 32) {
        int it = base + lane;
        int c0 = -1, c1 = -1;
        if (it < nf) {
          int tf = m.SN[CKI(w.fcav[it], m.capS)].w;
          if (tf >= 0 && (tf >> 2) < m.nT) {
            c0 = tf >> 2;
            int nb = tet_n_ptr(m, c0)[tf & 3];
            c1 = nb >= 0 ? (nb >> 2) : -1;
          } else {
            atomicAdd(&r.stats[ST_ITER], 1ULL);
          }
        }
        for (int side = 0; side < 2; ++side) {
          int c = side == 0 ? c0 : c1;
          bool pred = false, bl = false;
          if (c >= 0) {
            int res = hs_put(w.hset, hcap, c, 1, false);
            if (res < 0) retry = hf = true;
            pred = res == 1;
            bl = seed_blasts(m, r, c, i);
          }
          retry = __any_sync(FULLMASK, retry);
          blast |= __any_sync(FULLMASK, bl);
          wappend(w.cav, ncav, capc, pred, c, lane);
        }
        __syncwarp();
      }
      if (blast) goto done;
      if (retry || ncav > capc) {
        retry = true;
        goto done;
      }
    }
  }

  PHASE(2);  // facet part
  // ----------------------------------------------------------- tet part
  {
    int head = 0;
    bool listed = false;
    for (;;) {
      while (head < ncav) {
        int end = ncav;
        int items = (end - head) * 4;
        for (int base = 0; base < items; base += 32) {
          int it = base + lane;
          int cand = -1;
          if (it < items) {
            int t = w.cav[head + (it >> 2)], f = it & 3;
            TetRec rec = ld_tet(m, t);
            int nb = geti(rec.n, f);
            CKL(nb, m.nT);
            (void)CKI(t, m.nT);
            if (nb >= 0 && !face_sub(rec.v, f)) {
              int nt = nb >> 2;
              if (hs_find(w.hset, hcap, nt) == 0 && orient_rep(m, rec, f, p) > 0) cand = nt;
            }
          }
          unsigned grp = __match_any_sync(FULLMASK, cand);
          bool leader = cand >= 0 && (__ffs(grp) - 1) == lane;
          bool add = false, bl = false;
          if (leader) {
            bool in = tet_in_sphere(m, ld_tet(m, cand), p);
            ++ntested;
            int res = hs_put(w.hset, hcap, cand, in ? 1 : 2, false);
            if (res < 0) retry = hf = true;
            add = in && res == 1;
            bl = add && seed_blasts(m, r, cand, i);
          }
          retry = __any_sync(FULLMASK, retry);
          blast |= __any_sync(FULLMASK, bl);
          wappend(w.cav, ncav, capc, add, cand, lane);
          __syncwarp();
          if (blast || retry || ncav > capc) break;
        }
        head = end;
        if (blast || retry || ncav > capc) break;
      }
      if (blast) goto done;
      if (retry || ncav > capc) {
        retry = true;
        goto done;
      }
      // closure. The pass also lists the boundary faces: when it neither adds a
      // tet nor touches the set, that list is the final one.
      bool changed = false, fail = false, touched = false;
      int items = ncav * 4;
      nbnd = 0;
      for (int base = 0; base < items; base += 32) {
        int it = base + lane;
        int cand = -1;
        bool f_ = false, pred = false;
        int bi = 0, bo = -1, v0 = 0, v1 = 0, v2 = 0;
        if (it < items) {
          int t = w.cav[it >> 2], f = it & 3;
          TetRec rec = ld_tet(m, t);
          int nb = geti(rec.n, f);
          CKL(nb, m.nT);
          bool sub = face_sub(rec.v, f);
          bool removed = kFacets && sub && nf > 0 && in_list(w.fcav, nf, ts_ptr(m, t)[f]);
          bool interior = !sub && nb >= 0 && hs_find(w.hset, hcap, nb >> 2) == 1;
          pred = !removed && !interior;
          if (pred && orient_rep(m, rec, f, p) <= 0) {
            if (sub || nb < 0) f_ = true;
            else cand = nb >> 2;
          }
          bi = (t << 2) | f;
          bo = nb;
          int z[3], k = 0;
          for (int j = 0; j < 4; ++j)
            if (j != f) z[k++] = vid(geti(rec.v, j));
          v0 = z[0];
          v1 = z[1];
          v2 = z[2];
        }
        {
          unsigned bal = __ballot_sync(FULLMASK, pred);
          int pos = nbnd + __popc(bal & ((1u << lane) - 1));
          if (pred && pos < capb) {
            w.bin[pos] = bi;
            w.bout[pos] = bo;
            w.bv[3 * pos] = v0;
            w.bv[3 * pos + 1] = v1;
            w.bv[3 * pos + 2] = v2;
          }
          nbnd += __popc(bal);
        }
        fail |= __any_sync(FULLMASK, f_);
        touched |= __any_sync(FULLMASK, cand >= 0);
        unsigned grp = __match_any_sync(FULLMASK, cand);
        bool leader = cand >= 0 && (__ffs(grp) - 1) == lane;
        bool add = false, bl = false;
        if (leader) {
          // (a tet tested out before has its state forced to in)
          int res = hs_put(w.hset, hcap, cand, 1, true);
          if (res < 0) retry = hf = true;
          add = true;
          bl = seed_blasts(m, r, cand, i);
        }
        retry = __any_sync(FULLMASK, retry);
        blast |= __any_sync(FULLMASK, bl);
        __syncwarp();
        // a tet appended earlier in this pass is already in; skip duplicates
        if (add && in_list(w.cav, min(ncav, capc), cand)) add = false;
        __syncwarp();
        int before = ncav;
        wappend(w.cav, ncav, capc, add, cand, lane);
        changed |= ncav != before;
        __syncwarp();
        if (retry || ncav > capc) break;
      }
      cfail |= fail;
      if (blast) goto done;
      if (retry || ncav > capc) {
        retry = true;
        goto done;
      }
      listed = !touched;
      if (!changed) break;
    }
    // boundary faces, listed again when the last closure pass touched the set
    if (!listed) {
      nbnd = 0;
      int items = ncav * 4;
      for (int base = 0; base < items; base += 32) {
        int it = base + lane;
        bool pred = false;
        int bi = 0, bo = -1, v0 = 0, v1 = 0, v2 = 0;
        if (it < items) {
          int t = w.cav[it >> 2], f = it & 3;
          TetRec rec = ld_tet(m, t);
          int nb = geti(rec.n, f);
          bool sub = face_sub(rec.v, f);
          bool removed = kFacets && sub && nf > 0 && in_list(w.fcav, nf, ts_ptr(m, t)[f]);
          bool interior = !sub && nb >= 0 && hs_find(w.hset, hcap, nb >> 2) == 1;
          pred = !removed && !interior;
          bi = (t << 2) | f;
          bo = nb;
          CKL(nb, m.nT);
          int z[3], k = 0;
          for (int j = 0; j < 4; ++j)
            if (j != f) z[k++] = vid(geti(rec.v, j));
          v0 = z[0];
          v1 = z[1];
          v2 = z[2];
        }
        unsigned bal = __ballot_sync(FULLMASK, pred);
        int pos = nbnd + __popc(bal & ((1u << lane) - 1));
        if (pred && pos < capb) {
          w.bin[pos] = bi;
          w.bout[pos] = bo;
          w.bv[3 * pos] = v0;
          w.bv[3 * pos + 1] = v1;
          w.bv[3 * pos + 2] = v2;
        }
        nbnd += __popc(bal);
      }
    }
    __syncwarp();  // the lists written above are read by other lanes below
    if (nbnd > capb) {
      RETRY_NOTE(11);
      retry = true;
      goto done;
    }
    // the shell counts as touched
    for (int base = 0; base < nbnd; base += 32) {
      int it = base + lane;
      bool bl = it < nbnd && w.bout[it] >= 0 && seed_blasts(m, r, w.bout[it] >> 2, i);
      blast |= __any_sync(FULLMASK, bl);
    }
    if (blast) goto done;
  }
  PHASE(3);  // tet part: growth, closure, boundary, shell
  if (ncav > kCavLimit) {
    outcome = OUT_UNSPL;
    reason = RS_OVERFLOW;
    goto done;
  }
  if (cfail) {
    outcome = OUT_UNSPL;
    reason = RS_CLOSURE;
    goto done;
  }
  __syncwarp();

  // ------------------------------------------------ boundary table
  // (the tet set's storage: growth is done)
  {
    for (int k = lane; k < hcap; k += 32) w.hset[k] = -1;
    __syncwarp();
    bool full = false;
    for (int it = lane; it < 3 * nbnd; it += 32) {
      full |= !bt_put(w.hset, hcap, w.bv, C::CAP3, it, false);
      full |= !bt_put(w.hset, hcap, w.bv, C::CAP3, C::CAP3 + it, true);
    }
    if (__any_sync(FULLMASK, full)) {  // the table is too small for this region
      retry = hf = true;
      goto done;
    }
    __syncwarp();
  }
  // ------------------------------------------------ preservation checks
  {
    // every cavity vertex lies on a boundary face
    bool lost = false;
    int items = ncav * 4;
    for (int base = 0; base < items && !lost; base += 32) {
      int it = base + lane;
      bool miss = false;
      if (it < items) {
        int v = vid(geti(m.T[CKI(w.cav[it >> 2], m.capT)].v, it & 3));
        miss = !bt_find(w.hset, hcap, w.bv, C::CAP3, v, v, -1, nullptr);
      }
      lost = __any_sync(FULLMASK, miss);
    }
    // every facet boundary edge lies on a boundary face
    for (int base = 0; base < nfb && !lost; base += 32) {
      int it = base + lane;
      bool miss = false;
      if (it < nfb) {
        int u = w.fbv[3 * it], x = w.fbv[3 * it + 1];
        miss = !bt_find(w.hset, hcap, w.bv, C::CAP3, min(u, x), max(u, x), -1, nullptr);
      }
      lost = __any_sync(FULLMASK, miss);
    }
    if (lost) {
      outcome = OUT_UNSPL;
      reason = RS_CLOSURE;
      goto done;
    }
  }
  PHASE(4);  // preservation
  // ------------------------------------------------ star check
  {
    // topology first: every star edge is shared by at most two boundary faces;
    // each edge's partner (the other face's entry) is kept in the slab for
    // insertion
    bool topo = false, nondel = false;
    const int items = nbnd * 3;
    for (int it = lane; it < items; it += 32) {
      int a, b, other = -1;
      bt_key(w.bv, it, C::CAP3, a, b);
      int cnt = bt_find(w.hset, hcap, w.bv, C::CAP3, a, b, it, &other);
      topo |= cnt > 1;
      slab[L::OFF_PART + it] = cnt == 1 ? other : -1;
    }
    topo = __any_sync(FULLMASK, topo);
    if (!topo) {
      for (int base = 0; base < items; base += 32) {
        int it = base + lane;
        bool bad = false;
        if (it < items) {
          const int j = it / 3, q = it - 3 * j;
          const int pe = slab[L::OFF_PART + it];  // written by this lane above
          const int partner = pe >= 0 ? pe / 3 : -1;
          if (partner >= 0 && j < partner) {
            const int* F = w.bv + 3 * j;
            const int u = F[(q + 1) % 3], x = F[(q + 2) % 3];  // edge opposite face vertex q
            bool isnew = false;
            for (int z = 0; z < nfb && !isnew; ++z) {
              int a = w.fbv[3 * z], b = w.fbv[3 * z + 1];
              isnew = (a == u && b == x) || (a == x && b == u);
            }
            if (!isnew) {
              const int apex = w.bv[pe];  // the partner face's vertex off the shared edge
              int bij = w.bin[j];
              TetRec rec = ld_tet(m, bij >> 2);
              int f = bij & 3;
              D3 a = f == 0 ? p : vtx(m, vid(rec.v.x));
              D3 b = f == 1 ? p : vtx(m, vid(rec.v.y));
              D3 c = f == 2 ? p : vtx(m, vid(rec.v.z));
              D3 d = f == 3 ? p : vtx(m, vid(rec.v.w));
              bad = insphere(a, b, c, d, vtx(m, apex)) > 0;
            }
          }
        }
        nondel |= __any_sync(FULLMASK, bad);
      }
    }
    if (topo) {
      outcome = OUT_UNSPL;
      reason = RS_CLOSURE;
      goto done;
    }
    if (nondel) {
      outcome = OUT_UNSPL;
      reason = RS_STARDEL;
      goto done;
    }
  }
  PHASE(5);  // star check
  // ------------------------------------------------ shortest-edge guard
  {
    const double g2 = guard2_of(m, inst_of(r, i));
    bool g = false;
    int items = ncav * 4;
    for (int base = 0; base < items; base += 32) {
      int it = base + lane;
      bool near = false;
      if (it < items) {
        int v = vid(geti(m.T[CKI(w.cav[it >> 2], m.capT)].v, it & 3));
        near = dist2_fixed(p, vtx(m, v)) <= g2;
      }
      g |= __any_sync(FULLMASK, near);
    }
    if (g) {
      outcome = OUT_UNSPL;
      reason = RS_GUARD;
      goto done;
    }
  }
  PHASE(6);  // guard
  // ------------------------------------------------ encroachment
  {
    bool rej = false, runspl = false;
    if (cls == CLS_TET) {
      for (int base = 0; base < nbnd; base += 32) {
        int it = base + lane;
        bool enc = false, un = false;
        if (it < nbnd) {
          int bij = w.bin[it];
          int t = bij >> 2, f = bij & 3;
          if (face_sub(m.T[CKI(t, m.capT)].v, f)) {
            const int* F = w.bv + 3 * it;
            if (equatorial(vtx(m, F[0]), vtx(m, F[1]), vtx(m, F[2]), p) < 0) {
              int s = ts_ptr(m, t)[f];
              enc = true;
              if (s >= 0 && s < m.nS) {
                un = (m.Sflag[CKI(s, m.capS)] & F_UNSPL) != 0;
                m.Smust[CKI(s, m.capS)] = 1;
                m.dirtyS[CKI(s, m.capS)] = 1;
              } else {
                atomicAdd(&r.stats[ST_ITER], 1ULL);
              }
            }
          }
        }
        rej |= __any_sync(FULLMASK, enc);
        runspl |= __any_sync(FULLMASK, un);
      }
    }
    // subsegments on cavity tetrahedra: encroached, or deleted by the insertion
    int items = ncav * 6;
    for (int base = 0; base < items; base += 32) {
      int it = base + lane;
      bool flag = false, un = false;
      if (it < items) {
        int t = w.cav[it / 6], e = it % 6;
        int4 v = m.T[CKI(t, m.capT)].v;
        if (edge_bit(v, e)) {
          int u = vid(geti(v, edge_i(e))), x = vid(geti(v, edge_j(e)));
          bool split = sa >= 0 && ((u == sa && x == sb) || (u == sb && x == sa));
          if (!split) {
            bool enc = false;
            if (cls == CLS_TET || cls == CLS_SUBFACE) enc = diametral(vtx(m, u), vtx(m, x), p) < 0;
            if (!enc) enc = !bt_find(w.hset, hcap, w.bv, C::CAP3, min(u, x), max(u, x), -1, nullptr);
            if (enc) {
              int g = hash_lookup(m, ekey(u, x));
              if (g >= 0) {
                flag = true;
                un = (m.Gflag[CKI(g, m.capG)] & F_UNSPL) != 0;
                m.Gmust[CKI(g, m.capG)] = 1;
                m.dirtyG[CKI(g, m.capG)] = 1;
                if (r.candG && cls == CLS_SUBSEG && !r.candG[g]) {
                  atomicAdd(&r.stats[ST_NEWCAND], 1ULL);
                  if (m.instSt) atomicAdd(&m.instSt[inst_of(r, i) * IS_COUNT + IS_NEWCAND], 1ULL);
                }
              }
            }
          }
        }
      }
      rej |= __any_sync(FULLMASK, flag);
      runspl |= __any_sync(FULLMASK, un);
    }
    if (rej) {
      outcome = runspl ? OUT_UNSPL : OUT_REJECT;
      reason = runspl ? RS_ENCROACH_UNSPL : RS_ENCROACH;
      goto done;
    }
  }
  PHASE(7);  // encroachment
  // ------------------------------------------------ priority marks
  {
    const unsigned long long mk = (r.epoch << 32) | (unsigned long long)(unsigned)i;
    for (int k = lane; k < ncav; k += 32) atomicMin(&m.Tmark[CKI(w.cav[k], m.capT)], mk);
    for (int k = lane; k < nbnd; k += 32)
      if (w.bout[k] >= 0) atomicMin(&m.Tmark[CKI(w.bout[k] >> 2, m.capT)], mk);
    for (int k = lane; k < nf; k += 32) atomicMin(&m.Smark[CKI(w.fcav[k], m.capS)], mk);
    for (int k = lane; k < nfb; k += 32) {
      int sk = w.fbnd[k];
      int nb = sn_ptr(m, sk >> 2)[sk & 3];
      if (nb >= 0) atomicMin(&m.Smark[CKI(nb, m.capS)], mk);
    }
  }

  PHASE(8);  // marks
done:
  __syncwarp();
  const bool hfull = __any_sync(FULLMASK, hf);
  if (retry && hfull) RETRY_NOTE(13);
  else if (retry && ncav > capc) RETRY_NOTE(10);
  for (int o = 16; o > 0; o >>= 1) ntested += __shfl_xor_sync(FULLMASK, ntested, o);
  acc.tested += (unsigned long long)ntested;
  if (!retry) {
    acc.cav += (unsigned long long)ncav;
    acc.bnd += (unsigned long long)nbnd;
  }
  if (blast) {
    if (lane == 0) {
      set_status(r, i, OUT_BLASTED, RS_NONE);
      slab[0] = slab[1] = slab[2] = slab[3] = 0;
    }
    return false;
  }
  if (retry) {
    if (lane == 0) {
      set_status(r, i, OUT_RETRY, RS_NONE);
      slab[0] = slab[1] = slab[2] = slab[3] = 0;
    }
    return hfull;
  }
  if (lane == 0) {
    set_status(r, i, outcome, reason);
    slab[0] = ncav;
    slab[1] = nbnd;
    slab[2] = nf;
    slab[3] = nfb;
  }
  if (outcome == OUT_OK) {
    // lists for selection and insertion (tier 2 works in place)
    if (w.cav != slab + L::OFF_CAV) {
      for (int k = lane; k < ncav; k += 32) slab[L::OFF_CAV + k] = w.cav[k];
      for (int k = lane; k < nbnd; k += 32) {
        slab[L::OFF_BIN + k] = w.bin[k];
        slab[L::OFF_BOUT + k] = w.bout[k];
      }
      for (int k = lane; k < nf; k += 32) slab[L::OFF_FCAV + k] = w.fcav[k];
      for (int k = lane; k < nfb; k += 32) slab[L::OFF_FBND + k] = w.fbnd[k];
      for (int k = lane; k < 3 * nbnd; k += 32) slab[L::OFF_BV + k] = w.bv[k];
      for (int k = lane; k < 3 * nfb; k += 32) slab[L::OFF_FBV + k] = w.fbv[k];
    }
  } else if (outcome == OUT_REJECT || reason == RS_GUARD || reason == RS_STARDEL ||
             reason == RS_ENCROACH_UNSPL) {
    // the cavity is complete: keep its tets for the round report
    if (w.cav != slab + L::OFF_CAV)
      for (int k = lane; k < min(ncav, capc); k += 32) slab[L::OFF_CAV + k] = w.cav[k];
  }
  return false;
}

// Tier-2 growth of candidate i. With shs set, the hash set / boundary table
// first lives in shared memory (shcap slots), where its probes cost a fraction
// of a global atomic's latency; a region whose table fills it is grown again
// in the global workspace w.hset. There the table starts at 32,768 slots
// (enough for a region at the cavity limit) and is enlarged to Tier2::HCAP
// only when a region's boundary table fills it. A region is grown the same
// way whatever its table's size, so the result does not depend on where the
// table lives.
__device__ void grow_tier2(const DevMesh& m, const DevRound& r, int i, const Ws& w, int* slab,
                           int lane, GrowAcc& acc, int* shs = nullptr, int shcap = 0) {
  if (shs) {
    Ws ws = w;
    ws.hset = shs;
    const bool full = grow_one<Tier2>(m, r, i, ws, slab, lane, acc, shcap);
    __syncwarp();
    if (!full) return;
  }
  for (int hcap = 32768;; hcap = min(hcap * 4, Tier2::HCAP)) {
    const bool full = grow_one<Tier2>(m, r, i, w, slab, lane, acc, hcap);
    __syncwarp();
    if (!full || hcap >= Tier2::HCAP) break;
  }
}

// tier 1: shared-memory workspaces, one per warp
constexpr int kWarps1 = 8;
template <class C>
struct SmemT {
  int cav[C::CAPC];
  int hset[C::HCAP];
  int bin[C::CAPB];
  int bout[C::CAPB];
  int bv[3 * C::CAPB];
  int fcav[C::CAPF];
  int fbnd[C::CAPFB];
  int fbv[3 * C::CAPFB];
};
using Smem1 = SmemT<Tier1>;
using Smem1Big = SmemT<Tier1Big>;

// blocks per SM the register budget is sized for (build-time, CDR_G1_MINB)
#ifndef CDR_G1_MINB
#define CDR_G1_MINB 4
#endif
template <int kOnly>
__global__ void __launch_bounds__(32 * kWarps1, CDR_G1_MINB) k_grow1(DevMesh m, DevRound r) {
  extern __shared__ int smraw[];
  Smem1* sm = reinterpret_cast<Smem1*>(smraw) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  Ws w{sm->cav, sm->hset, sm->bin, sm->bout, sm->bv, sm->fcav, sm->fbnd, sm->fbv};
  int warp = blockIdx.x * kWarps1 + (threadIdx.x >> 5);
  int nw = gridDim.x * kWarps1;
  GrowAcc acc;
  for (int i = warp; i < r.n; i += nw) {
    int* slab = r.slab1 + (size_t)i * SlabLayout<Tier1>::STRIDE;
    grow_one<Tier1, kOnly>(m, r, i, w, slab, lane, acc);
    __syncwarp();
    if (lane == 0 && r.rflag) r.rflag[i] = r.status[i] == OUT_RETRY ? 1 : 0;
  }
  flush_acc(r, acc, lane);
}

// tier 1 of rounds with boundary or mixed candidates: larger workspaces, four
// warps per block
#ifndef CDR_W1BIG
#define CDR_W1BIG 4
#endif
constexpr int kWarps1Big = CDR_W1BIG;
__global__ void __launch_bounds__(32 * kWarps1Big, 3) k_grow1big(DevMesh m, DevRound r) {
  extern __shared__ int smraw[];
  Smem1Big* sm = reinterpret_cast<Smem1Big*>(smraw) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  Ws w{sm->cav, sm->hset, sm->bin, sm->bout, sm->bv, sm->fcav, sm->fbnd, sm->fbv};
  int warp = blockIdx.x * kWarps1Big + (threadIdx.x >> 5);
  int nw = gridDim.x * kWarps1Big;
  GrowAcc acc;
  for (int i = warp; i < r.n; i += nw) {
    int* slab = r.slab1 + (size_t)i * SlabLayout<Tier1Big>::STRIDE;
    grow_one<Tier1Big>(m, r, i, w, slab, lane, acc);
    __syncwarp();
    if (lane == 0 && r.rflag) r.rflag[i] = r.status[i] == OUT_RETRY ? 1 : 0;
  }
  flush_acc(r, acc, lane);
}

// tier 2: global-memory workspaces; the slab doubles as the list storage.
// (Hash sets in shared memory here cost residency and ran 9% slower on the
// 500k clustered workload: this launch is bound by the number of regions in
// flight, not by the latency of one.)
constexpr int kWs2Extra = Tier2::HCAP;
// In a fused round, tier-2 hash sets of kT2FusedSlots slots are cut from the
// block's tier-1 workspaces, which are free by then: there the slowest region
// holds up the whole cluster, so its latency is what counts.
constexpr int kT2FusedSlots = 8192;
constexpr int kFusedT2Chunks = (int)(sizeof(Smem1) * kFusedWarps / (kT2FusedSlots * sizeof(int)));
static_assert(kFusedT2Chunks >= 1, "a fused block holds at least one tier-2 hash set");
__global__ void k_grow2(DevMesh m, DevRound r) {
  int lane = threadIdx.x & 31;
  int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int nw = gridDim.x * (blockDim.x >> 5);
  using L = SlabLayout<Tier2>;
  if (warp >= r.nws2) return;  // no workspace for this warp
  nw = min(nw, r.nws2);
  int* extra = r.ws2 + (size_t)warp * kWs2Extra;
  GrowAcc acc;
  for (int j = warp; j < r.n2; j += nw) {
    int i = r.list2[j];
    int* slab = r.slab2 + (size_t)j * L::STRIDE;
    Ws w{slab + L::OFF_CAV, extra, slab + L::OFF_BIN, slab + L::OFF_BOUT,
         slab + L::OFF_BV, slab + L::OFF_FCAV, slab + L::OFF_FBND, slab + L::OFF_FBV};
    grow_tier2(m, r, i, w, slab, lane, acc);
    __syncwarp();
    if (lane == 0 && r.status[i] == OUT_RETRY) set_status(r, i, OUT_UNSPL, RS_OVERFLOW);
  }
  flush_acc(r, acc, lane);
}

// ============================================================== selection
__device__ __forceinline__ const int* slab_of(const DevRound& r, int i, bool& tier2) {
  int j = r.slab2_of ? r.slab2_of[i] : -1;
  tier2 = j >= 0;
  if (tier2) return r.slab2 + (size_t)j * SlabLayout<Tier2>::STRIDE;
  return r.slab1 + (size_t)i * r.s1.STRIDE;
}

// Selection (the "blast" step of Sec. 2): a region is kept if it holds every
// mark it placed. One warp per candidate; its lanes check the marks together.
__device__ bool holds_marks(const DevMesh& m, const DevRound& r, int i, int lane) {
  bool t2;
  const int* slab = slab_of(r, i, t2);
  int ncav = slab[0], nbnd = slab[1], nf = slab[2], nfb = slab[3];
  int offC = t2 ? SlabLayout<Tier2>::OFF_CAV : r.s1.OFF_CAV;
  int offBO = t2 ? SlabLayout<Tier2>::OFF_BOUT : r.s1.OFF_BOUT;
  int offF = t2 ? SlabLayout<Tier2>::OFF_FCAV : r.s1.OFF_FCAV;
  int offFB = t2 ? SlabLayout<Tier2>::OFF_FBND : r.s1.OFF_FBND;
  const unsigned long long mk = (r.epoch << 32) | (unsigned long long)(unsigned)i;
  bool lost = false;
  for (int k = lane; k < ncav; k += 32) lost |= m.Tmark[CKI(slab[offC + k], m.capT)] != mk;
  for (int k = lane; k < nbnd; k += 32) {
    int b = slab[offBO + k];
    if (b >= 0) lost |= m.Tmark[CKI(b >> 2, m.capT)] != mk;
  }
  for (int k = lane; k < nf; k += 32) lost |= m.Smark[CKI(slab[offF + k], m.capS)] != mk;
  for (int k = lane; k < nfb; k += 32) {
    int sk = slab[offFB + k];
    int nb = sn_ptr(m, sk >> 2)[sk & 3];
    if (nb >= 0) lost |= m.Smark[CKI(nb, m.capS)] != mk;
  }
  return !__any_sync(FULLMASK, lost);
}

// outcome counts of the candidates one warp selected
struct SelAcc {
  unsigned surv = 0, ok = 0, rej = 0, blast = 0, unspl = 0;
};
// select candidate i (called by a whole warp; lane 0 writes)
__device__ void select_one(const DevMesh& m, const DevRound& r, int i, int lane, SelAcc& a) {
  const int outcome = r.status[i] & 0xff;
  const bool surv = outcome == OUT_OK && holds_marks(m, r, i, lane);
  if (lane != 0) return;
  const int cls = cls_of(r, i);
  r.survived[i] = surv ? 1 : 0;
  int4 c = make_int4(0, 0, 0, 0);
  if (surv) {
    bool t2;
    const int* slab = slab_of(r, i, t2);
    c = make_int4(cls == CLS_POINT ? 0 : 1, slab[1], slab[3], cls == CLS_SUBSEG ? 1 : 0);
  }
  r.counts[i] = c;
  int e = r.cand[i];
  if (outcome == OUT_UNSPL) {
    if (cls == CLS_SUBSEG) {
      m.Gflag[CKI(e, m.capG)] |= F_UNSPL;
      m.dirtyG[CKI(e, m.capG)] = 1;
    } else if (cls == CLS_SUBFACE) {
      m.Sflag[CKI(e, m.capS)] |= F_UNSPL;
      m.dirtyS[CKI(e, m.capS)] = 1;
    } else if (cls == CLS_TET) {
      m.Tflag[CKI(e, m.capT)] |= F_UNSPL;
      m.candT[CKI(e, m.capT)] = 0;
    } else {
      r.point_state[e] = 2;
    }
  }
  if (outcome == OUT_OK) {
    if (surv) ++a.surv;
    else ++a.ok;
  } else if (outcome == OUT_REJECT) {
    ++a.rej;
  } else if (outcome == OUT_BLASTED) {
    ++a.blast;
  } else {
    ++a.unspl;
  }
  // per-instance counts for the stall rule and batch statistics (blasted
  // regions, the bulk of a large round, need none)
  if (m.instSt && (surv || outcome == OUT_UNSPL || outcome == OUT_REJECT)) {
    unsigned long long* q = m.instSt + (size_t)inst_of(r, i) * IS_COUNT;
    atomicAdd(&q[surv ? IS_SURV : (outcome == OUT_UNSPL ? IS_UNSPL : IS_REJECT)], 1ULL);
  }
}
__device__ void flush_sel(const DevRound& r, const SelAcc& a, int lane) {
  if (lane != 0) return;
  if (a.surv) atomicAdd(&r.stats[ST_SURV], (unsigned long long)a.surv);
  if (a.ok) atomicAdd(&r.stats[ST_OK], (unsigned long long)a.ok);
  if (a.rej) atomicAdd(&r.stats[ST_REJECT], (unsigned long long)a.rej);
  if (a.blast) atomicAdd(&r.stats[ST_BLAST], (unsigned long long)a.blast);
  if (a.unspl) atomicAdd(&r.stats[ST_UNSPL], (unsigned long long)a.unspl);
}

__global__ void k_select(DevMesh m, DevRound r) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nw = (gridDim.x * blockDim.x) >> 5;
  SelAcc a;
  for (int i = warp; i < r.n; i += nw) select_one(m, r, i, lane, a);
  flush_sel(r, a, lane);
}

// ============================================================== insertion
// One warp per kept point: new tetrahedra p + boundary face, links to the shell
// and inside the star, new subfaces p + facet boundary edge, retire the region.
// insert kept candidate i (called by a whole warp)
__device__ void insert_one(const DevMesh& m, const DevRound& r, int* hint, int i, int lane) {
  if (!r.survived[i]) return;
  bool t2;
  const int* slab = slab_of(r, i, t2);
#define SLAB_OFF(name) (t2 ? SlabLayout<Tier2>::name : r.s1.name)
  const int ncav = slab[0], nbnd = slab[1], nf = slab[2], nfb = slab[3];
  const int* cav = slab + SLAB_OFF(OFF_CAV);
  const int* bin = slab + SLAB_OFF(OFF_BIN);
  const int* bout = slab + SLAB_OFF(OFF_BOUT);
  const int* fcav = slab + SLAB_OFF(OFF_FCAV);
  const int* fbnd = slab + SLAB_OFF(OFF_FBND);
  const int* bv = slab + SLAB_OFF(OFF_BV);
  const int* fbv = slab + SLAB_OFF(OFF_FBV);
  const int* part = slab + SLAB_OFF(OFF_PART);
#undef SLAB_OFF
  const int4 off = r.offs[i];
  const int e = r.cand[i];
  const int cls = cls_of(r, i);
  const int inst = inst_of(r, i);
  const int vp = cls == CLS_POINT ? e : m.nV + off.x;
  const int t0 = m.nT + off.y;
  const int s0 = m.nS + off.z;
  int sa = -1, sb = -1;
  if (cls == CLS_SUBSEG) {
    int4 G = m.GV[CKI(e, m.capG)];
    sa = G.x;
    sb = G.y;
  }
  if (lane == 0 && cls != CLS_POINT) {
    m.V[CKI(vp, m.capV)] = r.sp[i];
    if (m.Vinst) m.Vinst[CKI(vp, m.capV)] = inst;
  }
  if (lane == 0) {
    atomicAdd(&r.stats[ST_NEWT], (unsigned long long)nbnd);
    atomicAdd(&r.stats[ST_DEADT], (unsigned long long)ncav);
  }
  // step 1: new tetrahedra (p replaces the vertex opposite each boundary face)
  for (int j = lane; j < nbnd; j += 32) {
    int t = bin[j] >> 2, f = bin[j] & 3;
    TetRec R = ld_tet(m, t);
    int nid = t0 + j;
    int4 nv;
    for (int k = 0; k < 4; ++k) seti(nv, k, k == f ? vp : vid(geti(R.v, k)));
    if (face_sub(R.v, f)) seti(nv, f, geti(nv, f) | (1 << kSubBit));
    for (int ed = 0; ed < 6; ++ed) {
      int a = edge_i(ed), b = edge_j(ed);
      bool mark;
      if (a != f && b != f) {
        mark = edge_bit(R.v, ed);
      } else {
        int other = vid(geti(R.v, a == f ? b : a));
        mark = cls == CLS_SUBSEG && (other == sa || other == sb);
      }
      if (mark) seti(nv, ed >> 1, geti(nv, ed >> 1) | (1 << (29 + (ed & 1))));
    }
    TetRec N;
    N.v = nv;
    N.n = make_int4(-1, -1, -1, -1);
    CKL(bout[j], m.nT);
    (void)CKI(t, m.nT);
    seti(N.n, f, bout[j]);
    m.T[CKI(nid, m.capT)] = N;
    int4 ts = make_int4(-1, -1, -1, -1);
    if (face_sub(R.v, f)) {
      int s = ts_ptr(m, t)[f];
      seti(ts, f, s);
      if (s >= 0 && s < m.nS) {
        m.SN[CKI(s, m.capS)].w = (nid << 2) | f;
        m.dirtyS[CKI(s, m.capS)] = 1;  // one of its tetrahedra is new
      } else {
        atomicAdd(&r.stats[ST_ITER], 1ULL);
      }
    }
    m.TS[CKI(nid, m.capT)] = ts;
    m.Tmark[CKI(nid, m.capT)] = ~0ULL;
    m.Tseed[CKI(nid, m.capT)] = ~0ULL;
    m.Tfwd[CKI(nid, m.capT)] = -1;
    if (bout[j] >= 0) tet_n_ptr(m, bout[j] >> 2)[bout[j] & 3] = (nid << 2) | f;
  }
  __syncwarp();
  // step 2: links inside the star, through the boundary faces' shared edges
  // (each edge's partner entry was recorded by growth's star check)
  for (int it = lane; it < nbnd * 3; it += 32) {
    int j = it / 3, q = it % 3;
    const int* F = bv + 3 * j;
    int t = bin[j] >> 2, f = bin[j] & 3;
    // position in tet j of the face vertex q (the apex across the new face)
    TetRec R = ld_tet(m, t);
    int g = -1;
    for (int k = 0; k < 4; ++k)
      if (k != f && vid(geti(R.v, k)) == F[q]) g = k;
    int link = -1;
    const int pe = part[it];
    if (pe >= 0) {
      const int k2 = pe / 3;
      const int apexv = bv[pe];  // vertex of face k2 off the shared edge
      int t2_ = bin[k2] >> 2, f2 = bin[k2] & 3;
      TetRec R2 = ld_tet(m, t2_);
      int h = -1;
      for (int k = 0; k < 4; ++k)
        if (k != f2 && vid(geti(R2.v, k)) == apexv) h = k;
      link = h >= 0 ? (((t0 + k2) << 2) | h) : -1;
    }
    CKL(link, m.nT + 0x7fffffff / 8);
    if (link >= 0 && (link >> 2) < t0) CKL(link, 0);  // must point into this star
    if (g >= 0) tet_n_ptr(m, t0 + j)[g] = link;
    else atomicAdd(&r.stats[ST_ITER], 1ULL);
  }
  __syncwarp();
  // step 3: new subfaces (p joined to each facet boundary edge)
  for (int k = lane; k < nfb; k += 32) {
    int s = fbnd[k] >> 2, ke = fbnd[k] & 3;
    int u = fbv[3 * k], x = fbv[3 * k + 1], fid = fbv[3 * k + 2];
    int ns = s0 + k;
    m.SV[CKI(ns, m.capS)] = make_int4(vp, u, x, fid);
    int outer = geti(m.SN[CKI(s, m.capS)], ke);
    int4 sn = make_int4(outer, -1, -1, -1);
    if (outer >= 0) {
      int* o = sn_ptr(m, outer);
      for (int q = 0; q < 3; ++q)
        if (o[q] == s) o[q] = ns;
    }
    // across (x, p) and (p, u): the other new subface of this facet there
    for (int k2 = 0; k2 < nfb; ++k2) {
      if (k2 == k || fbv[3 * k2 + 2] != fid) continue;
      int u2 = fbv[3 * k2], x2 = fbv[3 * k2 + 1];
      if (u2 == x || x2 == x) sn.y = s0 + k2;
      if (u2 == u || x2 == u) sn.z = s0 + k2;
    }
    if (sa >= 0 && (x == sa || x == sb)) sn.y = -1;  // a new subsegment bounds it
    if (sa >= 0 && (u == sa || u == sb)) sn.z = -1;
    // the new tetrahedra on either side of the new subface
    int tw = -1;
    for (int j = 0; j < nbnd; ++j) {
      const int* F = bv + 3 * j;
      bool hu = F[0] == u || F[1] == u || F[2] == u;
      bool hx = F[0] == x || F[1] == x || F[2] == x;
      if (!(hu && hx)) continue;
      int apexv = (F[0] != u && F[0] != x) ? F[0] : ((F[1] != u && F[1] != x) ? F[1] : F[2]);
      int t = bin[j] >> 2, f = bin[j] & 3;
      TetRec R = ld_tet(m, t);
      int g = -1;
      for (int q = 0; q < 4; ++q)
        if (q != f && vid(geti(R.v, q)) == apexv) g = q;
      int nid = t0 + j;
      if (g < 0) {
        atomicAdd(&r.stats[ST_ITER], 1ULL);
        continue;
      }
      ts_ptr(m, nid)[g] = ns;
      atomicOr(&tet_v_ptr(m, nid)[g], 1 << kSubBit);
      if (tw < 0) tw = (nid << 2) | g;
    }
    sn.w = tw;
    m.SN[CKI(ns, m.capS)] = sn;
    m.Sflag[CKI(ns, m.capS)] = 0;
    m.Smust[CKI(ns, m.capS)] = 0;
    m.dirtyS[CKI(ns, m.capS)] = 1;
    m.Smark[CKI(ns, m.capS)] = ~0ULL;
  }
  __syncwarp();
  // step 4: retire the cavity and the facet part
  for (int k = lane; k < ncav; k += 32) {
    int t = cav[k];
    m.Tflag[CKI(t, m.capT)] |= F_DEAD;
    m.Tfwd[CKI(t, m.capT)] = t0;
    if (m.candT) m.candT[CKI(t, m.capT)] = 0;
  }
  for (int k = lane; k < nf; k += 32) {
    m.Sflag[CKI(fcav[k], m.capS)] |= F_DEAD;
    if (m.candS) m.candS[CKI(fcav[k], m.capS)] = 0;
  }
  // step 5: the split subsegment becomes (a, p) and (p, b)
  if (cls == CLS_SUBSEG) {
    int ta = -1, tb = -1;
    for (int j = lane; j < nbnd; j += 32) {
      const int* F = bv + 3 * j;
      if (F[0] == sa || F[1] == sa || F[2] == sa) ta = t0 + j;
      if (F[0] == sb || F[1] == sb || F[2] == sb) tb = t0 + j;
    }
    for (int o = 16; o > 0; o >>= 1) {
      ta = max(ta, __shfl_xor_sync(FULLMASK, ta, o));
      tb = max(tb, __shfl_xor_sync(FULLMASK, tb, o));
    }
    if (lane == 0) {
      int4 G = m.GV[CKI(e, m.capG)];
      int g2 = m.nG + off.w;
      m.GV[CKI(e, m.capG)] = make_int4(G.x, vp, G.z, ta);
      m.GV[CKI(g2, m.capG)] = make_int4(vp, G.y, G.z, tb);
      m.Gflag[CKI(e, m.capG)] = 0;
      m.Gmust[CKI(e, m.capG)] = 0;
      m.Gflag[CKI(g2, m.capG)] = 0;
      m.Gmust[CKI(g2, m.capG)] = 0;
      m.dirtyG[CKI(e, m.capG)] = 1;
      m.dirtyG[CKI(g2, m.capG)] = 1;
      hash_insert(m, ekey(G.x, vp), e);
      hash_insert(m, ekey(vp, G.y), g2);
    }
  }
  __syncwarp();
  // step 6: subsegment tet references and quality of the new tetrahedra
  for (int j = lane; j < nbnd; j += 32) {
    int nid = t0 + j;
    int4 v = m.T[CKI(nid, m.capT)].v;
    for (int ed = 0; ed < 6; ++ed) {
      if (!edge_bit(v, ed)) continue;
      int a = vid(geti(v, edge_i(ed))), b = vid(geti(v, edge_j(ed)));
      if (a == vp || b == vp) continue;
      int g = hash_lookup(m, ekey(a, b));
      if (g >= 0) {
        m.GV[CKI(g, m.capG)].w = nid;
        if (m.dirtyG) m.dirtyG[CKI(g, m.capG)] = 1;  // its edge ring changed
      }
    }
    int s4[4] = {vid(v.x), vid(v.y), vid(v.z), vid(v.w)};
    sort4(s4);
    bool bad = tet_bad_fixed(vtx(m, s4[0]), vtx(m, s4[1]), vtx(m, s4[2]), vtx(m, s4[3]),
                             bound_of(m, r.B, inst));
    m.Tflag[CKI(nid, m.capT)] = bad ? F_BAD : 0;
    if (m.candT) m.candT[CKI(nid, m.capT)] = bad ? 1 : 0;
  }
  if (lane == 0 && cls == CLS_POINT) {
    r.point_state[e] = 1;
    hint[e] = t0;
  }
}

__global__ void k_insert(DevMesh m, DevRound r, int* hint) {
  int lane = threadIdx.x & 31;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < r.n; i += nw) {
    insert_one(m, r, hint, i, lane);
  }
}

// ================================================================ batches
// Append an instance built on its own (src) to the batch mesh d. Its ids move
// by the batch's current sizes (vertices ov, tets ot, subfaces os, subsegments
// og, facets of) and its segment ids by oseg; its vertices record the slot.
__global__ void k_append(DevMesh d, DevMesh src, int ov, int ot, int os, int og, int of, int oseg,
                         int slot) {
  const long tot = max(max((long)src.nV, (long)src.nT), max(max((long)src.nS, (long)src.nG), (long)src.nF));
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    if (i < src.nV) {
      d.V[CKI(ov + i, d.capV)] = src.V[i];
      d.Vinst[CKI(ov + i, d.capV)] = slot;
    }
    if (i < src.nT) {
      TetRec R = src.T[i];
      for (int k = 0; k < 4; ++k) {
        int v = geti(R.v, k);
        seti(R.v, k, ((v & kVidMask) + ov) | (v & ~kVidMask));
        int nb = geti(R.n, k);
        if (nb >= 0) seti(R.n, k, (((nb >> 2) + ot) << 2) | (nb & 3));
      }
      const long t = ot + i;
      d.T[CKI(t, d.capT)] = R;
      int4 ts = src.TS[i];
      for (int k = 0; k < 4; ++k)
        if (geti(ts, k) >= 0) seti(ts, k, geti(ts, k) + os);
      d.TS[CKI(t, d.capT)] = ts;
      d.Tflag[CKI(t, d.capT)] = src.Tflag[i];
      d.Tmark[CKI(t, d.capT)] = ~0ULL;
      d.Tseed[CKI(t, d.capT)] = ~0ULL;
      d.Tfwd[CKI(t, d.capT)] = -1;
    }
    if (i < src.nS) {
      int4 sv = src.SV[i];
      d.SV[CKI(os + i, d.capS)] = make_int4(sv.x + ov, sv.y + ov, sv.z + ov, sv.w + of);
      int4 sn = src.SN[i];
      for (int k = 0; k < 3; ++k)
        if (geti(sn, k) >= 0) seti(sn, k, geti(sn, k) + os);
      if (sn.w >= 0) sn.w = (((sn.w >> 2) + ot) << 2) | (sn.w & 3);
      d.SN[CKI(os + i, d.capS)] = sn;
      d.Sflag[CKI(os + i, d.capS)] = src.Sflag[i];
      d.Smust[CKI(os + i, d.capS)] = src.Smust[i];
      d.Smark[CKI(os + i, d.capS)] = ~0ULL;
    }
    if (i < src.nG) {
      int4 g = src.GV[i];
      d.GV[CKI(og + i, d.capG)] = make_int4(g.x + ov, g.y + ov, g.z + oseg, g.w >= 0 ? g.w + ot : -1);
      d.Gflag[CKI(og + i, d.capG)] = src.Gflag[i];
      d.Gmust[CKI(og + i, d.capG)] = src.Gmust[i];
    }
    if (i < src.nF) d.FQ[of + i] = src.FQ[i];
  }
}
void launch_append(const DevMesh& d, const DevMesh& src, int ov, int ot, int os, int og, int of,
                   int oseg, int slot, cudaStream_t s) {
  long tot = max(max((long)src.nV, (long)src.nT), max(max((long)src.nS, (long)src.nG), (long)src.nF));
  if (tot > 0) k_append<<<grid_for(tot, 256), 256, 0, s>>>(d, src, ov, ot, os, og, of, oseg, slot);
}

__device__ __forceinline__ int tet_inst(const DevMesh& m, int t) {
  return vinst(m, vid(m.T[CKI(t, m.capT)].v.x));
}
// Remove an instance: its elements die; its vertices leave the slot (which can
// then be reused).
__global__ void k_kill_instance(DevMesh m, int slot) {
  const long tot = (long)m.nT + m.nS + m.nG;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    if (i < m.nT) {
      if (tet_inst(m, (int)i) == slot) m.Tflag[CKI(i, m.capT)] |= F_DEAD;
    } else if (i < (long)m.nT + m.nS) {
      int s = (int)(i - m.nT);
      if (vinst(m, m.SV[CKI(s, m.capS)].x) == slot) m.Sflag[CKI(s, m.capS)] |= F_DEAD;
    } else {
      int g = (int)(i - m.nT - m.nS);
      if (vinst(m, m.GV[CKI(g, m.capG)].x) == slot) m.Gflag[CKI(g, m.capG)] |= F_DEAD;
    }
  }
}
__global__ void k_release_vertices(DevMesh m, int slot) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < m.nV; v += gridDim.x * blockDim.x)
    if (m.Vinst[CKI(v, m.capV)] == slot) m.Vinst[CKI(v, m.capV)] = -1;
}
void launch_kill_instance(const DevMesh& m, int slot, cudaStream_t s) {
  long tot = (long)m.nT + m.nS + m.nG;
  if (tot > 0) k_kill_instance<<<grid_for(tot, 256), 256, 0, s>>>(m, slot);
  if (m.nV > 0) k_release_vertices<<<grid_for(m.nV, 256), 256, 0, s>>>(m, slot);
}

// Export of one instance: flags of its vertices (kind 0), live tets (1),
// subfaces (2) and subsegments (3) as 0/1 ints.
__global__ void k_inst_flags(DevMesh m, int slot, int kind, int n, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool f;
    if (kind == 0) f = m.Vinst[CKI(i, m.capV)] == slot;
    else if (kind == 1) f = !(m.Tflag[CKI(i, m.capT)] & F_DEAD) && tet_inst(m, i) == slot;
    else if (kind == 2) f = !(m.Sflag[CKI(i, m.capS)] & F_DEAD) && vinst(m, m.SV[CKI(i, m.capS)].x) == slot;
    else f = !(m.Gflag[CKI(i, m.capG)] & F_DEAD) && vinst(m, m.GV[CKI(i, m.capG)].x) == slot;
    out[i] = f ? 1 : 0;
  }
}
// Gather the flagged entries (positions pos from an exclusive scan of the
// flags) with vertex ids renumbered by vpos and facet / segment ids shifted back.
__global__ void k_inst_gather(DevMesh m, int kind, int n, const int* flag, const int* pos,
                              const int* vpos, int of, int oseg, int4* out, uint8_t* oflag,
                              V4* oxyz) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    int d = pos[i];
    if (kind == 0) {
      oxyz[d] = m.V[CKI(i, m.capV)];
    } else if (kind == 1) {
      int4 v = m.T[CKI(i, m.capT)].v;
      out[d] = make_int4(vpos[vid(v.x)], vpos[vid(v.y)], vpos[vid(v.z)], vpos[vid(v.w)]);
      oflag[d] = m.Tflag[CKI(i, m.capT)] & F_UNSPL ? 2 : 0;
    } else if (kind == 2) {
      int4 S = m.SV[CKI(i, m.capS)];
      out[d] = make_int4(vpos[S.x], vpos[S.y], vpos[S.z], S.w - of);
      oflag[d] = (m.Smust[CKI(i, m.capS)] ? 1 : 0) | (m.Sflag[CKI(i, m.capS)] & F_UNSPL ? 2 : 0);
    } else {
      int4 G = m.GV[CKI(i, m.capG)];
      out[d] = make_int4(vpos[G.x], vpos[G.y], G.z - oseg, 0);
      oflag[d] = (m.Gmust[CKI(i, m.capG)] ? 1 : 0) | (m.Gflag[CKI(i, m.capG)] & F_UNSPL ? 2 : 0);
    }
  }
}
// keep the flags of bad tetrahedra (bad, not unsplittable)
__global__ void k_inst_bad(DevMesh m, int* flag, int n) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    if (flag[t] && !(m.Tflag[CKI(t, m.capT)] & F_BAD)) flag[t] = 0;
}
void launch_inst_bad(const DevMesh& m, int* flag, int n, cudaStream_t s) {
  if (n > 0) k_inst_bad<<<grid_for(n, 256), 256, 0, s>>>(m, flag, n);
}
void launch_inst_flags(const DevMesh& m, int slot, int kind, int n, int* out, cudaStream_t s) {
  if (n > 0) k_inst_flags<<<grid_for(n, 256), 256, 0, s>>>(m, slot, kind, n, out);
}
void launch_inst_gather(const DevMesh& m, int kind, int n, const int* flag, const int* pos,
                        const int* vpos, int of, int oseg, int4* out, uint8_t* oflag, V4* oxyz,
                        cudaStream_t s) {
  if (n > 0)
    k_inst_gather<<<grid_for(n, 256), 256, 0, s>>>(m, kind, n, flag, pos, vpos, of, oseg, out,
                                                   oflag, oxyz);
}

// ============================================================ maintenance
__global__ void k_follow_fwd(DevMesh m, int* hint, const int* state, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (state[i] != 0) continue;
    int t = hint[i];
    for (int it = 0; it < 1 << 20 && (m.Tflag[CKI(t, m.capT)] & F_DEAD); ++it) t = m.Tfwd[CKI(t, m.capT)];
    hint[i] = t;
  }
}

__global__ void k_compact_flags(DevMesh m, int* alive) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x)
    alive[t] = (m.Tflag[CKI(t, m.capT)] & F_DEAD) ? 0 : 1;
}
// newid = exclusive scan of alive; move live tets to T2 with remapped links
__global__ void k_compact_move(DevMesh m, const int* newid, TetRec* T2, int4* TS2,
                               unsigned char* F2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x) {
    if (m.Tflag[CKI(t, m.capT)] & F_DEAD) continue;
    TetRec R = m.T[CKI(t, m.capT)];
    for (int f = 0; f < 4; ++f) {
      int nb = geti(R.n, f);
      if (nb >= 0) seti(R.n, f, (newid[nb >> 2] << 2) | (nb & 3));
    }
    int d = newid[t];
    T2[d] = R;
    TS2[d] = m.TS[CKI(t, m.capT)];
    F2[d] = m.Tflag[CKI(t, m.capT)];
  }
}
__global__ void k_compact_hints(DevMesh m, const int* newid, int* hint, int nh) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += gridDim.x * blockDim.x) {
    int t = hint[i];
    for (int it = 0; it < 1 << 20 && (m.Tflag[CKI(t, m.capT)] & F_DEAD); ++it) t = m.Tfwd[CKI(t, m.capT)];
    hint[i] = newid[t];
  }
}
__global__ void k_compact_fix(DevMesh m, const int* newid) {
  int n = m.nS + m.nG;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < m.nS) {
      if (m.Sflag[CKI(i, m.capS)] & F_DEAD) continue;
      int w = m.SN[CKI(i, m.capS)].w;
      m.SN[CKI(i, m.capS)].w = (newid[w >> 2] << 2) | (w & 3);
    } else {
      int g = i - m.nS;
      if (m.Gflag[CKI(g, m.capG)] & F_DEAD) continue;
      m.GV[CKI(g, m.capG)].w = newid[m.GV[CKI(g, m.capG)].w];
    }
  }
}

// ================================================================= export
__global__ void k_live_flags(const unsigned char* flag, int n, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (flag[i] & F_DEAD) ? 0 : 1;
}
__global__ void k_gather_tets(DevMesh m, const int* pos, int4* out, unsigned char* oflag) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x) {
    if (m.Tflag[CKI(t, m.capT)] & F_DEAD) continue;
    int4 v = m.T[CKI(t, m.capT)].v;
    int d = pos[t];
    out[d] = make_int4(vid(v.x), vid(v.y), vid(v.z), vid(v.w));
    oflag[d] = (m.Tflag[CKI(t, m.capT)] & F_UNSPL) ? 2 : 0;
  }
}
__global__ void k_gather_subfaces(DevMesh m, const int* pos, int4* out, unsigned char* oflag) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m.nS; s += gridDim.x * blockDim.x) {
    if (m.Sflag[CKI(s, m.capS)] & F_DEAD) continue;
    int d = pos[s];
    out[d] = m.SV[CKI(s, m.capS)];
    oflag[d] = (m.Smust[CKI(s, m.capS)] ? 1 : 0) | ((m.Sflag[CKI(s, m.capS)] & F_UNSPL) ? 2 : 0);
  }
}
__global__ void k_gather_subsegs(DevMesh m, const int* pos, int4* out, unsigned char* oflag) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m.nG; g += gridDim.x * blockDim.x) {
    if (m.Gflag[CKI(g, m.capG)] & F_DEAD) continue;
    int d = pos[g];
    out[d] = m.GV[CKI(g, m.capG)];
    oflag[d] = (m.Gmust[CKI(g, m.capG)] ? 1 : 0) | ((m.Gflag[CKI(g, m.capG)] & F_UNSPL) ? 2 : 0);
  }
}
// cavity tets of each reported candidate as sorted vertex ids
__global__ void k_report_cav(DevMesh m, DevRound r, const int* offs, int4* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x) {
    bool t2;
    const int* slab = slab_of(r, i, t2);
    int n = offs[i + 1] - offs[i];
    const int* cav = slab + (t2 ? SlabLayout<Tier2>::OFF_CAV : r.s1.OFF_CAV);
    for (int k = 0; k < n; ++k) {
      int4 v = m.T[CKI(cav[k], m.capT)].v;
      int s[4] = {vid(v.x), vid(v.y), vid(v.z), vid(v.w)};
      sort4(s);
      out[offs[i] + k] = make_int4(s[0], s[1], s[2], s[3]);
    }
  }
}

// ================================================================ wrappers

void launch_init_tets(const DevMesh& m, const int4* tets, int n, cudaStream_t s) {
  k_init_tets<<<grid_for(n, 256), 256, 0, s>>>(m, tets, n);
}
void launch_face_keys(const DevMesh& m, unsigned long long* hi, unsigned int* lo, int* val,
                      cudaStream_t s) {
  k_face_keys<<<grid_for(4L * m.nT, 256), 256, 0, s>>>(m, hi, lo, val);
}
void launch_pair_faces(const DevMesh& m, const unsigned long long* hi, const unsigned int* lo,
                       const int* val, int n, int* err, cudaStream_t s) {
  k_pair_faces<<<grid_for(n, 256), 256, 0, s>>>(m, hi, lo, val, n, err);
}
void launch_label_subfaces(const DevMesh& m, const int4* tris, int n, const unsigned long long* hi,
                           const unsigned int* lo, const int* val, int nfaces, int* err,
                           cudaStream_t s) {
  k_label_subfaces<<<grid_for(n, 256), 256, 0, s>>>(m, tris, n, hi, lo, val, nfaces, err);
}
void launch_subface_edge_keys(const DevMesh& m, unsigned long long* hi, unsigned int* lo,
                              int* val, cudaStream_t s) {
  k_subface_edge_keys<<<grid_for(3L * m.nS, 256), 256, 0, s>>>(m, hi, lo, val);
}
void launch_pair_subface_edges(const DevMesh& m, const unsigned long long* hi,
                               const unsigned int* lo, const int* val, int n, int* err,
                               cudaStream_t s) {
  k_pair_subface_edges<<<grid_for(n, 256), 256, 0, s>>>(m, hi, lo, val, n, err);
}
void launch_hash_clear(const DevMesh& m, cudaStream_t s) {
  k_hash_clear<<<grid_for((long)m.hmask + 1, 256), 256, 0, s>>>(m);
}
void launch_hash_insert_subsegs(const DevMesh& m, int g0, int g1, cudaStream_t s) {
  if (g1 > g0) k_hash_insert_subsegs<<<grid_for(g1 - g0, 256), 256, 0, s>>>(m, g0, g1);
}
void launch_mark_edges(const DevMesh& m, cudaStream_t s) {
  k_mark_edges<<<grid_for(m.nT, 256), 256, 0, s>>>(m);
}
void launch_check_create(const DevMesh& m, int* err, cudaStream_t s) {
  k_check_create<<<grid_for((long)m.nT + m.nG, 256), 256, 0, s>>>(m, err);
}
void launch_recompute_bad(const DevMesh& m, double B, cudaStream_t s) {
  k_recompute_bad<<<grid_for(m.nT, 256), 256, 0, s>>>(m, B);
}
void launch_classify(const DevMesh& m, bool full, int* err, cudaStream_t s, const int4* add) {
  long n = add ? (long)m.capG + m.capS + (full ? m.capT : 0)
               : (long)m.nG + m.nS + (full ? m.nT : 0);
  if (n > 0) k_classify<<<grid_for(n, 256), 256, 0, s>>>(m, full ? 1 : 0, err, add);
}
void launch_prio(const DevMesh& m, int cls, const int* elems, int n, unsigned long long* keys,
                 cudaStream_t s) {
  if (n > 0) k_prio<<<grid_for(n, 256), 256, 0, s>>>(m, cls, elems, n, keys);
}
void launch_tiefix(const DevMesh& m, int cls, const unsigned long long* keys, int* elems, int n,
                   cudaStream_t s) {
  if (n > 1) k_tiefix<<<grid_for(n, 256), 256, 0, s>>>(m, cls, keys, elems, n);
}
void launch_split(const DevMesh& m, const DevRound& r, cudaStream_t s) {
  if (r.n > 0) k_split<<<grid_for(r.n, 256), 256, 0, s>>>(m, r);
}
void launch_locate(const DevMesh& m, const DevRound& r, int* hint, cudaStream_t s) {
  if (r.n > 0) k_locate<<<grid_for(r.n, 128), 128, 0, s>>>(m, r, hint);
}
void launch_seed(const DevMesh& m, const DevRound& r, cudaStream_t s) {
  if (r.n > 0) k_seed<<<grid_for(r.n, 256), 256, 0, s>>>(m, r);
}
void launch_grow1(const DevMesh& m, const DevRound& r, int blocks_per_sm, cudaStream_t s) {
  if (r.n <= 0) return;
  static bool attr = false;
  size_t smem = sizeof(Smem1) * kWarps1;
  if (!attr) {
    cudaFuncSetAttribute(k_grow1<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_grow1<CLS_TET>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  long blocks = ((long)r.n + kWarps1 - 1) / kWarps1;
  if (blocks > 152L * blocks_per_sm) blocks = 152L * blocks_per_sm;
  // a round of bad tetrahedra alone runs the tetrahedron-only growth; other
  // rounds the larger workspaces (the host set r.s1 to match: slab1_layout)
  if (grow1_tets_only(r)) {
    k_grow1<CLS_TET><<<(int)blocks, 32 * kWarps1, smem, s>>>(m, r);
    return;
  }
  static bool attr_big = false;
  const size_t smem_big = sizeof(Smem1Big) * kWarps1Big;
  if (!attr_big) {
    cudaFuncSetAttribute(k_grow1big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big);
    attr_big = true;
  }
  long bb = ((long)r.n + kWarps1Big - 1) / kWarps1Big;
  if (bb > 152L * 2 * blocks_per_sm) bb = 152L * 2 * blocks_per_sm;
  k_grow1big<<<(int)bb, 32 * kWarps1Big, smem_big, s>>>(m, r);
}
bool grow1_tets_only(const DevRound& r) { return r.cls == CLS_TET && !r.ccls; }
SlabOff slab1_layout(bool tets_only) {
  return tets_only ? slab_off<Tier1>() : slab_off<Tier1Big>();
}
void launch_grow2(const DevMesh& m, const DevRound& r, int nwarps, cudaStream_t s) {
  if (r.n2 <= 0 || r.nws2 <= 0) return;
  int blocks = (min(nwarps, r.nws2) + 1) / 2;  // two warps per block
  k_grow2<<<blocks, 64, 0, s>>>(m, r);
}
void launch_select(const DevMesh& m, const DevRound& r, cudaStream_t s) {
  if (r.n > 0) k_select<<<grid_for(32L * r.n, 256), 256, 0, s>>>(m, r);
}
void launch_insert(const DevMesh& m, const DevRound& r, int* hint, cudaStream_t s) {
  if (r.n > 0) k_insert<<<grid_for(32L * r.n, 256), 256, 0, s>>>(m, r, hint);
}
void launch_compact_flags(const DevMesh& m, int* alive, cudaStream_t s) {
  k_compact_flags<<<grid_for(m.nT, 256), 256, 0, s>>>(m, alive);
}
void launch_compact_move(const DevMesh& m, const int* newid, TetRec* T2, int4* TS2,
                         unsigned char* F2, int* hint, int nhint, cudaStream_t s) {
  if (nhint > 0) k_compact_hints<<<grid_for(nhint, 256), 256, 0, s>>>(m, newid, hint, nhint);
  k_compact_move<<<grid_for(m.nT, 256), 256, 0, s>>>(m, newid, T2, TS2, F2);
}
void launch_compact_fix(const DevMesh& m, const int* newid, cudaStream_t s) {
  k_compact_fix<<<grid_for((long)m.nS + m.nG, 256), 256, 0, s>>>(m, newid);
}
void launch_follow_fwd(const DevMesh& m, int* hint, const int* state, int n, cudaStream_t s) {
  if (n > 0) k_follow_fwd<<<grid_for(n, 256), 256, 0, s>>>(m, hint, state, n);
}
void launch_live_flags(const unsigned char* flag, int n, int* out, cudaStream_t s) {
  if (n > 0) k_live_flags<<<grid_for(n, 256), 256, 0, s>>>(flag, n, out);
}
void launch_gather_tets(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                        cudaStream_t s) {
  if (m.nT > 0) k_gather_tets<<<grid_for(m.nT, 256), 256, 0, s>>>(m, pos, out, oflag);
}
void launch_gather_subfaces(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                            cudaStream_t s) {
  if (m.nS > 0) k_gather_subfaces<<<grid_for(m.nS, 256), 256, 0, s>>>(m, pos, out, oflag);
}
void launch_gather_subsegs(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                           cudaStream_t s) {
  if (m.nG > 0) k_gather_subsegs<<<grid_for(m.nG, 256), 256, 0, s>>>(m, pos, out, oflag);
}
void launch_report_cav(const DevMesh& m, const DevRound& r, const int* offs, int4* out,
                       cudaStream_t s) {
  if (r.n > 0) k_report_cav<<<grid_for(r.n, 128), 128, 0, s>>>(m, r, offs, out);
}


// =========================================================== predicate probe
// Batch evaluation of the device predicates and formulas (for checking them
// against an exact reference). Each item holds 16 doubles of input.
__global__ void k_eval_pred(int kind, const double* in, int n, int* sign, double* outp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int sg;
    D3 o;
    eval_item(kind, in + 16 * (size_t)i, &sg, &o);
    sign[i] = sg;
    if (outp) {
      outp[3 * (size_t)i] = o.x;
      outp[3 * (size_t)i + 1] = o.y;
      outp[3 * (size_t)i + 2] = o.z;
    }
  }
}
void launch_eval_pred(int kind, const double* in, int n, int* sign, double* outp, cudaStream_t s) {
  if (n > 0) k_eval_pred<<<grid_for(n, 128), 128, 0, s>>>(kind, in, n, sign, outp);
}


// A subsegment round that inserted nothing, gave up nothing and flagged no new
// candidate would repeat itself: its refused candidates become unsplittable.
// Decided per instance from its round counters (run after selection).
// stall rule for candidate i; returns 1 if it was given up
__device__ int stall_one(const DevMesh& m, const DevRound& r, int i) {
  if (cls_of(r, i) != CLS_SUBSEG || (r.status[i] & 0xff) != OUT_REJECT) return 0;
  const unsigned long long* q = m.instSt + (size_t)inst_of(r, i) * IS_COUNT;
  if (q[IS_SURV] || q[IS_UNSPL] || q[IS_NEWCAND]) return 0;
  r.status[i] = OUT_UNSPL | (RS_STRUCT << 8);
  m.Gflag[CKI(r.cand[i], m.capG)] |= F_UNSPL;
  m.dirtyG[CKI(r.cand[i], m.capG)] = 1;
  atomicAdd(&m.instSt[(size_t)inst_of(r, i) * IS_COUNT + IS_STALLED], 1ULL);
  return 1;
}
__device__ void flush_stall(const DevRound& r, unsigned moved) {
  if (moved) {
    atomicAdd(&r.stats[ST_UNSPL], (unsigned long long)moved);
    atomicAdd(&r.stats[ST_REJECT], (unsigned long long)(-(long long)moved));
  }
}
__global__ void k_stall(DevMesh m, DevRound r) {
  unsigned moved = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x)
    moved += stall_one(m, r, i);
  flush_stall(r, moved);
}
void launch_count_inst(const DevMesh& m, const uint8_t* candG, const uint8_t* candS,
                       const uint8_t* candT, cudaStream_t s) {
  long tot = (long)m.nG + m.nS + m.nT;
  if (tot > 0) k_count_inst<<<grid_for(tot, 256), 256, 0, s>>>(m, candG, candS, candT);
}
void launch_round_flags(const DevMesh& m, const uint8_t* candG, const uint8_t* candS,
                        const uint8_t* candT, uint8_t* out, cudaStream_t s) {
  long tot = (long)m.nG + m.nS + m.nT;
  if (tot > 0) k_round_flags<<<grid_for(tot, 256), 256, 0, s>>>(m, candG, candS, candT, out);
}
void launch_decode_cands(const DevMesh& m, int* cand, uint8_t* ccls, int* cinst, int n,
                         cudaStream_t s) {
  if (n > 0) k_decode_cands<<<grid_for(n, 256), 256, 0, s>>>(m, cand, ccls, cinst, n);
}
void launch_stall(const DevMesh& m, const DevRound& r, cudaStream_t s) {
  if (r.n > 0) k_stall<<<grid_for(r.n, 256), 256, 0, s>>>(m, r);
}

// ============================================================ small rounds
// A round with few candidates (kFusedDefault by default, at most kFusedMax)
// runs in one thread-block cluster (kFusedBlocks blocks on as many SMs, one
// warp per candidate, or several in turn): split, locate
// (with the start claims), growth in tier 1 (shared-memory workspaces) and,
// for regions that do not fit, tier 2 (global workspaces; candidate i uses
// tier-2 slab i), selection, the stall rule, the allocation scan and
// insertion, with cluster barriers instead of separate launches and host
// synchronisations between the steps. The host reserves capacity for the
// largest possible growth (tier-2 caps) before the launch and reads the totals
// afterwards.
// every block's global writes are visible to the whole cluster after this
__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  cooperative_groups::this_cluster().sync();
}

// true if candidate a (key ka, class ca, element ea) comes before b: key, then
// class, then the sorted vertex ids (the order of the sort + tie fix path)
__device__ bool cand_before(const DevMesh& m, unsigned long long ka, int ca, int ea,
                            unsigned long long kb, int cb, int eb) {
  if (ka != kb) return ka < kb;
  if (ca != cb) return ca < cb;
  int x[4], y[4];
  int nk = elem_key(m, ca, ea, x);
  elem_key(m, cb, eb, y);
  for (int q = 0; q < nk; ++q)
    if (x[q] != y[q]) return x[q] < y[q];
  return ea < eb;
}

// Block-level ordering of a fused round's candidates (block 0): src holds the
// round's elements (cls >= 0) or concatenated indices (cls < 0); the sorted
// element ids go to cand, with their classes and instances for cls < 0.
__device__ void fused_order(const DevMesh& m, int cls, const int* src, int n, int* cand,
                            uint8_t* ccls, int* cinst) {
  __shared__ unsigned long long sk[kFusedMax];
  __shared__ int se[kFusedMax];
  __shared__ uint8_t sc[kFusedMax];
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int t = threadIdx.x; t < np2; t += blockDim.x) {
    if (t < n) {
      int c = cls;
      int e = cls >= 0 ? src[t] : decode_cand(m, src[t], c);
      sk[t] = prio_key(m, c, e);
      se[t] = e;
      sc[t] = (uint8_t)c;
    } else {
      sk[t] = ~0ULL;  // after every real key (classes 0..2 stay below 3 << 62)
      se[t] = 0x7fffffff;
      sc[t] = 3;
    }
  }
  __syncthreads();
  for (int size = 2; size <= np2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < np2; t += blockDim.x) {
        const int u = t ^ stride;
        if (u > t) {
          const bool up = (t & size) == 0;
          const bool after =
              (sk[t] == ~0ULL || sk[u] == ~0ULL)
                  ? sk[t] > sk[u]
                  : cand_before(m, sk[u], sc[u], se[u], sk[t], sc[t], se[t]);
          if (after == up) {
            unsigned long long k = sk[t];
            sk[t] = sk[u];
            sk[u] = k;
            int e = se[t];
            se[t] = se[u];
            se[u] = e;
            uint8_t c = sc[t];
            sc[t] = sc[u];
            sc[u] = c;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    cand[t] = se[t];
    if (cls < 0) {
      const int c = sc[t], e = se[t];
      ccls[t] = (uint8_t)c;
      const int v0 = c == CLS_SUBSEG ? m.GV[CKI(e, m.capG)].x
                                     : (c == CLS_SUBFACE ? m.SV[CKI(e, m.capS)].x
                                                         : vid(m.T[CKI(e, m.capT)].v.x));
      cinst[t] = vinst(m, v0);
    }
  }
}

__global__ void __launch_bounds__(32 * kFusedWarps, 1) k_round_fused(DevMesh m, DevRound r, int* hint,
                                                                      int4* offs, FusedOut* out,
                                                                      int do_stall, const int* src,
                                                                      int* cand_w, uint8_t* ccls_w,
                                                                      int* cinst_w) {
  extern __shared__ int smraw[];
  __shared__ int t2chunks;  // shared-memory hash sets handed out in the tier-2 phase
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
  const int warp = blockIdx.x * kFusedWarps + wib, nwarps = gridDim.x * kFusedWarps;
  if (threadIdx.x == 0) t2chunks = 0;
  if (src) {  // order the candidates first (instead of separate key, sort and tie launches)
    if (blockIdx.x == 0) fused_order(m, r.cls, src, r.n, cand_w, ccls_w, cinst_w);
    cluster_barrier();
  }
  for (int i = tid; i < r.n; i += nthreads) {
    split_one(m, r, i);
    locate_one(m, r, hint, i);
  }
  cluster_barrier();
  GrowAcc acc;
  {
    Smem1* sm = reinterpret_cast<Smem1*>(smraw) + wib;
    Ws w{sm->cav, sm->hset, sm->bin, sm->bout, sm->bv, sm->fcav, sm->fbnd, sm->fbv};
    for (int i = warp; i < r.n; i += nwarps) {
      int* slab = r.slab1 + (size_t)i * SlabLayout<Tier1>::STRIDE;
      grow_one<Tier1>(m, r, i, w, slab, lane, acc);
      __syncwarp();
    }
  }
  cluster_barrier();
  int t2c = -2;  // this warp's shared-memory tier-2 hash set: -2 none yet, -1 global
  for (int i = warp; i < r.n; i += nwarps) {
    if (r.status[i] != OUT_RETRY) continue;  // the same value in every lane
    using L = SlabLayout<Tier2>;
    int* slab = r.slab2 + (size_t)i * L::STRIDE;
    if (lane == 0) r.slab2_of[i] = i;
    __syncwarp();
    Ws w2{slab + L::OFF_CAV, r.ws2 + (size_t)warp * Tier2::HCAP, slab + L::OFF_BIN,
          slab + L::OFF_BOUT, slab + L::OFF_BV, slab + L::OFF_FCAV, slab + L::OFF_FBND,
          slab + L::OFF_FBV};
    // the tier-1 workspaces are free now: the first kFusedT2Chunks warps of
    // the block to meet a tier-2 region keep their hash sets there
    if (t2c < -1) {
      int c = 0;
      if (lane == 0) c = atomicAdd(&t2chunks, 1);
      t2c = __shfl_sync(FULLMASK, c, 0);
      if (t2c >= kFusedT2Chunks) t2c = -1;
    }
    int* shs = t2c >= 0 ? smraw + (size_t)t2c * kT2FusedSlots : nullptr;
    grow_tier2(m, r, i, w2, slab, lane, acc, shs, kT2FusedSlots);
    __syncwarp();
    if (lane == 0) {
      if (r.status[i] == OUT_RETRY) set_status(r, i, OUT_UNSPL, RS_OVERFLOW);
      atomicAdd(&out->n2, 1);
    }
  }
  flush_acc(r, acc, lane);
  cluster_barrier();
  SelAcc sa;
  for (int i = warp; i < r.n; i += nwarps) select_one(m, r, i, lane, sa);
  flush_sel(r, sa, lane);
  cluster_barrier();
  if (do_stall) {
    unsigned moved = 0;
    for (int i = tid; i < r.n; i += nthreads) moved += stall_one(m, r, i);
    flush_stall(r, moved);
    cluster_barrier();
  }
  if (warp == 0) {  // exclusive scan of the new-element counts
    int4 run = make_int4(0, 0, 0, 0);
    for (int base = 0; base < r.n; base += 32) {
      const int i = base + lane;
      const int4 c = i < r.n ? r.counts[i] : make_int4(0, 0, 0, 0);
      int4 inc = c;
      for (int o = 1; o < 32; o <<= 1) {
        int4 t;
        t.x = __shfl_up_sync(FULLMASK, inc.x, o);
        t.y = __shfl_up_sync(FULLMASK, inc.y, o);
        t.z = __shfl_up_sync(FULLMASK, inc.z, o);
        t.w = __shfl_up_sync(FULLMASK, inc.w, o);
        if (lane >= o) inc = make_int4(inc.x + t.x, inc.y + t.y, inc.z + t.z, inc.w + t.w);
      }
      if (i < r.n)
        offs[i] = make_int4(run.x + inc.x - c.x, run.y + inc.y - c.y, run.z + inc.z - c.z,
                            run.w + inc.w - c.w);
      run.x += __shfl_sync(FULLMASK, inc.x, 31);
      run.y += __shfl_sync(FULLMASK, inc.y, 31);
      run.z += __shfl_sync(FULLMASK, inc.z, 31);
      run.w += __shfl_sync(FULLMASK, inc.w, 31);
    }
    if (lane == 0) out->tot = run;
  }
  cluster_barrier();
  for (int i = warp; i < r.n; i += nwarps) insert_one(m, r, hint, i, lane);
}
void launch_round_fused(const DevMesh& m, const DevRound& r, int* hint, int4* offs, FusedOut* out,
                        bool do_stall, const int* src, int* cand_w, uint8_t* ccls_w, int* cinst_w,
                        cudaStream_t s) {
  static bool attr = false;
  const size_t smem = sizeof(Smem1) * kFusedWarps;
  if (!attr) {
    cudaFuncSetAttribute(k_round_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if (r.n <= 0) return;
  // as many blocks (a power of two, at most kFusedBlocks) as the round has
  // warps' worth of candidates: a small round synchronises fewer SMs
  int blocks = 1;
  while (blocks < kFusedBlocks && blocks * kFusedWarps < r.n) blocks <<= 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(32 * kFusedWarps, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = blocks;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_round_fused, m, r, hint, offs, out, do_stall ? 1 : 0, src, cand_w,
                     ccls_w, cinst_w);
}

// checked build: first out-of-bounds index seen (site line, index, bound), or 0
int checked_error(int* info, cudaStream_t s) {
#ifdef CDR_CHECKED
  int v[4] = {0, 0, 0, 0};
  cudaMemcpyFromSymbolAsync(v, g_chk, sizeof(v), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int k = 0; k < 4; ++k) info[k] = v[k];
  return v[0];
#else
  (void)s;
  info[0] = info[1] = info[2] = info[3] = 0;
  return 0;
#endif
}

// enqueue a copy of the exact-arithmetic overflow flag (no synchronisation)
void exact_overflow_copy_async(int* dst, cudaStream_t s) {
  cudaMemcpyFromSymbolAsync(dst, g_exact_overflow, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
}

// diagnostic build: read (and clear) the phase counters; 0 if not built in
int phase_counters(unsigned long long* out32, cudaStream_t s) {
#ifdef CDR_PHASES
  cudaMemcpyFromSymbolAsync(out32, g_phase, sizeof(g_phase), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  unsigned long long z[32] = {};
  cudaMemcpyToSymbolAsync(g_phase, z, sizeof(z), 0, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  return 1;
#else
  (void)out32;
  (void)s;
  return 0;
#endif
}

int exact_overflow_flag(cudaStream_t s, bool reset) {
  int v = 0;
  cudaMemcpyFromSymbolAsync(&v, g_exact_overflow, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (reset && v) {
    int z = 0;
    cudaMemcpyToSymbolAsync(g_exact_overflow, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  }
  return v;
}

}  // namespace cdr
