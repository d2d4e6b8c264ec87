// Host driver and C-ABI of the refinement library (see include/cdr.h).
//
// cdr_create builds the device mesh from a CDT with constraint labels (Sec. 1 of
// Chen & Tan, I3D 2019); cdr_round runs one round of the paper's refinement step
// (Sec. 2): classify, order by priority, split points, locate, grow regions,
// select disjoint regions, insert; cdr_refine repeats rounds until no candidate
// is left. Device memory comes from the caller's allocator (or cudaMallocAsync).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include "../../include/cdr.h"
#include "kernels.cuh"
#include "mesh.cuh"

using namespace cdr;

namespace {

// ------------------------------------------------------------ device buffers
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct cdr_handle {
  cudaStream_t stream = nullptr;
  cdr_allocator alloc{};
  bool has_alloc = false;
  int err = 0;  // sticky allocation / CUDA failure
  DevMesh m{};
  int capV = 0, capT = 0, capS = 0, capG = 0;
  int hcount = 0;
  long long deadT = 0;     // retired tetrahedra not yet compacted away
  bool deadKnown = true;   // false after removals: count them before deciding
  double lastB = -1.0;
  unsigned epoch = 0;
  bool dt_mode = false;
  // mesh arrays
  Buf bV, bT, bTS, bTflag, bTmark, bTseed, bTfwd, bSV, bSN, bSflag, bSmust, bSmark, bGV, bGflag, bGmust,
      bFQ, bHK, bHV;
  // classification: candidate flags and dirty marks, kept from round to round
  Buf bCandS, bCandG, bCandT, bDirtyS, bDirtyG;
  bool fullClassify = true;  // the next classification tests every element
  // the next round's classification and counts were enqueued behind the last
  // round and are already in pinCnt / pin->cerr (one-mesh refinement only)
  bool preCounted = false;
  // round buffers
  int capR = 0, capR2 = 0, capWs2 = 0;
  Buf bCand, bCand2, bKeys, bKeys2, bSp, bLoc, bStatus, bSurv, bCounts, bOffs, bSlab1, bSlab2of,
      bList2, bSlab2, bWs2, bCkey, bTmp, bStats, bErr, bI32, bFused;
  size_t tmpBytes = 0;
  // points (Delaunay mode)
  Buf bPts, bHint, bPstate;
  int npts = 0;
  // last round, for the report
  int lastN = 0, lastCls = -1, lastN2 = 0;
  SlabOff lastS1 = slab_off<Tier1>();  // tier-1 slab layout of the last round
  // profiling: events around each kernel group, accumulated per round
  bool prof = false;
  bool profGrowOnly = false;  // time the region-growth groups only
  cudaEvent_t ev[2 * 32] = {};
  bool fused = true;  // small rounds as one kernel
  // launch tuning (cdr_set_tuning)
  int fusedMax = kFusedDefault;  // rounds with at most this many candidates run fused
  int grow1PerSM = 8;         // growth grid: at most this many blocks per SM
  int tier2Warps = 152 * 4;   // warps (workspaces) for tier-2 growth
  int tier1Cav = 0;           // tier-1 cavity capacity (0: Tier1::CAPC)
  int tier1Bnd = 0;           // tier-1 boundary-face capacity (0: Tier1::CAPB)
  int compactMin = 1 << 19;   // no compaction below this many tetrahedra
  int compactPct = 50;        // compact once this percentage of the slots is dead
  double prof_ms[32] = {};
  long long prof_calls[32] = {};
  long long prof_ctr[32] = {};
  // instances: a plain handle holds one; a batch holds several as disconnected
  // parts of this mesh (Vinst set)
  int ninst = 1, capI = 0;
  Buf bVinst, bInstB, bInstG2, bInstCls, bInstCnt, bInstSt, bCcls, bCinst, bRflags;
  unsigned long long* pinCnt = nullptr;  // pinned: per-instance classification counts
  int* pinCls = nullptr;                 // pinned: per-instance class of the round
  unsigned long long* pinSt = nullptr;   // pinned: per-instance round counters
  std::vector<int> instCls;              // host copy of the round's classes
  // batch bookkeeping (host)
  bool batch = false;
  int mixed = 0;  // round kind: 0 one class, 1 every class, 2 subsegments + subfaces
  struct Inst {
    int state = 0;  // 0 free slot, 1 refining, 2 done
    int of = 0, nf = 0, oseg = 0, nseg = 0;
    double B = 0;
    cdr_stats st{};
  };
  std::vector<Inst> insts;
  std::vector<int> freeSlots;
  int segIds = 0;
  cdr_options opts{};
  // pinned host staging for the values a round reads back
  struct Pinned {
    unsigned long long c3[4];
    unsigned long long st[ST_COUNT];
    unsigned long long ctr[ST_COUNT];
    int4 lastOff, lastCnt;
    int cerr, n2, ovf;
  }* pin = nullptr;
  // checkpoint
  std::vector<Buf> ck;
  DevMesh ckm{};
  int ck_hcount = 0;
  long long ck_deadT = 0;
  bool has_ck = false;
};

namespace {

int set_err(cdr_handle* h, int e) {
  if (!h->err) h->err = e;
  return e;
}

void* dalloc(cdr_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc((uint64_t)bytes, h->alloc.ctx, (void*)h->stream);
  } else {
    if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) p = nullptr;
  }
  return p;
}
void dfree(cdr_handle* h, Buf& b) {
  if (!b.p) return;
  if (h->has_alloc) h->alloc.free(b.p, (uint64_t)b.bytes, h->alloc.ctx, (void*)h->stream);
  else cudaFreeAsync(b.p, h->stream);
  b.p = nullptr;
  b.bytes = 0;
}
// (re)allocate b to hold `bytes`, keeping the first `keep` bytes
bool ensure(cdr_handle* h, Buf& b, size_t bytes, size_t keep = 0) {
  if (b.bytes >= bytes && b.p) return true;
  size_t nb = std::max(bytes, b.bytes + b.bytes / 2);
  void* p = dalloc(h, nb);
  if (!p) {
    set_err(h, CDR_ERR_OOM);
    return false;
  }
  if (keep && b.p) cudaMemcpyAsync(p, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, h->stream);
  dfree(h, b);
  b.p = p;
  b.bytes = nb;
  return true;
}
template <class T>
T* ptr(Buf& b) {
  return reinterpret_cast<T*>(b.p);
}

int cuda_status(cdr_handle* h) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(h, CDR_ERR_CUDA);
  return h->err;
}

// bind the mesh pointers after any reallocation
void bind(cdr_handle* h) {
  DevMesh& m = h->m;
  m.V = ptr<V4>(h->bV);
  m.T = ptr<TetRec>(h->bT);
  m.TS = ptr<int4>(h->bTS);
  m.Tflag = ptr<uint8_t>(h->bTflag);
  m.Tmark = ptr<unsigned long long>(h->bTmark);
  m.Tseed = ptr<unsigned long long>(h->bTseed);
  m.Tfwd = ptr<int>(h->bTfwd);
  m.SV = ptr<int4>(h->bSV);
  m.SN = ptr<int4>(h->bSN);
  m.Sflag = ptr<uint8_t>(h->bSflag);
  m.Smust = ptr<uint8_t>(h->bSmust);
  m.Smark = ptr<unsigned long long>(h->bSmark);
  m.GV = ptr<int4>(h->bGV);
  m.Gflag = ptr<uint8_t>(h->bGflag);
  m.Gmust = ptr<uint8_t>(h->bGmust);
  m.FQ = ptr<V4>(h->bFQ);
  m.HK = ptr<unsigned long long>(h->bHK);
  m.HV = ptr<int>(h->bHV);
  m.Vinst = h->batch ? ptr<int>(h->bVinst) : nullptr;
  m.candT = ptr<uint8_t>(h->bCandT);
  m.candS = ptr<uint8_t>(h->bCandS);
  m.candG = ptr<uint8_t>(h->bCandG);
  m.dirtyS = ptr<uint8_t>(h->bDirtyS);
  m.dirtyG = ptr<uint8_t>(h->bDirtyG);
  m.capV = h->capV;
  m.capT = h->capT;
  m.capS = h->capS;
  m.capG = h->capG;
}

bool grow_verts(cdr_handle* h, int need) {
  if (need <= h->capV) return true;
  int cap = std::max(need, h->capV + h->capV / 2);
  if (cap > kMaxVerts) return false;
  if (!ensure(h, h->bV, (size_t)cap * sizeof(V4), (size_t)h->m.nV * sizeof(V4))) return false;
  if (h->batch && !ensure(h, h->bVinst, (size_t)cap * 4, (size_t)h->m.nV * 4)) return false;
  h->capV = cap;
  bind(h);
  return true;
}
bool grow_tets(cdr_handle* h, int need) {
  if (need <= h->capT) return true;
  int cap = std::max(need, h->capT + h->capT / 2);
  if (cap > kMaxTets) return false;
  size_t n = h->m.nT;
  bool ok = ensure(h, h->bT, cap * sizeof(TetRec), n * sizeof(TetRec)) &&
            ensure(h, h->bTS, cap * sizeof(int4), n * sizeof(int4)) &&
            ensure(h, h->bTflag, cap, n) &&
            ensure(h, h->bTmark, cap * sizeof(unsigned long long), n * 8) &&
            ensure(h, h->bTseed, cap * sizeof(unsigned long long), n * 8) &&
            ensure(h, h->bTfwd, cap * sizeof(int), n * 4) && ensure(h, h->bCandT, cap + 16, n);
  if (!ok) return false;
  h->capT = cap;
  bind(h);
  return true;
}
bool grow_subfaces(cdr_handle* h, int need) {
  if (need <= h->capS) return true;
  int cap = std::max(need, h->capS + h->capS / 2);
  size_t n = h->m.nS;
  bool ok = ensure(h, h->bSV, cap * sizeof(int4), n * sizeof(int4)) &&
            ensure(h, h->bSN, cap * sizeof(int4), n * sizeof(int4)) &&
            ensure(h, h->bSflag, cap, n) && ensure(h, h->bSmust, cap, n) &&
            ensure(h, h->bSmark, cap * 8, n * 8) && ensure(h, h->bCandS, cap + 16, n) &&
            ensure(h, h->bDirtyS, cap, n);
  if (!ok) return false;
  h->capS = cap;
  bind(h);
  return true;
}
bool grow_subsegs(cdr_handle* h, int need) {
  if (need <= h->capG) return true;
  int cap = std::max(need, h->capG + h->capG / 2);
  size_t n = h->m.nG;
  bool ok = ensure(h, h->bGV, cap * sizeof(int4), n * sizeof(int4)) &&
            ensure(h, h->bGflag, cap, n) && ensure(h, h->bGmust, cap, n) &&
            ensure(h, h->bCandG, cap + 16, n) && ensure(h, h->bDirtyG, cap, n);
  if (!ok) return false;
  h->capG = cap;
  bind(h);
  return true;
}
// subsegment hash: rebuild with a capacity of at least 4x the keys it will hold
bool rebuild_hash(cdr_handle* h, int keys) {
  size_t cap = 64;
  while (cap < (size_t)keys * 4) cap <<= 1;
  if (!ensure(h, h->bHK, cap * 8) || !ensure(h, h->bHV, cap * 4)) return false;
  bind(h);
  h->m.hmask = (int)cap - 1;
  launch_hash_clear(h->m, h->stream);
  launch_hash_insert_subsegs(h->m, 0, h->m.nG, h->stream);
  h->hcount = h->m.nG;
  return true;
}

// ------------------------------------------------------------- small kernels
__global__ void k_gather_u64(const unsigned long long* src, const int* perm, int n,
                             unsigned long long* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}
__global__ void k_gather_u32(const unsigned* src, const int* perm, int n, unsigned* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}
__global__ void k_iota(int* a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}
__global__ void k_xyz_to_v4(const double* xyz, int n, V4* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_v4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.0);
}
__global__ void k_init_subsegs(int4* GV, uint8_t* Gf, uint8_t* Gm, const int* segs,
                               const int* sid, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    GV[i] = make_int4(segs[2 * i], segs[2 * i + 1], sid[i], -1);
    Gf[i] = 0;
    Gm[i] = 0;
  }
}
// Element flags given with the input (a mesh exported between rounds), from
// the export's coding (tetrahedra bit1 unsplittable; subfaces and subsegments
// bit0 must split, bit1 unsplittable) into the device flags. Element i of
// each kind is input element i.
__global__ void k_apply_flags(DevMesh m, const uint8_t* tf, const uint8_t* sf, const uint8_t* gf) {
  const long n = (long)m.nT + m.nS + m.nG;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    if (i < m.nT) {
      if (tf && (tf[i] & 2)) m.Tflag[i] |= F_UNSPL;
    } else if (i < (long)m.nT + m.nS) {
      const long k = i - m.nT;
      if (!sf) continue;
      if (sf[k] & 2) m.Sflag[k] |= F_UNSPL;
      m.Smust[k] = (sf[k] & 1) ? 1 : 0;
    } else {
      const long k = i - m.nT - m.nS;
      if (!gf) continue;
      if (gf[k] & 2) m.Gflag[k] |= F_UNSPL;
      m.Gmust[k] = (gf[k] & 1) ? 1 : 0;
    }
  }
}
__global__ void k_scatter_slab2(const int* list2, int n2, int* slab2_of) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x)
    slab2_of[list2[j]] = j;
}
struct Int4Sum {
  __host__ __device__ int4 operator()(const int4& a, const int4& b) const {
    return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
  }
};
// points: one candidate per located tetrahedron (the smallest rank) this round
__global__ void k_point_prefilter(DevMesh m, int* status, const int* loc, int n,
                                  unsigned long long epoch, int pass) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (status[i] != OUT_OK) continue;
    unsigned long long mk = (epoch << 32) | (unsigned)i;
    if (pass == 0) atomicMin(&m.Tmark[loc[i]], mk);
    else if (m.Tmark[loc[i]] != mk) status[i] = OUT_UNSPL | (RS_NONE << 8) | (1 << 16);
  }
}
__global__ void k_point_flags(const int* state, int n, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    flag[i] = state[i] == 0 ? 1 : 0;
}
// a deferred point (bit 16 of its status) is neither marked nor counted
__global__ void k_undefer(int* status, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (status[i] & (1 << 16)) status[i] = OUT_REJECT | (RS_NONE << 8);
}

inline int gridn(long n, int b = 256) {
  long g = (n + b - 1) / b;
  return (int)std::max(1L, std::min(g, 152L * 32));
}

// CUB temporary storage
bool tmp_ensure(cdr_handle* h, size_t bytes) { return ensure(h, h->bTmp, bytes); }

// lexicographic sort of (hi, lo): sorted keys and the permutation of original
// indices (two stable radix passes, low key first)
bool sort2(cdr_handle* h, const unsigned long long* hi, const unsigned* lo, int n,
           unsigned long long* hi_s, unsigned* lo_s, int* perm) {
  Buf scr;
  if (!ensure(h, scr, (size_t)n * 20 + 256)) return false;
  char* base = ptr<char>(scr);
  unsigned long long* hi1 = reinterpret_cast<unsigned long long*>(base);
  int* idx0 = reinterpret_cast<int*>(base + (size_t)n * 8);
  unsigned* lo1 = reinterpret_cast<unsigned*>(base + (size_t)n * 12);
  int* perm1 = reinterpret_cast<int*>(base + (size_t)n * 16);
  k_iota<<<gridn(n), 256, 0, h->stream>>>(idx0, n);
  size_t tb = 0, tb2 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, lo, lo1, idx0, perm1, n, 0, 32, h->stream);
  cub::DeviceRadixSort::SortPairs(nullptr, tb2, hi1, hi_s, perm1, perm, n, 0, 64, h->stream);
  if (!tmp_ensure(h, std::max(tb, tb2))) return false;
  tb = h->bTmp.bytes;
  cub::DeviceRadixSort::SortPairs(h->bTmp.p, tb, lo, lo1, idx0, perm1, n, 0, 32, h->stream);
  k_gather_u64<<<gridn(n), 256, 0, h->stream>>>(hi, perm1, n, hi1);
  tb = h->bTmp.bytes;
  cub::DeviceRadixSort::SortPairs(h->bTmp.p, tb, hi1, hi_s, perm1, perm, n, 0, 64, h->stream);
  k_gather_u32<<<gridn(n), 256, 0, h->stream>>>(lo, perm, n, lo_s);
  cudaStreamSynchronize(h->stream);
  dfree(h, scr);
  return cuda_status(h) == 0;
}

__global__ void k_count_bad(DevMesh m, unsigned long long* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.nT; t += gridDim.x * blockDim.x)
    if ((m.Tflag[t] & (F_DEAD | F_BAD)) == F_BAD) atomicAdd(out, 1ULL);
}
// per-candidate report sizes: cavity size when the cavity is complete
__global__ void k_report_sizes(DevRound r, int* ncav, int* nbnd, int* nfcav) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x) {
    int j = r.slab2_of ? r.slab2_of[i] : -1;
    const int* slab = j >= 0 ? r.slab2 + (size_t)j * SlabLayout<Tier2>::STRIDE
                             : r.slab1 + (size_t)i * r.s1.STRIDE;
    int st = r.status[i];
    int oc = st & 0xff, rs = (st >> 8) & 0xff;
    bool full = oc == OUT_OK || (oc == OUT_REJECT && rs == RS_ENCROACH) || rs == RS_GUARD ||
                rs == RS_STARDEL || (rs == RS_ENCROACH_UNSPL && slab[0] > 0);
    ncav[i] = full ? slab[0] : 0;
    nbnd[i] = full ? slab[1] : 0;
    nfcav[i] = full ? slab[2] : 0;
  }
}

unsigned next_epoch(cdr_handle* h) { return 0xFFFFFFFFu - (++h->epoch); }

// kernel groups timed when profiling is on
enum { PG_CLASSIFY = 0, PG_ORDER, PG_SPLIT, PG_LOCATE, PG_GROW1, PG_GROW2, PG_SELECT, PG_SCAN,
       PG_INSERT, PG_COMPACT, PG_FUSED, PG_N };
inline void pmark(cdr_handle* h, int g, int which) {
  if (!h->prof) return;
  if (h->profGrowOnly && g != PG_GROW1 && g != PG_GROW2) return;
  if (!h->ev[2 * g + which]) cudaEventCreate(&h->ev[2 * g + which]);
  cudaEventRecord(h->ev[2 * g + which], h->stream);
}
// after the round's final synchronisation
inline void pcollect(cdr_handle* h, const bool* used) {
  if (!h->prof) return;
  for (int g = 0; g < PG_N; ++g) {
    if (!used[g]) continue;
    if (h->profGrowOnly && g != PG_GROW1 && g != PG_GROW2) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[2 * g], h->ev[2 * g + 1]) == cudaSuccess) {
      h->prof_ms[g] += ms;
      h->prof_calls[g] += 1;
    }
  }
}

bool ensure_pinned(cdr_handle* h) {
  if (h->pin) return true;
  void* p = nullptr;
  if (cudaMallocHost(&p, sizeof(*h->pin)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->pin = static_cast<decltype(h->pin)>(p);
  return true;
}

// per-instance device arrays and pinned staging for at least n instances
bool ensure_instances(cdr_handle* h, int n) {
  if (n <= h->capI && h->pinCnt) return true;
  int c = std::max(n, std::max(16, 2 * h->capI));
  if (!ensure(h, h->bInstB, (size_t)c * 8, (size_t)h->capI * 8) ||
      !ensure(h, h->bInstG2, (size_t)c * 8, (size_t)h->capI * 8) ||
      !ensure(h, h->bInstCls, (size_t)c * 4) || !ensure(h, h->bInstCnt, (size_t)c * 3 * 8) ||
      !ensure(h, h->bInstSt, (size_t)c * IS_COUNT * 8))
    return false;
  void* a = nullptr;
  void* b = nullptr;
  void* q = nullptr;
  if (cudaMallocHost(&a, (size_t)c * 3 * 8) != cudaSuccess ||
      cudaMallocHost(&b, (size_t)c * 4) != cudaSuccess ||
      cudaMallocHost(&q, (size_t)c * IS_COUNT * 8) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaFreeHost(a);
    if (b) cudaFreeHost(b);
    return false;
  }
  if (h->pinCnt) cudaFreeHost(h->pinCnt);
  if (h->pinCls) cudaFreeHost(h->pinCls);
  if (h->pinSt) cudaFreeHost(h->pinSt);
  h->pinCnt = static_cast<unsigned long long*>(a);
  h->pinCls = static_cast<int*>(b);
  h->pinSt = static_cast<unsigned long long*>(q);
  h->capI = c;
  DevMesh& m = h->m;
  m.instCls = ptr<int>(h->bInstCls);
  m.instCnt = ptr<unsigned long long>(h->bInstCnt);
  m.instSt = ptr<unsigned long long>(h->bInstSt);
  if (h->batch) {
    m.instB = ptr<double>(h->bInstB);
    m.instG2 = ptr<double>(h->bInstG2);
  }
  return true;
}

bool ensure_round(cdr_handle* h, int n) {
  if (n <= h->capR && h->bCand.p) return true;
  int c = std::max(n, 1024);
  bool ok = ensure(h, h->bCand, (size_t)c * 4) && ensure(h, h->bCand2, (size_t)c * 4) &&
            ensure(h, h->bKeys, (size_t)c * 8) && ensure(h, h->bKeys2, (size_t)c * 8) &&
            ensure(h, h->bSp, (size_t)c * sizeof(V4)) && ensure(h, h->bLoc, (size_t)c * 4) &&
            ensure(h, h->bStatus, (size_t)c * 4) && ensure(h, h->bSurv, (size_t)c * 4) &&
            ensure(h, h->bCounts, (size_t)c * 16) && ensure(h, h->bOffs, (size_t)(c + 1) * 16) &&
            ensure(h, h->bSlab1,
                   (size_t)c * std::max(SlabLayout<Tier1>::STRIDE, SlabLayout<Tier1Big>::STRIDE) *
                       4) &&
            ensure(h, h->bSlab2of, (size_t)c * 4) && ensure(h, h->bList2, (size_t)c * 4) &&
            ensure(h, h->bCkey, (size_t)c * 16) && ensure(h, h->bStats, 32 * 8) &&
            ensure(h, h->bErr, 64) && ensure(h, h->bI32, (size_t)(c + 1) * 4) &&
            ensure(h, h->bCcls, (size_t)c) && ensure(h, h->bCinst, (size_t)c * 4);
  if (ok) h->capR = c;
  return ok;
}

DevRound make_round(cdr_handle* h, int cls, int n, double B) {
  DevRound r{};
  r.cls = cls;
  r.n = n;
  r.t1cav = h->tier1Cav;
  r.t1bnd = h->tier1Bnd;
  r.s1 = slab_off<Tier1>();
  r.cand = ptr<int>(h->bCand2);
  r.given = ptr<double>(h->bPts);
  r.loc = ptr<int>(h->bLoc);
  r.sp = ptr<V4>(h->bSp);
  r.status = ptr<int>(h->bStatus);
  r.slab1 = ptr<int>(h->bSlab1);
  r.slab2 = ptr<int>(h->bSlab2);
  r.slab2_of = ptr<int>(h->bSlab2of);
  r.ws2 = ptr<int>(h->bWs2);
  r.n2 = 0;
  r.list2 = ptr<int>(h->bList2);
  r.survived = ptr<int>(h->bSurv);
  r.counts = ptr<int4>(h->bCounts);
  r.offs = ptr<int4>(h->bOffs);
  r.point_state = ptr<int>(h->bPstate);
  r.stats = ptr<unsigned long long>(h->bStats);
  r.candG = (cls == CLS_SUBSEG || cls < 0) ? ptr<uint8_t>(h->bCandG) : nullptr;
  r.B = B;
  if (cls < 0) {  // every instance serves its own class
    r.ccls = ptr<uint8_t>(h->bCcls);
    r.cinst = ptr<int>(h->bCinst);
  }
  return r;
}

struct RoundOut {
  int cls = -1;
  long long cand = 0, ins = 0, rej = 0, unspl = 0, blasted = 0;
};

// count the live tetrahedra; compact when more than half are dead
int maybe_compact(cdr_handle* h, bool force) {
  DevMesh& m = h->m;
  if (!force && m.nT < h->compactMin) return 0;
  if (!force && h->deadKnown && (long long)h->deadT * 100 < (long long)m.nT * h->compactPct)
    return 0;
  Buf alive, newid;
  if (!ensure(h, alive, (size_t)m.nT * 4 + 64) || !ensure(h, newid, (size_t)(m.nT + 1) * 4 + 64))
    return CDR_ERR_OOM;
  launch_compact_flags(m, ptr<int>(alive), h->stream);
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, ptr<int>(alive), ptr<int>(newid), m.nT, h->stream);
  if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
  tb = h->bTmp.bytes;
  cub::DeviceScan::ExclusiveSum(h->bTmp.p, tb, ptr<int>(alive), ptr<int>(newid), m.nT, h->stream);
  int last[2] = {0, 0};
  cudaMemcpyAsync(&last[0], ptr<int>(newid) + m.nT - 1, 4, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(&last[1], ptr<int>(alive) + m.nT - 1, 4, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  int live = last[0] + last[1];
  h->deadT = m.nT - live;
  h->deadKnown = true;
  if (!force && (long long)h->deadT * 100 < (long long)m.nT * h->compactPct) {
    dfree(h, alive);
    dfree(h, newid);
    return 0;
  }
  Buf T2, TS2, F2;
  if (!ensure(h, T2, (size_t)h->capT * sizeof(TetRec)) ||
      !ensure(h, TS2, (size_t)h->capT * sizeof(int4)) || !ensure(h, F2, (size_t)h->capT))
    return CDR_ERR_OOM;
  launch_compact_move(m, ptr<int>(newid), ptr<TetRec>(T2), ptr<int4>(TS2), ptr<uint8_t>(F2),
                      h->dt_mode ? ptr<int>(h->bHint) : nullptr, h->dt_mode ? h->npts : 0,
                      h->stream);
  launch_compact_fix(m, ptr<int>(newid), h->stream);
  cudaStreamSynchronize(h->stream);
  std::swap(h->bT, T2);
  std::swap(h->bTS, TS2);
  std::swap(h->bTflag, F2);
  dfree(h, T2);
  dfree(h, TS2);
  dfree(h, F2);
  m.nT = live;
  h->deadT = 0;
  h->fullClassify = true;
  bind(h);
  cudaMemsetAsync(h->bTmark.p, 0xff, (size_t)h->capT * 8, h->stream);
  cudaMemsetAsync(h->bTseed.p, 0xff, (size_t)h->capT * 8, h->stream);
  cudaMemsetAsync(h->bTfwd.p, 0xff, (size_t)h->capT * 4, h->stream);
  dfree(h, alive);
  dfree(h, newid);
  h->prof_ctr[13] += 1;  // compactions run
  return cuda_status(h);
}

// A refinement round with few candidates as one kernel (k_round_fused): the
// capacity for the largest growth the kernel could produce is reserved first,
// the totals are read back once at the end.
// Classification and per-instance candidate counts (Sec. 2: a round serves the
// first class with work), read back into pinCnt and pin->cerr at the next
// synchronisation. add: the last round's additions when the host has not read
// them yet (one-mesh handles only), else null.
void enqueue_classify(cdr_handle* h, const int4* add) {
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  const int ni = h->ninst;
  cudaMemsetAsync(h->bErr.p, 0, 64, s);
  pmark(h, PG_CLASSIFY, 0);
  launch_classify(m, h->fullClassify, ptr<int>(h->bErr), s, add);
  h->fullClassify = false;
  pmark(h, PG_CLASSIFY, 1);
  h->prof_ctr[15] += 2;  // classification + counts
  cudaMemsetAsync(h->bInstCnt.p, 0, (size_t)ni * 3 * 8, s);
  if (h->batch)
    launch_count_inst(m, ptr<uint8_t>(h->bCandG), ptr<uint8_t>(h->bCandS),
                      ptr<uint8_t>(h->bCandT), s);
  else
    launch_count_single(m, ptr<unsigned long long>(h->bInstCnt), s, add);
  cudaMemcpyAsync(h->pinCnt, h->bInstCnt.p, (size_t)ni * 3 * 8, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&h->pin->cerr, h->bErr.p, 4, cudaMemcpyDeviceToHost, s);
}

// Enqueue the next round's classification behind this round's kernels, so
// that the round's final synchronisation reads both: one-mesh refinement
// only, and not when the next round must test every element anyway.
bool enqueue_next_classify(cdr_handle* h, const int4* add) {
  if (h->batch || h->dt_mode || h->fullClassify) return false;
  enqueue_classify(h, add);
  return true;
}

int round_fused(cdr_handle* h, int cls, int n, double B, RoundOut* ro, bool unsorted) {
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  using T2 = Tier2;
  if (!grow_verts(h, m.nV + n) || !grow_tets(h, m.nT + n * T2::CAPB) ||
      !grow_subfaces(h, m.nS + n * T2::CAPFB) || !grow_subsegs(h, m.nG + n) ||
      !ensure(h, h->bSlab2, (size_t)n * SlabLayout<T2>::STRIDE * 4) ||
      !ensure(h, h->bWs2, (size_t)kFusedBlocks * kFusedWarps * T2::HCAP * 4) ||
      !ensure(h, h->bFused, sizeof(FusedOut)))
    return h->err ? h->err : CDR_ERR_OOM;
  if ((size_t)(h->hcount + 2 * n) * 2 > (size_t)m.hmask + 1) {
    if (!rebuild_hash(h, (m.nG + 2 * n) * 2)) return CDR_ERR_OOM;
  }
  DevRound r = make_round(h, cls, n, B);
  r.slab2 = ptr<int>(h->bSlab2);
  r.ws2 = ptr<int>(h->bWs2);
  r.nws2 = kFusedBlocks * kFusedWarps;
  r.ckey = ptr<int4>(h->bCkey);
  r.seed_epoch = next_epoch(h);
  r.epoch = next_epoch(h);
  cudaMemsetAsync(h->bStats.p, 0, ST_COUNT * 8, s);
  cudaMemsetAsync(h->bInstSt.p, 0, (size_t)h->ninst * IS_COUNT * 8, s);
  cudaMemsetAsync(h->bFused.p, 0, sizeof(FusedOut), s);
  const bool stall =
      cls == CLS_SUBSEG ||
      (cls < 0 && (std::find(h->instCls.begin(), h->instCls.end(), CLS_SUBSEG) != h->instCls.end() ||
                   std::find(h->instCls.begin(), h->instCls.end(), 3) != h->instCls.end() ||
                   std::find(h->instCls.begin(), h->instCls.end(), 4) != h->instCls.end()));
  bool used[PG_N] = {};
  pmark(h, PG_FUSED, 0);
  launch_round_fused(m, r, ptr<int>(h->bHint), ptr<int4>(h->bOffs), ptr<FusedOut>(h->bFused),
                     stall, unsorted ? ptr<int>(h->bCand) : nullptr, ptr<int>(h->bCand2),
                     ptr<uint8_t>(h->bCcls), ptr<int>(h->bCinst), s);
  pmark(h, PG_FUSED, 1);
  used[PG_FUSED] = true;
  h->prof_ctr[15] += 1;
  const bool next = enqueue_next_classify(
      h, reinterpret_cast<const int4*>(ptr<char>(h->bFused) + offsetof(FusedOut, tot)));
  FusedOut fo;
  cudaMemcpyAsync(&h->pin->lastOff, ptr<char>(h->bFused), sizeof(int4), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&h->pin->n2, ptr<char>(h->bFused) + offsetof(FusedOut, n2), 4,
                  cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h->pin->ctr, h->bStats.p, sizeof(h->pin->ctr), cudaMemcpyDeviceToHost, s);
  h->pin->ovf = 0;
  exact_overflow_copy_async(&h->pin->ovf, s);
  if (h->batch)
    cudaMemcpyAsync(h->pinSt, h->bInstSt.p, (size_t)h->ninst * IS_COUNT * 8,
                    cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (cuda_status(h)) return h->err;
  fo.tot = h->pin->lastOff;
  fo.n2 = h->pin->n2;
  h->prof_ctr[ST_RETRY] += fo.n2;  // regions re-grown in tier 2
  if (h->pin->ovf) {
    exact_overflow_flag(s, true);
    return set_err(h, CDR_ERR_INTERNAL);
  }
  {
    int info[4];
    if (checked_error(info, s)) {
      fprintf(stderr, "cdr checked build: bad index %d (bound %d) at kernels.cu:%d, round %u\n",
              info[2], info[3], info[1], h->epoch);
      return set_err(h, CDR_ERR_INTERNAL);
    }
  }
  const unsigned long long* ctr = h->pin->ctr;
  if (ctr[ST_ITER]) return set_err(h, CDR_ERR_INTERNAL);
  m.nV += fo.tot.x;
  m.nT += fo.tot.y;
  m.nS += fo.tot.z;
  m.nG += fo.tot.w;
  h->hcount += 2 * fo.tot.w;
  h->lastN = n;
  h->lastN2 = fo.n2;
  h->lastCls = cls;
  h->lastS1 = slab_off<Tier1>();
  if (ro) {
    ro->cls = cls;
    ro->cand = n;
    ro->ins = (long long)ctr[ST_SURV];
    ro->rej = (long long)ctr[ST_REJECT];
    ro->unspl = (long long)ctr[ST_UNSPL];
    ro->blasted = (long long)ctr[ST_OK] + (long long)ctr[ST_BLAST];
  }
  pcollect(h, used);
  // growth work of fused rounds is counted apart (16..18) from the separately
  // launched growth kernels (6..8), whose timings the roofline uses
  for (int k = 0; k < ST_COUNT && k < 15; ++k)
    if (k != ST_TESTED && k != ST_CAV && k != ST_BND) h->prof_ctr[k] += (long long)ctr[k];
  h->prof_ctr[16] += (long long)ctr[ST_TESTED];
  h->prof_ctr[17] += (long long)ctr[ST_CAV];
  h->prof_ctr[18] += (long long)ctr[ST_BND];
  h->deadT += (long long)ctr[ST_DEADT];
  h->preCounted = next;
  return cuda_status(h);
}

// whether a refinement round of n candidates runs as one kernel
inline bool use_fused(const cdr_handle* h, int n) { return h->fused && n <= h->fusedMax; }

// the shared body of a round once the ordered candidate list is in bCand2
// (unsorted: the candidates are still unordered in bCand; fused rounds only)
int round_core(cdr_handle* h, int cls, int n, double B, RoundOut* ro, bool unsorted = false) {
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  if (!ensure_pinned(h)) return CDR_ERR_OOM;
  if (cls != CLS_POINT && use_fused(h, n)) return round_fused(h, cls, n, B, ro, unsorted);
  if (unsorted) return set_err(h, CDR_ERR_INTERNAL);
  DevRound r = make_round(h, cls, n, B);
  cudaMemsetAsync(h->bStats.p, 0, ST_COUNT * 8, s);
  if (cls != CLS_POINT) cudaMemsetAsync(h->bInstSt.p, 0, (size_t)h->ninst * IS_COUNT * 8, s);
  r.ckey = ptr<int4>(h->bCkey);
  r.rflag = ptr<int>(h->bSurv);  // scratch until selection
  if (cls != CLS_POINT) r.seed_epoch = next_epoch(h);  // claims are made while locating
  bool used[PG_N] = {};
  pmark(h, PG_SPLIT, 0);
  launch_split(m, r, s);
  pmark(h, PG_SPLIT, 1);
  h->prof_ctr[15] += 1;
  used[PG_SPLIT] = true;
  if (cls == CLS_POINT)
    launch_follow_fwd(m, ptr<int>(h->bHint), ptr<int>(h->bPstate), h->npts, s);
  pmark(h, PG_LOCATE, 0);
  launch_locate(m, r, ptr<int>(h->bHint), s);
  pmark(h, PG_LOCATE, 1);
  h->prof_ctr[15] += cls == CLS_POINT ? 4 : 1;
  used[PG_LOCATE] = true;
  if (cls == CLS_POINT) {
    unsigned long long e0 = next_epoch(h);
    k_point_prefilter<<<gridn(n), 256, 0, s>>>(m, r.status, r.loc, n, e0, 0);
    k_point_prefilter<<<gridn(n), 256, 0, s>>>(m, r.status, r.loc, n, e0, 1);
  }
  if (cls == CLS_POINT) {
    r.seed_epoch = next_epoch(h);
    launch_seed(m, r, s);
    h->prof_ctr[15] += 1;
  }
  r.epoch = next_epoch(h);
  r.s1 = slab1_layout(grow1_tets_only(r));
  h->lastS1 = r.s1;
  pmark(h, PG_GROW1, 0);
  launch_grow1(m, r, h->grow1PerSM, s);
  pmark(h, PG_GROW1, 1);
  h->prof_ctr[15] += 1;
  used[PG_GROW1] = true;
  // tier 2 for regions that did not fit (flagged by the growth kernel)
  {
    int* flag = r.rflag;
    size_t tb = 0;
    int* nsel = ptr<int>(h->bErr) + 4;
    cub::DeviceSelect::Flagged(nullptr, tb, thrust::counting_iterator<int>(0), flag,
                               ptr<int>(h->bList2), nsel, n, s);
    if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
    tb = h->bTmp.bytes;
    cub::DeviceSelect::Flagged(h->bTmp.p, tb, thrust::counting_iterator<int>(0), flag,
                               ptr<int>(h->bList2), nsel, n, s);
    cudaMemcpyAsync(&h->pin->n2, nsel, 4, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int n2 = h->pin->n2;
    h->prof_ctr[ST_RETRY] += n2;  // regions re-grown in tier 2
    if (n2 > 0) {
      const size_t stride2 = SlabLayout<Tier2>::STRIDE;
      int warps = std::min(n2, h->tier2Warps);
      warps += warps & 1;  // the launch runs two warps per block
      if (!ensure(h, h->bSlab2, (size_t)n2 * stride2 * 4) ||
          !ensure(h, h->bWs2, (size_t)warps * Tier2::HCAP * 4))
        return CDR_ERR_OOM;
      r.slab2 = ptr<int>(h->bSlab2);
      r.ws2 = ptr<int>(h->bWs2);
      r.nws2 = warps;
      r.n2 = n2;
      k_scatter_slab2<<<gridn(n2), 256, 0, s>>>(r.list2, n2, r.slab2_of);
      pmark(h, PG_GROW2, 0);
      launch_grow2(m, r, warps, s);
      pmark(h, PG_GROW2, 1);
      h->prof_ctr[15] += 2;
      used[PG_GROW2] = true;
    }
    h->lastN2 = n2;
  }
  if (cls == CLS_POINT) k_undefer<<<gridn(n), 256, 0, s>>>(r.status, n);
  pmark(h, PG_SELECT, 0);
  launch_select(m, r, s);
  pmark(h, PG_SELECT, 1);
  h->prof_ctr[15] += cls == CLS_POINT ? 2 : 1;
  used[PG_SELECT] = true;
  // stall rule for instances serving subsegments (decided on the device)
  if (cls == CLS_SUBSEG ||
      (cls < 0 && (std::find(h->instCls.begin(), h->instCls.end(), CLS_SUBSEG) != h->instCls.end() ||
                   std::find(h->instCls.begin(), h->instCls.end(), 3) != h->instCls.end() ||
                   std::find(h->instCls.begin(), h->instCls.end(), 4) != h->instCls.end()))) {
    launch_stall(m, r, s);
    h->prof_ctr[15] += 1;
  }
  // allocation: exclusive scan of (verts, tets, subfaces, subsegs)
  {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveScan(nullptr, tb, r.counts, ptr<int4>(h->bOffs), Int4Sum(),
                                   make_int4(0, 0, 0, 0), n, s);
    if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
    tb = h->bTmp.bytes;
    cub::DeviceScan::ExclusiveScan(h->bTmp.p, tb, r.counts, ptr<int4>(h->bOffs), Int4Sum(),
                                   make_int4(0, 0, 0, 0), n, s);
  }
  cudaMemcpyAsync(&h->pin->lastOff, ptr<int4>(h->bOffs) + n - 1, 16, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&h->pin->lastCnt, r.counts + n - 1, 16, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h->pin->st, h->bStats.p, sizeof(h->pin->st), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (cuda_status(h)) return h->err;
  const int4 lastOff = h->pin->lastOff, lastCnt = h->pin->lastCnt;
  unsigned long long st[ST_COUNT];
  for (int k = 0; k < ST_COUNT; ++k) st[k] = h->pin->st[k];
  int4 tot = make_int4(lastOff.x + lastCnt.x, lastOff.y + lastCnt.y, lastOff.z + lastCnt.z,
                       lastOff.w + lastCnt.w);
  if (!grow_verts(h, m.nV + tot.x) || !grow_tets(h, m.nT + tot.y) ||
      !grow_subfaces(h, m.nS + tot.z) || !grow_subsegs(h, m.nG + tot.w))
    return h->err ? h->err : CDR_ERR_OOM;
  if ((size_t)(h->hcount + 2 * tot.w) * 2 > (size_t)m.hmask + 1) {
    if (!rebuild_hash(h, (m.nG + 2 * tot.w) * 2)) return CDR_ERR_OOM;
  }
  r = make_round(h, cls, n, B);  // rebind after any reallocation
  r.epoch = 0;
  r.n2 = h->lastN2;
  r.s1 = h->lastS1;  // the layout growth wrote its slabs in
  pmark(h, PG_INSERT, 0);
  launch_insert(m, r, ptr<int>(h->bHint), s);
  pmark(h, PG_INSERT, 1);
  h->prof_ctr[15] += 1;
  used[PG_INSERT] = true;
  m.nV += cls == CLS_POINT ? 0 : tot.x;
  m.nT += tot.y;
  m.nS += tot.z;
  m.nG += tot.w;
  h->hcount += 2 * tot.w;
  h->lastN = n;
  h->lastCls = cls;
  if (ro) {
    ro->cls = cls;
    ro->cand = n;
    ro->ins = (long long)st[ST_SURV];
    ro->rej = (long long)st[ST_REJECT];
    ro->unspl = (long long)st[ST_UNSPL];
    ro->blasted = (long long)st[ST_OK] + (long long)st[ST_BLAST];
  }
  // one synchronisation for the round's error flags and counters (and the
  // next round's counts)
  const bool next = cls != CLS_POINT && enqueue_next_classify(h, nullptr);
  const unsigned long long* ctr = h->pin->ctr;
  h->pin->ovf = 0;
  exact_overflow_copy_async(&h->pin->ovf, s);
  cudaMemcpyAsync(h->pin->ctr, h->bStats.p, sizeof(h->pin->ctr), cudaMemcpyDeviceToHost, s);
  if (h->batch && cls < 0)
    cudaMemcpyAsync(h->pinSt, h->bInstSt.p, (size_t)h->ninst * IS_COUNT * 8,
                    cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (h->pin->ovf) {
    exact_overflow_flag(s, true);  // clear it
    return set_err(h, CDR_ERR_INTERNAL);
  }
  {
    int info[4];
    if (checked_error(info, s)) {
      fprintf(stderr, "cdr checked build: bad index %d (bound %d) at kernels.cu:%d, round %u\n",
              info[2], info[3], info[1], h->epoch);
      return set_err(h, CDR_ERR_INTERNAL);
    }
  }
  if (ctr[ST_ITER]) return set_err(h, CDR_ERR_INTERNAL);  // a device invariant check failed
  pcollect(h, used);
  for (int k = 0; k < ST_COUNT && k < 15; ++k) h->prof_ctr[k] += (long long)ctr[k];
  h->deadT += (long long)ctr[ST_DEADT];
  h->preCounted = next;
  return cuda_status(h);
}

// order candidates in bCand[0..n) by priority into bCand2
int order_candidates(cdr_handle* h, int cls, int n) {
  cudaStream_t s = h->stream;
  launch_prio(h->m, cls, ptr<int>(h->bCand), n, ptr<unsigned long long>(h->bKeys), s);
  size_t tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, ptr<unsigned long long>(h->bKeys),
                                  ptr<unsigned long long>(h->bKeys2), ptr<int>(h->bCand),
                                  ptr<int>(h->bCand2), n, 0, 64, s);
  if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
  tb = h->bTmp.bytes;
  cub::DeviceRadixSort::SortPairs(h->bTmp.p, tb, ptr<unsigned long long>(h->bKeys),
                                  ptr<unsigned long long>(h->bKeys2), ptr<int>(h->bCand),
                                  ptr<int>(h->bCand2), n, 0, 64, s);
  launch_tiefix(h->m, cls, ptr<unsigned long long>(h->bKeys2), ptr<int>(h->bCand2), n, s);
  h->prof_ctr[15] += 2;  // priorities + tie fix
  return cuda_status(h);
}

// One round: every instance serves its own first non-empty class (subsegments,
// subfaces, bad tetrahedra; Sec. 2). With one instance this is the plain
// one-class round.
int refine_round(cdr_handle* h, double B, RoundOut* ro) {
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  if (!h->batch && B != h->lastB) {  // (a batch's bounds are per instance, set on entry)
    launch_recompute_bad(m, B, s);
    h->prof_ctr[15] += 1;
    h->lastB = B;
    h->fullClassify = true;
  }
  int st = maybe_compact(h, false);
  if (st) return st;
  if (!ensure_round(h, 1024) || !ensure_pinned(h) || !ensure_instances(h, h->ninst))
    return CDR_ERR_OOM;
  const int ni = h->ninst;
  // counts enqueued behind the last round stand unless the mesh or B changed
  // since (each such change asks for a full classification)
  const bool pre = h->preCounted && !h->fullClassify;
  h->preCounted = false;
  if (!pre) {
    enqueue_classify(h, nullptr);
    cudaStreamSynchronize(s);
  }
  if (cuda_status(h)) return h->err;
  if (h->pin->cerr) return set_err(h, CDR_ERR_INTERNAL);
  {
    bool used[PG_N] = {};
    used[PG_CLASSIFY] = true;
    pcollect(h, used);
  }
  h->instCls.assign(ni, -1);
  long long n = 0;
  for (int k = 0; k < ni; ++k) {
    int c0 = -1;
    for (int c = 0; c < 3 && c0 < 0; ++c)
      if (h->pinCnt[3 * k + c] > 0) c0 = c;
    if (c0 >= 0) {
      // classes taken: the first non-empty one, or up to hi in mixed rounds
      const int hi = h->mixed == 1 ? 2 : (h->mixed == 2 && c0 <= 1 ? 1 : c0);
      int present = 0;
      for (int c = c0; c <= hi; ++c)
        if (h->pinCnt[3 * k + c] > 0) {
          present |= 1 << c;
          n += (long long)h->pinCnt[3 * k + c];
        }
      // 0..2 one class; 3 every class; 4 subsegments and subfaces
      h->instCls[k] = (present & (present - 1)) ? (hi == 2 ? 3 : 4) : c0;
    }
    h->pinCls[k] = h->instCls[k];
  }
  if (ro) *ro = RoundOut();
  if (n == 0) return CDR_OK;
  if (n >= (1LL << 31) - 1) return set_err(h, CDR_ERR_OOM);
  if (!ensure_round(h, (int)n)) return CDR_ERR_OOM;
  if (!h->batch && h->instCls[0] < 3) {  // one instance, one class: its flagged elements
    const int cls = h->instCls[0];
    const uint8_t* flags = cls == 0 ? ptr<uint8_t>(h->bCandG)
                                    : (cls == 1 ? ptr<uint8_t>(h->bCandS) : ptr<uint8_t>(h->bCandT));
    const int nall = cls == 0 ? m.nG : (cls == 1 ? m.nS : m.nT);
    size_t tb = 0;
    int* nsel = ptr<int>(h->bErr) + 4;
    cub::DeviceSelect::Flagged(nullptr, tb, thrust::counting_iterator<int>(0), flags,
                               ptr<int>(h->bCand), nsel, nall, s);
    if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
    tb = h->bTmp.bytes;
    cub::DeviceSelect::Flagged(h->bTmp.p, tb, thrust::counting_iterator<int>(0), flags,
                               ptr<int>(h->bCand), nsel, nall, s);
    if (use_fused(h, (int)n)) {  // the kernel orders them itself
      st = round_core(h, cls, (int)n, B, ro, true);
      if (ro) ro->cls = cls;
      return st;
    }
    st = order_candidates(h, cls, (int)n);
    if (st) return st;
    st = round_core(h, cls, (int)n, B, ro);
    if (ro) ro->cls = cls;
    return st;
  }
  const long nall = (long)m.nG + m.nS + m.nT;
  if (!ensure(h, h->bRflags, (size_t)nall + 64)) return CDR_ERR_OOM;
  cudaMemcpyAsync(h->bInstCls.p, h->pinCls, (size_t)ni * 4, cudaMemcpyHostToDevice, s);
  launch_round_flags(m, ptr<uint8_t>(h->bCandG), ptr<uint8_t>(h->bCandS), ptr<uint8_t>(h->bCandT),
                     ptr<uint8_t>(h->bRflags), s);
  size_t tb = 0;
  int* nsel = ptr<int>(h->bErr) + 4;
  const uint8_t* flags = ptr<uint8_t>(h->bRflags);
  cub::DeviceSelect::Flagged(nullptr, tb, thrust::counting_iterator<int>(0), flags,
                             ptr<int>(h->bCand), nsel, (int)nall, s);
  if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
  tb = h->bTmp.bytes;
  cub::DeviceSelect::Flagged(h->bTmp.p, tb, thrust::counting_iterator<int>(0), flags,
                             ptr<int>(h->bCand), nsel, (int)nall, s);
  h->prof_ctr[15] += 1;
  if (use_fused(h, (int)n)) {  // the kernel orders and decodes them itself
    st = round_core(h, -1, (int)n, B, ro, true);
  } else {
    st = order_candidates(h, -1, (int)n);
    if (st) return st;
    launch_decode_cands(m, ptr<int>(h->bCand2), ptr<uint8_t>(h->bCcls), ptr<int>(h->bCinst),
                        (int)n, s);
    h->prof_ctr[15] += 1;
    st = round_core(h, -1, (int)n, B, ro);
  }
  if (ro) ro->cls = ni == 1 ? std::min(h->instCls[0], 3) : 3;  // 3: several classes or instances
  return st;
}

int count_bad(cdr_handle* h, long long* out) {
  if (!ensure(h, h->bStats, 32 * 8)) return CDR_ERR_OOM;
  unsigned long long* c = ptr<unsigned long long>(h->bStats) + 24;
  cudaMemsetAsync(c, 0, 8, h->stream);
  k_count_bad<<<gridn(h->m.nT), 256, 0, h->stream>>>(h->m, c);
  unsigned long long v = 0;
  cudaMemcpyAsync(&v, c, 8, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  *out = (long long)v;
  return cuda_status(h);
}

int live_count(cdr_handle* h, const uint8_t* flag, int n, int* out) {
  *out = 0;
  if (n == 0) return 0;
  Buf b;
  if (!ensure(h, b, (size_t)n * 4 + 64) || !ensure(h, h->bErr, 64)) return CDR_ERR_OOM;
  launch_live_flags(flag, n, ptr<int>(b), h->stream);
  int* sum = ptr<int>(h->bErr) + 8;
  size_t tb = 0;
  cub::DeviceReduce::Sum(nullptr, tb, ptr<int>(b), sum, n, h->stream);
  if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
  tb = h->bTmp.bytes;
  cub::DeviceReduce::Sum(h->bTmp.p, tb, ptr<int>(b), sum, n, h->stream);
  cudaMemcpyAsync(out, sum, 4, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  dfree(h, b);
  return cuda_status(h);
}

// dense positions of live entries (exclusive scan of live flags)
bool live_positions(cdr_handle* h, const uint8_t* flag, int n, Buf& pos) {
  Buf b;
  if (!ensure(h, b, (size_t)n * 4 + 64) || !ensure(h, pos, (size_t)n * 4 + 64)) return false;
  launch_live_flags(flag, n, ptr<int>(b), h->stream);
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, ptr<int>(b), ptr<int>(pos), n, h->stream);
  if (!tmp_ensure(h, tb)) return false;
  tb = h->bTmp.bytes;
  cub::DeviceScan::ExclusiveSum(h->bTmp.p, tb, ptr<int>(b), ptr<int>(pos), n, h->stream);
  cudaStreamSynchronize(h->stream);
  dfree(h, b);
  return true;
}

}  // namespace

// ===================================================================== API
extern "C" {

const char* cdr_status_string(int s) {
  switch (s) {
    case CDR_OK: return "ok";
    case CDR_ROUND_LIMIT: return "round limit reached with work left";
    case CDR_ERR_INVALID_INPUT: return "invalid input";
    case CDR_ERR_OOM: return "out of device memory";
    case CDR_ERR_CUDA: return "CUDA error";
    case CDR_ERR_ITER_LIMIT: return "a bounded device loop gave up";
    case CDR_ERR_INTERNAL: return "internal error (exact-arithmetic capacity or invariant)";
    case CDR_ERR_TOO_LARGE: return "more items than the fixed scratch of a no-allocation call holds";
  }
  return "unknown status";
}

int cdr_device_arch(void) { return 103; }

void cdr_destroy(cdr_handle* h) {
  if (!h) return;
  if (h->pin) cudaFreeHost(h->pin);
  if (h->pinCnt) cudaFreeHost(h->pinCnt);
  if (h->pinCls) cudaFreeHost(h->pinCls);
  if (h->pinSt) cudaFreeHost(h->pinSt);
  Buf* all[] = {&h->bV, &h->bT, &h->bTS, &h->bTflag, &h->bTmark, &h->bTseed, &h->bTfwd, &h->bSV, &h->bSN,
                &h->bSflag, &h->bSmust, &h->bSmark, &h->bGV, &h->bGflag, &h->bGmust, &h->bFQ,
                &h->bHK, &h->bHV, &h->bCandS, &h->bCandG, &h->bCandT, &h->bCand, &h->bCand2,
                &h->bKeys, &h->bKeys2, &h->bSp, &h->bLoc, &h->bStatus, &h->bSurv, &h->bCounts,
                &h->bOffs, &h->bSlab1, &h->bSlab2of, &h->bList2, &h->bSlab2, &h->bWs2, &h->bCkey,
                &h->bTmp, &h->bStats, &h->bErr, &h->bI32, &h->bPts, &h->bHint, &h->bPstate,
                &h->bVinst, &h->bInstB, &h->bInstG2, &h->bInstCls, &h->bInstCnt, &h->bInstSt,
                &h->bCcls, &h->bCinst, &h->bRflags, &h->bDirtyS, &h->bDirtyG, &h->bFused};
  for (Buf* b : all) dfree(h, *b);
  for (Buf& b : h->ck) dfree(h, b);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  cudaStreamSynchronize(h->stream);
  delete h;
}

}  // extern "C"

namespace {

// facet reference points: the facet's first listed triangle's first vertex
// moved along the dominant axis of that triangle's normal by the smallest power
// of two >= 4x the largest bounding-box extent
void facet_refs(const cdr_mesh_in* in, std::vector<V4>& fq) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < in->n_verts; ++i)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], in->xyz[3 * i + k]);
      hi[k] = std::max(hi[k], in->xyz[3 * i + k]);
    }
  double ex = 0.0;
  for (int k = 0; k < 3; ++k) ex = std::max(ex, hi[k] - lo[k]);
  double s = 1.0;
  while (s < 4.0 * ex) s *= 2.0;
  while (s * 0.5 >= 4.0 * ex && s > 1e-300) s *= 0.5;
  fq.assign(in->n_facets, make_v4(0, 0, 0, 0));
  std::vector<char> done(in->n_facets, 0);
  for (int i = 0; i < in->n_tris; ++i) {
    int f = in->facet_id[i];
    if (done[f]) continue;
    done[f] = 1;
    const double* A = in->xyz + 3 * in->tris[3 * i];
    const double* B = in->xyz + 3 * in->tris[3 * i + 1];
    const double* C = in->xyz + 3 * in->tris[3 * i + 2];
    double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
    double vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
    double n[3] = {uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx};
    int kk = 0;
    for (int k = 1; k < 3; ++k)
      if (std::fabs(n[k]) > std::fabs(n[kk])) kk = k;
    double q[3] = {A[0], A[1], A[2]};
    q[kk] = A[kk] + s;
    fq[f] = make_v4(q[0], q[1], q[2], 0.0);
  }
}

double default_guard2(const double* xyz, int n) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], xyz[3 * i + k]);
      hi[k] = std::max(hi[k], xyz[3 * i + k]);
    }
  double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
  double diag2 = dx * dx + dy * dy + dz * dz;
  return diag2 * 1e-18;
}

// shared by cdr_create and cdr_delaunay_box: allocate, upload vertices and
// tetrahedra, build neighbours from sorted face keys. The sorted keys stay in
// bKeys / bCand2 / bI32 for subface labelling.
int build_mesh(cdr_handle* h, const double* xyz, int nv, const int* tets, int nt, int capV,
               int capT) {
  DevMesh& m = h->m;
  h->capV = h->capT = 0;
  if (!grow_verts(h, capV) || !grow_tets(h, capT)) return h->err ? h->err : CDR_ERR_OOM;
  Buf tmp;
  if (!ensure(h, tmp, (size_t)std::max((size_t)nv * 24, (size_t)nt * 16) + 64)) return CDR_ERR_OOM;
  cudaMemcpyAsync(tmp.p, xyz, (size_t)nv * 24, cudaMemcpyHostToDevice, h->stream);
  k_xyz_to_v4<<<gridn(nv), 256, 0, h->stream>>>(ptr<double>(tmp), nv, m.V);
  m.nV = nv;
  cudaStreamSynchronize(h->stream);
  cudaMemcpyAsync(tmp.p, tets, (size_t)nt * 16, cudaMemcpyHostToDevice, h->stream);
  launch_init_tets(m, ptr<int4>(tmp), nt, h->stream);
  m.nT = nt;
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp);
  int nf = 4 * nt;
  Buf bhi, blo;
  if (!ensure(h, bhi, (size_t)nf * 8 + 64) || !ensure(h, blo, (size_t)nf * 4 + 64) ||
      !ensure(h, h->bKeys, (size_t)nf * 8 + 64) || !ensure(h, h->bCand2, (size_t)nf * 4 + 64) ||
      !ensure(h, h->bI32, (size_t)nf * 4 + 64))
    return CDR_ERR_OOM;
  launch_face_keys(m, ptr<unsigned long long>(bhi), ptr<unsigned>(blo), nullptr, h->stream);
  if (!sort2(h, ptr<unsigned long long>(bhi), ptr<unsigned>(blo), nf,
             ptr<unsigned long long>(h->bKeys), ptr<unsigned>(h->bCand2), ptr<int>(h->bI32)))
    return h->err ? h->err : CDR_ERR_OOM;
  dfree(h, bhi);
  dfree(h, blo);
  if (!ensure(h, h->bErr, 64)) return CDR_ERR_OOM;
  cudaMemsetAsync(h->bErr.p, 0, 64, h->stream);
  launch_pair_faces(m, ptr<unsigned long long>(h->bKeys), ptr<unsigned>(h->bCand2),
                    ptr<int>(h->bI32), nf, ptr<int>(h->bErr), h->stream);
  return cuda_status(h);
}

}  // namespace

extern "C" int cdr_create(const cdr_mesh_in* in, const cdr_options* opt, const cdr_allocator* alloc,
                          void* stream, cdr_handle** out) {
  if (!in || !out) return CDR_ERR_INVALID_INPUT;
  *out = nullptr;
  if (in->n_verts < 4 || in->n_tets < 1 || in->n_segs < 0 || in->n_tris < 0 || in->n_facets < 0 ||
      !in->xyz || !in->tets || (in->n_segs && (!in->segs || !in->seg_id)) ||
      (in->n_tris && (!in->tris || !in->facet_id)) || in->n_verts >= kMaxVerts ||
      in->n_tets >= kMaxTets / 8)
    return CDR_ERR_INVALID_INPUT;
  for (long i = 0; i < 4L * in->n_tets; ++i)
    if (in->tets[i] < 0 || in->tets[i] >= in->n_verts) return CDR_ERR_INVALID_INPUT;
  for (long i = 0; i < 2L * in->n_segs; ++i)
    if (in->segs[i] < 0 || in->segs[i] >= in->n_verts) return CDR_ERR_INVALID_INPUT;
  for (long i = 0; i < 3L * in->n_tris; ++i)
    if (in->tris[i] < 0 || in->tris[i] >= in->n_verts) return CDR_ERR_INVALID_INPUT;
  for (int i = 0; i < in->n_tris; ++i)
    if (in->facet_id[i] < 0 || in->facet_id[i] >= in->n_facets) return CDR_ERR_INVALID_INPUT;
  for (long i = 0; i < 3L * in->n_verts; ++i)
    if (!std::isfinite(in->xyz[i])) return CDR_ERR_INVALID_INPUT;
  if (in->tet_flag)
    for (int i = 0; i < in->n_tets; ++i)
      if (in->tet_flag[i] & ~2) return CDR_ERR_INVALID_INPUT;
  if (in->subface_flag)
    for (int i = 0; i < in->n_tris; ++i)
      if (in->subface_flag[i] & ~3) return CDR_ERR_INVALID_INPUT;
  if (in->subseg_flag)
    for (int i = 0; i < in->n_segs; ++i)
      if (in->subseg_flag[i] & ~3) return CDR_ERR_INVALID_INPUT;

  cdr_handle* h = new (std::nothrow) cdr_handle();
  if (!h) return CDR_ERR_OOM;
  h->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  int rf = (opt && opt->reserve_factor > 0) ? opt->reserve_factor : 4;
  h->mixed = opt ? opt->mixed_rounds : 0;
  h->m.walk_limit = (opt && opt->walk_limit > 0) ? opt->walk_limit : 100000;
  h->m.guard2 = (opt && opt->guard2 > 0) ? opt->guard2 : default_guard2(in->xyz, in->n_verts);
  h->m.nF = in->n_facets;

  int st = build_mesh(h, in->xyz, in->n_verts, in->tets, in->n_tets,
                      std::max(in->n_verts * rf, 1024), std::max(in->n_tets * rf, 4096));
  if (st) {
    cdr_destroy(h);
    return st;
  }
  DevMesh& m = h->m;
  // subsegments + hash
  if (!grow_subsegs(h, std::max(in->n_segs * rf, 256)) ||
      !grow_subfaces(h, std::max(in->n_tris * rf, 256))) {
    cdr_destroy(h);
    return CDR_ERR_OOM;
  }
  {
    Buf tmp;
    if (!ensure(h, tmp, (size_t)in->n_segs * 12 + 64)) {
      cdr_destroy(h);
      return CDR_ERR_OOM;
    }
    if (in->n_segs) {
      cudaMemcpyAsync(tmp.p, in->segs, (size_t)in->n_segs * 8, cudaMemcpyHostToDevice, h->stream);
      cudaMemcpyAsync(ptr<char>(tmp) + (size_t)in->n_segs * 8, in->seg_id, (size_t)in->n_segs * 4,
                      cudaMemcpyHostToDevice, h->stream);
      k_init_subsegs<<<gridn(in->n_segs), 256, 0, h->stream>>>(
          m.GV, m.Gflag, m.Gmust, ptr<int>(tmp),
          reinterpret_cast<int*>(ptr<char>(tmp) + (size_t)in->n_segs * 8), in->n_segs);
    }
    m.nG = in->n_segs;
    cudaStreamSynchronize(h->stream);
    dfree(h, tmp);
    if (!rebuild_hash(h, std::max(in->n_segs * rf, 256))) {
      cdr_destroy(h);
      return CDR_ERR_OOM;
    }
    h->hcount = in->n_segs;
  }
  // facet reference points
  {
    std::vector<V4> fq;
    if (in->facet_ref) {
      fq.resize(in->n_facets);
      for (int f = 0; f < in->n_facets; ++f)
        fq[f] = make_v4(in->facet_ref[3 * f], in->facet_ref[3 * f + 1], in->facet_ref[3 * f + 2], 0);
    } else {
      facet_refs(in, fq);
    }
    if (!ensure(h, h->bFQ, std::max<size_t>(fq.size(), 1) * sizeof(V4))) {
      cdr_destroy(h);
      return CDR_ERR_OOM;
    }
    bind(h);
    if (!fq.empty())
      cudaMemcpyAsync(h->bFQ.p, fq.data(), fq.size() * sizeof(V4), cudaMemcpyHostToDevice,
                      h->stream);
    cudaStreamSynchronize(h->stream);
  }
  // subfaces: label faces, then facet adjacency
  {
    int ns = in->n_tris;
    Buf tris;
    if (!ensure(h, tris, (size_t)ns * 16 + 64)) {
      cdr_destroy(h);
      return CDR_ERR_OOM;
    }
    std::vector<int4> ht(ns);
    for (int i = 0; i < ns; ++i)
      ht[i] = make_int4(in->tris[3 * i], in->tris[3 * i + 1], in->tris[3 * i + 2], in->facet_id[i]);
    if (ns) cudaMemcpyAsync(tris.p, ht.data(), (size_t)ns * 16, cudaMemcpyHostToDevice, h->stream);
    m.nS = ns;
    if (ns)
      launch_label_subfaces(m, ptr<int4>(tris), ns, ptr<unsigned long long>(h->bKeys),
                            ptr<unsigned>(h->bCand2), ptr<int>(h->bI32), 4 * m.nT,
                            ptr<int>(h->bErr), h->stream);
    cudaStreamSynchronize(h->stream);
    dfree(h, tris);
    dfree(h, h->bKeys);
    dfree(h, h->bCand2);
    dfree(h, h->bI32);
    if (ns) {
      int ne = 3 * ns;
      Buf bhi, blo, shi, slo, sperm;
      if (!ensure(h, bhi, (size_t)ne * 8 + 64) || !ensure(h, blo, (size_t)ne * 4 + 64) ||
          !ensure(h, shi, (size_t)ne * 8 + 64) || !ensure(h, slo, (size_t)ne * 4 + 64) ||
          !ensure(h, sperm, (size_t)ne * 4 + 64)) {
        cdr_destroy(h);
        return CDR_ERR_OOM;
      }
      launch_subface_edge_keys(m, ptr<unsigned long long>(bhi), ptr<unsigned>(blo), nullptr,
                               h->stream);
      if (!sort2(h, ptr<unsigned long long>(bhi), ptr<unsigned>(blo), ne,
                 ptr<unsigned long long>(shi), ptr<unsigned>(slo), ptr<int>(sperm))) {
        cdr_destroy(h);
        return CDR_ERR_OOM;
      }
      launch_pair_subface_edges(m, ptr<unsigned long long>(shi), ptr<unsigned>(slo),
                                ptr<int>(sperm), ne, ptr<int>(h->bErr), h->stream);
      cudaStreamSynchronize(h->stream);
      dfree(h, bhi);
      dfree(h, blo);
      dfree(h, shi);
      dfree(h, slo);
      dfree(h, sperm);
    }
  }
  // element flags of a mesh exported between rounds
  if ((in->tet_flag && in->n_tets) || (in->subface_flag && in->n_tris) ||
      (in->subseg_flag && in->n_segs)) {
    Buf fl;
    const size_t nt = in->n_tets, ns = in->n_tris, ng = in->n_segs;
    if (!ensure(h, fl, nt + ns + ng + 64)) {
      cdr_destroy(h);
      return CDR_ERR_OOM;
    }
    uint8_t* d = ptr<uint8_t>(fl);
    if (in->tet_flag && nt) cudaMemcpyAsync(d, in->tet_flag, nt, cudaMemcpyHostToDevice, h->stream);
    if (in->subface_flag && ns)
      cudaMemcpyAsync(d + nt, in->subface_flag, ns, cudaMemcpyHostToDevice, h->stream);
    if (in->subseg_flag && ng)
      cudaMemcpyAsync(d + nt + ns, in->subseg_flag, ng, cudaMemcpyHostToDevice, h->stream);
    k_apply_flags<<<gridn((long)nt + ns + ng), 256, 0, h->stream>>>(
        m, in->tet_flag ? d : nullptr, in->subface_flag ? d + nt : nullptr,
        in->subseg_flag ? d + nt + ns : nullptr);
    cudaStreamSynchronize(h->stream);
    dfree(h, fl);
  }
  launch_mark_edges(m, h->stream);
  launch_check_create(m, ptr<int>(h->bErr), h->stream);
  int err = 0;
  cudaMemcpyAsync(&err, h->bErr.p, 4, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  if (cuda_status(h)) {
    int e = h->err;
    cdr_destroy(h);
    return e;
  }
  if (err) {
    cdr_destroy(h);
    return CDR_ERR_INVALID_INPUT;
  }
  *out = h;
  return CDR_OK;
}

// ===================================================================== API
extern "C" {

int cdr_round(cdr_handle* h, double B, int32_t* cls, cdr_stats* stats) {
  if (!h || !(B > 0)) return CDR_ERR_INVALID_INPUT;
  if (h->batch) return CDR_ERR_INVALID_INPUT;
  if (h->err) return h->err;
  if (h->dt_mode) return CDR_ERR_INVALID_INPUT;
  RoundOut ro;
  int st = refine_round(h, B, &ro);
  if (cls) *cls = st ? -1 : ro.cls;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->rounds = ro.cls >= 0 ? 1 : 0;
    if (ro.cls >= 0 && ro.cls < 3) stats->rounds_by_class[ro.cls] = 1;
    stats->candidates = ro.cand;
    stats->steiner_inserted = ro.ins;
    stats->rejected = ro.rej;
    stats->blasted = ro.blasted;
    stats->unsplittable = ro.unspl;
    stats->n_verts = h->m.nV;
  }
  return st;
}

int cdr_refine(cdr_handle* h, double B, int32_t max_rounds, cdr_stats* stats) {
  if (!h || !(B > 0) || max_rounds < 0) return CDR_ERR_INVALID_INPUT;
  if (h->batch) return CDR_ERR_INVALID_INPUT;
  if (h->err) return h->err;
  if (h->dt_mode) return CDR_ERR_INVALID_INPUT;
  cdr_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  int st = CDR_OK;
  bool done = false;
  for (int r = 0; r < max_rounds; ++r) {
    RoundOut ro;
    st = refine_round(h, B, &ro);
    if (st) break;
    if (ro.cls < 0) {
      done = true;
      break;
    }
    acc.rounds++;
    if (ro.cls < 3) acc.rounds_by_class[ro.cls]++;
    acc.candidates += ro.cand;
    acc.steiner_inserted += ro.ins;
    acc.rejected += ro.rej;
    acc.blasted += ro.blasted;
    acc.unsplittable += ro.unspl;
  }
  if (!st && !done) st = CDR_ROUND_LIMIT;
  if (stats) {
    acc.n_verts = h->m.nV;
    long long bad = 0;
    if (count_bad(h, &bad) == 0) acc.n_bad_left = bad;
    int nt = 0, ns = 0, ng = 0;
    live_count(h, h->m.Tflag, h->m.nT, &nt);
    live_count(h, h->m.Sflag, h->m.nS, &ns);
    live_count(h, h->m.Gflag, h->m.nG, &ng);
    acc.n_tets = nt;
    acc.n_subfaces = ns;
    acc.n_subsegs = ng;
    *stats = acc;
  }
  return st;
}

int cdr_export_sizes(cdr_handle* h, cdr_sizes* out) {
  if (!h || !out) return CDR_ERR_INVALID_INPUT;
  int nt = 0, ns = 0, ng = 0;
  int st = live_count(h, h->m.Tflag, h->m.nT, &nt);
  if (!st) st = live_count(h, h->m.Sflag, h->m.nS, &ns);
  if (!st) st = live_count(h, h->m.Gflag, h->m.nG, &ng);
  out->n_verts = h->m.nV;
  out->n_tets = nt;
  out->n_subfaces = ns;
  out->n_subsegs = ng;
  out->n_facets = h->m.nF;
  return st;
}

int cdr_export(cdr_handle* h, const cdr_mesh_out* out) {
  if (!h || !out) return CDR_ERR_INVALID_INPUT;
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  if (out->xyz && m.nV > 0) {
    std::vector<V4> v(m.nV);
    cudaMemcpyAsync(v.data(), m.V, (size_t)m.nV * sizeof(V4), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int i = 0; i < m.nV; ++i) {
      out->xyz[3 * i] = v[i].x;
      out->xyz[3 * i + 1] = v[i].y;
      out->xyz[3 * i + 2] = v[i].z;
    }
  }
  struct Part {
    const uint8_t* flag;
    int n;
    int kind;
  } parts[3] = {{m.Tflag, m.nT, 0}, {m.Sflag, m.nS, 1}, {m.Gflag, m.nG, 2}};
  for (auto& p : parts) {
    if (p.n == 0) continue;
    Buf pos, dense, dflag;
    if (!live_positions(h, p.flag, p.n, pos) || !ensure(h, dense, (size_t)p.n * 16 + 64) ||
        !ensure(h, dflag, (size_t)p.n + 64))
      return CDR_ERR_OOM;
    if (p.kind == 0) launch_gather_tets(m, ptr<int>(pos), ptr<int4>(dense), ptr<uint8_t>(dflag), s);
    if (p.kind == 1)
      launch_gather_subfaces(m, ptr<int>(pos), ptr<int4>(dense), ptr<uint8_t>(dflag), s);
    if (p.kind == 2)
      launch_gather_subsegs(m, ptr<int>(pos), ptr<int4>(dense), ptr<uint8_t>(dflag), s);
    int live = 0;
    live_count(h, p.flag, p.n, &live);
    std::vector<int4> d(live);
    std::vector<uint8_t> f(live);
    if (live) {
      cudaMemcpyAsync(d.data(), dense.p, (size_t)live * 16, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(f.data(), dflag.p, (size_t)live, cudaMemcpyDeviceToHost, s);
    }
    cudaStreamSynchronize(s);
    dfree(h, pos);
    dfree(h, dense);
    dfree(h, dflag);
    for (int i = 0; i < live; ++i) {
      if (p.kind == 0 && out->tets) {
        out->tets[4 * i] = d[i].x;
        out->tets[4 * i + 1] = d[i].y;
        out->tets[4 * i + 2] = d[i].z;
        out->tets[4 * i + 3] = d[i].w;
      }
      if (p.kind == 0 && out->tet_flag) out->tet_flag[i] = f[i];
      if (p.kind == 1 && out->subfaces) {
        out->subfaces[4 * i] = d[i].x;
        out->subfaces[4 * i + 1] = d[i].y;
        out->subfaces[4 * i + 2] = d[i].z;
        out->subfaces[4 * i + 3] = d[i].w;
      }
      if (p.kind == 1 && out->subface_flag) out->subface_flag[i] = f[i];
      if (p.kind == 2 && out->subsegs) {
        out->subsegs[3 * i] = d[i].x;
        out->subsegs[3 * i + 1] = d[i].y;
        out->subsegs[3 * i + 2] = d[i].z;
      }
      if (p.kind == 2 && out->subseg_flag) out->subseg_flag[i] = f[i];
    }
  }
  if (out->facet_ref && m.nF > 0) {
    std::vector<V4> q(m.nF);
    cudaMemcpyAsync(q.data(), m.FQ, (size_t)m.nF * sizeof(V4), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int f = 0; f < m.nF; ++f) {
      out->facet_ref[3 * f] = q[f].x;
      out->facet_ref[3 * f + 1] = q[f].y;
      out->facet_ref[3 * f + 2] = q[f].z;
    }
  }
  return cuda_status(h);
}

int cdr_round_report(cdr_handle* h, int32_t* n_cand, int64_t* n_cav_total, int32_t* keys,
                     double* pts, int32_t* outcome, int32_t* reason, int32_t* survived,
                     int32_t* n_cav, int32_t* n_bnd, int32_t* n_fcav, int32_t* cav) {
  if (!h || !n_cand || !n_cav_total) return CDR_ERR_INVALID_INPUT;
  cudaStream_t s = h->stream;
  int n = h->lastN;
  *n_cand = n;
  *n_cav_total = 0;
  if (n == 0) return CDR_OK;
  DevRound r = make_round(h, h->lastCls, n, 0.0);
  r.n2 = h->lastN2;
  r.s1 = h->lastS1;
  Buf b;
  if (!ensure(h, b, (size_t)n * 12 + 64)) return CDR_ERR_OOM;
  int* dn = ptr<int>(b);
  k_report_sizes<<<gridn(n), 256, 0, s>>>(r, dn, dn + n, dn + 2 * n);
  std::vector<int> nc(3 * (size_t)n);
  cudaMemcpyAsync(nc.data(), dn, (size_t)n * 12, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  long long tot = 0;
  std::vector<int> offs(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    offs[i] = (int)tot;
    tot += nc[i];
  }
  offs[n] = (int)tot;
  *n_cav_total = tot;
  std::vector<int4> k(n);
  std::vector<V4> p(n);
  std::vector<int> st(n), sv(n);
  cudaMemcpyAsync(k.data(), h->bCkey.p, (size_t)n * 16, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(p.data(), h->bSp.p, (size_t)n * sizeof(V4), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(st.data(), h->bStatus.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(sv.data(), h->bSurv.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < n; ++i) {
    if (keys) {
      keys[4 * i] = k[i].x;
      keys[4 * i + 1] = k[i].y;
      keys[4 * i + 2] = k[i].z;
      keys[4 * i + 3] = k[i].w;
    }
    if (pts) {
      pts[3 * i] = p[i].x;
      pts[3 * i + 1] = p[i].y;
      pts[3 * i + 2] = p[i].z;
    }
    if (outcome) outcome[i] = st[i] & 0xff;
    if (reason) reason[i] = (st[i] >> 8) & 0xff;
    if (survived) survived[i] = sv[i];
    if (n_cav) n_cav[i] = nc[i];
    if (n_bnd) n_bnd[i] = nc[n + i];
    if (n_fcav) n_fcav[i] = nc[2 * n + i];
  }
  if (cav && tot > 0) {
    Buf doffs, dout;
    if (!ensure(h, doffs, (size_t)(n + 1) * 4) || !ensure(h, dout, (size_t)tot * 16))
      return CDR_ERR_OOM;
    cudaMemcpyAsync(doffs.p, offs.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s);
    launch_report_cav(h->m, r, ptr<int>(doffs), ptr<int4>(dout), s);
    cudaMemcpyAsync(cav, dout.p, (size_t)tot * 16, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    dfree(h, doffs);
    dfree(h, dout);
  }
  dfree(h, b);
  return cuda_status(h);
}

int cdr_checkpoint(cdr_handle* h) {
  if (!h) return CDR_ERR_INVALID_INPUT;
  if (h->batch) return CDR_ERR_INVALID_INPUT;
  DevMesh& m = h->m;
  struct {
    Buf* b;
    size_t bytes;
  } parts[] = {{&h->bV, (size_t)m.nV * sizeof(V4)},
               {&h->bT, (size_t)m.nT * sizeof(TetRec)},
               {&h->bTS, (size_t)m.nT * 16},
               {&h->bTflag, (size_t)m.nT},
               {&h->bTfwd, (size_t)m.nT * 4},
               {&h->bSV, (size_t)m.nS * 16},
               {&h->bSN, (size_t)m.nS * 16},
               {&h->bSflag, (size_t)m.nS},
               {&h->bSmust, (size_t)m.nS},
               {&h->bGV, (size_t)m.nG * 16},
               {&h->bGflag, (size_t)m.nG},
               {&h->bGmust, (size_t)m.nG},
               {&h->bHK, h->bHK.bytes},
               {&h->bHV, h->bHV.bytes}};
  for (Buf& b : h->ck) dfree(h, b);
  h->ck.clear();
  for (auto& p : parts) {
    Buf c;
    if (!ensure(h, c, p.bytes + 16)) return CDR_ERR_OOM;
    if (p.bytes) cudaMemcpyAsync(c.p, p.b->p, p.bytes, cudaMemcpyDeviceToDevice, h->stream);
    c.bytes = p.bytes;  // payload size
    h->ck.push_back(c);
  }
  h->ckm = m;
  h->ck_hcount = h->hcount;
  h->ck_deadT = h->deadT;
  h->has_ck = true;
  cudaStreamSynchronize(h->stream);
  return cuda_status(h);
}

int cdr_restore(cdr_handle* h) {
  if (!h || !h->has_ck) return CDR_ERR_INVALID_INPUT;
  if (h->batch) return CDR_ERR_INVALID_INPUT;
  DevMesh c = h->ckm;
  if (!grow_verts(h, c.nV) || !grow_tets(h, c.nT) || !grow_subfaces(h, c.nS) ||
      !grow_subsegs(h, c.nG))
    return CDR_ERR_OOM;
  if (!ensure(h, h->bHK, h->ck[12].bytes) || !ensure(h, h->bHV, h->ck[13].bytes)) return CDR_ERR_OOM;
  Buf* dst[] = {&h->bV,  &h->bT,     &h->bTS,    &h->bTflag, &h->bTfwd,  &h->bSV,  &h->bSN,
                &h->bSflag, &h->bSmust, &h->bGV, &h->bGflag, &h->bGmust, &h->bHK, &h->bHV};
  for (int i = 0; i < 14; ++i)
    if (h->ck[i].bytes)
      cudaMemcpyAsync(dst[i]->p, h->ck[i].p, h->ck[i].bytes, cudaMemcpyDeviceToDevice, h->stream);
  DevMesh& m = h->m;
  m.nV = c.nV;
  m.nT = c.nT;
  m.nS = c.nS;
  m.nG = c.nG;
  m.hmask = c.hmask;
  h->hcount = h->ck_hcount;
  h->deadT = h->ck_deadT;
  h->deadKnown = true;
  h->fullClassify = true;
  h->lastB = -1.0;
  h->lastN = 0;
  h->err = 0;
  bind(h);
  cudaMemsetAsync(h->bTmark.p, 0xff, (size_t)h->capT * 8, h->stream);
  cudaMemsetAsync(h->bTseed.p, 0xff, (size_t)h->capT * 8, h->stream);
  cudaMemsetAsync(h->bSmark.p, 0xff, (size_t)h->capS * 8, h->stream);
  cudaStreamSynchronize(h->stream);
  return cuda_status(h);
}

int cdr_delaunay_box(const double* xyz, int32_t n, const cdr_options* opt,
                     const cdr_allocator* alloc, void* stream, cdr_handle** out,
                     int32_t* n_skipped, int32_t* n_rounds) {
  if (!xyz || !out || n < 8 || n >= kMaxVerts) return CDR_ERR_INVALID_INPUT;
  *out = nullptr;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      double v = xyz[3 * i + k];
      if (!std::isfinite(v)) return CDR_ERR_INVALID_INPUT;
      lo[k] = std::min(lo[k], v);
      hi[k] = std::max(hi[k], v);
    }
  int corner[8];
  for (int c = 0; c < 8; ++c) corner[c] = -1;
  std::vector<int> state(n, 0);
  for (int i = 0; i < n; ++i) {
    int code = 0;
    bool ok = true, onb = false;
    for (int k = 0; k < 3; ++k) {
      double v = xyz[3 * i + k];
      if (v == hi[k]) code |= 1 << k;
      else if (v != lo[k]) ok = false;
      if (v == hi[k] || v == lo[k]) onb = true;
    }
    if (ok && corner[code] < 0) {
      corner[code] = i;
      state[i] = 1;
    } else if (onb) {
      return CDR_ERR_INVALID_INPUT;  // only the corners may lie on the box
    }
  }
  for (int c = 0; c < 8; ++c)
    if (corner[c] < 0) return CDR_ERR_INVALID_INPUT;
  // the cube as six tetrahedra around its main diagonal; an odd axis order
  // gives a negatively oriented tuple, fixed by swapping two vertices
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const bool odd[6] = {false, true, true, false, false, true};
  std::vector<int> tets;
  for (int q = 0; q < 6; ++q) {
    int b1 = 1 << perm[q][0], b2 = b1 | (1 << perm[q][1]);
    int t[4] = {corner[0], corner[b1], corner[b2], corner[7]};
    if (odd[q]) std::swap(t[1], t[2]);
    tets.insert(tets.end(), t, t + 4);
  }
  cdr_handle* h = new (std::nothrow) cdr_handle();
  if (!h) return CDR_ERR_OOM;
  h->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  h->dt_mode = true;
  h->m.walk_limit = (opt && opt->walk_limit > 0) ? opt->walk_limit : 100000;
  h->m.guard2 = 0.0;  // exact duplicates only
  int st = build_mesh(h, xyz, n, tets.data(), 6, n, std::max(8 * n, 4096));
  dfree(h, h->bKeys);
  dfree(h, h->bCand2);
  dfree(h, h->bI32);
  if (!st && (!grow_subsegs(h, 16) || !grow_subfaces(h, 16) || !rebuild_hash(h, 16) ||
              !ensure(h, h->bFQ, 64)))
    st = CDR_ERR_OOM;
  if (st) {
    cdr_destroy(h);
    return st;
  }
  bind(h);
  h->npts = n;
  if (!ensure(h, h->bPts, (size_t)n * 24) || !ensure(h, h->bHint, (size_t)n * 4) ||
      !ensure(h, h->bPstate, (size_t)n * 4)) {
    cdr_destroy(h);
    return CDR_ERR_OOM;
  }
  cudaStream_t s = h->stream;
  cudaMemcpyAsync(h->bPts.p, xyz, (size_t)n * 24, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(h->bHint.p, 0, (size_t)n * 4, s);
  cudaMemcpyAsync(h->bPstate.p, state.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
  int rounds = 0;
  for (;;) {
    if (!ensure_round(h, n)) {
      st = CDR_ERR_OOM;
      break;
    }
    int* flag = ptr<int>(h->bI32);
    k_point_flags<<<gridn(n), 256, 0, s>>>(ptr<int>(h->bPstate), n, flag);
    size_t tb = 0;
    int* nsel = ptr<int>(h->bErr) + 4;
    cub::DeviceSelect::Flagged(nullptr, tb, thrust::counting_iterator<int>(0), flag,
                               ptr<int>(h->bCand), nsel, n, s);
    if (!tmp_ensure(h, tb)) {
      st = CDR_ERR_OOM;
      break;
    }
    tb = h->bTmp.bytes;
    cub::DeviceSelect::Flagged(h->bTmp.p, tb, thrust::counting_iterator<int>(0), flag,
                               ptr<int>(h->bCand), nsel, n, s);
    int nc = 0;
    cudaMemcpyAsync(&nc, nsel, 4, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (nc == 0) break;
    st = order_candidates(h, CLS_POINT, nc);
    if (!st) st = round_core(h, CLS_POINT, nc, 1.0, nullptr);
    if (st) break;
    ++rounds;
    if (h->m.nT > (1 << 20) && (rounds % 8) == 0) {
      st = maybe_compact(h, false);
      if (st) break;
    }
  }
  if (!st) {
    cudaMemcpyAsync(state.data(), h->bPstate.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int sk = 0;
    for (int i = 0; i < n; ++i) sk += state[i] == 2;
    if (n_skipped) *n_skipped = sk;
    if (n_rounds) *n_rounds = rounds;
    st = cuda_status(h);
  }
  if (st) {
    cdr_destroy(h);
    return st;
  }
  *out = h;
  return CDR_OK;
}

// ===================================================================== batches
// Diagnostic builds only (CDR_PHASES): cycles and region counts per phase of
// region growth since the last call. Not part of the declared interface.
int cdr_debug_phases(cdr_handle* h, unsigned long long* out32) {
  if (!h || !out32) return CDR_ERR_INVALID_INPUT;
  return phase_counters(out32, h->stream) ? CDR_OK : CDR_ERR_INVALID_INPUT;
}

int cdr_batch_create(const cdr_options* opt, const cdr_allocator* alloc, void* stream,
                     cdr_handle** out) {
  if (!out) return CDR_ERR_INVALID_INPUT;
  *out = nullptr;
  cdr_handle* h = new (std::nothrow) cdr_handle();
  if (!h) return CDR_ERR_OOM;
  h->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  h->batch = true;
  h->mixed = opt ? opt->mixed_rounds : 0;
  h->ninst = 0;
  if (opt) h->opts = *opt;
  h->opts.reserve_factor = 1;  // an instance is built at its own size, then appended
  h->m.walk_limit = (opt && opt->walk_limit > 0) ? opt->walk_limit : 100000;
  h->m.nV = h->m.nT = h->m.nS = h->m.nG = h->m.nF = 0;
  if (!grow_verts(h, 4096) || !grow_tets(h, 16384) || !grow_subfaces(h, 4096) ||
      !grow_subsegs(h, 1024) || !rebuild_hash(h, 1024) || !ensure(h, h->bFQ, 64 * sizeof(V4)) ||
      !ensure_instances(h, 16) || !ensure_pinned(h)) {
    int e = h->err ? h->err : CDR_ERR_OOM;
    cdr_destroy(h);
    return e;
  }
  bind(h);
  int st = cuda_status(h);
  if (st) {
    cdr_destroy(h);
    return st;
  }
  *out = h;
  return CDR_OK;
}

int cdr_batch_add(cdr_handle* h, const cdr_mesh_in* in, double B, int32_t* slot) {
  if (!h || !h->batch || !in || !(B > 0) || !slot) return CDR_ERR_INVALID_INPUT;
  if (h->err) return h->err;
  *slot = -1;
  cdr_allocator al = h->alloc;
  cdr_handle* t = nullptr;
  int st = cdr_create(in, &h->opts, h->has_alloc ? &al : nullptr, h->stream, &t);
  if (st) return st;
  DevMesh& d = h->m;
  const DevMesh& sm = t->m;
  if ((long)d.nV + sm.nV >= kMaxVerts || (long)d.nT + sm.nT >= kMaxTets / 8) {
    cdr_destroy(t);
    return CDR_ERR_OOM;
  }
  int k;
  if (!h->freeSlots.empty()) {
    k = h->freeSlots.back();
    h->freeSlots.pop_back();
  } else {
    k = h->ninst++;
    h->insts.emplace_back();
  }
  if (!ensure_instances(h, h->ninst) || !grow_verts(h, d.nV + sm.nV) ||
      !grow_tets(h, d.nT + sm.nT) || !grow_subfaces(h, d.nS + sm.nS) ||
      !grow_subsegs(h, d.nG + sm.nG) ||
      !ensure(h, h->bFQ, (size_t)(d.nF + sm.nF + 1) * sizeof(V4), (size_t)d.nF * sizeof(V4))) {
    cdr_destroy(t);
    return h->err ? h->err : CDR_ERR_OOM;
  }
  bind(h);
  int nseg = 0;
  for (int i = 0; i < in->n_segs; ++i) nseg = std::max(nseg, in->seg_id[i] + 1);
  launch_append(d, sm, d.nV, d.nT, d.nS, d.nG, d.nF, h->segIds, k, h->stream);
  const double b = B, g2 = sm.guard2;
  cudaMemcpyAsync(ptr<double>(h->bInstB) + k, &b, 8, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(ptr<double>(h->bInstG2) + k, &g2, 8, cudaMemcpyHostToDevice, h->stream);
  const int g0 = d.nG;
  cdr_handle::Inst& I = h->insts[k];
  I = cdr_handle::Inst();
  I.state = 1;
  I.of = d.nF;
  I.nf = sm.nF;
  I.oseg = h->segIds;
  I.nseg = nseg;
  I.B = B;
  d.nV += sm.nV;
  d.nT += sm.nT;
  d.nS += sm.nS;
  d.nG += sm.nG;
  d.nF += sm.nF;
  h->segIds += nseg;
  if ((size_t)(h->hcount + sm.nG) * 2 > (size_t)d.hmask + 1) {
    if (!rebuild_hash(h, d.nG * 2)) {
      cdr_destroy(t);
      return CDR_ERR_OOM;
    }
  } else {
    launch_hash_insert_subsegs(d, g0, d.nG, h->stream);
    h->hcount += sm.nG;
  }
  launch_recompute_bad(d, 0.0, h->stream);  // per-instance bounds
  h->fullClassify = true;
  cudaStreamSynchronize(h->stream);
  cdr_destroy(t);
  st = cuda_status(h);
  if (!st) *slot = k;
  return st;
}

int cdr_batch_round(cdr_handle* h, int32_t* n_active) {
  if (!h || !h->batch) return CDR_ERR_INVALID_INPUT;
  if (h->err) return h->err;
  if (n_active) *n_active = 0;
  if (h->ninst == 0) return CDR_OK;
  RoundOut ro;
  int st = refine_round(h, 1.0, &ro);
  if (st) return st;
  int active = 0;
  const bool ran = ro.cand > 0;
  for (int k = 0; k < h->ninst; ++k) {
    cdr_handle::Inst& I = h->insts[k];
    if (I.state != 1) continue;
    int c = k < (int)h->instCls.size() ? h->instCls[k] : -1;
    if (c < 0) {
      I.state = 2;
      continue;
    }
    ++active;
    I.st.rounds++;
    if (c < 3) {
      I.st.rounds_by_class[c]++;
      I.st.candidates += (long long)h->pinCnt[3 * k + c];
    } else {
      I.st.candidates += (long long)(h->pinCnt[3 * k] + h->pinCnt[3 * k + 1] +
                                     (c == 3 ? h->pinCnt[3 * k + 2] : 0));
    }
    if (ran) {
      const unsigned long long* q = h->pinSt + (size_t)k * IS_COUNT;
      I.st.steiner_inserted += (long long)q[IS_SURV];
      I.st.rejected += (long long)q[IS_REJECT] - (long long)q[IS_STALLED];
      I.st.unsplittable += (long long)q[IS_UNSPL] + (long long)q[IS_STALLED];
    }
  }
  if (n_active) *n_active = active;
  return CDR_OK;
}

int cdr_batch_refine(cdr_handle* h, int32_t max_rounds, int32_t* rounds) {
  if (!h || !h->batch || max_rounds < 0) return CDR_ERR_INVALID_INPUT;
  int r = 0, st = CDR_OK, active = 1;
  while (r < max_rounds) {
    st = cdr_batch_round(h, &active);
    if (st || active == 0) break;
    ++r;
  }
  if (rounds) *rounds = r;
  if (!st && active > 0) st = CDR_ROUND_LIMIT;
  return st;
}

namespace {
// live entries of instance k of one kind (0 vertices, 1 tets, 2 subfaces,
// 3 subsegments, 4 bad tets left) and, if pos is given, their positions
int inst_count(cdr_handle* h, int k, int kind, Buf* flag, Buf* pos, int* out) {
  DevMesh& m = h->m;
  int n = kind == 0 ? m.nV : (kind == 1 || kind == 4 ? m.nT : (kind == 2 ? m.nS : m.nG));
  *out = 0;
  if (n == 0) return CDR_OK;
  Buf f;
  if (!ensure(h, f, (size_t)n * 4 + 64) || !ensure(h, h->bErr, 64)) return CDR_ERR_OOM;
  launch_inst_flags(m, k, kind == 4 ? 1 : kind, n, ptr<int>(f), h->stream);
  if (kind == 4) launch_inst_bad(m, ptr<int>(f), n, h->stream);
  int* sum = ptr<int>(h->bErr) + 8;
  size_t tb = 0;
  cub::DeviceReduce::Sum(nullptr, tb, ptr<int>(f), sum, n, h->stream);
  if (!tmp_ensure(h, tb)) return CDR_ERR_OOM;
  tb = h->bTmp.bytes;
  cub::DeviceReduce::Sum(h->bTmp.p, tb, ptr<int>(f), sum, n, h->stream);
  if (pos) {
    if (!ensure(h, *pos, (size_t)n * 4 + 64)) return CDR_ERR_OOM;
    size_t tb2 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb2, ptr<int>(f), ptr<int>(*pos), n, h->stream);
    if (!tmp_ensure(h, tb2)) return CDR_ERR_OOM;
    tb2 = h->bTmp.bytes;
    cub::DeviceScan::ExclusiveSum(h->bTmp.p, tb2, ptr<int>(f), ptr<int>(*pos), n, h->stream);
  }
  cudaMemcpyAsync(&h->pin->n2, sum, 4, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  *out = h->pin->n2;
  if (flag) {
    dfree(h, *flag);
    *flag = f;
  } else {
    dfree(h, f);
  }
  return cuda_status(h);
}
}  // namespace

int cdr_batch_stats(cdr_handle* h, int32_t slot, cdr_stats* stats, int32_t* state) {
  if (!h || !h->batch || slot < 0 || slot >= h->ninst) return CDR_ERR_INVALID_INPUT;
  const cdr_handle::Inst& I = h->insts[slot];
  if (state) *state = I.state;
  if (stats) {
    *stats = I.st;
    if (I.state != 0 && ensure_pinned(h)) {
      int nv = 0, nt = 0, ns = 0, ng = 0, nb = 0;
      int st = inst_count(h, slot, 0, nullptr, nullptr, &nv);
      if (!st) st = inst_count(h, slot, 1, nullptr, nullptr, &nt);
      if (!st) st = inst_count(h, slot, 2, nullptr, nullptr, &ns);
      if (!st) st = inst_count(h, slot, 3, nullptr, nullptr, &ng);
      if (!st) st = inst_count(h, slot, 4, nullptr, nullptr, &nb);
      if (st) return st;
      stats->n_verts = nv;
      stats->n_tets = nt;
      stats->n_subfaces = ns;
      stats->n_subsegs = ng;
      stats->n_bad_left = nb;
    }
  }
  return CDR_OK;
}

int cdr_batch_export_sizes(cdr_handle* h, int32_t slot, cdr_sizes* out) {
  if (!h || !h->batch || !out || slot < 0 || slot >= h->ninst || h->insts[slot].state == 0)
    return CDR_ERR_INVALID_INPUT;
  if (!ensure_pinned(h)) return CDR_ERR_OOM;
  int nv = 0, nt = 0, ns = 0, ng = 0;
  int st = inst_count(h, slot, 0, nullptr, nullptr, &nv);
  if (!st) st = inst_count(h, slot, 1, nullptr, nullptr, &nt);
  if (!st) st = inst_count(h, slot, 2, nullptr, nullptr, &ns);
  if (!st) st = inst_count(h, slot, 3, nullptr, nullptr, &ng);
  if (st) return st;
  out->n_verts = nv;
  out->n_tets = nt;
  out->n_subfaces = ns;
  out->n_subsegs = ng;
  out->n_facets = h->insts[slot].nf;
  return CDR_OK;
}

int cdr_batch_export(cdr_handle* h, int32_t slot, const cdr_mesh_out* out) {
  if (!h || !h->batch || !out || slot < 0 || slot >= h->ninst || h->insts[slot].state == 0)
    return CDR_ERR_INVALID_INPUT;
  if (!ensure_pinned(h)) return CDR_ERR_OOM;
  DevMesh& m = h->m;
  cudaStream_t s = h->stream;
  const cdr_handle::Inst& I = h->insts[slot];
  Buf vflag, vpos;
  int nv = 0;
  int st = inst_count(h, slot, 0, &vflag, &vpos, &nv);
  if (st) return st;
  Buf dense;
  if (!ensure(h, dense, (size_t)std::max(nv, 1) * sizeof(V4))) return CDR_ERR_OOM;
  launch_inst_gather(m, 0, m.nV, ptr<int>(vflag), ptr<int>(vpos), ptr<int>(vpos), 0, 0, nullptr,
                     nullptr, ptr<V4>(dense), s);
  if (out->xyz && nv > 0) {
    std::vector<V4> v(nv);
    cudaMemcpyAsync(v.data(), dense.p, (size_t)nv * sizeof(V4), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int i = 0; i < nv; ++i) {
      out->xyz[3 * i] = v[i].x;
      out->xyz[3 * i + 1] = v[i].y;
      out->xyz[3 * i + 2] = v[i].z;
    }
  }
  dfree(h, dense);
  dfree(h, vflag);
  for (int kind = 1; kind <= 3; ++kind) {
    Buf f, pos;
    int live = 0;
    st = inst_count(h, slot, kind, &f, &pos, &live);
    if (st) return st;
    int n = kind == 1 ? m.nT : (kind == 2 ? m.nS : m.nG);
    Buf d4, d1;
    if (!ensure(h, d4, (size_t)std::max(live, 1) * 16) || !ensure(h, d1, (size_t)std::max(live, 1)))
      return CDR_ERR_OOM;
    launch_inst_gather(m, kind, n, ptr<int>(f), ptr<int>(pos), ptr<int>(vpos), I.of, I.oseg,
                       ptr<int4>(d4), ptr<uint8_t>(d1), nullptr, s);
    std::vector<int4> d(live);
    std::vector<uint8_t> fl(live);
    if (live) {
      cudaMemcpyAsync(d.data(), d4.p, (size_t)live * 16, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(fl.data(), d1.p, (size_t)live, cudaMemcpyDeviceToHost, s);
    }
    cudaStreamSynchronize(s);
    dfree(h, f);
    dfree(h, pos);
    dfree(h, d4);
    dfree(h, d1);
    for (int i = 0; i < live; ++i) {
      if (kind == 1) {
        if (out->tets) {
          out->tets[4 * i] = d[i].x;
          out->tets[4 * i + 1] = d[i].y;
          out->tets[4 * i + 2] = d[i].z;
          out->tets[4 * i + 3] = d[i].w;
        }
        if (out->tet_flag) out->tet_flag[i] = fl[i];
      } else if (kind == 2) {
        if (out->subfaces) {
          out->subfaces[4 * i] = d[i].x;
          out->subfaces[4 * i + 1] = d[i].y;
          out->subfaces[4 * i + 2] = d[i].z;
          out->subfaces[4 * i + 3] = d[i].w;
        }
        if (out->subface_flag) out->subface_flag[i] = fl[i];
      } else {
        if (out->subsegs) {
          out->subsegs[3 * i] = d[i].x;
          out->subsegs[3 * i + 1] = d[i].y;
          out->subsegs[3 * i + 2] = d[i].z;
        }
        if (out->subseg_flag) out->subseg_flag[i] = fl[i];
      }
    }
  }
  dfree(h, vpos);
  if (out->facet_ref && I.nf > 0) {
    std::vector<V4> q(I.nf);
    cudaMemcpyAsync(q.data(), m.FQ + I.of, (size_t)I.nf * sizeof(V4), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int f = 0; f < I.nf; ++f) {
      out->facet_ref[3 * f] = q[f].x;
      out->facet_ref[3 * f + 1] = q[f].y;
      out->facet_ref[3 * f + 2] = q[f].z;
    }
  }
  return cuda_status(h);
}

int cdr_batch_finished(cdr_handle* h, int32_t* slots, int32_t cap, int32_t* n) {
  if (!h || !h->batch || !n || cap < 0 || (cap > 0 && !slots)) return CDR_ERR_INVALID_INPUT;
  int c = 0;
  for (int k = 0; k < h->ninst; ++k)
    if (h->insts[k].state == 2) {
      if (c < cap) slots[c] = k;
      ++c;
    }
  *n = c;
  return CDR_OK;
}

int cdr_batch_remove(cdr_handle* h, int32_t slot) {
  if (!h || !h->batch || slot < 0 || slot >= h->ninst || h->insts[slot].state == 0)
    return CDR_ERR_INVALID_INPUT;
  launch_kill_instance(h->m, slot, h->stream);
  cudaStreamSynchronize(h->stream);
  h->deadKnown = false;
  h->fullClassify = true;
  h->insts[slot] = cdr_handle::Inst();
  h->freeSlots.push_back(slot);
  return cuda_status(h);
}

int cdr_eval_predicates(int32_t kind, const double* in, int32_t n, int32_t* sign, double* out,
                        void* stream) {
  if (kind < 0 || kind > 11 || n < 0 || !in || !sign) return CDR_ERR_INVALID_INPUT;
  if (n == 0) return CDR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  double* din = nullptr;
  int* dsg = nullptr;
  double* dout = nullptr;
  if (cudaMalloc(&din, (size_t)n * 16 * 8) != cudaSuccess ||
      cudaMalloc(&dsg, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&dout, (size_t)n * 3 * 8) != cudaSuccess) {
    cudaFree(din);
    cudaFree(dsg);
    cudaFree(dout);
    return CDR_ERR_OOM;
  }
  cudaMemcpyAsync(din, in, (size_t)n * 16 * 8, cudaMemcpyHostToDevice, s);
  launch_eval_pred(kind, din, n, dsg, dout, s);
  cudaMemcpyAsync(sign, dsg, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  if (out) cudaMemcpyAsync(out, dout, (size_t)n * 3 * 8, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  int ov = exact_overflow_flag(s, true);
  cudaFree(din);
  cudaFree(dsg);
  cudaFree(dout);
  if (cudaGetLastError() != cudaSuccess) return CDR_ERR_CUDA;
  return ov ? CDR_ERR_INTERNAL : CDR_OK;
}

int cdr_set_tuning(cdr_handle* h, const cdr_tuning* t) {
  if (!h || !t) return CDR_ERR_INVALID_INPUT;
  if (t->fused_max < -1 || t->fused_max > kFusedMax || t->grow1_blocks_per_sm < 0 ||
      t->grow1_blocks_per_sm > 32 || t->tier2_warps < 0 || t->tier2_warps > 152 * 32 ||
      t->tier1_cavity < 0 || t->tier1_cavity > Tier1::CAPC || t->tier1_boundary < 0 ||
      t->tier1_boundary > Tier1::CAPB || t->compact_min_tets < 0 || t->compact_dead_pct < 0 ||
      t->compact_dead_pct > 100)
    return CDR_ERR_INVALID_INPUT;
  h->tier1Cav = t->tier1_cavity;
  h->tier1Bnd = t->tier1_boundary;
  h->compactMin = t->compact_min_tets > 0 ? t->compact_min_tets : (1 << 19);
  h->compactPct = t->compact_dead_pct > 0 ? t->compact_dead_pct : 50;
  h->fused = t->fused_max != -1;
  h->fusedMax = t->fused_max > 0 ? t->fused_max : kFusedDefault;
  h->grow1PerSM = t->grow1_blocks_per_sm > 0 ? t->grow1_blocks_per_sm : 8;
  int w = t->tier2_warps > 0 ? t->tier2_warps : 152 * 4;
  h->tier2Warps = w + (w & 1);  // tier-2 launches run two warps per block
  return CDR_OK;
}

int cdr_profile(cdr_handle* h, int32_t enable, int32_t reset, double* ms, int64_t* calls,
                int64_t* counters) {
  if (!h) return CDR_ERR_INVALID_INPUT;
  if (reset) {
    for (int g = 0; g < 32; ++g) {
      h->prof_ms[g] = 0;
      h->prof_calls[g] = 0;
      h->prof_ctr[g] = 0;
    }
  }
  if (ms)
    for (int g = 0; g < 32; ++g) ms[g] = h->prof_ms[g];
  if (calls)
    for (int g = 0; g < 32; ++g) calls[g] = h->prof_calls[g];
  if (counters)
    for (int g = 0; g < 32; ++g) counters[g] = h->prof_ctr[g];
  if (enable >= 0) {
    h->prof = enable != 0;
    h->profGrowOnly = enable == 2;
  }
  return CDR_OK;
}

}  // extern "C"
