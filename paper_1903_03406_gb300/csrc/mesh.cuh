// Device mesh layout and the per-round buffers.
//
// Layout (GB300: every gather is a 32-byte sector, the mesh of the 100k-point
// workload fits the 129 MB L2):
//   V      V4 per vertex (x, y, z, unused)            one sector per vertex
//   T      TetRec per tetrahedron: int4 v, int4 n           one sector per tet
//          v.k : vertex id (bits 0..27) | face k is a subface (bit 28) |
//                edge marks (bits 29..30 of v.x, v.y, v.z: subsegment on edges
//                01 02 | 03 12 | 13 23)
//          n.k : neighbour across face k as (tet << 2 | its face), -1 on the hull
//   TS     int4 per tet: subface id on each face (-1), read only for marked faces
//   Tflag  bit0 dead, bit1 bad, bit2 unsplittable
//   Tmark  64-bit priority marks (round epoch << 32 | candidate rank)
//   Tseed  64-bit claims of start tetrahedra, same encoding
//   Tfwd   for a dead tet, one tet of the star that replaced it
//   SV     int4 per subface (a, b, c, facet)
//   SN     int4 per subface: facet neighbour across edge k (opposite vertex k),
//          -1 across a subsegment; .w = one adjacent tet as (tet << 2 | face)
//   Sflag  bit0 dead, bit2 unsplittable; Smust: split first (set by refusals)
//   GV     int4 per subsegment (a, b, segment id, one tet containing the edge)
//   Gflag  bit0 dead, bit2 unsplittable; Gmust as Smust
//   FQ     V4 per facet: reference point off the facet's plane
//   HK/HV  open-addressing hash (min<<32|max) -> subsegment id
// Paper passages: elements, subsegments, subfaces (Sec. 1, Sec. 2).
#pragma once
#include <cstdint>

namespace cdr {

// 32-byte vertex / point record: one sector per gather
struct __align__(32) V4 {
  double x, y, z, w;
};
__host__ __device__ inline V4 make_v4(double x, double y, double z, double w) {
  V4 v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = w;
  return v;
}

constexpr int kVidMask = 0x0FFFFFFF;
constexpr int kSubBit = 28;
constexpr int kMaxVerts = 1 << 28;
constexpr int kMaxTets = 1 << 29;

enum : uint8_t { F_DEAD = 1, F_BAD = 2, F_UNSPL = 4 };
enum { CLS_SUBSEG = 0, CLS_SUBFACE = 1, CLS_TET = 2, CLS_POINT = 3 };
enum { OUT_OK = 0, OUT_REJECT = 1, OUT_UNSPL = 2, OUT_RETRY = 3, OUT_BLASTED = 4 };
enum {
  RS_NONE = 0,
  RS_BADPOINT = 1,
  RS_WALK_SUBFACE = 2,
  RS_WALK_SUBSEG = 3,
  RS_WALK_LIMIT = 4,
  RS_WALK_HULL = 5,
  RS_CLOSURE = 6,
  RS_OVERFLOW = 7,
  RS_GUARD = 8,
  RS_ENCROACH = 9,
  RS_STRUCT = 10,
  RS_ENCROACH_UNSPL = 11,
  RS_STARDEL = 12,
};

struct __align__(32) TetRec {
  int4 v;
  int4 n;
};

struct DevMesh {
  V4* V;
  TetRec* T;
  int4* TS;
  uint8_t* Tflag;
  unsigned long long* Tmark;
  unsigned long long* Tseed;  // start-tetrahedron claims (round epoch << 32 | rank)
  int* Tfwd;
  int4* SV;
  int4* SN;
  uint8_t* Sflag;
  uint8_t* Smust;
  unsigned long long* Smark;
  int4* GV;
  uint8_t* Gflag;
  uint8_t* Gmust;
  V4* FQ;
  unsigned long long* HK;
  int* HV;
  int hmask;
  int nV, nT, nS, nG, nF;
  int capV, capT, capS, capG;  // allocated sizes (bounds of the checked build)
  double guard2;
  int walk_limit;
  // Candidate flags kept from round to round, and the subfaces / subsegments
  // whose flag must be recomputed (created or touched by the last round).
  uint8_t* candT;
  uint8_t* candS;
  uint8_t* candG;
  uint8_t* dirtyS;
  uint8_t* dirtyG;
  // Instances: independent meshes held as disconnected parts of this mesh
  // (batched refinement). Each vertex records its instance; an element belongs
  // to the instance of its vertices. Vinst == nullptr means one instance (0)
  // whose bound is the round's B and whose guard is guard2.
  int* Vinst;
  const double* instB;          // per instance: quality bound B
  const double* instG2;         // per instance: squared shortest-edge guard
  const int* instCls;           // per instance: class served this round (-1: none)
  unsigned long long* instCnt;  // per instance: classification counts [3]
  unsigned long long* instSt;   // per instance: round counters [IS_COUNT]
  int ninst;
};

// per-instance round counters
enum { IS_SURV = 0, IS_UNSPL, IS_NEWCAND, IS_REJECT, IS_STALLED, IS_COUNT };

// Tier capacities of the region-growth workspace. Tier 1 lives in shared
// memory (one workspace per warp); candidates whose region does not fit are
// re-run in tier 2, whose workspace lives in global memory. Tier 2's cavity cap
// is the method's limit: a larger cavity makes the element unsplittable.
template <int CAPC_, int CAPB_, int CAPF_, int CAPFB_, int HCAP_>
struct Caps {
  static constexpr int CAPC = CAPC_, CAPB = CAPB_, CAPF = CAPF_, CAPFB = CAPFB_, HCAP = HCAP_;
  static constexpr int CAP3 = 3 * CAPB_;  // boundary-table entries below this are edges
};
// HCAP: the tet hash set of growth, reused afterwards as the table of boundary
// edges and vertices (at most 3 CAPB edges + CAPB/2 + 2 vertices: 338 entries,
// two thirds of tier 1's 512 slots; a full table sends the region to tier 2).
// Tier 1's boundary-face capacity and table size can be set at build time
// (CDR_T1_CAPB, CDR_T1_HCAP) to trade shared memory per warp against the share
// of regions that move to tier 2; results do not depend on them.
#ifndef CDR_T1_CAPB
#define CDR_T1_CAPB 96
#endif
#ifndef CDR_T1_HCAP
#define CDR_T1_HCAP 512
#endif
using Tier1 = Caps<64, CDR_T1_CAPB, 32, 48, CDR_T1_HCAP>;
// Tier 1 of rounds with subsegment, subface or mixed candidates: their regions
// (a subsegment's midpoint, a facet part) are larger than a bad tetrahedron's,
// so their workspaces hold twice the cavity and three times the boundary, in
// blocks of fewer warps.
#ifndef CDR_T1BIG_CAV
#define CDR_T1BIG_CAV 128
#endif
#ifndef CDR_T1BIG_BND
#define CDR_T1BIG_BND 288
#endif
#ifndef CDR_T1BIG_HCAP
#define CDR_T1BIG_HCAP 2048
#endif
using Tier1Big = Caps<CDR_T1BIG_CAV, CDR_T1BIG_BND, 64, 96, CDR_T1BIG_HCAP>;
using Tier2 = Caps<4096, 16384, 8192, 24576, 131072>;
constexpr int kCavLimit = 4096;

// Per-candidate slab in global memory (written by growth, read by selection
// and insertion): counts then lists.
template <class C>
struct SlabLayout {
  static constexpr int OFF_CAV = 4;
  static constexpr int OFF_BIN = OFF_CAV + C::CAPC;
  static constexpr int OFF_BOUT = OFF_BIN + C::CAPB;
  static constexpr int OFF_FCAV = OFF_BOUT + C::CAPB;
  static constexpr int OFF_FBND = OFF_FCAV + C::CAPF;
  static constexpr int OFF_BV = OFF_FBND + C::CAPFB;   // 3 vertex ids per boundary face
  static constexpr int OFF_FBV = OFF_BV + 3 * C::CAPB;  // (u, x, facet) per facet edge
  static constexpr int OFF_PART = OFF_FBV + 3 * C::CAPFB;  // per boundary-face edge: the
                                                           // other face's edge (3 k + q), or -1
  static constexpr int STRIDE = OFF_PART + 3 * C::CAPB;
};

// Offsets of a tier-1 slab's lists (the layout of the workspace caps the
// round's growth kernel used), read by selection, insertion and the report.
struct SlabOff {
  int OFF_CAV, OFF_BIN, OFF_BOUT, OFF_FCAV, OFF_FBND, OFF_BV, OFF_FBV, OFF_PART, STRIDE;
};
template <class C>
inline SlabOff slab_off() {
  using L = SlabLayout<C>;
  return SlabOff{L::OFF_CAV,  L::OFF_BIN, L::OFF_BOUT, L::OFF_FCAV, L::OFF_FBND,
                 L::OFF_BV,   L::OFF_FBV, L::OFF_PART, L::STRIDE};
}

struct DevRound {
  int cls;
  int n;                       // candidates
  const int* cand;             // element ids in priority order
  const double* given;         // CLS_POINT: point coordinates (xyz), by element id
  int* loc;                    // located tet / subface (or start hint for points)
  V4* sp;                 // splitting points
  int* status;                 // outcome | reason << 8
  unsigned long long epoch;    // mark = epoch << 32 | rank
  unsigned long long seed_epoch;  // start claims of this round
  int* slab1;                  // tier-1 slabs (n * STRIDE1)
  int* slab2;                  // tier-2 slabs (n2 * STRIDE2)
  int* slab2_of;               // candidate -> tier-2 slab index (-1)
  int* ws2;                    // tier-2 workspaces (per warp)
  int nws2;                    // tier-2 workspaces allocated
  int n2;                      // tier-2 candidates
  const int* list2;            // tier-2 candidate indices
  int* survived;
  int4* counts;                // new (verts, tets, subfaces, subsegs) per candidate
  const int4* offs;            // exclusive scan of counts
  int* point_state;            // CLS_POINT: 0 pending, 1 inserted, 2 skipped
  unsigned long long* stats;   // device counters
  const uint8_t* candG;        // this round's subsegment candidates (classification)
  double B;
  // Per-candidate class and instance (rounds in which every instance serves
  // its own first non-empty class); nullptr: every candidate has class cls
  // and instance 0.
  const uint8_t* ccls;
  const int* cinst;
  int4* ckey;                  // per candidate: sorted vertex ids (round report)
  int* rflag;                  // per candidate: 1 if its region needs tier 2
  int t1cav, t1bnd;            // tier-1 cavity / boundary-face capacities in use
                               // (0: the compile-time Tier1 sizes)
  SlabOff s1;                  // layout of the tier-1 slabs (Tier1 or Tier1Big)
};

// device counters
enum {
  ST_REJECT = 0,
  ST_UNSPL,
  ST_OK,
  ST_SURV,
  ST_RETRY,
  ST_ITER,
  ST_TESTED,  // neighbour tetrahedra tested (insphere) by region growth
  ST_CAV,     // cavity tetrahedra of evaluated regions
  ST_BND,     // boundary faces of evaluated regions
  ST_NEWT,    // tetrahedra written by insertion
  ST_NEWCAND,  // refusals that flagged a subsegment not yet a candidate
  ST_BLAST,    // regions stopped on a higher-priority start tetrahedron
  ST_DEADT,    // tetrahedra retired by insertion
  ST_COUNT
};

}  // namespace cdr
