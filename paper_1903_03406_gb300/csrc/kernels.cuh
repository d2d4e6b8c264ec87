// Launch wrappers exported by kernels.cu to the host driver (api.cu).
#pragma once
#include <cuda_runtime.h>

#include "mesh.cuh"

namespace cdr {

// create / labels
void launch_init_tets(const DevMesh& m, const int4* tets, int n, cudaStream_t s);
void launch_face_keys(const DevMesh& m, unsigned long long* hi, unsigned int* lo, int* val,
                      cudaStream_t s);
void launch_pair_faces(const DevMesh& m, const unsigned long long* hi, const unsigned int* lo,
                       const int* val, int n, int* err, cudaStream_t s);
void launch_label_subfaces(const DevMesh& m, const int4* tris, int n, const unsigned long long* hi,
                           const unsigned int* lo, const int* val, int nfaces, int* err,
                           cudaStream_t s);
void launch_subface_edge_keys(const DevMesh& m, unsigned long long* hi, unsigned int* lo,
                              int* val, cudaStream_t s);
void launch_pair_subface_edges(const DevMesh& m, const unsigned long long* hi,
                               const unsigned int* lo, const int* val, int n, int* err,
                               cudaStream_t s);
void launch_hash_clear(const DevMesh& m, cudaStream_t s);
void launch_hash_insert_subsegs(const DevMesh& m, int g0, int g1, cudaStream_t s);
void launch_mark_edges(const DevMesh& m, cudaStream_t s);
void launch_check_create(const DevMesh& m, int* err, cudaStream_t s);
void launch_recompute_bad(const DevMesh& m, double B, cudaStream_t s);

// classification and queues
// add: counts added by the last round that the host has not read yet, or null
void launch_classify(const DevMesh& m, bool full, int* err, cudaStream_t s,
                     const int4* add = nullptr);
void launch_prio(const DevMesh& m, int cls, const int* elems, int n, unsigned long long* keys,
                 cudaStream_t s);
void launch_tiefix(const DevMesh& m, int cls, const unsigned long long* keys, int* elems, int n,
                   cudaStream_t s);
void launch_count_inst(const DevMesh& m, const uint8_t* candG, const uint8_t* candS,
                       const uint8_t* candT, cudaStream_t s);
void launch_count_single(const DevMesh& m, unsigned long long* cnt, cudaStream_t s,
                         const int4* add = nullptr);
void launch_round_flags(const DevMesh& m, const uint8_t* candG, const uint8_t* candS,
                        const uint8_t* candT, uint8_t* out, cudaStream_t s);
void launch_decode_cands(const DevMesh& m, int* cand, uint8_t* ccls, int* cinst, int n,
                         cudaStream_t s);

// one round
void launch_split(const DevMesh& m, const DevRound& r, cudaStream_t s);
void launch_locate(const DevMesh& m, const DevRound& r, int* hint, cudaStream_t s);
void launch_seed(const DevMesh& m, const DevRound& r, cudaStream_t s);
void launch_grow1(const DevMesh& m, const DevRound& r, int blocks_per_sm, cudaStream_t s);
// does the separately launched tier-1 growth of this round use the
// tetrahedron-only kernel (Tier1 slabs) rather than the larger one (Tier1Big)
bool grow1_tets_only(const DevRound& r);
SlabOff slab1_layout(bool tets_only);
void launch_grow2(const DevMesh& m, const DevRound& r, int nwarps, cudaStream_t s);
void launch_select(const DevMesh& m, const DevRound& r, cudaStream_t s);
void launch_insert(const DevMesh& m, const DevRound& r, int* hint, cudaStream_t s);
void launch_stall(const DevMesh& m, const DevRound& r, cudaStream_t s);

// rounds with few candidates: the whole round in one block
constexpr int kFusedBlocks = 8;  // one cluster (the portable maximum)
constexpr int kFusedWarps = 16;  // per block
constexpr int kFusedDefault = kFusedBlocks * kFusedWarps;  // one warp per candidate
constexpr int kFusedMax = 4 * kFusedDefault;  // the largest setting: four per warp
struct FusedOut {
  int4 tot;  // new vertices, tetrahedra, subfaces, subsegments
  int n2;    // regions grown in tier 2
};
// src: the round's candidates before ordering (elements, or concatenated
// indices when r.cls < 0), ordered by the kernel into cand_w (and ccls_w,
// cinst_w); nullptr if r.cand is already in priority order
void launch_round_fused(const DevMesh& m, const DevRound& r, int* hint, int4* offs, FusedOut* out,
                        bool do_stall, const int* src, int* cand_w, uint8_t* ccls_w, int* cinst_w,
                        cudaStream_t s);

// maintenance
void launch_compact_flags(const DevMesh& m, int* alive, cudaStream_t s);
void launch_compact_move(const DevMesh& m, const int* newid, TetRec* T2, int4* TS2,
                         unsigned char* F2, int* hint, int nhint, cudaStream_t s);
void launch_compact_fix(const DevMesh& m, const int* newid, cudaStream_t s);
void launch_follow_fwd(const DevMesh& m, int* hint, const int* state, int n, cudaStream_t s);

// export helpers
void launch_live_flags(const unsigned char* flag, int n, int* out, cudaStream_t s);
void launch_gather_tets(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                        cudaStream_t s);
void launch_gather_subfaces(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                            cudaStream_t s);
void launch_gather_subsegs(const DevMesh& m, const int* pos, int4* out, unsigned char* oflag,
                           cudaStream_t s);
void launch_report_cav(const DevMesh& m, const DevRound& r, const int* offs, int4* out,
                       cudaStream_t s);

// batches
void launch_append(const DevMesh& d, const DevMesh& src, int ov, int ot, int os, int og, int of,
                   int oseg, int slot, cudaStream_t s);
void launch_kill_instance(const DevMesh& m, int slot, cudaStream_t s);
void launch_inst_flags(const DevMesh& m, int slot, int kind, int n, int* out, cudaStream_t s);
void launch_inst_bad(const DevMesh& m, int* flag, int n, cudaStream_t s);
void launch_inst_gather(const DevMesh& m, int kind, int n, const int* flag, const int* pos,
                        const int* vpos, int of, int oseg, int4* out, uint8_t* oflag, V4* oxyz,
                        cudaStream_t s);

void launch_eval_pred(int kind, const double* in, int n, int* sign, double* outp, cudaStream_t s);
int exact_overflow_flag(cudaStream_t s, bool reset);
void exact_overflow_copy_async(int* dst, cudaStream_t s);
int checked_error(int* info, cudaStream_t s);
int phase_counters(unsigned long long* out32, cudaStream_t s);

}  // namespace cdr
