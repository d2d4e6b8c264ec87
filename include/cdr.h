/* cdr.h -- constrained Delaunay refinement on one GB300 (sm_103a).
 *
 * The library implements the per-round parallel refinement step of gQM3D
 * (Chen & Tan, "Computing Three-dimensional Constrained Delaunay Refinement
 * Using the GPU", I3D 2019):
 *   Sec. 1  -- problem: given a piecewise linear complex G = (P, E, F), a
 *              constrained Delaunay triangulation (CDT) T conforming to G and a
 *              constant B, add Steiner points until (most) tetrahedra have
 *              circumradius / shortest edge <= B, keeping T a CDT of G.
 *   Sec. 2  -- rounds: subsegments, then subfaces, then bad tetrahedra are split;
 *              splitting points are midpoints / circumcentres; each point's
 *              Delaunay region is grown, regions are made disjoint by
 *              predetermined priorities ("grow-and-blast"), and the surviving
 *              points are inserted concurrently.
 *
 * Conventions used by every call:
 *   - Coordinates are FP64, row-major (x, y, z) per vertex.
 *   - Ids are int32. A tetrahedron (a, b, c, d) is positively oriented:
 *     (b - a) . ((c - a) x (d - a)) > 0.
 *   - Constraint labels: a subsegment is a mesh edge lying on a PLC segment (E),
 *     given with that segment's id; a subface is a mesh face lying in a PLC
 *     polygon (F), given with that polygon's (facet's) id. Each PLC polygon edge
 *     is itself a segment.
 *   - All pointers passed in are HOST pointers unless stated otherwise. The
 *     library copies every input; the caller keeps ownership of its buffers.
 *   - Device memory comes from the caller's allocator when one is given (the
 *     Python binding passes PyTorch's caching allocator), else from
 *     cudaMallocAsync on the handle's stream. The handle owns its device buffers
 *     until cdr_destroy.
 *   - One handle is used by one host thread at a time. No call throws; every
 *     call returns a status code (CDR_OK = 0), see cdr_status_string.
 *   - Errors leave the handle usable unless stated (CDR_ERR_CUDA and
 *     CDR_ERR_INTERNAL may leave it in an unspecified state; destroy it).
 */
#ifndef CDR_H_
#define CDR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CDR_OK = 0,
  CDR_ROUND_LIMIT = 1,        /* informational: max_rounds reached with work left */
  CDR_ERR_INVALID_INPUT = -1, /* malformed mesh / labels / arguments             */
  CDR_ERR_OOM = -2,           /* the allocator returned NULL                      */
  CDR_ERR_CUDA = -3,          /* a CUDA call failed                               */
  CDR_ERR_ITER_LIMIT = -4,    /* a bounded device loop gave up                    */
  CDR_ERR_INTERNAL = -5,      /* exact-arithmetic capacity or an invariant failed */
  CDR_ERR_TOO_LARGE = -6      /* more items than a fixed-capacity call can hold   */
};

typedef struct cdr_handle cdr_handle;

/* Device memory provider. alloc returns device memory of at least `bytes` bytes
 * usable on `stream` (NULL on failure); free releases it. */
typedef struct {
  void* (*alloc)(uint64_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, uint64_t bytes, void* ctx, void* stream);
  void* ctx;
} cdr_allocator;

/* The input: a CDT with its constraint labels (Sec. 1).
 *   xyz[n_verts*3]            vertex coordinates
 *   tets[n_tets*4]            positively oriented tetrahedra
 *   segs[n_segs*2], seg_id[]  subsegments (mesh edges) and their PLC segment ids
 *   tris[n_tris*3], facet_id[] subfaces (mesh faces) and their PLC facet ids;
 *                              facet ids are 0 .. n_facets-1
 *   facet_ref[n_facets*3]     optional (NULL = derived) per-facet reference point
 *                              used to read circles and sides inside a facet; the
 *                              derived point is the facet's first listed triangle's
 *                              first vertex moved along the dominant axis of that
 *                              triangle's normal by the smallest power of two that
 *                              is >= 4x the largest bounding-box extent.
 *   tet_flag[n_tets]          optional (NULL = none) element flags, coded as
 *   subface_flag[n_tris]      cdr_mesh_out's (tetrahedra: bit1 unsplittable;
 *   subseg_flag[n_segs]       subfaces and subsegments: bit0 must split, bit1
 *                              unsplittable). With them, a mesh exported
 *                              between rounds and created again (by cdr_create
 *                              or cdr_batch_add) refines on exactly as the
 *                              uninterrupted refinement would: a checkpoint on
 *                              the host. Other bits: CDR_ERR_INVALID_INPUT.
 * Every hull face must be a subface (the domain is closed by facets). */
typedef struct {
  const double* xyz;
  int32_t n_verts;
  const int32_t* tets;
  int32_t n_tets;
  const int32_t* segs;
  const int32_t* seg_id;
  int32_t n_segs;
  const int32_t* tris;
  const int32_t* facet_id;
  int32_t n_tris;
  int32_t n_facets;
  const double* facet_ref;
  const uint8_t* tet_flag;
  const uint8_t* subface_flag;
  const uint8_t* subseg_flag;
} cdr_mesh_in;

/* Options. Zero-initialised fields select the defaults given. */
typedef struct {
  double guard2;        /* squared shortest-edge guard; <= 0: (1e-9 * bbox diagonal)^2 */
  int32_t walk_limit;   /* point-location step limit; 0: 100000                         */
  int32_t reserve_factor; /* initial capacity multiple of the input sizes; 0: 4          */
  int32_t mixed_rounds; /* 0: each round serves one class, the first non-empty of
                           subsegments, subfaces, bad tetrahedra (Sec. 2's order);
                           1: each round takes every flagged element, and the
                           class decides priority first, so a subsegment still
                           beats a subface and a subface beats a tetrahedron;
                           2: subsegments and subfaces together, bad
                           tetrahedra only once both are done (fewer rounds) */
} cdr_options;

/* Per-call statistics. */
typedef struct {
  int32_t rounds;
  int32_t rounds_by_class[3]; /* subsegment, subface, tetrahedron rounds        */
  int64_t candidates;         /* splitting points evaluated                     */
  int64_t steiner_inserted;   /* points inserted                                */
  int64_t rejected;           /* points refused for encroachment (split first)  */
  int64_t blasted;            /* eligible points that lost a priority conflict  */
  int64_t unsplittable;       /* elements given up (guard, closure, overflow)   */
  int64_t n_verts, n_tets, n_subfaces, n_subsegs;
  int64_t n_bad_left;         /* bad tetrahedra left (all unsplittable)         */
} cdr_stats;

/* Sizes of the live mesh, for cdr_export. */
typedef struct {
  int32_t n_verts, n_tets, n_subfaces, n_subsegs, n_facets;
} cdr_sizes;

/* Export buffers (host, caller-owned, sized from cdr_export_sizes). Any pointer
 * may be NULL to skip that array.
 *   xyz[n_verts*3]
 *   tets[n_tets*4]            live tetrahedra, positively oriented
 *   tet_flag[n_tets]          bit1: unsplittable
 *   subfaces[n_subfaces*4]    a, b, c, facet id
 *   subface_flag[n_subfaces]  bit0: must split (encroached by a refused point),
 *                             bit1: unsplittable
 *   subsegs[n_subsegs*3]      a, b, segment id
 *   subseg_flag[n_subsegs]    as subface_flag
 *   facet_ref[n_facets*3]     the facet reference points in use */
typedef struct {
  double* xyz;
  int32_t* tets;
  uint8_t* tet_flag;
  int32_t* subfaces;
  uint8_t* subface_flag;
  int32_t* subsegs;
  uint8_t* subseg_flag;
  double* facet_ref;
} cdr_mesh_out;

/* Create a handle from a CDT with constraint labels (Sec. 1). The mesh is
 * validated (index ranges, labels present as edges / faces, faces shared by at
 * most two tetrahedra, every hull face a subface): CDR_ERR_INVALID_INPUT.
 * stream is a cudaStream_t (NULL = legacy default stream). alloc may be NULL. */
int cdr_create(const cdr_mesh_in* in, const cdr_options* opt, const cdr_allocator* alloc,
               void* stream, cdr_handle** out);

/* Refine (Sec. 2) with bound B until no encroached subsegment, encroached
 * subface or bad tetrahedron is left (apart from unsplittable ones), or
 * max_rounds rounds ran (then CDR_ROUND_LIMIT). stats may be NULL. */
int cdr_refine(cdr_handle* h, double B, int32_t max_rounds, cdr_stats* stats);

/* Exactly one round (Sec. 2) with bound B. *cls receives the class served
 * (0 subsegments, 1 subfaces, 2 tetrahedra, 3 several classes in a mixed
 * round; -1 = nothing left). stats
 * (nullable) receives that round's counts. */
int cdr_round(cdr_handle* h, double B, int32_t* cls, cdr_stats* stats);

/* Sizes of the live mesh. */
int cdr_export_sizes(cdr_handle* h, cdr_sizes* out);

/* Copy the live mesh into caller buffers (see cdr_mesh_out). */
int cdr_export(cdr_handle* h, const cdr_mesh_out* out);

/* Report of the last round, candidate by candidate in priority order (used to
 * check a round against a reference implementation). Two-call protocol:
 * call with all pointers NULL to get *n_cand and *n_cav_total, then with
 * buffers:
 *   keys[n_cand*4]      the element's sorted vertex ids (-1 padded)
 *   pts[n_cand*3]       splitting point
 *   outcome[n_cand]     0 eligible, 1 refused (encroachment), 2 unsplittable,
 *                       4 stopped on a higher-priority start tetrahedron
 *   reason[n_cand]      detail code: 0 none, 1 degenerate or non-finite point,
 *                       2 / 3 the walk crossed a subface / subsegment,
 *                       4 walk or ring step limit, 5 the walk left the hull,
 *                       6 the region failed a validity check (closure, star,
 *                       boundary vertices), 7 cavity over the limit,
 *                       8 shortest-edge guard, 9 encroaches a subface or
 *                       subsegment, 10 given up by the stall rule of
 *                       subsegment rounds, 11 encroaches only unsplittable
 *                       elements, 12 would delete a subsegment
 *   survived[n_cand]    1 if inserted
 *   n_cav[n_cand], n_bnd[n_cand], n_fcav[n_cand]  region sizes
 *   cav[n_cav_total*4]  each candidate's cavity tetrahedra as sorted vertex ids,
 *                       concatenated in candidate order (eligible candidates) */
int cdr_round_report(cdr_handle* h, int32_t* n_cand, int64_t* n_cav_total, int32_t* keys,
                     double* pts, int32_t* outcome, int32_t* reason, int32_t* survived,
                     int32_t* n_cav, int32_t* n_bnd, int32_t* n_fcav, int32_t* cav);

/* Save the current mesh on the device / restore it (for repeated timing). */
int cdr_checkpoint(cdr_handle* h);
int cdr_restore(cdr_handle* h);

/* Release the handle and all its device memory. NULL is ignored. */
void cdr_destroy(cdr_handle* h);

/* Delaunay tetrahedralisation of points whose bounding-box corners are among
 * them and whose other points lie strictly inside the box, built on the device
 * by the same grow / select / insert rounds with plain points as candidates.
 * The result (export: vertices = the points in input order, tetrahedra) has no
 * constraint labels. Points that coincide with an earlier point are skipped
 * (*n_skipped). */
int cdr_delaunay_box(const double* xyz, int32_t n, const cdr_options* opt,
                     const cdr_allocator* alloc, void* stream, cdr_handle** out,
                     int32_t* n_skipped, int32_t* n_rounds);

/* ------------------------------------------------------------------ batches
 * Many independent refinements (instances) advance together, each round being
 * one pass of every kernel over all instances' candidates (Sec. 2's round, with
 * every instance serving its own first non-empty class: subsegments, then
 * subfaces, then bad tetrahedra). The instances live as disconnected parts of
 * one device-resident mesh. An element's priority depends only on its
 * geometry and the relative order of its vertex ids, so an instance's result is
 * the same whether it is refined alone (cdr_create + cdr_refine) or in a
 * batch, whenever it joins. Instances can join (cdr_batch_add) and leave
 * (cdr_batch_remove) between rounds.
 *
 * Create an empty batch. opt: walk_limit and guard2 apply to every instance
 * (guard2 <= 0: each instance's own default); alloc, stream as for cdr_create.
 * The batch is a cdr_handle: cdr_destroy releases it, cdr_export copies the
 * whole multi-instance mesh, and cdr_refine / cdr_round / cdr_checkpoint /
 * cdr_restore reject it (CDR_ERR_INVALID_INPUT). */
int cdr_batch_create(const cdr_options* opt, const cdr_allocator* alloc, void* stream,
                     cdr_handle** out);

/* Admit an instance: a CDT with labels as for cdr_create (validated the same
 * way) and its bound B. *slot receives its slot (slots of removed instances
 * are reused). The input is copied; the call synchronises the batch's stream.
 * CDR_ERR_OOM if the batch would exceed 2^28 vertices or the device memory. */
int cdr_batch_add(cdr_handle* b, const cdr_mesh_in* in, double B, int32_t* slot);

/* One round for every instance with work left. *n_active (nullable) receives
 * the number of instances that had candidates this round (0: all done). */
int cdr_batch_round(cdr_handle* b, int32_t* n_active);

/* Rounds until no instance has work left or max_rounds rounds ran (then
 * CDR_ROUND_LIMIT). *rounds (nullable) receives the rounds run. */
int cdr_batch_refine(cdr_handle* b, int32_t max_rounds, int32_t* rounds);

/* Statistics of one instance (accumulated over the rounds it took part in;
 * the sizes and n_bad_left are those of its current mesh) and its state:
 * 0 free slot, 1 refining, 2 done. */
int cdr_batch_stats(cdr_handle* b, int32_t slot, cdr_stats* stats, int32_t* state);

/* Sizes and copy of one instance's mesh, in the layout of cdr_export_sizes /
 * cdr_export, with vertex ids, facet ids and segment ids local to the
 * instance (vertices in the order the instance created them). */
int cdr_batch_export_sizes(cdr_handle* b, int32_t slot, cdr_sizes* out);
int cdr_batch_export(cdr_handle* b, int32_t slot, const cdr_mesh_out* out);

/* Slots of the instances that have finished (state 2), in slot order: up to
 * cap of them into slots[], their total count into *n. Host-side, no device
 * work. */
int cdr_batch_finished(cdr_handle* b, int32_t* slots, int32_t cap, int32_t* n);

/* Remove an instance: its elements are retired and its slot freed. */
int cdr_batch_remove(cdr_handle* b, int32_t slot);

/* Text for a status code. */
const char* cdr_status_string(int status);

/* Timing of the kernel groups of each round with CUDA events recorded on the
 * handle's stream, and device work counters (always accumulated).
 *   enable   1 on, 2 on for the region-growth groups (4, 5) only, 0 off,
 *            -1 unchanged;  reset  nonzero clears the totals first
 *   ms[32]   accumulated milliseconds per group: 0 classify, 1 order, 2 split,
 *            3 locate, 4 grow (tier 1), 5 grow (tier 2), 6 select, 7 scan,
 *            8 insert, 9 compact, 10 whole rounds run as one kernel (rounds
 *            with at most cdr_tuning.fused_max candidates, 128 by default)
 *   calls[32] launches timed per group
 *   counters[32] 0 refused, 1 unsplittable, 2 eligible-but-blasted, 3 inserted,
 *            4 retried in tier 2, 5 invariant failures, 6 neighbour tetrahedra
 *            tested by growth, 7 cavity tetrahedra, 8 boundary faces (6..8 in
 *            rounds with separately launched growth kernels), 9 new
 *            tetrahedra written, 10 refusals flagging a new candidate, 11 regions
 *            stopped on a higher-priority start, 12 tetrahedra retired by
 *            insertion, 13 compactions of the tetrahedron arrays,
 *            15 kernels of this library launched (library
 *            primitives such as sorts and scans excluded), 16..18 as 6..8 in
 *            rounds run as one kernel
 * Any output pointer may be NULL. */
int cdr_profile(cdr_handle* h, int32_t enable, int32_t reset, double* ms, int64_t* calls,
                int64_t* counters);

/* Launch tuning of a handle (one mesh or a batch). Results do not depend on
 * it, only speed; zero fields select the defaults.
 *   fused_max            rounds with at most this many candidates (1..512) run
 *                        as one kernel (above 128, a warp takes several
 *                        candidates in turn); -1: never; 0: 128
 *   grow1_blocks_per_sm  at most this many blocks per SM in the region-growth
 *                        grid (1..32); 0: 8
 *   tier2_warps          warps (each with a global workspace) for regions that
 *                        outgrow tier 1 (1..4864); 0: 608
 *   tier1_cavity         cavity tetrahedra a tier-1 (shared-memory) workspace
 *                        holds before the region is re-grown in tier 2 (1..64);
 *                        0: 64
 *   tier1_boundary       cavity boundary faces a tier-1 workspace holds
 *                        (1..96); 0: 96
 *   compact_min_tets     tetrahedron slots below which the dead ones are never
 *                        compacted away; 0: 524288
 *   compact_dead_pct     the tetrahedron arrays are compacted once at least this
 *                        percentage of their slots is dead (1..100); 0: 50 */
typedef struct {
  int32_t fused_max;
  int32_t grow1_blocks_per_sm;
  int32_t tier2_warps;
  int32_t tier1_cavity;
  int32_t tier1_boundary;
  int32_t compact_min_tets;
  int32_t compact_dead_pct;
} cdr_tuning;
int cdr_set_tuning(cdr_handle* h, const cdr_tuning* t);

/* Library self-description: sm architecture compiled for, e.g. 103. */
int cdr_device_arch(void);

/* Evaluate one device predicate or formula over a batch (a checking aid for the
 * geometry every round relies on; Sec. 1 bad-tetrahedron rule, Sec. 2 splitting
 * points and Delaunay-region tests).
 *   in[n*16]  per item: points a, b, c, d, e as (x, y, z) in doubles 0..14;
 *             for kind 7 the bound B sits in double 12
 *   kind      0 orient3d(a,b,c,d) sign       1 insphere(a,b,c,d; e) sign (> 0:
 *             strictly inside, abcd positively oriented)
 *             2 diametral (a-c).(b-c) sign   3 equatorial(a,b,c; d) sign (< 0:
 *             strictly inside the smallest sphere through a, b, c)
 *             4 tetrahedron circumcentre of (a,b,c,d)   5 circumcentre of (a,b,c)
 *             6 midpoint of (a,b)            7 bad tetrahedron (a,b,c,d) for B
 *             8..11 the exact-arithmetic paths of 0, 1, 3, 2 alone
 *   sign[n]   the sign (kinds 4..7: 1 = ok / bad, 0 = degenerate / not bad)
 *   out[n*3]  (nullable) the point computed by kinds 4..6
 * Uses cudaMalloc / cudaFree for its own buffers and synchronises `stream`.
 * CDR_ERR_INTERNAL if the exact arithmetic ran out of capacity. */
int cdr_eval_predicates(int32_t kind, const double* in, int32_t n, int32_t* sign, double* out,
                        void* stream);

/* Largest batch cdr_eval_predicates_noalloc accepts. */
#define CDR_EVAL_NOALLOC_MAX_ITEMS 16384

/* cdr_eval_predicates without device allocation. The paper has no counterpart:
 * this is a convenience for callers that cannot allocate device memory. Two
 * kinds of caller cannot: one that keeps kernels running on other streams
 * (cudaFree waits for the whole device, so each call would stall that work),
 * and one whose device memory is held by a caching allocator such as
 * PyTorch's (cudaMalloc can fail while the memory sits reserved in the cache).
 *
 * Arguments, results, layout and error codes are those of cdr_eval_predicates.
 * The device copies of in, sign and out live in one fixed array in the
 * library's device image (2.44 MiB, present on every GPU that loads the
 * library until the process exits), so:
 *   - n > CDR_EVAL_NOALLOC_MAX_ITEMS returns CDR_ERR_TOO_LARGE and does nothing;
 *   - no call allocates or frees device memory (cudaMalloc, cudaFree or any
 *     allocating library routine);
 *   - every call looks the array up on the current device
 *     (cudaGetSymbolAddress); no address is cached, so a call after
 *     cudaDeviceReset finds the array where the reloaded library put it;
 *   - the call copies through pageable host memory and synchronises `stream`,
 *     so it cannot be made on a stream that is being captured into a graph;
 *   - every call on a device shares the array, and the exact-arithmetic
 *     overflow flag it reads back (one word in the library's image). Calls
 *     whose device work overlaps (other streams, other host threads) race on
 *     both, so their results and their CDR_ERR_INTERNAL status are undefined:
 *     serialise them. Each call synchronises `stream` before it returns, so
 *     calls from one host thread never overlap.
 * The array keeps the last call's contents; each call clears what must start
 * at zero (the exact-arithmetic overflow flag) and writes every output slot
 * it reads back. */
int cdr_eval_predicates_noalloc(int32_t kind, const double* in, int32_t n, int32_t* sign,
                                double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CDR_H_ */
