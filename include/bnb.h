/*
 * bnb.h -- C ABI of libbnb: GB300 (sm_103a) kernels for Bernstein bounds for
 * caustics (Fan, Wang, Wang, Li, Guo, Yan, Guo, Guo; ACM TOG 44(4), 2025).
 *
 * Three calls make up the path:
 *   bnb_bound_tuples      precomputation pass (Sec. 3 "Overall pipeline",
 *                         Secs. 4.3-4.5): per (emitter, specular triangle,
 *                         subdivision cell) a conservative receiver box U_k and
 *                         irradiance bound [E_lo, E_hi].
 *   bnb_build_index       bound storage (Sec. 6.1 "Bound storage"): the boxes
 *                         binned into a uniform texture-space grid; per grid
 *                         cell the sorted list of tuples with the per-tuple
 *                         bound E~ = m * max E_hi (Eq. eq_pertuple_b).
 *   bnb_sample_and_solve  rendering pass (Sec. 5, Algorithm 1; Sec. 6.1
 *                         "Root-finding"): per shading point, select each
 *                         listed tuple with P = min(gamma E~, 1) (Sec. 5.4),
 *                         solve for the path with Newton's method and return
 *                         sum E(T)/P.
 *
 * Conventions (all calls):
 *   - Every array pointer is a DEVICE pointer owned by the caller; the library
 *     never allocates device memory.  Scratch comes from the caller's workspace
 *     `ws` of `ws_bytes` bytes (256-byte aligned), sized by the matching
 *     *_ws() query.  Small structs (receiver, cfgs) are read on the host.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls enqueue kernels on it and return without synchronizing.
 *   - Return values are host-detected: BNB_OK, or BNB_ERR_INVALID for a bad
 *     argument (nothing is launched), BNB_ERR_UNSUPPORTED, or BNB_ERR_CUDA when
 *     a launch fails.  Conditions only the device can see (an output or
 *     workspace too small) are written to the device word `*status` of the
 *     output struct (0 = ok, BNB_ERR_CAPACITY) and the device counters hold the
 *     size that was needed; the outputs are then incomplete and the caller
 *     re-calls with larger buffers.  The library does not reset `*status`: the
 *     caller zeroes it (and the counters) before a call.  The same codes also
 *     go to a device error word that bnb_stream_status() reads and clears.
 *   - No C++ exception crosses the ABI.  Calls on different streams with
 *     disjoint outputs and workspaces may run concurrently.
 */
#ifndef BNB_H_
#define BNB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define BNB_OK 0
#define BNB_ERR_INVALID (-1)
#define BNB_ERR_CAPACITY (-2)
#define BNB_ERR_CUDA (-3)
#define BNB_ERR_UNSUPPORTED (-4)
#define BNB_ERR_TIMEOUT (-5)

/* Surface kinds (scattering type at the specular vertex, Eq. eq_refr_rational). */
#define BNB_REFLECT 0
#define BNB_REFRACT 1

/* Cell record flags (bits 0..7); bits 24..29 of `flags` hold the cell depth. */
#define BNB_CELL_LIVE 1u           /* box and irradiance bound valid, box meets [0,1]^2 */
#define BNB_CELL_SPLIT 2u          /* superseded by its four children (denominator sign test failed) */
#define BNB_CELL_CULL_BEHIND 4u    /* every path of the cell hits the receiver plane behind x1 (t < 0) */
#define BNB_CELL_CULL_EMPTY 8u     /* the box misses the receiver region [0,1]^2 */
#define BNB_CELL_FOLD 16u          /* Jacobian numerator changes sign: E_hi = +inf */
#define BNB_CELL_POS_UNBOUNDED 32u /* reciprocal rule / universal set used after the split limit */
#define BNB_CELL_QSIGN_FP64 64u    /* the float32 sign test was inconclusive; float64 decided it */
#define BNB_CELL_TIR 128u          /* refraction: total internal reflection on the whole cell */
#define BNB_CELL_DEPTH_SHIFT 24

/* A triangle mesh with per-vertex normals (Table 1: p_{i,0..2}, n_{i,0..2}).
 * SoA float32 device arrays of n_verts entries; int32 index arrays of n_tris.
 * Normals are interpolated un-normalized (Eq. eq_ni); they need not be unit. */
typedef struct bnb_surface {
  int32_t n_verts, n_tris;
  const float *px, *py, *pz;
  const float *nx, *ny, *nz;
  const int32_t *i0, *i1, *i2;
  int32_t kind; /* BNB_REFLECT or BNB_REFRACT */
  float eta;    /* refraction: index of the incident side / index of the transmitted side */
} bnb_surface;

/* Planar receiver T_k: x = p0 + u e1 + v e2 with texture coordinates (u,v) in
 * [0,1]^2 (host values).  Eq. eq_rct maps a path to (u,v). */
typedef struct bnb_receiver {
  float p0[3], e1[3], e2[3];
} bnb_receiver;

/* Point emitters x_0 with isotropic intensity I_0 (device arrays of n).  Each
 * emitter is part of the tuple key (Sec. 3: multiple emitters are treated as
 * part of the tuple); area lights are passed as their stratified samples. */
typedef struct bnb_emitters {
  int32_t n;
  const float *x, *y, *z, *intensity;
} bnb_emitters;

typedef struct bnb_bound_cfg {
  int32_t depth;           /* base 4-way subdivision depth D of T1's domain: 4^D cells per tuple (0..10) */
  int32_t max_extra_split; /* extra splits of a cell whose denominator sign test fails (0..4) */
  int32_t irradiance;      /* 1: irradiance bound (Sec. 4.4); 0: position only, e_hi = +inf;
                            * 2 (single refraction only, else BNB_ERR_UNSUPPORTED): the bound of 1
                            * intersected with the implicit-differentiation bound of every live
                            * record (bnb_implicit_irradiance, mode 1), after the whole pass;
                            * adaptive stopping decisions use the bound of 1 */
  int32_t fp64;            /* 1: the whole bound pass in float64 (same arithmetic, u = 2^-53) */
  /* Adaptive subdivision (Sec. 6.1 "Domain subdivision"), on when adapt_depth > depth: a live cell
   * with a bounded box at depth < adapt_depth is subdivided again unless its receiver box has area
   * (u_hi - u_lo)(v_hi - v_lo) < sigma or e_hi < alpha * e_lo, both taken in float32 on the stored
   * record (e_hi = +inf never stops by the ratio).  Sign-test splits may then go max_extra_split
   * levels below adapt_depth.  One emitter/triangle pass, not the batched or the two-vertex pass. */
  int32_t adapt_depth;     /* 0 or depth..15 (adapt_depth + max_extra_split <= 15) */
  float sigma;             /* >= 0 */
  float alpha;             /* >= 0 */
  int32_t block_threads;   /* block size of the float32 base pass (one persistent block per SM):
                              reflection 256, 320 or 384 (0: 384), refraction 128 or 256 (0: 256);
                              other values of the set are ignored by the other pass, and the
                              float64 and two-vertex passes ignore it.  The records do not depend
                              on it (the autotuner picks the fastest); values outside {0, 128, 256,
                              320, 384} are BNB_ERR_INVALID. */
  int64_t split_capacity;  /* split-queue entries per level (0: 4096 + n_base / 32); a level that
                              queues more raises BNB_ERR_CAPACITY */
} bnb_bound_cfg;

/* Per-cell bound records, SoA device arrays of `capacity` entries.  Slots
 * [0, n_base) hold the base cells in work order
 *     w = (emitter * n_tris + tri) * 4^depth + cell
 * (the 4^depth cells of one tuple are contiguous); children of split cells
 * are appended after n_base in no particular order.  Boxes are in receiver
 * texture coordinates, clipped to [0,1]^2, rounded outward. */
typedef struct bnb_cell_bounds {
  int64_t capacity;
  int64_t *count;  /* device int64: records produced (n_base + children); may exceed capacity */
  int32_t *status; /* device int32: BNB_OK or BNB_ERR_CAPACITY */
  float *u_lo, *u_hi, *v_lo, *v_hi, *e_hi;
  float *e_lo;                    /* optional (NULL: the lower irradiance bound is neither computed nor written) */
  int32_t *emitter, *tri0, *tri1; /* tri1 = -1 for single scattering */
  uint32_t *cell;                 /* base-4 digits of the cell path, most significant first */
  uint32_t *flags;                /* BNB_CELL_* | depth << BNB_CELL_DEPTH_SHIFT */
  float *e_hi_min;                /* optional (NULL: not written): the exact-arithmetic Bernstein bound
                                     that e_hi rounds outward lies in [e_hi_min, e_hi]; 0 when e_hi = +inf */
  /* host fields, written by bnb_bound_tuples for the index pass */
  int64_t n_base;
  int32_t depth;
  int32_t n_emitters;
  int32_t n_tris;
} bnb_cell_bounds;

/* Texture-space grid index (CSR).  Tuple keys: emitter << 48 | (tri1 + 1) << 24 | tri0. */
typedef struct bnb_index {
  int32_t grid_res; /* G: G x G cells over [0,1]^2, cell (i,j) = j * G + i */
  int64_t capacity; /* entries key/etilde can hold */
  int64_t *count;   /* device int64[2]: [0] entries in the index, [1] pre-merge entries needed */
  int32_t *status;  /* device int32: BNB_OK or BNB_ERR_CAPACITY */
  int64_t *offsets; /* device, G*G + 1 */
  uint64_t *key;    /* device, capacity; ascending within each grid cell */
  float *etilde;    /* device, capacity; per-tuple bound E~ (may be +inf) */
} bnb_index;

typedef struct bnb_sample_cfg {
  float gamma;                /* P = min(gamma * E~, 1) (Sec. 5.4) */
  uint64_t seed;              /* Philox4x32-10 key; counter = (point, tuple key) */
  int32_t newton_iters;       /* damped float32 Newton steps (<= 64) */
  int32_t polish_iters;       /* float64 polish steps (<= 8) */
  float tol;                  /* acceptance: |hit - target| < tol scene units */
  int64_t worklist_capacity;  /* selected (point, tuple) pairs the workspace holds */
  /* 0: Algorithm 1, one draw per listed tuple.  1: bin-packed selection (Sec. 5.3): the listed
   * tuples of a point, in list order, are packed greedily into groups whose probabilities sum to at
   * most 1 (a tuple that does not fit, fl(sum + P) > 1, opens the next group); one draw per group
   * (counter = (point, key of the group's first tuple)) selects the tuple whose float32 cumulative
   * interval [sum before it, sum with it) holds the draw, none past the group's sum.  Each tuple is
   * still selected with probability P; at most one per group. */
  int32_t bins;
  /* 0: Newton from the centroid (Det, Sec. 6.1).  > 0: stochastic starts with the reciprocal
   * weighting (Stoc, Sec. 6.1): per selected tuple Newton from a uniform random start (Philox4x32-10,
   * counter = (point, key), key = seed + (trial + 1) * 0x9E3779B97F4A7C15, two 24-bit uniforms folded
   * into the triangle); an accepted root is weighted by the number N of further random starts up to
   * the first that reaches it again (within 1e-4), N capped at stoc_trials (unbiased for roots reached
   * from more than ~1 / stoc_trials of the triangle).  One specular vertex only. */
  int32_t stoc_trials;
} bnb_sample_cfg;

typedef struct bnb_sample_stats {
  int64_t *counters;  /* device int64[4]: |U| summed, |S| summed (= worklist entries needed), roots found,
                         |B| summed (groups drawn; bins = 1 only, else 0) */
  int32_t *status;    /* device int32: BNB_OK or BNB_ERR_CAPACITY */
  int32_t *sel_count; /* optional device int32[n_points]: |S| per shading point (NULL: not written) */
  /* Optional per-selection outputs (NULL: not written), worklist_capacity entries each, in worklist
   * order: points ascending, and within a point its selected tuples in index (key) order.  Entries
   * [0, min(counters[1], worklist_capacity)) are written. */
  int64_t *sel_point; /* shading point of the selection */
  uint64_t *sel_key;  /* its tuple key */
  double *root_u1;    /* 2 per selection: the barycentric coordinates (u, v) in T1 of the accepted root
                         (the polished float64 iterate; the first accepted start with stoc_trials > 0),
                         or (NaN, NaN) when the selection contributes no root */
} bnb_sample_stats;

/* Precomputation pass.  Bounds every (emitter, triangle of s1, cell) with
 * Secs. 4.3-4.4: x1, n1 (Eqs. eq_xi, eq_ni), the reflected or refracted
 * direction (Eq. eq_refr_rational), receiver coordinates (Eq. eq_rct) and, for
 * reflection, irradiance (Eqs. eq_dwda, eq_irr_term3a) as Bernstein forms on
 * the cell, their ratio bound (Eq. eq_bbound), |d0|^-3 carried by a remainder
 * variable (Sec. 4.3).  Refraction (s1->kind = BNB_REFRACT, normals facing the
 * incident side, eta in (0, 1e6)) carries sqrt(beta) by a remainder variable
 * (Sec. 4.3), culls cells in total internal reflection (flag TIR) and reports
 * e_hi = +inf (its irradiance is not bounded).  Requires out->capacity >= n_base =
 * em->n * s1->n_tris * 4^depth.  ws: bnb_bound_tuples_ws() bytes.
 *
 * Two specular vertices (s2 != NULL; each surface BNB_REFLECT, or BNB_REFRACT with
 * eta in (0, 1e6), else BNB_ERR_UNSUPPORTED): chains x0 -> T1 (s1) -> T2 (s2) ->
 * receiver, each vertex reflecting or refracting by its surface's kind.
 * Tuple construction (Sec. 6.1): for every (emitter, T1, cell at `depth`), the
 * triangles T2 whose xy box meets the footprint of the cell's scattered rays on
 * T2's z-range (from the x1 box and the ratio bounds of d~1x/d~1z, d~1y/d~1z) are
 * candidates; each candidate is one record (tri1 = T2), records of one cell
 * contiguous, cells in base order.  Its box is the composite position bound:
 * u2 reduced to degree 1 plus a remainder (Sec. 6.1 "Degree reduction"), then
 * the second reflection or refraction and the receiver forms.  Irradiance (cfg->irradiance = 1;
 * 0: e_hi = +inf, so P = 1 in the rendering pass; 2 is not supported for chains): per live
 * record, E = I0 |C1| / (|x1 - x0|^3 |N_k| |det du_k/du1|) (Eq. eq_dwda through both vertices) is
 * bounded by evaluating the chain map (unit normals, mirror law or vector Snell, ray/plane hits)
 * in float32 interval arithmetic rounded outward, with forward-mode derivatives, over the cell's
 * barycentric bounding box (then its 2 x 2 and 4 x 4 sub-boxes that meet the cell when the whole
 * box is not certified); e_hi = +inf where the Jacobian's determinant cannot be kept away from 0,
 * e_lo (when given) the matching lower bound, e_hi_min = 0.  A float32
 * sign test that cannot decide is redone in float64 (QSIGN_FP64); a certified
 * mixed-sign denominator gives the full box (POS_UNBOUNDED; no splits:
 * max_extra_split is ignored).  *count receives the number
 * of candidates; when it exceeds out->capacity, status = BNB_ERR_CAPACITY and the
 * records are invalid: re-call with capacity >= *count.  Host fields: n_base = 0
 * and depth = 0 (the index pass takes every record on its own). */
int32_t bnb_bound_tuples(const bnb_surface *s1, const bnb_surface *s2, const bnb_receiver *rec,
                         const bnb_emitters *em, const bnb_bound_cfg *cfg, bnb_cell_bounds *out,
                         void *ws, size_t ws_bytes, void *stream);
size_t bnb_bound_tuples_ws(const bnb_surface *s1, const bnb_surface *s2, const bnb_emitters *em,
                           const bnb_bound_cfg *cfg);

/* Bound pass for callers that cannot allocate device memory.  The paper has no counterpart: this
 * is an interface for callers with no device allocator of their own (a plug-in or callback inside
 * an application whose device memory is owned by another runtime, or a program that forbids
 * allocation after start-up).  Same inputs, outputs and results as bnb_bound_tuples, but the
 * scratch comes from a fixed 8 MiB array inside the library (each GPU that loads the library holds
 * it until the process exits) instead of a caller workspace.
 *   - Returns BNB_ERR_CAPACITY, launching nothing, when bnb_bound_tuples_ws() for these arguments
 *     exceeds 8 MiB; that query is the exact test.  One surface: 80 B per triangle plus two split
 *     queues of 16 B per entry (default 4096 + n_base / 32 entries each), e.g. up to ~50k
 *     triangles with ~2M base cells.  Two surfaces: 80 B per triangle of each surface, about
 *     20 B per triangle of s2 for its grid, and 16 B per base cell of s1, so at most ~0.45M
 *     base cells (a 48^2 slab face at depth 2, 73,728 base cells, needs about 2 MB).
 *   - The first call in a CUDA context, with that context current, looks up the array's device
 *     address in it (cudaGetSymbolAddress) and caches it per context (by the driver's context id),
 *     so calls from another device, from a context created through the driver API, or after
 *     cudaDeviceReset look it up again; make the first call in each context before any stream
 *     capture there.
 *   - All calls share the one array, which keeps the last call's contents; each call clears what
 *     must start at zero on its stream.  Calls whose kernels overlap on the GPU (on different
 *     streams, or from different threads) race on the array: serialize them.
 *   - Calls no allocating function (no cudaMalloc/cudaFree, no library allocator). */
int32_t bnb_bound_tuples_noalloc(const bnb_surface *s1, const bnb_surface *s2, const bnb_receiver *rec,
                                 const bnb_emitters *em, const bnb_bound_cfg *cfg, bnb_cell_bounds *out,
                                 void *stream);

/* Bound storage (Sec. 6.1) over the records of one bnb_bound_tuples call (its
 * host fields must be set).  m multiplies the bound (Eq. eq_pertuple_b; the
 * paper uses m = 1).  pre_capacity: pre-merge (grid cell, tuple) entries the
 * workspace holds; bnb_build_index_ws(cells, grid_res, pre_capacity) bytes
 * (32 B per pre-merge entry plus 40 B per grid cell).  The pre-merge entries are
 * kept in 64 partitions of pre_capacity / 64 (tuple T, or a record emitted on
 * its own, in the partition given by a hash of T); out->count[1] reports 64 x
 * the largest partition's count, the pre_capacity these records need (it
 * depends on the records only).  Entries that do not fit are dropped and status
 * is BNB_ERR_CAPACITY. */
int32_t bnb_build_index(const bnb_cell_bounds *cells, float m, int64_t pre_capacity, bnb_index *out,
                        void *ws, size_t ws_bytes, void *stream);
size_t bnb_build_index_ws(const bnb_cell_bounds *cells, int32_t grid_res, int64_t pre_capacity);

/* Rendering pass for n_points shading points (receiver texture coordinates
 * su, sv, device float arrays).  E_out[p] (device float, n_points) receives the
 * estimate sum_{T in S} E(T) / P_T (Sec. 5.3) with E the path irradiance
 * I0 dOmega0/dA_k of Eq. eq_dwda (visibility and Fresnel ignored, Sec. 4.4).
 * With s2 != NULL (pair tuples of a two-vertex bound pass, surfaces as there)
 * every listed key names (emitter, T1, T2) and the Newton solve runs
 * through the chain x0 -> T1 -> T2 -> receiver; a root is accepted when u1 lies in
 * the closed T1, u2 in the closed T2 and both hits are in front.
 * ws: bnb_sample_and_solve_ws(s1, s2, n_points, cfg->worklist_capacity) bytes. */
int32_t bnb_sample_and_solve(const bnb_surface *s1, const bnb_surface *s2, const bnb_receiver *rec,
                             const bnb_emitters *em, const bnb_index *index, const float *su, const float *sv,
                             int64_t n_points, const bnb_sample_cfg *cfg, float *E_out,
                             bnb_sample_stats *stats, void *ws, size_t ws_bytes, void *stream);
size_t bnb_sample_and_solve_ws(const bnb_surface *s1, const bnb_surface *s2, int64_t n_points,
                               int64_t worklist_capacity);

/* gamma for a target expected sample count (Sec. 5.4: gamma and E|S| are in one-to-one
 * correspondence, so the sampling density is set by E|S|).  With the selection rule of
 * bnb_sample_and_solve (a 24-bit draw below P = min(gamma (x) E~, 1), product rounded up) a listed
 * tuple is selected with probability exactly ceil(P 2^24) / 2^24, and
 *     E|S|(gamma) = sum over grid cells g of w_g * sum over g's listed tuples of that probability, / W,
 * with w_g the number of shading points (su, sv: device float arrays of n_points >= 1) whose grid
 * cell is g and W = n_points; su = sv = NULL weighs every grid cell once (W = G^2, n_points
 * ignored).  The sum is formed in integers on the device and bisected over the bit patterns of
 * the non-negative finite floats: *gamma_out (device float) receives the smallest gamma with
 * E|S|(gamma) >= target, or FLT_MAX when no gamma reaches it.  Deterministic.  target >= 0.
 * ws: bnb_gamma_for_target_ws(grid_res) bytes (the weights and the bisection state); ~65 small
 * launches on the stream, no host synchronization. */
int32_t bnb_gamma_for_target(const bnb_index *index, const float *su, const float *sv, int64_t n_points,
                             double target, float *gamma_out, void *ws, size_t ws_bytes, void *stream);
size_t bnb_gamma_for_target_ws(int32_t grid_res);

/* ---- Batched rendering pass ------------------------------------------------
 * The paper renders one frame at a time; these calls serve many rendering
 * requests at once.  A job is one request's shading points against one scene
 * whose bound pass and index are already resident on the device.  The job
 * table and the job count are DEVICE memory and every launch is sized from the
 * capacities in bnb_batch_cfg only, so one launch sequence can be captured in a
 * CUDA graph and replayed with a rewritten job table.  The Philox counter is
 * the point's index within its job, so a job's estimate does not depend on
 * which other jobs share the batch; with emitter_on NULL it is bit-identical
 * to bnb_sample_and_solve on that job's points with the job's gamma and seed. */

/* Triangles of s in the packed layout the batched pass reads (80 bytes per
 * triangle: p0, p1, p2, n0, n1, n2 as 18 floats in five 16-byte words).
 * `packed` is a device buffer of bnb_pack_surface_bytes(s) bytes, 16-byte
 * aligned, owned by the caller; it stays valid while the caller keeps it. */
size_t bnb_pack_surface_bytes(const bnb_surface *s);
int32_t bnb_pack_surface(const bnb_surface *s, void *packed, size_t packed_bytes, void *stream);

/* One job of a batch (the table is a device array of these, 8-byte aligned).
 * All pointers are device pointers that stay valid until the batch is done. */
typedef struct bnb_job {
  const void *packed_tris;         /* bnb_pack_surface output of the scene's specular surface */
  int32_t n_tris, n_emitters;
  const float *ex, *ey, *ez, *ei;  /* the scene's emitters (as passed to bnb_bound_tuples) */
  const uint8_t *emitter_on;       /* optional, n_emitters bytes: the job renders the emitters whose byte
                                      is nonzero; the other emitters' tuples are skipped (NULL: all) */
  float rp0[3], re1[3], re2[3];    /* the scene's receiver */
  int32_t grid_res;                /* index of the scene (bnb_build_index output) */
  int32_t kind;                    /* the surface's BNB_REFLECT or BNB_REFRACT */
  float eta;                       /* refraction: the surface's eta */
  int32_t reserved0;               /* 0 */
  const int64_t *offsets;
  const uint64_t *key;
  const float *etilde;
  int64_t index_capacity;
  const float *su, *sv;            /* the request's shading points, n_points each */
  int64_t n_points;
  float gamma;                     /* as bnb_sample_cfg */
  uint32_t reserved;                /* 0 */
  uint64_t seed;
  float *E_out;                    /* n_points estimates */
} bnb_job;

typedef struct bnb_batch_cfg {
  int32_t max_jobs;          /* capacity of the job table (1..65536) */
  int32_t newton_iters;      /* as bnb_sample_cfg */
  int64_t max_points;        /* capacity: sum of the jobs' n_points */
  int64_t worklist_capacity; /* capacity: selected (point, tuple) pairs of the whole batch */
  int32_t polish_iters;
  float tol;
  int32_t block_threads;     /* launch shape of the per-point and per-tuple kernels: 0 = 256, else 64..512, multiple of 32 */
  int32_t blocks_per_sm;     /* resident-grid factor: grids hold at most #SMs x this many blocks (0 = 8; 1..64) */
} bnb_batch_cfg;

/* Runs every job of jobs[0 .. *n_jobs) (device int32, read on the device).
 * Device-side overflows (sum of n_points > max_points, *n_jobs > max_jobs,
 * more selections than worklist_capacity) set *stats->status =
 * BNB_ERR_CAPACITY; stats->counters as bnb_sample_and_solve, summed over the
 * batch; stats->sel_count, sel_point, sel_key and root_u1 are not written.  The caller zeroes status and
 * counters before each batch.  ws: bnb_sample_and_solve_batched_ws(cfg) bytes. */
int32_t bnb_sample_and_solve_batched(const bnb_job *jobs, const int32_t *n_jobs, const bnb_batch_cfg *cfg,
                                     bnb_sample_stats *stats, void *ws, size_t ws_bytes, void *stream);
size_t bnb_sample_and_solve_batched_ws(const bnb_batch_cfg *cfg);

/* ---- Batched bound pass ------------------------------------------------------
 * The precomputation of many scenes in one persistent launch (no counterpart in
 * the paper).  A job is one scene: its packed triangles (bnb_pack_surface), its
 * emitters and receiver, the subdivision depth and its own record outputs.  The
 * job table and the job count are DEVICE memory; the launch is sized by the
 * device's SM count only, so it can be captured in a CUDA graph.  Each cell is
 * bounded by the same cell program as bnb_bound_tuples; jobs take no extra
 * split levels: a cell whose denominator has mixed sign is bounded at once by
 * the reciprocal rule (reflection) or the universal box (refraction), a valid
 * but looser bound than splitting.  Base records land at the job's work index
 * (as in bnb_bound_tuples); the job's *count receives its number of base
 * cells.  The caller zeroes every job's count and status before the call. */
typedef struct bnb_bound_job {
  const void *packed_tris;            /* bnb_pack_surface output of the scene's specular surface */
  const float *ex, *ey, *ez, *ei;     /* the scene's emitters */
  int32_t n_tris, n_emitters;
  int32_t kind, depth;                /* BNB_REFLECT / BNB_REFRACT; base depth 0..10 */
  float eta;                          /* refraction: eta' */
  int32_t irradiance;                 /* as bnb_bound_cfg */
  float rp0[3], re1[3], re2[3];       /* the scene's receiver */
  int32_t reserved;                   /* 0 */
  int64_t capacity;                   /* records the outputs hold: >= n_emitters * n_tris * 4^depth */
  int64_t *count;                     /* device int64 */
  int32_t *status;                    /* device int32 */
  float *u_lo, *u_hi, *v_lo, *v_hi, *e_hi;
  float *e_lo;                        /* optional (NULL: not written) */
  int32_t *emitter, *tri0, *tri1;
  uint32_t *cell, *flags;
} bnb_bound_job;

/* Bounds every base cell of jobs[0 .. *n_jobs) (n_jobs: device int32, at most
 * max_jobs, 1..65536).  ws: bnb_bound_tuples_batched_ws(max_jobs) bytes. */
int32_t bnb_bound_tuples_batched(const bnb_bound_job *jobs, const int32_t *n_jobs, int32_t max_jobs, void *ws,
                                 size_t ws_bytes, void *stream);
size_t bnb_bound_tuples_batched_ws(int32_t max_jobs);

/* Human-readable name of a status code (static string). */
const char *bnb_status_string(int32_t status);

/* Reads and clears the device error word (no counterpart in the paper: the error reporting of this
 * GPU library).  Every kernel that meets a condition only the
 * device can see (BNB_ERR_CAPACITY: an output, split queue, index or worklist too small) raises it
 * both in the status word of its call's output struct and in a device error word that keeps the
 * first code raised since the last read.  This call synchronizes `stream` (all work enqueued on it
 * has finished when it returns), then takes the word with an atomic exchange against 0, so a code
 * raised concurrently is reported either now or by the next call, never lost.  Returns BNB_OK when
 * no kernel raised anything since the last read, the first code raised otherwise, or BNB_ERR_CUDA
 * when the stream itself failed (a launch or fault error).  The word belongs to the CUDA context
 * current on the calling thread, not to the stream: it collects codes from every stream and call
 * in that context, so callers that share a context also share the word.  The per-struct status
 * words are not touched.  Not for use during stream capture (it synchronizes). */
int32_t bnb_stream_status(void *stream);

/* ABI version of this header (increments on any struct or signature change). */
/* Implicit-differentiation irradiance bound (Sec. 4.4 "Implicit differentiation", with the
 * specular polynomials F, G of its footnote) of single-refraction records, on the stream.
 * For every record r < n (n = -1: min(*cells->count, capacity), read on the device) that is
 * BNB_CELL_LIVE with tri1 < 0: the cell's barycentric coordinates and the receiver
 * coordinates of its box [u_lo, u_hi] x [v_lo, v_hi] are independent variables (the 4D
 * superset of the path manifold); |du1/du_k| = |det B| / |det A| with A = d(F,G)/d(u1,v1),
 * B = d(F,G)/d(u_k,v_k), and E = I0 |C1| |det B| / (|d0|^3 |N_k| |det A|) (Eq. eq_dwda) is
 * bounded by coefficient ratios (Eq. eq_bbound) in float64 with tracked rounding error; the
 * tighter of b = (1,0,0) and (0,1,0) is kept, +inf / 0 when neither certifies det A's sign.
 *   mode 0: e_hi (and e_lo when non-NULL) receive the implicit bound, rounded outward;
 *   mode 1: e_hi = min(e_hi, implicit), e_lo = max(e_lo, implicit).
 * Other records are left unchanged.  s1: BNB_REFRACT with eta in (0, 1e6), else
 * BNB_ERR_UNSUPPORTED / BNB_ERR_INVALID.  The records' emitter, tri0, tri1, cell, flags and
 * box arrays must be valid device arrays; record indices outside the scene are skipped.
 * No workspace; one warp per record (48 KB of shared memory per 64-thread block). */
int32_t bnb_implicit_irradiance(const bnb_surface *s1, const bnb_receiver *rec, const bnb_emitters *em,
                                const bnb_cell_bounds *cells, int64_t n, int32_t mode, void *stream);

/* FP32 FMA throughput probe (no counterpart in the paper): the measured denominator of the
 * roofline of the ALU-bound bound kernels.  Launches grid_blocks x block_threads threads
 * (block_threads a multiple of 32, at most 1024) on the stream; each runs `iters` rounds of 16
 * independent FMA chains, as scalar FFMA (paired = 0) or paired FFMA2 (paired = 1, two FMAs per
 * instruction), and writes one float to sink[thread] (device, grid_blocks * block_threads floats,
 * caller-owned) so that no chain is dead code.  FLOPs per launch = grid_blocks * block_threads *
 * iters * 32 * (paired ? 2 : 1).  The caller times it (CUDA events on the stream). */
int32_t bnb_ffma_probe(int32_t grid_blocks, int32_t block_threads, int32_t iters, int32_t paired, float *sink,
                       void *stream);

int32_t bnb_abi_version(void);  /* 11 */

#ifdef __cplusplus
}
#endif

#endif /* BNB_H_ */
