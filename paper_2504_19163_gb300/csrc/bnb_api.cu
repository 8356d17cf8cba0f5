// C ABI of libbnb (declared in include/bnb.h): argument checks, workspace
// layout and the launch sequence of each call.  No call allocates memory or
// synchronizes the stream.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"

namespace bnb {
size_t index_ws_bytes(int32_t G, int64_t pre_cap);
cudaError_t launch_build_index(const bnb_cell_bounds* c, float m, int64_t pre_cap, bnb_index* out, void* ws,
                               cudaStream_t st);
size_t sample_ws_bytes(int64_t n_tris, int64_t n_tris2, int64_t n_points, int64_t wl_cap);
cudaError_t launch_sample_and_solve(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                                    const bnb_emitters* em, const bnb_index* idx, const float* su, const float* sv,
                                    int64_t n_points, const bnb_sample_cfg* cfg, float* E_out,
                                    bnb_sample_stats* stats, void* ws, cudaStream_t st);
size_t pair_ws_bytes(int64_t n_tris1, int64_t n_tris2, int64_t n_base);
cudaError_t launch_bound_pairs(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                               const bnb_emitters* em, int32_t depth, bool fp64, bool irradiance, bnb_cell_bounds* out,
                               void* ws, cudaStream_t st);
cudaError_t launch_implicit(const bnb_surface* s1, const bnb_receiver* rec, const bnb_emitters* em,
                            const bnb_cell_bounds* cells, int64_t n, int32_t mode, cudaStream_t st);
size_t gamma_ws_bytes(int32_t G);
cudaError_t launch_gamma_for_target(const bnb_index* idx, const float* su, const float* sv, int64_t n_points,
                                    double target, float* gamma_out, void* ws, cudaStream_t st);
size_t batch_ws_bytes(const bnb_batch_cfg* c);
size_t bound_batch_ws_bytes(int32_t max_jobs);
cudaError_t launch_bound_batched(const bnb_bound_job* jobs, const int32_t* n_jobs, int32_t max_jobs, void* ws,
                                 cudaStream_t st);
cudaError_t launch_sample_and_solve_batched(const bnb_job* jobs, const int32_t* n_jobs, const bnb_batch_cfg* c,
                                            bnb_sample_stats* stats, void* ws, cudaStream_t st);
}  // namespace bnb

using namespace bnb;

namespace {

constexpr int kMaxBaseDepth = 10;
constexpr int kMaxExtra = 4;

bool surface_ok(const bnb_surface* s) {
  if (!s || s->n_tris < 0 || s->n_verts < 0) return false;
  if (s->n_tris > 0 && (!s->px || !s->py || !s->pz || !s->nx || !s->ny || !s->nz || !s->i0 || !s->i1 || !s->i2))
    return false;
  if (s->n_tris > (1 << 24) - 2) return false;  // tuple key holds 24 bits per triangle index
  return true;
}

bool emitters_ok(const bnb_emitters* e) {
  if (!e || e->n < 0 || e->n > 65535) return false;
  if (e->n > 0 && (!e->x || !e->y || !e->z || !e->intensity)) return false;
  return true;
}

bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

// Two specular vertices: each reflecting, or refracting with eta' in (0, 1e6).
bool vertex_ok(const bnb_surface* s) {
  return s->kind == BNB_REFLECT || (s->kind == BNB_REFRACT && s->eta > 0.0f && s->eta < 1e6f);
}
bool pair_ok(const bnb_surface* s1, const bnb_surface* s2) { return vertex_ok(s1) && vertex_ok(s2); }

int64_t n_base_of(const bnb_surface* s1, const bnb_emitters* em, int depth) {
  return (int64_t)em->n * (int64_t)s1->n_tris * ((int64_t)1 << (2 * depth));
}

int64_t split_queue_cap(int64_t n_base) { return 4096 + n_base / 32; }

int64_t queue_cap(const bnb_bound_cfg* cfg, int64_t n_base) {
  return cfg->split_capacity > 0 ? cfg->split_capacity : split_queue_cap(n_base);
}

// Adaptive-subdivision fields: off (adapt_depth <= depth) or within the cell-id depth limit.
bool adapt_ok(const bnb_bound_cfg* cfg) {
  if (cfg->adapt_depth < 0 || cfg->adapt_depth > kMaxDepth || cfg->split_capacity < 0) return false;
  if (cfg->adapt_depth > cfg->depth && cfg->adapt_depth + cfg->max_extra_split > kMaxDepth) return false;
  return cfg->sigma >= 0.0f && cfg->alpha >= 0.0f;  // NaN fails
}

struct BoundWs {
  float4* tri;
  SplitItem* q[2];
  int64_t* qcount;  // [2]
  size_t bytes;
};

BoundWs carve_bound_ws(void* base, int64_t n_tris, int64_t qcap) {
  BoundWs w{};
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  w.tri = (float4*)take((size_t)n_tris * kTriF4 * sizeof(float4));
  w.q[0] = (SplitItem*)take((size_t)qcap * sizeof(SplitItem));
  w.q[1] = (SplitItem*)take((size_t)qcap * sizeof(SplitItem));
  w.qcount = (int64_t*)take(2 * sizeof(int64_t));
  w.bytes = o;
  return w;
}

}  // namespace

extern "C" {

int32_t bnb_abi_version(void) { return 11; }

const char* bnb_status_string(int32_t s) {
  switch (s) {
    case BNB_OK: return "ok";
    case BNB_ERR_INVALID: return "invalid argument";
    case BNB_ERR_CAPACITY: return "output or workspace capacity exceeded";
    case BNB_ERR_CUDA: return "CUDA launch error";
    case BNB_ERR_UNSUPPORTED: return "unsupported configuration";
    case BNB_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

size_t bnb_bound_tuples_ws(const bnb_surface* s1, const bnb_surface* s2, const bnb_emitters* em,
                           const bnb_bound_cfg* cfg) {
  if (!surface_ok(s1) || !emitters_ok(em) || !cfg || cfg->depth < 0 || cfg->depth > kMaxBaseDepth) return 0;
  if (cfg->split_capacity < 0) return 0;
  const int64_t nb = n_base_of(s1, em, cfg->depth);
  if (s2 != nullptr) return surface_ok(s2) ? pair_ws_bytes(s1->n_tris, s2->n_tris, nb) : 0;
  return carve_bound_ws(nullptr, s1->n_tris, queue_cap(cfg, nb)).bytes;
}

int32_t bnb_bound_tuples(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                         const bnb_emitters* em, const bnb_bound_cfg* cfg, bnb_cell_bounds* out, void* ws,
                         size_t ws_bytes, void* stream) {
  if (!surface_ok(s1) || !emitters_ok(em) || !rec || !cfg || !out) return BNB_ERR_INVALID;
  if (s2 != nullptr) {
    if (!surface_ok(s2)) return BNB_ERR_INVALID;
    if (!pair_ok(s1, s2)) return BNB_ERR_UNSUPPORTED;
    if (cfg->depth < 0 || cfg->depth > kMaxBaseDepth) return BNB_ERR_INVALID;
    if (!out->count || !out->status || out->capacity < 0) return BNB_ERR_INVALID;
    if (out->capacity > 0 && (!out->u_lo || !out->u_hi || !out->v_lo || !out->v_hi || !out->e_hi ||
                              !out->emitter || !out->tri0 || !out->tri1 || !out->cell || !out->flags))
      return BNB_ERR_INVALID;
    const int64_t nb = n_base_of(s1, em, cfg->depth);
    const size_t need = pair_ws_bytes(s1->n_tris, s2->n_tris, nb);
    if (ws_bytes < need || (need > 0 && (!ws || !aligned256(ws)))) return BNB_ERR_INVALID;
    out->n_base = 0;  // records are not in base-cell order: every record is indexed on its own
    out->depth = 0;
    out->n_emitters = em->n;
    out->n_tris = s1->n_tris;
    if (cfg->irradiance < 0 || cfg->irradiance > 1) return BNB_ERR_INVALID;
    return launch_bound_pairs(s1, s2, rec, em, cfg->depth, cfg->fp64 != 0, cfg->irradiance != 0, out, ws,
                              (cudaStream_t)stream) ==
                   cudaSuccess
               ? BNB_OK
               : BNB_ERR_CUDA;
  }
  if (s1->kind != BNB_REFLECT && s1->kind != BNB_REFRACT) return BNB_ERR_INVALID;
  if (s1->kind == BNB_REFRACT && !(s1->eta > 0.0f && s1->eta < 1e6f)) return BNB_ERR_INVALID;
  if (cfg->irradiance < 0 || cfg->irradiance > 2) return BNB_ERR_INVALID;
  if (cfg->irradiance == 2 && s1->kind != BNB_REFRACT) return BNB_ERR_UNSUPPORTED;
  if (cfg->block_threads != 0 && cfg->block_threads != 128 && cfg->block_threads != 256 &&
      cfg->block_threads != 320 && cfg->block_threads != 384)
    return BNB_ERR_INVALID;
  if (cfg->depth < 0 || cfg->depth > kMaxBaseDepth || cfg->max_extra_split < 0 || cfg->max_extra_split > kMaxExtra ||
      cfg->depth + cfg->max_extra_split > kMaxDepth || !adapt_ok(cfg))
    return BNB_ERR_INVALID;
  const int64_t nb = n_base_of(s1, em, cfg->depth);
  if (!out->count || !out->status) return BNB_ERR_INVALID;
  if (out->capacity < nb) return BNB_ERR_INVALID;
  if (out->capacity > 0 && (!out->u_lo || !out->u_hi || !out->v_lo || !out->v_hi || !out->e_hi ||
                            !out->emitter || !out->tri0 || !out->tri1 || !out->cell || !out->flags))
    return BNB_ERR_INVALID;
  const int64_t qcap = queue_cap(cfg, nb);
  const BoundWs need = carve_bound_ws(nullptr, s1->n_tris, qcap);
  if (ws_bytes < need.bytes || (need.bytes > 0 && (!ws || !aligned256(ws)))) return BNB_ERR_INVALID;
  out->n_base = nb;
  out->depth = cfg->depth;
  out->n_emitters = em->n;
  out->n_tris = s1->n_tris;
  if (nb == 0) return BNB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  BoundWs w = carve_bound_ws(ws, s1->n_tris, qcap);
  if (launch_pack_tris(s1, w.tri, st) != cudaSuccess) return BNB_ERR_CUDA;
  if (cudaMemsetAsync(w.qcount, 0, 2 * sizeof(int64_t), st) != cudaSuccess) return BNB_ERR_CUDA;
  BoundParams P{};
  P.tri = w.tri;
  P.n_tris = s1->n_tris;
  P.n_emitters = em->n;
  P.ex = em->x;
  P.ey = em->y;
  P.ez = em->z;
  P.ei = em->intensity;
  for (int c = 0; c < 3; ++c) {
    P.rp0[c] = rec->p0[c];
    P.re1[c] = rec->e1[c];
    P.re2[c] = rec->e2[c];
  }
  P.depth = cfg->depth;
  P.block_threads = cfg->block_threads;
  const bool adaptive = cfg->adapt_depth > cfg->depth;
  P.adapt_depth = adaptive ? cfg->adapt_depth : 0;
  P.sigma = cfg->sigma;
  P.alpha = cfg->alpha;
  // sign-test splits may go max_extra_split levels below the deepest adaptive level
  P.max_depth = (adaptive ? cfg->adapt_depth : cfg->depth) + cfg->max_extra_split;
  P.irradiance = cfg->irradiance ? 1 : 0;
  P.kind = s1->kind;
  P.eta = s1->eta;
  P.n_base = nb;
  P.capacity = out->capacity;
  P.count = out->count;
  P.status = out->status;
  P.u_lo = out->u_lo;
  P.u_hi = out->u_hi;
  P.v_lo = out->v_lo;
  P.v_hi = out->v_hi;
  P.e_lo = out->e_lo;
  P.e_hi = out->e_hi;
  P.emitter = out->emitter;
  P.tri0 = out->tri0;
  P.tri1 = out->tri1;
  P.cell = out->cell;
  P.flags = out->flags;
  P.e_hi_min = out->e_hi_min;
  P.q_cap = qcap;
  P.q_out = w.q[0];
  P.q_out_count = w.qcount + 0;
  const bool fp64 = cfg->fp64 != 0;
  if (launch_bound_base(P, fp64, st) != cudaSuccess) return BNB_ERR_CUDA;
  for (int lvl = 0; lvl < P.max_depth - cfg->depth; ++lvl) {
    const int cur = lvl & 1, nxt = cur ^ 1;
    if (cudaMemsetAsync(w.qcount + nxt, 0, sizeof(int64_t), st) != cudaSuccess) return BNB_ERR_CUDA;
    P.q_out = w.q[nxt];
    P.q_out_count = w.qcount + nxt;
    if (launch_bound_split(P, w.q[cur], w.qcount + cur, fp64, st) != cudaSuccess) return BNB_ERR_CUDA;
  }
  // implicit differentiation: intersect each live record's bound with the implicit one
  if (cfg->irradiance == 2 && launch_implicit(s1, rec, em, out, -1, 1, st) != cudaSuccess) return BNB_ERR_CUDA;
  return BNB_OK;
}

int32_t bnb_implicit_irradiance(const bnb_surface* s1, const bnb_receiver* rec, const bnb_emitters* em,
                                const bnb_cell_bounds* cells, int64_t n, int32_t mode, void* stream) {
  if (!surface_ok(s1) || !emitters_ok(em) || !rec || !cells) return BNB_ERR_INVALID;
  if (s1->kind != BNB_REFRACT) return BNB_ERR_UNSUPPORTED;
  if (!(s1->eta > 0.0f && s1->eta < 1e6f)) return BNB_ERR_INVALID;
  if (mode != 0 && mode != 1) return BNB_ERR_INVALID;
  if (n < -1 || n > cells->capacity || (n < 0 && !cells->count)) return BNB_ERR_INVALID;
  if (n == 0 || cells->capacity == 0) return BNB_OK;
  if (!cells->u_lo || !cells->u_hi || !cells->v_lo || !cells->v_hi || !cells->e_hi || !cells->emitter ||
      !cells->tri0 || !cells->tri1 || !cells->cell || !cells->flags)
    return BNB_ERR_INVALID;
  return launch_implicit(s1, rec, em, cells, n, mode, (cudaStream_t)stream) == cudaSuccess ? BNB_OK : BNB_ERR_CUDA;
}

size_t bnb_build_index_ws(const bnb_cell_bounds* cells, int32_t grid_res, int64_t pre_capacity) {
  (void)cells;
  if (grid_res < 1 || grid_res > 4096 || pre_capacity < 0) return 0;
  return index_ws_bytes(grid_res, pre_capacity);
}

int32_t bnb_build_index(const bnb_cell_bounds* cells, float m, int64_t pre_capacity, bnb_index* out, void* ws,
                        size_t ws_bytes, void* stream) {
  if (!cells || !out || !cells->count) return BNB_ERR_INVALID;
  if (out->grid_res < 1 || out->grid_res > 4096 || !out->count || !out->status || !out->offsets) return BNB_ERR_INVALID;
  if (out->capacity < 0 || (out->capacity > 0 && (!out->key || !out->etilde))) return BNB_ERR_INVALID;
  if (pre_capacity < 0 || !(m >= 0.0f)) return BNB_ERR_INVALID;
  if (cells->depth < 0 || cells->depth > kMaxBaseDepth || cells->n_base < 0) return BNB_ERR_INVALID;
  if (cells->n_base % ((int64_t)1 << (2 * cells->depth)) != 0) return BNB_ERR_INVALID;
  if (cells->n_base > 0 && (!cells->u_lo || !cells->u_hi || !cells->v_lo || !cells->v_hi || !cells->e_hi ||
                            !cells->emitter || !cells->tri0 || !cells->tri1 || !cells->flags))
    return BNB_ERR_INVALID;
  const size_t need = index_ws_bytes(out->grid_res, pre_capacity);
  if (ws_bytes < need || !ws || !aligned256(ws)) return BNB_ERR_INVALID;
  return launch_build_index(cells, m, pre_capacity, out, ws, (cudaStream_t)stream) == cudaSuccess ? BNB_OK
                                                                                                  : BNB_ERR_CUDA;
}

size_t bnb_sample_and_solve_ws(const bnb_surface* s1, const bnb_surface* s2, int64_t n_points,
                               int64_t worklist_capacity) {
  if (!surface_ok(s1) || (s2 && !surface_ok(s2)) || n_points < 0 || worklist_capacity < 0) return 0;
  return sample_ws_bytes(s1->n_tris, s2 ? s2->n_tris : 0, n_points, worklist_capacity);
}

int32_t bnb_sample_and_solve(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                             const bnb_emitters* em, const bnb_index* index, const float* su, const float* sv,
                             int64_t n_points, const bnb_sample_cfg* cfg, float* E_out, bnb_sample_stats* stats,
                             void* ws, size_t ws_bytes, void* stream) {
  if (!surface_ok(s1) || !emitters_ok(em) || !rec || !index || !cfg || !stats) return BNB_ERR_INVALID;
  if (s2 != nullptr && !surface_ok(s2)) return BNB_ERR_INVALID;
  if (s2 != nullptr && !pair_ok(s1, s2)) return BNB_ERR_UNSUPPORTED;
  if (s1->kind != BNB_REFLECT && s1->kind != BNB_REFRACT) return BNB_ERR_INVALID;
  if (s1->kind == BNB_REFRACT && !(s1->eta > 0.0f && s1->eta < 1e6f)) return BNB_ERR_INVALID;
  if (n_points < 0 || (n_points > 0 && (!su || !sv || !E_out))) return BNB_ERR_INVALID;
  if (!stats->counters || !stats->status || !index->offsets) return BNB_ERR_INVALID;
  if (index->grid_res < 1 || index->grid_res > 4096) return BNB_ERR_INVALID;
  if (cfg->worklist_capacity < 0 || cfg->newton_iters < 0 || cfg->newton_iters > 64 || cfg->polish_iters < 0 ||
      cfg->polish_iters > 8 || !(cfg->gamma >= 0.0f) || !(cfg->tol > 0.0f) || (cfg->bins != 0 && cfg->bins != 1) ||
      cfg->stoc_trials < 0 || cfg->stoc_trials > (1 << 20))
    return BNB_ERR_INVALID;
  if (s2 != nullptr && cfg->stoc_trials > 0) return BNB_ERR_UNSUPPORTED;
  const size_t need = sample_ws_bytes(s1->n_tris, s2 ? s2->n_tris : 0, n_points, cfg->worklist_capacity);
  if (ws_bytes < need || !ws || !aligned256(ws)) return BNB_ERR_INVALID;
  return launch_sample_and_solve(s1, s2, rec, em, index, su, sv, n_points, cfg, E_out, stats, ws,
                                 (cudaStream_t)stream) == cudaSuccess
             ? BNB_OK
             : BNB_ERR_CUDA;
}

size_t bnb_gamma_for_target_ws(int32_t grid_res) {
  if (grid_res < 1 || grid_res > 4096) return 0;
  return gamma_ws_bytes(grid_res);
}

int32_t bnb_gamma_for_target(const bnb_index* index, const float* su, const float* sv, int64_t n_points,
                             double target, float* gamma_out, void* ws, size_t ws_bytes, void* stream) {
  if (!index || !gamma_out || !index->offsets) return BNB_ERR_INVALID;
  if (index->grid_res < 1 || index->grid_res > 4096 || index->capacity < 0) return BNB_ERR_INVALID;
  if (index->capacity > 0 && !index->etilde) return BNB_ERR_INVALID;
  if (!(target >= 0.0) || !(target < 1e300)) return BNB_ERR_INVALID;  // NaN fails
  if ((su == nullptr) != (sv == nullptr) || n_points < 0) return BNB_ERR_INVALID;
  if (su != nullptr && n_points == 0) return BNB_ERR_INVALID;
  const size_t need = gamma_ws_bytes(index->grid_res);
  if (ws_bytes < need || !ws || !aligned256(ws)) return BNB_ERR_INVALID;
  return launch_gamma_for_target(index, su, sv, n_points, target, gamma_out, ws, (cudaStream_t)stream) ==
                 cudaSuccess
             ? BNB_OK
             : BNB_ERR_CUDA;
}

size_t bnb_pack_surface_bytes(const bnb_surface* s) {
  if (!surface_ok(s)) return 0;
  return (size_t)s->n_tris * kTriF4 * sizeof(float4);
}

int32_t bnb_pack_surface(const bnb_surface* s, void* packed, size_t packed_bytes, void* stream) {
  if (!surface_ok(s)) return BNB_ERR_INVALID;
  const size_t need = (size_t)s->n_tris * kTriF4 * sizeof(float4);
  if (packed_bytes < need || (need > 0 && (!packed || ((uintptr_t)packed & 15u) != 0))) return BNB_ERR_INVALID;
  if (need == 0) return BNB_OK;
  return launch_pack_tris(s, (float4*)packed, (cudaStream_t)stream) == cudaSuccess ? BNB_OK : BNB_ERR_CUDA;
}

static bool batch_cfg_ok(const bnb_batch_cfg* c) {
  if (!c) return false;
  if (c->max_jobs < 1 || c->max_jobs > 65536 || c->max_points < 0 || c->worklist_capacity < 0) return false;
  if (c->newton_iters < 0 || c->newton_iters > 64 || c->polish_iters < 0 || c->polish_iters > 8) return false;
  if (!(c->tol > 0.0f)) return false;
  if (c->block_threads != 0 && (c->block_threads < 64 || c->block_threads > 512 || c->block_threads % 32 != 0))
    return false;
  if (c->blocks_per_sm < 0 || c->blocks_per_sm > 64) return false;
  return true;
}

size_t bnb_sample_and_solve_batched_ws(const bnb_batch_cfg* cfg) {
  if (!batch_cfg_ok(cfg)) return 0;
  return batch_ws_bytes(cfg);
}

int32_t bnb_sample_and_solve_batched(const bnb_job* jobs, const int32_t* n_jobs, const bnb_batch_cfg* cfg,
                                     bnb_sample_stats* stats, void* ws, size_t ws_bytes, void* stream) {
  if (!jobs || !n_jobs || !batch_cfg_ok(cfg) || !stats || !stats->counters || !stats->status) return BNB_ERR_INVALID;
  if (((uintptr_t)jobs & 7u) != 0) return BNB_ERR_INVALID;
  const size_t need = batch_ws_bytes(cfg);
  if (ws_bytes < need || !ws || !aligned256(ws)) return BNB_ERR_INVALID;
  return launch_sample_and_solve_batched(jobs, n_jobs, cfg, stats, ws, (cudaStream_t)stream) == cudaSuccess
             ? BNB_OK
             : BNB_ERR_CUDA;
}

size_t bnb_bound_tuples_batched_ws(int32_t max_jobs) {
  if (max_jobs < 1 || max_jobs > 65536) return 0;
  return bound_batch_ws_bytes(max_jobs);
}

int32_t bnb_bound_tuples_batched(const bnb_bound_job* jobs, const int32_t* n_jobs, int32_t max_jobs, void* ws,
                                 size_t ws_bytes, void* stream) {
  if (!jobs || !n_jobs || max_jobs < 1 || max_jobs > 65536) return BNB_ERR_INVALID;
  if (((uintptr_t)jobs & 7u) != 0) return BNB_ERR_INVALID;
  if (ws_bytes < bound_batch_ws_bytes(max_jobs) || !ws || !aligned256(ws)) return BNB_ERR_INVALID;
  return launch_bound_batched(jobs, n_jobs, max_jobs, ws, (cudaStream_t)stream) == cudaSuccess ? BNB_OK
                                                                                               : BNB_ERR_CUDA;
}

}  // extern "C"
