// Sample and solve kernels: the rendering pass (Sec. 5, Algorithm 1; Sec. 6.1
// "Root-finding").
//
//   sample_k (count)  per shading point: grid cell of (u,v), then for every
//                     listed tuple P = min(gamma E~, 1) (float32 product rounded
//                     up, so P > 0 whenever E~ > 0) and one Philox4x32-10
//                     uniform r (key = seed, counter = (point, tuple key));
//                     the tuple is selected when r < P.  Counts per point.  With
//                     bins = 1, the bin-packed form (Sec. 5.3): the list is
//                     packed greedily into groups of probability sum <= 1 and
//                     one draw per group selects at most one of its tuples.
//   scan              -> worklist offsets (point order, then key order).
//   (bins = 0 and long lists: sample_warp_k, the same with a warp per point)
//   sample_k (fill)   the same selections, writing (point, key, P): the count pass keeps
//                     the list positions of a point's first kSelCache selections,
//                     so only points with more selections walk their list again.
//   solve32_k         per selected tuple: Newton's method in T1's barycentric
//                     coordinates from the centroid (deterministic init), float32
//                     damped steps; tuples left with a possible root are listed.
//   polish_k          per listed tuple: float64 polish steps, acceptance tests,
//                     contribution E(root) / P.
//   (pair tuples, s2 given: solve32_pair_k / polish_pair_k through the two-vertex
//    chain x0 -> T1 -> T2 -> receiver, Newton in T1's barycentric coordinates)
//   reduce_k          per point, contributions summed in worklist order.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"
#include "bnb_path.cuh"

namespace bnb {

struct SampleParams {
  const int64_t* offsets;
  const uint64_t* key;
  const float* etilde;
  int64_t index_capacity;
  int32_t G;
  const float *su, *sv;
  int64_t n_points;
  float gamma;
  uint64_t seed;
  int64_t* n_sel;      // per point
  const int64_t* woff; // per point + 1 (fill pass)
  int64_t wl_cap;
  int64_t* wl_point;
  uint64_t* wl_key;
  float* wl_p;
  int64_t* counters;   // device int64[4]
  int32_t* status;
  int32_t* sel_count;  // optional, per point
  int64_t* sel_point;  // optional, per selection (worklist order)
  uint64_t* sel_key;   // optional, per selection
  int32_t bins;        // 1: bin-packed selection (one draw per group), 0: one draw per tuple
  int32_t* sel_cache;  // [kSelCache][n_points]: list positions (from the cell's start) of the selections
};

constexpr int kSelCache = 8;

template <bool FILL>
__global__ void __launch_bounds__(256) sample_k(SampleParams P, const int32_t* __restrict__ mode) {
  if (!P.bins && *mode != 0) return;  // the long-list form runs instead (sample_warp_k)
  long long nu = 0, ns = 0, nb = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n_points;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int g = grid_col_s(P.sv[p], P.G) * P.G + grid_col_s(P.su[p], P.G);
    const int64_t s = P.offsets[g];
    const int64_t e = min(P.offsets[g + 1], P.index_capacity);
    int64_t cnt = 0;
    int64_t out = FILL ? P.woff[p] : 0;
    if (FILL) {
      const int64_t c = P.n_sel[p];
      if (c <= kSelCache) {  // the count pass kept every selection's list position
        for (int q = 0; q < (int)c; ++q) {
          const int64_t j = s + P.sel_cache[(int64_t)q * P.n_points + p];
          const uint64_t k = P.key[j];
          if (out < P.wl_cap) {
            P.wl_point[out] = p;
            P.wl_key[out] = k;
            P.wl_p[out] = fminf(__fmul_ru(P.gamma, P.etilde[j]), 1.0f);
            if (P.sel_point) P.sel_point[out] = p;
            if (P.sel_key) P.sel_key[out] = k;
          } else {
            raise_status(P.status, BNB_ERR_CAPACITY);
          }
          ++out;
        }
        continue;
      }
    }
    // bins: the current group's running probability sum and draw (groups are runs of the list)
    float acc = 0.0f, rb = 0.0f;
    bool open = false;
    for (int64_t j = s; j < e; ++j) {
      const float Pt = fminf(__fmul_ru(P.gamma, P.etilde[j]), 1.0f);
      const uint64_t k = P.key[j];
      bool sel;
      if (P.bins) {
        if (!open || __fadd_rn(acc, Pt) > 1.0f) {  // the tuple does not fit: it opens the next group
          open = true;
          acc = 0.0f;
          rb = uniform24(P.seed, p, k);
          ++nb;
        }
        const float lo = acc;
        acc = __fadd_rn(acc, Pt);
        sel = rb >= lo && rb < acc;
      } else {
        sel = uniform24(P.seed, p, k) < Pt;
      }
      if (sel) {
        if (FILL) {
          if (out < P.wl_cap) {
            P.wl_point[out] = p;
            P.wl_key[out] = k;
            P.wl_p[out] = Pt;
            if (P.sel_point) P.sel_point[out] = p;
            if (P.sel_key) P.sel_key[out] = k;
          } else {
            raise_status(P.status, BNB_ERR_CAPACITY);
          }
          ++out;
        } else if (cnt < kSelCache) {
          P.sel_cache[cnt * P.n_points + p] = (int32_t)(j - s);
        }
        ++cnt;
      }
    }
    if (!FILL) {
      P.n_sel[p] = cnt;
      if (P.sel_count) P.sel_count[p] = (int32_t)cnt;
    }
    nu += (e > s ? e - s : 0);
    ns += cnt;
  }
  if (!FILL) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nu += __shfl_xor_sync(0xffffffffu, nu, o);
      ns += __shfl_xor_sync(0xffffffffu, ns, o);
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (nu) atomicAdd((unsigned long long*)&P.counters[0], (unsigned long long)nu);
      if (ns) atomicAdd((unsigned long long*)&P.counters[1], (unsigned long long)ns);
      if (nb) atomicAdd((unsigned long long*)&P.counters[3], (unsigned long long)nb);
    }
  }
}

// One draw per listed tuple (bins = 0) with a warp per shading point, for long lists: lane l
// takes list entries l, l + 32, ... (coalesced loads, 32 draws at once); a ballot per 32 entries
// keeps the selections in list order, so the counts, the kept positions and the worklist are
// those of sample_k.  *mode (set by sample_mode_k) picks this kernel or sample_k; the other one
// returns at once.
constexpr int kLongList = 32;  // mean entries per grid cell from which the warp form runs

__global__ void sample_mode_k(const int64_t* __restrict__ offsets, int32_t G, int64_t capacity,
                              int32_t* __restrict__ mode) {
  const int64_t cells = (int64_t)G * G;
  const int64_t entries = min(offsets[cells], capacity);
  *mode = entries >= (int64_t)kLongList * cells ? 1 : 0;
}

template <bool FILL>
__global__ void __launch_bounds__(256) sample_warp_k(SampleParams P, const int32_t* __restrict__ mode) {
  if (*mode == 0) return;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  long long nu = 0, ns = 0;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); p < P.n_points; p += warps) {
    const int g = grid_col_s(P.sv[p], P.G) * P.G + grid_col_s(P.su[p], P.G);
    const int64_t s = P.offsets[g];
    const int64_t e = min(P.offsets[g + 1], P.index_capacity);
    int64_t out = FILL ? P.woff[p] : 0;
    if (FILL) {
      const int64_t c = P.n_sel[p];
      if (c <= kSelCache) {  // the count pass kept every selection's list position
        if (lane < (int)c) {
          const int64_t j = s + P.sel_cache[(int64_t)lane * P.n_points + p];
          const uint64_t k = P.key[j];
          const int64_t o = out + lane;
          if (o < P.wl_cap) {
            P.wl_point[o] = p;
            P.wl_key[o] = k;
            P.wl_p[o] = fminf(__fmul_ru(P.gamma, P.etilde[j]), 1.0f);
            if (P.sel_point) P.sel_point[o] = p;
            if (P.sel_key) P.sel_key[o] = k;
          } else {
            raise_status(P.status, BNB_ERR_CAPACITY);
          }
        }
        continue;
      }
    }
    int64_t cnt = 0;
    for (int64_t j0 = s; j0 < e; j0 += 32) {
      const int64_t j = j0 + lane;
      bool sel = false;
      float Pt = 0.0f;
      uint64_t k = 0;
      if (j < e) {
        Pt = fminf(__fmul_ru(P.gamma, P.etilde[j]), 1.0f);
        k = P.key[j];
        sel = uniform24(P.seed, p, k) < Pt;
      }
      const unsigned m = __ballot_sync(0xffffffffu, sel);
      if (sel) {
        const int64_t rank = cnt + __popc(m & below);
        if (FILL) {
          const int64_t o = out + rank;
          if (o < P.wl_cap) {
            P.wl_point[o] = p;
            P.wl_key[o] = k;
            P.wl_p[o] = Pt;
            if (P.sel_point) P.sel_point[o] = p;
            if (P.sel_key) P.sel_key[o] = k;
          } else {
            raise_status(P.status, BNB_ERR_CAPACITY);
          }
        } else if (rank < kSelCache) {
          P.sel_cache[rank * P.n_points + p] = (int32_t)(j - s);
        }
      }
      cnt += __popc(m);
    }
    if (!FILL && lane == 0) {
      P.n_sel[p] = cnt;
      if (P.sel_count) P.sel_count[p] = (int32_t)cnt;
      nu += (e > s ? e - s : 0);
      ns += cnt;
    }
  }
  if (!FILL) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nu += __shfl_xor_sync(0xffffffffu, nu, o);
      ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if (lane == 0) {
      if (nu) atomicAdd((unsigned long long*)&P.counters[0], (unsigned long long)nu);
      if (ns) atomicAdd((unsigned long long*)&P.counters[1], (unsigned long long)ns);
    }
  }
}

struct SolveParams {
  const float4* tri;
  int32_t n_tris, n_emitters;
  const float *ex, *ey, *ez, *ei;
  float rp0[3], re1[3], re2[3];
  const float *su, *sv;
  const int64_t* wl_point;
  const uint64_t* wl_key;
  const float* wl_p;
  const int64_t* n_wl;  // device: selections
  int64_t wl_cap;
  int32_t newton_iters, polish_iters;
  float tol;
  float eta;  // refraction: eta'
  int32_t stoc_trials;  // > 0: stochastic starts with the reciprocal weighting, capped at this count
  uint64_t seed;
  // pair tuples (s2 given): T2's packed triangles and eta'
  const float4* tri2;
  int32_t n_tris2;
  float eta2;
  int32_t kind1, kind2;
  float* contrib;
  int64_t* counters;
  double* root_u1;  // optional: (u, v) of the accepted root per selection, NaN when none
  // tuples handed from the float32 phase to the float64 polish
  int64_t* pl_count;
  int64_t* pl_idx;
  float *pl_u, *pl_v;
};

__device__ __forceinline__ void put_root(const SolveParams& S, int64_t i, double u, double v) {
  if (S.root_u1) {
    S.root_u1[2 * i] = u;
    S.root_u1[2 * i + 1] = v;
  }
}

__device__ __forceinline__ void put_no_root(const SolveParams& S, int64_t i) {
  put_root(S, i, __longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
}

// float32 Newton phase over every selection: contributions of the tuples without an admissible
// root are 0 now; the others go to the polish list with their float32 root.
template <bool REFRACT>
__global__ void __launch_bounds__(256) solve32_k(SolveParams S) {
  const int64_t n = min(*S.n_wl, S.wl_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = S.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    bool need = false;
    float u = 0.0f, v = 0.0f;
    if (t < S.n_tris && e < S.n_emitters) {  // a key from another scene has no path and reads nothing
      float pf[3][3], nf[3][3];
      load_tri_s(S.tri, t, pf, nf);
      const float x0[3] = {__ldg(S.ex + e), __ldg(S.ey + e), __ldg(S.ez + e)};
      const int64_t pt = S.wl_point[i];
      need = newton32<REFRACT>(pf, nf, x0, __ldg(S.ei + e), S.rp0, S.re1, S.re2, S.su[pt], S.sv[pt], S.newton_iters,
                               S.eta, u, v);
    }
    if (!need) {
      S.contrib[i] = 0.0f;
      put_no_root(S, i);
    }
    const int64_t j = warp_append(need, S.pl_count);
    if (need) {
      S.pl_idx[j] = i;
      S.pl_u[j] = u;
      S.pl_v[j] = v;
    }
  }
}

// float64 polish of the listed tuples, acceptance tests, contribution E(root) / P.
template <bool REFRACT>
__global__ void __launch_bounds__(256) polish_k(SolveParams S) {
  const int64_t n = *S.pl_count;
  long long roots = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = S.pl_idx[j];
    const uint64_t k = S.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    float pf[3][3], nf[3][3];
    load_tri_s(S.tri, t, pf, nf);
    const float x0[3] = {__ldg(S.ex + e), __ldg(S.ey + e), __ldg(S.ez + e)};
    const int64_t pt = S.wl_point[i];
    double ur = 0.0, vr = 0.0;
    const double E = polish64<REFRACT>(pf, nf, x0, __ldg(S.ei + e), S.rp0, S.re1, S.re2, S.su[pt], S.sv[pt],
                                       S.polish_iters, S.tol, S.eta, S.pl_u[j], S.pl_v[j], &ur, &vr);
    float c = 0.0f;
    if (E >= 0.0) {
      c = (float)(E / (double)S.wl_p[i]);
      ++roots;
      put_root(S, i, ur, vr);
    } else {
      put_no_root(S, i);
    }
    S.contrib[i] = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd((unsigned long long*)&S.counters[2], (unsigned long long)roots);
}

// Stochastic starts with the reciprocal weighting (Sec. 6.1 "Stoc"): per selected tuple, Newton from
// a uniform random start (the float32 phase and the float64 polish); an accepted root u* is weighted
// by the number N of further random starts up to the first whose accepted root lies within 1e-4 of
// u* (geometric, mean 1 / P(reach u*)), N capped at stoc_trials.  contrib = E(u*) N / P.
template <bool REFRACT>
__global__ void __launch_bounds__(256) solve_stoc_k(SolveParams S) {
  const int64_t n = min(*S.n_wl, S.wl_cap);
  long long roots = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = S.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    float c = 0.0f;
    if (t < S.n_tris && e < S.n_emitters) {
      float pf[3][3], nf[3][3];
      load_tri_s(S.tri, t, pf, nf);
      const float x0[3] = {__ldg(S.ex + e), __ldg(S.ey + e), __ldg(S.ez + e)};
      const float I0 = __ldg(S.ei + e);
      const int64_t pt = S.wl_point[i];
      const float tu = S.su[pt], tv = S.sv[pt];
      auto solve_from = [&](int trial, double& ur, double& vr) -> double {
        float u, v;
        stoc_start(S.seed, pt, k, trial, u, v);
        if (!newton32_from<REFRACT>(pf, nf, x0, I0, S.rp0, S.re1, S.re2, tu, tv, S.newton_iters, S.eta, u, v))
          return -1.0;
        return polish64<REFRACT>(pf, nf, x0, I0, S.rp0, S.re1, S.re2, tu, tv, S.polish_iters, S.tol, S.eta, u, v,
                                 &ur, &vr);
      };
      double ur = 0.0, vr = 0.0;
      const double E = solve_from(0, ur, vr);
      if (E >= 0.0) {
        int nw = 1;
        for (; nw < S.stoc_trials; ++nw) {
          double u2 = 0.0, v2 = 0.0;
          const double E2 = solve_from(nw, u2, v2);
          if (E2 >= 0.0 && fabs(u2 - ur) <= 1e-4 && fabs(v2 - vr) <= 1e-4) break;
        }
        c = (float)(E * (double)nw / (double)S.wl_p[i]);
        ++roots;
        put_root(S, i, ur, vr);
      } else {
        put_no_root(S, i);
      }
    } else {
      put_no_root(S, i);
    }
    S.contrib[i] = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd((unsigned long long*)&S.counters[2], (unsigned long long)roots);
}

// Pair tuples (key tri1 >= 0): the same two phases through the two-vertex chain.
__device__ __forceinline__ bool pair_geom(const SolveParams& S, uint64_t k, PairGeom& G) {
  const int e = (int)(k >> 48), t1 = (int)(k & 0xFFFFFFull), t2 = (int)((k >> 24) & 0xFFFFFFull) - 1;
  if (t1 >= S.n_tris || t2 < 0 || t2 >= S.n_tris2 || e >= S.n_emitters) return false;
  load_tri_s(S.tri, t1, G.p1, G.n1);
  load_tri_s(S.tri2, t2, G.p2, G.n2);
  G.x0[0] = __ldg(S.ex + e);
  G.x0[1] = __ldg(S.ey + e);
  G.x0[2] = __ldg(S.ez + e);
  G.I0 = __ldg(S.ei + e);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    G.rp0[c] = S.rp0[c];
    G.re1[c] = S.re1[c];
    G.re2[c] = S.re2[c];
  }
  G.eta1 = S.eta;
  G.eta2 = S.eta2;
  G.kind1 = S.kind1;
  G.kind2 = S.kind2;
  return true;
}

__global__ void __launch_bounds__(256) solve32_pair_k(SolveParams S) {
  const int64_t n = min(*S.n_wl, S.wl_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    PairGeom G;
    bool need = false;
    float u = 0.0f, v = 0.0f;
    if (pair_geom(S, S.wl_key[i], G)) {
      const int64_t pt = S.wl_point[i];
      need = newton32_pair(G, S.su[pt], S.sv[pt], S.newton_iters, u, v);
    }
    if (!need) {
      S.contrib[i] = 0.0f;
      put_no_root(S, i);
    }
    const int64_t j = warp_append(need, S.pl_count);
    if (need) {
      S.pl_idx[j] = i;
      S.pl_u[j] = u;
      S.pl_v[j] = v;
    }
  }
}

// Two blocks per SM (128 registers): more warps on the float64 chain polish than one block at 233.
__global__ void __launch_bounds__(256, 2) polish_pair_k(SolveParams S) {
  const int64_t n = *S.pl_count;
  long long roots = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = S.pl_idx[j];
    PairGeom G;
    pair_geom(S, S.wl_key[i], G);  // listed by solve32_pair_k: the key is valid
    const int64_t pt = S.wl_point[i];
    double ur = 0.0, vr = 0.0;
    const double E = polish64_pair(G, S.su[pt], S.sv[pt], S.polish_iters, S.tol, S.pl_u[j], S.pl_v[j], &ur, &vr);
    float c = 0.0f;
    if (E >= 0.0) {
      c = (float)(E / (double)S.wl_p[i]);
      ++roots;
      put_root(S, i, ur, vr);
    } else {
      put_no_root(S, i);
    }
    S.contrib[i] = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd((unsigned long long*)&S.counters[2], (unsigned long long)roots);
}

__global__ void reduce_k(const int64_t* __restrict__ woff, const float* __restrict__ contrib, int64_t n_points,
                         int64_t wl_cap, float* __restrict__ E_out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_points; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = woff[p], b = min(woff[p + 1], wl_cap);
    float s = 0.0f;
    for (int64_t j = a; j < b; ++j) s += contrib[j];
    E_out[p] = s;
  }
}

// ------------------------------------------------------------------ host side
struct SampleWs {
  float4* tri;
  float4* tri2;
  int64_t* n_sel;
  int64_t* woff;
  int64_t* wl_point;
  uint64_t* wl_key;
  float* wl_p;
  float* contrib;
  int64_t* pl_count;
  int64_t* pl_idx;
  float *pl_u, *pl_v;
  int32_t* sel_cache;
  int32_t* mode;
  void* scan;
  size_t bytes;
};

static SampleWs carve_sample_ws(void* base, int64_t n_tris, int64_t n_tris2, int64_t n_points, int64_t wl_cap) {
  SampleWs w{};
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  w.tri = (float4*)take((size_t)n_tris * kTriF4 * sizeof(float4));
  w.tri2 = (float4*)take((size_t)n_tris2 * kTriF4 * sizeof(float4));
  w.n_sel = (int64_t*)take((size_t)n_points * 8);
  w.woff = (int64_t*)take((size_t)(n_points + 1) * 8);
  w.wl_point = (int64_t*)take((size_t)wl_cap * 8);
  w.wl_key = (uint64_t*)take((size_t)wl_cap * 8);
  w.wl_p = (float*)take((size_t)wl_cap * 4);
  w.contrib = (float*)take((size_t)wl_cap * 4);
  w.pl_count = (int64_t*)take(8);
  w.pl_idx = (int64_t*)take((size_t)wl_cap * 8);
  w.pl_u = (float*)take((size_t)wl_cap * 4);
  w.pl_v = (float*)take((size_t)wl_cap * 4);
  w.sel_cache = (int32_t*)take((size_t)n_points * kSelCache * 4);
  w.mode = (int32_t*)take(4);
  w.scan = take(scan_ws_bytes(n_points));
  w.bytes = o;
  return w;
}

size_t sample_ws_bytes(int64_t n_tris, int64_t n_tris2, int64_t n_points, int64_t wl_cap) {
  return carve_sample_ws(nullptr, n_tris, n_tris2, n_points, wl_cap).bytes;
}

cudaError_t launch_sample_and_solve(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                                    const bnb_emitters* em, const bnb_index* idx, const float* su, const float* sv,
                                    int64_t n_points, const bnb_sample_cfg* cfg, float* E_out,
                                    bnb_sample_stats* stats, void* ws, cudaStream_t st) {
  SampleWs w = carve_sample_ws(ws, s1->n_tris, s2 ? s2->n_tris : 0, n_points, cfg->worklist_capacity);
  cudaError_t e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = launch_pack_tris(s1, w.tri, st)) != cudaSuccess) return e;
  if (s2 && (e = launch_pack_tris(s2, w.tri2, st)) != cudaSuccess) return e;
  if (n_points == 0) return cudaSuccess;
  SampleParams P{};
  P.offsets = idx->offsets;
  P.key = idx->key;
  P.etilde = idx->etilde;
  P.index_capacity = idx->capacity;
  P.G = idx->grid_res;
  P.su = su;
  P.sv = sv;
  P.n_points = n_points;
  P.gamma = cfg->gamma;
  P.seed = cfg->seed;
  P.n_sel = w.n_sel;
  P.woff = w.woff;
  P.wl_cap = cfg->worklist_capacity;
  P.wl_point = w.wl_point;
  P.wl_key = w.wl_key;
  P.wl_p = w.wl_p;
  P.counters = stats->counters;
  P.status = stats->status;
  P.sel_count = stats->sel_count;
  P.sel_point = stats->sel_point;
  P.sel_key = stats->sel_key;
  P.bins = cfg->bins;
  P.sel_cache = w.sel_cache;
  const int64_t pblocks = std::min<int64_t>((n_points + 255) / 256, (int64_t)sms * 32);
  const int64_t wblocks = std::min<int64_t>((n_points * 32 + 255) / 256, (int64_t)sms * 64);
  sample_mode_k<<<1, 1, 0, st>>>(idx->offsets, idx->grid_res, idx->capacity, w.mode);
  sample_k<false><<<(unsigned)pblocks, 256, 0, st>>>(P, w.mode);
  if (!P.bins) sample_warp_k<false><<<(unsigned)wblocks, 256, 0, st>>>(P, w.mode);
  if ((e = launch_exclusive_scan(w.n_sel, w.woff, n_points, w.scan, st)) != cudaSuccess) return e;
  sample_k<true><<<(unsigned)pblocks, 256, 0, st>>>(P, w.mode);
  if (!P.bins) sample_warp_k<true><<<(unsigned)wblocks, 256, 0, st>>>(P, w.mode);
  SolveParams S{};
  S.tri = w.tri;
  S.n_tris = s1->n_tris;
  S.n_emitters = em->n;
  S.ex = em->x;
  S.ey = em->y;
  S.ez = em->z;
  S.ei = em->intensity;
  for (int c = 0; c < 3; ++c) {
    S.rp0[c] = rec->p0[c];
    S.re1[c] = rec->e1[c];
    S.re2[c] = rec->e2[c];
  }
  S.su = su;
  S.sv = sv;
  S.wl_point = w.wl_point;
  S.wl_key = w.wl_key;
  S.wl_p = w.wl_p;
  S.n_wl = w.woff + n_points;
  S.wl_cap = cfg->worklist_capacity;
  S.newton_iters = cfg->newton_iters;
  S.polish_iters = cfg->polish_iters;
  S.tol = cfg->tol;
  S.contrib = w.contrib;
  S.counters = stats->counters;
  S.root_u1 = stats->root_u1;
  S.pl_count = w.pl_count;
  S.pl_idx = w.pl_idx;
  S.pl_u = w.pl_u;
  S.pl_v = w.pl_v;
  if ((e = cudaMemsetAsync(w.pl_count, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
  S.eta = s1->eta;
  S.tri2 = w.tri2;
  S.n_tris2 = s2 ? s2->n_tris : 0;
  S.eta2 = s2 ? s2->eta : 1.0f;
  S.kind1 = s1->kind;
  S.kind2 = s2 ? s2->kind : BNB_REFLECT;
  S.stoc_trials = cfg->stoc_trials;
  S.seed = cfg->seed;
  if (!s2 && cfg->stoc_trials > 0) {
    if (s1->kind == BNB_REFRACT)
      solve_stoc_k<true><<<sms * 16, 256, 0, st>>>(S);
    else
      solve_stoc_k<false><<<sms * 16, 256, 0, st>>>(S);
  } else if (s2) {
    solve32_pair_k<<<sms * 16, 256, 0, st>>>(S);
    polish_pair_k<<<sms * 16, 256, 0, st>>>(S);
  } else if (s1->kind == BNB_REFRACT) {
    solve32_k<true><<<sms * 16, 256, 0, st>>>(S);
    polish_k<true><<<sms * 16, 256, 0, st>>>(S);
  } else {
    solve32_k<false><<<sms * 16, 256, 0, st>>>(S);
    polish_k<false><<<sms * 16, 256, 0, st>>>(S);
  }
  reduce_k<<<(unsigned)pblocks, 256, 0, st>>>(w.woff, w.contrib, n_points, cfg->worklist_capacity, E_out);
  return cudaGetLastError();
}

}  // namespace bnb
