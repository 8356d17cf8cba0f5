// Sample and solve kernels: the rendering pass (Sec. 5, Algorithm 1; Sec. 6.1
// "Root-finding").
//
//   sample_k (count)  per shading point: grid cell of (u,v), then for every
//                     listed tuple P = min(gamma E~, 1) (float32 product rounded
//                     up, so P > 0 whenever E~ > 0) and one Philox4x32-10
//                     uniform r (key = seed, counter = (point, tuple key));
//                     the tuple is selected when r < P.  Counts per point.
//   scan              -> worklist offsets (point order, then key order).
//   sample_k (fill)   the same draws, writing (point, key, P).
//   solve_k           per selected tuple: Newton's method in T1's barycentric
//                     coordinates from the centroid (deterministic init), float32
//                     damped steps then float64 polish steps, acceptance tests,
//                     contribution E(root) / P.
//   reduce_k          per point, contributions summed in worklist order.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"

namespace bnb {

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ float uniform24(uint64_t seed, int64_t point, uint64_t key) {
  uint32_t c[4] = {(uint32_t)point, (uint32_t)((uint64_t)point >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (float)(c[0] >> 8) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ int grid_col_s(float x, int G) {
  const float p = __fmul_rn(fminf(fmaxf(x, 0.0f), 1.0f), (float)G);
  return min(G - 1, max(0, (int)floorf(p)));
}

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
};

template <bool FILL>
__global__ void __launch_bounds__(256) sample_k(SampleParams P) {
  long long nu = 0, ns = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n_points;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int g = grid_col_s(P.sv[p], P.G) * P.G + grid_col_s(P.su[p], P.G);
    const int64_t s = P.offsets[g];
    const int64_t e = min(P.offsets[g + 1], P.index_capacity);
    int64_t cnt = 0;
    int64_t out = FILL ? P.woff[p] : 0;
    for (int64_t j = s; j < e; ++j) {
      const float Pt = fminf(__fmul_ru(P.gamma, P.etilde[j]), 1.0f);
      const uint64_t k = P.key[j];
      const float r = uniform24(P.seed, p, k);
      if (r < Pt) {
        if (FILL) {
          if (out < P.wl_cap) {
            P.wl_point[out] = p;
            P.wl_key[out] = k;
            P.wl_p[out] = Pt;
          } else {
            atomicCAS(P.status, 0, BNB_ERR_CAPACITY);
          }
          ++out;
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
    }
    if ((threadIdx.x & 31) == 0) {
      if (nu) atomicAdd((unsigned long long*)&P.counters[0], (unsigned long long)nu);
      if (ns) atomicAdd((unsigned long long*)&P.counters[1], (unsigned long long)ns);
    }
  }
}

// ------------------------------------------------------------------ path evaluation (rational form)
// For barycentrics (u, v) in T1: x1, interpolated n1, d0 = x1 - x0, reflected d~ (Eq.
// eq_refr_rational), receiver coordinates (Eq. eq_rct), their Jacobian by the product
// rule, and the path irradiance of Eq. eq_dwda.
template <typename T>
struct Path {
  T uk, vk, J00, J01, J10, J11, t, E;
  bool ok;
};

template <typename T>
__device__ __forceinline__ Path<T> eval_path(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0f)[3],
                                            float I0, const float (&rp0)[3], const float (&re1)[3],
                                            const float (&re2)[3], T u, T v) {
  T p0[3], e1[3], e2[3], n0[3], f1[3], f2[3], x[3], n[3], d[3], P0[3], E1[3], E2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p0[c] = (T)pf[0][c];
    e1[c] = (T)pf[1][c] - p0[c];
    e2[c] = (T)pf[2][c] - p0[c];
    n0[c] = (T)nf[0][c];
    f1[c] = (T)nf[1][c] - n0[c];
    f2[c] = (T)nf[2][c] - n0[c];
    x[c] = p0[c] + u * e1[c] + v * e2[c];
    n[c] = n0[c] + u * f1[c] + v * f2[c];
    d[c] = x[c] - (T)x0f[c];
    P0[c] = (T)rp0[c];
    E1[c] = (T)re1[c];
    E2[c] = (T)re2[c];
  }
  auto dot = [](const T* a, const T* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  auto cross = [](const T* a, const T* b, T* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
  };
  const T nn = dot(n, n), dn = dot(d, n);
  T dt[3], w[3], g[3], he2w[3], hwe1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dt[c] = nn * d[c] - T(2) * dn * n[c];
    w[c] = x[c] - P0[c];
  }
  cross(E2, E1, g);
  cross(E2, w, he2w);
  cross(w, E1, hwe1);
  const T Q = dot(dt, g), A = dot(dt, he2w), B = dot(hwe1, dt);
  T dA[2], dB[2], dQ[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T* dx = j == 0 ? e1 : e2;
    const T* dnv = j == 0 ? f1 : f2;
    const T dnn = T(2) * dot(n, dnv);
    const T ddn = dot(dx, n) + dot(d, dnv);
    T ddt[3], c1[3], c2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ddt[c] = dnn * d[c] + nn * dx[c] - T(2) * (ddn * n[c] + dn * dnv[c]);
    cross(E2, dx, c1);
    cross(dx, E1, c2);
    dQ[j] = dot(ddt, g);
    dA[j] = dot(ddt, he2w) + dot(dt, c1);
    dB[j] = dot(c2, dt) + dot(hwe1, ddt);
  }
  Path<T> r;
  const T iq = T(1) / Q;
  r.uk = A * iq;
  r.vk = B * iq;
  r.J00 = (dA[0] * Q - A * dQ[0]) * iq * iq;
  r.J01 = (dA[1] * Q - A * dQ[1]) * iq * iq;
  r.J10 = (dB[0] * Q - B * dQ[0]) * iq * iq;
  r.J11 = (dB[1] * Q - B * dQ[1]) * iq * iq;
  r.t = dot(hwe1, E2) * iq;
  const T det = r.J00 * r.J11 - r.J01 * r.J10;
  T N1[3], Nk[3], r0[3];
  cross(e1, e2, N1);
  cross(E1, E2, Nk);
#pragma unroll
  for (int c = 0; c < 3; ++c) r0[c] = p0[c] - (T)x0f[c];
  const T C1 = dot(r0, N1);
  const T s = dot(d, d);
  r.E = (T)I0 * fabs(C1) / (s * sqrt(s) * sqrt(dot(Nk, Nk)) * fabs(det));
  r.ok = isfinite(r.uk) && isfinite(r.vk) && isfinite(det) && Q != T(0);
  return r;
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
  float* contrib;
  int64_t* counters;
};

__device__ __forceinline__ void load_tri_s(const float4* __restrict__ tri, int t, float (&p)[3][3],
                                           float (&n)[3][3]) {
  const float4* b = tri + (int64_t)t * kTriF4;
  const float4 a0 = __ldg(b), a1 = __ldg(b + 1), a2 = __ldg(b + 2), a3 = __ldg(b + 3), a4 = __ldg(b + 4);
  p[0][0] = a0.x; p[0][1] = a0.y; p[0][2] = a0.z; p[1][0] = a0.w;
  p[1][1] = a1.x; p[1][2] = a1.y; p[2][0] = a1.z; p[2][1] = a1.w;
  p[2][2] = a2.x; n[0][0] = a2.y; n[0][1] = a2.z; n[0][2] = a2.w;
  n[1][0] = a3.x; n[1][1] = a3.y; n[1][2] = a3.z; n[2][0] = a3.w;
  n[2][1] = a4.x; n[2][2] = a4.y;
}

template <typename T>
__device__ __forceinline__ bool newton_step(const Path<T>& P, T tu, T tv, bool damped, T& u, T& v, T& step) {
  const T det = P.J00 * P.J11 - P.J01 * P.J10;
  if (!P.ok || !(det != T(0)) || !isfinite(det)) return false;
  const T fu = P.uk - tu, fv = P.vk - tv;
  T du = -(P.J11 * fu - P.J01 * fv) / det;
  T dv = -(-P.J10 * fu + P.J00 * fv) / det;
  const T mx = fmax(fabs(du), fabs(dv));
  if (damped && mx > T(0.5)) {
    du *= T(0.5) / mx;
    dv *= T(0.5) / mx;
  }
  u += du;
  v += dv;
  step = mx;
  return isfinite(u) && isfinite(v);
}

__global__ void __launch_bounds__(256) solve_k(SolveParams S) {
  const int64_t n = min(*S.n_wl, S.wl_cap);
  long long roots = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = S.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    if (t >= S.n_tris || e >= S.n_emitters) {  // key from another scene: no path, no read
      S.contrib[i] = 0.0f;
      continue;
    }
    float pf[3][3], nf[3][3];
    load_tri_s(S.tri, t, pf, nf);
    const float x0[3] = {__ldg(S.ex + e), __ldg(S.ey + e), __ldg(S.ez + e)};
    const float I0 = __ldg(S.ei + e);
    const int64_t pt = S.wl_point[i];
    const float tuf = S.su[pt], tvf = S.sv[pt];
    // float32 damped Newton from the centroid
    float u = 1.0f / 3.0f, v = 1.0f / 3.0f;
    bool good = true;
    for (int it = 0; it < S.newton_iters; ++it) {
      const Path<float> P = eval_path<float>(pf, nf, x0, I0, S.rp0, S.re1, S.re2, u, v);
      float step;
      if (!newton_step<float>(P, tuf, tvf, true, u, v, step)) {
        good = false;
        break;
      }
      if (step < 1e-6f) break;
    }
    float c = 0.0f;
    if (good) {
      // float64 polish and acceptance
      double ud = u, vd = v;
      for (int it = 0; it < S.polish_iters && good; ++it) {
        const Path<double> P = eval_path<double>(pf, nf, x0, I0, S.rp0, S.re1, S.re2, ud, vd);
        double step;
        good = newton_step<double>(P, (double)tuf, (double)tvf, false, ud, vd, step);
      }
      if (good) {
        const Path<double> P = eval_path<double>(pf, nf, x0, I0, S.rp0, S.re1, S.re2, ud, vd);
        const double fu = P.uk - (double)tuf, fv = P.vk - (double)tvf;
        const double r0 = fu * S.re1[0] + fv * S.re2[0], r1 = fu * S.re1[1] + fv * S.re2[1],
                     r2 = fu * S.re1[2] + fv * S.re2[2];
        const double res = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
        const bool inside = ud >= 0.0 && vd >= 0.0 && ud + vd <= 1.0;
        if (P.ok && res < (double)S.tol && inside && P.t > 0.0 && isfinite(P.E)) {
          c = (float)(P.E / (double)S.wl_p[i]);
          ++roots;
        }
      }
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
  int64_t* n_sel;
  int64_t* woff;
  int64_t* wl_point;
  uint64_t* wl_key;
  float* wl_p;
  float* contrib;
  void* scan;
  size_t bytes;
};

static SampleWs carve_sample_ws(void* base, int64_t n_tris, int64_t n_points, int64_t wl_cap) {
  SampleWs w{};
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  w.tri = (float4*)take((size_t)n_tris * kTriF4 * sizeof(float4));
  w.n_sel = (int64_t*)take((size_t)n_points * 8);
  w.woff = (int64_t*)take((size_t)(n_points + 1) * 8);
  w.wl_point = (int64_t*)take((size_t)wl_cap * 8);
  w.wl_key = (uint64_t*)take((size_t)wl_cap * 8);
  w.wl_p = (float*)take((size_t)wl_cap * 4);
  w.contrib = (float*)take((size_t)wl_cap * 4);
  w.scan = take(scan_ws_bytes(n_points));
  w.bytes = o;
  return w;
}

size_t sample_ws_bytes(int64_t n_tris, int64_t n_points, int64_t wl_cap) {
  return carve_sample_ws(nullptr, n_tris, n_points, wl_cap).bytes;
}

cudaError_t launch_sample_and_solve(const bnb_surface* s1, const bnb_receiver* rec, const bnb_emitters* em,
                                    const bnb_index* idx, const float* su, const float* sv, int64_t n_points,
                                    const bnb_sample_cfg* cfg, float* E_out, bnb_sample_stats* stats, void* ws,
                                    cudaStream_t st) {
  SampleWs w = carve_sample_ws(ws, s1->n_tris, n_points, cfg->worklist_capacity);
  cudaError_t e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = launch_pack_tris(s1, w.tri, st)) != cudaSuccess) return e;
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
  const int64_t pblocks = std::min<int64_t>((n_points + 255) / 256, (int64_t)sms * 32);
  sample_k<false><<<(unsigned)pblocks, 256, 0, st>>>(P);
  if ((e = launch_exclusive_scan(w.n_sel, w.woff, n_points, w.scan, st)) != cudaSuccess) return e;
  sample_k<true><<<(unsigned)pblocks, 256, 0, st>>>(P);
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
  solve_k<<<sms * 16, 256, 0, st>>>(S);
  reduce_k<<<(unsigned)pblocks, 256, 0, st>>>(w.woff, w.contrib, n_points, cfg->worklist_capacity, E_out);
  return cudaGetLastError();
}

}  // namespace bnb
