// Device functions shared by the per-call and the batched rendering pass: Philox4x32-10
// selection draws, the rational-form path evaluation of one tuple, and Newton steps.
#pragma once

#include <stdint.h>

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

// ------------------------------------------------------------------ path evaluation (rational form)
// For barycentrics (u, v) in T1: x1, interpolated n1, d0 = x1 - x0, the reflected or refracted
// d~ (Eq. eq_refr_rational; refraction with eta' = eta, sqrt(beta) and its derivative
// d beta / (2 sqrt(beta))), receiver coordinates (Eq. eq_rct), their Jacobian by the product
// rule, and the path irradiance of Eq. eq_dwda.  ok is false where no refracted path exists.
template <typename T>
struct Path {
  T uk, vk, J00, J01, J10, J11, t, E;
  bool ok;
};

template <typename T, bool REFRACT>
__device__ __forceinline__ Path<T> eval_path(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0f)[3],
                                            float I0, const float (&rp0)[3], const float (&re1)[3],
                                            const float (&re2)[3], T u, T v, float etaf) {
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
  const T nn = dot(n, n), dn = dot(d, n), ss = dot(d, d);
  const T eta = (T)etaf;
  T W = T(0);
  bool tir = false;
  if constexpr (REFRACT) {
    const T beta = (T(1) - eta * eta) * nn * ss + eta * eta * dn * dn;
    tir = !(beta > T(0));
    W = sqrt(fmax(beta, T(0)));
  }
  T dt[3], w[3], g[3], he2w[3], hwe1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (REFRACT)
      dt[c] = eta * (nn * d[c] - dn * n[c]) - W * n[c];
    else
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
    if constexpr (REFRACT) {
      const T dbeta = (T(1) - eta * eta) * (dnn * ss + nn * T(2) * dot(d, dx)) + eta * eta * T(2) * dn * ddn;
      const T dW = dbeta / (T(2) * W);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        ddt[c] = eta * (dnn * d[c] + nn * dx[c] - ddn * n[c] - dn * dnv[c]) - dW * n[c] - W * dnv[c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) ddt[c] = dnn * d[c] + nn * dx[c] - T(2) * (ddn * n[c] + dn * dnv[c]);
    }
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
  r.E = (T)I0 * fabs(C1) / (ss * sqrt(ss) * sqrt(dot(Nk, Nk)) * fabs(det));
  r.ok = !tir && isfinite(r.uk) && isfinite(r.vk) && isfinite(det) && Q != T(0);
  return r;
}

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

// One tuple's Newton solve at a receiver point (Sec. 6.1 "Root-finding", deterministic init) in
// two phases, so that the float64 work runs only for the tuples that need it:
//
//   newton32  float32 damped steps from the centroid.  Returns false when the tuple has no
//             admissible root: a step failed (non-finite or singular), or the iteration converged
//             (last step below 1e-6, so the root is known to about 1e-6) more than kOutside = 1e-3
//             outside the triangle, a distance the float64 polish, whose steps from there are of
//             the size of the float32 root error, cannot cover.  Otherwise (u, v) is the start of
//             the polish.
//   polish64  float64 polish steps and the acceptance tests.  Returns the path irradiance E
//             (float64), or a negative value when no admissible root is found.
template <bool REFRACT>
__device__ __forceinline__ bool newton32(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0)[3],
                                         float I0, const float (&rp0)[3], const float (&re1)[3], const float (&re2)[3],
                                         float tuf, float tvf, int newton_iters, float eta, float& u, float& v) {
  u = 1.0f / 3.0f;
  v = 1.0f / 3.0f;
  bool converged = false;
  for (int it = 0; it < newton_iters; ++it) {
    const Path<float> P = eval_path<float, REFRACT>(pf, nf, x0, I0, rp0, re1, re2, u, v, eta);
    float step;
    if (!newton_step<float>(P, tuf, tvf, true, u, v, step)) return false;
    if (step < 1e-6f) {
      converged = true;
      break;
    }
  }
  constexpr float kOutside = 1e-3f;
  return !(converged && fminf(fminf(u, v), 1.0f - u - v) < -kOutside);
}

template <bool REFRACT>
__device__ __forceinline__ double polish64(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0)[3],
                                           float I0, const float (&rp0)[3], const float (&re1)[3],
                                           const float (&re2)[3], float tuf, float tvf, int polish_iters, float tol,
                                           float eta, float u, float v) {
  double ud = u, vd = v;
  bool good = true;
  for (int it = 0; it < polish_iters && good; ++it) {
    const Path<double> P = eval_path<double, REFRACT>(pf, nf, x0, I0, rp0, re1, re2, ud, vd, eta);
    double step;
    good = newton_step<double>(P, (double)tuf, (double)tvf, false, ud, vd, step);
  }
  if (!good) return -1.0;
  const Path<double> P = eval_path<double, REFRACT>(pf, nf, x0, I0, rp0, re1, re2, ud, vd, eta);
  const double fu = P.uk - (double)tuf, fv = P.vk - (double)tvf;
  const double r0 = fu * re1[0] + fv * re2[0], r1 = fu * re1[1] + fv * re2[1], r2 = fu * re1[2] + fv * re2[2];
  const double res = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
  const bool inside = ud >= 0.0 && vd >= 0.0 && ud + vd <= 1.0;
  if (P.ok && res < (double)tol && inside && P.t > 0.0 && isfinite(P.E)) return P.E;
  return -1.0;
}

// Appends the calling lane to a device list when `need` is set (one atomic per warp); returns the
// lane's list position, or -1.  Every lane active at the call must make it.
__device__ __forceinline__ int64_t warp_append(bool need, int64_t* count) {
  const unsigned active = __activemask();
  const unsigned m = __ballot_sync(active, need);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(active) - 1;
  unsigned long long base = 0;
  if (lane == leader && m != 0u) base = atomicAdd((unsigned long long*)count, (unsigned long long)__popc(m));
  base = __shfl_sync(active, base, leader);
  if (!need) return -1;
  return (int64_t)base + __popc(m & ((1u << lane) - 1u));
}

}  // namespace bnb
