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

// DERIV = false: the receiver coordinates, t and ok only (no Jacobian, no E).
template <typename T, bool REFRACT, bool DERIV = true>
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
  T dA[2] = {T(0), T(0)}, dB[2] = {T(0), T(0)}, dQ[2] = {T(0), T(0)};
#pragma unroll
  for (int j = 0; j < (DERIV ? 2 : 0); ++j) {
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
  if constexpr (!DERIV) {
    r.J00 = r.J01 = r.J10 = r.J11 = T(0);
    r.E = T(0);
    r.t = dot(hwe1, E2) * iq;
    r.ok = !tir && isfinite(r.uk) && isfinite(r.vk) && Q != T(0);
    return r;
  }
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
// From the start (u, v) given on entry (the deterministic start is the centroid).
template <bool REFRACT>
__device__ __forceinline__ bool newton32_from(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0)[3],
                                              float I0, const float (&rp0)[3], const float (&re1)[3],
                                              const float (&re2)[3], float tuf, float tvf, int newton_iters, float eta,
                                              float& u, float& v) {
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
__device__ __forceinline__ bool newton32(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0)[3],
                                         float I0, const float (&rp0)[3], const float (&re1)[3], const float (&re2)[3],
                                         float tuf, float tvf, int newton_iters, float eta, float& u, float& v) {
  u = 1.0f / 3.0f;
  v = 1.0f / 3.0f;
  return newton32_from<REFRACT>(pf, nf, x0, I0, rp0, re1, re2, tuf, tvf, newton_iters, eta, u, v);
}

// The float64 polish, mixed precision: Newton steps whose residual is evaluated in float64 (the
// receiver coordinates only) and whose Jacobian is the float32 one at the float32 root (iterative
// refinement: from a root known to ~1e-6 with a Jacobian accurate to ~1e-6 one step leaves
// ~1e-12); the acceptance tests in float64 at the polished root, E from the float32 derivatives
// there (relative error ~1e-6).  The polished root is returned through ur, vr when given.
template <bool REFRACT>
__device__ __forceinline__ double polish64(const float (&pf)[3][3], const float (&nf)[3][3], const float (&x0)[3],
                                           float I0, const float (&rp0)[3], const float (&re1)[3],
                                           const float (&re2)[3], float tuf, float tvf, int polish_iters, float tol,
                                           float eta, float u, float v, double* ur = nullptr,
                                           double* vr = nullptr) {
  const Path<float> Pf = eval_path<float, REFRACT>(pf, nf, x0, I0, rp0, re1, re2, u, v, eta);
  const double J00 = Pf.J00, J01 = Pf.J01, J10 = Pf.J10, J11 = Pf.J11;
  const double det = J00 * J11 - J01 * J10;
  if (!Pf.ok || !(det != 0.0) || !isfinite(det)) return -1.0;
  double ud = u, vd = v;
  for (int it = 0; it < polish_iters; ++it) {
    const Path<double> H = eval_path<double, REFRACT, false>(pf, nf, x0, I0, rp0, re1, re2, ud, vd, eta);
    if (!H.ok) return -1.0;
    const double fu = H.uk - (double)tuf, fv = H.vk - (double)tvf;
    ud -= (J11 * fu - J01 * fv) / det;
    vd -= (-J10 * fu + J00 * fv) / det;
    if (!isfinite(ud) || !isfinite(vd)) return -1.0;
  }
  if (ur) *ur = ud;
  if (vr) *vr = vd;
  const Path<double> H = eval_path<double, REFRACT, false>(pf, nf, x0, I0, rp0, re1, re2, ud, vd, eta);
  if (!H.ok) return -1.0;
  const double fu = H.uk - (double)tuf, fv = H.vk - (double)tvf;
  const double r0 = fu * re1[0] + fv * re2[0], r1 = fu * re1[1] + fv * re2[1], r2 = fu * re1[2] + fv * re2[2];
  const double res = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
  const bool inside = ud >= 0.0 && vd >= 0.0 && ud + vd <= 1.0;
  if (!(res < (double)tol && inside && H.t > 0.0)) return -1.0;
  const Path<float> Pe = eval_path<float, REFRACT>(pf, nf, x0, I0, rp0, re1, re2, (float)ud, (float)vd, eta);
  if (!Pe.ok || !isfinite(Pe.E)) return -1.0;
  return (double)Pe.E;
}

// Start of stochastic trial t (t >= 0) of (point, tuple key) (Sec. 6.1 "Stoc"): the first two
// outputs of Philox4x32-10 with counter (point, key) and key seed + (t + 1) * 0x9E3779B97F4A7C15
// (mod 2^64), as 24-bit integers (a, b) folded into the triangle (a + b > 2^24 -> 2^24 - a, 2^24 - b,
// decided on the integers), scaled by 2^-24 (exact in float32).
__device__ __forceinline__ void stoc_start(uint64_t seed, int64_t point, uint64_t key, int t, float& u, float& v) {
  const uint64_t k = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
  uint32_t c[4] = {(uint32_t)point, (uint32_t)((uint64_t)point >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
  philox4x32_10(c, (uint32_t)k, (uint32_t)(k >> 32));
  uint32_t a = c[0] >> 8, b = c[1] >> 8;
  if (a + b > (1u << 24)) {
    a = (1u << 24) - a;
    b = (1u << 24) - b;
  }
  u = (float)a * (1.0f / 16777216.0f);
  v = (float)b * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------------ two-vertex chains
// x0 -> x1 on T1 -> x2 on T2 -> receiver with refraction at both vertices, in the same
// un-normalized rational forms (Eqs. eq_xi, eq_ni, eq_refr_rational, eq_rct; d1 = x2 - x1),
// differentiated in (u1, v1) by forward-mode duals.
template <typename T>
struct Dl {
  T v, du, dv;
};
template <typename T>
__device__ __forceinline__ Dl<T> operator+(Dl<T> a, Dl<T> b) { return {a.v + b.v, a.du + b.du, a.dv + b.dv}; }
template <typename T>
__device__ __forceinline__ Dl<T> operator-(Dl<T> a, Dl<T> b) { return {a.v - b.v, a.du - b.du, a.dv - b.dv}; }
template <typename T>
__device__ __forceinline__ Dl<T> operator*(Dl<T> a, Dl<T> b) {
  return {a.v * b.v, a.du * b.v + a.v * b.du, a.dv * b.v + a.v * b.dv};
}
template <typename T>
__device__ __forceinline__ Dl<T> operator*(T s, Dl<T> a) { return {s * a.v, s * a.du, s * a.dv}; }
template <typename T>
__device__ __forceinline__ Dl<T> operator/(Dl<T> a, Dl<T> b) {
  const T i = T(1) / b.v, q = a.v * i;
  return {q, (a.du - q * b.du) * i, (a.dv - q * b.dv) * i};
}
template <typename T>
__device__ __forceinline__ Dl<T> dl_sqrt(Dl<T> a) {
  const T s = sqrt(a.v), h = T(0.5) / s;
  return {s, a.du * h, a.dv * h};
}
template <typename T>
__device__ __forceinline__ Dl<T> dl_dot(const Dl<T> (&a)[3], const Dl<T> (&b)[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
template <typename T>
__device__ __forceinline__ Dl<T> dl_dotc(const Dl<T> (&a)[3], const T (&b)[3]) {
  return b[0] * a[0] + b[1] * a[1] + b[2] * a[2];
}
template <typename T>
__device__ __forceinline__ void dl_cross_cd(const T (&a)[3], const Dl<T> (&b)[3], Dl<T> (&r)[3]) {  // a x b
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ void dl_cross_dc(const Dl<T> (&a)[3], const T (&b)[3], Dl<T> (&r)[3]) {  // a x b
  r[0] = b[2] * a[1] - b[1] * a[2];
  r[1] = b[0] * a[2] - b[2] * a[0];
  r[2] = b[1] * a[0] - b[0] * a[1];
}

// The triangles and constants of one pair tuple; kind1 / kind2: BNB_REFLECT or BNB_REFRACT.
struct PairGeom {
  float p1[3][3], n1[3][3], p2[3][3], n2[3][3], x0[3], I0, rp0[3], re1[3], re2[3], eta1, eta2;
  int kind1, kind2;
};

template <typename T>
struct Path2 : Path<T> {
  T u2, v2, t2;  // barycentrics of the hit on T2's plane; ray parameter of the receiver hit
};

// d~ = eta' ((n.n) d - (d.n) n) - sqrt(beta) n; false when beta <= 0 (no refracted path).
// Reflection: d~ = (n.n) d - 2 (d.n) n.
template <typename T>
__device__ __forceinline__ bool dl_refract(const Dl<T> (&n)[3], const Dl<T> (&d)[3], int kind, T eta,
                                           Dl<T> (&out)[3]) {
  const Dl<T> nn = dl_dot(n, n), dn = dl_dot(d, n), ss = dl_dot(d, d);
  if (kind == BNB_REFLECT) {
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = nn * d[c] - T(2) * (dn * n[c]);
    return true;
  }
  const Dl<T> beta = (T(1) - eta * eta) * (nn * ss) + (eta * eta) * (dn * dn);
  if (!(beta.v > T(0))) return false;
  const Dl<T> W = dl_sqrt(beta);
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = eta * (nn * d[c] - dn * n[c]) - W * n[c];
  return true;
}

// Plane coordinates (Eq. eq_rct) of the ray x + t d on o + a e1 + b e2, and its parameter t.
template <typename T>
__device__ __forceinline__ void dl_plane(const Dl<T> (&x)[3], const Dl<T> (&d)[3], const T (&o)[3], const T (&e1)[3],
                                         const T (&e2)[3], Dl<T>& a, Dl<T>& b, Dl<T>& t) {
  Dl<T> w[3], h1[3], h2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) w[c] = x[c] - Dl<T>{o[c], T(0), T(0)};
  const T g[3] = {e2[1] * e1[2] - e2[2] * e1[1], e2[2] * e1[0] - e2[0] * e1[2], e2[0] * e1[1] - e2[1] * e1[0]};
  dl_cross_cd(e2, w, h1);
  dl_cross_dc(w, e1, h2);
  const Dl<T> q = dl_dotc(d, g);
  a = dl_dot(d, h1) / q;
  b = dl_dot(h2, d) / q;
  t = dl_dotc(h2, e2) / q;
}

template <typename T>
__device__ __forceinline__ Path2<T> eval_pair(const PairGeom& G, T u, T v) {
  Path2<T> r{};
  r.ok = false;
  T e1[3], e2[3], f1[3], f2[3], o2[3], e21[3], e22[3], R0[3], R1[3], R2[3];
  Dl<T> x1[3], n1[3], d0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    e1[c] = (T)G.p1[1][c] - (T)G.p1[0][c];
    e2[c] = (T)G.p1[2][c] - (T)G.p1[0][c];
    f1[c] = (T)G.n1[1][c] - (T)G.n1[0][c];
    f2[c] = (T)G.n1[2][c] - (T)G.n1[0][c];
    x1[c] = {(T)G.p1[0][c] + u * e1[c] + v * e2[c], e1[c], e2[c]};
    n1[c] = {(T)G.n1[0][c] + u * f1[c] + v * f2[c], f1[c], f2[c]};
    d0[c] = {x1[c].v - (T)G.x0[c], e1[c], e2[c]};
    o2[c] = (T)G.p2[0][c];
    e21[c] = (T)G.p2[1][c] - o2[c];
    e22[c] = (T)G.p2[2][c] - o2[c];
    R0[c] = (T)G.rp0[c];
    R1[c] = (T)G.re1[c];
    R2[c] = (T)G.re2[c];
  }
  Dl<T> t1d[3];
  if (!dl_refract(n1, d0, G.kind1, (T)G.eta1, t1d)) return r;
  Dl<T> u2, v2, s1;
  dl_plane(x1, t1d, o2, e21, e22, u2, v2, s1);
  Dl<T> x2[3], n2[3], d1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x2[c] = Dl<T>{o2[c], T(0), T(0)} + e21[c] * u2 + e22[c] * v2;
    n2[c] = Dl<T>{(T)G.n2[0][c], T(0), T(0)} + ((T)G.n2[1][c] - (T)G.n2[0][c]) * u2 +
            ((T)G.n2[2][c] - (T)G.n2[0][c]) * v2;
    d1[c] = x2[c] - x1[c];
  }
  Dl<T> t2d[3];
  if (!dl_refract(n2, d1, G.kind2, (T)G.eta2, t2d)) return r;
  Dl<T> uk, vk, s2;
  dl_plane(x2, t2d, R0, R1, R2, uk, vk, s2);
  r.uk = uk.v;
  r.vk = vk.v;
  r.J00 = uk.du;
  r.J01 = uk.dv;
  r.J10 = vk.du;
  r.J11 = vk.dv;
  r.t = s1.v;
  r.t2 = s2.v;
  r.u2 = u2.v;
  r.v2 = v2.v;
  const T det = r.J00 * r.J11 - r.J01 * r.J10;
  const T N1[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const T Nk[3] = {R1[1] * R2[2] - R1[2] * R2[1], R1[2] * R2[0] - R1[0] * R2[2], R1[0] * R2[1] - R1[1] * R2[0]};
  T C1 = T(0), ss = T(0), nk = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C1 += ((T)G.p1[0][c] - (T)G.x0[c]) * N1[c];
    ss += d0[c].v * d0[c].v;
    nk += Nk[c] * Nk[c];
  }
  // GGT (Eq. eq_dwda) through both vertices: I0 |d0.N1| / (|d0|^3 |N_k| |det du_k/du_1|)
  r.E = (T)G.I0 * fabs(C1) / (ss * sqrt(ss) * sqrt(nk) * fabs(det));
  r.ok = isfinite(r.uk) && isfinite(r.vk) && isfinite(det) && isfinite(r.u2) && isfinite(r.v2);
  return r;
}

// Pair counterpart of newton32: the same damped float32 phase, also rejecting a root converged more
// than kOutside outside T2.
__device__ __forceinline__ bool newton32_pair(const PairGeom& G, float tuf, float tvf, int newton_iters, float& u,
                                              float& v) {
  u = 1.0f / 3.0f;
  v = 1.0f / 3.0f;
  bool converged = false;
  Path2<float> P{};
  for (int it = 0; it < newton_iters; ++it) {
    P = eval_pair<float>(G, u, v);
    float step;
    if (!newton_step<float>(P, tuf, tvf, true, u, v, step)) return false;
    if (step < 1e-6f) {
      converged = true;
      break;
    }
  }
  constexpr float kOutside = 1e-3f;
  if (!converged) return true;
  if (fminf(fminf(u, v), 1.0f - u - v) < -kOutside) return false;
  return !(fminf(fminf(P.u2, P.v2), 1.0f - P.u2 - P.v2) < -kOutside);
}

// The chain's values only (no derivatives): receiver coordinates, T2 barycentrics and both ray
// parameters; ok is false where a vertex has no refracted path.
template <typename T>
struct Hit2 {
  T uk, vk, u2, v2, t1, t2;
  bool ok;
};

template <typename T>
__device__ __forceinline__ Hit2<T> eval_pair_value(const PairGeom& G, T u, T v) {
  Hit2<T> h{};
  h.ok = false;
  auto dot = [](const T* a, const T* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  auto cross = [](const T* a, const T* b, T* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
  };
  auto refract = [&](const T* n, const T* d, int kind, T eta, T* out) {
    const T nn = dot(n, n), dn = dot(d, n), ss = dot(d, d);
    if (kind == BNB_REFLECT) {
#pragma unroll
      for (int c = 0; c < 3; ++c) out[c] = nn * d[c] - T(2) * (dn * n[c]);
      return true;
    }
    const T beta = (T(1) - eta * eta) * (nn * ss) + (eta * eta) * (dn * dn);
    if (!(beta > T(0))) return false;
    const T W = sqrt(beta);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = eta * (nn * d[c] - dn * n[c]) - W * n[c];
    return true;
  };
  auto plane = [&](const T* x, const T* d, const T* o, const T* e1, const T* e2, T& a, T& b, T& t) {
    T w[3], g[3], h1[3], h2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = x[c] - o[c];
    cross(e2, e1, g);
    cross(e2, w, h1);
    cross(w, e1, h2);
    const T q = dot(d, g);
    a = dot(d, h1) / q;
    b = dot(h2, d) / q;
    t = dot(h2, e2) / q;
  };
  T x1[3], n1[3], d0[3], o2[3], e21[3], e22[3], R0[3], R1[3], R2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T p0 = (T)G.p1[0][c];
    x1[c] = p0 + u * ((T)G.p1[1][c] - p0) + v * ((T)G.p1[2][c] - p0);
    const T m0 = (T)G.n1[0][c];
    n1[c] = m0 + u * ((T)G.n1[1][c] - m0) + v * ((T)G.n1[2][c] - m0);
    d0[c] = x1[c] - (T)G.x0[c];
    o2[c] = (T)G.p2[0][c];
    e21[c] = (T)G.p2[1][c] - o2[c];
    e22[c] = (T)G.p2[2][c] - o2[c];
    R0[c] = (T)G.rp0[c];
    R1[c] = (T)G.re1[c];
    R2[c] = (T)G.re2[c];
  }
  T t1d[3];
  if (!refract(n1, d0, G.kind1, (T)G.eta1, t1d)) return h;
  plane(x1, t1d, o2, e21, e22, h.u2, h.v2, h.t1);
  T x2[3], n2[3], d1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x2[c] = o2[c] + h.u2 * e21[c] + h.v2 * e22[c];
    const T m0 = (T)G.n2[0][c];
    n2[c] = m0 + h.u2 * ((T)G.n2[1][c] - m0) + h.v2 * ((T)G.n2[2][c] - m0);
    d1[c] = x2[c] - x1[c];
  }
  T t2d[3];
  if (!refract(n2, d1, G.kind2, (T)G.eta2, t2d)) return h;
  plane(x2, t2d, R0, R1, R2, h.uk, h.vk, h.t2);
  h.ok = isfinite(h.uk) && isfinite(h.vk) && isfinite(h.u2) && isfinite(h.v2);
  return h;
}

// Mixed-precision polish: Newton steps whose residual is evaluated in float64 (the chain's values
// only) and whose Jacobian is the float32 one at the float32 root (iterative refinement: from a
// root known to ~1e-6 with a Jacobian accurate to ~1e-6, one step leaves ~1e-12).  Acceptance
// tests in float64 at the polished root; E from the float32 derivatives there.
__device__ __forceinline__ double polish64_pair(const PairGeom& G, float tuf, float tvf, int polish_iters, float tol,
                                                float u, float v, double* ur = nullptr, double* vr = nullptr) {
  const Path2<float> Pf = eval_pair<float>(G, u, v);
  const double J00 = Pf.J00, J01 = Pf.J01, J10 = Pf.J10, J11 = Pf.J11;
  const double det = J00 * J11 - J01 * J10;
  if (!Pf.ok || !(det != 0.0) || !isfinite(det)) return -1.0;
  double ud = u, vd = v;
  for (int it = 0; it < polish_iters; ++it) {
    const Hit2<double> H = eval_pair_value<double>(G, ud, vd);
    if (!H.ok) return -1.0;
    const double fu = H.uk - (double)tuf, fv = H.vk - (double)tvf;
    ud -= (J11 * fu - J01 * fv) / det;
    vd -= (-J10 * fu + J00 * fv) / det;
    if (!isfinite(ud) || !isfinite(vd)) return -1.0;
  }
  if (ur) *ur = ud;
  if (vr) *vr = vd;
  const Hit2<double> H = eval_pair_value<double>(G, ud, vd);
  if (!H.ok) return -1.0;
  const double fu = H.uk - (double)tuf, fv = H.vk - (double)tvf;
  const double r0 = fu * G.re1[0] + fv * G.re2[0], r1 = fu * G.re1[1] + fv * G.re2[1], r2 = fu * G.re1[2] + fv * G.re2[2];
  const double res = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
  const bool in1 = ud >= 0.0 && vd >= 0.0 && ud + vd <= 1.0;
  const bool in2 = H.u2 >= 0.0 && H.v2 >= 0.0 && H.u2 + H.v2 <= 1.0;
  if (!(res < (double)tol && in1 && in2 && H.t1 > 0.0 && H.t2 > 0.0)) return -1.0;
  const Path2<float> Pe = eval_pair<float>(G, (float)ud, (float)vd);
  if (!Pe.ok || !isfinite(Pe.E)) return -1.0;
  return (double)Pe.E;
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
