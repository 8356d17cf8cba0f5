// Bound kernel (header-only so that the float32 and float64 instantiations compile
// in parallel): conservative receiver box and irradiance bound per
// (emitter, triangle, subdivision cell) for single reflection.
//
// Per cell (one thread), in the cell's barycentric coordinates mu:
//   x1, n1 (Eqs. eq_xi, eq_ni)        degree 1: coefficients are the corner values
//   d0 = x1 - x0                       degree 1
//   d~ = (n.n) d0 - 2 (d0.n) n         degree 3 (Eq. eq_refr_rational, reflection)
//   Q  = (d~ x e_k2) . e_k1            degree 3 (Eq. eq_rct denominator)
//   A  = (d~ x e_k2) . (x1 - p')       degree 4 (numerator of u_k - u_c)
//   B  = ((x1 - p') x e_k1) . d~       degree 4 (numerator of v_k - v_c)
// with the receiver origin moved to p' = p_k0 + u_c e_k1 + v_c e_k2, the hit of
// the cell's centroid ray.  In exact arithmetic A/Q = u_k - u_c and the
// Jacobian numerator below is unchanged; in float32 the small A, B avoid the
// cancellation that an O(1) origin causes.  Directional derivatives along the
// cell edges are propagated by the product rule from the leaves (forward mode)
// instead of by differencing coefficients, so they keep their own precision.
//
// Irradiance (Eqs. eq_dwda, eq_irr_term3a):
//   det(d u_k / d mu) = M / Q^3,  M = Q (A1 B2 - A2 B1) - B (A1 Q2 - A2 Q1) - A (Q1 B2 - Q2 B1)
//   E = I0 |(p10 - x0).N1| |det A_cell| |Q|^3 s^(-3/2) / (|N_k| |M|),  s = d0.d0
// where s^(-3/2) is replaced by the chord a s + b plus the remainder term
// (1-xi) dlo + xi dhi (Sec. 4.3 "Remainder variables"); the ratio bound of
// Eq. eq_bbound runs over the degree-11 x degree-1 (xi) product domain.
//
// Rounding: every coefficient carries a rigorous error bound (bnb_poly.cuh);
// coefficient intervals, ratio bounds and the chord terms are rounded outward,
// so the float32 result encloses the exact-arithmetic Bernstein bound.  When
// the float32 sign test of Q cannot decide, Q is recomputed in float64 and that
// decides whether the cell is split.
#pragma once
#include <float.h>

#include <algorithm>

#include "bnb_internal.cuh"
#include "bnb_poly.cuh"

namespace bnb {

// ------------------------------------------------------------------ helpers
template <typename T>
__host__ __device__ constexpr T cup(double x) {  // constant rounded up into T (x >= 0)
  return (T)(x * (1.0 + 4.0 * FP<T>::u));
}

template <typename T>
__host__ __device__ constexpr T tiny_pos() {
  return sizeof(T) == 4 ? (T)1e-30 : (T)1e-290;
}

// gamma_k and multinomials as compile-time constants.
template <typename T, int K>
constexpr T GAM = gam<T>(K);
template <typename T, int N, int I>
constexpr T MULT = (T)mult_c(N, I);
template <typename T, int N, int I>
constexpr T MULTUP = cup<T>(mult_c(N, I));

__device__ __forceinline__ void load_tri(const float4* __restrict__ tri, int t, float (&p)[3][3], float (&n)[3][3]) {
  const float4* b = tri + (int64_t)t * kTriF4;
  const float4 a0 = __ldg(b), a1 = __ldg(b + 1), a2 = __ldg(b + 2), a3 = __ldg(b + 3), a4 = __ldg(b + 4);
  p[0][0] = a0.x; p[0][1] = a0.y; p[0][2] = a0.z; p[1][0] = a0.w;
  p[1][1] = a1.x; p[1][2] = a1.y; p[2][0] = a1.z; p[2][1] = a1.w;
  p[2][2] = a2.x; n[0][0] = a2.y; n[0][1] = a2.z; n[0][2] = a2.w;
  n[1][0] = a3.x; n[1][1] = a3.y; n[1][2] = a3.z; n[2][0] = a3.w;
  n[2][1] = a4.x; n[2][2] = a4.y;
}

// Corners of cell `id` at `depth` in T1's (u,v): children of (C0,C1,C2) are
// (C0,m01,m02), (m01,C1,m12), (m02,m12,C2), (m12,m02,m01).  Dyadic, exact.
template <typename T>
__device__ __forceinline__ void cell_corners(uint32_t id, int depth, T (&cu)[3], T (&cv)[3]) {
  cu[0] = 0; cu[1] = 1; cu[2] = 0;
  cv[0] = 0; cv[1] = 0; cv[2] = 1;
  for (int d = depth - 1; d >= 0; --d) {
    const int k = (id >> (2 * d)) & 3;
    const T mu01 = (cu[0] + cu[1]) * T(0.5), mv01 = (cv[0] + cv[1]) * T(0.5);
    const T mu02 = (cu[0] + cu[2]) * T(0.5), mv02 = (cv[0] + cv[2]) * T(0.5);
    const T mu12 = (cu[1] + cu[2]) * T(0.5), mv12 = (cv[1] + cv[2]) * T(0.5);
    if (k == 0) { cu[1] = mu01; cv[1] = mv01; cu[2] = mu02; cv[2] = mv02; }
    else if (k == 1) { cu[0] = mu01; cv[0] = mv01; cu[2] = mu12; cv[2] = mv12; }
    else if (k == 2) { cu[0] = mu02; cv[0] = mv02; cu[1] = mu12; cv[1] = mv12; }
    else { cu[0] = mu12; cv[0] = mv12; cu[1] = mu02; cv[1] = mv02; cu[2] = mu01; cv[2] = mv01; }
  }
}

// Corner k of a degree-1 form: (1,0,0) -> 0, (0,1,0) -> 2, (0,0,1) -> 1.
__device__ __forceinline__ constexpr int corner_idx(int k) { return k == 0 ? 0 : (k == 1 ? 2 : 1); }

// ------------------------------------------------------------------ leaves
// ------------------------------------------------------------------ float-float helpers
// Error-free transformations (Knuth TwoSum; FMA-based TwoProd) for the few constants whose
// computation cancels: the reflected direction at the triangle's first vertex.
template <typename T>
struct FF {
  T hi, lo;
};
template <typename T>
__device__ __forceinline__ FF<T> two_sum(T a, T b) {
  const T s = a + b;
  const T bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
template <typename T>
__device__ __forceinline__ FF<T> two_prod(T a, T b) {
  const T p = a * b;
  return {p, FP<T>::fma_rn(a, b, -p)};
}
template <typename T>
__device__ __forceinline__ FF<T> ff_norm(T hi, T lo) {  // fast two-sum renormalization
  const T s = hi + lo;
  return {s, lo - (s - hi)};
}
template <typename T>
__device__ __forceinline__ FF<T> ff_add(FF<T> x, FF<T> y) {
  FF<T> s = two_sum(x.hi, y.hi);
  return ff_norm(s.hi, s.lo + (x.lo + y.lo));
}
template <typename T>
__device__ __forceinline__ FF<T> ff_mul(FF<T> x, FF<T> y) {
  FF<T> p = two_prod(x.hi, y.hi);
  return ff_norm(p.hi, p.lo + FP<T>::fma_rn(x.hi, y.lo, x.lo * y.hi));
}
template <typename T>
__device__ __forceinline__ FF<T> ff_of(T a) {
  return {a, T(0)};
}

// ------------------------------------------------------------------ leaves
// Every leaf is expanded around the triangle's first vertex p0 and first normal n0:
//   x1 = p0 + XL,  n1 = n0 + S,  d0 = x1 - x0 = r0 + XL  (r0 = p0 - x0),
// with XL, S degree-1 forms whose coefficients are O(cell size).  Big constants are handled
// in float-float (below); only small quantities are rounded in working precision.
template <typename T>
struct Leaves {
  TP<T, 1> XL[3], S[3], N[3], D0[3];
  TP<T, 0> DX[2][3], DN[2][3];
  T n0[3];
  FF<T> r0[3];
};

template <typename T, bool DERIV>
__device__ __forceinline__ void make_leaves(const T (&p)[3][3], const T (&n)[3][3], const T (&x0)[3], const T (&cu)[3],
                                            const T (&cv)[3], Leaves<T>& L) {
  using F = FP<T>;
  constexpr T g3 = GAM<T, 3>, g4 = GAM<T, 4>, uu = (T)FP<T>::u, up2 = (T)(1.0 + 2.0 * FP<T>::u);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T e1 = p[1][c] - p[0][c], e2 = p[2][c] - p[0][c];
    const T f1 = n[1][c] - n[0][c], f2 = n[2][c] - n[0][c];
    T xm = T(0), sm = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      L.XL[c].c[corner_idx(k)] = F::fma_rn(cv[k], e2, cu[k] * e1);
      L.S[c].c[corner_idx(k)] = F::fma_rn(cv[k], f2, cu[k] * f1);
      xm = fmax(xm, F::fma_ru(fabs(cu[k]), fabs(e1), F::mul_ru(fabs(cv[k]), fabs(e2))));
      sm = fmax(sm, F::fma_ru(fabs(cu[k]), fabs(f1), F::mul_ru(fabs(cv[k]), fabs(f2))));
    }
    L.XL[c].B = F::mul_ru(xm, up2);
    L.XL[c].E = F::mul_ru(g3, xm);
    L.S[c].B = F::mul_ru(sm, up2);
    L.S[c].E = F::mul_ru(g3, sm);
    L.n0[c] = n[0][c];
    L.r0[c] = two_sum(p[0][c], -x0[c]);  // exact
    // rounded full leaves (used where no cancellation follows)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      L.N[c].c[i] = n[0][c] + L.S[c].c[i];
      L.D0[c].c[i] = L.r0[c].hi + L.XL[c].c[i];
    }
    L.N[c].B = F::add_ru(fabs(n[0][c]), L.S[c].B);
    L.N[c].E = F::add_ru(L.S[c].E, F::mul_ru(uu, F::add_ru(L.N[c].B, L.S[c].E)));
    const T r0m = F::add_ru(fabs(L.r0[c].hi), fabs(L.r0[c].lo));
    L.D0[c].B = F::add_ru(r0m, L.XL[c].B);
    L.D0[c].E = F::add_ru(F::add_ru(L.XL[c].E, fabs(L.r0[c].lo)),
                          F::mul_ru(uu, F::add_ru(F::add_ru(fabs(L.r0[c].hi), L.XL[c].B), L.XL[c].E)));
    if constexpr (DERIV) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const T du = cu[j + 1] - cu[0], dv = cv[j + 1] - cv[0];  // exact
        L.DX[j][c].c[0] = F::fma_rn(du, e1, dv * e2);
        L.DN[j][c].c[0] = F::fma_rn(du, f1, dv * f2);
        const T mx = F::fma_ru(fabs(du), fabs(e1), F::mul_ru(fabs(dv), fabs(e2)));
        const T mn = F::fma_ru(fabs(du), fabs(f1), F::mul_ru(fabs(dv), fabs(f2)));
        L.DX[j][c].B = F::mul_ru(mx, up2);
        L.DX[j][c].E = F::mul_ru(g4, mx);
        L.DN[j][c].B = F::mul_ru(mn, up2);
        L.DN[j][c].E = F::mul_ru(g4, mn);
      }
    }
  }
}

template <typename T, int N>
__device__ __forceinline__ void scale2(TP<T, N>& p) {  // exact doubling
#pragma unroll
  for (int i = 0; i < nc(N); ++i) p.c[i] = p.c[i] * T(2);
  p.B = p.B * T(2);
  p.E = p.E * T(2);
}

// p += c * ONE_N (the constant c in degree-N scaled form: c * C(N;g)); cerr bounds |c - exact|.
template <typename T, int N>
__device__ __forceinline__ void add_const(TP<T, N>& p, T c, T cerr) {
  using F = FP<T>;
  static_for<nc(N)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    p.c[i] = F::fma_rn(c, MULT<T, N, i>, p.c[i]);
  });
  const T mag = F::add_ru(F::add_ru(fabs(c), p.B), p.E);
  p.E = F::add_ru(F::add_ru(p.E, cerr), F::mul_ru((T)FP<T>::u, mag));
  p.B = F::add_ru(F::add_ru(p.B, fabs(c)), cerr);
}

// Round a float-float value carrying a relative float-float error budget to a tracked constant.
template <typename T>
__device__ __forceinline__ void ff_round(FF<T> x, T mag, T& v, T& err) {
  using F = FP<T>;
  v = x.hi + x.lo;
  // |x - exact| <= 16 u^2 mag (a few float-float operations), |v - x| <= u |v|
  const T ffe = F::mul_ru((T)(16.0 * FP<T>::u * FP<T>::u), mag);
  err = F::add_ru(F::add_ru(ffe, F::mul_ru((T)FP<T>::u, fabs(v))), fabs(x.hi + x.lo - v));
}

// ------------------------------------------------------------------ reflected direction
template <typename T>
struct Dir {
  TP<T, 3> DT[3];
  TP<T, 2> DDT[2][3];
};

// d~ = (n.n) d0 - 2 (d0.n) n  (Eq. eq_refr_rational, reflection), expanded around (p0, n0):
//   n.n  = c0 + NV,  NV = 2 n0.S + S.S        (c0 = n0.n0)
//   d0.n = k0 + DV,  DV = r0.S + n0.XL + XL.S  (k0 = r0.n0)
//   d~_c = [c0 r0_c - 2 k0 n0_c] + c0 XL_c + r0_c NV + NV XL_c - 2 k0 S_c - 2 n0_c DV - 2 DV S_c.
// The bracket (where the reflection cancels) is computed in float-float.
template <typename T, bool DERIV>
__device__ __forceinline__ void reflect_dir(const Leaves<T>& L, Dir<T>& D) {
  using F = FP<T>;
  const T uu = (T)FP<T>::u;
  // float-float constants
  FF<T> c0 = ff_of(T(0)), k0 = ff_of(T(0));
  T c0m = T(0), k0m = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    c0 = ff_add(c0, two_prod(L.n0[c], L.n0[c]));
    k0 = ff_add(k0, ff_mul(L.r0[c], ff_of(L.n0[c])));
    c0m = F::fma_ru(fabs(L.n0[c]), fabs(L.n0[c]), c0m);
    k0m = F::fma_ru(F::add_ru(fabs(L.r0[c].hi), fabs(L.r0[c].lo)), fabs(L.n0[c]), k0m);
  }
  T c0f, c0e, k0f, k0e;
  ff_round(c0, c0m, c0f, c0e);
  ff_round(k0, k0m, k0f, k0e);
  // NV (degree 2) and DV (degree 2)
  TP<T, 2> NV, DV;
  {
    TP<T, 1> n1, d1;
    tp_zero(n1);
    tp_zero(d1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac_s(n1, T(2) * L.n0[c], L.S[c]);
      mac_s(d1, L.n0[c], L.XL[c]);
      mac(d1, tconst<T>(L.r0[c].hi, fabs(L.r0[c].lo)), L.S[c]);
    }
    elevate(NV, n1);
    elevate(DV, d1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(NV, L.S[c], L.S[c]);
      mac(DV, L.XL[c], L.S[c]);
    }
  }
  const TP<T, 0> c0t = tconst<T>(c0f, c0e), k2t = tconst<T>(T(2) * k0f, T(2) * k0e);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // constant part K_c = c0 r0_c - 2 k0 n0_c in float-float
    const FF<T> K = ff_add(ff_mul(c0, L.r0[c]), ff_mul(ff_of(T(-2) * L.n0[c]), k0));
    const T Km = F::fma_ru(c0m, F::add_ru(fabs(L.r0[c].hi), fabs(L.r0[c].lo)), F::mul_ru(T(2), F::mul_ru(k0m, fabs(L.n0[c]))));
    T Kf, Ke;
    ff_round(K, Km, Kf, Ke);
    // variable part, by degree
    TP<T, 1> V1;
    tp_zero(V1);
    mac(V1, c0t, L.XL[c]);
    mac<true>(V1, k2t, L.S[c]);
    TP<T, 2> V2;
    elevate(V2, V1);
    mac(V2, tconst<T>(L.r0[c].hi, fabs(L.r0[c].lo)), NV);
    mac_s<true>(V2, T(2) * L.n0[c], DV);
    elevate(D.DT[c], V2);
    mac(D.DT[c], NV, L.XL[c]);
    TP<T, 2> DV2 = DV;
    scale2(DV2);
    mac<true>(D.DT[c], DV2, L.S[c]);
    add_const(D.DT[c], Kf, Ke);
    renorm(D.DT[c]);
  }
  if constexpr (DERIV) {
    // full n.n and 2 d0.n (rounded; their error is O(u) of their size) for the derivative chain
    TP<T, 2> NN = NV, DN2 = DV;
    add_const(NN, c0f, c0e);
    add_const(DN2, k0f, k0e);
    scale2(DN2);
    (void)uu;
    // the two edge directions j = 0, 1 run as pairs
    TP<T, 1> DNN[2], DDN2[2];  // D(n.n) = 2 n.Dn ; 2 D(d0.n)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      tp_zero(DNN[j]);
      tp_zero(DDN2[j]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac2(DNN[0], L.N[c], L.DN[0][c], DNN[1], L.N[c], L.DN[1][c]);
      mac2(DDN2[0], L.N[c], L.DX[0][c], DDN2[1], L.N[c], L.DX[1][c]);
      mac2(DDN2[0], L.D0[c], L.DN[0][c], DDN2[1], L.D0[c], L.DN[1][c]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      scale2(DNN[j]);
      scale2(DDN2[j]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      tp_zero(D.DDT[0][c]);
      tp_zero(D.DDT[1][c]);
      mac2(D.DDT[0][c], DNN[0], L.D0[c], D.DDT[1][c], DNN[1], L.D0[c]);
      mac2(D.DDT[0][c], NN, L.DX[0][c], D.DDT[1][c], NN, L.DX[1][c]);
      mac2<true>(D.DDT[0][c], DDN2[0], L.N[c], D.DDT[1][c], DDN2[1], L.N[c]);
      mac2<true>(D.DDT[0][c], DN2, L.DN[0][c], D.DDT[1][c], DN2, L.DN[1][c]);
      renorm(D.DDT[0][c]);
      renorm(D.DDT[1][c]);
    }
  }
}

// Tracked constant vector g = e2 x e1 (receiver) and cross products with exact vectors.
template <typename T>
__device__ __forceinline__ TP<T, 0> cross_comp(T a1, T b2, T a2, T b1) {  // a1*b2 - a2*b1
  using F = FP<T>;
  const T v = F::fma_rn(a1, b2, -(a2 * b1));
  const T mag = F::fma_ru(fabs(a1), fabs(b2), F::mul_ru(fabs(a2), fabs(b1)));
  return tconst<T>(v, F::mul_ru(GAM<T, 2>, mag));
}

template <typename T>
__device__ __forceinline__ TP<T, 3> q_of(const Dir<T>& D, const T (&e1)[3], const T (&e2)[3]) {
  TP<T, 0> g[3] = {cross_comp<T>(e2[1], e1[2], e2[2], e1[1]), cross_comp<T>(e2[2], e1[0], e2[0], e1[2]),
                   cross_comp<T>(e2[0], e1[1], e2[1], e1[0])};
  TP<T, 3> Q;
  tp_zero(Q);
#pragma unroll
  for (int c = 0; c < 3; ++c) mac(Q, D.DT[c], g[c]);
  return Q;
}

// ------------------------------------------------------------------ ratio helpers
// Track min/max of p/q over a coefficient with intervals [pl,ph] / [ql,qh], ql > 0, given
// Reciprocals of positive interval ends for the ratio bounds, each within the relative error
// FP<T>::rcp_rel of the exact value.  rcp_hi(x) stands for 1/x where an upper-side value is needed
// (x is clamped to rcp_big, which can only enlarge the result); rcp_lo(x) where a lower-side value
// is needed (0 above rcp_big).
template <typename T>
__device__ __forceinline__ T rcp_hi(T x) {
  return FP<T>::rcp_fast(fmin(x, (T)FP<T>::rcp_big));
}
template <typename T>
__device__ __forceinline__ T rcp_lo(T x) {
  return x > (T)FP<T>::rcp_big ? T(0) : FP<T>::rcp_fast(x);
}
// rl = rcp_hi(ql), rh = rcp_lo(qh).  Each ratio carries the reciprocal's error and one product
// rounding; the caller widens the final min/max by the relative factor of widen_lo / widen_hi.
template <typename T>
__device__ __forceinline__ void ratio_acc(T pl, T ph, T rl, T rh, T& mn, T& mx) {
  mn = fmin(mn, pl * (pl >= T(0) ? rh : rl));
  mx = fmax(mx, ph * (ph >= T(0) ? rl : rh));
}
// A ratio p = fl(n * r) with r = (1/d)(1 + d1), |d1| <= rcp_rel, satisfies
// n/d = p / ((1 + d1)(1 + d2)), |d2| <= u: the exact ratio lies within the relative distance
// rcp_rel + u + (rcp_rel + u)^2 < rcp_rel + 1.5 u of p.
template <typename T>
constexpr T kWiden = (T)(FP<T>::rcp_rel + 1.5 * FP<T>::u);
template <typename T>
__device__ __forceinline__ T widen_lo(T x) {
  return FP<T>::fma_rd(-fabs(x), kWiden<T>, x);
}
template <typename T>
__device__ __forceinline__ T widen_hi(T x) {
  return FP<T>::fma_ru(fabs(x), kWiden<T>, x);
}

// Interval of coefficient i of a tracked polynomial (scaled form).
template <int i, typename T, int N>
__device__ __forceinline__ void coef_iv(const TP<T, N>& p, T& lo, T& hi) {
  constexpr T C = MULTUP<T, N, i>;
  lo = FP<T>::fma_rd(-p.E, C, p.c[i]);
  hi = FP<T>::fma_ru(p.E, C, p.c[i]);
}

// Compile-time coefficient G of a degree-M x degree-2 product, summing over the 6 degree-2 terms.
template <int M, int G, int Bi>
struct Term2 {
  static constexpr int gg1 = g1_of(M + 2, G) - g1_of(2, Bi);
  static constexpr int gg2 = g2_of(M + 2, G) - g2_of(2, Bi);
  static constexpr bool valid = gg1 >= 0 && gg2 >= 0 && gg1 + gg2 <= M;
  static constexpr int a = valid ? idx_of(M, gg1, gg2) : 0;
  static constexpr double c2 = mult_c(2, Bi);
};

template <bool LO, typename T, int M, int G, int... Bi>
__device__ __forceinline__ void coef3(const T* __restrict__ p, const T* __restrict__ f0, const T* __restrict__ f1,
                                      const T* __restrict__ m, T& n0, T& n1, T& mm, std::integer_sequence<int, Bi...>) {
  // n0 = sum f0[b] p[G-b] (only when LO), n1 = sum f1[b] p[G-b], mm = sum C(2;b) m[G-b]
  n0 = T(0);
  n1 = T(0);
  mm = T(0);
  ((Term2<M, G, Bi>::valid ? (n0 = LO ? FP<T>::fma_rn(f0[Bi], p[Term2<M, G, Bi>::a], n0) : n0,
                              n1 = FP<T>::fma_rn(f1[Bi], p[Term2<M, G, Bi>::a], n1),
                              mm = FP<T>::fma_rn((T)Term2<M, G, Bi>::c2, m[Term2<M, G, Bi>::a], mm), 0)
                           : 0),
   ...);
}

template <typename T>
struct IrrAcc {
  T eh_mx, el_mn;  // ratio max (xi = 1 side) and min (xi = 0 side)
  T eh_in;         // lower end of the enclosure of the exact max (inner interval ends)
  bool unbounded;
  T EN0, EN1, EM;  // coefficient error bounds (classical)
};

// LO: also the lower irradiance bound (xi = 0 side) and the inner end of the enclosure of the
// exact upper bound; both are skipped when the caller does not ask for e_lo / e_hi_min.
template <bool LO, typename T, int G>
__device__ __forceinline__ void irr_step(const TP<T, 9>& Q3, const T (&F0)[6], const T (&F1)[6], const TP<T, 9>& M,
                                         IrrAcc<T>& acc) {
  T n0, n1, mm;
  coef3<LO, T, 9, G>(Q3.c, F0, F1, M.c, n0, n1, mm, std::make_integer_sequence<int, 6>{});
  constexpr T C = MULTUP<T, 11, G>;
  const T ml = FP<T>::fma_rd(-acc.EM, C, mm), mh = FP<T>::fma_ru(acc.EM, C, mm);
  if (!(ml > tiny_pos<T>())) acc.unbounded = true;
  const T n1h = FP<T>::fma_ru(acc.EN1, C, n1);
  if constexpr (LO) {
    const T rl = rcp_hi(ml), rh = rcp_lo(mh);
    acc.eh_mx = fmax(acc.eh_mx, n1h * (n1h >= T(0) ? rl : rh));
    const T n0l = FP<T>::fma_rd(-acc.EN0, C, n0);
    acc.el_mn = fmin(acc.el_mn, n0l * (n0l >= T(0) ? rh : rl));
    const T n1l = FP<T>::fma_rd(-acc.EN1, C, n1);
    acc.eh_in = fmax(acc.eh_in, n1l * (n1l >= T(0) ? rh : rl));
  } else {
    // only the reciprocal the numerator's sign selects: rcp_hi(ml) for n1h >= 0, rcp_lo(mh) below
    const bool pos = n1h >= T(0);
    T r = FP<T>::rcp_fast(fmin(pos ? ml : mh, (T)FP<T>::rcp_big));
    if (!pos && mh > (T)FP<T>::rcp_big) r = T(0);
    acc.eh_mx = fmax(acc.eh_mx, n1h * r);
  }
}

template <bool LO, typename T, int... G>
__device__ __forceinline__ void irr_all(const TP<T, 9>& Q3, const T (&F0)[6], const T (&F1)[6], const TP<T, 9>& M,
                                        IrrAcc<T>& acc, std::integer_sequence<int, G...>) {
  (irr_step<LO, T, G>(Q3, F0, F1, M, acc), ...);
}


// irradiance term G with the numerator and denominator sums paired: (n1, mm) += (F1[b], C(2;b)) (Q3, M)[G-b]
template <int G, int... Bi>
__device__ __forceinline__ float2 coef3_f2(const float2* __restrict__ QM, const float2 (&FC)[6],
                                           std::integer_sequence<int, Bi...>) {
  float2 acc = make_float2(0.0f, 0.0f);
  ((Term2<9, G, Bi>::valid ? (acc = __ffma2_rn(FC[Bi], QM[Term2<9, G, Bi>::a], acc), 0) : 0), ...);
  return acc;
}

template <int G>
__device__ __forceinline__ void irr_step_f2(const float2* __restrict__ QM, const float2 (&FC)[6], IrrAcc<float>& acc) {
  const float2 nm = coef3_f2<G>(QM, FC, std::make_integer_sequence<int, 6>{});
  const float n1 = nm.x, mm = nm.y;
  constexpr float C = MULTUP<float, 11, G>;
  const float ml = FP<float>::fma_rd(-acc.EM, C, mm), mh = FP<float>::fma_ru(acc.EM, C, mm);
  if (!(ml > tiny_pos<float>())) acc.unbounded = true;
  const float n1h = FP<float>::fma_ru(acc.EN1, C, n1);
  const bool pos = n1h >= 0.0f;
  float r = FP<float>::rcp_fast(fminf(pos ? ml : mh, (float)FP<float>::rcp_big));
  if (!pos && mh > (float)FP<float>::rcp_big) r = 0.0f;
  acc.eh_mx = fmaxf(acc.eh_mx, n1h * r);
}

template <int... G>
__device__ __forceinline__ void irr_all_f2(const float2* __restrict__ QM, const float2 (&FC)[6], IrrAcc<float>& acc,
                                           std::integer_sequence<int, G...>) {
  (irr_step_f2<G>(QM, FC, acc), ...);
}

// Chord of f(s) = s^(-3/2) on [sl, sh] with rigorous remainder bounds dlo <= f - (a s + b) <= dhi.
template <typename T>
__device__ __forceinline__ T f_hi(T s) {  // >= s^(-3/2)
  using F = FP<T>;
  return F::div_ru(T(1), F::mul_rd(s, F::sqrt_rd(s)));
}
template <typename T>
__device__ __forceinline__ T f_lo(T s) {  // <= s^(-3/2)
  using F = FP<T>;
  return F::div_rd(T(1), F::mul_ru(s, F::sqrt_ru(s)));
}

template <typename T>
__device__ __forceinline__ void chord_remainder(T sl, T sh, T& a, T& b, T& dlo, T& dhi) {
  using F = FP<T>;
  if (!(sh > sl * (T)(1.0 + 64.0 * FP<T>::u))) {
    a = T(0);
    b = (f_hi(sl) + f_lo(sh)) * T(0.5);
    dlo = F::add_rd(f_lo(sh), -b);  // f decreasing: f(s) >= f(sh)
    dhi = F::add_ru(f_hi(sl), -b);  // f(s) <= f(sl)
    return;
  }
  const T fl = (f_hi(sl) + f_lo(sl)) * T(0.5), fh = (f_hi(sh) + f_lo(sh)) * T(0.5);
  a = (fh - fl) / (sh - sl);
  b = F::fma_rn(-a, sl, fl);
  // f - r is convex: its maximum is at an end point ...
  const T g_sl = F::add_ru(f_hi(sl), -F::fma_rd(a, sl, b));
  const T g_sh = F::add_ru(f_hi(sh), -F::fma_rd(a, sh, b));
  dhi = fmax(g_sl, g_sh);
  // ... and it lies above its tangent at t (near the stationary point f'(t) = a).
  T t;
  if constexpr (sizeof(T) == 4) t = powf(-a / 1.5f, -0.4f); else t = pow(-a / 1.5, -0.4);
  t = fmin(fmax(t, sl), sh);
  const T gt = F::add_rd(f_lo(t), -F::fma_ru(a, t, b));
  const T fp_lo = F::mul_rd(T(-1.5), F::div_ru(f_hi(t), t));  // f'(t) = -1.5 f(t) / t
  const T fp_hi = F::mul_ru(T(-1.5), F::div_rd(f_lo(t), t));
  const T gp_lo = F::add_rd(fp_lo, -a), gp_hi = F::add_ru(fp_hi, -a);
  const T dl = F::add_rd(sl, -t), dh = F::add_ru(sh, -t);  // dl <= 0 <= dh
  const T m = fmin(fmin(F::mul_rd(gp_lo, dl), F::mul_rd(gp_lo, dh)), fmin(F::mul_rd(gp_hi, dl), F::mul_rd(gp_hi, dh)));
  dlo = F::add_rd(gt, m);
  dlo = fmin(dlo, dhi);
}

// ------------------------------------------------------------------ records
// raise_status (bnb_internal.cuh): the record's status word and the device error word

template <typename T>
__device__ __forceinline__ float f_dn(T x) {
  if constexpr (sizeof(T) == 8) return __double2float_rd(x); else return x;
}
template <typename T>
__device__ __forceinline__ float f_up(T x) {
  if constexpr (sizeof(T) == 8) return __double2float_ru(x); else return x;
}

__device__ __forceinline__ void put_rec(const BoundParams& P, int64_t slot, float ul, float uh, float vl, float vh,
                                        float el, float eh, int e, int t, uint32_t id, uint32_t flags,
                                        float eh_min = 0.0f) {
  if (slot < 0) {
    slot = (int64_t)atomicAdd((unsigned long long*)P.count, 1ull);
    if (slot >= P.capacity) {
      raise_status(P.status, BNB_ERR_CAPACITY);
      return;
    }
  }
  P.u_lo[slot] = ul;
  P.u_hi[slot] = uh;
  P.v_lo[slot] = vl;
  P.v_hi[slot] = vh;
  if (P.e_lo) P.e_lo[slot] = el;
  P.e_hi[slot] = eh;
  P.emitter[slot] = e;
  P.tri0[slot] = t;
  P.tri1[slot] = -1;
  P.cell[slot] = id;
  P.flags[slot] = flags;
  if (P.e_hi_min) P.e_hi_min[slot] = eh_min;
}

// Adaptive subdivision (Sec. 6.1 "Domain subdivision"): a live cell with a bounded box above the
// depth limit is queued for its four children (its record becomes SPLIT) unless its receiver box
// has area below sigma or E_hi < alpha E_lo.  The decision is taken on the float32 values the
// record stores, with round-to-nearest differences and products.  Returns true when queued.
__device__ __forceinline__ bool adapt_split(const BoundParams& P, int64_t slot, float ul, float uh, float vl, float vh,
                                            float el, float eh, int e, int t, uint32_t id, int depth, uint32_t flags) {
  if (depth >= P.adapt_depth) return false;
  if (__fmul_rn(__fsub_rn(uh, ul), __fsub_rn(vh, vl)) < P.sigma) return false;
  if (eh < __fmul_rn(P.alpha, el)) return false;
  const int64_t qi = (int64_t)atomicAdd((unsigned long long*)P.q_out_count, 1ull);
  if (qi < P.q_cap) {
    P.q_out[qi] = SplitItem{e, t, id, depth};
  } else {
    raise_status(P.status, BNB_ERR_CAPACITY);
  }
  put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, (flags & ~(BNB_CELL_LIVE | BNB_CELL_FOLD)) | BNB_CELL_SPLIT);
  return true;
}

// Reciprocal rule after the split limit (Sec. 4.1): with the denominator of mixed sign, bound
// q/p when p has one sign; p/q then lies in 1/[rl, rh]; return the hull of that set and [0,1].
template <typename T>
__device__ void recip01(const TP<T, 4>& P4, const TP<T, 4>& Q4, int sp, T& lo, T& hi) {
  using F = FP<T>;
  lo = T(0);
  hi = T(1);
  if (sp == 0) return;  // universal set
  T mn = F::inf(), mx = -F::inf();
  bool bad = false;
  static_for<nc(4)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr T C = MULTUP<T, 4, i>;
    T pl = F::fma_rd(-P4.E, C, P4.c[i]), ph = F::fma_ru(P4.E, C, P4.c[i]);
    T ql = F::fma_rd(-Q4.E, C, Q4.c[i]), qh = F::fma_ru(Q4.E, C, Q4.c[i]);
    if (sp < 0) {  // divide by the positive -p
      T t = pl;
      pl = -ph;
      ph = -t;
      t = ql;
      ql = -qh;
      qh = -t;
    }
    if (!(pl > tiny_pos<T>())) bad = true;
    mn = fmin(mn, F::div_rd(ql, ql >= T(0) ? ph : pl));
    mx = fmax(mx, F::div_ru(qh, qh >= T(0) ? pl : ph));
  });
  if (bad) return;  // universal set
  // r = q/p in [mn, mx]; p/q = 1/r
  T L = T(1), H = T(0);
  auto add = [&](T a, T b) {
    a = fmax(a, T(0));
    b = fmin(b, T(1));
    if (a <= b) {
      L = fmin(L, a);
      H = fmax(H, b);
    }
  };
  if (mn > T(0) || mx < T(0)) {
    add(F::div_rd(T(1), mx), F::div_ru(T(1), mn));
  } else {
    add(-F::inf(), mn < T(0) ? F::div_ru(T(1), mn) : -F::inf());
    add(mx > T(0) ? F::div_rd(T(1), mx) : F::inf(), F::inf());
  }
  lo = L;
  hi = H;
}

// ------------------------------------------------------------------ one cell
// K = I0 |(p10 - x0).N1| |det A_cell| / |N_k| (|det A_cell| = 4^-depth, exact), rounded outward:
// the constant factor of the path irradiance (Eq. eq_dwda) on a cell.
template <typename T>
__device__ __forceinline__ void cell_K(const T (&p)[3][3], const T (&x0)[3], const T (&e1)[3], const T (&e2)[3],
                                       float I0f, int depth, T& Klo, T& Khi) {
  using F = FP<T>;
  T a[3], b[3], r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a[c] = p[1][c] - p[0][c];
    b[c] = p[2][c] - p[0][c];
    r[c] = p[0][c] - x0[c];
  }
  const T N1[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const T C1 = r[0] * N1[0] + r[1] * N1[1] + r[2] * N1[2];
  T mag = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int i = (c + 1) % 3, j = (c + 2) % 3;
    mag = F::fma_ru(fabs(r[c]), F::fma_ru(fabs(a[i]), fabs(b[j]), F::mul_ru(fabs(a[j]), fabs(b[i]))), mag);
  }
  const T cerr = F::mul_ru(GAM<T, 10>, mag);
  const T C1hi = F::add_ru(fabs(C1), cerr), C1lo = fmax(F::add_rd(fabs(C1), -cerr), T(0));
  T nkl2 = T(0), nkh2 = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int i = (c + 1) % 3, j = (c + 2) % 3;
    const T v = e1[i] * e2[j] - e1[j] * e2[i];
    const T err = F::mul_ru(GAM<T, 2>, F::fma_ru(fabs(e1[i]), fabs(e2[j]), F::mul_ru(fabs(e1[j]), fabs(e2[i]))));
    const T lo = fmax(F::add_rd(fabs(v), -err), T(0)), hi = F::add_ru(fabs(v), err);
    nkl2 = F::fma_rd(lo, lo, nkl2);
    nkh2 = F::fma_ru(hi, hi, nkh2);
  }
  const T nkl = F::sqrt_rd(nkl2), nkh = F::sqrt_ru(nkh2);
  T detA;
  if constexpr (sizeof(T) == 4) detA = ldexpf(1.0f, -2 * depth); else detA = ldexp(1.0, -2 * depth);
  const T I0 = (T)I0f;
  Khi = F::div_ru(F::mul_ru(F::mul_ru(I0, C1hi), detA), nkl);
  Klo = F::div_rd(F::mul_rd(F::mul_rd(I0, C1lo), detA), nkh);
}

static __device__ __noinline__ void process_cell_fp64(const BoundParams& P, int e, int t, uint32_t id, int depth,
                                                      int64_t slot);

template <typename T>
__device__ __forceinline__ void process_cell(const BoundParams& P, int e, int t, uint32_t id, int depth, int64_t slot,
                                             uint32_t extra_flags = 0) {
  using F = FP<T>;
  float pf[3][3], nf[3][3];
  load_tri(P.tri, t, pf, nf);
  const float x0f[3] = {__ldg(P.ex + e), __ldg(P.ey + e), __ldg(P.ez + e)};
  const float I0f = __ldg(P.ei + e);
  T p[3][3], n[3][3], x0[3], e1[3], e2[3], rp0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      p[a][b] = (T)pf[a][b];
      n[a][b] = (T)nf[a][b];
    }
    x0[a] = (T)x0f[a];
    e1[a] = (T)P.re1[a];
    e2[a] = (T)P.re2[a];
    rp0[a] = (T)P.rp0[a];
  }
  const uint32_t dflag = ((uint32_t)depth << BNB_CELL_DEPTH_SHIFT) | extra_flags;
  T cu[3], cv[3];
  cell_corners<T>(id, depth, cu, cv);

  // Receiver origin: the hit of the centroid ray, rounded to 2^-16 (any finite value is valid).
  T uc, vc;
  {
    T xc[3], ncn[3], d[3];
    const T third = T(1) / T(3);
    const T w1 = (cu[0] + cu[1] + cu[2]) * third, w2 = (cv[0] + cv[1] + cv[2]) * third, w0 = T(1) - w1 - w2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xc[c] = w0 * p[0][c] + w1 * p[1][c] + w2 * p[2][c];
      ncn[c] = w0 * n[0][c] + w1 * n[1][c] + w2 * n[2][c];
      d[c] = xc[c] - x0[c];
    }
    const T nn = ncn[0] * ncn[0] + ncn[1] * ncn[1] + ncn[2] * ncn[2];
    const T dn = d[0] * ncn[0] + d[1] * ncn[1] + d[2] * ncn[2];
    T dt[3], w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dt[c] = nn * d[c] - T(2) * dn * ncn[c];
      w[c] = xc[c] - rp0[c];
    }
    const T g0 = e2[1] * e1[2] - e2[2] * e1[1], g1 = e2[2] * e1[0] - e2[0] * e1[2], g2 = e2[0] * e1[1] - e2[1] * e1[0];
    const T Qc = dt[0] * g0 + dt[1] * g1 + dt[2] * g2;
    const T hu0 = e2[1] * w[2] - e2[2] * w[1], hu1 = e2[2] * w[0] - e2[0] * w[2], hu2 = e2[0] * w[1] - e2[1] * w[0];
    const T hv0 = w[1] * e1[2] - w[2] * e1[1], hv1 = w[2] * e1[0] - w[0] * e1[2], hv2 = w[0] * e1[1] - w[1] * e1[0];
    uc = (dt[0] * hu0 + dt[1] * hu1 + dt[2] * hu2) / Qc;
    vc = (dt[0] * hv0 + dt[1] * hv1 + dt[2] * hv2) / Qc;
    if (!(fabs(uc) < T(4))) uc = T(0.5);
    if (!(fabs(vc) < T(4))) vc = T(0.5);
    uc = rint(uc * T(65536)) * T(1.0 / 65536);
    vc = rint(vc * T(65536)) * T(1.0 / 65536);
  }

  Leaves<T> L;
  make_leaves<T, true>(p, n, x0, cu, cv, L);
  Dir<T> D;
  reflect_dir<T, true>(L, D);
  TP<T, 3> Q = q_of<T>(D, e1, e2);
  renorm(Q);
  uint32_t flags = dflag;
  const int sq = cert_sign(Q);
  if constexpr (sizeof(T) == 4) {
    // The float32 intervals cannot decide the denominator's sign: the split decision, the
    // reciprocal rule and the bounds of this cell are taken in float64 (flag QSIGN_FP64).
    if (sq == 0) {
      process_cell_fp64(P, e, t, id, depth, slot);
      return;
    }
  }
  // Receiver-side linear terms: W = x1 - p', h_u = e2 x W, h_v = W x e1 and their derivatives.
  TP<T, 1> hu[3], hv[3];
  TP<T, 0> Dhu[2][3], Dhv[2][3];
  auto build_h = [&](T ou, T ov) {
    constexpr T g2e = GAM<T, 2>, uu = (T)FP<T>::u;
    TP<T, 1> W[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // q = p_{1,0} - p' with p' = p_k0 + ou e_k1 + ov e_k2 (p' exact by definition, computed with error perr)
      const T pc = F::fma_rn(ov, e2[c], F::fma_rn(ou, e1[c], rp0[c]));
      const T pmag = F::fma_ru(fabs(ov), fabs(e2[c]), F::fma_ru(fabs(ou), fabs(e1[c]), fabs(rp0[c])));
      const T perr = F::mul_ru(g2e, pmag);
      const T q = p[0][c] - pc;
      const T qerr = F::add_ru(perr, F::mul_ru(uu, F::add_ru(F::add_ru(fabs(p[0][c]), fabs(pc)), perr)));
#pragma unroll
      for (int i = 0; i < 3; ++i) W[c].c[i] = L.XL[c].c[i] + q;
      W[c].B = F::add_ru(F::add_ru(L.XL[c].B, fabs(q)), qerr);
      W[c].E = F::add_ru(F::add_ru(L.XL[c].E, qerr),
                         F::mul_ru(uu, F::add_ru(F::add_ru(L.XL[c].B, L.XL[c].E), F::add_ru(fabs(q), qerr))));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      tp_zero(hu[c]);
      mac_s(hu[c], e2[a], W[b]);
      mac_s<true>(hu[c], e2[b], W[a]);
      tp_zero(hv[c]);
      mac_s(hv[c], e1[b], W[a]);
      mac_s<true>(hv[c], e1[a], W[b]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        tp_zero(Dhu[j][c]);
        mac_s(Dhu[j][c], e2[a], L.DX[j][b]);
        mac_s<true>(Dhu[j][c], e2[b], L.DX[j][a]);
        tp_zero(Dhv[j][c]);
        mac_s(Dhv[j][c], e1[b], L.DX[j][a]);
        mac_s<true>(Dhv[j][c], e1[a], L.DX[j][b]);
      }
    }
  };

  if (sq == 0) {
    // Mixed-sign denominator (Sec. 4.1): reciprocal rule with the literal origin p_k0; a cell
    // whose reciprocal bound misses [0,1]^2 is culled, otherwise split (up to the limit) or,
    // at the limit, kept with that box and an unbounded irradiance.
    build_h(T(0), T(0));
    TP<T, 4> A4, B4;
    tp_zero(A4);
    tp_zero(B4);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(A4, D.DT[c], hu[c]);
      mac(B4, D.DT[c], hv[c]);
    }
    TP<T, 4> Q4;
    elevate(Q4, Q);
    T ul, uh, vl, vh;
    recip01(A4, Q4, cert_sign(A4), ul, uh);
    recip01(B4, Q4, cert_sign(B4), vl, vh);
    if (ul > uh || vl > vh) {
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_CULL_EMPTY);
    } else if (depth < P.max_depth) {
      const int64_t qi = (int64_t)atomicAdd((unsigned long long*)P.q_out_count, 1ull);
      if (qi < P.q_cap) {
        P.q_out[qi] = SplitItem{e, t, id, depth};
      } else {
        raise_status(P.status, BNB_ERR_CAPACITY);
      }
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_SPLIT);
    } else {
      put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id,
              flags | BNB_CELL_LIVE | BNB_CELL_POS_UNBOUNDED);
    }
    return;
  }
  // Normalize the denominator sign (exact negation of every polynomial that scales with d~).
  if (sq < 0) {
    negate(Q);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      negate(D.DT[c]);
      negate(D.DDT[0][c]);
      negate(D.DDT[1][c]);
    }
  }
  build_h(uc, vc);
  // Forward culling: t = Tn / Q with Tn = (W x e1) . e2 = h_v . e2; every path behind x1 -> cull.
  {
    TP<T, 1> Tn;
    tp_zero(Tn);
#pragma unroll
    for (int c = 0; c < 3; ++c) mac_s(Tn, e2[c], hv[c]);
    // Q was normalized by negating d~ only; Tn does not contain d~, so apply the sign here.
    if (sq < 0) negate(Tn);
    if (cert_sign(Tn) < 0) {
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_CULL_BEHIND);
      return;
    }
  }
  TP<T, 4> A, B;
  TP<T, 3> DA[2], DB[2];
  TP<T, 2> DQ[2];
  {
    TP<T, 0> g[3] = {cross_comp<T>(e2[1], e1[2], e2[2], e1[1]), cross_comp<T>(e2[2], e1[0], e2[0], e1[2]),
                     cross_comp<T>(e2[0], e1[1], e2[1], e1[0])};
    tp_zero(A);
    tp_zero(B);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      tp_zero(DA[j]);
      tp_zero(DB[j]);
      tp_zero(DQ[j]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac2(A, D.DT[c], hu[c], B, D.DT[c], hv[c]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        mac2(DA[j], D.DDT[j][c], hu[c], DB[j], D.DDT[j][c], hv[c]);
        mac2(DA[j], D.DT[c], Dhu[j][c], DB[j], D.DT[c], Dhv[j][c]);
      }
      mac2(DQ[0], D.DDT[0][c], g[c], DQ[1], D.DDT[1][c], g[c]);
    }
    renorm(A);
    renorm(B);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      renorm(DA[j]);
      renorm(DB[j]);
      renorm(DQ[j]);
    }
  }
  // Position bound: ratios of degree-4 forms (Q elevated once).
  T ul, uh, vl, vh;
  {
    TP<T, 4> Q4;
    elevate(Q4, Q);
    T umn = F::inf(), umx = -F::inf(), vmn = F::inf(), vmx = -F::inf();
    static_for<nc(4)>([&](auto I) {
      constexpr int i = decltype(I)::value;
      T ql, qh, al, ah, bl, bh;
      coef_iv<i>(Q4, ql, qh);
      coef_iv<i>(A, al, ah);
      coef_iv<i>(B, bl, bh);
      // Q > 0 is certified; a float32 interval reaching down to 0 makes the ratio unbounded
      // on the side of the numerator's sign only.
      const bool open = !(ql > tiny_pos<T>());
      const T rl = open ? F::inf() : rcp_hi(ql), rh = rcp_lo(qh);
      ratio_acc(al, ah, rl, rh, umn, umx);
      ratio_acc(bl, bh, rl, rh, vmn, vmx);
      if (open) {  // 0 * inf: a zero numerator end stays 0
        if (al == T(0)) umn = fmin(umn, T(0));
        if (ah == T(0)) umx = fmax(umx, T(0));
        if (bl == T(0)) vmn = fmin(vmn, T(0));
        if (bh == T(0)) vmx = fmax(vmx, T(0));
      }
    });
    ul = F::add_rd(uc, widen_lo(umn));
    uh = F::add_ru(uc, widen_hi(umx));
    vl = F::add_rd(vc, widen_lo(vmn));
    vh = F::add_ru(vc, widen_hi(vmx));
    ul = fmax(ul, T(0));
    uh = fmin(uh, T(1));
    vl = fmax(vl, T(0));
    vh = fmin(vh, T(1));
    if (!(ul <= uh) || !(vl <= vh)) {
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_CULL_EMPTY);
      return;
    }
  }
  flags |= BNB_CELL_LIVE;
  if (!P.irradiance) {
    if (!adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, depth, flags))
      put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, flags);
    return;
  }
  // Jacobian numerator M (degree 9):
  //   X = DA1 DB2 - DA2 DB1,  Y = DA1 DQ2 - DA2 DQ1,  Z = DQ1 DB2 - DQ2 DB1,  M = Q X - B Y - A Z.
  // (Q^3 is formed later, next to its use, which keeps fewer forms live at once.)
  TP<T, 9> M, Q3;
  tp_zero(M);
  {
    TP<T, 6> X;
    tp_zero(X);
    mac(X, DA[0], DB[1]);
    mac<true>(X, DA[1], DB[0]);
    renorm(X);
    TP<T, 5> Y, Z;
    tp_zero(Y);
    mac(Y, DA[0], DQ[1]);
    mac<true>(Y, DA[1], DQ[0]);
    renorm(Y);
    tp_zero(Z);
    mac(Z, DQ[0], DB[1]);
    mac<true>(Z, DQ[1], DB[0]);
    renorm(Z);
    mac(M, Q, X);
    // B Y and A Z (the largest products) as one rolled loop, negated copies of B and A
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      TP<T, 4> a = t ? A : B;
      negate(a);
      mac(M, a, t ? Z : Y);
    }
  }
  renorm(M);
  const int sm = cert_sign(M);
  if (sm == 0) {
    if (!adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, depth,
                     flags | BNB_CELL_FOLD))
      put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, flags | BNB_CELL_FOLD);
    return;
  }
  if (sm < 0) negate(M);
  // s = d0.d0 and its range from the classical coefficients.
  TP<T, 2> S;
  tp_zero(S);
#pragma unroll
  for (int c = 0; c < 3; ++c) mac(S, L.D0[c], L.D0[c]);
  renorm(S);
  T sl = F::inf(), sh = T(0);
  static_for<nc(2)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const T cl = S.c[i] * (T)(1.0 / mult_c(2, i));  // exact: C in {1, 2}
    sl = fmin(sl, F::add_rd(cl, -S.E));
    sh = fmax(sh, F::add_ru(cl, S.E));
  });
  if (!(sl > tiny_pos<T>())) {
    if (!adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, depth,
                     flags | BNB_CELL_FOLD))
      put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, flags | BNB_CELL_FOLD);
    return;
  }
  T ca, cb, dlo, dhi;
  chord_remainder<T>(sl, sh, ca, cb, dlo, dhi);
  // F_j = a s + (b + delta_j) (degree 2), j = 0 (delta = dlo), 1 (delta = dhi).
  T F0[6], F1[6];
  T FB, FE0, FE1;
  {
    const T c0 = cb + dlo, c1 = cb + dhi;
    const T uu = (T)FP<T>::u;
    static_for<6>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr T one = MULT<T, 2, i>;
      F0[i] = F::fma_rn(ca, S.c[i], c0 * one);
      F1[i] = F::fma_rn(ca, S.c[i], c1 * one);
    });
    const T as = F::mul_ru(fabs(ca), F::add_ru(S.B, S.E));
    FB = F::add_ru(F::mul_ru(fabs(ca), S.B), F::mul_ru(fmax(fabs(c0), fabs(c1)), (T)(1.0 + 2.0 * FP<T>::u)));
    const T base = F::mul_ru(fabs(ca), S.E);
    FE0 = F::add_ru(F::add_ru(base, F::mul_ru(uu, fabs(c0))), F::mul_ru(GAM<T, 2>, F::add_ru(as, fabs(c0))));
    FE1 = F::add_ru(F::add_ru(base, F::mul_ru(uu, fabs(c1))), F::mul_ru(GAM<T, 2>, F::add_ru(as, fabs(c1))));
  }
  {
    TP<T, 6> Q2;
    tp_zero(Q2);
    mac(Q2, Q, Q);
    renorm(Q2);
    tp_zero(Q3);
    mac(Q3, Q2, Q);
    renorm(Q3);
  }
  IrrAcc<T> acc;
  acc.eh_mx = -F::inf();
  acc.el_mn = F::inf();
  acc.eh_in = -F::inf();
  acc.unbounded = false;
  {
    T rB = T(0), rE = T(0);
    track_mac<6>(rB, rE, Q3.B, Q3.E, FB, FE0);
    acc.EN0 = rE;
    rB = T(0);
    rE = T(0);
    track_mac<6>(rB, rE, Q3.B, Q3.E, FB, FE1);
    acc.EN1 = rE;
    rB = T(0);
    rE = T(0);
    track_mac<6>(rB, rE, M.B, M.E, T(1), T(0));
    acc.EM = rE;
  }
  // uniform across the launch (adaptive subdivision needs E_lo for its ratio test)
  const bool want_lo = P.e_lo != nullptr || P.e_hi_min != nullptr || P.adapt_depth > 0;
  if (want_lo) {
    irr_all<true, T>(Q3, F0, F1, M, acc, std::make_integer_sequence<int, nc(11)>{});
  } else if constexpr (sizeof(T) == 4) {
    float2 QM[nc(9)];
#pragma unroll
    for (int i = 0; i < nc(9); ++i) QM[i] = make_float2(Q3.c[i], M.c[i]);
    float2 FC[6];
    static_for<6>([&](auto I) {
      constexpr int b = decltype(I)::value;
      FC[b] = make_float2(F1[b], (float)mult_c(2, b));
    });
    irr_all_f2(QM, FC, acc, std::make_integer_sequence<int, nc(11)>{});
  } else {
    irr_all<false, T>(Q3, F0, F1, M, acc, std::make_integer_sequence<int, nc(11)>{});
  }
  if (acc.unbounded) {
    if (!adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, depth,
                     flags | BNB_CELL_FOLD))
      put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), 0.f, F::inf(), e, t, id, flags | BNB_CELL_FOLD);
    return;
  }
  // K = I0 |(p10 - x0).N1| |det A_cell| / |N_k|   (|det A_cell| = 4^-depth, exact)
  T Klo, Khi;
  cell_K<T>(p, x0, e1, e2, I0f, depth, Klo, Khi);
  T eh = F::mul_ru(Khi, widen_hi(acc.eh_mx));
  T el = want_lo ? fmax(F::mul_rd(Klo, widen_lo(acc.el_mn)), T(0)) : T(0);
  if (!(eh >= T(0))) eh = F::inf();  // NaN guard: never report a finite bound by accident
  T ehm = fmax(F::mul_rd(Klo, widen_lo(acc.eh_in)), T(0));
  if (!(ehm <= eh)) ehm = T(0);
  if (adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), f_dn(el), f_up(eh), e, t, id, depth, flags)) return;
  put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), f_dn(el), f_up(eh), e, t, id, flags, f_dn(ehm));
}

static __device__ __noinline__ void process_cell_fp64(const BoundParams& P, int e, int t, uint32_t id, int depth,
                                                      int64_t slot) {
  process_cell<double>(P, e, t, id, depth, slot, BNB_CELL_QSIGN_FP64);
}

// ------------------------------------------------------------------ refraction (one vertex)
// Eq. eq_refr_rational, refraction: d~ = eta' ((n.n) d0 - (d0.n) n) - sqrt(beta) n with
// beta = (1 - eta'^2)(n.n)(d0.d0) + eta'^2 (d0.n)^2.  sqrt(beta) is replaced by the remainder
// form a beta + b + (1 - xi) dlo + xi dhi (Sec. 4.3 "Remainder variables"), xi in [0, 1], with
// the chord of sqrt on the cell's range of beta; d~, Q, P_u, P_v are affine in it, so each is
// carried as its two faces xi = 0 and xi = 1 and the ratio bound runs over both.  Normals face
// the incident side.  The irradiance of refraction is not bounded (E_hi = +inf).

// Range [lo, hi] of the classical coefficients of a tracked degree-4 form (rigorous).
template <typename T>
__device__ __forceinline__ void classical_range4(const TP<T, 4>& p, T& lo, T& hi) {
  using F = FP<T>;
  lo = F::inf();
  hi = -F::inf();
  static_for<nc(4)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr T C = MULT<T, 4, i>;  // a small integer, exact
    lo = fmin(lo, F::div_rd(F::fma_rd(-p.E, C, p.c[i]), C));
    hi = fmax(hi, F::div_ru(F::fma_ru(p.E, C, p.c[i]), C));
  });
}

// Chord a x + b of sqrt on [lo, hi] (0 <= lo <= hi, computed in round-to-nearest; any a, b are
// admissible) and a rigorous range [dlo, dhi] of sqrt(x) - (a x + b) over [lo, hi]:
//   dlo: sqrt minus a line is concave, so its minimum is at an end of the interval;
//   dhi: sqrt(x) <= sqrt(x0) + (x - x0) / (2 sqrt(x0)) for any x0 > 0 (tangent of a concave
//        function); that bound minus the line is linear in x, so its maximum is at an end.
//        x0 = 1 / (4 a^2), where the chord's slope is attained, makes the bound tight.
template <typename T>
__device__ __forceinline__ void sqrt_chord(T lo, T hi, T& a, T& b, T& dlo, T& dhi) {
  using F = FP<T>;
  if (!(hi > lo)) {
    a = T(0);
    b = sqrt(hi);
    dlo = F::add_rd(F::sqrt_rd(lo), -b);
    dhi = F::add_ru(F::sqrt_ru(hi), -b);
    return;
  }
  const T sl = sqrt(lo), sh = sqrt(hi);
  a = (sh - sl) / (hi - lo);
  if (!(a > T(0)) || !(a < F::inf())) a = T(0);
  b = sl - a * lo;
  auto low_at = [&](T x) { return F::add_rd(F::sqrt_rd(x), -F::fma_ru(a, x, b)); };
  dlo = fmin(low_at(lo), low_at(hi));
  T x0 = a > T(0) ? T(1) / (T(4) * a * a) : hi;
  x0 = fmin(fmax(x0, lo), hi);
  if (!(x0 > T(0))) x0 = hi;
  const T s0u = F::sqrt_ru(x0), s0d = F::sqrt_rd(x0);
  const T klo = F::div_rd(T(1), F::mul_ru(T(2), s0u)), khi = F::div_ru(T(1), F::mul_rd(T(2), s0d));
  auto up_at = [&](T x) {
    const T dx = F::add_ru(x, -x0);  // >= x - x0
    // g'(x0) in [klo, khi]; an upper bound of g'(x0) (x - x0) on either side of x0
    const T lin = dx >= T(0) ? F::mul_ru(khi, dx) : F::mul_ru(klo, dx);
    return F::add_ru(F::add_ru(s0u, lin), -F::fma_rd(a, x, b));
  };
  dhi = fmax(up_at(lo), up_at(hi));
}

// ---- refraction irradiance (Eqs. eq_dwda, eq_irr_term3a) with W = sqrt(beta) kept as a symbol.
// A pair (p0, p1) stands for p0 + W p1; products reduce W^2 to beta, exact on real paths.  The
// edge derivatives of d~ are scaled by 2W, which clears d sqrt(beta) = d beta / (2W):
//   2W d_j d~ = (-(d_j beta) n - 2 beta d_j n) + W (2 d_j G),   G = eta' ((n.n) d0 - (d0.n) n),
// so the Jacobian numerator of (A/Q, B/Q) built from 2W-scaled derivatives is M' = 4 beta M and
//   E = K |Q|^3 4 beta s^(-3/2) / |M'|.
// W is then replaced by the position bound's remainder form (two xi1 faces) and s^(-3/2) by its
// chord (two xi2 faces); the ratio bound runs over the four faces.
template <typename T, int N>
struct WPr {
  TP<T, N> p0;
  TP<T, N - 2> p1;
};

template <typename T, int N>
__device__ __forceinline__ void wp_zero(WPr<T, N>& r) {
  tp_zero(r.p0);
  tp_zero(r.p1);
}

// r (+/-)= a * b  with W^2 = beta
template <bool NEG = false, typename T, int M, int N>
__device__ __forceinline__ void wp_mac(WPr<T, M + N>& r, const WPr<T, M>& a, const WPr<T, N>& b, const TP<T, 4>& beta) {
  mac<NEG>(r.p0, a.p0, b.p0);
  TP<T, M + N - 4> t;
  tp_zero(t);
  mac(t, a.p1, b.p1);
  renorm(t);
  mac<NEG>(r.p0, t, beta);
  mac<NEG>(r.p1, a.p0, b.p1);
  mac<NEG>(r.p1, a.p1, b.p0);
}

// r += a * q for a plain form q
template <typename T, int M, int N>
__device__ __forceinline__ void wp_mac_p(WPr<T, M + N>& r, const WPr<T, M>& a, const TP<T, N>& q) {
  mac(r.p0, a.p0, q);
  mac(r.p1, a.p1, q);
}

template <typename T, int N>
__device__ __forceinline__ void wp_negate(WPr<T, N>& r) {  // exact: coefficients only
  negate(r.p0);
  negate(r.p1);
}

template <typename T, int N>
__device__ __forceinline__ void wp_renorm(WPr<T, N>& r) {
  renorm(r.p0);
  renorm(r.p1);
}

// The face p0 + W_j p1 of a pair (degree N + 2).
template <typename T, int N>
__device__ __forceinline__ void wp_face(TP<T, N + 2>& r, const WPr<T, N>& a, const TP<T, 4>& Wj) {
  TP<T, N + 1> e1;
  elevate(e1, a.p0);
  elevate(r, e1);
  mac(r, Wj, a.p1);
  renorm(r);
}

template <typename T>
__device__ __forceinline__ void refract_irradiance(const Leaves<T>& L, const TP<T, 2>& NN, const TP<T, 2>& DN,
                                                   const TP<T, 2>& SS, const TP<T, 4>& beta, T eta,
                                                   const TP<T, 3> (&TG3)[3], const TP<T, 1> (&hu)[3],
                                                   const TP<T, 1> (&hv)[3], const TP<T, 0> (&g)[3], const T (&e1)[3],
                                                   const T (&e2)[3], int sq, T ca, T cb, T dlo, T dhi, T Klo, T Khi,
                                                   T& el, T& eh, uint32_t& fold) {
  using F = FP<T>;
  const T uu = (T)FP<T>::u;
  const T e2v = eta * eta, e2err = F::mul_ru(uu, e2v);
  const T c1 = T(1) - e2v, c1err = F::add_ru(e2err, F::mul_ru(uu, fabs(c1)));
  // d~ pairs and their 2W-scaled edge derivatives
  WPr<T, 3> dt[3];
  WPr<T, 4> Dt[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dt[c].p0 = TG3[c];
    tp_zero(dt[c].p1);
    mac_s<true>(dt[c].p1, T(1), L.N[c]);
  }
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    // d(n.n) = 2 n.dn, d(d0.n) = dx.n + d0.dn, d(d0.d0) = 2 d0.dx   (degree 1)
    TP<T, 1> dNN, dDN, dSS;
    tp_zero(dNN);
    tp_zero(dDN);
    tp_zero(dSS);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(dNN, L.N[c], L.DN[j][c]);
      mac(dDN, L.N[c], L.DX[j][c]);
      mac(dDN, L.D0[c], L.DN[j][c]);
      mac(dSS, L.D0[c], L.DX[j][c]);
    }
    scale2(dNN);
    scale2(dSS);
    // d beta = (1 - eta^2)(d(n.n) s + (n.n) d s) + 2 eta^2 (d0.n) d(d0.n)   (degree 3)
    TP<T, 3> dB, t1;
    tp_zero(t1);
    mac(t1, dNN, SS);
    mac(t1, NN, dSS);
    renorm(t1);
    tp_zero(dB);
    mac(dB, tconst<T>(c1, c1err), t1);
    TP<T, 3> t2;
    tp_zero(t2);
    mac(t2, DN, dDN);
    scale2(t2);
    mac(dB, tconst<T>(e2v, e2err), t2);
    renorm(dB);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // d G_c = eta' (d(n.n) d0_c + (n.n) dx_c - d(d0.n) n_c - (d0.n) dn_c)   (degree 2)
      TP<T, 2> dG, dGe;
      tp_zero(dG);
      mac(dG, dNN, L.D0[c]);
      mac(dG, NN, L.DX[j][c]);
      mac<true>(dG, dDN, L.N[c]);
      mac<true>(dG, DN, L.DN[j][c]);
      tp_zero(dGe);
      mac_s(dGe, eta, dG);
      scale2(dGe);
      Dt[j][c].p1 = dGe;
      tp_zero(Dt[j][c].p0);
      mac<true>(Dt[j][c].p0, dB, L.N[c]);
      TP<T, 0> dn2 = L.DN[j][c];
      scale2(dn2);
      mac<true>(Dt[j][c].p0, dn2, beta);
      renorm(Dt[j][c].p0);
    }
  }
  // Q, A, B and their scaled derivatives
  WPr<T, 3> Qw;
  WPr<T, 4> Aw, Bw, Qt[2];
  WPr<T, 5> At[2], Bt[2];
  wp_zero(Qw);
  wp_zero(Aw);
  wp_zero(Bw);
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    wp_zero(Qt[j]);
    wp_zero(At[j]);
    wp_zero(Bt[j]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mac(Qw.p0, g[c], dt[c].p0);
    mac(Qw.p1, g[c], dt[c].p1);
    wp_mac_p(Aw, dt[c], hu[c]);
    wp_mac_p(Bw, dt[c], hv[c]);
  }
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const TP<T, 0> dhu[3] = {cross_comp<T>(e2[1], L.DX[j][2].c[0], e2[2], L.DX[j][1].c[0]),
                             cross_comp<T>(e2[2], L.DX[j][0].c[0], e2[0], L.DX[j][2].c[0]),
                             cross_comp<T>(e2[0], L.DX[j][1].c[0], e2[1], L.DX[j][0].c[0])};
    const TP<T, 0> dhv[3] = {cross_comp<T>(L.DX[j][1].c[0], e1[2], L.DX[j][2].c[0], e1[1]),
                             cross_comp<T>(L.DX[j][2].c[0], e1[0], L.DX[j][0].c[0], e1[2]),
                             cross_comp<T>(L.DX[j][0].c[0], e1[1], L.DX[j][1].c[0], e1[0])};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(Qt[j].p0, g[c], Dt[j][c].p0);
      mac(Qt[j].p1, g[c], Dt[j][c].p1);
      wp_mac_p(At[j], Dt[j][c], hu[c]);
      wp_mac_p(Bt[j], Dt[j][c], hv[c]);
      // 2W d~ . d(h) = (-2 beta n . dh) + W (2 G . dh)
      TP<T, 1> n2;
      tp_zero(n2);
      mac_s(n2, T(-2), L.N[c]);
      TP<T, 3> G2 = TG3[c];
      scale2(G2);
      TP<T, 1> nu, nv;
      tp_zero(nu);
      tp_zero(nv);
      mac(nu, dhu[c], n2);
      mac(nv, dhv[c], n2);
      mac(At[j].p0, nu, beta);
      mac(Bt[j].p0, nv, beta);
      mac(At[j].p1, dhu[c], G2);
      mac(Bt[j].p1, dhv[c], G2);
    }
    wp_renorm(Qt[j]);
    wp_renorm(At[j]);
    wp_renorm(Bt[j]);
  }
  wp_renorm(Qw);
  wp_renorm(Aw);
  wp_renorm(Bw);
  // M' = Q (A1 B2 - A2 B1) - B (A1 Q2 - A2 Q1) - A (Q1 B2 - Q2 B1).  The two products of each
  // difference run as one rolled loop, the subtracted one through an exactly negated copy of an
  // operand (the same FMAs, term for term), so each product shape is compiled once.
  WPr<T, 10> X;
  wp_zero(X);
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {
    WPr<T, 5> b = Bt[1 - t];
    if (t) wp_negate(b);
    wp_mac(X, At[t], b, beta);
  }
  wp_renorm(X);
  // Y = A1 Q2 - A2 Q1 and Z = Q1 B2 - Q2 B1 = B2 Q1 - B1 Q2: four products of one shape in one loop
  WPr<T, 9> YZ[2];
  wp_zero(YZ[0]);
  wp_zero(YZ[1]);
#pragma unroll 1
  for (int t = 0; t < 4; ++t) {
    const int h = t >> 1, k = t & 1;
    const WPr<T, 5>& a = h == 0 ? At[k] : Bt[1 - k];
    WPr<T, 4> q = h == 0 ? Qt[1 - k] : Qt[k];
    if (k) wp_negate(q);
    wp_mac(YZ[h], a, q, beta);
  }
  WPr<T, 9>& Y = YZ[0];
  WPr<T, 9>& Z = YZ[1];
  wp_renorm(Y);
  wp_renorm(Z);
  WPr<T, 13> Mp;
  wp_zero(Mp);
  wp_mac(Mp, Qw, X, beta);
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {
    WPr<T, 4> a = t ? Aw : Bw;
    wp_negate(a);
    wp_mac(Mp, a, t ? Z : Y, beta);
  }
  wp_renorm(Mp);
  WPr<T, 9> Q3;
  {
    WPr<T, 6> Q2;
    wp_zero(Q2);
    wp_mac(Q2, Qw, Qw, beta);
    wp_renorm(Q2);
    wp_zero(Q3);
    wp_mac(Q3, Q2, Qw, beta);
    wp_renorm(Q3);
  }
  // chord of s^(-3/2) on the range of s = d0.d0 (second remainder variable)
  T sl = F::inf(), sh = T(0);
  static_for<nc(2)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const T cl = SS.c[i] * (T)(1.0 / mult_c(2, i));  // exact: C in {1, 2}
    sl = fmin(sl, F::add_rd(cl, -SS.E));
    sh = fmax(sh, F::add_ru(cl, SS.E));
  });
  if (!(sl > tiny_pos<T>())) {
    fold = BNB_CELL_FOLD;
    return;
  }
  T sa, sb, sdlo, sdhi;
  chord_remainder<T>(sl, sh, sa, sb, sdlo, sdhi);
  TP<T, 2> Fk[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T ck = sb + (k == 0 ? sdlo : sdhi);
    tp_zero(Fk[k]);
    mac_s(Fk[k], sa, SS);
    add_const(Fk[k], ck, F::mul_ru(uu, fabs(ck)));
  }
  TP<T, 4> beta4 = beta;
  scale2(beta4);
  scale2(beta4);
  T mn = F::inf(), mx = -F::inf();
  int sm0 = 0;
  // the face loops stay rolled: one copy of their long bodies keeps the program within reach of
  // the instruction caches (unrolled, the four copies made the kernel wait on instruction fetch)
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    TP<T, 4> Wj;
    tp_zero(Wj);
    mac_s(Wj, ca, beta);
    const T cj = cb + (j == 0 ? dlo : dhi);
    add_const(Wj, cj, F::mul_ru(uu, fabs(cj)));
    TP<T, 15> Mj;
    wp_face(Mj, Mp, Wj);
    const int sm = cert_sign(Mj);
    if (sm == 0 || (j == 1 && sm != sm0)) {
      fold = BNB_CELL_FOLD;
      return;
    }
    sm0 = sm;
    if (sm < 0) negate(Mj);
    TP<T, 17> Den;
    {
      TP<T, 16> m16;
      elevate(m16, Mj);
      elevate(Den, m16);
    }
    TP<T, 11> Q3j;
    wp_face(Q3j, Q3, Wj);
    if (sq < 0) negate(Q3j);
    TP<T, 15> Nb;
    tp_zero(Nb);
    mac(Nb, Q3j, beta4);
    renorm(Nb);
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
      TP<T, 17> Nm;
      tp_zero(Nm);
      mac(Nm, Nb, Fk[k]);
      renorm(Nm);
      bool open = false;
      static_for<nc(17)>([&](auto I) {
        constexpr int i = decltype(I)::value;
        T nl, nh, dl, dh;
        coef_iv<i>(Nm, nl, nh);
        coef_iv<i>(Den, dl, dh);
        open = open || !(dl > tiny_pos<T>());
        ratio_acc(nl, nh, rcp_hi(dl), rcp_lo(dh), mn, mx);
      });
      if (open) {
        fold = BNB_CELL_FOLD;
        return;
      }
    }
  }
  eh = F::mul_ru(Khi, widen_hi(mx));
  if (!(eh >= T(0))) eh = F::inf();
  el = fmax(F::mul_rd(Klo, widen_lo(mn)), T(0));
}

static __device__ __noinline__ void process_cell_refract_fp64(const BoundParams& P, int e, int t, uint32_t id,
                                                              int depth, int64_t slot);

template <typename T>
__device__ __forceinline__ void process_cell_refract(const BoundParams& P, int e, int t, uint32_t id, int depth,
                                                     int64_t slot, uint32_t extra_flags = 0) {
  using F = FP<T>;
  float pf[3][3], nf[3][3];
  load_tri(P.tri, t, pf, nf);
  const float x0f[3] = {__ldg(P.ex + e), __ldg(P.ey + e), __ldg(P.ez + e)};
  T p[3][3], n[3][3], x0[3], e1[3], e2[3], rp0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      p[a][b] = (T)pf[a][b];
      n[a][b] = (T)nf[a][b];
    }
    x0[a] = (T)x0f[a];
    e1[a] = (T)P.re1[a];
    e2[a] = (T)P.re2[a];
    rp0[a] = (T)P.rp0[a];
  }
  const T eta = (T)P.eta;
  uint32_t flags = ((uint32_t)depth << BNB_CELL_DEPTH_SHIFT) | extra_flags;
  T cu[3], cv[3];
  cell_corners<T>(id, depth, cu, cv);

  // Receiver origin: the hit of the centroid's refracted ray, rounded to 2^-16 (any value is valid).
  T uc = T(0.5), vc = T(0.5);
  {
    T xc[3], ncn[3], d[3];
    const T third = T(1) / T(3);
    const T w1 = (cu[0] + cu[1] + cu[2]) * third, w2 = (cv[0] + cv[1] + cv[2]) * third, w0 = T(1) - w1 - w2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xc[c] = w0 * p[0][c] + w1 * p[1][c] + w2 * p[2][c];
      ncn[c] = w0 * n[0][c] + w1 * n[1][c] + w2 * n[2][c];
      d[c] = xc[c] - x0[c];
    }
    const T nn = ncn[0] * ncn[0] + ncn[1] * ncn[1] + ncn[2] * ncn[2];
    const T dn = d[0] * ncn[0] + d[1] * ncn[1] + d[2] * ncn[2];
    const T ss = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const T bc = (T(1) - eta * eta) * nn * ss + eta * eta * dn * dn;
    if (bc > T(0)) {
      const T wc = sqrt(bc);
      T dt[3], w[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dt[c] = eta * (nn * d[c] - dn * ncn[c]) - wc * ncn[c];
        w[c] = xc[c] - rp0[c];
      }
      const T g0 = e2[1] * e1[2] - e2[2] * e1[1], g1 = e2[2] * e1[0] - e2[0] * e1[2],
              g2 = e2[0] * e1[1] - e2[1] * e1[0];
      const T Qc = dt[0] * g0 + dt[1] * g1 + dt[2] * g2;
      const T hu0 = e2[1] * w[2] - e2[2] * w[1], hu1 = e2[2] * w[0] - e2[0] * w[2], hu2 = e2[0] * w[1] - e2[1] * w[0];
      const T hv0 = w[1] * e1[2] - w[2] * e1[1], hv1 = w[2] * e1[0] - w[0] * e1[2], hv2 = w[0] * e1[1] - w[1] * e1[0];
      uc = (dt[0] * hu0 + dt[1] * hu1 + dt[2] * hu2) / Qc;
      vc = (dt[0] * hv0 + dt[1] * hv1 + dt[2] * hv2) / Qc;
    }
    if (!(fabs(uc) < T(4))) uc = T(0.5);
    if (!(fabs(vc) < T(4))) vc = T(0.5);
    uc = rint(uc * T(65536)) * T(1.0 / 65536);
    vc = rint(vc * T(65536)) * T(1.0 / 65536);
  }

  Leaves<T> L;
  make_leaves<T, true>(p, n, x0, cu, cv, L);
  // n.n, d0.n, d0.d0 (degree 2) and beta (degree 4)
  TP<T, 2> NN, DN, SS;
  tp_zero(NN);
  tp_zero(DN);
  tp_zero(SS);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mac(NN, L.N[c], L.N[c]);
    mac(DN, L.D0[c], L.N[c]);
    mac(SS, L.D0[c], L.D0[c]);
  }
  renorm(NN);
  renorm(DN);
  renorm(SS);
  TP<T, 4> beta;
  tp_zero(beta);
  {
    TP<T, 4> A1, A2;
    tp_zero(A1);
    tp_zero(A2);
    mac(A1, NN, SS);
    mac(A2, DN, DN);
    const T uu = (T)FP<T>::u;
    const T e2v = eta * eta, e2err = F::mul_ru(uu, e2v);
    const T c1 = T(1) - e2v, c1err = F::add_ru(e2err, F::mul_ru(uu, fabs(c1)));
    mac(beta, tconst<T>(c1, c1err), A1);
    mac(beta, tconst<T>(e2v, e2err), A2);
    renorm(beta);
  }
  T blo, bhi;
  classical_range4(beta, blo, bhi);
  if (!(bhi > T(0))) {  // total internal reflection on the whole cell: no refracted path
    put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_TIR);
    return;
  }
  T ca, cb, dlo, dhi;
  sqrt_chord<T>(fmax(blo, T(0)), bhi, ca, cb, dlo, dhi);
  // tangential part eta' ((n.n) d0 - (d0.n) n) (degree 3, elevated to 5)
  TP<T, 3> TG3[3];
  TP<T, 5> TG5[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    TP<T, 3> tg;
    tp_zero(tg);
    mac(tg, NN, L.D0[c]);
    mac<true>(tg, DN, L.N[c]);
    tp_zero(TG3[c]);
    mac_s(TG3[c], eta, tg);
    TP<T, 4> t4;
    elevate(t4, TG3[c]);
    elevate(TG5[c], t4);
  }
  // receiver-side linear terms with the origin p' = p_k0 + uc e_k1 + vc e_k2
  TP<T, 1> hu[3], hv[3];
  {
    constexpr T g2e = GAM<T, 2>, uu = (T)FP<T>::u;
    TP<T, 1> W[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T pc = F::fma_rn(vc, e2[c], F::fma_rn(uc, e1[c], rp0[c]));
      const T pmag = F::fma_ru(fabs(vc), fabs(e2[c]), F::fma_ru(fabs(uc), fabs(e1[c]), fabs(rp0[c])));
      const T perr = F::mul_ru(g2e, pmag);
      const T q = p[0][c] - pc;
      const T qerr = F::add_ru(perr, F::mul_ru(uu, F::add_ru(F::add_ru(fabs(p[0][c]), fabs(pc)), perr)));
#pragma unroll
      for (int i = 0; i < 3; ++i) W[c].c[i] = L.XL[c].c[i] + q;
      W[c].B = F::add_ru(F::add_ru(L.XL[c].B, fabs(q)), qerr);
      W[c].E = F::add_ru(F::add_ru(L.XL[c].E, qerr),
                         F::mul_ru(uu, F::add_ru(F::add_ru(L.XL[c].B, L.XL[c].E), F::add_ru(fabs(q), qerr))));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      tp_zero(hu[c]);
      mac_s(hu[c], e2[a], W[b]);
      mac_s<true>(hu[c], e2[b], W[a]);
      tp_zero(hv[c]);
      mac_s(hv[c], e1[b], W[a]);
      mac_s<true>(hv[c], e1[a], W[b]);
    }
  }
  const TP<T, 0> g[3] = {cross_comp<T>(e2[1], e1[2], e2[2], e1[1]), cross_comp<T>(e2[2], e1[0], e2[0], e1[2]),
                         cross_comp<T>(e2[0], e1[1], e2[1], e1[0])};
  // the two xi faces: W_j = a beta + b + d_j, d~ = TG - W_j n, Q, A = d~.h_u, B = d~.h_v
  TP<T, 5> Qf[2];
  TP<T, 6> Af[2], Bf[2];
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    TP<T, 4> Wj;
    tp_zero(Wj);
    mac_s(Wj, ca, beta);
    const T cj = cb + (j == 0 ? dlo : dhi);
    add_const(Wj, cj, F::mul_ru((T)FP<T>::u, fabs(cj)));
    tp_zero(Qf[j]);
    tp_zero(Af[j]);
    tp_zero(Bf[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      TP<T, 5> DT = TG5[c];
      mac<true>(DT, Wj, L.N[c]);
      renorm(DT);
      mac(Qf[j], g[c], DT);
      mac(Af[j], DT, hu[c]);
      mac(Bf[j], DT, hv[c]);
    }
    renorm(Qf[j]);
    renorm(Af[j]);
    renorm(Bf[j]);
  }
  const int s0 = cert_sign(Qf[0]), s1 = cert_sign(Qf[1]);
  if constexpr (sizeof(T) == 4) {
    if (s0 == 0 || s1 == 0) {  // the float32 intervals cannot decide: float64 decides (flag QSIGN_FP64)
      process_cell_refract_fp64(P, e, t, id, depth, slot);
      return;
    }
  }
  const int sq = s0 == s1 ? s0 : 0;
  if (sq == 0) {
    // mixed-sign denominator: split up to the limit, then the universal box
    if (depth < P.max_depth) {
      const int64_t qi = (int64_t)atomicAdd((unsigned long long*)P.q_out_count, 1ull);
      if (qi < P.q_cap) {
        P.q_out[qi] = SplitItem{e, t, id, depth};
      } else {
        raise_status(P.status, BNB_ERR_CAPACITY);
      }
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_SPLIT);
    } else {
      put_rec(P, slot, 0.f, 1.f, 0.f, 1.f, 0.f, F::inf(), e, t, id, flags | BNB_CELL_LIVE | BNB_CELL_POS_UNBOUNDED);
    }
    return;
  }
  if (sq < 0) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      negate(Qf[j]);
      negate(Af[j]);
      negate(Bf[j]);
    }
  }
  {  // forward culling: t = Tn / Q with Tn = h_v . e2 (independent of d~)
    TP<T, 1> Tn;
    tp_zero(Tn);
#pragma unroll
    for (int c = 0; c < 3; ++c) mac_s(Tn, e2[c], hv[c]);
    if (sq < 0) negate(Tn);
    if (cert_sign(Tn) < 0) {
      put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_CULL_BEHIND);
      return;
    }
  }
  T umn = F::inf(), umx = -F::inf(), vmn = F::inf(), vmx = -F::inf();
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    TP<T, 6> Q6;
    elevate(Q6, Qf[j]);
    static_for<nc(6)>([&](auto I) {
      constexpr int i = decltype(I)::value;
      T ql, qh, al, ah, bl, bh;
      coef_iv<i>(Q6, ql, qh);
      coef_iv<i>(Af[j], al, ah);
      coef_iv<i>(Bf[j], bl, bh);
      const bool open = !(ql > tiny_pos<T>());
      const T rl = open ? F::inf() : rcp_hi(ql), rh = rcp_lo(qh);
      ratio_acc(al, ah, rl, rh, umn, umx);
      ratio_acc(bl, bh, rl, rh, vmn, vmx);
      if (open) {
        if (al == T(0)) umn = fmin(umn, T(0));
        if (ah == T(0)) umx = fmax(umx, T(0));
        if (bl == T(0)) vmn = fmin(vmn, T(0));
        if (bh == T(0)) vmx = fmax(vmx, T(0));
      }
    });
  }
  T ul = fmax(F::add_rd(uc, widen_lo(umn)), T(0));
  T uh = fmin(F::add_ru(uc, widen_hi(umx)), T(1));
  T vl = fmax(F::add_rd(vc, widen_lo(vmn)), T(0));
  T vh = fmin(F::add_ru(vc, widen_hi(vmx)), T(1));
  if (!(ul <= uh) || !(vl <= vh)) {
    put_rec(P, slot, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, e, t, id, flags | BNB_CELL_CULL_EMPTY);
    return;
  }
  // Irradiance: float32 only; a cell whose sign test fell back to float64 keeps E_hi = +inf.
  T el = T(0), eh = F::inf();
  uint32_t fold = 0;
  if constexpr (sizeof(T) == 4) {
    if (P.irradiance) {
      T Klo, Khi;
      cell_K<T>(p, x0, e1, e2, __ldg(P.ei + e), depth, Klo, Khi);
      refract_irradiance<T>(L, NN, DN, SS, beta, eta, TG3, hu, hv, g, e1, e2, sq, ca, cb, dlo, dhi, Klo, Khi, el,
                            eh, fold);
      if (fold) {
        el = T(0);
        eh = F::inf();
      }
    }
  }
  if (adapt_split(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), f_dn(el), f_up(eh), e, t, id, depth,
                  flags | BNB_CELL_LIVE | fold))
    return;
  put_rec(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), f_dn(el), f_up(eh), e, t, id,
          flags | BNB_CELL_LIVE | fold);
}

static __device__ __noinline__ void process_cell_refract_fp64(const BoundParams& P, int e, int t, uint32_t id,
                                                              int depth, int64_t slot) {
  process_cell_refract<double>(P, e, t, id, depth, slot, BNB_CELL_QSIGN_FP64);
}

// ------------------------------------------------------------------ kernels
// One 384-thread block per SM, persistent.  Every round starts with a block barrier so the
// twelve warps walk the (long, straight-line) cell program together and share instruction
// fetches; the round count is uniform across the block, so every thread reaches every barrier.
// 384 threads cap the registers at 168 (some spilling to L1): on the 256^2 mirror this beat 256
// threads at 255 registers by 6.5%, while 192 and 512 threads were slower.
constexpr int kBoundThreads = 384;
// The refraction cell program (irradiance in degree-17 forms) needs the full register file: 256
// threads (255 registers) ran the 420^2 water workload in 560 ms against 694 ms with 384 threads.
template <int KIND>
constexpr int kThreadsOf = KIND == 1 ? 256 : kBoundThreads;

// The refraction cell program (with its irradiance part) is long: compiled once, as a function
// that the base and the split kernels call.
static __device__ __noinline__ void process_cell_refract_f32(const BoundParams& P, int e, int t, uint32_t id,
                                                             int depth, int64_t slot) {
  process_cell_refract<float>(P, e, t, id, depth, slot);
}

// KIND 0: reflection, 1: refraction (separate instantiations: each kernel holds one cell program).
template <typename T, int KIND>
__device__ __forceinline__ void process_any(const BoundParams& P, int e, int t, uint32_t id, int depth, int64_t slot) {
  if constexpr (KIND == 0)
    process_cell<T>(P, e, t, id, depth, slot);
  else if constexpr (sizeof(T) == 4)
    process_cell_refract_f32(P, e, t, id, depth, slot);
  else
    process_cell_refract<T>(P, e, t, id, depth, slot);
}

// Refraction: the same kernel also bounds the children of queued split cells (q_in != nullptr), so
// its long cell program is reachable from one kernel entry only.  THREADS: the block size (one
// resident block per SM), which sets the register budget per thread (65,536 / THREADS, at most
// 255); the reflection pass is compiled for 256, 320 and 384 threads, the schedules the
// autotuner chooses from.
template <typename T, int KIND, int THREADS = kThreadsOf<KIND>>
__global__ void __launch_bounds__(THREADS, 1) bound_base_k(BoundParams P, const SplitItem* __restrict__ q_in,
                                                           const int64_t* __restrict__ q_in_count) {
  if constexpr (KIND == 1) {
    if (q_in != nullptr) {
      const int64_t n = min(*q_in_count, P.q_cap);
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 4 * n;
           i += (int64_t)gridDim.x * blockDim.x) {
        const SplitItem it = q_in[i >> 2];
        process_any<T, KIND>(P, it.emitter, it.tri, it.cell * 4u + (uint32_t)(i & 3), it.depth + 1, -1);
      }
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd((unsigned long long*)P.count, (unsigned long long)P.n_base);
  const int64_t per_tuple = (int64_t)1 << (2 * P.depth);
  const int64_t per_em = per_tuple * P.n_tris;
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  const int64_t rounds = (P.n_base + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    __syncthreads();
    const int64_t w = r * stride + (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (w < P.n_base) {
      const int e = (int)(w / per_em);
      const int64_t rr = w - (int64_t)e * per_em;
      const int t = (int)(rr / per_tuple);
      const uint32_t c = (uint32_t)(rr - (int64_t)t * per_tuple);
      process_any<T, KIND>(P, e, t, c, P.depth, w);
    }
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(128) bound_split_k(BoundParams P, const SplitItem* __restrict__ q_in,
                                                      const int64_t* __restrict__ q_in_count) {
  const int64_t n = min(*q_in_count, P.q_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 4 * n; i += (int64_t)gridDim.x * blockDim.x) {
    const SplitItem it = q_in[i >> 2];
    process_any<T, KIND>(P, it.emitter, it.tri, it.cell * 4u + (uint32_t)(i & 3), it.depth + 1, -1);
  }
}

template <typename T>
int grid_for_T(int64_t n, int block) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + block - 1) / block;
  const int64_t cap = (int64_t)sms;  // one resident block per SM
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

template <typename T, int KIND, int THREADS = kThreadsOf<KIND>>
cudaError_t launch_bound_base_T(const BoundParams& p, cudaStream_t st) {
  bound_base_k<T, KIND, THREADS><<<grid_for_T<T>(p.n_base, THREADS), THREADS, 0, st>>>(p, nullptr, nullptr);
  return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t launch_bound_split_T(const BoundParams& p, const SplitItem* q_in, const int64_t* q_in_count,
                                 cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if constexpr (KIND == 1)
    bound_base_k<T, KIND><<<sms, kThreadsOf<KIND>, 0, st>>>(p, q_in, q_in_count);
  else
    bound_split_k<T, KIND><<<sms * 2, 128, 0, st>>>(p, q_in, q_in_count);
  return cudaGetLastError();
}

}  // namespace bnb
