// Scaled Bernstein-Bezier polynomials on a triangle with rigorous rounding-error
// tracking, for the bound kernel.
//
// A degree-n polynomial on a cell with barycentric coordinates mu is held by
// its scaled coefficients c_g = C(n;g) b_g, where b_g are the classical
// Bernstein coefficients of Sec. 4.1 and C(n;g) = n!/(g0! g1! g2!).  In that
// form p(mu) = sum_g c_g mu^g, so a product is a plain convolution of the
// coefficient arrays, degree elevation adds the three neighbours, and the ratio
// of two same-degree forms has the same coefficient ratios as the classical
// forms (Eq. eq_bbound needs only those ratios).
//
// Every polynomial carries two scalars: B >= max_g |b_g| of the exact value and
// E >= max_g |b^_g - b_g|, the absolute error of the computed classical
// coefficients (so the scaled coefficient g is within E*C(n;g) of exact).  The
// update rules follow from the convex-combination form of the classical
// product (|b(pq)| <= max|b(p)| max|b(q)|) and the standard bound for a
// k-term FMA chain, |fl(s) - s| <= gamma_k sum |terms|, gamma_k = k u/(1-k u).
// B and E are themselves computed with upward rounding.  The final coefficient
// interval [c - E C, c + E C] is therefore rigorous for the float32 run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace bnb {

// ---------------------------------------------------------------- index maps
__host__ __device__ constexpr int nc(int n) { return (n + 1) * (n + 2) / 2; }
__host__ __device__ constexpr int g1_of(int n, int i) {
  int g1 = 0;
  while (i >= n + 1 - g1) {
    i -= n + 1 - g1;
    ++g1;
  }
  return g1;
}
__host__ __device__ constexpr int g2_of(int n, int i) {
  int g1 = 0;
  while (i >= n + 1 - g1) {
    i -= n + 1 - g1;
    ++g1;
  }
  return i;
}
__host__ __device__ constexpr int idx_of(int n, int g1, int g2) { return g1 * (n + 1) - g1 * (g1 - 1) / 2 + g2; }
__host__ __device__ constexpr double binom_c(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
__host__ __device__ constexpr double mult_c(int n, int i) {  // C(n; g) for coefficient i
  return binom_c(n, g1_of(n, i)) * binom_c(n - g1_of(n, i), g2_of(n, i));
}
// Number of (a, b) pairs that meet in one output coefficient of a degree-M x degree-N product.
__host__ __device__ constexpr int kterms(int M, int N) { return nc(M < N ? M : N); }

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1, so that every index and
// every table value derived from it (multinomials, gamma_k) is a constant expression.
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- arithmetic traits
template <typename T>
struct FP;

template <>
struct FP<float> {
  static constexpr double u = 5.9604644775390625e-08;  // 2^-24
  __device__ static __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  __device__ static __forceinline__ float fma_ru(float a, float b, float c) { return __fmaf_ru(a, b, c); }
  __device__ static __forceinline__ float fma_rd(float a, float b, float c) { return __fmaf_rd(a, b, c); }
  __device__ static __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
  __device__ static __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
  __device__ static __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
  __device__ static __forceinline__ float mul_rd(float a, float b) { return __fmul_rd(a, b); }
  __device__ static __forceinline__ float div_ru(float a, float b) { return __fdiv_ru(a, b); }
  __device__ static __forceinline__ float div_rd(float a, float b) { return __fdiv_rd(a, b); }
  __device__ static __forceinline__ float sqrt_ru(float a) { return __fsqrt_ru(a); }
  __device__ static __forceinline__ float sqrt_rd(float a) { return __fsqrt_rd(a); }
  __device__ static __forceinline__ float rcp_rn(float a) { return __frcp_rn(a); }
  // Hardware reciprocal approximation (rcp.approx.ftz.f32, one MUFU operation): relative error at
  // most rcp_rel = 2^-23 (1 ulp) for normal inputs up to rcp_big, checked exhaustively over that
  // range by the test suite.  Inputs above rcp_big would give flushed subnormal results.
  static constexpr double rcp_rel = 1.1920928955078125e-07;  // 2^-23
  static constexpr float rcp_big = 1.329227995784916e36f;    // 2^120
  __device__ static __forceinline__ float rcp_fast(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
  }
  __device__ static __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

template <>
struct FP<double> {
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
  __device__ static __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ static __forceinline__ double fma_ru(double a, double b, double c) { return __fma_ru(a, b, c); }
  __device__ static __forceinline__ double fma_rd(double a, double b, double c) { return __fma_rd(a, b, c); }
  __device__ static __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
  __device__ static __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
  __device__ static __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }
  __device__ static __forceinline__ double mul_rd(double a, double b) { return __dmul_rd(a, b); }
  __device__ static __forceinline__ double div_ru(double a, double b) { return __ddiv_ru(a, b); }
  __device__ static __forceinline__ double div_rd(double a, double b) { return __ddiv_rd(a, b); }
  __device__ static __forceinline__ double sqrt_ru(double a) { return __dsqrt_ru(a); }
  __device__ static __forceinline__ double sqrt_rd(double a) { return __dsqrt_rd(a); }
  __device__ static __forceinline__ double rcp_rn(double a) { return __drcp_rn(a); }
  // float64: the correctly rounded reciprocal (relative error at most u).
  static constexpr double rcp_rel = 1.1102230246251565e-16;  // 2^-53
  static constexpr double rcp_big = 1e300;
  __device__ static __forceinline__ double rcp_fast(double a) { return __drcp_rn(a); }
  __device__ static __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

// gamma_k rounded up into T (computed in double with a safety factor).
template <typename T>
__host__ __device__ constexpr T gam(int k) {
  return (T)((double)k * FP<T>::u / (1.0 - (double)k * FP<T>::u) * 1.0000001 + 1e-300);
}

// ---------------------------------------------------------------- tracked polynomial
template <typename T, int N>
struct TP {
  T c[nc(N)];
  T B;  // >= max |classical coefficient| (exact value)
  T E;  // >= max |computed - exact| over classical coefficients
};

template <typename T, int N>
__device__ __forceinline__ void tp_zero(TP<T, N>& r) {
#pragma unroll
  for (int i = 0; i < nc(N); ++i) r.c[i] = T(0);
  r.B = T(0);
  r.E = T(0);
}

// Error/bound update for r <- r + sign * p * q computed as a k-term FMA chain per coefficient.
template <int K, typename T>
__device__ __forceinline__ void track_mac(T& rB, T& rE, T pB, T pE, T qB, T qE) {
  using F = FP<T>;
  T p1 = F::add_ru(pB, pE), q1 = F::add_ru(qB, qE);
  T inh = F::fma_ru(pE, q1, F::mul_ru(pB, qE));
  T mag = F::fma_ru(p1, q1, F::add_ru(rB, rE));
  constexpr T g = gam<T>(K);  // K FMAs per output coefficient, one rounding each
  rE = F::add_ru(F::add_ru(rE, inh), F::mul_ru(g, mag));
  rB = F::fma_ru(pB, qB, rB);
}

// Compile-time pair tables: output index of (a, b) in a degree-M x degree-N product.
template <int M, int N, int I>
struct Pair {
  static constexpr int a = I / nc(N);
  static constexpr int b = I % nc(N);
  static constexpr int g = idx_of(M + N, g1_of(M, a) + g1_of(N, b), g2_of(M, a) + g2_of(N, b));
};

template <typename T, int M, int N, bool NEG, int... I>
__device__ __forceinline__ void conv_acc(T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                                         std::integer_sequence<int, I...>) {
  if constexpr (NEG) {
    ((r[Pair<M, N, I>::g] = FP<T>::fma_rn(-p[Pair<M, N, I>::a], q[Pair<M, N, I>::b], r[Pair<M, N, I>::g])), ...);
  } else {
    ((r[Pair<M, N, I>::g] = FP<T>::fma_rn(p[Pair<M, N, I>::a], q[Pair<M, N, I>::b], r[Pair<M, N, I>::g])), ...);
  }
}

// r += p * q   (NEG: r -= p * q)
template <bool NEG = false, typename T, int M, int N>
__device__ __forceinline__ void mac(TP<T, M + N>& r, const TP<T, M>& p, const TP<T, N>& q) {
  conv_acc<T, M, N, NEG>(r.c, p.c, q.c, std::make_integer_sequence<int, nc(M) * nc(N)>{});
  track_mac<kterms(M, N)>(r.B, r.E, p.B, p.E, q.B, q.E);
}

// Two independent products of the same shape, r1 (+/-)= p1 q1 and r2 (+/-)= p2 q2, one paired FMA
// (__ffma2_rn) per term; each lane runs exactly the FMA chain of mac().
template <typename T, int M, int N, bool NEG, int... I>
__device__ __forceinline__ void conv_acc2(T* __restrict__ r1, T* __restrict__ r2, const T* __restrict__ p1,
                                          const T* __restrict__ q1, const T* __restrict__ p2,
                                          const T* __restrict__ q2, std::integer_sequence<int, I...>) {
  if constexpr (sizeof(T) == 4) {
    (([&] {
       constexpr int a = Pair<M, N, I>::a, b = Pair<M, N, I>::b, g = Pair<M, N, I>::g;
       const float2 pp = NEG ? make_float2(-p1[a], -p2[a]) : make_float2(p1[a], p2[a]);
       const float2 acc = __ffma2_rn(pp, make_float2(q1[b], q2[b]), make_float2(r1[g], r2[g]));
       r1[g] = acc.x;
       r2[g] = acc.y;
     }()),
     ...);
  } else {
    conv_acc<T, M, N, NEG>(r1, p1, q1, std::integer_sequence<int, I...>{});
    conv_acc<T, M, N, NEG>(r2, p2, q2, std::integer_sequence<int, I...>{});
  }
}

template <bool NEG = false, typename T, int M, int N>
__device__ __forceinline__ void mac2(TP<T, M + N>& r1, const TP<T, M>& p1, const TP<T, N>& q1, TP<T, M + N>& r2,
                                     const TP<T, M>& p2, const TP<T, N>& q2) {
  conv_acc2<T, M, N, NEG>(r1.c, r2.c, p1.c, q1.c, p2.c, q2.c, std::make_integer_sequence<int, nc(M) * nc(N)>{});
  track_mac<kterms(M, N)>(r1.B, r1.E, p1.B, p1.E, q1.B, q1.E);
  track_mac<kterms(M, N)>(r2.B, r2.E, p2.B, p2.E, q2.B, q2.E);
}

// r += s * p for an exact scalar s (a float input such as a receiver edge component).
template <bool NEG = false, typename T, int N>
__device__ __forceinline__ void mac_s(TP<T, N>& r, T s, const TP<T, N>& p) {
  T ss = NEG ? -s : s;
#pragma unroll
  for (int i = 0; i < nc(N); ++i) r.c[i] = FP<T>::fma_rn(ss, p.c[i], r.c[i]);
  track_mac<1>(r.B, r.E, fabs(s), T(0), p.B, p.E);
}

// Degree elevation by one (scaled form: sum of the up-to-three lower neighbours).
template <typename T, int N>
__device__ __forceinline__ void elevate(TP<T, N + 1>& r, const TP<T, N>& p) {
  static_for<nc(N + 1)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int g1 = g1_of(N + 1, i), g2 = g2_of(N + 1, i), g0 = N + 1 - g1 - g2;
    T s = T(0);
    if constexpr (g0 >= 1) s = s + p.c[idx_of(N, g1, g2)];
    if constexpr (g1 >= 1) s = s + p.c[idx_of(N, g1 - 1, g2)];
    if constexpr (g2 >= 1) s = s + p.c[idx_of(N, g1, g2 - 1)];
    r.c[i] = s;
  });
  using F = FP<T>;
  constexpr T g2 = gam<T>(2);
  r.B = p.B;
  r.E = F::add_ru(p.E, F::mul_ru(g2, F::add_ru(p.B, p.E)));
}

// Re-derive B from the computed coefficients: max_g |c_g| / C(n;g) + E.  Tightens B after
// a cancellation (a small result computed from large operands).
template <typename T, int N>
__device__ __forceinline__ void renorm(TP<T, N>& p) {
  using F = FP<T>;
  T m = T(0);
  static_for<nc(N)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    // 1/C rounded up, then |c| * (1/C) rounded up, is >= |c| / C.
    constexpr T inv = (T)(1.0 / mult_c(N, i) * (1.0 + 4.0 * FP<T>::u));
    m = fmax(m, F::mul_ru(fabs(p.c[i]), inv));
  });
  T nb = F::add_ru(m, p.E);
  p.B = fmin(p.B, nb);
}

// Sign of every coefficient interval: +1 all > 0, -1 all < 0, 0 otherwise.
template <typename T, int N>
__device__ __forceinline__ int cert_sign(const TP<T, N>& p) {
  using F = FP<T>;
  bool pos = true, neg = true;
  static_for<nc(N)>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr T C = (T)(mult_c(N, i) * (1.0 + 4.0 * FP<T>::u));
    const T lo = F::fma_rd(-p.E, C, p.c[i]);
    const T hi = F::fma_ru(p.E, C, p.c[i]);
    pos = pos && (lo > T(0));
    neg = neg && (hi < T(0));
  });
  return pos ? 1 : (neg ? -1 : 0);
}

template <typename T, int N>
__device__ __forceinline__ void negate(TP<T, N>& p) {
#pragma unroll
  for (int i = 0; i < nc(N); ++i) p.c[i] = -p.c[i];
}

// Tracked degree-0 scalar (a constant computed from inputs).
template <typename T>
__device__ __forceinline__ TP<T, 0> tconst(T v, T err) {
  TP<T, 0> r;
  r.c[0] = v;
  r.B = FP<T>::add_ru(fabs(v), err);
  r.E = err;
  return r;
}

}  // namespace bnb
