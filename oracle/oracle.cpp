// FP64 CPU oracle for Bernstein bounds for caustics (Fan et al., TOG 2025).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA path is checked against.  Only the test-suite, the smoke check and the
// CPU-baseline leg of the benchmark load it; the library path never does.  It
// shares no code, header or table with the CUDA sources.
//
// What it follows, step by step:
//   * Sec. 4.1, Eq. (1) and Eq. "eq_bbound": classical Bernstein coefficients
//     on a simplex; a ratio p/q is bounded by the min/max of b(p)/b(q) when all
//     b(q) are non-zero and share a sign; otherwise the reciprocal rule, then the
//     universal set.  Products use the textbook weights C(m;a)C(n;b)/C(m+n;a+b),
//     elevation and directional derivatives their textbook formulas.
//   * Sec. 4.3, Eqs. "eq_xi", "eq_ni", "eq_rct", "eq_refr_rational": the vertex,
//     interpolated normal, reflected direction and the Moller-form receiver
//     coordinates as polynomials in the cell's barycentric coordinates.
//   * Sec. 4.4, Eqs. "eq_dwda" and "eq_irr_term3a": irradiance through the GGT
//     chain rule, det(du_k/du_1) = M / Q^3, and the non-rational |d_0|^3 carried
//     by a remainder variable xi (Sec. 4.3, "Remainder variables") around a chord
//     of f(s) = s^(-3/2).
//   * Sec. 4.5, Eq. "eq_pertuple_b": per-tuple bound m * max over covering pieces.
//   * Sec. 6.1 "Bound storage": uniform texture-space grid, splat to every
//     overlapped cell.
//   * Sec. 5.3, Algorithm 1, and Sec. 5.4: independent selection of each tuple
//     with P = min(gamma * E~, 1), estimate sum E(T)/P over selected tuples.
//   * Sec. 6.1 "Root-finding": Newton's method with deterministic initialization.
//   * Two specular vertices (each reflecting or refracting; the TT chains of Table
//     "tab:perf"): Sec. 6.1 "Tuple construction" (candidate T2 of a cell from the bound
//     of x1 and of the direction ratios) and "Degree reduction" (u2 reduced to degree 1
//     plus a remainder, then the second vertex), and a direct-geometry chain evaluator.
//   * Sec. 4.4 "Implicit differentiation": the irradiance of a single refraction from
//     the specular polynomials F, G of the section's footnote over the cell and the
//     receiver box, |du1/du_k| = |det B| / |det A|, bounded by coefficient ratios.
//   * Sec. 6.1 "Domain subdivision" (adaptive stopping), Sec. 5.3 bin packing and the
//     stochastic Newton starts ("Stoc") with their reciprocal weighting.
//
// Readings where the paper is silent (cell split order, chord closed form,
// forward culling, grid inclusion, RNG, Newton details) are listed in the
// repository's design notes; the code below states each one where it is used.
//
// Precision: every quantity is double.  Where a floating-point value decides an
// integer and the CUDA path takes that decision in float32 (grid cell of a box
// edge, selection r < P), this file repeats the same float32 operation.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Small vector algebra
// ---------------------------------------------------------------------------
struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

// ---------------------------------------------------------------------------
// Classical Bernstein polynomials on the 1-simplex (dim 1) or 2-simplex (dim 2)
// Coefficient order (dim 2): g1 = 0..n outer, g2 = 0..n-g1 inner, g0 = n-g1-g2.
// ---------------------------------------------------------------------------
// Pascal's triangle up to degree 96, built once (exact integers up to 2^53).
constexpr int kMaxDeg = 96;
struct BinomTable {
  double t[kMaxDeg + 1][kMaxDeg + 1];
  BinomTable() {
    for (int n = 0; n <= kMaxDeg; ++n)
      for (int k = 0; k <= kMaxDeg; ++k)
        t[n][k] = (k == 0 || k == n) ? 1.0 : (k > n ? 0.0 : t[n - 1][k - 1] + t[n - 1][k]);
  }
};
const BinomTable kBinom;
double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  return kBinom.t[n][k];
}

struct Poly {
  int dim = 2;
  int n = 0;
  std::vector<double> c;  // classical Bernstein coefficients
};

int psize(int dim, int n) { return dim == 1 ? n + 1 : (n + 1) * (n + 2) / 2; }
int pidx(int dim, int n, int g1, int g2) {
  if (dim == 1) return g1;
  return g1 * (n + 1) - g1 * (g1 - 1) / 2 + g2;
}
// multinomial n! / (g0! g1! g2!)
double multinom(int n, int g1, int g2) { return binom(n, g1) * binom(n - g1, g2); }

template <class F>
void for_each_index(int dim, int n, F f) {
  if (dim == 1) {
    for (int g1 = 0; g1 <= n; ++g1) f(g1, 0);
  } else {
    for (int g1 = 0; g1 <= n; ++g1)
      for (int g2 = 0; g2 <= n - g1; ++g2) f(g1, g2);
  }
}

Poly pconst(int dim, int n, double v) {
  Poly p;
  p.dim = dim;
  p.n = n;
  p.c.assign(psize(dim, n), v);  // partition of unity
  return p;
}

// Degree-1 polynomial from its values at the simplex corners (linear precision).
Poly paffine(double f0, double f1, double f2) {
  Poly p;
  p.dim = 2;
  p.n = 1;
  p.c.assign(3, 0.0);
  p.c[pidx(2, 1, 0, 0)] = f0;
  p.c[pidx(2, 1, 1, 0)] = f1;
  p.c[pidx(2, 1, 0, 1)] = f2;
  return p;
}

// Product in classical form: (pq)_g = sum_{a+b=g} C(m;a) C(n;b) / C(m+n;g) p_a q_b.
Poly pmul(const Poly& p, const Poly& q) {
  Poly r;
  r.dim = p.dim;
  r.n = p.n + q.n;
  r.c.assign(psize(r.dim, r.n), 0.0);
  for_each_index(p.dim, p.n, [&](int a1, int a2) {
    double pa = p.c[pidx(p.dim, p.n, a1, a2)];
    double wa = multinom(p.n, a1, a2);
    for_each_index(q.dim, q.n, [&](int b1, int b2) {
      int g1 = a1 + b1, g2 = a2 + b2;
      double w = wa * multinom(q.n, b1, b2) / multinom(r.n, g1, g2);
      r.c[pidx(r.dim, r.n, g1, g2)] += w * pa * q.c[pidx(q.dim, q.n, b1, b2)];
    });
  });
  return r;
}

// Degree elevation by one: b'_g = sum_i (g_i / (n+1)) b_{g - e_i}.
Poly pelevate(const Poly& p) {
  Poly r;
  r.dim = p.dim;
  r.n = p.n + 1;
  r.c.assign(psize(r.dim, r.n), 0.0);
  for_each_index(r.dim, r.n, [&](int g1, int g2) {
    int g0 = r.n - g1 - g2;
    double s = 0.0;
    if (g0 >= 1) s += (double)g0 / r.n * p.c[pidx(p.dim, p.n, g1, g2)];
    if (g1 >= 1) s += (double)g1 / r.n * p.c[pidx(p.dim, p.n, g1 - 1, g2)];
    if (g2 >= 1) s += (double)g2 / r.n * p.c[pidx(p.dim, p.n, g1, g2 - 1)];
    r.c[pidx(r.dim, r.n, g1, g2)] = s;
  });
  return r;
}

Poly pelevate_to(Poly p, int n) {
  while (p.n < n) p = pelevate(p);
  return p;
}

Poly padd(Poly p, Poly q, double sq = 1.0) {
  int n = std::max(p.n, q.n);
  p = pelevate_to(p, n);
  q = pelevate_to(q, n);
  for (size_t i = 0; i < p.c.size(); ++i) p.c[i] += sq * q.c[i];
  return p;
}

Poly pscale(Poly p, double s) {
  for (auto& v : p.c) v *= s;
  return p;
}

// Derivative along the j-th barycentric direction (d/dmu_j with mu_0 = 1 - mu_1 - mu_2):
// coefficient at b (degree n-1) = n (b_{b+e_j} - b_{b+e_0}).
Poly pderiv(const Poly& p, int j) {
  Poly r;
  r.dim = p.dim;
  r.n = p.n - 1;
  r.c.assign(psize(r.dim, r.n), 0.0);
  for_each_index(r.dim, r.n, [&](int b1, int b2) {
    double up = (j == 1) ? p.c[pidx(p.dim, p.n, b1 + 1, b2)] : p.c[pidx(p.dim, p.n, b1, b2 + 1)];
    double base = p.c[pidx(p.dim, p.n, b1, b2)];
    r.c[pidx(r.dim, r.n, b1, b2)] = p.n * (up - base);
  });
  return r;
}

// Direct evaluation sum_g b_g C(n;g) mu^g.
double peval(const Poly& p, double m1, double m2) {
  double m0 = 1.0 - m1 - m2;
  double s = 0.0;
  for_each_index(p.dim, p.n, [&](int g1, int g2) {
    int g0 = p.n - g1 - g2;
    s += p.c[pidx(p.dim, p.n, g1, g2)] * multinom(p.n, g1, g2) * std::pow(m0, g0) *
         std::pow(m1, g1) * std::pow(m2, g2);
  });
  return s;
}

double pmin(const Poly& p) { return *std::min_element(p.c.begin(), p.c.end()); }
double pmax(const Poly& p) { return *std::max_element(p.c.begin(), p.c.end()); }

// +1 / -1 when every coefficient is non-zero with that sign, 0 otherwise (Eq. eq_bbound).
int psign(const Poly& p) {
  bool pos = true, neg = true;
  for (double v : p.c) {
    if (!(v > 0.0)) pos = false;
    if (!(v < 0.0)) neg = false;
  }
  return pos ? 1 : (neg ? -1 : 0);
}

struct PV {  // polynomial 3-vector
  Poly x, y, z;
};
PV pv_affine(V3 a, V3 b, V3 c) { return {paffine(a.x, b.x, c.x), paffine(a.y, b.y, c.y), paffine(a.z, b.z, c.z)}; }
Poly pv_dot(const PV& a, const PV& b) { return padd(padd(pmul(a.x, b.x), pmul(a.y, b.y)), pmul(a.z, b.z)); }
Poly pv_dotc(const PV& a, V3 b) { return padd(padd(pscale(a.x, b.x), pscale(a.y, b.y)), pscale(a.z, b.z)); }
PV pv_mul(const Poly& s, const PV& a) { return {pmul(s, a.x), pmul(s, a.y), pmul(s, a.z)}; }
PV pv_sub(const PV& a, const PV& b, double sb = 1.0) { return {padd(a.x, b.x, -sb), padd(a.y, b.y, -sb), padd(a.z, b.z, -sb)}; }
PV pv_subc(const PV& a, V3 c) {
  PV r = a;
  for (auto& v : r.x.c) v -= c.x;
  for (auto& v : r.y.c) v -= c.y;
  for (auto& v : r.z.c) v -= c.z;
  return r;
}
PV pv_scale(const PV& a, double s) { return {pscale(a.x, s), pscale(a.y, s), pscale(a.z, s)}; }
PV pv_elev(const PV& a, int n) { return {pelevate_to(a.x, n), pelevate_to(a.y, n), pelevate_to(a.z, n)}; }
PV pv_crossc(const PV& a, V3 b) {  // a x b, b constant
  return {padd(pscale(a.y, b.z), pscale(a.z, b.y), -1.0), padd(pscale(a.z, b.x), pscale(a.x, b.z), -1.0),
          padd(pscale(a.x, b.y), pscale(a.y, b.x), -1.0)};
}

// p0 + W p1 with W = sqrt(beta) kept as a symbol: products reduce W^2 to beta, which is exact
// wherever W = sqrt(beta) (refraction, Sec. 4.4 with the derivative of sqrt carried exactly).
struct WP {
  Poly p0, p1;
};
WP wp_add(const WP& a, const WP& b, double sb = 1.0) { return {padd(a.p0, b.p0, sb), padd(a.p1, b.p1, sb)}; }
WP wp_mul(const WP& a, const WP& b, const Poly& beta) {
  return {padd(pmul(a.p0, b.p0), pmul(pmul(a.p1, b.p1), beta)), padd(pmul(a.p0, b.p1), pmul(a.p1, b.p0))};
}
WP wp_mulp(const WP& a, const Poly& q) { return {pmul(a.p0, q), pmul(a.p1, q)}; }
Poly wp_at(const WP& a, const Poly& W) { return padd(a.p0, pmul(W, a.p1)); }  // W replaced by a polynomial

// ---------------------------------------------------------------------------
// Scene views (own definitions; the field layout is the documented interface)
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {
typedef struct {
  int32_t n_verts, n_tris;
  const float *px, *py, *pz, *nx, *ny, *nz;
  const int32_t *i0, *i1, *i2;
  int32_t kind;  // 0 reflect, 1 refract
  float eta;     // n_incident / n_transmitted
} orc_surface;
typedef struct {
  float p0[3], e1[3], e2[3];
} orc_receiver;
typedef struct {
  int32_t n;
  const float *x, *y, *z, *intensity;
} orc_emitters;
typedef struct {
  int32_t emitter, tri0, tri1;
  uint32_t cell;   // base-4 digits of the cell path, most significant first
  uint32_t flags;  // bits 0..7 flags, bits 24..29 depth
  int32_t pad;
  double u_lo, u_hi, v_lo, v_hi, e_lo, e_hi;
  double q_cond, m_cond;  // min|b| / max|b| of Q and M (diagnostics for tolerance rules)
} orc_record;
}

namespace {

enum : uint32_t {
  F_LIVE = 1u,
  F_SPLIT = 2u,
  F_CULL_BEHIND = 4u,
  F_CULL_EMPTY = 8u,
  F_FOLD = 16u,
  F_POS_UNBOUNDED = 32u,
  F_TIR = 128u,
};

struct Tri {
  V3 p[3], n[3];
};

Tri get_tri(const orc_surface* s, int t) {
  Tri T;
  int id[3] = {s->i0[t], s->i1[t], s->i2[t]};
  for (int k = 0; k < 3; ++k) {
    int v = id[k];
    T.p[k] = {(double)s->px[v], (double)s->py[v], (double)s->pz[v]};
    T.n[k] = {(double)s->nx[v], (double)s->ny[v], (double)s->nz[v]};
  }
  return T;
}

struct Rec {
  V3 p0, e1, e2;
};
Rec get_rec(const orc_receiver* r) {
  return {{r->p0[0], r->p0[1], r->p0[2]}, {r->e1[0], r->e1[1], r->e1[2]}, {r->e2[0], r->e2[1], r->e2[2]}};
}

struct UV {
  double u, v;
};

// Cell corners for a base-4 path (Sec. 6.1 "Domain subdivision", on the simplex):
// children of (C0,C1,C2) are (C0,m01,m02), (m01,C1,m12), (m02,m12,C2), (m12,m02,m01).
void child_corners(const UV in[3], int k, UV out[3]) {
  UV m01 = {(in[0].u + in[1].u) / 2, (in[0].v + in[1].v) / 2};
  UV m02 = {(in[0].u + in[2].u) / 2, (in[0].v + in[2].v) / 2};
  UV m12 = {(in[1].u + in[2].u) / 2, (in[1].v + in[2].v) / 2};
  if (k == 0) { out[0] = in[0]; out[1] = m01; out[2] = m02; }
  if (k == 1) { out[0] = m01; out[1] = in[1]; out[2] = m12; }
  if (k == 2) { out[0] = m02; out[1] = m12; out[2] = in[2]; }
  if (k == 3) { out[0] = m12; out[1] = m02; out[2] = m01; }
}

void cell_corners(uint32_t id, int depth, UV C[3]) {
  C[0] = {0, 0};
  C[1] = {1, 0};
  C[2] = {0, 1};
  for (int d = depth - 1; d >= 0; --d) {
    int k = (id >> (2 * d)) & 3;
    UV o[3];
    child_corners(C, k, o);
    C[0] = o[0]; C[1] = o[1]; C[2] = o[2];
  }
}

// Chord of f(s) = s^(-3/2) on [s_lo, s_hi] and the range [dlo, dhi] of f - r.
// f is convex and decreasing: the chord lies above f, so f - r <= 0 with the
// minimum where f'(s*) = a.  A degenerate interval gives a = 0, b = f, d = 0.
void chord_inv32(double s_lo, double s_hi, double* a, double* b, double* dlo, double* dhi) {
  auto f = [](double s) { return 1.0 / (s * std::sqrt(s)); };
  if (!(s_hi > s_lo)) {
    *a = 0.0;
    *b = f(s_lo);
    *dlo = 0.0;
    *dhi = 0.0;
    return;
  }
  *a = (f(s_hi) - f(s_lo)) / (s_hi - s_lo);
  *b = f(s_lo) - *a * s_lo;
  double ss = std::pow(-*a / 1.5, -0.4);
  ss = std::min(std::max(ss, s_lo), s_hi);
  *dlo = std::min(0.0, f(ss) - (*a * ss + *b));
  *dhi = 0.0;
}

// Chord r(beta) = a beta + b of g(beta) = sqrt(beta) on [lo, hi] (lo >= 0) and the range
// [dlo, dhi] of g - r (Sec. 4.3, "Remainder variables", linear r built from the range of beta
// on the current cell).  g is concave: the chord lies below g, so g - r >= 0, zero at both
// ends and largest where g'(b*) = a, i.e. b* = 1 / (4 a^2).  A degenerate interval gives
// a = 0, b = g(lo), d = 0.
void chord_sqrt(double lo, double hi, double* a, double* b, double* dlo, double* dhi) {
  if (!(hi > lo)) {
    *a = 0.0;
    *b = std::sqrt(lo);
    *dlo = 0.0;
    *dhi = 0.0;
    return;
  }
  *a = (std::sqrt(hi) - std::sqrt(lo)) / (hi - lo);
  *b = std::sqrt(lo) - *a * lo;
  double bs = 1.0 / (4.0 * *a * *a);
  bs = std::min(std::max(bs, lo), hi);
  *dlo = 0.0;
  *dhi = std::max(0.0, std::sqrt(bs) - (*a * bs + *b));
}

// Ratio bound [min, max] of b(p)/b(q) (same degree; q must have uniform sign).
void ratio_bound(const Poly& p, const Poly& q, double* lo, double* hi) {
  double l = std::numeric_limits<double>::infinity(), h = -l;
  for (size_t i = 0; i < p.c.size(); ++i) {
    double r = p.c[i] / q.c[i];
    l = std::min(l, r);
    h = std::max(h, r);
  }
  *lo = l;
  *hi = h;
}

// Reciprocal rule (Sec. 4.1): when q has mixed signs but p does not, q/p is
// bounded; p/q then lies in 1/[r_lo, r_hi] (two rays when 0 is inside).  The
// result is returned already intersected with [0,1] as its hull; empty -> lo > hi.
void reciprocal_bound01(const Poly& p, const Poly& q, double* lo, double* hi) {
  if (psign(p) == 0) {
    *lo = 0.0;
    *hi = 1.0;  // universal set, intersected with [0,1]
    return;
  }
  double rl, rh;
  ratio_bound(q, p, &rl, &rh);
  double L = 1.0, H = 0.0;  // empty
  auto add = [&](double a, double b) {  // add [a,b] ∩ [0,1] to the hull
    a = std::max(a, 0.0);
    b = std::min(b, 1.0);
    if (a <= b) {
      L = std::min(L, a);
      H = std::max(H, b);
    }
  };
  const double inf = std::numeric_limits<double>::infinity();
  if (rl > 0.0 || rh < 0.0) {
    add(1.0 / rh, 1.0 / rl);
  } else {
    // r in [rl, 0] -> p/q in (-inf, 1/rl];  r in [0, rh] -> p/q in [1/rh, inf)
    add(-inf, rl < 0.0 ? 1.0 / rl : -inf);
    add(rh > 0.0 ? 1.0 / rh : inf, inf);
  }
  *lo = L;
  *hi = H;
}

struct Ctx {
  const orc_surface* s1;
  Rec rec;
  const orc_emitters* em;
  int irradiance;
  int max_total_depth;
  // adaptive subdivision (Sec. 6.1 "Domain subdivision"): off when adapt_depth <= the base depth
  int adapt_depth = 0;
  float sigma = 0.0f, alpha = 0.0f;
};

float f32_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
  return f;
}
float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}

// Adaptive subdivision (Sec. 6.1 "Domain subdivision"): a live cell with a bounded box, above the
// depth limit, is subdivided again unless its receiver box (U_k) has area below sigma or its
// irradiance bounds satisfy E_hi < alpha E_lo.  The decision is taken on the record as stored in
// float32 (box rounded outward, area and alpha E_lo as float32 products), the precision in which
// the CUDA path takes it.  Returns true (and turns r into a SPLIT record) when the cell splits.
bool adaptive_split(const Ctx& cx, orc_record& r, int depth) {
  if (depth >= cx.adapt_depth || !(r.flags & F_LIVE) || (r.flags & F_POS_UNBOUNDED)) return false;
  const float du = f32_up(r.u_hi) - f32_down(r.u_lo), dv = f32_up(r.v_hi) - f32_down(r.v_lo);
  const float area = du * dv;
  if (area < cx.sigma) return false;
  const float el = f32_down(r.e_lo), eh = f32_up(r.e_hi);
  if (eh < cx.alpha * el) return false;
  r.flags = (r.flags & ~(F_LIVE | F_FOLD)) | F_SPLIT;
  r.u_lo = r.u_hi = r.v_lo = r.v_hi = r.e_lo = r.e_hi = 0.0;
  return true;
}

double cond_of(const Poly& p) {
  double mn = std::numeric_limits<double>::infinity(), mx = 0.0;
  for (double v : p.c) {
    mn = std::min(mn, std::fabs(v));
    mx = std::max(mx, std::fabs(v));
  }
  return mx > 0 ? mn / mx : 0.0;
}

// Bound one cell of one (emitter, triangle) tuple for single reflection.
void bound_cell_reflect(const Ctx& cx, int e, int t, uint32_t id, int depth, std::vector<orc_record>& out) {
  UV C[3];
  cell_corners(id, depth, C);
  Tri T = get_tri(cx.s1, t);
  V3 x0 = {cx.em->x[e], cx.em->y[e], cx.em->z[e]};
  double I0 = cx.em->intensity[e];
  V3 e11 = T.p[1] - T.p[0], e12 = T.p[2] - T.p[0];
  V3 n1d = T.n[1] - T.n[0], n2d = T.n[2] - T.n[0];
  V3 xc[3], nc[3];
  for (int k = 0; k < 3; ++k) {
    xc[k] = T.p[0] + C[k].u * e11 + C[k].v * e12;  // Eq. eq_xi
    nc[k] = T.n[0] + C[k].u * n1d + C[k].v * n2d;  // Eq. eq_ni
  }
  PV x1 = pv_affine(xc[0], xc[1], xc[2]);
  PV n1 = pv_affine(nc[0], nc[1], nc[2]);
  PV d0 = pv_subc(x1, x0);
  // Eq. eq_refr_rational, reflection: d~ = (n.n) d0 - 2 (d0.n) n
  Poly nn = pv_dot(n1, n1);
  Poly dn = pv_dot(d0, n1);
  PV dt = pv_sub(pv_mul(nn, d0), pv_mul(dn, n1), 2.0);
  // Eq. eq_rct with receiver (p_k0, e_k1, e_k2)
  const Rec& R = cx.rec;
  PV w = pv_subc(x1, R.p0);
  PV dxe2 = pv_crossc(dt, R.e2);
  Poly Q = pv_dotc(dxe2, R.e1);
  Poly Pu = pv_dot(dxe2, w);
  Poly Pv = pv_dot(pv_crossc(w, R.e1), dt);
  Poly Tn = pv_dotc(pv_crossc(w, R.e1), R.e2);  // t = Tn / Q (forward distance)

  orc_record r;
  std::memset(&r, 0, sizeof(r));
  r.emitter = e;
  r.tri0 = t;
  r.tri1 = -1;
  r.cell = id;
  r.flags = (uint32_t)depth << 24;
  r.q_cond = cond_of(Q);

  int sq = psign(Q);
  if (sq == 0) {
    // Mixed-sign denominator (Sec. 4.1): bound the reciprocal q/p where p has one sign; the
    // result (possibly two rays) is intersected with the receiver region [0,1] as a hull, and
    // the universal set when p also has mixed signs.  A cell whose reciprocal bound misses
    // the receiver is culled; otherwise it is split (up to the extra-split limit) and, at the
    // limit, kept with this box and an unbounded irradiance.
    Poly Q4 = pelevate_to(Q, 4);
    reciprocal_bound01(Pu, Q4, &r.u_lo, &r.u_hi);
    reciprocal_bound01(Pv, Q4, &r.v_lo, &r.v_hi);
    if (r.u_lo > r.u_hi || r.v_lo > r.v_hi) {
      r.u_lo = r.u_hi = r.v_lo = r.v_hi = 0.0;
      r.flags |= F_CULL_EMPTY;
      out.push_back(r);
      return;
    }
    if (depth < cx.max_total_depth) {  // split and bound the four children
      r.u_lo = r.u_hi = r.v_lo = r.v_hi = 0.0;
      r.flags |= F_SPLIT;
      out.push_back(r);
      for (int k = 0; k < 4; ++k) bound_cell_reflect(cx, e, t, id * 4u + (uint32_t)k, depth + 1, out);
      return;
    }
    r.e_lo = 0.0;
    r.e_hi = std::numeric_limits<double>::infinity();
    r.flags |= F_LIVE | F_POS_UNBOUNDED;
    out.push_back(r);
    return;
  }
  // Forward culling: the hit is behind x1 on the whole cell when t < 0 everywhere.
  int st = psign(Tn);
  if (st != 0 && st != sq) {
    r.flags |= F_CULL_BEHIND;
    out.push_back(r);
    return;
  }
  Poly Q4 = pelevate(Q);
  double ul, uh, vl, vh;
  ratio_bound(Pu, Q4, &ul, &uh);
  ratio_bound(Pv, Q4, &vl, &vh);
  r.u_lo = std::max(ul, 0.0);
  r.u_hi = std::min(uh, 1.0);
  r.v_lo = std::max(vl, 0.0);
  r.v_hi = std::min(vh, 1.0);
  if (r.u_lo > r.u_hi || r.v_lo > r.v_hi) {
    r.flags |= F_CULL_EMPTY;
    out.push_back(r);
    return;
  }
  r.flags |= F_LIVE;
  auto finish = [&]() {
    const bool split = adaptive_split(cx, r, depth);
    out.push_back(r);
    if (split)
      for (int k = 0; k < 4; ++k) bound_cell_reflect(cx, e, t, id * 4u + (uint32_t)k, depth + 1, out);
  };
  if (!cx.irradiance) {
    r.e_lo = 0.0;
    r.e_hi = std::numeric_limits<double>::infinity();
    finish();
    return;
  }
  // Eq. eq_irr_term3a: det(du_k/dmu) = M / Q^3 with a = Pu, b = Pv.
  Poly a1 = pderiv(Pu, 1), a2 = pderiv(Pu, 2);
  Poly b1 = pderiv(Pv, 1), b2 = pderiv(Pv, 2);
  Poly q1 = pderiv(Q, 1), q2 = pderiv(Q, 2);
  Poly X = padd(pmul(a1, b2), pmul(a2, b1), -1.0);
  Poly Y = padd(pmul(a1, q2), pmul(a2, q1), -1.0);
  Poly Z = padd(pmul(q1, b2), pmul(q2, b1), -1.0);
  Poly M = padd(padd(pmul(Q, X), pmul(Pv, Y), -1.0), pmul(Pu, Z), -1.0);
  r.m_cond = cond_of(M);
  int sm = psign(M);
  // Eq. eq_dwda: E = I0 * |d0.N1|/|d0|^3 * |N1|... collapsed to
  //   E = I0 |C1| |detA| |Q|^3 s^(-3/2) / (|N_k| |M|),  s = d0.d0,
  // with C1 = (p10 - x0).N1 (N1 = e11 x e12, constant on the triangle),
  // detA = det[C1 - C0, C2 - C0] (cell -> triangle barycentrics).
  V3 N1 = cross(e11, e12);
  double C1 = dot(T.p[0] - x0, N1);
  V3 Nk = cross(R.e1, R.e2);
  double detA = (C[1].u - C[0].u) * (C[2].v - C[0].v) - (C[1].v - C[0].v) * (C[2].u - C[0].u);
  double K = I0 * std::fabs(C1) * std::fabs(detA) / norm(Nk);
  if (sm == 0) {
    r.flags |= F_FOLD;
    r.e_lo = 0.0;
    r.e_hi = std::numeric_limits<double>::infinity();
    finish();
    return;
  }
  Poly s = pv_dot(d0, d0);
  double a, b, dlo, dhi;
  chord_inv32(pmin(s), pmax(s), &a, &b, &dlo, &dhi);
  Poly Q3 = pmul(pmul(Q, Q), Q);
  if (sq < 0) Q3 = pscale(Q3, -1.0);  // |Q|^3 on a cell where Q has one sign
  Poly Mn = pelevate_to(M, 11);
  if (sm < 0) Mn = pscale(Mn, -1.0);
  double lo = std::numeric_limits<double>::infinity(), hi = -lo;
  for (int j = 0; j < 2; ++j) {  // remainder variable xi in {0, 1}: delta = dlo, dhi
    Poly F = padd(pscale(s, a), pconst(2, 2, b + (j == 0 ? dlo : dhi)));
    Poly N = pmul(Q3, F);
    double l, h;
    ratio_bound(N, Mn, &l, &h);
    lo = std::min(lo, l);
    hi = std::max(hi, h);
  }
  r.e_lo = K * lo;
  r.e_hi = K * hi;
  finish();
}

// Bound one cell of one (emitter, triangle) tuple for single refraction (Eq. eq_refr_rational,
// refraction; Sec. 4.3 "Remainder variables").  sqrt(beta) is replaced by
//   r~(beta, xi) = a beta + b + (1 - xi) dlo + xi dhi,   xi in [0, 1],
// with the chord of sqrt on the cell's range of beta; every quantity below is affine in r~,
// so it is a degree-(n, 1) Bernstein form on the product of the cell and [0, 1] (xi), stored
// as its two faces xi = 0 and xi = 1, and the ratio bound runs over the coefficients of both
// faces.  Readings: the normals face the incident side (d0.n < 0 on real paths); a cell where
// beta < 0 everywhere has no refracted path (total internal reflection: flag TIR); beta < 0
// elsewhere is clipped from the chord's range (no path exists there); a mixed-sign denominator
// is split up to the extra-split limit and then kept with the universal box [0,1]^2.
void bound_cell_refract(const Ctx& cx, int e, int t, uint32_t id, int depth, std::vector<orc_record>& out) {
  UV C[3];
  cell_corners(id, depth, C);
  Tri T = get_tri(cx.s1, t);
  V3 x0 = {cx.em->x[e], cx.em->y[e], cx.em->z[e]};
  V3 e11 = T.p[1] - T.p[0], e12 = T.p[2] - T.p[0];
  V3 n1d = T.n[1] - T.n[0], n2d = T.n[2] - T.n[0];
  V3 xc[3], nc[3];
  for (int k = 0; k < 3; ++k) {
    xc[k] = T.p[0] + C[k].u * e11 + C[k].v * e12;  // Eq. eq_xi
    nc[k] = T.n[0] + C[k].u * n1d + C[k].v * n2d;  // Eq. eq_ni
  }
  PV x1 = pv_affine(xc[0], xc[1], xc[2]);
  PV n1 = pv_affine(nc[0], nc[1], nc[2]);
  PV d0 = pv_subc(x1, x0);
  const double eta = cx.s1->eta;
  Poly nn = pv_dot(n1, n1), dn = pv_dot(d0, n1), ss = pv_dot(d0, d0);
  // beta = (1 - eta'^2) (n.n)(d0.d0) + eta'^2 (d0.n)^2   (degree 4)
  Poly beta = padd(pscale(pmul(nn, ss), 1.0 - eta * eta), pscale(pmul(dn, dn), eta * eta));
  const Rec& R = cx.rec;
  PV w = pv_subc(x1, R.p0);
  Poly Tn = pv_dotc(pv_crossc(w, R.e1), R.e2);  // t = Tn / Q (forward distance)

  orc_record r;
  std::memset(&r, 0, sizeof(r));
  r.emitter = e;
  r.tri0 = t;
  r.tri1 = -1;
  r.cell = id;
  r.flags = (uint32_t)depth << 24;

  const double blo = pmin(beta), bhi = pmax(beta);
  if (!(bhi > 0.0)) {
    r.flags |= F_TIR;
    out.push_back(r);
    return;
  }
  double a, b, dlo, dhi;
  chord_sqrt(std::max(blo, 0.0), bhi, &a, &b, &dlo, &dhi);
  // tangential part eta' ((n.n) d0 - (d0.n) n), degree 3, elevated to 5
  PV tang = pv_elev(pv_scale(pv_sub(pv_mul(nn, d0), pv_mul(dn, n1)), eta), 5);
  Poly Qf[2], Puf[2], Pvf[2];
  for (int j = 0; j < 2; ++j) {
    Poly W = padd(pscale(beta, a), pconst(2, 4, b + (j == 0 ? dlo : dhi)));  // r~ at xi = j
    PV dt = pv_sub(tang, pv_mul(W, n1));                                    // degree 5
    PV dxe2 = pv_crossc(dt, R.e2);
    Qf[j] = pv_dotc(dxe2, R.e1);                // Eq. eq_rct
    Puf[j] = pv_dot(dxe2, w);
    Pvf[j] = pv_dot(pv_crossc(w, R.e1), dt);
  }
  r.q_cond = std::min(cond_of(Qf[0]), cond_of(Qf[1]));
  const int s0 = psign(Qf[0]), s1 = psign(Qf[1]);
  const int sq = s0 == s1 ? s0 : 0;
  if (sq == 0) {
    if (depth < cx.max_total_depth) {
      r.flags |= F_SPLIT;
      out.push_back(r);
      for (int k = 0; k < 4; ++k) bound_cell_refract(cx, e, t, id * 4u + (uint32_t)k, depth + 1, out);
      return;
    }
    r.u_lo = r.v_lo = 0.0;
    r.u_hi = r.v_hi = 1.0;
    r.e_hi = std::numeric_limits<double>::infinity();
    r.flags |= F_LIVE | F_POS_UNBOUNDED;
    out.push_back(r);
    return;
  }
  int st = psign(Tn);
  if (st != 0 && st != sq) {
    r.flags |= F_CULL_BEHIND;
    out.push_back(r);
    return;
  }
  double ul = std::numeric_limits<double>::infinity(), uh = -ul, vl = ul, vh = -ul;
  for (int j = 0; j < 2; ++j) {
    Poly Q6 = pelevate(Qf[j]);
    double l, h;
    ratio_bound(Puf[j], Q6, &l, &h);
    ul = std::min(ul, l);
    uh = std::max(uh, h);
    ratio_bound(Pvf[j], Q6, &l, &h);
    vl = std::min(vl, l);
    vh = std::max(vh, h);
  }
  r.u_lo = std::max(ul, 0.0);
  r.u_hi = std::min(uh, 1.0);
  r.v_lo = std::max(vl, 0.0);
  r.v_hi = std::min(vh, 1.0);
  if (r.u_lo > r.u_hi || r.v_lo > r.v_hi) {
    r.u_lo = r.u_hi = r.v_lo = r.v_hi = 0.0;
    r.flags |= F_CULL_EMPTY;
    out.push_back(r);
    return;
  }
  r.flags |= F_LIVE;
  r.e_lo = 0.0;
  r.e_hi = std::numeric_limits<double>::infinity();
  auto finish = [&]() {
    const bool split = adaptive_split(cx, r, depth);
    out.push_back(r);
    if (split)
      for (int k = 0; k < 4; ++k) bound_cell_refract(cx, e, t, id * 4u + (uint32_t)k, depth + 1, out);
  };
  if (!cx.irradiance) {
    finish();
    return;
  }
  // Irradiance (Eqs. eq_dwda, eq_irr_term3a) with sqrt(beta) kept as the symbol W: the
  // derivatives of d~ are scaled by 2W, which clears dW = d beta / (2W):
  //   2W d_j d~ = (-(d_j beta) n - 2 beta d_j n) + W (2 d_j G),   G = eta' ((n.n) d0 - (d0.n) n),
  // and the same scaling of d_j A, d_j B, d_j Q gives M' = (2W)^2 M = 4 beta M, so
  //   E = I0 |C1| |detA| |Q|^3 4 beta s^(-3/2) / (|N_k| |M'|).
  // W is then replaced by the remainder form (xi1) and s^(-3/2) by its chord (xi2); the ratio
  // bound runs over the (cell, xi1, xi2) product domain.  A mixed-sign M' is a fold (E = +inf).
  {
    Poly beta_d[2] = {pderiv(beta, 1), pderiv(beta, 2)};
    Poly G[3], nc3[3] = {n1.x, n1.y, n1.z}, d0c[3] = {d0.x, d0.y, d0.z};
    for (int c = 0; c < 3; ++c) G[c] = pscale(padd(pmul(nn, d0c[c]), pmul(dn, nc3[c]), -1.0), eta);
    WP dt[3], Dt[2][3];
    for (int c = 0; c < 3; ++c) {
      dt[c] = {G[c], pscale(nc3[c], -1.0)};
      for (int j = 0; j < 2; ++j)
        Dt[j][c] = {padd(pscale(pmul(beta_d[j], nc3[c]), -1.0), pscale(pmul(beta, pderiv(nc3[c], j + 1)), -2.0)),
                    pscale(pderiv(G[c], j + 1), 2.0)};
    }
    const V3 gv = cross(R.e2, R.e1);
    const double g[3] = {gv.x, gv.y, gv.z};
    PV hu = pv_crossc(w, R.e2);  // h_u = e2 x w  ->  w x e2 negated below
    hu = pv_scale(hu, -1.0);
    PV hv = pv_crossc(w, R.e1);  // h_v = w x e1
    Poly huc[3] = {hu.x, hu.y, hu.z}, hvc[3] = {hv.x, hv.y, hv.z};
    auto zero = [](int n) { return WP{pconst(2, n, 0.0), pconst(2, n, 0.0)}; };
    WP Qw = zero(0), Aw = zero(0), Bw = zero(0), Qt[2] = {zero(0), zero(0)}, At[2] = {zero(0), zero(0)},
       Bt[2] = {zero(0), zero(0)};
    for (int c = 0; c < 3; ++c) {
      Qw = wp_add(Qw, {pscale(dt[c].p0, g[c]), pscale(dt[c].p1, g[c])});
      Aw = wp_add(Aw, wp_mulp(dt[c], huc[c]));
      Bw = wp_add(Bw, wp_mulp(dt[c], hvc[c]));
      for (int j = 0; j < 2; ++j) {
        Qt[j] = wp_add(Qt[j], {pscale(Dt[j][c].p0, g[c]), pscale(Dt[j][c].p1, g[c])});
        const Poly dhu = pderiv(huc[c], j + 1), dhv = pderiv(hvc[c], j + 1);
        // 2W d~ . d_j h = (-2 beta n . d_j h) + W (2 G . d_j h)
        const WP tu = {pscale(pmul(pmul(beta, nc3[c]), dhu), -2.0), pscale(pmul(G[c], dhu), 2.0)};
        const WP tv = {pscale(pmul(pmul(beta, nc3[c]), dhv), -2.0), pscale(pmul(G[c], dhv), 2.0)};
        At[j] = wp_add(At[j], wp_add(wp_mulp(Dt[j][c], huc[c]), tu));
        Bt[j] = wp_add(Bt[j], wp_add(wp_mulp(Dt[j][c], hvc[c]), tv));
      }
    }
    WP X = wp_add(wp_mul(At[0], Bt[1], beta), wp_mul(At[1], Bt[0], beta), -1.0);
    WP Y = wp_add(wp_mul(At[0], Qt[1], beta), wp_mul(At[1], Qt[0], beta), -1.0);
    WP Z = wp_add(wp_mul(Qt[0], Bt[1], beta), wp_mul(Qt[1], Bt[0], beta), -1.0);
    WP Mp = wp_add(wp_add(wp_mul(Qw, X, beta), wp_mul(Bw, Y, beta), -1.0), wp_mul(Aw, Z, beta), -1.0);
    WP Q3 = wp_mul(wp_mul(Qw, Qw, beta), Qw, beta);
    Poly Mf[2], Q3f[2];
    int sm[2];
    for (int j = 0; j < 2; ++j) {
      Poly W = padd(pscale(beta, a), pconst(2, 4, b + (j == 0 ? dlo : dhi)));
      Mf[j] = wp_at(Mp, W);
      Q3f[j] = pscale(wp_at(Q3, W), (double)sq);
      sm[j] = psign(Mf[j]);
    }
    r.m_cond = std::min(cond_of(Mf[0]), cond_of(Mf[1]));
    if (sm[0] == 0 || sm[0] != sm[1]) {
      r.flags |= F_FOLD;
      finish();
      return;
    }
    V3 N1 = cross(e11, e12);
    double C1 = dot(T.p[0] - x0, N1);
    V3 Nk = cross(R.e1, R.e2);
    double detA = (C[1].u - C[0].u) * (C[2].v - C[0].v) - (C[1].v - C[0].v) * (C[2].u - C[0].u);
    double K = cx.em->intensity[e] * std::fabs(C1) * std::fabs(detA) / norm(Nk);
    double sa, sb, sdlo, sdhi;
    chord_inv32(pmin(ss), pmax(ss), &sa, &sb, &sdlo, &sdhi);
    const Poly beta4 = pscale(beta, 4.0);
    double lo = std::numeric_limits<double>::infinity(), hi = -lo;
    for (int j = 0; j < 2; ++j) {
      const Poly num0 = pmul(Q3f[j], beta4);
      Poly den = pscale(Mf[j], (double)sm[j]);
      for (int k = 0; k < 2; ++k) {
        Poly F = padd(pscale(ss, sa), pconst(2, 2, sb + (k == 0 ? sdlo : sdhi)));
        Poly N = pmul(num0, F);
        double l, h;
        ratio_bound(N, pelevate_to(den, N.n), &l, &h);
        lo = std::min(lo, l);
        hi = std::max(hi, h);
      }
    }
    r.e_lo = K * std::max(lo, 0.0);
    r.e_hi = K * hi;
  }
  finish();
}

void decode_work(int64_t i, int n_tris, int depth, int* e, int* t, uint32_t* c) {
  int64_t per = (int64_t)1 << (2 * depth);
  *c = (uint32_t)(i % per);
  int64_t tup = i / per;
  *t = (int)(tup % n_tris);
  *e = (int)(tup / n_tris);
}

template <class F>
void parallel_for(int64_t n, int n_threads, F f) {
  if (n_threads <= 1 || n < 2 * n_threads) {
    f(0, (int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + n_threads - 1) / n_threads;
  for (int k = 0; k < n_threads; ++k) {
    int64_t a = k * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=]() { f(k, a, b); });
  }
  for (auto& x : th) x.join();
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Uniform in [0,1) with 24 bits, from the first output word.
float philox_uniform(uint64_t seed, int64_t point, uint64_t key) {
  uint32_t ctr[4] = {(uint32_t)point, (uint32_t)((uint64_t)point >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, k, o);
  return (float)(o[0] >> 8) * (1.0f / 16777216.0f);
}

// float32 product rounded toward +inf, emulated exactly: the double product of
// two floats is exact, then rounded up to the next float when needed.
float fmul_ru32(float a, float b) {
  double p = (double)a * (double)b;
  float f = (float)p;
  if ((double)f < p) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}

// ---------------------------------------------------------------------------
// Path evaluation within a tuple (rational form, forward-mode derivatives)
// ---------------------------------------------------------------------------
struct PathEval {
  double uk, vk;       // receiver coordinates of the hit
  double J[2][2];      // d(uk,vk)/d(u1,v1)
  double t, Q;         // ray parameter numerator/denominator sign info
  double E;            // irradiance I0 dOmega0/dA_k (GGT), V = F = 1
  bool ok;
};

// kind 0: reflection, 1: refraction with eta' = eta (Eq. eq_refr_rational).  For refraction the
// derivative of sqrt(beta) is d beta / (2 sqrt(beta)); ok is false where beta <= 0 (no path).
PathEval eval_path(const Tri& T, V3 x0, double I0, const Rec& R, double u, double v, int kind, double eta) {
  PathEval P;
  V3 e1 = T.p[1] - T.p[0], e2 = T.p[2] - T.p[0];
  V3 dn1 = T.n[1] - T.n[0], dn2 = T.n[2] - T.n[0];
  V3 x = T.p[0] + u * e1 + v * e2;
  V3 n = T.n[0] + u * dn1 + v * dn2;
  V3 d0 = x - x0;
  V3 dx[2] = {e1, e2}, dnn[2] = {dn1, dn2};
  double nn = dot(n, n), dn = dot(d0, n), ss = dot(d0, d0);
  double W = 0.0;
  V3 dt;
  if (kind == 0) {
    dt = nn * d0 - 2.0 * dn * n;
  } else {
    const double beta = (1.0 - eta * eta) * nn * ss + eta * eta * dn * dn;
    if (!(beta > 0.0)) {
      P = PathEval{};
      P.ok = false;
      return P;
    }
    W = std::sqrt(beta);
    dt = eta * (nn * d0 - dn * n) - W * n;
  }
  V3 w = x - R.p0;
  V3 g = cross(R.e2, R.e1);
  double Q = dot(dt, g);
  V3 he2w = cross(R.e2, w), hwe1 = cross(w, R.e1);
  double A = dot(dt, he2w), B = dot(hwe1, dt);
  double dA[2], dB[2], dQ[2];
  for (int j = 0; j < 2; ++j) {
    double dnn_j = 2.0 * dot(n, dnn[j]);
    double ddn_j = dot(dx[j], n) + dot(d0, dnn[j]);
    V3 ddt;
    if (kind == 0) {
      ddt = dnn_j * d0 + nn * dx[j] - 2.0 * (ddn_j * n + dn * dnn[j]);
    } else {
      const double dss_j = 2.0 * dot(d0, dx[j]);
      const double dbeta_j = (1.0 - eta * eta) * (dnn_j * ss + nn * dss_j) + eta * eta * 2.0 * dn * ddn_j;
      const double dW_j = dbeta_j / (2.0 * W);
      ddt = eta * (dnn_j * d0 + nn * dx[j] - ddn_j * n - dn * dnn[j]) - dW_j * n - W * dnn[j];
    }
    dQ[j] = dot(ddt, g);
    dA[j] = dot(ddt, he2w) + dot(dt, cross(R.e2, dx[j]));
    dB[j] = dot(cross(dx[j], R.e1), dt) + dot(hwe1, ddt);
  }
  P.Q = Q;
  P.t = dot(hwe1, R.e2) / Q;
  P.uk = A / Q;
  P.vk = B / Q;
  for (int j = 0; j < 2; ++j) {
    P.J[0][j] = (dA[j] * Q - A * dQ[j]) / (Q * Q);
    P.J[1][j] = (dB[j] * Q - B * dQ[j]) / (Q * Q);
  }
  double detJ = P.J[0][0] * P.J[1][1] - P.J[0][1] * P.J[1][0];
  V3 N1 = cross(e1, e2);
  double C1 = dot(T.p[0] - x0, N1);
  double s = ss;
  P.E = I0 * std::fabs(C1) / (s * std::sqrt(s) * norm(cross(R.e1, R.e2)) * std::fabs(detJ));
  P.ok = std::isfinite(P.uk) && std::isfinite(P.vk) && std::isfinite(detJ) && Q != 0.0;
  return P;
}

// Independent direct-geometry evaluator: normalized normal, vector reflection,
// ray/plane hit, and the Jacobian by forward-mode dual numbers through those
// operations.  Used only by the pins (containment sweeps).
struct Dual {
  double v, d[2];
};
Dual dmk(double v, double a, double b) { return {v, {a, b}}; }
Dual operator+(Dual a, Dual b) { return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1]}}; }
Dual operator-(Dual a, Dual b) { return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1]}}; }
Dual operator*(Dual a, Dual b) { return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1]}}; }
Dual operator/(Dual a, Dual b) {
  double iv = 1.0 / b.v;
  return {a.v * iv, {(a.d[0] - a.v * iv * b.d[0]) * iv, (a.d[1] - a.v * iv * b.d[1]) * iv}};
}
Dual dsqrt(Dual a) {
  double s = std::sqrt(a.v);
  return {s, {a.d[0] / (2 * s), a.d[1] / (2 * s)}};
}
Dual dc(double v) { return {v, {0, 0}}; }
struct DV3 {
  Dual x, y, z;
};
DV3 operator+(DV3 a, DV3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
DV3 operator-(DV3 a, DV3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
DV3 operator*(Dual s, DV3 a) { return {s * a.x, s * a.y, s * a.z}; }
Dual ddot(DV3 a, DV3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
DV3 dconst(V3 a) { return {dc(a.x), dc(a.y), dc(a.z)}; }

bool eval_direct_reflect(const Tri& T, V3 x0, double I0, const Rec& R, double u, double v, double* uk,
                         double* vk, double* E, double* tt) {
  Dual U = dmk(u, 1, 0), W = dmk(v, 0, 1);
  DV3 p0 = dconst(T.p[0]), e1 = dconst(T.p[1] - T.p[0]), e2 = dconst(T.p[2] - T.p[0]);
  DV3 x = p0 + U * e1 + W * e2;
  DV3 n = dconst(T.n[0]) + U * dconst(T.n[1] - T.n[0]) + W * dconst(T.n[2] - T.n[0]);
  Dual ln = dsqrt(ddot(n, n));
  DV3 nh = {n.x / ln, n.y / ln, n.z / ln};
  DV3 d = x - dconst(x0);
  DV3 r = d - (dc(2.0) * ddot(d, nh)) * nh;  // mirror reflection of the incident direction
  V3 Nk = cross(R.e1, R.e2);
  DV3 Nkd = dconst(Nk);
  Dual t = ddot(dconst(R.p0) - x, Nkd) / ddot(r, Nkd);
  DV3 X = x + t * r;
  // receiver coordinates via the dual basis of (e1, e2) in the receiver plane
  double g11 = dot(R.e1, R.e1), g12 = dot(R.e1, R.e2), g22 = dot(R.e2, R.e2);
  double det = g11 * g22 - g12 * g12;
  DV3 rel = X - dconst(R.p0);
  Dual a = ddot(rel, dconst(R.e1)), b = ddot(rel, dconst(R.e2));
  Dual Uk = (dc(g22) * a - dc(g12) * b) / dc(det);
  Dual Vk = (dc(g11) * b - dc(g12) * a) / dc(det);
  double detJ = Uk.d[0] * Vk.d[1] - Uk.d[1] * Vk.d[0];
  V3 N1 = cross(T.p[1] - T.p[0], T.p[2] - T.p[0]);
  V3 dd = {d.x.v, d.y.v, d.z.v};
  double s = dot(dd, dd);
  // GGT (Eq. eq_dwda): dOmega0/dA1 |dx1/du1| = |d0.N1| / |d0|^3, |du_k/dx_k| = 1/|N_k|
  *E = I0 * std::fabs(dot(dd, N1)) / (s * std::sqrt(s)) / (std::fabs(detJ) * norm(Nk));
  *uk = Uk.v;
  *vk = Vk.v;
  *tt = t.v;
  return std::isfinite(Uk.v) && std::isfinite(Vk.v);
}

// Direct geometry for refraction: unit normal and unit incident direction, the textbook vector
// form of Snell's law t = eta i + (eta c1 - sqrt(1 - eta^2 (1 - c1^2))) n with c1 = -i.n (the
// normal faces the incident side), ray/plane hit, Jacobian by duals.  Returns false under total
// internal reflection.
bool eval_direct_refract(const Tri& T, V3 x0, double I0, const Rec& R, double eta, double u, double v, double* uk,
                         double* vk, double* E, double* tt) {
  Dual U = dmk(u, 1, 0), W = dmk(v, 0, 1);
  DV3 p0 = dconst(T.p[0]), e1 = dconst(T.p[1] - T.p[0]), e2 = dconst(T.p[2] - T.p[0]);
  DV3 x = p0 + U * e1 + W * e2;
  DV3 n = dconst(T.n[0]) + U * dconst(T.n[1] - T.n[0]) + W * dconst(T.n[2] - T.n[0]);
  Dual ln = dsqrt(ddot(n, n));
  DV3 nh = {n.x / ln, n.y / ln, n.z / ln};
  DV3 d = x - dconst(x0);
  Dual ld = dsqrt(ddot(d, d));
  DV3 ih = {d.x / ld, d.y / ld, d.z / ld};
  Dual c1 = dc(0.0) - ddot(ih, nh);
  Dual k = dc(1.0) - dc(eta * eta) * (dc(1.0) - c1 * c1);
  if (!(k.v > 0.0)) return false;
  DV3 tdir = dc(eta) * ih + (dc(eta) * c1 - dsqrt(k)) * nh;
  V3 Nk = cross(R.e1, R.e2);
  DV3 Nkd = dconst(Nk);
  Dual t = ddot(dconst(R.p0) - x, Nkd) / ddot(tdir, Nkd);
  DV3 X = x + t * tdir;
  double g11 = dot(R.e1, R.e1), g12 = dot(R.e1, R.e2), g22 = dot(R.e2, R.e2);
  double det = g11 * g22 - g12 * g12;
  DV3 rel = X - dconst(R.p0);
  Dual a = ddot(rel, dconst(R.e1)), b = ddot(rel, dconst(R.e2));
  Dual Uk = (dc(g22) * a - dc(g12) * b) / dc(det);
  Dual Vk = (dc(g11) * b - dc(g12) * a) / dc(det);
  double detJ = Uk.d[0] * Vk.d[1] - Uk.d[1] * Vk.d[0];
  V3 N1 = cross(T.p[1] - T.p[0], T.p[2] - T.p[0]);
  V3 dd = {d.x.v, d.y.v, d.z.v};
  double s = dot(dd, dd);
  *E = I0 * std::fabs(dot(dd, N1)) / (s * std::sqrt(s)) / (std::fabs(detJ) * norm(Nk));
  *uk = Uk.v;
  *vk = Vk.v;
  *tt = t.v;
  return std::isfinite(Uk.v) && std::isfinite(Vk.v);
}

// ---------------------------------------------------------------------------
// Two specular vertices: chains x0 -> T1 -> T2 -> receiver with refraction at both
// vertices (the TT chains of Table "tab:perf", e.g. the glass slab).
//
//   * Tuple construction (Sec. 6.1): for one cell of T1, every refracted ray that reaches
//     the z-band of a triangle T2 crosses it at x2 = x1 + s d~1 (s > 0), so
//     x2.xy = x1.xy + (x2.z - x1.z) (d~1x / d~1z, d~1y / d~1z).  The box of x1 (its
//     corner values) and the ratio bounds of the two direction ratios (Eq. eq_bbound,
//     over both xi1 faces) give an xy footprint; T2 is a candidate of the cell when its
//     xy box meets the footprint for T2's own z-range.
//   * Composite position bound: u2 = P2 / Q2 (Eq. eq_rct with d~1 of Eq.
//     eq_refr_rational) is reduced to degree 1 plus a remainder (Sec. 6.1 "Degree
//     reduction"): l(u1) interpolates u2 at the cell corners (at xi1 = 1/2) and the
//     ratio bound of (P2 - l Q2) / Q2 over the cell and xi1 bounds u2 - l.  The
//     reduction drops xi1.  The second vertex is then built from that degree-1 form
//     with its remainder carried as a radius: a "model" p + e, |e| <= r on the cell,
//     with r(a b) = |a| r_b + |b| r_a + r_a r_b (|a| the largest classical coefficient,
//     a bound of |a| on the cell).  The second refraction and the receiver forms are
//     those of a single refraction, and the final ratio bound divides the coefficient
//     intervals [b - r, b + r].
//   * The irradiance of a chain is not bounded (e_hi = +inf, so P = 1 in Algorithm 1).
// ---------------------------------------------------------------------------
double pmaxabs(const Poly& p) {
  double m = 0.0;
  for (double v : p.c) m = std::max(m, std::fabs(v));
  return m;
}

struct MP {  // model: polynomial p plus a remainder bounded by r on the whole cell
  Poly p;
  double r = 0.0;
};
MP mp_add(const MP& a, const MP& b, double sb = 1.0) { return {padd(a.p, b.p, sb), a.r + std::fabs(sb) * b.r}; }
MP mp_mul(const MP& a, const MP& b) { return {pmul(a.p, b.p), pmaxabs(a.p) * b.r + pmaxabs(b.p) * a.r + a.r * b.r}; }
MP mp_scale(const MP& a, double s) { return {pscale(a.p, s), std::fabs(s) * a.r}; }
MP mp_shift(MP a, double c) {
  for (auto& v : a.p.c) v += c;
  return a;
}
MP mp_elev(const MP& a, int n) { return {pelevate_to(a.p, n), a.r}; }
// +1 / -1 when every coefficient interval [b - r, b + r] lies above / below zero.
int mp_sign(const MP& a) {
  bool pos = true, neg = true;
  for (double v : a.p.c) {
    if (!(v - a.r > 0.0)) pos = false;
    if (!(v + a.r < 0.0)) neg = false;
  }
  return pos ? 1 : (neg ? -1 : 0);
}
// Ratio bound with interval coefficients (p/q is a weighted mean of (b_p + e_p)/(b_q + e_q) for the
// one pair of remainders e_p, e_q at each point); sq = the certified sign of q's intervals.
void mp_ratio_bound(const MP& p, const MP& q, int sq, double* lo, double* hi) {
  double l = std::numeric_limits<double>::infinity(), h = -l;
  for (size_t i = 0; i < p.p.c.size(); ++i) {
    double pl = p.p.c[i] - p.r, ph = p.p.c[i] + p.r, ql = q.p.c[i] - q.r, qh = q.p.c[i] + q.r;
    if (sq < 0) {
      double t = pl;
      pl = -ph;
      ph = -t;
      t = ql;
      ql = -qh;
      qh = -t;
    }
    l = std::min(l, pl >= 0.0 ? pl / qh : pl / ql);
    h = std::max(h, ph >= 0.0 ? ph / ql : ph / qh);
  }
  *lo = l;
  *hi = h;
}
double mp_cond(const MP& a) {
  double mn = std::numeric_limits<double>::infinity(), mx = 0.0;
  for (double v : a.p.c) {
    mn = std::min(mn, std::fabs(v) - a.r);
    mx = std::max(mx, std::fabs(v));
  }
  return mx > 0 ? std::max(mn, 0.0) / mx : 0.0;
}

struct MV {
  MP x, y, z;
};
MP mv_dot(const MV& a, const MV& b) { return mp_add(mp_add(mp_mul(a.x, b.x), mp_mul(a.y, b.y)), mp_mul(a.z, b.z)); }
MP mv_dotc(const MV& a, V3 c) { return mp_add(mp_add(mp_scale(a.x, c.x), mp_scale(a.y, c.y)), mp_scale(a.z, c.z)); }
MV mv_mul(const MP& s, const MV& a) { return {mp_mul(s, a.x), mp_mul(s, a.y), mp_mul(s, a.z)}; }
MV mv_sub(const MV& a, const MV& b) { return {mp_add(a.x, b.x, -1.0), mp_add(a.y, b.y, -1.0), mp_add(a.z, b.z, -1.0)}; }
MV mv_scale(const MV& a, double s) { return {mp_scale(a.x, s), mp_scale(a.y, s), mp_scale(a.z, s)}; }
MV mv_elev(const MV& a, int n) { return {mp_elev(a.x, n), mp_elev(a.y, n), mp_elev(a.z, n)}; }
MV mv_crossc(const MV& a, V3 b) {  // a x b, b constant
  return {mp_add(mp_scale(a.y, b.z), mp_scale(a.z, b.y), -1.0), mp_add(mp_scale(a.z, b.x), mp_scale(a.x, b.z), -1.0),
          mp_add(mp_scale(a.x, b.y), mp_scale(a.y, b.x), -1.0)};
}

// The first vertex on one cell of T1: x1 (degree 1) and the scattered d~1 on the faces xi1 = 0, 1
// (degree 5): refraction as in the single-refraction bound; reflection (kind 0) has no remainder,
// d~1 = (n.n) d0 - 2 (d0.n) n on both faces (degree 3, elevated).
struct Vertex1 {
  bool tir = false;
  PV x1;
  PV dt[2];
  double ca = 0.0, cb = 0.0, dlo = 0.0, dhi = 0.0;  // refraction: chord of sqrt(beta) and its remainder range
};

Vertex1 first_vertex(const Tri& T, V3 x0, int kind, double eta, const UV C[3]) {
  Vertex1 S;
  V3 e11 = T.p[1] - T.p[0], e12 = T.p[2] - T.p[0];
  V3 n1d = T.n[1] - T.n[0], n2d = T.n[2] - T.n[0];
  V3 xc[3], nc[3];
  for (int k = 0; k < 3; ++k) {
    xc[k] = T.p[0] + C[k].u * e11 + C[k].v * e12;  // Eq. eq_xi
    nc[k] = T.n[0] + C[k].u * n1d + C[k].v * n2d;  // Eq. eq_ni
  }
  S.x1 = pv_affine(xc[0], xc[1], xc[2]);
  PV n1 = pv_affine(nc[0], nc[1], nc[2]);
  PV d0 = pv_subc(S.x1, x0);
  Poly nn = pv_dot(n1, n1), dn = pv_dot(d0, n1), ss = pv_dot(d0, d0);
  if (kind == 0) {  // Eq. eq_refr_rational, reflection
    S.dt[0] = S.dt[1] = pv_elev(pv_sub(pv_mul(nn, d0), pv_mul(dn, n1), 2.0), 5);
    return S;
  }
  Poly beta = padd(pscale(pmul(nn, ss), 1.0 - eta * eta), pscale(pmul(dn, dn), eta * eta));
  const double blo = pmin(beta), bhi = pmax(beta);
  if (!(bhi > 0.0)) {
    S.tir = true;
    return S;
  }
  double a, b, dlo, dhi;
  chord_sqrt(std::max(blo, 0.0), bhi, &a, &b, &dlo, &dhi);
  S.ca = a;
  S.cb = b;
  S.dlo = dlo;
  S.dhi = dhi;
  PV tang = pv_elev(pv_scale(pv_sub(pv_mul(nn, d0), pv_mul(dn, n1)), eta), 5);
  for (int j = 0; j < 2; ++j) {
    Poly W = padd(pscale(beta, a), pconst(2, 4, b + (j == 0 ? dlo : dhi)));
    S.dt[j] = pv_sub(tang, pv_mul(W, n1));
  }
  return S;
}

// The cell's ray bundle for tuple construction: the x1 box (corner values), the certified sign of
// d~1z and the ratio bounds of d~1x / d~1z, d~1y / d~1z over both xi1 faces.  kind 0: no refracted
// ray (total internal reflection); 1: bounded; 2: the sign of d~1z is not certified.
struct Bundle {
  int kind = 0, sz = 0;
  double x[2], y[2], z[2], rx[2], ry[2];
};

Bundle ray_bundle(const Vertex1& S) {
  Bundle B;
  if (S.tir) return B;
  const int s0 = psign(S.dt[0].z), s1 = psign(S.dt[1].z);
  if (s0 == 0 || s0 != s1) {
    B.kind = 2;
    return B;
  }
  B.kind = 1;
  B.sz = s0;
  B.rx[0] = B.ry[0] = std::numeric_limits<double>::infinity();
  B.rx[1] = B.ry[1] = -std::numeric_limits<double>::infinity();
  for (int j = 0; j < 2; ++j) {
    double l, h;
    ratio_bound(S.dt[j].x, S.dt[j].z, &l, &h);
    B.rx[0] = std::min(B.rx[0], l);
    B.rx[1] = std::max(B.rx[1], h);
    ratio_bound(S.dt[j].y, S.dt[j].z, &l, &h);
    B.ry[0] = std::min(B.ry[0], l);
    B.ry[1] = std::max(B.ry[1], h);
  }
  B.x[0] = pmin(S.x1.x);
  B.x[1] = pmax(S.x1.x);
  B.y[0] = pmin(S.x1.y);
  B.y[1] = pmax(S.x1.y);
  B.z[0] = pmin(S.x1.z);
  B.z[1] = pmax(S.x1.z);
  return B;
}

// Footprint f = {xlo, xhi, ylo, yhi} of a bounded bundle on the band zlo <= z <= zhi.  Returns
// false when no forward ray reaches the band.
bool footprint(const Bundle& B, double zlo, double zhi, double f[4]) {
  double dzl = zlo - B.z[1], dzh = zhi - B.z[0];
  if (B.sz < 0)
    dzh = std::min(dzh, 0.0);
  else
    dzl = std::max(dzl, 0.0);
  if (dzl > dzh) return false;
  auto span = [&](const double x[2], const double r[2], double* ol, double* oh) {
    const double p[4] = {dzl * r[0], dzl * r[1], dzh * r[0], dzh * r[1]};
    *ol = x[0] + *std::min_element(p, p + 4);
    *oh = x[1] + *std::max_element(p, p + 4);
  };
  span(B.x, B.rx, &f[0], &f[1]);
  span(B.y, B.ry, &f[2], &f[3]);
  return true;
}

struct Box3 {
  double lo[3], hi[3];
};
Box3 tri_box(const Tri& T) {
  Box3 b;
  for (int c = 0; c < 3; ++c) {
    auto comp = [&](const V3& v) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); };
    b.lo[c] = std::min(comp(T.p[0]), std::min(comp(T.p[1]), comp(T.p[2])));
    b.hi[c] = std::max(comp(T.p[0]), std::max(comp(T.p[1]), comp(T.p[2])));
  }
  return b;
}

// Candidate test of T2 for a cell (Sec. 6.1 "Tuple construction"); *gap > 0 is the distance by which
// T2's xy box misses the footprint for T2's own z-range (<= 0: they meet), +inf when no ray reaches
// T2's band, -inf when every triangle is a candidate.
bool pair_candidate(const Bundle& B, const Box3& b, double* gap) {
  const double inf = std::numeric_limits<double>::infinity();
  if (B.kind == 0) {
    *gap = inf;
    return false;
  }
  if (B.kind == 2) {
    *gap = -inf;
    return true;
  }
  double f[4];
  if (!footprint(B, b.lo[2], b.hi[2], f)) {
    *gap = inf;
    return false;
  }
  *gap = std::max(std::max(b.lo[0] - f[1], f[0] - b.hi[0]), std::max(b.lo[1] - f[3], f[2] - b.hi[1]));
  return *gap <= 0.0;
}

// Direct geometry of the chain: unit normals, the vector form of Snell's law (or of the mirror law) at
// each vertex,
// ray/plane hits (T2's plane, then the receiver's), derivatives by duals.  u2, v2: barycentrics of
// the hit on T2's plane; t1, t2: ray parameters of the two hits (forward when > 0).
struct PairEval {
  double uk, vk, detJ, u2, v2, t1, t2, E;
  double J[2][2];
  bool ok;
};

void plane_coords(DV3 rel, V3 a, V3 b, Dual* U, Dual* V) {  // rel = U a + V b in the plane of a, b
  const double g11 = dot(a, a), g12 = dot(a, b), g22 = dot(b, b);
  const double det = g11 * g22 - g12 * g12;
  Dual pa = ddot(rel, dconst(a)), pb = ddot(rel, dconst(b));
  *U = (dc(g22) * pa - dc(g12) * pb) / dc(det);
  *V = (dc(g11) * pb - dc(g12) * pa) / dc(det);
}

bool snell(DV3 ih, DV3 n, double eta, DV3* out) {  // ih unit incident direction, n normal (any length)
  Dual ln = dsqrt(ddot(n, n));
  DV3 nh = {n.x / ln, n.y / ln, n.z / ln};
  if (eta < 0.0) {  // a mirror (kind 0, passed as eta < 0): r = i - 2 (i.n) n
    *out = ih - (dc(2.0) * ddot(ih, nh)) * nh;
    return true;
  }
  Dual c1 = dc(0.0) - ddot(ih, nh);
  Dual k = dc(1.0) - dc(eta * eta) * (dc(1.0) - c1 * c1);
  if (!(k.v > 0.0)) return false;
  *out = dc(eta) * ih + (dc(eta) * c1 - dsqrt(k)) * nh;
  return true;
}

// eta1 / eta2 < 0 mark a reflecting vertex.
PairEval eval_pair_direct(const Tri& A, const Tri& B, V3 x0, double I0, const Rec& R, double eta1, double eta2,
                          double u, double v) {
  PairEval P{};
  P.ok = false;
  Dual U = dmk(u, 1, 0), W = dmk(v, 0, 1);
  DV3 x1 = dconst(A.p[0]) + U * dconst(A.p[1] - A.p[0]) + W * dconst(A.p[2] - A.p[0]);
  DV3 n1 = dconst(A.n[0]) + U * dconst(A.n[1] - A.n[0]) + W * dconst(A.n[2] - A.n[0]);
  DV3 d0 = x1 - dconst(x0);
  Dual l0 = dsqrt(ddot(d0, d0));
  DV3 i1 = {d0.x / l0, d0.y / l0, d0.z / l0};
  DV3 r1;
  if (!snell(i1, n1, eta1, &r1)) return P;
  const V3 e21 = B.p[1] - B.p[0], e22 = B.p[2] - B.p[0], N2 = cross(e21, e22);
  Dual s1 = ddot(dconst(B.p[0]) - x1, dconst(N2)) / ddot(r1, dconst(N2));
  DV3 x2 = x1 + s1 * r1;
  Dual U2, V2;
  plane_coords(x2 - dconst(B.p[0]), e21, e22, &U2, &V2);
  DV3 n2 = dconst(B.n[0]) + U2 * dconst(B.n[1] - B.n[0]) + V2 * dconst(B.n[2] - B.n[0]);
  Dual lr = dsqrt(ddot(r1, r1));
  DV3 i2 = {r1.x / lr, r1.y / lr, r1.z / lr};
  DV3 r2;
  if (!snell(i2, n2, eta2, &r2)) return P;
  const V3 Nk = cross(R.e1, R.e2);
  Dual s2 = ddot(dconst(R.p0) - x2, dconst(Nk)) / ddot(r2, dconst(Nk));
  DV3 X = x2 + s2 * r2;
  Dual Uk, Vk;
  plane_coords(X - dconst(R.p0), R.e1, R.e2, &Uk, &Vk);
  P.uk = Uk.v;
  P.vk = Vk.v;
  P.J[0][0] = Uk.d[0];
  P.J[0][1] = Uk.d[1];
  P.J[1][0] = Vk.d[0];
  P.J[1][1] = Vk.d[1];
  P.detJ = Uk.d[0] * Vk.d[1] - Uk.d[1] * Vk.d[0];
  P.u2 = U2.v;
  P.v2 = V2.v;
  P.t1 = s1.v;
  P.t2 = s2.v;
  V3 dd = {d0.x.v, d0.y.v, d0.z.v};
  const double s = dot(dd, dd);
  const V3 N1 = cross(A.p[1] - A.p[0], A.p[2] - A.p[0]);
  // GGT (Eq. eq_dwda) through both vertices: |d0.N1| / |d0|^3 / (|det du_k/du_1| |N_k|)
  P.E = I0 * std::fabs(dot(dd, N1)) / (s * std::sqrt(s)) / (std::fabs(P.detJ) * norm(Nk));
  P.ok = std::isfinite(P.uk) && std::isfinite(P.vk) && std::isfinite(P.detJ) && std::isfinite(P.u2) &&
         std::isfinite(P.v2);
  return P;
}

struct Ctx2 {
  const orc_surface *s1, *s2;
  Rec rec;
  const orc_emitters* em;
};
// The vertex law for the direct evaluator: eta' for refraction, -1 for reflection.
double law(const orc_surface* s) { return s->kind == 0 ? -1.0 : (double)s->eta; }

// Expansion point of the second vertex's receiver forms: the receiver coordinates of the chain
// through the cell's centroid (no containment test), rounded to 2^-16; per coordinate 0.5 where
// that chain has no refracted path or the coordinate is not below 4 in magnitude.  Any point gives
// a valid bound.
void centroid_hit(const Ctx2& cx, const Tri& A, const Tri& B, V3 x0, const UV C[3], double* uc, double* vc) {
  const double cu = (C[0].u + C[1].u + C[2].u) / 3.0, cv = (C[0].v + C[1].v + C[2].v) / 3.0;
  PairEval P = eval_pair_direct(A, B, x0, 1.0, cx.rec, law(cx.s1), law(cx.s2), cu, cv);
  const double a = P.ok && std::fabs(P.uk) < 4.0 ? P.uk : 0.5;
  const double b = P.ok && std::fabs(P.vk) < 4.0 ? P.vk : 0.5;
  *uc = std::nearbyint(a * 65536.0) / 65536.0;
  *vc = std::nearbyint(b * 65536.0) / 65536.0;
}

// Intermediate quantities of one pair record, for the pins that evaluate the remainder forms
// pointwise (the bound must hold over the whole product domain of the cell and the remainder
// variables, not only on true chains).
struct PairDiag {
  double chord1[4];      // vertex 1: a, b, delta_lo, delta_hi of W1 = a beta1 + b + delta (0 for reflection)
  double rx[2], ry[2];   // ratio bounds of d~1x / d~1z, d~1y / d~1z over both xi1 faces (tuple construction)
  double u2box[4];       // ratio bounds of u2, v2 over the cell and both xi1 faces
  double lu[3], lv[3];   // degree-1 interpolant of u2, v2 at the cell corners (barycentric order of C)
  double rho[4];         // remainder ranges: u2 - l_u in [rho0, rho1], v2 - l_v in [rho2, rho3]
  double chord2[4];      // vertex 2: a, b, delta_lo, delta_hi of W2 (0 for reflection)
  double uc, vc;         // expansion point of the receiver forms
  int32_t stage;         // 0: no intermediate, 1: vertex 1 only, 2: through u2, 3: complete
  int32_t pad;
};

void bound_cell_pair(const Ctx2& cx, int e, int t1, uint32_t id, int depth, int t2, orc_record& r,
                     PairDiag* dg = nullptr) {
  UV C[3];
  cell_corners(id, depth, C);
  const Tri A = get_tri(cx.s1, t1), B = get_tri(cx.s2, t2);
  const V3 x0 = {cx.em->x[e], cx.em->y[e], cx.em->z[e]};
  const Rec& R = cx.rec;
  std::memset(&r, 0, sizeof(r));
  r.emitter = e;
  r.tri0 = t1;
  r.tri1 = t2;
  r.cell = id;
  r.flags = (uint32_t)depth << 24;
  const double inf = std::numeric_limits<double>::infinity();
  auto unbounded = [&]() {
    r.u_lo = r.v_lo = 0.0;
    r.u_hi = r.v_hi = 1.0;
    r.e_hi = inf;
    r.flags |= F_LIVE | F_POS_UNBOUNDED;
  };
  const Vertex1 S = first_vertex(A, x0, cx.s1->kind, cx.s1->eta, C);
  if (dg) {
    std::memset(dg, 0, sizeof(*dg));
    dg->chord1[0] = S.ca;
    dg->chord1[1] = S.cb;
    dg->chord1[2] = S.dlo;
    dg->chord1[3] = S.dhi;
    const Bundle Bd = ray_bundle(S);
    dg->rx[0] = Bd.rx[0];
    dg->rx[1] = Bd.rx[1];
    dg->ry[0] = Bd.ry[0];
    dg->ry[1] = Bd.ry[1];
    dg->stage = Bd.kind == 1 ? 1 : 0;
  }
  if (S.tir) {
    r.flags |= F_TIR;
    return;
  }
  // u2 on T2's plane (Eq. eq_rct), both xi1 faces
  const V3 p20 = B.p[0], e21 = B.p[1] - p20, e22 = B.p[2] - p20;
  const PV w2 = pv_subc(S.x1, p20);
  Poly Q2[2], A2[2], B2[2], Q2e[2];
  for (int j = 0; j < 2; ++j) {
    PV dxe = pv_crossc(S.dt[j], e22);
    Q2[j] = pv_dotc(dxe, e21);
    A2[j] = pv_dot(dxe, w2);
    B2[j] = pv_dot(pv_crossc(w2, e21), S.dt[j]);
    Q2e[j] = pelevate(Q2[j]);
  }
  r.q_cond = std::min(cond_of(Q2[0]), cond_of(Q2[1]));
  const int s0 = psign(Q2[0]), s1 = psign(Q2[1]);
  const int sq = s0 == s1 ? s0 : 0;
  if (sq == 0) {
    unbounded();
    return;
  }
  const int st = psign(pv_dotc(pv_crossc(w2, e21), e22));
  if (st != 0 && st != sq) {
    r.flags |= F_CULL_BEHIND;
    return;
  }
  double u2l = inf, u2h = -inf, v2l = inf, v2h = -inf;
  for (int j = 0; j < 2; ++j) {
    double l, h;
    ratio_bound(A2[j], Q2e[j], &l, &h);
    u2l = std::min(u2l, l);
    u2h = std::max(u2h, h);
    ratio_bound(B2[j], Q2e[j], &l, &h);
    v2l = std::min(v2l, l);
    v2h = std::max(v2h, h);
  }
  if (u2h < 0.0 || v2h < 0.0 || u2l + v2l > 1.0) {  // no ray of the cell meets the closed triangle T2
    r.flags |= F_CULL_EMPTY;
    return;
  }
  // Degree reduction of u2, v2 to the corner interpolant at xi1 = 1/2 plus a remainder
  const int cidx[3] = {pidx(2, 6, 0, 0), pidx(2, 6, 6, 0), pidx(2, 6, 0, 6)};
  double lu[3], lv[3];
  for (int k = 0; k < 3; ++k) {
    const double q = Q2e[0].c[cidx[k]] + Q2e[1].c[cidx[k]];
    lu[k] = (A2[0].c[cidx[k]] + A2[1].c[cidx[k]]) / q;
    lv[k] = (B2[0].c[cidx[k]] + B2[1].c[cidx[k]]) / q;
  }
  const Poly Lu = paffine(lu[0], lu[1], lu[2]), Lv = paffine(lv[0], lv[1], lv[2]);
  double rul = inf, ruh = -inf, rvl = inf, rvh = -inf;
  for (int j = 0; j < 2; ++j) {
    double l, h;
    ratio_bound(padd(A2[j], pmul(Lu, Q2[j]), -1.0), Q2e[j], &l, &h);
    rul = std::min(rul, l);
    ruh = std::max(ruh, h);
    ratio_bound(padd(B2[j], pmul(Lv, Q2[j]), -1.0), Q2e[j], &l, &h);
    rvl = std::min(rvl, l);
    rvh = std::max(rvh, h);
  }
  if (dg) {
    dg->u2box[0] = u2l;
    dg->u2box[1] = u2h;
    dg->u2box[2] = v2l;
    dg->u2box[3] = v2h;
    for (int k = 0; k < 3; ++k) {
      dg->lu[k] = lu[k];
      dg->lv[k] = lv[k];
    }
    dg->rho[0] = rul;
    dg->rho[1] = ruh;
    dg->rho[2] = rvl;
    dg->rho[3] = rvh;
    dg->stage = 2;
  }
  const MP U2 = {mp_shift(MP{Lu, 0.0}, 0.5 * (rul + ruh)).p, 0.5 * (ruh - rul)};
  const MP V2 = {mp_shift(MP{Lv, 0.0}, 0.5 * (rvl + rvh)).p, 0.5 * (rvh - rvl)};
  // Second vertex: x2, n2 (Eqs. eq_xi, eq_ni on T2) affine in (U2, V2), d1 = x2 - x1
  const V3 n20 = B.n[0], f21 = B.n[1] - n20, f22 = B.n[2] - n20;
  auto on_t2 = [&](double base, double a, double b) { return mp_shift(mp_add(mp_scale(U2, a), mp_scale(V2, b)), base); };
  const MV x2 = {on_t2(p20.x, e21.x, e22.x), on_t2(p20.y, e21.y, e22.y), on_t2(p20.z, e21.z, e22.z)};
  const MV n2 = {on_t2(n20.x, f21.x, f22.x), on_t2(n20.y, f21.y, f22.y), on_t2(n20.z, f21.z, f22.z)};
  const MV d1 = mv_sub(x2, MV{{S.x1.x, 0.0}, {S.x1.y, 0.0}, {S.x1.z, 0.0}});
  const double eta = cx.s2->eta;
  const MP nn = mv_dot(n2, n2), dn = mv_dot(d1, n2), ss = mv_dot(d1, d1);
  MV dtf[2];  // d~2 on the faces xi2 = 0, 1 (degree 5)
  if (cx.s2->kind == 0) {  // reflection: (n.n) d1 - 2 (d1.n) n, no remainder
    dtf[0] = dtf[1] = mv_elev(mv_sub(mv_mul(nn, d1), mv_scale(mv_mul(dn, n2), 2.0)), 5);
  } else {
    const MP beta = mp_add(mp_scale(mp_mul(nn, ss), 1.0 - eta * eta), mp_scale(mp_mul(dn, dn), eta * eta));
    const double blo = pmin(beta.p) - beta.r, bhi = pmax(beta.p) + beta.r;
    if (!(bhi > 0.0)) {
      r.flags |= F_TIR;
      return;
    }
    double a, b, dlo, dhi;
    chord_sqrt(std::max(blo, 0.0), bhi, &a, &b, &dlo, &dhi);
    if (dg) {
      dg->chord2[0] = a;
      dg->chord2[1] = b;
      dg->chord2[2] = dlo;
      dg->chord2[3] = dhi;
    }
    const MV tang = mv_elev(mv_scale(mv_sub(mv_mul(nn, d1), mv_mul(dn, n2)), eta), 5);
    for (int j = 0; j < 2; ++j) {
      const MP Wj = mp_shift(mp_scale(beta, a), b + (j == 0 ? dlo : dhi));
      dtf[j] = mv_sub(tang, mv_mul(Wj, n2));
    }
  }
  double uc, vc;
  centroid_hit(cx, A, B, x0, C, &uc, &vc);
  if (dg) {
    dg->uc = uc;
    dg->vc = vc;
    dg->stage = 3;
  }
  const V3 pp = R.p0 + uc * R.e1 + vc * R.e2;
  const MV w3 = {mp_shift(x2.x, -pp.x), mp_shift(x2.y, -pp.y), mp_shift(x2.z, -pp.z)};
  MP Q3[2], A3[2], B3[2];
  for (int j = 0; j < 2; ++j) {
    const MV& dt = dtf[j];
    const MV dxe = mv_crossc(dt, R.e2);
    Q3[j] = mv_dotc(dxe, R.e1);
    A3[j] = mv_dot(dxe, w3);
    B3[j] = mv_dot(mv_crossc(w3, R.e1), dt);
  }
  r.m_cond = std::min(mp_cond(Q3[0]), mp_cond(Q3[1]));
  const int m0 = mp_sign(Q3[0]), m1 = mp_sign(Q3[1]);
  const int sq3 = m0 == m1 ? m0 : 0;
  if (sq3 == 0) {
    unbounded();
    return;
  }
  const int st3 = mp_sign(mv_dotc(mv_crossc(w3, R.e1), R.e2));
  if (st3 != 0 && st3 != sq3) {
    r.flags |= F_CULL_BEHIND;
    return;
  }
  double ul = inf, uh = -inf, vl = inf, vh = -inf;
  for (int j = 0; j < 2; ++j) {
    const MP Qe = mp_elev(Q3[j], 6);
    double l, h;
    mp_ratio_bound(A3[j], Qe, sq3, &l, &h);
    ul = std::min(ul, l);
    uh = std::max(uh, h);
    mp_ratio_bound(B3[j], Qe, sq3, &l, &h);
    vl = std::min(vl, l);
    vh = std::max(vh, h);
  }
  r.u_lo = std::max(uc + ul, 0.0);
  r.u_hi = std::min(uc + uh, 1.0);
  r.v_lo = std::max(vc + vl, 0.0);
  r.v_hi = std::min(vc + vh, 1.0);
  if (r.u_lo > r.u_hi || r.v_lo > r.v_hi) {
    r.u_lo = r.u_hi = r.v_lo = r.v_hi = 0.0;
    r.flags |= F_CULL_EMPTY;
    return;
  }
  r.flags |= F_LIVE;
  r.e_lo = 0.0;
  r.e_hi = inf;
}

// ---------------------------------------------------------------------------
// Irradiance of two-vertex chains (Eq. eq_dwda through both vertices).  The irradiance at the
// receiver is E = I0 |d0.N1| / |d0|^3 * |det du1/du_k| / |N_k| (the direct evaluator's GGT form);
// here both factors are enclosed over the whole cell by evaluating the chain map of
// eval_pair_direct (unit normals, vector Snell or mirror law at each vertex, ray/plane hits) in
// interval arithmetic with forward-mode derivatives along T1's two barycentric directions: the
// cell's barycentric bounding box is the input interval, every operation rounds outward by one ulp,
// and the hit on T2's plane is intersected with T2's closed domain (only chains through T2 count).
// The Jacobian du_k/du1 of every chain of the cell lies in the resulting interval matrix, so when its
// interval determinant excludes 0, E_hi = I0 |C1| / (s_lo^(3/2) |N_k| min |det|) bounds the
// irradiance of every chain of the record from above (and E_lo from below); otherwise, or when a
// division or square root cannot be certified, E_hi = +inf.  (The paper bounds chain irradiance by
// implicit differentiation with Bernstein forms; its details are in the unavailable supplement.)
struct Iv {
  double lo, hi;
};
double out_dn(double x) { return std::nextafter(x, -std::numeric_limits<double>::infinity()); }
double out_up(double x) { return std::nextafter(x, std::numeric_limits<double>::infinity()); }
Iv ic(double a) { return {a, a}; }
Iv iadd(Iv a, Iv b) { return {out_dn(a.lo + b.lo), out_up(a.hi + b.hi)}; }
Iv isub(Iv a, Iv b) { return {out_dn(a.lo - b.hi), out_up(a.hi - b.lo)}; }
Iv imul(Iv a, Iv b) {
  const double p0 = a.lo * b.lo, p1 = a.lo * b.hi, p2 = a.hi * b.lo, p3 = a.hi * b.hi;
  return {out_dn(std::min(std::min(p0, p1), std::min(p2, p3))), out_up(std::max(std::max(p0, p1), std::max(p2, p3)))};
}
// a / b; ok = false when b contains 0
Iv idiv(Iv a, Iv b, bool& ok) {
  if (!(b.lo > 0.0 || b.hi < 0.0)) {
    ok = false;
    return {-std::numeric_limits<double>::infinity(), std::numeric_limits<double>::infinity()};
  }
  const double q0 = a.lo / b.lo, q1 = a.lo / b.hi, q2 = a.hi / b.lo, q3 = a.hi / b.hi;
  return {out_dn(std::min(std::min(q0, q1), std::min(q2, q3))), out_up(std::max(std::max(q0, q1), std::max(q2, q3)))};
}
// sqrt of the non-negative part; ok = false when a has none
Iv isqrt(Iv a, bool& ok) {
  if (!(a.hi >= 0.0)) {
    ok = false;
    return {0.0, 0.0};
  }
  return {std::max(0.0, out_dn(std::sqrt(std::max(a.lo, 0.0)))), out_up(std::sqrt(a.hi))};
}

struct ID {  // interval value and its derivatives along T1's barycentric directions u, v
  Iv v, d[2];
};
ID idc(double a) { return {ic(a), {ic(0.0), ic(0.0)}}; }
ID operator+(ID a, ID b) { return {iadd(a.v, b.v), {iadd(a.d[0], b.d[0]), iadd(a.d[1], b.d[1])}}; }
ID operator-(ID a, ID b) { return {isub(a.v, b.v), {isub(a.d[0], b.d[0]), isub(a.d[1], b.d[1])}}; }
ID operator*(ID a, ID b) {
  return {imul(a.v, b.v),
          {iadd(imul(a.d[0], b.v), imul(a.v, b.d[0])), iadd(imul(a.d[1], b.v), imul(a.v, b.d[1]))}};
}
ID idivd(ID a, ID b, bool& ok) {
  const Iv q = idiv(a.v, b.v, ok);
  return {q, {idiv(isub(a.d[0], imul(q, b.d[0])), b.v, ok), idiv(isub(a.d[1], imul(q, b.d[1])), b.v, ok)}};
}
ID isqrtd(ID a, bool& ok) {
  const Iv r = isqrt(a.v, ok);
  const Iv r2 = imul(ic(2.0), r);
  return {r, {idiv(a.d[0], r2, ok), idiv(a.d[1], r2, ok)}};
}
struct IV3 {
  ID x, y, z;
};
IV3 operator+(IV3 a, IV3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
IV3 operator-(IV3 a, IV3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
IV3 operator*(ID s, IV3 a) { return {s * a.x, s * a.y, s * a.z}; }
ID idot(IV3 a, IV3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
IV3 iconst(V3 a) { return {idc(a.x), idc(a.y), idc(a.z)}; }
IV3 idivs(IV3 a, ID s, bool& ok) { return {idivd(a.x, s, ok), idivd(a.y, s, ok), idivd(a.z, s, ok)}; }

// Unit normal, then the mirror law or vector Snell (as snell(); eta < 0: a mirror); ok = false
// when the discriminant's range reaches 0 (total internal reflection on part of the cell).
IV3 isnell(IV3 ih, IV3 n, double eta, bool& ok) {
  const ID ln = isqrtd(idot(n, n), ok);
  const IV3 nh = idivs(n, ln, ok);
  if (eta < 0.0) return ih - (idc(2.0) * idot(ih, nh)) * nh;
  const ID c1 = idc(0.0) - idot(ih, nh);
  const ID k = idc(1.0) - idc(eta * eta) * (idc(1.0) - c1 * c1);
  if (!(k.v.lo > 0.0)) ok = false;
  return idc(eta) * ih + (idc(eta) * c1 - isqrtd(k, ok)) * nh;
}

void iplane_coords(IV3 rel, V3 a, V3 b, ID* U, ID* V, bool& ok) {  // as plane_coords
  const double g11 = dot(a, a), g12 = dot(a, b), g22 = dot(b, b);
  const double det = g11 * g22 - g12 * g12;
  const ID pa = idot(rel, iconst(a)), pb = idot(rel, iconst(b));
  *U = idivd(idc(g22) * pa - idc(g12) * pb, idc(det), ok);
  *V = idivd(idc(g11) * pb - idc(g12) * pa, idc(det), ok);
}

// [E_lo, E_hi] of every chain of (emitter e, T1, T2) whose u1 lies in the box U x W of T1's
// barycentric coordinates.  Returns 0 (bounds certified), 1 (no chain of the box meets T2's closed
// domain: [0, 0]) or 2 (not certified: a division, square root or the Jacobian's sign undecided).
int chain_box(const Ctx2& cx, const Tri& A, const Tri& B, V3 x0, double I0, Iv Ub, Iv Wb, double* elo, double* ehi,
              double* diag = nullptr) {
  const Rec& R = cx.rec;
  bool ok = true;
  const ID U = {Ub, {ic(1.0), ic(0.0)}};
  const ID W = {Wb, {ic(0.0), ic(1.0)}};
  const IV3 x1 = iconst(A.p[0]) + U * iconst(A.p[1] - A.p[0]) + W * iconst(A.p[2] - A.p[0]);
  const IV3 n1 = iconst(A.n[0]) + U * iconst(A.n[1] - A.n[0]) + W * iconst(A.n[2] - A.n[0]);
  const IV3 d0 = x1 - iconst(x0);
  const ID s0 = idot(d0, d0);
  const IV3 i1 = idivs(d0, isqrtd(s0, ok), ok);
  const IV3 r1 = isnell(i1, n1, law(cx.s1), ok);
  const V3 e21 = B.p[1] - B.p[0], e22 = B.p[2] - B.p[0], N2 = cross(e21, e22);
  const ID t = idivd(idot(iconst(B.p[0]) - x1, iconst(N2)), idot(r1, iconst(N2)), ok);
  const IV3 x2 = x1 + t * r1;
  ID U2, V2;
  iplane_coords(x2 - iconst(B.p[0]), e21, e22, &U2, &V2, ok);
  if (!ok) return 2;
  // only chains through the closed triangle T2 count: clip the values to its barycentric box
  U2.v = {std::max(U2.v.lo, 0.0), std::min(U2.v.hi, 1.0)};
  V2.v = {std::max(V2.v.lo, 0.0), std::min(V2.v.hi, 1.0)};
  if (U2.v.lo > U2.v.hi || V2.v.lo > V2.v.hi || U2.v.lo + V2.v.lo > 1.0) return 1;
  const IV3 n2 = iconst(B.n[0]) + U2 * iconst(B.n[1] - B.n[0]) + V2 * iconst(B.n[2] - B.n[0]);
  const IV3 i2 = idivs(r1, isqrtd(idot(r1, r1), ok), ok);
  const IV3 r2 = isnell(i2, n2, law(cx.s2), ok);
  const V3 Nk = cross(R.e1, R.e2);
  const ID t2h = idivd(idot(iconst(R.p0) - x2, iconst(Nk)), idot(r2, iconst(Nk)), ok);
  const IV3 X = x2 + t2h * r2;
  ID Uk, Vk;
  iplane_coords(X - iconst(R.p0), R.e1, R.e2, &Uk, &Vk, ok);
  if (!ok) return 2;
  const Iv det = isub(imul(Uk.d[0], Vk.d[1]), imul(Uk.d[1], Vk.d[0]));
  if (diag) {  // s = |d0|^2 and det du_k/du1 over the box
    diag[0] = s0.v.lo;
    diag[1] = s0.v.hi;
    diag[2] = det.lo;
    diag[3] = det.hi;
  }
  if (!(det.lo > 0.0 || det.hi < 0.0)) return 2;  // a fold may lie in the box
  const double dmin = det.lo > 0.0 ? det.lo : -det.hi, dmax = det.lo > 0.0 ? det.hi : -det.lo;
  const Iv s = s0.v;
  if (!(s.lo > 0.0)) return 2;
  // |C1| = |(p10 - x0).N1| (constant on T1) with its float64 rounding error, |N_k|
  const V3 a1 = A.p[1] - A.p[0], b1 = A.p[2] - A.p[0], r0 = A.p[0] - x0;
  const V3 N1 = cross(a1, b1);
  const double c1 = std::fabs(dot(r0, N1)), nk = norm(Nk);
  const double mag = std::fabs(r0.x) * (std::fabs(a1.y * b1.z) + std::fabs(a1.z * b1.y)) +
                     std::fabs(r0.y) * (std::fabs(a1.z * b1.x) + std::fabs(a1.x * b1.z)) +
                     std::fabs(r0.z) * (std::fabs(a1.x * b1.y) + std::fabs(a1.y * b1.x));
  const double cerr = 2e-15 * mag;
  const double num_hi = out_up(I0 * out_up(c1 + cerr));
  const double num_lo = std::max(0.0, out_dn(I0 * out_dn(c1 - cerr)));
  const double s32_lo = out_dn(s.lo * out_dn(std::sqrt(s.lo))), s32_hi = out_up(s.hi * out_up(std::sqrt(s.hi)));
  *ehi = out_up(num_hi / out_dn(out_dn(s32_lo * out_dn(nk * (1.0 - 1e-15))) * dmin));
  *elo = std::max(0.0, out_dn(num_lo / out_up(out_up(s32_hi * out_up(nk * (1.0 + 1e-15))) * dmax)));
  return 0;
}

// Whether the box [u0, u1] x [v0, v1] meets the triangle with corners C (separating axes: the
// coordinate axes and the triangle's edge normals); a box separated by at most 1e-6 counts as
// meeting it, so boxes that touch the cell are always kept.
bool box_meets_cell(const UV C[3], double u0, double u1, double v0, double v1) {
  const double mu = std::min(std::min(C[0].u, C[1].u), C[2].u), Mu = std::max(std::max(C[0].u, C[1].u), C[2].u);
  const double mv = std::min(std::min(C[0].v, C[1].v), C[2].v), Mv = std::max(std::max(C[0].v, C[1].v), C[2].v);
  const double eps = 1e-6;
  if (u0 > Mu + eps || u1 < mu - eps || v0 > Mv + eps || v1 < mv - eps) return false;
  for (int k = 0; k < 3; ++k) {
    const UV a = C[k], b = C[(k + 1) % 3], c = C[(k + 2) % 3];
    const double nu = -(b.v - a.v), nv = b.u - a.u;  // normal of edge a-b
    const double side = nu * (c.u - a.u) + nv * (c.v - a.v);  // the triangle's side
    const double len = std::sqrt(nu * nu + nv * nv);
    double mn = std::numeric_limits<double>::infinity(), mx = -mn;
    for (int q = 0; q < 4; ++q) {
      const double pu = (q & 1) ? u1 : u0, pv = (q & 2) ? v1 : v0;
      const double d = nu * (pu - a.u) + nv * (pv - a.v);
      mn = std::min(mn, d);
      mx = std::max(mx, d);
    }
    if (side > 0.0 && mx < -eps * len) return false;
    if (side < 0.0 && mn > eps * len) return false;
  }
  return true;
}

// [E_lo, E_hi] of every chain of (emitter e, cell of T1, T2); E_hi = +inf when not certified,
// [0, 0] when no chain of the cell passes through T2's closed domain.  The cell's barycentric
// bounding box is tried whole; when that is not certified, its 2 x 2 and then 4 x 4 sub-boxes that
// meet the cell (interval widths shrink with the box): the bound is the hull over the sub-boxes
// of the first level at which every kept sub-box is certified or meets no chain.
void chain_irradiance(const Ctx2& cx, int e, int t1, uint32_t id, int depth, int t2, double* elo, double* ehi) {
  const double inf = std::numeric_limits<double>::infinity();
  UV C[3];
  cell_corners(id, depth, C);
  const Tri A = get_tri(cx.s1, t1), B = get_tri(cx.s2, t2);
  const V3 x0 = {cx.em->x[e], cx.em->y[e], cx.em->z[e]};
  const double I0 = cx.em->intensity[e];
  const double u0 = std::min(std::min(C[0].u, C[1].u), C[2].u), u1 = std::max(std::max(C[0].u, C[1].u), C[2].u);
  const double v0 = std::min(std::min(C[0].v, C[1].v), C[2].v), v1 = std::max(std::max(C[0].v, C[1].v), C[2].v);
  for (int level = 0; level < 3; ++level) {
    const int m = 1 << level;
    double lo = inf, hi = 0.0;
    bool certified = true;
    for (int j = 0; j < m && certified; ++j) {
      for (int i = 0; i < m && certified; ++i) {
        const double a0 = u0 + (u1 - u0) * i / m, a1 = u0 + (u1 - u0) * (i + 1) / m;
        const double b0 = v0 + (v1 - v0) * j / m, b1 = v0 + (v1 - v0) * (j + 1) / m;
        if (level > 0 && !box_meets_cell(C, a0, a1, b0, b1)) continue;
        double l = 0.0, h = 0.0;
        const int rc = chain_box(cx, A, B, x0, I0, Iv{a0, a1}, Iv{b0, b1}, &l, &h);
        if (rc == 2) certified = false;
        if (rc == 0) {
          lo = std::min(lo, l);
          hi = std::max(hi, h);
        }
      }
    }
    if (certified) {
      *elo = lo == inf ? 0.0 : lo;
      *ehi = hi;
      return;
    }
  }
  *elo = 0.0;
  *ehi = inf;
}

}  // namespace

// ===========================================================================
// C ABI (loaded by the tests through ctypes)
// ===========================================================================
extern "C" {

// Bernstein helpers exposed for the pins.  dim in {1,2}; coefficient order as above.
int orc_bb_size(int dim, int n) { return psize(dim, n); }
void orc_bb_mul(int dim, int m, const double* p, int n, const double* q, double* out) {
  Poly P{dim, m, std::vector<double>(p, p + psize(dim, m))};
  Poly Qp{dim, n, std::vector<double>(q, q + psize(dim, n))};
  Poly R = pmul(P, Qp);
  std::copy(R.c.begin(), R.c.end(), out);
}
void orc_bb_elevate(int dim, int n, const double* p, double* out) {
  Poly P{dim, n, std::vector<double>(p, p + psize(dim, n))};
  Poly R = pelevate(P);
  std::copy(R.c.begin(), R.c.end(), out);
}
void orc_bb_deriv(int n, const double* p, int j, double* out) {
  Poly P{2, n, std::vector<double>(p, p + psize(2, n))};
  Poly R = pderiv(P, j);
  std::copy(R.c.begin(), R.c.end(), out);
}
double orc_bb_eval(int dim, int n, const double* p, double m1, double m2) {
  Poly P{dim, n, std::vector<double>(p, p + psize(dim, n))};
  return peval(P, m1, m2);
}
void orc_chord_sqrt(double lo, double hi, double* out4) { chord_sqrt(lo, hi, &out4[0], &out4[1], &out4[2], &out4[3]); }
void orc_chord_inv32(double s_lo, double s_hi, double* out4) {
  chord_inv32(s_lo, s_hi, &out4[0], &out4[1], &out4[2], &out4[3]);
}
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }
float orc_philox_uniform(uint64_t seed, int64_t point, uint64_t key) { return philox_uniform(seed, point, key); }
void orc_cell_corners(uint32_t id, int depth, double* out6) {
  UV C[3];
  cell_corners(id, depth, C);
  for (int k = 0; k < 3; ++k) {
    out6[2 * k] = C[k].u;
    out6[2 * k + 1] = C[k].v;
  }
}

// Bound the given base cells (flat work indices, or all when work == NULL).
// Records of cells that split follow their parent (flag SPLIT) in depth-first
// order.  Returns 0, or -2 when cap is too small (n_out then holds the need).
int orc_bound(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int32_t depth,
              int32_t max_extra_split, int32_t irradiance, const int64_t* work, int64_t n_work,
              orc_record* out, int64_t cap, int64_t* n_out, int32_t n_threads, int32_t adapt_depth, float sigma,
              float alpha) {
  if (s1->kind != 0 && s1->kind != 1) return -4;
  // sign-test splits may go max_extra_split levels below the deepest adaptive level
  Ctx cx{s1, get_rec(rec), em, irradiance, std::max(depth, adapt_depth) + max_extra_split, adapt_depth, sigma, alpha};
  int64_t total = work ? n_work : (int64_t)em->n * s1->n_tris * ((int64_t)1 << (2 * depth));
  int nt = std::max(1, (int)n_threads);
  std::vector<std::vector<orc_record>> parts(nt);
  parallel_for(total, nt, [&](int k, int64_t a, int64_t b) {
    auto& v = parts[k];
    for (int64_t i = a; i < b; ++i) {
      int e, t;
      uint32_t c;
      decode_work(work ? work[i] : i, s1->n_tris, depth, &e, &t, &c);
      if (s1->kind == 0)
        bound_cell_reflect(cx, e, t, c, depth, v);
      else
        bound_cell_refract(cx, e, t, c, depth, v);
    }
  });
  int64_t n = 0;
  for (auto& v : parts) n += (int64_t)v.size();
  *n_out = n;
  if (n > cap) return -2;
  int64_t o = 0;
  for (auto& v : parts)
    for (auto& r : v) out[o++] = r;
  return 0;
}

// Index (Sec. 6.1 "Bound storage"): for each LIVE record, the closed range of
// grid cells its box overlaps, i = floor(u*G) clamped to [0, G-1] (float32
// product, as the CUDA path takes this decision).  Per (grid cell, tuple key)
// the tuple bound is m * max over covering records (Eq. eq_pertuple_b), kept in
// float32 (round-up product).  Keys: emitter<<48 | (tri1+1)<<24 | tri0.
int orc_index(const float* u_lo, const float* u_hi, const float* v_lo, const float* v_hi, const float* e_hi,
              const int32_t* emitter, const int32_t* tri0, const int32_t* tri1, const uint32_t* flags, int64_t n,
              int32_t G, float m, int64_t* offsets, uint64_t* key, float* etilde, int64_t cap, int64_t* n_out) {
  std::vector<std::map<uint64_t, float>> cells((size_t)G * G);
  for (int64_t r = 0; r < n; ++r) {
    if (!(flags[r] & F_LIVE)) continue;
    auto gi = [&](float x) {
      float p = x * (float)G;  // float32 product
      int i = (int)std::floor(p);
      return std::min(G - 1, std::max(0, i));
    };
    int i0 = gi(u_lo[r]), i1 = gi(u_hi[r]), j0 = gi(v_lo[r]), j1 = gi(v_hi[r]);
    uint64_t k = ((uint64_t)(uint32_t)emitter[r] << 48) | ((uint64_t)(uint32_t)(tri1[r] + 1) << 24) |
                 (uint64_t)(uint32_t)tri0[r];
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        auto& mp = cells[(size_t)j * G + i];
        auto it = mp.find(k);
        if (it == mp.end())
          mp[k] = e_hi[r];
        else
          it->second = std::max(it->second, e_hi[r]);
      }
  }
  int64_t tot = 0;
  offsets[0] = 0;
  for (size_t g = 0; g < cells.size(); ++g) {
    tot += (int64_t)cells[g].size();
    offsets[g + 1] = tot;
  }
  *n_out = tot;
  if (tot > cap) return -2;
  int64_t o = 0;
  for (auto& mp : cells)
    for (auto& kv : mp) {
      key[o] = kv.first;
      etilde[o] = fmul_ru32(m, kv.second);
      ++o;
    }
  return 0;
}

// Algorithm 1 (Sec. 5.3) with P = min(gamma E~, 1) (Sec. 5.4): one uniform per
// (point, tuple) from Philox4x32-10 keyed by the seed, counter (point, key);
// select when r < P.  The probability is the float32 product rounded up, so
// P > 0 whenever E~ > 0 (unbiasedness condition of Sec. 5.3).
int orc_sample(const int64_t* offsets, const uint64_t* key, const float* etilde, int32_t G, const float* su,
               const float* sv, int64_t n_points, float gamma, uint64_t seed, int64_t* wl_point, uint64_t* wl_key,
               float* wl_p, int64_t cap, int64_t* n_out, int64_t* n_U, int32_t bins, int64_t* n_B) {
  int64_t o = 0, nu = 0, nb = 0;
  for (int64_t p = 0; p < n_points; ++p) {
    auto gi = [&](float x) {
      int i = (int)std::floor(x * (float)G);
      return std::min(G - 1, std::max(0, i));
    };
    int64_t g = (int64_t)gi(sv[p]) * G + gi(su[p]);
    // bins (Sec. 5.3): the listed tuples packed greedily in list order into groups whose
    // probabilities sum to at most 1 (a tuple that does not fit closes the group and opens the
    // next); one draw per group (counter = (point, key of its first tuple)) picks the tuple whose
    // cumulative interval [c_prev, c) holds it, or none past the group's total.  Float32 sums.
    float acc = 0.0f, rb = 0.0f;
    bool open = false;
    for (int64_t j = offsets[g]; j < offsets[g + 1]; ++j) {
      ++nu;
      float P = std::fmin(fmul_ru32(gamma, etilde[j]), 1.0f);  // fmin: a NaN product (0 * inf) selects
      bool sel;
      if (bins) {
        if (!open || acc + P > 1.0f) {
          open = true;
          acc = 0.0f;
          rb = philox_uniform(seed, p, key[j]);
          ++nb;
        }
        const float lo = acc;
        acc = acc + P;
        sel = rb >= lo && rb < acc;
      } else {
        sel = philox_uniform(seed, p, key[j]) < P;
      }
      if (sel) {
        if (o < cap) {
          wl_point[o] = p;
          wl_key[o] = key[j];
          wl_p[o] = P;
        }
        ++o;
      }
    }
  }
  *n_out = o;
  *n_U = nu;
  if (n_B) *n_B = nb;
  return o > cap ? -2 : 0;
}

}  // extern "C"

namespace {

// Newton's method for one tuple from the start (u, v): newton_iters damped steps (step clamped to
// 0.5 in barycentric units; once a step is below 1e-6 the damped phase ends), then polish_iters
// full steps; the root is accepted when the hit is within tol scene units of the target, u1 lies in
// the closed triangle and the hit is in front (t > 0).  Returns E(root) >= 0, or -1.
double newton_from(const Tri& T, V3 x0, double I0, const Rec& R, int kind, double eta, double tu, double tv,
                   int newton_iters, int polish_iters, double tol, double* u_io, double* v_io) {
  double u = *u_io, v = *v_io;
  for (int it = 0; it < newton_iters + polish_iters; ++it) {
    PathEval P = eval_path(T, x0, I0, R, u, v, kind, eta);
    double det = P.J[0][0] * P.J[1][1] - P.J[0][1] * P.J[1][0];
    if (!P.ok || !(det != 0.0) || !std::isfinite(det)) return -1.0;
    double fu = P.uk - tu, fv = P.vk - tv;
    double du = -(P.J[1][1] * fu - P.J[0][1] * fv) / det;
    double dv = -(-P.J[1][0] * fu + P.J[0][0] * fv) / det;
    double mx = std::max(std::fabs(du), std::fabs(dv));
    bool damped = it < newton_iters;
    if (damped && mx > 0.5) {
      du *= 0.5 / mx;
      dv *= 0.5 / mx;
    }
    u += du;
    v += dv;
    if (!std::isfinite(u) || !std::isfinite(v)) return -1.0;
    if (damped && mx < 1e-6) it = newton_iters - 1;  // converged: go to the polish steps
  }
  *u_io = u;
  *v_io = v;
  PathEval P = eval_path(T, x0, I0, R, u, v, kind, eta);
  if (!P.ok) return -1.0;
  V3 res = (P.uk - tu) * R.e1 + (P.vk - tv) * R.e2;
  bool inside = u >= 0.0 && v >= 0.0 && u + v <= 1.0;
  if (norm(res) < tol && inside && P.t > 0.0 && std::isfinite(P.E)) return P.E;
  return -1.0;
}

// Start of stochastic trial t (t >= 0) for (point, tuple key): the first two outputs of
// Philox4x32-10 with counter (point, key) and key seed + (t + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
// as 24-bit uniforms (a, b), folded into the triangle (a + b > 1 -> (1 - a, 1 - b)).
void stoc_start(uint64_t seed, int64_t point, uint64_t key, int t, double* u, double* v) {
  const uint64_t k = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
  const uint32_t ctr[4] = {(uint32_t)point, (uint32_t)((uint64_t)point >> 32), (uint32_t)key, (uint32_t)(key >> 32)};
  const uint32_t kk[2] = {(uint32_t)k, (uint32_t)(k >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, kk, o);
  double a = (double)(o[0] >> 8) * (1.0 / 16777216.0), b = (double)(o[1] >> 8) * (1.0 / 16777216.0);
  if (a + b > 1.0) {
    a = 1.0 - a;
    b = 1.0 - b;
  }
  *u = a;
  *v = b;
}

}  // namespace

extern "C" {

// Newton root-finding in the tuple's triangle (Sec. 6.1).  stoc_trials = 0: deterministic start at
// the centroid (Det).  stoc_trials > 0: stochastic start with the unbiased reciprocal weighting
// (Stoc, Sec. 6.1 after Zeltner et al. 2020): a root u* found from a uniform random start is
// weighted by the number N of further random starts up to the first that reaches u* again (within
// 1e-4 in barycentrics), E[N] = 1 / P(reach u*), capped at stoc_trials (N = stoc_trials when no
// start in the cap reaches it).  contrib = E(root) N / P; status 1 root, 0 none; trials[i] = N.
int orc_solve(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, const int64_t* wl_point,
              const uint64_t* wl_key, const float* wl_p, int64_t n_wl, const float* su, const float* sv,
              int32_t newton_iters, int32_t polish_iters, double tol, double* contrib, double* root_u,
              double* root_v, int32_t* status, int32_t n_threads, int32_t stoc_trials, uint64_t seed,
              int32_t* trials) {
  Rec R = get_rec(rec);
  parallel_for(n_wl, std::max(1, (int)n_threads), [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      uint64_t k = wl_key[i];
      int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFu);
      Tri T = get_tri(s1, t);
      V3 x0 = {em->x[e], em->y[e], em->z[e]};
      double I0 = em->intensity[e];
      const int64_t pt = wl_point[i];
      double tu = su[pt], tv = sv[pt];
      double u = 1.0 / 3.0, v = 1.0 / 3.0;
      if (stoc_trials > 0) stoc_start(seed, pt, k, 0, &u, &v);
      const double E = newton_from(T, x0, I0, R, s1->kind, s1->eta, tu, tv, newton_iters, polish_iters, tol, &u, &v);
      contrib[i] = 0.0;
      status[i] = 0;
      root_u[i] = u;
      root_v[i] = v;
      if (trials) trials[i] = 0;
      if (!(E >= 0.0)) continue;
      int n = 1;
      if (stoc_trials > 0) {
        for (n = 1; n < stoc_trials; ++n) {
          double u2, v2;
          stoc_start(seed, pt, k, n, &u2, &v2);
          const double E2 =
              newton_from(T, x0, I0, R, s1->kind, s1->eta, tu, tv, newton_iters, polish_iters, tol, &u2, &v2);
          if (E2 >= 0.0 && std::fabs(u2 - u) <= 1e-4 && std::fabs(v2 - v) <= 1e-4) break;
        }
      }
      status[i] = 1;
      contrib[i] = E * n / (double)wl_p[i];
      if (trials) trials[i] = n;
    }
  });
  return 0;
}

// Every root of tuple (e, t) at target (tu, tv): Newton from an n x n grid of starts over the
// triangle (Det steps), distinct accepted roots (1e-7 apart) summed.  For the pins.
int orc_roots(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int32_t e, int32_t t,
              double tu, double tv, int32_t n, int32_t newton_iters, int32_t polish_iters, double tol,
              double* sum_E, int32_t* n_roots) {
  const Rec R = get_rec(rec);
  const Tri T = get_tri(s1, t);
  const V3 x0 = {em->x[e], em->y[e], em->z[e]};
  std::vector<std::array<double, 3>> found;
  for (int i = 0; i <= n; ++i)
    for (int j = 0; i + j <= n; ++j) {
      double u = (i + 1.0 / 3.0) / (n + 1.0), v = (j + 1.0 / 3.0) / (n + 1.0);
      const double E = newton_from(T, x0, em->intensity[e], R, s1->kind, s1->eta, tu, tv, newton_iters,
                                   polish_iters, tol, &u, &v);
      if (!(E >= 0.0)) continue;
      bool dup = false;
      for (auto& f : found) dup = dup || (std::fabs(f[0] - u) < 1e-7 && std::fabs(f[1] - v) < 1e-7);
      if (!dup) found.push_back({u, v, E});
    }
  double s = 0.0;
  for (auto& f : found) s += f[2];
  *sum_E = s;
  *n_roots = (int32_t)found.size();
  return 0;
}

// Rational-form path evaluation at given (u1, v1) of one tuple (for pins).
int orc_eval_path(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int32_t e, int32_t t,
                  const double* u, const double* v, int64_t n, double* uk, double* vk, double* E, double* tt) {
  Rec R = get_rec(rec);
  Tri T = get_tri(s1, t);
  V3 x0 = {em->x[e], em->y[e], em->z[e]};
  for (int64_t i = 0; i < n; ++i) {
    PathEval P = eval_path(T, x0, em->intensity[e], R, u[i], v[i], s1->kind, s1->eta);
    const double nan = std::numeric_limits<double>::quiet_NaN();
    uk[i] = P.ok ? P.uk : nan;
    vk[i] = P.ok ? P.vk : nan;
    E[i] = P.ok ? P.E : nan;
    tt[i] = P.ok ? P.t : nan;
  }
  return 0;
}

// Direct-geometry evaluation (normalized normals, vector reflection, duals).
int orc_eval_direct(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int32_t e, int32_t t,
                    const double* u, const double* v, int64_t n, double* uk, double* vk, double* E, double* tt) {
  Rec R = get_rec(rec);
  Tri T = get_tri(s1, t);
  V3 x0 = {em->x[e], em->y[e], em->z[e]};
  for (int64_t i = 0; i < n; ++i) {
    bool ok;
    if (s1->kind == 0)
      ok = eval_direct_reflect(T, x0, em->intensity[e], R, u[i], v[i], &uk[i], &vk[i], &E[i], &tt[i]);
    else
      ok = eval_direct_refract(T, x0, em->intensity[e], R, s1->eta, u[i], v[i], &uk[i], &vk[i], &E[i], &tt[i]);
    if (!ok) uk[i] = vk[i] = E[i] = tt[i] = std::numeric_limits<double>::quiet_NaN();
  }
  return 0;
}

// Candidate pairs (Sec. 6.1 "Tuple construction") by brute force over every triangle of s2:
// items (emitter, tri0, cell, tri1) in that lexicographic order, for both surfaces refractive.
int orc_pair_candidates(const orc_surface* s1, const orc_surface* s2, const orc_emitters* em, int32_t depth,
                        int32_t* out_e, int32_t* out_t1, uint32_t* out_cell, int32_t* out_t2, int64_t cap,
                        int64_t* n_out, int32_t n_threads) {
  if (s1->kind < 0 || s1->kind > 1 || s2->kind < 0 || s2->kind > 1) return -4;
  std::vector<Box3> boxes(s2->n_tris);
  for (int t = 0; t < s2->n_tris; ++t) boxes[t] = tri_box(get_tri(s2, t));
  const int64_t total = (int64_t)em->n * s1->n_tris * ((int64_t)1 << (2 * depth));
  const int nt = std::max(1, (int)n_threads);
  std::vector<std::vector<std::array<int64_t, 4>>> parts(nt);
  parallel_for(total, nt, [&](int k, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      int e, t;
      uint32_t c;
      decode_work(i, s1->n_tris, depth, &e, &t, &c);
      UV C[3];
      cell_corners(c, depth, C);
      const V3 x0 = {em->x[e], em->y[e], em->z[e]};
      const Bundle B = ray_bundle(first_vertex(get_tri(s1, t), x0, s1->kind, s1->eta, C));
      if (B.kind == 0) continue;
      for (int t2 = 0; t2 < s2->n_tris; ++t2) {
        double gap;
        if (pair_candidate(B, boxes[t2], &gap)) parts[k].push_back({e, t, (int64_t)c, t2});
      }
    }
  });
  int64_t n = 0;
  for (auto& v : parts) n += (int64_t)v.size();
  *n_out = n;
  if (n > cap) return -2;
  int64_t o = 0;
  for (auto& v : parts)
    for (auto& q : v) {
      out_e[o] = (int32_t)q[0];
      out_t1[o] = (int32_t)q[1];
      out_cell[o] = (uint32_t)q[2];
      out_t2[o] = (int32_t)q[3];
      ++o;
    }
  return 0;
}

// Footprint gap of each queried (emitter, tri0, cell, tri1) (see pair_candidate).
int orc_pair_gap(const orc_surface* s1, const orc_surface* s2, const orc_emitters* em, int32_t depth,
                 const int32_t* e, const int32_t* t1, const uint32_t* cell, const int32_t* t2, int64_t n,
                 double* gap) {
  for (int64_t i = 0; i < n; ++i) {
    UV C[3];
    cell_corners(cell[i], depth, C);
    const V3 x0 = {em->x[e[i]], em->y[e[i]], em->z[e[i]]};
    pair_candidate(ray_bundle(first_vertex(get_tri(s1, t1[i]), x0, s1->kind, s1->eta, C)), tri_box(get_tri(s2, t2[i])),
                   &gap[i]);
  }
  return 0;
}

// Records of the given pair items (composite position bound; e_hi = +inf).
int orc_bound_pairs(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec, const orc_emitters* em,
                    int32_t depth, const int32_t* e, const int32_t* t1, const uint32_t* cell, const int32_t* t2,
                    int64_t n, orc_record* out, int32_t n_threads) {
  if (s1->kind < 0 || s1->kind > 1 || s2->kind < 0 || s2->kind > 1) return -4;
  Ctx2 cx{s1, s2, get_rec(rec), em};
  parallel_for(n, std::max(1, (int)n_threads), [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) bound_cell_pair(cx, e[i], t1[i], cell[i], depth, t2[i], out[i]);
  });
  return 0;
}

// Records of the given pair items with their intermediate quantities (one PairDiag each).
int orc_bound_pairs_diag(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec,
                         const orc_emitters* em, int32_t depth, const int32_t* e, const int32_t* t1,
                         const uint32_t* cell, const int32_t* t2, int64_t n, orc_record* out, PairDiag* diag) {
  if (s1->kind < 0 || s1->kind > 1 || s2->kind < 0 || s2->kind > 1) return -4;
  Ctx2 cx{s1, s2, get_rec(rec), em};
  for (int64_t i = 0; i < n; ++i) bound_cell_pair(cx, e[i], t1[i], cell[i], depth, t2[i], out[i], &diag[i]);
  return 0;
}
int orc_pair_diag_size(void) { return (int)sizeof(PairDiag); }

// Irradiance bounds [e_lo, e_hi] of the given pair items (chain_irradiance; +inf when not certified).
int orc_chain_irradiance(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec,
                         const orc_emitters* em, int32_t depth, const int32_t* e, const int32_t* t1,
                         const uint32_t* cell, const int32_t* t2, int64_t n, double* e_lo, double* e_hi,
                         int32_t n_threads) {
  if (s1->kind < 0 || s1->kind > 1 || s2->kind < 0 || s2->kind > 1) return -4;
  Ctx2 cx{s1, s2, get_rec(rec), em};
  parallel_for(n, std::max(1, (int)n_threads), [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) chain_irradiance(cx, e[i], t1[i], cell[i], depth, t2[i], &e_lo[i], &e_hi[i]);
  });
  return 0;
}

// One box of the chain bound with its factors: out = {rc, s_lo, s_hi, det_lo, det_hi, e_lo, e_hi} for the
// box [u0, u1] x [v0, v1] of T1's barycentric coordinates (rc: 0 certified, 1 no chain, 2 not certified).
int orc_chain_box(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec, const orc_emitters* em,
                  int32_t e, int32_t t1, int32_t t2, double u0, double u1, double v0, double v1, double* out) {
  Ctx2 cx{s1, s2, get_rec(rec), em};
  const Tri A = get_tri(s1, t1), B = get_tri(s2, t2);
  const V3 x0 = {em->x[e], em->y[e], em->z[e]};
  double d[4] = {0, 0, 0, 0}, l = 0.0, h = 0.0;
  const int rc = chain_box(cx, A, B, x0, em->intensity[e], Iv{u0, u1}, Iv{v0, v1}, &l, &h, d);
  const double vals[7] = {(double)rc, d[0], d[1], d[2], d[3], l, h};
  for (int k = 0; k < 7; ++k) out[k] = vals[k];
  return 0;
}

// Direct chain evaluation at (u1, v1): out[i*8 + 0..7] = uk, vk, E, u2, v2, t1, t2, detJ (NaN: no path).
int orc_eval_pair(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec, const orc_emitters* em,
                  int32_t e, int32_t t1, int32_t t2, const double* u, const double* v, int64_t n, double* out) {
  const Rec R = get_rec(rec);
  const Tri A = get_tri(s1, t1), B = get_tri(s2, t2);
  const V3 x0 = {em->x[e], em->y[e], em->z[e]};
  for (int64_t i = 0; i < n; ++i) {
    PairEval P = eval_pair_direct(A, B, x0, em->intensity[e], R, law(s1), law(s2), u[i], v[i]);
    const double nan = std::numeric_limits<double>::quiet_NaN();
    const double vals[8] = {P.uk, P.vk, P.E, P.u2, P.v2, P.t1, P.t2, P.detJ};
    for (int k = 0; k < 8; ++k) out[i * 8 + k] = P.ok ? vals[k] : nan;
  }
  return 0;
}

// Newton root-finding for pair tuples (Sec. 6.1 "Root-finding", deterministic init) with the same
// schedule as orc_solve; a root is accepted when the hit is within tol scene units of the target,
// u1 lies in the closed T1, u2 in the closed T2, and both ray parameters are positive.
int orc_solve_pair(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec, const orc_emitters* em,
                   const int64_t* wl_point, const uint64_t* wl_key, const float* wl_p, int64_t n_wl, const float* su,
                   const float* sv, int32_t newton_iters, int32_t polish_iters, double tol, double* contrib,
                   double* root_u, double* root_v, int32_t* status, int32_t n_threads) {
  const Rec R = get_rec(rec);
  parallel_for(n_wl, std::max(1, (int)n_threads), [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      const uint64_t k = wl_key[i];
      const int e = (int)(k >> 48), t1 = (int)(k & 0xFFFFFFu), t2 = (int)((k >> 24) & 0xFFFFFFu) - 1;
      contrib[i] = 0.0;
      status[i] = 0;
      root_u[i] = root_v[i] = 0.0;
      if (t2 < 0 || t2 >= s2->n_tris || t1 >= s1->n_tris) continue;
      const Tri A = get_tri(s1, t1), B = get_tri(s2, t2);
      const V3 x0 = {em->x[e], em->y[e], em->z[e]};
      const double I0 = em->intensity[e];
      const double tu = su[wl_point[i]], tv = sv[wl_point[i]];
      double u = 1.0 / 3.0, v = 1.0 / 3.0;
      bool bad = false;
      for (int it = 0; it < newton_iters + polish_iters; ++it) {
        PairEval P = eval_pair_direct(A, B, x0, I0, R, law(s1), law(s2), u, v);
        const double det = P.detJ;
        if (!P.ok || !(det != 0.0) || !std::isfinite(det)) {
          bad = true;
          break;
        }
        const double fu = P.uk - tu, fv = P.vk - tv;
        double du = -(P.J[1][1] * fu - P.J[0][1] * fv) / det;
        double dv = -(-P.J[1][0] * fu + P.J[0][0] * fv) / det;
        const double mx = std::max(std::fabs(du), std::fabs(dv));
        const bool damped = it < newton_iters;
        if (damped && mx > 0.5) {
          du *= 0.5 / mx;
          dv *= 0.5 / mx;
        }
        u += du;
        v += dv;
        if (!std::isfinite(u) || !std::isfinite(v)) {
          bad = true;
          break;
        }
        if (damped && mx < 1e-6) it = newton_iters - 1;
      }
      root_u[i] = u;
      root_v[i] = v;
      if (bad) continue;
      PairEval P = eval_pair_direct(A, B, x0, I0, R, law(s1), law(s2), u, v);
      if (!P.ok) continue;
      const V3 res = (P.uk - tu) * R.e1 + (P.vk - tv) * R.e2;
      const bool in1 = u >= 0.0 && v >= 0.0 && u + v <= 1.0;
      const bool in2 = P.u2 >= 0.0 && P.v2 >= 0.0 && P.u2 + P.v2 <= 1.0;
      if (norm(res) < tol && in1 && in2 && P.t1 > 0.0 && P.t2 > 0.0 && std::isfinite(P.E)) {
        status[i] = 1;
        contrib[i] = P.E / (double)wl_p[i];
      }
    }
  });
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Implicit differentiation for a single refraction (Sec. 4.4 "Implicit
// differentiation"; the specular polynomials F, G of its footnote).
//
//   * Variables: u1 in the cell (the cell's barycentric coordinates, a 2-simplex) and the
//     receiver coordinates u_k in the record's position box [u_lo, u_hi] x [v_lo, v_hi]
//     (box coordinates s, t in [0, 1]), treated as independent: the 4D superset of the
//     2D manifold of refracted paths.  Polynomials are classical Bernstein forms on
//     simplex x interval x interval ("tensor" forms below), degree (n; p, q).
//   * With d0 = x1 - x0, d1 = x_k - x1, n1 the interpolated normal and b a fixed vector,
//     A = (d0 x n1).b and C = (d1 x n1).b, the constraints are
//       F = eta'^2 |d1|^2 A^2 - |d0|^2 C^2   (Snell's law squared along b; the paper's
//           eta is the transmitted-over-incident ratio 1/eta', and F is scaled by the
//           constant eta'^2, which cancels in the Jacobian),
//       G = (d0 x n1).d1                      (coplanarity).
//   * Partial derivatives by the product rule with the constant derivative vectors:
//     d x1/du1 = p1 - p0, d n1/du1 = n1 - n0 (and v1 likewise), d x_k/du_k = e1 of the
//     receiver (v_k: e2).
//   * The implicit-function theorem gives |d u1 / d u_k| = |det B| / |det A| with
//     A = d(F, G)/d(u1, v1) (degree (7; 3, 3)) and B = d(F, G)/d(u_k, v_k) (degree (7; 1, 1),
//     elevated to (7; 3, 3)); with Eq. eq_dwda the irradiance is
//       E = I0 |C1| |det B| / (|d0|^3 |N_k| |det A|),  C1 = (p0 - x0).N1.
//   * Bound (Eq. eq_bbound): when every coefficient of det A is non-zero with one sign,
//     |det B / det A| lies in [min, max] of the coefficient ratios (0 below when they
//     change sign); |d0|^2 lies in [min, max] of its coefficients.  E_hi is the smaller
//     and E_lo the larger of the bounds from b1 = (1, 0, 0) and b2 = (0, 1, 0); with
//     neither certified, E_hi = +inf and E_lo = 0.
// ---------------------------------------------------------------------------
namespace {

struct TPl {  // classical Bernstein coefficients, index (simplex g) * (p+1)(q+1) + i (q+1) + j
  int n = 0, p = 0, q = 0;
  std::vector<double> c;
};

int tsize(int n, int p, int q) { return psize(2, n) * (p + 1) * (q + 1); }

TPl tconst(double v) { return {0, 0, 0, {v}}; }

TPl tmul(const TPl& a, const TPl& b) {
  TPl r;
  r.n = a.n + b.n;
  r.p = a.p + b.p;
  r.q = a.q + b.q;
  r.c.assign(tsize(r.n, r.p, r.q), 0.0);
  const int ba = (a.p + 1) * (a.q + 1), bb = (b.p + 1) * (b.q + 1), br = (r.p + 1) * (r.q + 1);
  for_each_index(2, a.n, [&](int a1, int a2) {
    for_each_index(2, b.n, [&](int b1, int b2) {
      const double ws = multinom(a.n, a1, a2) * multinom(b.n, b1, b2) / multinom(r.n, a1 + b1, a2 + b2);
      const int ia = pidx(2, a.n, a1, a2), ib = pidx(2, b.n, b1, b2), ir = pidx(2, r.n, a1 + b1, a2 + b2);
      for (int i = 0; i <= a.p; ++i)
        for (int k = 0; k <= b.p; ++k) {
          const double wi = binom(a.p, i) * binom(b.p, k) / binom(r.p, i + k);
          for (int j = 0; j <= a.q; ++j)
            for (int l = 0; l <= b.q; ++l) {
              const double wj = binom(a.q, j) * binom(b.q, l) / binom(r.q, j + l);
              r.c[ir * br + (i + k) * (r.q + 1) + (j + l)] +=
                  ws * wi * wj * a.c[ia * ba + i * (a.q + 1) + j] * b.c[ib * bb + k * (b.q + 1) + l];
            }
        }
    });
  });
  return r;
}

// Elevation to (n; p, q): the product with the constant 1 of degree (n - a.n; p - a.p, q - a.q).
TPl televate(const TPl& a, int n, int p, int q) {
  if (a.n == n && a.p == p && a.q == q) return a;
  TPl one{n - a.n, p - a.p, q - a.q, {}};
  one.c.assign(tsize(one.n, one.p, one.q), 1.0);
  return tmul(a, one);
}

TPl tadd(const TPl& a, const TPl& b, double sb = 1.0) {
  const int n = std::max(a.n, b.n), p = std::max(a.p, b.p), q = std::max(a.q, b.q);
  TPl r = televate(a, n, p, q);
  const TPl e = televate(b, n, p, q);
  for (size_t i = 0; i < r.c.size(); ++i) r.c[i] += sb * e.c[i];
  return r;
}

TPl tscale(TPl a, double s) {
  for (auto& v : a.c) v *= s;
  return a;
}

struct TV {
  TPl x, y, z;
};
TV tv_const(V3 a) { return {tconst(a.x), tconst(a.y), tconst(a.z)}; }
TPl tv_dot(const TV& a, const TV& b) { return tadd(tadd(tmul(a.x, b.x), tmul(a.y, b.y)), tmul(a.z, b.z)); }
TV tv_cross(const TV& a, const TV& b) {
  return {tadd(tmul(a.y, b.z), tmul(a.z, b.y), -1.0), tadd(tmul(a.z, b.x), tmul(a.x, b.z), -1.0),
          tadd(tmul(a.x, b.y), tmul(a.y, b.x), -1.0)};
}
TV tv_sub(const TV& a, const TV& b) { return {tadd(a.x, b.x, -1.0), tadd(a.y, b.y, -1.0), tadd(a.z, b.z, -1.0)}; }
TV tv_add(const TV& a, const TV& b) { return {tadd(a.x, b.x), tadd(a.y, b.y), tadd(a.z, b.z)}; }

// Degree (1; 0, 0) from the values at the cell corners.
TV tv_simplex(V3 f0, V3 f1, V3 f2) {
  auto one = [&](double a, double b, double c) {
    TPl r{1, 0, 0, std::vector<double>(3)};
    r.c[pidx(2, 1, 0, 0)] = a;
    r.c[pidx(2, 1, 1, 0)] = b;
    r.c[pidx(2, 1, 0, 1)] = c;
    return r;
  };
  return {one(f0.x, f1.x, f2.x), one(f0.y, f1.y, f2.y), one(f0.z, f1.z, f2.z)};
}

// Degree (0; 1, 1): a0 + s es + t et on [0, 1]^2.
TV tv_box(V3 a0, V3 es, V3 et) {
  auto one = [&](double a, double s, double t) { return TPl{0, 1, 1, {a, a + t, a + s, a + s + t}}; };
  return {one(a0.x, es.x, et.x), one(a0.y, es.y, et.y), one(a0.z, es.z, et.z)};
}

double teval(const TPl& a, double l1, double l2, double s, double t) {
  double sum = 0.0;
  const double l0 = 1.0 - l1 - l2;
  const int bs = (a.p + 1) * (a.q + 1);
  for_each_index(2, a.n, [&](int g1, int g2) {
    const int g0 = a.n - g1 - g2;
    const double bsx = multinom(a.n, g1, g2) * std::pow(l0, g0) * std::pow(l1, g1) * std::pow(l2, g2);
    for (int i = 0; i <= a.p; ++i)
      for (int j = 0; j <= a.q; ++j)
        sum += bsx * binom(a.p, i) * std::pow(s, i) * std::pow(1.0 - s, a.p - i) * binom(a.q, j) * std::pow(t, j) *
               std::pow(1.0 - t, a.q - j) * a.c[pidx(2, a.n, g1, g2) * bs + i * (a.q + 1) + j];
  });
  return sum;
}

struct ImplicitForms {
  TPl F, G, detA, detB, L0;
};

// The forms of the implicit Jacobian for one cell C (corners in T's (u, v)), one receiver box and
// one vector b; detA and detB at degree (7; 3, 3).
ImplicitForms implicit_forms(const Tri& T, V3 x0, double eta, const Rec& R, const UV C[3], double ul, double uh,
                             double vl, double vh, V3 b) {
  const V3 Eu = T.p[1] - T.p[0], Ev = T.p[2] - T.p[0], Nu = T.n[1] - T.n[0], Nv = T.n[2] - T.n[0];
  auto X = [&](const UV& c) { return T.p[0] + c.u * Eu + c.v * Ev; };
  auto Nn = [&](const UV& c) { return T.n[0] + c.u * Nu + c.v * Nv; };
  const TV x1 = tv_simplex(X(C[0]), X(C[1]), X(C[2]));
  const TV n1 = tv_simplex(Nn(C[0]), Nn(C[1]), Nn(C[2]));
  const TV xk = tv_box(R.p0 + ul * R.e1 + vl * R.e2, (uh - ul) * R.e1, (vh - vl) * R.e2);
  const TV d0 = tv_sub(x1, tv_const(x0));
  const TV d1 = tv_sub(xk, x1);
  const TV B = tv_const(b);
  const TV d0n = tv_cross(d0, n1);
  const TPl A = tv_dot(d0n, B);
  const TPl Cc = tv_dot(tv_cross(d1, n1), B);
  const TPl L1 = tv_dot(d1, d1), L0 = tv_dot(d0, d0);
  const double e2 = eta * eta;
  ImplicitForms out;
  out.F = tadd(tscale(tmul(L1, tmul(A, A)), e2), tmul(L0, tmul(Cc, Cc)), -1.0);
  out.G = tv_dot(d0n, d1);
  // derivatives along T's u or v (edge E, normal difference N)
  auto dF_dG_1 = [&](V3 E, V3 N, TPl* dF, TPl* dG) {
    const TV Ec = tv_const(E), Nc = tv_const(N);
    const TV dd0n = tv_add(tv_cross(Ec, n1), tv_cross(d0, Nc));          // d(d0 x n1)
    const TPl dA = tv_dot(dd0n, B);
    const TPl dC = tv_dot(tv_sub(tv_cross(d1, Nc), tv_cross(Ec, n1)), B);  // d(d1 x n1).b, d d1 = -E
    const TPl dL1 = tscale(tv_dot(d1, Ec), -2.0), dL0 = tscale(tv_dot(d0, Ec), 2.0);
    *dF = tadd(tscale(tadd(tmul(dL1, tmul(A, A)), tscale(tmul(L1, tmul(A, dA)), 2.0)), e2),
               tadd(tmul(dL0, tmul(Cc, Cc)), tscale(tmul(L0, tmul(Cc, dC)), 2.0)), -1.0);
    *dG = tadd(tv_dot(dd0n, d1), tv_dot(d0n, Ec), -1.0);
  };
  // derivatives along the receiver's u_k or v_k (edge e)
  auto dF_dG_k = [&](V3 e, TPl* dF, TPl* dG) {
    const TV ec = tv_const(e);
    const TPl dC = tv_dot(tv_cross(ec, n1), B);
    const TPl dL1 = tscale(tv_dot(d1, ec), 2.0);
    *dF = tadd(tscale(tmul(dL1, tmul(A, A)), e2), tscale(tmul(L0, tmul(Cc, dC)), 2.0), -1.0);
    *dG = tv_dot(d0n, ec);
  };
  TPl Fu, Gu, Fv, Gv, Fuk, Guk, Fvk, Gvk;
  dF_dG_1(Eu, Nu, &Fu, &Gu);
  dF_dG_1(Ev, Nv, &Fv, &Gv);
  dF_dG_k(R.e1, &Fuk, &Guk);
  dF_dG_k(R.e2, &Fvk, &Gvk);
  out.detA = televate(tadd(tmul(Fu, Gv), tmul(Fv, Gu), -1.0), 7, 3, 3);
  out.detB = televate(tadd(tmul(Fuk, Gvk), tmul(Fvk, Guk), -1.0), 7, 3, 3);
  out.L0 = L0;
  return out;
}

// E_lo, E_hi of one refraction record by implicit differentiation (header comment above).
void implicit_irradiance(const Tri& T, V3 x0, double I0, double eta, const Rec& R, const UV C[3], double ul,
                         double uh, double vl, double vh, int b_mask, double* e_lo, double* e_hi) {
  const double inf = std::numeric_limits<double>::infinity();
  const V3 N1 = cross(T.p[1] - T.p[0], T.p[2] - T.p[0]);
  const double k = I0 * std::fabs(dot(T.p[0] - x0, N1)) / norm(cross(R.e1, R.e2));
  double hi = inf, lo = 0.0;
  const V3 bs[2] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}};
  for (int ib = 0; ib < 2; ++ib) {
    if (!(b_mask & (1 << ib))) continue;
    const V3& b = bs[ib];
    const ImplicitForms f = implicit_forms(T, x0, eta, R, C, ul, uh, vl, vh, b);
    bool pos = true, neg = true;
    for (double v : f.detA.c) {
      if (!(v > 0.0)) pos = false;
      if (!(v < 0.0)) neg = false;
    }
    if (!pos && !neg) continue;
    double rmin = inf, rmax = -inf;
    for (size_t i = 0; i < f.detA.c.size(); ++i) {
      const double r = f.detB.c[i] / f.detA.c[i];
      rmin = std::min(rmin, r);
      rmax = std::max(rmax, r);
    }
    const double amax = std::max(std::fabs(rmin), std::fabs(rmax));
    const double amin = rmin > 0.0 ? rmin : (rmax < 0.0 ? -rmax : 0.0);
    const double s_lo = *std::min_element(f.L0.c.begin(), f.L0.c.end());
    const double s_hi = *std::max_element(f.L0.c.begin(), f.L0.c.end());
    hi = std::min(hi, s_lo > 0.0 ? k * amax / (s_lo * std::sqrt(s_lo)) : inf);
    lo = std::max(lo, k * amin / (s_hi * std::sqrt(s_hi)));
  }
  *e_lo = lo;
  *e_hi = hi;
}

}  // namespace

extern "C" {

// Implicit-differentiation irradiance bounds of n single-refraction records (emitter, tri0,
// cell id at depth, position box): e_lo[i], e_hi[i].  b_mask: 1 = b (1,0,0) only, 2 = (0,1,0)
// only, 3 = both (the tighter of the two).
int orc_implicit_bound(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int64_t n,
                       const int32_t* emitter, const int32_t* tri0, const uint32_t* cell, const int32_t* depth,
                       const double* u_lo, const double* u_hi, const double* v_lo, const double* v_hi, double* e_lo,
                       double* e_hi, int n_threads, int b_mask) {
  if (s1->kind != 1) return -1;
  const Rec R = get_rec(rec);
  parallel_for(n, n_threads, [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      const int e = emitter[i];
      UV C[3];
      cell_corners(cell[i], depth[i], C);
      const V3 x0 = {em->x[e], em->y[e], em->z[e]};
      implicit_irradiance(get_tri(s1, tri0[i]), x0, em->intensity[e], s1->eta, R, C, u_lo[i], u_hi[i], v_lo[i],
                          v_hi[i], b_mask, &e_lo[i], &e_hi[i]);
    }
  });
  return 0;
}

// The implicit forms of one record evaluated at n points (cell barycentrics l1, l2; box
// coordinates s, t), for b = (1,0,0) (which_b 0) or (0,1,0) (1): out[5 i + 0..4] = F, G,
// det A, det B, |d0|^2.
int orc_implicit_eval(const orc_surface* s1, const orc_receiver* rec, const orc_emitters* em, int32_t e, int32_t t,
                      uint32_t cell, int32_t depth, double ul, double uh, double vl, double vh, int32_t which_b,
                      int64_t n, const double* l1, const double* l2, const double* s, const double* tt, double* out) {
  if (s1->kind != 1) return -1;
  UV C[3];
  cell_corners(cell, depth, C);
  const V3 x0 = {em->x[e], em->y[e], em->z[e]};
  const V3 b = which_b == 0 ? V3{1.0, 0.0, 0.0} : V3{0.0, 1.0, 0.0};
  const ImplicitForms f = implicit_forms(get_tri(s1, t), x0, s1->eta, get_rec(rec), C, ul, uh, vl, vh, b);
  for (int64_t i = 0; i < n; ++i) {
    out[5 * i + 0] = teval(f.F, l1[i], l2[i], s[i], tt[i]);
    out[5 * i + 1] = teval(f.G, l1[i], l2[i], s[i], tt[i]);
    out[5 * i + 2] = teval(f.detA, l1[i], l2[i], s[i], tt[i]);
    out[5 * i + 3] = teval(f.detB, l1[i], l2[i], s[i], tt[i]);
    out[5 * i + 4] = teval(f.L0, l1[i], l2[i], s[i], tt[i]);
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Implicit differentiation for two-vertex chains whose first vertex reflects (Sec. 4.4
// "Implicit differentiation": the specular constraint at the last specular vertex x2 in u1
// and u_k, with u2 substituted by its rational function of u1).
//
//   * First vertex (reflection, Eq. eq_refr_rational): d~1 = (n1.n1) d0 - 2 (d0.n1) n1, exact
//     (no square root), so u2 = U2/Q2, v2 = V2/Q2 on T2's plane (Eq. eq_rct, Moller form) is
//     an exact rational function of u1, and x2 = X2/Q2, n2 = N2/Q2 with
//     X2 = p20 Q2 + U2 e21 + V2 e22, N2 = n20 Q2 + U2 (n21 - n20) + V2 (n22 - n20).
//   * Constraints at x2 with d1 = x2 - x1 = D1/Q2, d2 = x_k - x2 = D2/Q2 (D1 = X2 - x1 Q2,
//     D2 = x_k Q2 - X2) and A = (D1 x N2).b, C = (D2 x N2).b:
//       F~ = eta2'^2 |D2|^2 A^2 - |D1|^2 C^2  (eta2' = 1 for a reflecting second vertex),
//       G~ = (D1 x N2).D2,
//     the section's F and G times powers of Q2 (functions of u1 alone): on the path manifold,
//     where F = G = 0, the derivatives scale by the same factors and |du1/du_k| is unchanged.
//   * Derivatives along u1 are taken in the cell's barycentric coordinates (Bernstein
//     differencing), then det d(F,G)/d(u1,v1) = det d(F,G)/d(l1,l2) / det M with M the cell's
//     edge matrix in T1's (u, v); along u_k by the product rule (d D2/du_k = e1 Q2, v_k: e2 Q2).
//   * E = I0 |C1| |det B| |det M| / (|d0|^3 |N_k| |det A_l|), bounded like the single-vertex
//     case over the cell x the record's receiver box; the tighter of b = x and y.
// ---------------------------------------------------------------------------
namespace {

// d/d l_j (j = 1, 2) of a tensor form in the simplex's barycentric coordinates (l0 = 1 - l1 - l2):
// degree n - 1 with classical coefficients n (c_{g + e_j} - c_{g + e_0}).
TPl tderiv_simplex(const TPl& a, int j) {
  TPl r{a.n - 1, a.p, a.q, {}};
  r.c.assign(tsize(r.n, r.p, r.q), 0.0);
  const int bs = (a.p + 1) * (a.q + 1);
  for_each_index(2, r.n, [&](int g1, int g2) {
    const int ij = j == 1 ? pidx(2, a.n, g1 + 1, g2) : pidx(2, a.n, g1, g2 + 1);
    const int i0 = pidx(2, a.n, g1, g2);
    const int ir = pidx(2, r.n, g1, g2);
    for (int k = 0; k < bs; ++k) r.c[ir * bs + k] = a.n * (a.c[ij * bs + k] - a.c[i0 * bs + k]);
  });
  return r;
}

TV tv_scale_poly(const TPl& s, const TV& a) { return {tmul(s, a.x), tmul(s, a.y), tmul(s, a.z)}; }
TV tv_constmul(const TPl& s, V3 c) { return {tscale(s, c.x), tscale(s, c.y), tscale(s, c.z)}; }
TPl tv_comp(const TV& a, int c) { return c == 0 ? a.x : (c == 1 ? a.y : a.z); }

struct ChainForms {
  TPl F, G, detA, detB, L0;
  double detM;
};

// Forms of one reflecting-first chain record (cell C of T1 = A, second vertex on T2 = Bt with the
// law eta2 (< 0: mirror), receiver box) for the vector component b (0: x, 1: y).
ChainForms chain_forms(const Tri& A, const Tri& Bt, V3 x0, double eta2, const Rec& R, const UV C[3], double ul,
                       double uh, double vl, double vh, int bc) {
  const V3 Eu = A.p[1] - A.p[0], Ev = A.p[2] - A.p[0], Nu = A.n[1] - A.n[0], Nv = A.n[2] - A.n[0];
  auto X = [&](const UV& c) { return A.p[0] + c.u * Eu + c.v * Ev; };
  auto Nn = [&](const UV& c) { return A.n[0] + c.u * Nu + c.v * Nv; };
  const TV x1 = tv_simplex(X(C[0]), X(C[1]), X(C[2]));
  const TV n1 = tv_simplex(Nn(C[0]), Nn(C[1]), Nn(C[2]));
  const TV d0 = tv_sub(x1, tv_const(x0));
  const TPl nn = tv_dot(n1, n1), dn = tv_dot(d0, n1);
  const TV dt = tv_sub(tv_scale_poly(nn, d0), tv_scale_poly(tscale(dn, 2.0), n1));  // reflected, degree 3
  const V3 p20 = Bt.p[0], e21 = Bt.p[1] - p20, e22 = Bt.p[2] - p20;
  const V3 n20 = Bt.n[0], dn21 = Bt.n[1] - n20, dn22 = Bt.n[2] - n20;
  const TV w2 = tv_sub(x1, tv_const(p20));
  const TV dxe = tv_cross(dt, tv_const(e22));
  const TPl Q2 = tv_dot(dxe, tv_const(e21));
  const TPl U2 = tv_dot(dxe, w2);
  const TPl V2 = tv_dot(tv_cross(w2, tv_const(e21)), dt);
  const TV X2 = tv_add(tv_add(tv_constmul(Q2, p20), tv_constmul(U2, e21)), tv_constmul(V2, e22));
  const TV N2 = tv_add(tv_add(tv_constmul(Q2, n20), tv_constmul(U2, dn21)), tv_constmul(V2, dn22));
  const TV D1 = tv_sub(X2, tv_scale_poly(Q2, x1));
  const TV xk = tv_box(R.p0 + ul * R.e1 + vl * R.e2, (uh - ul) * R.e1, (vh - vl) * R.e2);
  const TV D2 = tv_sub(tv_scale_poly(Q2, xk), X2);
  const TV D1N = tv_cross(D1, N2), D2N = tv_cross(D2, N2);
  const TPl Ab = tv_comp(D1N, bc), Cb = tv_comp(D2N, bc);
  const TPl L1 = tv_dot(D2, D2), L1b = tv_dot(D1, D1);
  const double e2 = eta2 < 0.0 ? 1.0 : eta2 * eta2;
  ChainForms out;
  out.F = tadd(tscale(tmul(L1, tmul(Ab, Ab)), e2), tmul(L1b, tmul(Cb, Cb)), -1.0);
  out.G = tv_dot(D1N, D2);
  const TPl F1 = tderiv_simplex(out.F, 1), F2 = tderiv_simplex(out.F, 2);
  const TPl G1 = tderiv_simplex(out.G, 1), G2 = tderiv_simplex(out.G, 2);
  out.detA = televate(tadd(tmul(F1, G2), tmul(F2, G1), -1.0), 34, 3, 3);
  auto dk = [&](V3 e, TPl* dF, TPl* dG) {
    const TV eQ = tv_constmul(Q2, e);  // d D2 / d u_k
    const TPl dC = tv_comp(tv_cross(eQ, N2), bc);
    *dF = tadd(tscale(tmul(tscale(tv_dot(D2, eQ), 2.0), tmul(Ab, Ab)), e2), tmul(L1b, tscale(tmul(Cb, dC), 2.0)),
               -1.0);
    *dG = tv_dot(D1N, eQ);
  };
  TPl Fu, Gu, Fv, Gv;
  dk(R.e1, &Fu, &Gu);
  dk(R.e2, &Fv, &Gv);
  out.detB = televate(tadd(tmul(Fu, Gv), tmul(Fv, Gu), -1.0), 34, 3, 3);
  out.L0 = tv_dot(d0, d0);
  out.detM = (C[1].u - C[0].u) * (C[2].v - C[0].v) - (C[2].u - C[0].u) * (C[1].v - C[0].v);
  return out;
}

double chain_k(const Tri& A, V3 x0, double I0, const Rec& R) {
  const V3 N1 = cross(A.p[1] - A.p[0], A.p[2] - A.p[0]);
  return I0 * std::fabs(dot(A.p[0] - x0, N1)) / norm(cross(R.e1, R.e2));
}

}  // namespace

extern "C" {

// Implicit-differentiation irradiance bounds of n chain records (emitter, tri0 on s1, cell at
// depth, tri1 on s2, receiver box) whose first vertex reflects: e_lo[i], e_hi[i].  b_mask as in
// orc_implicit_bound.  Returns -1 unless s1 reflects.
int orc_implicit_bound_pairs(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec,
                             const orc_emitters* em, int64_t n, const int32_t* emitter, const int32_t* tri0,
                             const uint32_t* cell, const int32_t* depth, const int32_t* tri1, const double* u_lo,
                             const double* u_hi, const double* v_lo, const double* v_hi, double* e_lo, double* e_hi,
                             int n_threads, int b_mask) {
  if (s1->kind != 0) return -1;
  const Rec R = get_rec(rec);
  const double inf = std::numeric_limits<double>::infinity();
  parallel_for(n, n_threads, [&](int, int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      const int e = emitter[i];
      UV C[3];
      cell_corners(cell[i], depth[i], C);
      const V3 x0 = {em->x[e], em->y[e], em->z[e]};
      const Tri A = get_tri(s1, tri0[i]), Bt = get_tri(s2, tri1[i]);
      const double k = chain_k(A, x0, em->intensity[e], R);
      double hi = inf, lo = 0.0;
      for (int bc = 0; bc < 2; ++bc) {
        if (!(b_mask & (1 << bc))) continue;
        const ChainForms f = chain_forms(A, Bt, x0, law(s2), R, C, u_lo[i], u_hi[i], v_lo[i], v_hi[i], bc);
        bool pos = true, neg = true;
        for (double v : f.detA.c) {
          if (!(v > 0.0)) pos = false;
          if (!(v < 0.0)) neg = false;
        }
        if (!pos && !neg) continue;
        double rmin = inf, rmax = -inf;
        for (size_t j = 0; j < f.detA.c.size(); ++j) {
          const double r = f.detB.c[j] / f.detA.c[j];
          rmin = std::min(rmin, r);
          rmax = std::max(rmax, r);
        }
        const double amax = std::max(std::fabs(rmin), std::fabs(rmax));
        const double amin = rmin > 0.0 ? rmin : (rmax < 0.0 ? -rmax : 0.0);
        const double s_lo = *std::min_element(f.L0.c.begin(), f.L0.c.end());
        const double s_hi = *std::max_element(f.L0.c.begin(), f.L0.c.end());
        const double m = std::fabs(f.detM);
        hi = std::min(hi, s_lo > 0.0 ? k * m * amax / (s_lo * std::sqrt(s_lo)) : inf);
        lo = std::max(lo, k * m * amin / (s_hi * std::sqrt(s_hi)));
      }
      e_lo[i] = lo;
      e_hi[i] = hi;
    }
  });
  return 0;
}

// The chain forms of one record at n points (cell barycentrics l1, l2; box coordinates s, t), for
// b component which_b: out[3 i + 0..2] = F~, G~ and the irradiance I0 |C1| |det B| |det M| /
// (|d0|^3 |N_k| |det A_l|).
int orc_implicit_eval_pair(const orc_surface* s1, const orc_surface* s2, const orc_receiver* rec,
                           const orc_emitters* em, int32_t e, int32_t t1, uint32_t cell, int32_t depth, int32_t t2,
                           double ul, double uh, double vl, double vh, int32_t which_b, int64_t n, const double* l1,
                           const double* l2, const double* s, const double* tt, double* out) {
  if (s1->kind != 0) return -1;
  UV C[3];
  cell_corners(cell, depth, C);
  const V3 x0 = {em->x[e], em->y[e], em->z[e]};
  const Rec R = get_rec(rec);
  const Tri A = get_tri(s1, t1), Bt = get_tri(s2, t2);
  const ChainForms f = chain_forms(A, Bt, x0, law(s2), R, C, ul, uh, vl, vh, which_b);
  const double k = chain_k(A, x0, em->intensity[e], R);
  for (int64_t i = 0; i < n; ++i) {
    const double L0 = teval(f.L0, l1[i], l2[i], s[i], tt[i]);
    out[3 * i + 0] = teval(f.F, l1[i], l2[i], s[i], tt[i]);
    out[3 * i + 1] = teval(f.G, l1[i], l2[i], s[i], tt[i]);
    out[3 * i + 2] = k * std::fabs(teval(f.detB, l1[i], l2[i], s[i], tt[i]) * f.detM) /
                     (L0 * std::sqrt(L0) * std::fabs(teval(f.detA, l1[i], l2[i], s[i], tt[i])));
  }
  return 0;
}

}  // extern "C"
