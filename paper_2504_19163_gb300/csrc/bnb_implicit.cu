// Implicit-differentiation irradiance bound of single-refraction records (Sec. 4.4,
// "Implicit differentiation", with the specular polynomials F, G of the section's footnote).
//
// A post-pass over bound records: for a live record (emitter, T1, cell, position box) the
// cell's barycentric coordinates and the receiver coordinates of the box are independent
// variables (the 4D superset of the paths' 2D manifold).  With d0 = x1 - x0, d1 = x_k - x1,
// n1 the interpolated normal and b = (1,0,0) or (0,1,0), A = (d0 x n1).b, C = (d1 x n1).b:
//   F = eta'^2 |d1|^2 A^2 - |d0|^2 C^2   (Snell's law squared along b, scaled by the constant
//                                         eta'^2 = (incident/transmitted)^2, which cancels),
//   G = (d0 x n1).d1,
// whose partial derivatives follow from the product rule with constant derivative vectors
// (T1's edges and normal differences, the receiver's edges).  The implicit-function theorem
// gives |du1/du_k| = |det B| / |det A|, A = d(F,G)/d(u1,v1), B = d(F,G)/d(u_k,v_k), and with
// Eq. eq_dwda E = I0 |C1| |det B| / (|d0|^3 |N_k| |det A|).  Bound (Eq. eq_bbound): when every
// coefficient of det A (degree 7 on the cell x 3 x 3 on the box) is non-zero with one sign,
// |det B / det A| lies between the coefficient ratios; |d0|^2 between its coefficients.  The
// result is the tighter of the two b vectors; neither certified: E_hi = +inf, E_lo = 0.
//
// Layout: one warp per record, its polynomials in shared memory (float64, scaled Bernstein
// coefficients on simplex x interval x interval, so products are plain convolutions), each
// with a bound B of its classical coefficients and a radius E of their rounding error (the
// product rule of the other bound kernels, u = 2^-53).  Lanes split every product's output
// coefficients.  Persistent grid over records.
#include <stdint.h>

#include <algorithm>

#include "bnb_bound_impl.cuh"  // cell_corners
#include "bnb_internal.cuh"

namespace bnb {
namespace {

constexpr int kImpWarps = 2;                 // records in flight per block
constexpr int kImpThreads = 32 * kImpWarps;
constexpr int kImpScratch = 3072;            // doubles of shared memory per warp (24 KB)
constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53

__device__ __forceinline__ int nsx(int n) { return (n + 1) * (n + 2) / 2; }
__device__ __forceinline__ int tsz(int n, int p, int q) { return nsx(n) * (p + 1) * (q + 1); }
__device__ __forceinline__ int sidx_of(int n, int g1, int g2) { return g1 * (n + 1) - g1 * (g1 - 1) / 2 + g2; }

// Small binomials and multinomials (exact in double): C(n, k) for n < 32 from a table built at
// compile time by Pascal's rule (integers below 2^53, so every sum is exact), else the product
// formula, whose every partial value is an integer too.
struct BinomTable {
  double v[32][32];
};
constexpr BinomTable binom_table() {
  BinomTable t{};
  for (int n = 0; n < 32; ++n) {
    t.v[n][0] = 1.0;
    for (int k = 1; k <= n; ++k) t.v[n][k] = t.v[n - 1][k - 1] + (k < n ? t.v[n - 1][k] : 0.0);
  }
  return t;
}
__device__ const BinomTable g_binom = binom_table();

__device__ __forceinline__ double dbinom(int n, int k) {
  if (n < 32) return __ldg(&g_binom.v[n][k]);
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}
__device__ __forceinline__ double dmultinom(int n, int g1, int g2) { return dbinom(n, g1) * dbinom(n - g1, g2); }

// gamma_K = K u / (1 - K u), rounded up.
__device__ __forceinline__ double gam64(int K) { return __ddiv_ru((double)K * kU64, 1.0 - (double)K * kU64); }

// A polynomial of degree (n; p, q): scaled coefficients in warp-private shared memory, indexed
// (simplex index) * (p+1)(q+1) + i (q+1) + j; B >= max |classical coefficient| of the exact value,
// E >= max |computed - exact| over the classical coefficients.
struct Ten {
  double* c;
  int n, p, q;
  double B, E;
  int cap;   // coefficients allocated
  int* err;  // set when an operation's result would not fit (the write is skipped)
};

// Bump allocator over the warp's scratch; an overflow sets err (no access past the end).
struct Arena {
  double* base;
  int off;
  int err;
  __device__ Ten make(int n, int p, int q) {
    const int m = tsz(n, p, q);
    if (off + m > kImpScratch) {
      err = 1;
      return Ten{base, n, p, q, 0.0, 0.0, 0, &err};  // capacity 0: every write is skipped
    }
    Ten t{base + off, n, p, q, 0.0, 0.0, m, &err};
    off += m;
    return t;
  }
};

// Rounding bookkeeping of r (+)= a * b, computed as an FMA chain of at most K terms per output.
__device__ __forceinline__ void track_mul(Ten& r, double aB, double aE, double bB, double bE, int K, bool acc) {
  const double a1 = __dadd_ru(aB, aE), b1 = __dadd_ru(bB, bE);
  const double inh = __fma_ru(aE, b1, __dmul_ru(aB, bE));
  const double rB0 = acc ? r.B : 0.0, rE0 = acc ? r.E : 0.0;
  const double mag = __fma_ru(a1, b1, __dadd_ru(rB0, rE0));
  r.E = __dadd_ru(__dadd_ru(rE0, inh), __dmul_ru(gam64(K), mag));
  r.B = __fma_ru(aB, bB, rB0);
}

// r (+)= sgn * a * b (sgn exact: +-1 or +-2).  bc == nullptr: b is the constant 1 of degree
// (bn; bp, bq) (degree elevation).  r must not alias a or b.
__device__ void tmul(Ten& r, const Ten& a, const double* bc, int bn, int bp, int bq, double bB, double bE, double sgn,
                     bool acc, int lane) {
  const int rn = a.n + bn, rp = a.p + bp, rq = a.q + bq;
  if (!acc) {
    r.n = rn;
    r.p = rp;
    r.q = rq;
  }
  const int rs = tsz(rn, rp, rq), rbox = (rp + 1) * (rq + 1);
  const int abox = (a.p + 1) * (a.q + 1), bbox = (bp + 1) * (bq + 1);
  if (rs > r.cap || (acc && (rn != r.n || rp != r.p || rq != r.q))) {
    *r.err = 1;
    return;
  }
  const double isgn = 1.0 / sgn;
  for (int o = lane; o < rs; o += 32) {
    const int si = o / rbox, bx = o - si * rbox;
    const int i = bx / (rq + 1), j = bx - i * (rq + 1);
    int g1 = 0, t = si;
    while (t > rn - g1) {
      t -= rn - g1 + 1;
      ++g1;
    }
    const int g2 = t;
    // sgn is +-1 or +-2: scaling by it is exact and commutes with rounding, so the chain runs on
    // s / sgn with the plain products and is scaled back once (the same value as scaling each term)
    double s = acc ? r.c[o] * isgn : 0.0;
    for (int a1 = max(0, g1 - bn); a1 <= min(g1, a.n); ++a1) {
      const int b1 = g1 - a1;
      for (int a2 = max(0, g2 - (bn - b1)); a2 <= min(g2, a.n - a1); ++a2) {
        const int b2 = g2 - a2;
        const double* ap = a.c + sidx_of(a.n, a1, a2) * abox;
        const int bsi = sidx_of(bn, b1, b2);
        const double wb = bc ? 0.0 : dmultinom(bn, b1, b2);
        for (int ia = max(0, i - bp); ia <= min(i, a.p); ++ia) {
          const int ib = i - ia;
          for (int ja = max(0, j - bq); ja <= min(j, a.q); ++ja) {
            const int jb = j - ja;
            const double bv = bc ? bc[bsi * bbox + ib * (bq + 1) + jb] : wb * dbinom(bp, ib) * dbinom(bq, jb);
            s = fma(ap[ia * (a.q + 1) + ja], bv, s);
          }
        }
      }
    }
    r.c[o] = s * sgn;
  }
  __syncwarp();
  const int K = nsx(min(a.n, bn)) * (min(a.p, bp) + 1) * (min(a.q, bq) + 1);
  track_mul(r, fabs(sgn) * a.B, fabs(sgn) * a.E, bB, bE, K, acc);
}

__device__ __forceinline__ void tmul(Ten& r, const Ten& a, const Ten& b, double sgn, bool acc, int lane) {
  tmul(r, a, b.c, b.n, b.p, b.q, b.B, b.E, sgn, acc, lane);
}

// r = a elevated to (n; p, q).
__device__ __forceinline__ void televate(Ten& r, const Ten& a, int n, int p, int q, int lane) {
  tmul(r, a, nullptr, n - a.n, p - a.p, q - a.q, 1.0, 0.0, 1.0, false, lane);
}

// r (+)= s * a (same degree; one FMA per coefficient).  r may alias a when !acc.
__device__ __forceinline__ void tscale(Ten& r, double s, const Ten& a, bool acc, int lane) {
  const int m = tsz(a.n, a.p, a.q);
  if (m > r.cap || (acc && (a.n != r.n || a.p != r.p || a.q != r.q))) {
    *r.err = 1;
    return;
  }
  for (int o = lane; o < m; o += 32) r.c[o] = fma(s, a.c[o], acc ? r.c[o] : 0.0);
  __syncwarp();
  const double aB = a.B, aE = a.E;
  if (!acc) {
    r.n = a.n;
    r.p = a.p;
    r.q = a.q;
  }
  track_mul(r, fabs(s), 0.0, aB, aE, 1, acc);
}

struct TV3 {
  Ten x, y, z;
  __device__ Ten& operator[](int k) { return k == 0 ? x : (k == 1 ? y : z); }
};

__device__ __forceinline__ TV3 make3(Arena& ar, int n, int p, int q) {
  return TV3{ar.make(n, p, q), ar.make(n, p, q), ar.make(n, p, q)};
}

// r = a . b (three products).
__device__ __forceinline__ void tdot(Ten& r, TV3& a, TV3& b, int lane) {
  tmul(r, a.x, b.x, 1.0, false, lane);
  tmul(r, a.y, b.y, 1.0, true, lane);
  tmul(r, a.z, b.z, 1.0, true, lane);
}

// r = a . c for a constant vector c.
__device__ __forceinline__ void tdotc(Ten& r, TV3& a, const double (&c)[3], int lane) {
  tscale(r, c[0], a.x, false, lane);
  tscale(r, c[1], a.y, true, lane);
  tscale(r, c[2], a.z, true, lane);
}

// r = a x b.
__device__ __forceinline__ void tcross(TV3& r, TV3& a, TV3& b, int lane) {
  tmul(r.x, a.y, b.z, 1.0, false, lane);
  tmul(r.x, a.z, b.y, -1.0, true, lane);
  tmul(r.y, a.z, b.x, 1.0, false, lane);
  tmul(r.y, a.x, b.z, -1.0, true, lane);
  tmul(r.z, a.x, b.y, 1.0, false, lane);
  tmul(r.z, a.y, b.x, -1.0, true, lane);
}

// r = c x a (constant c), or r += c x a.
__device__ __forceinline__ void tcrossc(TV3& r, const double (&c)[3], TV3& a, bool acc, int lane) {
  tscale(r.x, c[1], a.z, acc, lane);
  tscale(r.x, -c[2], a.y, true, lane);
  tscale(r.y, c[2], a.x, acc, lane);
  tscale(r.y, -c[0], a.z, true, lane);
  tscale(r.z, c[0], a.y, acc, lane);
  tscale(r.z, -c[1], a.x, true, lane);
}

// (a x N)_c for a constant N: a_{c+1} N_{c+2} - a_{c+2} N_{c+1}.
__device__ __forceinline__ void tcross_comp(Ten& r, TV3& a, const double (&N)[3], int c, int lane) {
  const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
  tscale(r, N[c2], a[c1], false, lane);
  tscale(r, -N[c1], a[c2], true, lane);
}

// Degree (1; 0, 0) from corner values f[k] (corner k at the simplex vertex g_k = 1); E covers the
// roundings of the corner arithmetic.
__device__ __forceinline__ void tsimplex(Ten& r, double f0, double f1, double f2, int lane) {
  if (r.cap < 3) {
    *r.err = 1;
    return;
  }
  if (lane == 0) {
    r.c[sidx_of(1, 0, 0)] = f0;
    r.c[sidx_of(1, 1, 0)] = f1;
    r.c[sidx_of(1, 0, 1)] = f2;
  }
  __syncwarp();
  r.n = 1;
  r.p = r.q = 0;
  r.B = fmax(fabs(f0), fmax(fabs(f1), fabs(f2)));
  r.E = __dmul_ru(gam64(4), r.B);
}

// Degree (0; 1, 1): a0 + s es + t et on the box [0,1]^2.
__device__ __forceinline__ void tbox(Ten& r, double a0, double es, double et, int lane) {
  if (r.cap < 4) {
    *r.err = 1;
    return;
  }
  if (lane == 0) {
    r.c[0] = a0;
    r.c[1] = a0 + et;
    r.c[2] = a0 + es;
    r.c[3] = a0 + es + et;
  }
  __syncwarp();
  r.n = 0;
  r.p = r.q = 1;
  r.B = fmax(fmax(fabs(r.c[0]), fabs(r.c[1])), fmax(fabs(r.c[2]), fabs(r.c[3])));
  r.E = __dmul_ru(gam64(8), r.B);
}

// r = a - k for a degree-(1; 0, 0) form and a constant k (scaled weights of 1 are all 1 there).
__device__ __forceinline__ void tsubc1(Ten& r, const Ten& a, double k, int lane) {
  if (r.cap < 3 || a.n != 1 || a.p != 0 || a.q != 0) {
    *r.err = 1;
    return;
  }
  for (int o = lane; o < 3; o += 32) r.c[o] = a.c[o] - k;
  __syncwarp();
  r.n = 1;
  r.p = r.q = 0;
  r.B = __dadd_ru(a.B, fabs(k));
  r.E = __dadd_ru(a.E, __dmul_ru(gam64(1), __dadd_ru(__dadd_ru(a.B, a.E), fabs(k))));
}

struct ImpParams {
  const float *px, *py, *pz, *nx, *ny, *nz;
  const int32_t *i0, *i1, *i2;
  int32_t n_verts, n_tris;
  float eta;
  const float *ex, *ey, *ez, *ei;
  int32_t n_emitters;
  float rp0[3], re1[3], re2[3];
  const int32_t *emitter, *tri0, *tri1;
  const uint32_t *cell, *flags;
  const float *u_lo, *u_hi, *v_lo, *v_hi;
  float *e_hi, *e_lo;
  int64_t n;             // records; < 0: min(*count, capacity)
  const int64_t* count;
  int64_t capacity;
  int32_t mode;          // 0: write the implicit bound; 1: intersect with the stored bound
};

struct ImpGeom {
  double p[3][3], nv[3][3], x0[3], I0, cu[3], cv[3], ul, uh, vl, vh, eta, R0[3], R1[3], R2[3];
};

// E_lo, E_hi of one record (all lanes return the same values).  *bad: scratch overflow.
__device__ void implicit_record(const ImpGeom& g, double* scratch, int lane, double* e_lo, double* e_hi, bool* bad) {
  Arena ar{scratch, 0, 0};
  double Eu[3], Ev[3], Nu[3], Nv[3], X[3][3], Nn[3][3];
  for (int c = 0; c < 3; ++c) {
    Eu[c] = g.p[1][c] - g.p[0][c];
    Ev[c] = g.p[2][c] - g.p[0][c];
    Nu[c] = g.nv[1][c] - g.nv[0][c];
    Nv[c] = g.nv[2][c] - g.nv[0][c];
    for (int k = 0; k < 3; ++k) {
      X[k][c] = g.p[0][c] + g.cu[k] * Eu[c] + g.cv[k] * Ev[c];
      Nn[k][c] = g.nv[0][c] + g.cu[k] * Nu[c] + g.cv[k] * Nv[c];
    }
  }
  TV3 x1 = make3(ar, 1, 0, 0), n1 = make3(ar, 1, 0, 0), xk = make3(ar, 0, 1, 1);
  TV3 x1e = make3(ar, 1, 1, 1), xke = make3(ar, 1, 1, 1);
  TV3 d0 = make3(ar, 1, 0, 0), d1 = make3(ar, 1, 1, 1), d0n = make3(ar, 2, 0, 0), d1n = make3(ar, 2, 1, 1);
  Ten L1 = ar.make(2, 2, 2), L0 = ar.make(2, 0, 0);
  for (int c = 0; c < 3; ++c) {
    tsimplex(x1[c], X[0][c], X[1][c], X[2][c], lane);
    tsimplex(n1[c], Nn[0][c], Nn[1][c], Nn[2][c], lane);
    const double a0 = g.R0[c] + g.ul * g.R1[c] + g.vl * g.R2[c];
    tbox(xk[c], a0, (g.uh - g.ul) * g.R1[c], (g.vh - g.vl) * g.R2[c], lane);
    tsubc1(d0[c], x1[c], g.x0[c], lane);
    televate(x1e[c], x1[c], 1, 1, 1, lane);
    televate(xke[c], xk[c], 1, 1, 1, lane);
    tscale(d1[c], 1.0, xke[c], false, lane);
    tscale(d1[c], -1.0, x1e[c], true, lane);
  }
  tcross(d0n, d0, n1, lane);
  tcross(d1n, d1, n1, lane);
  tdot(L1, d1, d1, lane);
  tdot(L0, d0, d0, lane);
  // b-independent parts of the derivatives along T1's u, v (edge E, normal difference N)
  TV3 dd0n[2] = {make3(ar, 1, 0, 0), make3(ar, 1, 0, 0)}, Exn1[2] = {make3(ar, 1, 0, 0), make3(ar, 1, 0, 0)};
  Ten dL1[2] = {ar.make(1, 1, 1), ar.make(1, 1, 1)}, dL0[2] = {ar.make(1, 0, 0), ar.make(1, 0, 0)};
  Ten dG[2] = {ar.make(2, 1, 1), ar.make(2, 1, 1)};
  Ten t6 = ar.make(2, 0, 0), t24 = ar.make(2, 1, 1);
  for (int dir = 0; dir < 2; ++dir) {
    const double (&E)[3] = dir == 0 ? Eu : Ev;
    const double(&N)[3] = dir == 0 ? Nu : Nv;
    const double mN[3] = {-N[0], -N[1], -N[2]};
    tcrossc(Exn1[dir], E, n1, false, lane);  // E x n1
    tcrossc(dd0n[dir], E, n1, false, lane);
    tcrossc(dd0n[dir], mN, d0, true, lane);  // + d0 x N
    tdotc(dL1[dir], d1, E, lane);
    tscale(dL1[dir], -2.0, dL1[dir], false, lane);
    tdotc(dL0[dir], d0, E, lane);
    tscale(dL0[dir], 2.0, dL0[dir], false, lane);
    tdot(dG[dir], dd0n[dir], d1, lane);  // dG = d(d0 x n1).d1 - (d0 x n1).E
    tdotc(t6, d0n, E, lane);
    televate(t24, t6, 2, 1, 1, lane);
    tscale(dG[dir], -1.0, t24, true, lane);
  }
  // along the receiver's u_k, v_k (edge e)
  TV3 exn1[2] = {make3(ar, 1, 0, 0), make3(ar, 1, 0, 0)};
  Ten dL1k[2] = {ar.make(1, 1, 1), ar.make(1, 1, 1)}, dGk[2] = {ar.make(2, 0, 0), ar.make(2, 0, 0)};
  for (int dir = 0; dir < 2; ++dir) {
    const double (&e)[3] = dir == 0 ? g.R1 : g.R2;
    tcrossc(exn1[dir], e, n1, false, lane);
    tdotc(dL1k[dir], d1, e, lane);
    tscale(dL1k[dir], 2.0, dL1k[dir], false, lane);
    tdotc(dGk[dir], d0n, e, lane);
  }
  const int mark = ar.off;
  const double e2 = g.eta * g.eta;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double hi = inf, lo = 0.0;
  for (int c = 0; c < 2; ++c) {  // b = (1,0,0), then (0,1,0): A, C are the c-th components
    ar.off = mark;
    Ten& A = d0n[c];
    Ten& C = d1n[c];
    Ten A2 = ar.make(4, 0, 0), A2e = ar.make(4, 0, 0), C2 = ar.make(4, 2, 2);
    tmul(A2, A, A, 1.0, false, lane);
    tscale(A2e, e2, A2, false, lane);  // eta'^2 A^2
    tmul(C2, C, C, 1.0, false, lane);
    Ten AdA = ar.make(3, 0, 0), CdC = ar.make(3, 2, 2), T84 = ar.make(5, 1, 1), dC = ar.make(1, 1, 1),
        t12 = ar.make(1, 1, 1);
    Ten Fd[2] = {ar.make(5, 2, 2), ar.make(5, 2, 2)};
    for (int dir = 0; dir < 2; ++dir) {
      const double(&N)[3] = dir == 0 ? Nu : Nv;
      // dC = (d1 x N - E x n1).b
      tcross_comp(dC, d1, N, c, lane);
      televate(t12, Exn1[dir][c], 1, 1, 1, lane);
      tscale(dC, -1.0, t12, true, lane);
      // dF = eta'^2 (dL1 A^2 + 2 L1 A dA) - (dL0 C^2 + 2 L0 C dC)
      tmul(T84, dL1[dir], A2e, 1.0, false, lane);
      televate(Fd[dir], T84, 5, 2, 2, lane);
      tmul(AdA, A, dd0n[dir][c], 1.0, false, lane);
      tscale(AdA, e2, AdA, false, lane);
      tmul(Fd[dir], L1, AdA, 2.0, true, lane);
      tmul(Fd[dir], dL0[dir], C2, -1.0, true, lane);
      tmul(CdC, C, dC, 1.0, false, lane);
      tmul(Fd[dir], L0, CdC, -2.0, true, lane);
    }
    Ten CdCk = ar.make(3, 1, 1);
    Ten Fk[2] = {ar.make(5, 1, 1), ar.make(5, 1, 1)};
    for (int dir = 0; dir < 2; ++dir) {
      // dF = eta'^2 dL1 A^2 - 2 L0 C dC,  dC = (e x n1).b
      tmul(Fk[dir], dL1k[dir], A2e, 1.0, false, lane);
      tmul(CdCk, C, exn1[dir][c], 1.0, false, lane);
      tmul(Fk[dir], L0, CdCk, -2.0, true, lane);
    }
    Ten detA = ar.make(7, 3, 3), detB7 = ar.make(7, 1, 1), detB = ar.make(7, 3, 3);
    tmul(detA, Fd[0], dG[1], 1.0, false, lane);
    tmul(detA, Fd[1], dG[0], -1.0, true, lane);
    tmul(detB7, Fk[0], dGk[1], 1.0, false, lane);
    tmul(detB7, Fk[1], dGk[0], -1.0, true, lane);
    televate(detB, detB7, 7, 3, 3, lane);
    if (ar.err || detA.n != 7 || detA.p != 3 || detA.q != 3 || detB.n != 7 || detB.p != 3 || detB.q != 3) {
      ar.err = 1;
      break;
    }
    // coefficient ratios: scaled coefficients share the weight w of their index, so the classical
    // radius E becomes E w
    bool pos = true, neg = true, bpos = true, bneg = true;
    double rmax = 0.0, rmin = inf;
    for (int o = lane; o < 576; o += 32) {
      const int si = o / 16, bx = o - si * 16, i = bx / 4, j = bx - i * 4;
      int g1 = 0, t = si;
      while (t > 7 - g1) {
        t -= 8 - g1;
        ++g1;
      }
      const double w = dmultinom(7, g1, t) * dbinom(3, i) * dbinom(3, j);
      const double a = detA.c[o], b = detB.c[o];
      const double ea = __dmul_ru(detA.E, w), eb = __dmul_ru(detB.E, w);
      pos = pos && __dsub_rd(a, ea) > 0.0;
      neg = neg && __dadd_ru(a, ea) < 0.0;
      bpos = bpos && __dsub_rd(b, eb) > 0.0;
      bneg = bneg && __dadd_ru(b, eb) < 0.0;
      const double alo = __dsub_rd(fabs(a), ea), ahi = __dadd_ru(fabs(a), ea);
      const double bhi = __dadd_ru(fabs(b), eb), blo = fmax(0.0, __dsub_rd(fabs(b), eb));
      rmax = fmax(rmax, alo > 0.0 ? __ddiv_ru(bhi, alo) : inf);
      rmin = fmin(rmin, __ddiv_rd(blo, ahi));
    }
    pos = __all_sync(0xffffffffu, pos);
    neg = __all_sync(0xffffffffu, neg);
    bpos = __all_sync(0xffffffffu, bpos);
    bneg = __all_sync(0xffffffffu, bneg);
    for (int s = 16; s > 0; s >>= 1) {
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, s));
      rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, s));
    }
    if (!pos && !neg) continue;
    const double amin = (bpos || bneg) ? rmin : 0.0;
    // |d0|^2 range: classical coefficients of degree 2 (weights 1 or 2) +- E
    double s_lo = inf, s_hi = 0.0;
    for (int g1 = 0; g1 <= 2; ++g1)
      for (int g2 = 0; g2 <= 2 - g1; ++g2) {
        const double v = L0.c[sidx_of(2, g1, g2)] / dmultinom(2, g1, g2);
        s_lo = fmin(s_lo, __dsub_rd(v, L0.E));
        s_hi = fmax(s_hi, __dadd_ru(v, L0.E));
      }
    if (s_lo > 0.0) {
      const double den_lo = __dmul_rd(s_lo, __dsqrt_rd(s_lo));
      hi = fmin(hi, __ddiv_ru(rmax, den_lo));
    }
    const double den_hi = __dmul_ru(s_hi, __dsqrt_ru(s_hi));
    lo = fmax(lo, __ddiv_rd(amin, den_hi));
  }
  *bad = ar.err != 0;
  *e_lo = lo;
  *e_hi = hi;
}

__global__ void __launch_bounds__(kImpThreads) implicit_k(ImpParams P) {
  extern __shared__ double imp_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* scratch = imp_smem + (size_t)warp * kImpScratch;
  int64_t n = P.n;
  if (n < 0) n = min(*P.count, P.capacity);
  const int64_t stride = (int64_t)gridDim.x * kImpWarps;
  for (int64_t r = (int64_t)blockIdx.x * kImpWarps + warp; r < n; r += stride) {
    const uint32_t fl = P.flags[r];
    if (!(fl & BNB_CELL_LIVE) || P.tri1[r] >= 0) continue;
    const int t = P.tri0[r], e = P.emitter[r];
    const int depth = (int)((fl >> BNB_CELL_DEPTH_SHIFT) & 63u);
    if (t < 0 || t >= P.n_tris || e < 0 || e >= P.n_emitters || depth > 15) continue;
    const int vi[3] = {P.i0[t], P.i1[t], P.i2[t]};
    if (min(vi[0], min(vi[1], vi[2])) < 0 || max(vi[0], max(vi[1], vi[2])) >= P.n_verts) continue;
    ImpGeom g;
    for (int k = 0; k < 3; ++k) {
      g.p[k][0] = P.px[vi[k]];
      g.p[k][1] = P.py[vi[k]];
      g.p[k][2] = P.pz[vi[k]];
      g.nv[k][0] = P.nx[vi[k]];
      g.nv[k][1] = P.ny[vi[k]];
      g.nv[k][2] = P.nz[vi[k]];
      g.R0[k] = P.rp0[k];
      g.R1[k] = P.re1[k];
      g.R2[k] = P.re2[k];
    }
    g.x0[0] = P.ex[e];
    g.x0[1] = P.ey[e];
    g.x0[2] = P.ez[e];
    g.I0 = P.ei[e];
    g.eta = P.eta;
    cell_corners<double>(P.cell[r], depth, g.cu, g.cv);
    g.ul = P.u_lo[r];
    g.uh = P.u_hi[r];
    g.vl = P.v_lo[r];
    g.vh = P.v_hi[r];
    double lo, hi;
    bool bad;
    implicit_record(g, scratch, lane, &lo, &hi, &bad);
    if (bad) continue;
    // I0 |C1| / |N_k|, C1 = (p0 - x0).N1; a relative 1e-12 covers the roundings of these constants
    // and of the double-precision corner arithmetic that seeded the forms
    double E1[3], E2[3], N1[3], Nk[3], d[3];
    for (int c = 0; c < 3; ++c) {
      E1[c] = g.p[1][c] - g.p[0][c];
      E2[c] = g.p[2][c] - g.p[0][c];
      d[c] = g.p[0][c] - g.x0[c];
    }
    for (int c = 0; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      N1[c] = E1[c1] * E2[c2] - E1[c2] * E2[c1];
      Nk[c] = g.R1[c1] * g.R2[c2] - g.R1[c2] * g.R2[c1];
    }
    const double k = g.I0 * fabs(d[0] * N1[0] + d[1] * N1[1] + d[2] * N1[2]) /
                     sqrt(Nk[0] * Nk[0] + Nk[1] * Nk[1] + Nk[2] * Nk[2]);
    double ehi = __dmul_ru(__dmul_ru(k, 1.0 + 1e-12), hi);
    double elo = __dmul_rd(__dmul_rd(k, 1.0 - 1e-12), lo);
    if (P.mode == 1) {
      ehi = fmin(ehi, (double)P.e_hi[r]);
      if (P.e_lo) elo = fmax(elo, (double)P.e_lo[r]);
    }
    if (lane == 0) {
      P.e_hi[r] = __double2float_ru(ehi);
      if (P.e_lo) P.e_lo[r] = __double2float_rd(elo);
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_implicit(const bnb_surface* s1, const bnb_receiver* rec, const bnb_emitters* em,
                            const bnb_cell_bounds* cells, int64_t n, int32_t mode, cudaStream_t st) {
  ImpParams P{};
  P.px = s1->px;
  P.py = s1->py;
  P.pz = s1->pz;
  P.nx = s1->nx;
  P.ny = s1->ny;
  P.nz = s1->nz;
  P.i0 = s1->i0;
  P.i1 = s1->i1;
  P.i2 = s1->i2;
  P.n_verts = s1->n_verts;
  P.n_tris = s1->n_tris;
  P.eta = s1->eta;
  P.ex = em->x;
  P.ey = em->y;
  P.ez = em->z;
  P.ei = em->intensity;
  P.n_emitters = em->n;
  for (int c = 0; c < 3; ++c) {
    P.rp0[c] = rec->p0[c];
    P.re1[c] = rec->e1[c];
    P.re2[c] = rec->e2[c];
  }
  P.emitter = cells->emitter;
  P.tri0 = cells->tri0;
  P.tri1 = cells->tri1;
  P.cell = cells->cell;
  P.flags = cells->flags;
  P.u_lo = cells->u_lo;
  P.u_hi = cells->u_hi;
  P.v_lo = cells->v_lo;
  P.v_hi = cells->v_hi;
  P.e_hi = cells->e_hi;
  P.e_lo = cells->e_lo;
  P.n = n;
  P.count = cells->count;
  P.capacity = cells->capacity;
  P.mode = mode;
  const size_t smem = (size_t)kImpWarps * kImpScratch * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(implicit_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per_sm = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, implicit_k, kImpThreads, smem)) != cudaSuccess)
    return err;
  int64_t blocks = (int64_t)sms * max(per_sm, 1);
  if (n >= 0) blocks = std::min<int64_t>(blocks, (n + kImpWarps - 1) / kImpWarps);
  if (blocks <= 0) return cudaSuccess;
  implicit_k<<<(unsigned)blocks, kImpThreads, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace bnb
