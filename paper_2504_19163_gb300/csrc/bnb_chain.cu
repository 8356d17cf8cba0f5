// Irradiance bound of two-vertex chains (Eq. eq_dwda through both vertices), a post-pass over the
// records of the pair bound pass.
//
// The irradiance of a chain x0 -> x1 (T1) -> x2 (T2) -> receiver is
//     E = I0 |C1| / (|x1 - x0|^3 |N_k| |det du_k/du1|),   C1 = (p10 - x0).N1 constant on T1,
// with u1 T1's barycentric coordinates and u_k the receiver's.  Per record the chain map (unit
// normals, the mirror law or vector Snell at each vertex, ray/plane hits) is evaluated in float32
// interval arithmetic with forward-mode derivatives along T1's two barycentric directions, every
// operation rounded outward (__f*_rd / __f*_ru); the input is the cell's barycentric bounding box,
// and the hit on T2's plane is clipped to T2's closed domain (only chains through T2 count).  Every
// chain of the box then has s = |x1 - x0|^2 and det du_k/du1 in the computed intervals, so when the
// determinant's interval excludes 0
//     E_hi = I0 |C1|_hi / (s_lo^(3/2) |N_k|_lo min|det|),  E_lo = I0 |C1|_lo / (s_hi^(3/2) |N_k|_hi max|det|).
// When the whole box is not certified (a division, square root or the determinant's sign left
// open), its 2 x 2 and then 4 x 4 sub-boxes that meet the cell are tried; the bound is the hull
// over the sub-boxes of the first level where every kept sub-box is certified or meets no chain,
// else E_hi = +inf.  Thread per record; the records' boxes and flags are not changed.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"

namespace bnb {

namespace {

struct If {
  float lo, hi;
};

__device__ __forceinline__ If ic(float a) { return {a, a}; }
__device__ __forceinline__ If iadd(If a, If b) { return {__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi)}; }
__device__ __forceinline__ If isub(If a, If b) { return {__fadd_rd(a.lo, -b.hi), __fadd_ru(a.hi, -b.lo)}; }
__device__ __forceinline__ If imul(If a, If b) {
  const float l = fminf(fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
                        fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)));
  const float h = fmaxf(fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi)),
                        fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi)));
  return {l, h};
}
// a / b; ok = false when b contains 0
__device__ __forceinline__ If idiv(If a, If b, bool& ok) {
  if (!(b.lo > 0.0f || b.hi < 0.0f)) {
    ok = false;
    return {-INFINITY, INFINITY};
  }
  const float l = fminf(fminf(__fdiv_rd(a.lo, b.lo), __fdiv_rd(a.lo, b.hi)),
                        fminf(__fdiv_rd(a.hi, b.lo), __fdiv_rd(a.hi, b.hi)));
  const float h = fmaxf(fmaxf(__fdiv_ru(a.lo, b.lo), __fdiv_ru(a.lo, b.hi)),
                        fmaxf(__fdiv_ru(a.hi, b.lo), __fdiv_ru(a.hi, b.hi)));
  return {l, h};
}
// sqrt of the non-negative part; ok = false when there is none
__device__ __forceinline__ If isqrt(If a, bool& ok) {
  if (!(a.hi >= 0.0f)) {
    ok = false;
    return {0.0f, 0.0f};
  }
  return {__fsqrt_rd(fmaxf(a.lo, 0.0f)), __fsqrt_ru(a.hi)};
}

struct ID {  // interval value and its derivatives along T1's barycentric directions u, v
  If v, d0, d1;
};
__device__ __forceinline__ ID idc(If a) { return {a, ic(0.0f), ic(0.0f)}; }
__device__ __forceinline__ ID operator+(const ID& a, const ID& b) {
  return {iadd(a.v, b.v), iadd(a.d0, b.d0), iadd(a.d1, b.d1)};
}
__device__ __forceinline__ ID operator-(const ID& a, const ID& b) {
  return {isub(a.v, b.v), isub(a.d0, b.d0), isub(a.d1, b.d1)};
}
__device__ __forceinline__ ID operator*(const ID& a, const ID& b) {
  return {imul(a.v, b.v), iadd(imul(a.d0, b.v), imul(a.v, b.d0)), iadd(imul(a.d1, b.v), imul(a.v, b.d1))};
}
__device__ __forceinline__ ID idivd(const ID& a, const ID& b, bool& ok) {
  const If q = idiv(a.v, b.v, ok);
  return {q, idiv(isub(a.d0, imul(q, b.d0)), b.v, ok), idiv(isub(a.d1, imul(q, b.d1)), b.v, ok)};
}
__device__ __forceinline__ ID isqrtd(const ID& a, bool& ok) {
  const If r = isqrt(a.v, ok);
  const If r2 = imul(ic(2.0f), r);
  return {r, idiv(a.d0, r2, ok), idiv(a.d1, r2, ok)};
}

struct IV {
  ID x, y, z;
};
__device__ __forceinline__ IV operator+(const IV& a, const IV& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ IV operator-(const IV& a, const IV& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ IV operator*(const ID& s, const IV& a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ ID idot(const IV& a, const IV& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ IV idivs(const IV& a, const ID& s, bool& ok) {
  return {idivd(a.x, s, ok), idivd(a.y, s, ok), idivd(a.z, s, ok)};
}

// Constant 3-vectors as intervals: a point, or the difference of two points (rounded outward).
struct CV {
  If x, y, z;
};
__device__ __forceinline__ CV cpt(const float (&a)[3]) { return {ic(a[0]), ic(a[1]), ic(a[2])}; }
__device__ __forceinline__ CV cdiff(const float (&a)[3], const float (&b)[3]) {
  return {isub(ic(a[0]), ic(b[0])), isub(ic(a[1]), ic(b[1])), isub(ic(a[2]), ic(b[2]))};
}
__device__ __forceinline__ CV ccross(const CV& a, const CV& b) {
  return {isub(imul(a.y, b.z), imul(a.z, b.y)), isub(imul(a.z, b.x), imul(a.x, b.z)),
          isub(imul(a.x, b.y), imul(a.y, b.x))};
}
__device__ __forceinline__ If cdot(const CV& a, const CV& b) {
  return iadd(iadd(imul(a.x, b.x), imul(a.y, b.y)), imul(a.z, b.z));
}
__device__ __forceinline__ IV iconst(const CV& a) { return {idc(a.x), idc(a.y), idc(a.z)}; }

// Unit normal, then the mirror law (eta < 0) or vector Snell; ok = false when the discriminant's
// range reaches 0 (total internal reflection on part of the box).
__device__ __forceinline__ IV isnell(const IV& ih, const IV& n, float eta, bool& ok) {
  const ID ln = isqrtd(idot(n, n), ok);
  const IV nh = idivs(n, ln, ok);
  if (eta < 0.0f) return ih - (idc(ic(2.0f)) * idot(ih, nh)) * nh;
  const ID c1 = idc(ic(0.0f)) - idot(ih, nh);
  const ID e2 = idc(imul(ic(eta), ic(eta)));
  const ID k = idc(ic(1.0f)) - e2 * (idc(ic(1.0f)) - c1 * c1);
  if (!(k.v.lo > 0.0f)) ok = false;
  return idc(ic(eta)) * ih + (idc(ic(eta)) * c1 - isqrtd(k, ok)) * nh;
}

// rel = U a + V b in the plane of a, b (the dual basis of (a, b))
__device__ __forceinline__ void iplane(const IV& rel, const CV& a, const CV& b, ID& U, ID& V, bool& ok) {
  const If g11 = cdot(a, a), g12 = cdot(a, b), g22 = cdot(b, b);
  const If det = isub(imul(g11, g22), imul(g12, g12));
  const ID pa = idot(rel, iconst(a)), pb = idot(rel, iconst(b));
  U = idivd(idc(g22) * pa - idc(g12) * pb, idc(det), ok);
  V = idivd(idc(g11) * pb - idc(g12) * pa, idc(det), ok);
}

struct ChainCtx {
  float p1[3][3], n1[3][3], p2[3][3], n2[3][3];
  float x0[3];
  float I0;
  float eta1, eta2;  // < 0: a mirror
  float rp0[3], re1[3], re2[3];
};

// One box of T1's barycentric coordinates.  Returns 0 (bounds certified), 1 (no chain of the box
// meets T2's closed domain) or 2 (not certified).
__device__ int chain_box(const ChainCtx& c, If Ub, If Wb, float& elo, float& ehi) {
  bool ok = true;
  const ID U = {Ub, ic(1.0f), ic(0.0f)};
  const ID W = {Wb, ic(0.0f), ic(1.0f)};
  const IV x1 = iconst(cpt(c.p1[0])) + U * iconst(cdiff(c.p1[1], c.p1[0])) + W * iconst(cdiff(c.p1[2], c.p1[0]));
  const IV n1 = iconst(cpt(c.n1[0])) + U * iconst(cdiff(c.n1[1], c.n1[0])) + W * iconst(cdiff(c.n1[2], c.n1[0]));
  const IV d0 = x1 - iconst(cpt(c.x0));
  const ID s0 = idot(d0, d0);
  const IV i1 = idivs(d0, isqrtd(s0, ok), ok);
  const IV r1 = isnell(i1, n1, c.eta1, ok);
  const CV e21 = cdiff(c.p2[1], c.p2[0]), e22 = cdiff(c.p2[2], c.p2[0]);
  const CV N2 = ccross(e21, e22);
  const ID t = idivd(idot(iconst(cpt(c.p2[0])) - x1, iconst(N2)), idot(r1, iconst(N2)), ok);
  const IV x2 = x1 + t * r1;
  ID U2, V2;
  iplane(x2 - iconst(cpt(c.p2[0])), e21, e22, U2, V2, ok);
  if (!ok) return 2;
  // only chains through the closed triangle T2 count: clip the values to its barycentric box
  U2.v = {fmaxf(U2.v.lo, 0.0f), fminf(U2.v.hi, 1.0f)};
  V2.v = {fmaxf(V2.v.lo, 0.0f), fminf(V2.v.hi, 1.0f)};
  if (U2.v.lo > U2.v.hi || V2.v.lo > V2.v.hi || __fadd_rd(U2.v.lo, V2.v.lo) > 1.0f) return 1;
  const IV n2 = iconst(cpt(c.n2[0])) + U2 * iconst(cdiff(c.n2[1], c.n2[0])) + V2 * iconst(cdiff(c.n2[2], c.n2[0]));
  const IV i2 = idivs(r1, isqrtd(idot(r1, r1), ok), ok);
  const IV r2 = isnell(i2, n2, c.eta2, ok);
  const CV E1 = cpt(c.re1), E2 = cpt(c.re2);
  const CV Nk = ccross(E1, E2);
  const ID t2 = idivd(idot(iconst(cpt(c.rp0)) - x2, iconst(Nk)), idot(r2, iconst(Nk)), ok);
  const IV X = x2 + t2 * r2;
  ID Uk, Vk;
  iplane(X - iconst(cpt(c.rp0)), E1, E2, Uk, Vk, ok);
  if (!ok) return 2;
  const If det = isub(imul(Uk.d0, Vk.d1), imul(Uk.d1, Vk.d0));
  if (!(det.lo > 0.0f || det.hi < 0.0f)) return 2;  // a fold may lie in the box
  const float dmin = det.lo > 0.0f ? det.lo : -det.hi, dmax = det.lo > 0.0f ? det.hi : -det.lo;
  const If s = s0.v;
  if (!(s.lo > 0.0f)) return 2;
  // |C1| = |(p10 - x0).N1| and |N_k| as intervals
  const CV a1 = cdiff(c.p1[1], c.p1[0]), b1 = cdiff(c.p1[2], c.p1[0]), r0 = cdiff(c.p1[0], c.x0);
  const If C1 = cdot(r0, ccross(a1, b1));
  const float c1lo = C1.lo > 0.0f ? C1.lo : (C1.hi < 0.0f ? -C1.hi : 0.0f);
  const float c1hi = fmaxf(fabsf(C1.lo), fabsf(C1.hi));
  bool okn = true;
  const If nk = isqrt(cdot(Nk, Nk), okn);
  if (!okn || !(nk.lo > 0.0f)) return 2;
  const float s32lo = __fmul_rd(s.lo, __fsqrt_rd(s.lo)), s32hi = __fmul_ru(s.hi, __fsqrt_ru(s.hi));
  const float den_lo = __fmul_rd(__fmul_rd(s32lo, nk.lo), dmin);
  if (!(den_lo > 0.0f)) return 2;
  ehi = __fdiv_ru(__fmul_ru(c.I0, c1hi), den_lo);
  elo = fmaxf(__fdiv_rd(__fmul_rd(c.I0, c1lo), __fmul_ru(__fmul_ru(s32hi, nk.hi), dmax)), 0.0f);
  return 0;
}

// Whether the box [u0, u1] x [v0, v1] meets the triangle with corners (cu, cv) (separating axes:
// the coordinate axes and the edge normals); a box separated by at most 1e-6 counts as meeting it.
__device__ __forceinline__ bool box_meets_cell(const float (&cu)[3], const float (&cv)[3], float u0, float u1, float v0,
                                               float v1) {
  const float eps = 1e-6f;
  const float mu = fminf(fminf(cu[0], cu[1]), cu[2]), Mu = fmaxf(fmaxf(cu[0], cu[1]), cu[2]);
  const float mv = fminf(fminf(cv[0], cv[1]), cv[2]), Mv = fmaxf(fmaxf(cv[0], cv[1]), cv[2]);
  if (u0 > Mu + eps || u1 < mu - eps || v0 > Mv + eps || v1 < mv - eps) return false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    const float nu = -(cv[k1] - cv[k]), nv = cu[k1] - cu[k];
    const float side = nu * (cu[k2] - cu[k]) + nv * (cv[k2] - cv[k]);
    const float len = sqrtf(nu * nu + nv * nv);
    float mn = INFINITY, mx = -INFINITY;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float pu = (q & 1) ? u1 : u0, pv = (q & 2) ? v1 : v0;
      const float d = nu * (pu - cu[k]) + nv * (pv - cv[k]);
      mn = fminf(mn, d);
      mx = fmaxf(mx, d);
    }
    if (side > 0.0f && mx < -eps * len) return false;
    if (side < 0.0f && mn > eps * len) return false;
  }
  return true;
}

struct ChainParams {
  const float4* ptri1;  // packed triangles of s1 and s2
  const float4* ptri2;
  int32_t n_tris1, n_tris2, n_emitters;
  const float *ex, *ey, *ez, *ei;
  float eta1, eta2;  // < 0: a mirror
  float rp0[3], re1[3], re2[3];
  int32_t depth;
  int64_t capacity;
  const int64_t* count;
  const int32_t *emitter, *tri0, *tri1;
  const uint32_t *cell, *flags;
  float *e_lo, *e_hi;
};

__device__ __forceinline__ void unpack(const float4* __restrict__ tri, int t, float (&p)[3][3], float (&n)[3][3]) {
  const float4* q = tri + (int64_t)t * kTriF4;
  float f[20];
#pragma unroll
  for (int i = 0; i < kTriF4; ++i) {
    const float4 v = __ldg(q + i);
    f[4 * i] = v.x;
    f[4 * i + 1] = v.y;
    f[4 * i + 2] = v.z;
    f[4 * i + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[k][c] = f[3 * k + c];
      n[k][c] = f[9 + 3 * k + c];
    }
}

// Three 128-thread blocks per SM (168 registers): the interval products are chains of dependent
// directed-rounding operations, and twelve warps hide more of their latency than eight at 255.
__global__ void __launch_bounds__(128, 3) chain_irradiance_k(ChainParams P) {
  const int64_t n = min(*P.count, P.capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!(P.flags[i] & BNB_CELL_LIVE)) continue;
    const int e = P.emitter[i], t1 = P.tri0[i], t2 = P.tri1[i];
    if (e < 0 || e >= P.n_emitters || t1 < 0 || t1 >= P.n_tris1 || t2 < 0 || t2 >= P.n_tris2) continue;
    ChainCtx c;
    unpack(P.ptri1, t1, c.p1, c.n1);
    unpack(P.ptri2, t2, c.p2, c.n2);
    c.x0[0] = __ldg(P.ex + e);
    c.x0[1] = __ldg(P.ey + e);
    c.x0[2] = __ldg(P.ez + e);
    c.I0 = __ldg(P.ei + e);
    c.eta1 = P.eta1;
    c.eta2 = P.eta2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      c.rp0[k] = P.rp0[k];
      c.re1[k] = P.re1[k];
      c.re2[k] = P.re2[k];
    }
    // the cell's corners in T1's barycentric coordinates (base-4 path, most significant first)
    float cu[3] = {0.0f, 1.0f, 0.0f}, cv[3] = {0.0f, 0.0f, 1.0f};
    const uint32_t id = P.cell[i];
    for (int l = P.depth - 1; l >= 0; --l) {
      const int ch = (int)((id >> (2 * l)) & 3u);
      const float mu01 = 0.5f * (cu[0] + cu[1]), mv01 = 0.5f * (cv[0] + cv[1]);
      const float mu02 = 0.5f * (cu[0] + cu[2]), mv02 = 0.5f * (cv[0] + cv[2]);
      const float mu12 = 0.5f * (cu[1] + cu[2]), mv12 = 0.5f * (cv[1] + cv[2]);
      float nu[3], nv[3];
      if (ch == 0) {
        nu[0] = cu[0], nv[0] = cv[0], nu[1] = mu01, nv[1] = mv01, nu[2] = mu02, nv[2] = mv02;
      } else if (ch == 1) {
        nu[0] = mu01, nv[0] = mv01, nu[1] = cu[1], nv[1] = cv[1], nu[2] = mu12, nv[2] = mv12;
      } else if (ch == 2) {
        nu[0] = mu02, nv[0] = mv02, nu[1] = mu12, nv[1] = mv12, nu[2] = cu[2], nv[2] = cv[2];
      } else {
        nu[0] = mu12, nv[0] = mv12, nu[1] = mu02, nv[1] = mv02, nu[2] = mu01, nv[2] = mv01;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cu[k] = nu[k];
        cv[k] = nv[k];
      }
    }
    const float u0 = fminf(fminf(cu[0], cu[1]), cu[2]), u1 = fmaxf(fmaxf(cu[0], cu[1]), cu[2]);
    const float v0 = fminf(fminf(cv[0], cv[1]), cv[2]), v1 = fmaxf(fmaxf(cv[0], cv[1]), cv[2]);
    float lo = INFINITY, hi = 0.0f;
    bool certified = false;
    for (int level = 0; level < 3 && !certified; ++level) {
      const int m = 1 << level;
      lo = INFINITY;
      hi = 0.0f;
      certified = true;
      for (int j = 0; j < m && certified; ++j) {
        for (int q = 0; q < m && certified; ++q) {
          // exact: dyadic corners, m a power of two
          const float a0 = u0 + (u1 - u0) * (float)q / (float)m, a1 = u0 + (u1 - u0) * (float)(q + 1) / (float)m;
          const float b0 = v0 + (v1 - v0) * (float)j / (float)m, b1 = v0 + (v1 - v0) * (float)(j + 1) / (float)m;
          if (level > 0 && !box_meets_cell(cu, cv, a0, a1, b0, b1)) continue;
          float l = 0.0f, h = 0.0f;
          const int rc = chain_box(c, If{a0, a1}, If{b0, b1}, l, h);
          if (rc == 2) certified = false;
          if (rc == 0) {
            lo = fminf(lo, l);
            hi = fmaxf(hi, h);
          }
        }
      }
    }
    if (certified) {
      P.e_hi[i] = hi;
      if (P.e_lo) P.e_lo[i] = lo == INFINITY ? 0.0f : lo;
    } else {
      P.e_hi[i] = INFINITY;
      if (P.e_lo) P.e_lo[i] = 0.0f;
    }
  }
}

}  // namespace

cudaError_t launch_chain_irradiance(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                                    const bnb_emitters* em, int32_t depth, const float4* tri1, const float4* tri2,
                                    const bnb_cell_bounds* out, cudaStream_t st) {
  ChainParams P{};
  P.ptri1 = tri1;
  P.ptri2 = tri2;
  P.n_tris1 = s1->n_tris;
  P.n_tris2 = s2->n_tris;
  P.n_emitters = em->n;
  P.ex = em->x;
  P.ey = em->y;
  P.ez = em->z;
  P.ei = em->intensity;
  P.eta1 = s1->kind == BNB_REFLECT ? -1.0f : s1->eta;
  P.eta2 = s2->kind == BNB_REFLECT ? -1.0f : s2->eta;
  for (int k = 0; k < 3; ++k) {
    P.rp0[k] = rec->p0[k];
    P.re1[k] = rec->e1[k];
    P.re2[k] = rec->e2[k];
  }
  P.depth = depth;
  P.capacity = out->capacity;
  P.count = out->count;
  P.emitter = out->emitter;
  P.tri0 = out->tri0;
  P.tri1 = out->tri1;
  P.cell = out->cell;
  P.flags = out->flags;
  P.e_lo = out->e_lo;
  P.e_hi = out->e_hi;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  chain_irradiance_k<<<sms * 8, 128, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace bnb
