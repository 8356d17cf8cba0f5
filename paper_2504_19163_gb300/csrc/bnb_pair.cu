// Two specular vertices: the bound pass of chains x0 -> T1 -> T2 -> receiver, each vertex
// reflecting or refracting (e.g. the TT chains of Table "tab:perf" through a glass slab).
//
//   s2 grid        s2_bbox_k, s2_bin_k, scan, s2_fill_k, s2_sort_k: a uniform grid over the xy box
//                  of s2; every triangle is listed once, in the grid cell of its xy box's lower
//                  corner (cells sorted by triangle index), and a query widens its range by the
//                  largest extent of a triangle box in grid cells.
//   pair_cand_k    per base cell (emitter, T1, cell) (Sec. 6.1 "Tuple construction"): the x1 box
//                  and the ratio bounds of the refracted direction give the xy footprint of the
//                  cell's rays on a z-band; T2 is a candidate when its xy box meets the footprint
//                  for T2's own z-range.  Count pass, scan, then the same search writing
//                  (emitter, tri0 = T1, tri1 = T2, cell) into the output records.
//   pair_bound_k   per record: u2 (Eq. eq_rct with d~1 of Eq. eq_refr_rational, both xi1 faces)
//                  is reduced to its corner interpolant plus a remainder (Sec. 6.1 "Degree
//                  reduction"); the second refraction and the receiver forms are then built from
//                  those degree-1 forms, whose remainder rides in the tracked error E (a sup-norm
//                  bound on the cell, propagated by the same rules as rounding error), and the
//                  ratio bound divides the coefficient intervals.  e_hi = +inf (no irradiance
//                  bound for chains).  Denominator sign tests that float32 cannot decide are
//                  redone in float64 (flag QSIGN_FP64); a certified mixed sign gives the full box
//                  (flag POS_UNBOUNDED; chains are not split).
#include <algorithm>
#include <cmath>

#include "bnb_bound_impl.cuh"

namespace bnb {

struct S2Grid {
  float x0, y0, inv_x, inv_y;  // column of x: floor((x - x0) * inv_x) clamped to [0, G - 1]
  float zlo, zhi;              // z range of s2
  int32_t mx, my;              // largest extent of a triangle's xy box, in grid columns / rows
};

struct PairParams {
  const float4* ptri1;  // packed s1
  const float4* ptri2;  // packed s2
  int32_t n_tris1, n_tris2, n_emitters;
  const float *ex, *ey, *ez;
  float rp0[3], re1[3], re2[3];
  float eta1, eta2;
  int32_t kind1, kind2;  // BNB_REFLECT or BNB_REFRACT per vertex
  int32_t depth;
  int64_t n_base;
  int32_t G;
  S2Grid* grid;
  const int64_t* cell_off;  // G*G + 1
  const int32_t* cell_tri;  // n_tris2
  int64_t* cand_count;      // n_base
  const int64_t* cand_off;  // n_base + 1
  int64_t capacity;
  int64_t* count;
  int32_t* status;
  float *u_lo, *u_hi, *v_lo, *v_hi, *e_lo, *e_hi;
  int32_t *emitter, *tri0, *tri1;
  uint32_t *cell, *flags;
  float* e_hi_min;
};

// ------------------------------------------------------------------ s2 grid
__device__ __forceinline__ int grid_cell_of(float x, float x0, float inv, int G) {
  const float f = (x - x0) * inv;  // monotone in x
  if (!(f > 0.0f)) return 0;
  return (int)fminf(f, (float)(G - 1));
}

__device__ __forceinline__ void tri_box(const float4* tri, int t, float (&lo)[3], float (&hi)[3]) {
  float p[3][3], n[3][3];
  load_tri(tri, t, p, n);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    lo[c] = fminf(p[0][c], fminf(p[1][c], p[2][c]));
    hi[c] = fmaxf(p[0][c], fmaxf(p[1][c], p[2][c]));
  }
}

__global__ void __launch_bounds__(1024) s2_bbox_k(const float4* __restrict__ tri, int n, int G, S2Grid* grid) {
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    float a[3], b[3];
    tri_box(tri, t, a, b);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], a[c]);
      hi[c] = fmaxf(hi[c], b[c]);
    }
  }
  __shared__ float s[6][32];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s[c][wid] = lo[c];
      s[3 + c][wid] = hi[c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        lo[c] = fminf(lo[c], s[c][w]);
        hi[c] = fmaxf(hi[c], s[3 + c][w]);
      }
    }
    S2Grid g;
    g.x0 = lo[0];
    g.y0 = lo[1];
    g.inv_x = hi[0] > lo[0] ? (float)G / (hi[0] - lo[0]) : 0.0f;
    g.inv_y = hi[1] > lo[1] ? (float)G / (hi[1] - lo[1]) : 0.0f;
    g.zlo = lo[2];
    g.zhi = hi[2];
    g.mx = 0;
    g.my = 0;
    *grid = g;
  }
}

__global__ void s2_bin_k(const float4* __restrict__ tri, int n, int G, S2Grid* grid, int32_t* __restrict__ tri_cell,
                         int64_t* __restrict__ cell_count) {
  const S2Grid g = *grid;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    float a[3], b[3];
    tri_box(tri, t, a, b);
    const int ix0 = grid_cell_of(a[0], g.x0, g.inv_x, G), ix1 = grid_cell_of(b[0], g.x0, g.inv_x, G);
    const int iy0 = grid_cell_of(a[1], g.y0, g.inv_y, G), iy1 = grid_cell_of(b[1], g.y0, g.inv_y, G);
    const int cell = iy0 * G + ix0;
    tri_cell[t] = cell;
    atomicAdd((unsigned long long*)(cell_count + cell), 1ull);
    atomicMax(&grid->mx, ix1 - ix0);
    atomicMax(&grid->my, iy1 - iy0);
  }
}

__global__ void s2_fill_k(int n, const int32_t* __restrict__ tri_cell, const int64_t* __restrict__ cell_off,
                          int64_t* __restrict__ cursor, int32_t* __restrict__ cell_tri) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int c = tri_cell[t];
    const int64_t k = (int64_t)atomicAdd((unsigned long long*)(cursor + c), 1ull);
    cell_tri[cell_off[c] + k] = t;
  }
}

// Each grid cell's list in ascending triangle order (insertion sort; lists are short).
__global__ void s2_sort_k(int cells, const int64_t* __restrict__ cell_off, int32_t* __restrict__ cell_tri) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
    const int64_t a = cell_off[c], b = cell_off[c + 1];
    for (int64_t i = a + 1; i < b; ++i) {
      const int32_t v = cell_tri[i];
      int64_t j = i - 1;
      while (j >= a && cell_tri[j] > v) {
        cell_tri[j + 1] = cell_tri[j];
        --j;
      }
      cell_tri[j + 1] = v;
    }
  }
}

// ------------------------------------------------------------------ vertex faces
// The scattered direction at a vertex from degree-1 forms n and d (tracked errors may hold
// remainders), on the two faces of a remainder variable: refraction (Eq. eq_refr_rational)
// d~ = eta' ((n.n) d - (d.n) n) - r~(beta) n with sqrt(beta)'s remainder (Sec. 4.3); reflection
// d~ = (n.n) d - 2 (d.n) n on both faces (no remainder).  Returns false when beta <= 0 on the whole
// cell (total internal reflection).
template <typename T>
__device__ __forceinline__ bool vertex_faces(const TP<T, 1> (&N)[3], const TP<T, 1> (&D)[3], int kind, T eta,
                                             TP<T, 5> (&DT)[2][3]) {
  using F = FP<T>;
  if (kind == BNB_REFLECT) {
    TP<T, 2> NN, DN2;
    tp_zero(NN);
    tp_zero(DN2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(NN, N[c], N[c]);
      mac(DN2, D[c], N[c]);
    }
    renorm(NN);
    renorm(DN2);
    scale2(DN2);  // 2 (d.n), exact
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      TP<T, 3> r;
      tp_zero(r);
      mac(r, NN, D[c]);
      mac<true>(r, DN2, N[c]);
      TP<T, 4> r4;
      elevate(r4, r);
      elevate(DT[0][c], r4);
      renorm(DT[0][c]);
      DT[1][c] = DT[0][c];
    }
    return true;
  }
  TP<T, 2> NN, DN, SS;
  tp_zero(NN);
  tp_zero(DN);
  tp_zero(SS);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mac(NN, N[c], N[c]);
    mac(DN, D[c], N[c]);
    mac(SS, D[c], D[c]);
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
  if (!(bhi > T(0))) return false;
  T ca, cb, dlo, dhi;
  sqrt_chord<T>(fmax(blo, T(0)), bhi, ca, cb, dlo, dhi);
  TP<T, 5> TG5[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    TP<T, 3> tg, tg3;
    tp_zero(tg);
    mac(tg, NN, D[c]);
    mac<true>(tg, DN, N[c]);
    tp_zero(tg3);
    mac_s(tg3, eta, tg);
    TP<T, 4> t4;
    elevate(t4, tg3);
    elevate(TG5[c], t4);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    TP<T, 4> Wj;
    tp_zero(Wj);
    mac_s(Wj, ca, beta);
    const T cj = cb + (j == 0 ? dlo : dhi);
    add_const(Wj, cj, F::mul_ru((T)FP<T>::u, fabs(cj)));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      DT[j][c] = TG5[c];
      mac<true>(DT[j][c], Wj, N[c]);
      renorm(DT[j][c]);
    }
  }
  return true;
}

template <typename T>
__device__ __forceinline__ TP<T, 0> diff_const(T a, T b) {  // a - b with its rounding error
  const T v = a - b;
  return tconst<T>(v, FP<T>::mul_ru((T)FP<T>::u, fabs(v)));
}

// The first vertex of a cell of T1: leaves (x1 = p0 + XL, n1, d0) and the refracted faces.
template <typename T>
__device__ __forceinline__ bool first_vertex(const PairParams& P, int e, int t1, uint32_t id, T (&p)[3][3],
                                             Leaves<T>& L, TP<T, 5> (&DT)[2][3], T (&cu)[3], T (&cv)[3]) {
  float pf[3][3], nf[3][3];
  load_tri(P.ptri1, t1, pf, nf);
  T n[3][3], x0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      p[a][b] = (T)pf[a][b];
      n[a][b] = (T)nf[a][b];
    }
  }
  x0[0] = (T)__ldg(P.ex + e);
  x0[1] = (T)__ldg(P.ey + e);
  x0[2] = (T)__ldg(P.ez + e);
  cell_corners<T>(id, P.depth, cu, cv);
  make_leaves<T, false>(p, n, x0, cu, cv, L);
  return vertex_faces<T>(L.N, L.D0, P.kind1, (T)P.eta1, DT);
}

// Ratio bound [lo, hi] of num/den over both faces (den's certified sign sq; degrees 5 and 5).
template <typename T, int N>
__device__ __forceinline__ void face_ratio(const TP<T, N> (&num)[2], const TP<T, N> (&den)[2], int sq, T& lo, T& hi) {
  using F = FP<T>;
  T mn = F::inf(), mx = -F::inf();
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    static_for<nc(N)>([&](auto I) {
      constexpr int i = decltype(I)::value;
      T ql, qh, al, ah;
      coef_iv<i>(den[j], ql, qh);
      coef_iv<i>(num[j], al, ah);
      if (sq < 0) {
        T t = ql;
        ql = -qh;
        qh = -t;
        t = al;
        al = -ah;
        ah = -t;
      }
      const bool open = !(ql > tiny_pos<T>());
      const T rl = open ? F::inf() : rcp_hi(ql), rh = rcp_lo(qh);
      ratio_acc(al, ah, rl, rh, mn, mx);
      if (open) {
        if (al == T(0)) mn = fmin(mn, T(0));
        if (ah == T(0)) mx = fmax(mx, T(0));
      }
    });
  }
  lo = widen_lo(mn);
  hi = widen_hi(mx);
}

// ------------------------------------------------------------------ candidates
// The cell's ray bundle: kind 0 no refracted ray, 1 bounded, 2 the sign of d~z is not certified.
struct Bundle {
  int kind, sz;
  float x[2], y[2], z[2], rx[2], ry[2];
};

__device__ __forceinline__ Bundle bundle_of(const PairParams& P, int e, int t1, uint32_t id) {
  using F = FP<float>;
  Bundle B{};
  float p[3][3], cu[3], cv[3];
  Leaves<float> L;
  TP<float, 5> DT[2][3];
  if (!first_vertex<float>(P, e, t1, id, p, L, DT, cu, cv)) return B;
  const int s0 = cert_sign(DT[0][2]), s1 = cert_sign(DT[1][2]);
  if (s0 == 0 || s0 != s1) {
    B.kind = 2;
    return B;
  }
  B.kind = 1;
  B.sz = s0;
  TP<float, 5> dx[2] = {DT[0][0], DT[1][0]}, dy[2] = {DT[0][1], DT[1][1]}, dz[2] = {DT[0][2], DT[1][2]};
  face_ratio<float, 5>(dx, dz, s0, B.rx[0], B.rx[1]);
  face_ratio<float, 5>(dy, dz, s0, B.ry[0], B.ry[1]);
  float* box[3] = {B.x, B.y, B.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float lo = F::inf(), hi = -F::inf();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = L.XL[c].c[corner_idx(k)];
      lo = fminf(lo, F::add_rd(p[0][c], F::add_rd(v, -L.XL[c].E)));
      hi = fmaxf(hi, F::add_ru(p[0][c], F::add_ru(v, L.XL[c].E)));
    }
    box[c][0] = lo;
    box[c][1] = hi;
  }
  return B;
}

// Footprint {xlo, xhi, ylo, yhi} of a bounded bundle on the band [zlo, zhi] (outward rounding);
// false when no forward ray reaches the band.
__device__ __forceinline__ bool footprint(const Bundle& B, float zlo, float zhi, float (&f)[4]) {
  using F = FP<float>;
  float dzl = F::add_rd(zlo, -B.z[1]), dzh = F::add_ru(zhi, -B.z[0]);
  if (B.sz < 0)
    dzh = fminf(dzh, 0.0f);
  else
    dzl = fmaxf(dzl, 0.0f);
  if (!(dzl <= dzh)) return false;
  auto span = [&](const float (&x)[2], const float (&r)[2], float& ol, float& oh) {
    const float l = fminf(fminf(F::mul_rd(dzl, r[0]), F::mul_rd(dzl, r[1])),
                          fminf(F::mul_rd(dzh, r[0]), F::mul_rd(dzh, r[1])));
    const float h = fmaxf(fmaxf(F::mul_ru(dzl, r[0]), F::mul_ru(dzl, r[1])),
                          fmaxf(F::mul_ru(dzh, r[0]), F::mul_ru(dzh, r[1])));
    ol = F::add_rd(x[0], l);
    oh = F::add_ru(x[1], h);
  };
  span(B.x, B.rx, f[0], f[1]);
  span(B.y, B.ry, f[2], f[3]);
  return true;
}

template <bool FILL>
__global__ void __launch_bounds__(128) pair_cand_k(PairParams P) {
  const int64_t per_tuple = (int64_t)1 << (2 * P.depth);
  const int64_t per_em = per_tuple * P.n_tris1;
  const S2Grid g = *P.grid;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < P.n_base;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(w / per_em);
    const int64_t rr = w - (int64_t)e * per_em;
    const int t1 = (int)(rr / per_tuple);
    const uint32_t id = (uint32_t)(rr - (int64_t)t1 * per_tuple);
    const Bundle B = bundle_of(P, e, t1, id);
    int64_t n = 0;
    int64_t slot = FILL ? P.cand_off[w] : 0;
    auto emit = [&](int t2) {
      if (FILL) {
        if (slot < P.capacity) {
          P.emitter[slot] = e;
          P.tri0[slot] = t1;
          P.tri1[slot] = t2;
          P.cell[slot] = id;
          P.flags[slot] = (uint32_t)P.depth << BNB_CELL_DEPTH_SHIFT;
        }
        ++slot;
      }
      ++n;
    };
    float f[4];
    bool all = B.kind == 2;
    bool any = B.kind != 0;
    if (B.kind == 1) {
      any = footprint(B, g.zlo, g.zhi, f);
      if (any && !(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]) && isfinite(f[3]))) all = true;
    }
    if (all) {
      for (int t2 = 0; t2 < P.n_tris2; ++t2) emit(t2);
    } else if (any) {
      const int qx0 = grid_cell_of(f[0], g.x0, g.inv_x, P.G), qx1 = grid_cell_of(f[1], g.x0, g.inv_x, P.G);
      const int qy0 = grid_cell_of(f[2], g.y0, g.inv_y, P.G), qy1 = grid_cell_of(f[3], g.y0, g.inv_y, P.G);
      for (int iy = max(0, qy0 - g.my); iy <= qy1; ++iy) {
        for (int ix = max(0, qx0 - g.mx); ix <= qx1; ++ix) {
          const int64_t a = P.cell_off[iy * P.G + ix], b = P.cell_off[iy * P.G + ix + 1];
          for (int64_t k = a; k < b; ++k) {
            const int t2 = P.cell_tri[k];
            float lo[3], hi[3], ft[4];
            tri_box(P.ptri2, t2, lo, hi);
            if (!footprint(B, lo[2], hi[2], ft)) continue;
            if (lo[0] <= ft[1] && ft[0] <= hi[0] && lo[1] <= ft[3] && ft[2] <= hi[1]) emit(t2);
          }
        }
      }
    }
    if (!FILL) P.cand_count[w] = n;
  }
}

__global__ void pair_total_k(const int64_t* __restrict__ cand_off, int64_t n_base, int64_t capacity,
                             int64_t* __restrict__ count, int32_t* __restrict__ status) {
  const int64_t total = cand_off[n_base];
  *count = total;
  if (total > capacity) raise_status(status, BNB_ERR_CAPACITY);
}

// ------------------------------------------------------------------ composite bound
__device__ __forceinline__ void put_pair(const PairParams& P, int64_t slot, float ul, float uh, float vl, float vh,
                                         uint32_t flags) {
  P.u_lo[slot] = ul;
  P.u_hi[slot] = uh;
  P.v_lo[slot] = vl;
  P.v_hi[slot] = vh;
  if (P.e_lo) P.e_lo[slot] = 0.0f;
  P.e_hi[slot] = (flags & BNB_CELL_LIVE) ? __int_as_float(0x7f800000) : 0.0f;
  if (P.e_hi_min) P.e_hi_min[slot] = 0.0f;
  P.flags[slot] = flags;
}

// Receiver coordinates of the chain through the cell centroid (un-normalized forms, exact square
// roots, no containment test), rounded to 2^-16; per coordinate 0.5 where the chain has no
// scattered path (total internal reflection) or the coordinate is not below 4 in magnitude.  The expansion point of the second
// vertex's receiver forms (any point is valid).
template <typename T>
__device__ __forceinline__ void centroid_hit(const PairParams& P, const T (&p)[3][3], const float (&nf1)[3][3],
                                             const float (&pf2)[3][3], const float (&nf2)[3][3], const T (&x0)[3],
                                             const T (&cu)[3], const T (&cv)[3], T& uc, T& vc) {
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
      for (int c = 0; c < 3; ++c) out[c] = nn * d[c] - T(2) * dn * n[c];
      return true;
    }
    const T beta = (T(1) - eta * eta) * nn * ss + eta * eta * dn * dn;
    if (!(beta > T(0))) return false;
    const T W = sqrt(beta);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = eta * (nn * d[c] - dn * n[c]) - W * n[c];
    return true;
  };
  auto plane = [&](const T* x, const T* d, const T* o, const T* e1, const T* e2, T& a, T& b) {
    T w[3], g[3], h1[3], h2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = x[c] - o[c];
    cross(e2, e1, g);
    cross(e2, w, h1);
    cross(w, e1, h2);
    const T q = dot(d, g);
    a = dot(d, h1) / q;
    b = dot(h2, d) / q;
  };
  const T third = T(1) / T(3);
  const T w1 = (cu[0] + cu[1] + cu[2]) * third, w2 = (cv[0] + cv[1] + cv[2]) * third, w0 = T(1) - w1 - w2;
  T x1[3], n1[3], d0[3], t1[3], o2[3], e21[3], e22[3], x2[3], n2[3], d1[3], t2[3], R0[3], R1[3], R2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x1[c] = w0 * p[0][c] + w1 * p[1][c] + w2 * p[2][c];
    n1[c] = w0 * (T)nf1[0][c] + w1 * (T)nf1[1][c] + w2 * (T)nf1[2][c];
    d0[c] = x1[c] - x0[c];
    o2[c] = (T)pf2[0][c];
    e21[c] = (T)pf2[1][c] - o2[c];
    e22[c] = (T)pf2[2][c] - o2[c];
    R0[c] = (T)P.rp0[c];
    R1[c] = (T)P.re1[c];
    R2[c] = (T)P.re2[c];
  }
  T a = T(0.5), b = T(0.5);
  if (refract(n1, d0, P.kind1, (T)P.eta1, t1)) {
    T u2, v2;
    plane(x1, t1, o2, e21, e22, u2, v2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x2[c] = o2[c] + u2 * e21[c] + v2 * e22[c];
      n2[c] = (T)nf2[0][c] + u2 * ((T)nf2[1][c] - (T)nf2[0][c]) + v2 * ((T)nf2[2][c] - (T)nf2[0][c]);
      d1[c] = x2[c] - x1[c];
    }
    if (refract(n2, d1, P.kind2, (T)P.eta2, t2)) plane(x2, t2, R0, R1, R2, a, b);
  }
  if (!(fabs(a) < T(4))) a = T(0.5);
  if (!(fabs(b) < T(4))) b = T(0.5);
  uc = rint(a * T(65536)) * T(1.0 / 65536);
  vc = rint(b * T(65536)) * T(1.0 / 65536);
}

// Bound of record `slot`.  Returns false (nothing written) when a float32 sign test is undecided.
template <typename T>
__device__ __forceinline__ bool process_pair(const PairParams& P, int64_t slot, uint32_t extra_flags) {
  using F = FP<T>;
  const int e = P.emitter[slot], t1 = P.tri0[slot], t2 = P.tri1[slot];
  const uint32_t id = P.cell[slot];
  const uint32_t flags = ((uint32_t)P.depth << BNB_CELL_DEPTH_SHIFT) | extra_flags;
  T p[3][3], cu[3], cv[3];
  Leaves<T> L;
  TP<T, 5> DT[2][3];
  if (!first_vertex<T>(P, e, t1, id, p, L, DT, cu, cv)) {
    put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_TIR);
    return true;
  }
  float pf2[3][3], nf2[3][3];
  load_tri(P.ptri2, t2, pf2, nf2);
  // u2 on T2's plane (Eq. eq_rct), both xi1 faces; T2's edges are rounded differences (tracked)
  TP<T, 0> E21[3], E22[3], G2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    E21[c] = diff_const<T>((T)pf2[1][c], (T)pf2[0][c]);
    E22[c] = diff_const<T>((T)pf2[2][c], (T)pf2[0][c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    tp_zero(G2[c]);
    mac(G2[c], E22[a], E21[b]);
    mac<true>(G2[c], E22[b], E21[a]);
  }
  TP<T, 1> hu2[3], hv2[3];
  {
    TP<T, 1> W2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T q = p[0][c] - (T)pf2[0][c];
      W2[c] = L.XL[c];
      add_const(W2[c], q, F::mul_ru((T)FP<T>::u, fabs(q)));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      tp_zero(hu2[c]);
      mac(hu2[c], E22[a], W2[b]);
      mac<true>(hu2[c], E22[b], W2[a]);
      tp_zero(hv2[c]);
      mac(hv2[c], E21[b], W2[a]);
      mac<true>(hv2[c], E21[a], W2[b]);
    }
  }
  TP<T, 5> Q2[2];
  TP<T, 6> A2[2], B2[2], Q6[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    tp_zero(Q2[j]);
    tp_zero(A2[j]);
    tp_zero(B2[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(Q2[j], G2[c], DT[j][c]);
      mac(A2[j], DT[j][c], hu2[c]);
      mac(B2[j], DT[j][c], hv2[c]);
    }
    renorm(Q2[j]);
    renorm(A2[j]);
    renorm(B2[j]);
    elevate(Q6[j], Q2[j]);
  }
  const int s0 = cert_sign(Q2[0]), s1 = cert_sign(Q2[1]);
  if constexpr (sizeof(T) == 4) {
    if (s0 == 0 || s1 == 0) return false;
  }
  const int sq = s0 == s1 ? s0 : 0;
  if (sq == 0) {
    put_pair(P, slot, 0.f, 1.f, 0.f, 1.f, flags | BNB_CELL_LIVE | BNB_CELL_POS_UNBOUNDED);
    return true;
  }
  {  // forward: t = ((x1 - p20) x e21) . e22 / Q2
    TP<T, 1> Tn;
    tp_zero(Tn);
#pragma unroll
    for (int c = 0; c < 3; ++c) mac(Tn, E22[c], hv2[c]);
    if (cert_sign(Tn) * sq < 0) {
      put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_CULL_BEHIND);
      return true;
    }
  }
  T u2l, u2h, v2l, v2h;
  face_ratio<T, 6>(A2, Q6, sq, u2l, u2h);
  face_ratio<T, 6>(B2, Q6, sq, v2l, v2h);
  if (u2h < T(0) || v2h < T(0) || F::add_rd(u2l, v2l) > T(1)) {  // no ray of the cell meets T2
    put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_CULL_EMPTY);
    return true;
  }
  // degree reduction: corner interpolant l at xi1 = 1/2 plus the ratio bound of (P2 - l Q2) / Q2
  TP<T, 1> U2, V2;
  {
    constexpr int k6[3] = {0, idx_of(6, 6, 0), idx_of(6, 0, 6)};
    T lu[3], lv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T q = Q6[0].c[k6[k]] + Q6[1].c[k6[k]];
      lu[k] = (A2[0].c[k6[k]] + A2[1].c[k6[k]]) / q;
      lv[k] = (B2[0].c[k6[k]] + B2[1].c[k6[k]]) / q;
    }
    auto reduce = [&](const T (&l)[3], const TP<T, 6> (&Num)[2], TP<T, 1>& out) {
      TP<T, 1> Lf;
      T lm = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Lf.c[corner_idx(k)] = l[k];
        lm = fmax(lm, fabs(l[k]));
      }
      Lf.B = lm;
      Lf.E = T(0);
      TP<T, 6> R[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        R[j] = Num[j];
        mac<true>(R[j], Lf, Q2[j]);
        renorm(R[j]);
      }
      T rl, rh;
      face_ratio<T, 6>(R, Q6, sq, rl, rh);
      const T mid = (rl + rh) * T(0.5);
      const T rad = fmax(F::add_ru(rh, -mid), F::add_ru(mid, -rl));
      T cm = T(0), em = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        out.c[corner_idx(k)] = l[k] + mid;
        cm = fmax(cm, fabs(out.c[corner_idx(k)]));
        em = fmax(em, F::add_ru(fabs(l[k]), fabs(mid)));
      }
      out.E = F::add_ru(rad, F::mul_ru((T)FP<T>::u, em));
      out.B = F::add_ru(cm, out.E);
    };
    reduce(lu, A2, U2);
    reduce(lv, B2, V2);
  }
  // second vertex: x2 = p20 + U2 e21 + V2 e22, n2 = n20 + U2 f21 + V2 f22, d1 = x2 - x1
  TP<T, 1> X2[3], N2[3], D1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const TP<T, 0> F21 = diff_const<T>((T)nf2[1][c], (T)nf2[0][c]), F22 = diff_const<T>((T)nf2[2][c], (T)nf2[0][c]);
    tp_zero(X2[c]);
    mac(X2[c], E21[c], U2);
    mac(X2[c], E22[c], V2);
    add_const(X2[c], (T)pf2[0][c], T(0));
    renorm(X2[c]);
    tp_zero(N2[c]);
    mac(N2[c], F21, U2);
    mac(N2[c], F22, V2);
    add_const(N2[c], (T)nf2[0][c], T(0));
    renorm(N2[c]);
    D1[c] = X2[c];
    add_const(D1[c], -p[0][c], T(0));
    mac_s<true>(D1[c], T(1), L.XL[c]);
    renorm(D1[c]);
  }
  TP<T, 5> DT2[2][3];
  if (!vertex_faces<T>(N2, D1, P.kind2, (T)P.eta2, DT2)) {
    put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_TIR);
    return true;
  }
  // receiver forms around the chain through the cell centroid
  T uc, vc;
  {
    float nf1[3][3], pf1[3][3];
    load_tri(P.ptri1, t1, pf1, nf1);
    const T x0[3] = {(T)__ldg(P.ex + e), (T)__ldg(P.ey + e), (T)__ldg(P.ez + e)};
    centroid_hit<T>(P, p, nf1, pf2, nf2, x0, cu, cv, uc, vc);
  }
  T e1[3], e2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    e1[c] = (T)P.re1[c];
    e2[c] = (T)P.re2[c];
  }
  TP<T, 1> hu[3], hv[3];
  {
    constexpr T g2e = GAM<T, 2>;
    TP<T, 1> W3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T pc = F::fma_rn(vc, e2[c], F::fma_rn(uc, e1[c], (T)P.rp0[c]));
      const T pmag = F::fma_ru(fabs(vc), fabs(e2[c]), F::fma_ru(fabs(uc), fabs(e1[c]), fabs((T)P.rp0[c])));
      W3[c] = X2[c];
      add_const(W3[c], -pc, F::mul_ru(g2e, pmag));
      renorm(W3[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      tp_zero(hu[c]);
      mac_s(hu[c], e2[a], W3[b]);
      mac_s<true>(hu[c], e2[b], W3[a]);
      tp_zero(hv[c]);
      mac_s(hv[c], e1[b], W3[a]);
      mac_s<true>(hv[c], e1[a], W3[b]);
      renorm(hu[c]);  // the remainder's growth in the products below scales with these bounds
      renorm(hv[c]);
    }
  }
  const TP<T, 0> g[3] = {cross_comp<T>(e2[1], e1[2], e2[2], e1[1]), cross_comp<T>(e2[2], e1[0], e2[0], e1[2]),
                         cross_comp<T>(e2[0], e1[1], e2[1], e1[0])};
  TP<T, 5> Q3[2];
  TP<T, 6> A3[2], B3[2], Q36[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    tp_zero(Q3[j]);
    tp_zero(A3[j]);
    tp_zero(B3[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mac(Q3[j], g[c], DT2[j][c]);
      mac(A3[j], DT2[j][c], hu[c]);
      mac(B3[j], DT2[j][c], hv[c]);
    }
    renorm(Q3[j]);
    renorm(A3[j]);
    renorm(B3[j]);
    elevate(Q36[j], Q3[j]);
  }
  const int m0 = cert_sign(Q3[0]), m1 = cert_sign(Q3[1]);
  if constexpr (sizeof(T) == 4) {
    if (m0 == 0 || m1 == 0) return false;
  }
  const int sq3 = m0 == m1 ? m0 : 0;
  if (sq3 == 0) {
    put_pair(P, slot, 0.f, 1.f, 0.f, 1.f, flags | BNB_CELL_LIVE | BNB_CELL_POS_UNBOUNDED);
    return true;
  }
  {  // forward: t = h_v . e2 / Q3
    TP<T, 1> Tn;
    tp_zero(Tn);
#pragma unroll
    for (int c = 0; c < 3; ++c) mac_s(Tn, e2[c], hv[c]);
    if (cert_sign(Tn) * sq3 < 0) {
      put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_CULL_BEHIND);
      return true;
    }
  }
  T ul, uh, vl, vh;
  face_ratio<T, 6>(A3, Q36, sq3, ul, uh);
  face_ratio<T, 6>(B3, Q36, sq3, vl, vh);
  ul = fmax(F::add_rd(uc, ul), T(0));
  uh = fmin(F::add_ru(uc, uh), T(1));
  vl = fmax(F::add_rd(vc, vl), T(0));
  vh = fmin(F::add_ru(vc, vh), T(1));
  if (!(ul <= uh) || !(vl <= vh)) {
    put_pair(P, slot, 0.f, 0.f, 0.f, 0.f, flags | BNB_CELL_CULL_EMPTY);
    return true;
  }
  put_pair(P, slot, f_dn(ul), f_up(uh), f_dn(vl), f_up(vh), flags | BNB_CELL_LIVE);
  return true;
}

static __device__ __noinline__ void process_pair_fp64(const PairParams& P, int64_t slot) {
  process_pair<double>(P, slot, BNB_CELL_QSIGN_FP64);
}

// Persistent: the blocks resident on the GPU step through the records in rounds with a block
// barrier per round, so the warps of a block walk the long record program together and share its
// instruction fetches.  Three 128-thread blocks per SM (<= 170 registers, ~3 KB of spills) ran the
// slab48 bound stage in 0.600 ms against 0.688 ms with two (255 registers) and 0.733 ms with four.
constexpr int kPairThreads = 128;

template <bool FP64>
__global__ void __launch_bounds__(kPairThreads, 3) pair_bound_k(PairParams P) {
  const int64_t n = min(*P.count, P.capacity);
  const int64_t stride = (int64_t)gridDim.x * kPairThreads;
  const int64_t rounds = (n + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    __syncthreads();
    const int64_t i = r * stride + (int64_t)blockIdx.x * kPairThreads + threadIdx.x;
    if (i >= n) continue;
    if constexpr (FP64) {
      process_pair<double>(P, i, 0u);
    } else {
      if (!process_pair<float>(P, i, 0u)) process_pair_fp64(P, i);
    }
  }
}

// ------------------------------------------------------------------ host side
int32_t pair_grid_res(int32_t n_tris2) {
  int g = (int)sqrt((double)n_tris2 / 2.0);
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

struct PairWs {
  float4* tri1;
  float4* tri2;
  S2Grid* grid;
  int32_t* tri_cell;
  int64_t* cell_count;  // G*G, zeroed
  int64_t* cursor;      // G*G, zeroed
  int64_t* cell_off;    // G*G + 1
  int32_t* cell_tri;
  int64_t* cand_count;  // n_base
  int64_t* cand_off;    // n_base + 1
  void* scan;
  size_t bytes;
};

static PairWs carve_pair_ws(void* base, int64_t n_tris1, int64_t n_tris2, int64_t n_base) {
  PairWs w{};
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  const int64_t G = pair_grid_res((int32_t)n_tris2), cells = G * G;
  w.tri1 = (float4*)take((size_t)n_tris1 * kTriF4 * sizeof(float4));
  w.tri2 = (float4*)take((size_t)n_tris2 * kTriF4 * sizeof(float4));
  w.grid = (S2Grid*)take(sizeof(S2Grid));
  w.tri_cell = (int32_t*)take((size_t)n_tris2 * 4);
  w.cell_count = (int64_t*)take((size_t)cells * 8);
  w.cursor = (int64_t*)take((size_t)cells * 8);
  w.cell_off = (int64_t*)take((size_t)(cells + 1) * 8);
  w.cell_tri = (int32_t*)take((size_t)n_tris2 * 4);
  w.cand_count = (int64_t*)take((size_t)n_base * 8);
  w.cand_off = (int64_t*)take((size_t)(n_base + 1) * 8);
  w.scan = take(std::max(scan_ws_bytes(n_base), scan_ws_bytes(cells)));
  w.bytes = o;
  return w;
}

size_t pair_ws_bytes(int64_t n_tris1, int64_t n_tris2, int64_t n_base) {
  return carve_pair_ws(nullptr, n_tris1, n_tris2, n_base).bytes;
}

cudaError_t launch_chain_irradiance(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                                    const bnb_emitters* em, int32_t depth, const float4* tri1, const float4* tri2,
                                    const bnb_cell_bounds* out, cudaStream_t st);  // bnb_chain.cu

cudaError_t launch_bound_pairs(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                               const bnb_emitters* em, int32_t depth, bool fp64, bool irradiance, bnb_cell_bounds* out,
                               void* ws, cudaStream_t st) {
  const int64_t n_base = (int64_t)em->n * s1->n_tris * ((int64_t)1 << (2 * depth));
  PairWs w = carve_pair_ws(ws, s1->n_tris, s2->n_tris, n_base);
  const int G = pair_grid_res(s2->n_tris);
  const int64_t cells = (int64_t)G * G;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if ((e = cudaMemsetAsync(out->count, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
  if (n_base == 0 || s2->n_tris == 0) return cudaSuccess;
  if ((e = launch_pack_tris(s1, w.tri1, st)) != cudaSuccess) return e;
  if ((e = launch_pack_tris(s2, w.tri2, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.cell_count, 0, (size_t)((char*)w.cell_off - (char*)w.cell_count), st)) != cudaSuccess)
    return e;
  const int n2 = s2->n_tris;
  const int b2 = (int)std::min<int64_t>((n2 + 255) / 256, (int64_t)sms * 8);
  s2_bbox_k<<<1, 1024, 0, st>>>(w.tri2, n2, G, w.grid);
  s2_bin_k<<<b2, 256, 0, st>>>(w.tri2, n2, G, w.grid, w.tri_cell, w.cell_count);
  if ((e = launch_exclusive_scan(w.cell_count, w.cell_off, cells, w.scan, st)) != cudaSuccess) return e;
  s2_fill_k<<<b2, 256, 0, st>>>(n2, w.tri_cell, w.cell_off, w.cursor, w.cell_tri);
  s2_sort_k<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>((int)cells, w.cell_off, w.cell_tri);
  PairParams P{};
  P.ptri1 = w.tri1;
  P.ptri2 = w.tri2;
  P.n_tris1 = s1->n_tris;
  P.n_tris2 = n2;
  P.n_emitters = em->n;
  P.ex = em->x;
  P.ey = em->y;
  P.ez = em->z;
  for (int c = 0; c < 3; ++c) {
    P.rp0[c] = rec->p0[c];
    P.re1[c] = rec->e1[c];
    P.re2[c] = rec->e2[c];
  }
  P.eta1 = s1->eta;
  P.eta2 = s2->eta;
  P.kind1 = s1->kind;
  P.kind2 = s2->kind;
  P.depth = depth;
  P.n_base = n_base;
  P.G = G;
  P.grid = w.grid;
  P.cell_off = w.cell_off;
  P.cell_tri = w.cell_tri;
  P.cand_count = w.cand_count;
  P.cand_off = w.cand_off;
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
  const int cb = (int)std::min<int64_t>((n_base + 127) / 128, (int64_t)sms * 16);
  pair_cand_k<false><<<cb, 128, 0, st>>>(P);
  if ((e = launch_exclusive_scan(w.cand_count, w.cand_off, n_base, w.scan, st)) != cudaSuccess) return e;
  pair_cand_k<true><<<cb, 128, 0, st>>>(P);
  pair_total_k<<<1, 1, 0, st>>>(w.cand_off, n_base, out->capacity, out->count, out->status);
  int per_sm = 1;  // resident blocks per SM of the record kernel
  if (fp64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_bound_k<true>, kPairThreads, 0);
    pair_bound_k<true><<<sms * std::max(1, per_sm), kPairThreads, 0, st>>>(P);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_bound_k<false>, kPairThreads, 0);
    pair_bound_k<false><<<sms * std::max(1, per_sm), kPairThreads, 0, st>>>(P);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // chain irradiance bounds of the live records (a post-pass; otherwise e_hi stays +inf)
  if (irradiance) return launch_chain_irradiance(s1, s2, rec, em, depth, w.tri1, w.tri2, out, st);
  return cudaSuccess;
}

}  // namespace bnb
