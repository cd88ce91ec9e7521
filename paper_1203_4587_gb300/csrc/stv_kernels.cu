// Algorithm 2 with a spatio-temporal analysis operator
//   R x = (D_t x, w D_x x, w D_y x)
// (non-circular differences along t, the horizontal index i and the vertical
// index j) and an m-update by conjugate gradients, as Section IV-B suggests
// when (mu2/mu1 I + R'R)^{-1} is not used in closed form.  With e = d1 - v
// and p = m - d2 (so d2 = x - p), iteration k is
//
//   rhs = R'(v - d1) + rho (x + d2) = -R'e + rho (2x - p),
//   r = rhs - M m (M = rho I + R'R)                            k_stv_rhs
//   cg steps from m:                                           k_stv_dir, k_stv_update
//     p_j = r_j + (gamma_j / gamma_{j-1}) p_{j-1},  q = M p_j
//     alpha = gamma_j / <p_j, q>,  m += alpha p_j,  r -= alpha q,  gamma_{j+1} = <r, r>
//   d1' = e + R m'  (= d1 - (v - R m')),  p' = m' - d2 = m' + p - x,
//   and already the next threshold step on (m', d1'):
//   v' = S(R m' + d1', lambda/(2 mu1)),  e' = d1' - v'          k_stv_finish
//
// after which the inverse step forms x' = A (H'y + mu2 p') (k_col_inverse);
// the next d2 is x' - p'.  d1 itself is never stored.  A solve starts from
// m = p = x = H'y, d1 = 0: k_stv_init forms e = -S(R m).  The prior term
// ||R x||_1 of J at the incoming x is summed by k_stv_rhs (k_stv_prior for
// the final x).
//
// Fields are [Nt][Nx][Ny]; a "row" is one image column (t, i) of Ny
// elements, with neighbours at +-1 (j), +-Ny (i) and +-Nx Ny (t).  A block
// walks P.rows (<= kStvRows) consecutive rows; (t, i) of its first row is found once and
// stepped, and an element's row within the block comes from an FP32
// reciprocal that is exact at these sizes (see row_of).  e keeps its three
// components padded to the grid, with zeros where a difference leaves it
// (they stay zero: S(0) = 0), so R'e needs no cases beyond the first index of
// each axis.
//
// 3D volumes: slices stacked along z (each with its own mask, coils and
// inverses) add w_z D_z to R.  The slices of a volume are consecutive
// descriptors of one launch; an element's z-neighbours are the same element
// of the neighbouring descriptors' fields, and e carries a fourth component.
// A volume of one slice runs exactly the 2D arithmetic.
//
// CG inner products are sums over the whole slice (over the whole volume).  A thread adds its
// elements (rows * Ny / 256 of them, at most 64) in FP32 with Kahan's
// compensated summation (error about 2 eps, not n eps); the block sums
// its threads in FP64 and writes a partial, and the last block of the slice
// to finish (an atomic counter after a fence) adds the partials in block
// order, so results do not depend on scheduling.  alpha and beta are formed
// in FP64 from those sums.  (GB300's FP64 pipe runs at 1/64 of FP32: FP64
// products per element would cost more than the memory traffic.)
#include "kahan.cuh"
#include "kernels.h"

namespace recon {

namespace {

// Where the threads of this block are: rows [row0, row0 + nrows) of the slice.
struct Blk {
  int row0, nrows;
  int t0, i0;      // (t, i) of row0
  float inv_ny;
};

__device__ __forceinline__ Blk blk_of(const StvSlice& P) {
  Blk b;
  b.row0 = ((int)blockIdx.x - P.tile0) * P.rows;
  b.nrows = min(P.rows, P.Nt * P.Nx - b.row0);
  b.t0 = b.row0 / P.Nx;
  b.i0 = b.row0 - b.t0 * P.Nx;
  b.inv_ny = 1.f / (float)P.Ny;
  return b;
}

// Row within the block of local element e < rows * Ny <= kStvRows * Ny: (e + 1/2)/Ny has
// fractional part >= 1/(2 Ny) >= 2^-11 away from an integer, and its FP32
// rounding error is below 2^14 * 2^-24, so the truncation is exact.
__device__ __forceinline__ int row_of(const Blk& b, int e) {
  return __float2int_rz(((float)e + 0.5f) * b.inv_ny);
}

struct Pos {
  int idx, t, i, j;
};

__device__ __forceinline__ Pos pos_of(const StvSlice& P, const Blk& b, int e) {
  const int r = row_of(b, e);
  Pos q;
  q.j = e - r * P.Ny;
  q.i = b.i0 + r;
  q.t = b.t0;
  while (q.i >= P.Nx) { q.i -= P.Nx; ++q.t; }   // at most P.rows steps
  q.idx = (b.row0 + r) * P.Ny + q.j;
  return q;
}

// (D_t f, w D_x f, w D_y f, w_z D_z f) at q, zero where the difference leaves
// the grid; fz is the same field of the slice above (null: none)
__device__ __forceinline__ void diffs(const StvSlice& P, const float2* __restrict__ f, const float2* fz,
                                      const Pos& q, float2 (&d)[4]) {
  const float2 c = f[q.idx];
  const float2 z = make_float2(0.f, 0.f);
  d[0] = (q.t + 1 < P.Nt) ? c_sub(f[q.idx + P.Nx * P.Ny], c) : z;
  d[1] = (q.i + 1 < P.Nx) ? c_scale(c_sub(f[q.idx + P.Ny], c), P.ws) : z;
  d[2] = (q.j + 1 < P.Ny) ? c_scale(c_sub(f[q.idx + 1], c), P.ws) : z;
  d[3] = fz ? c_scale(c_sub(fz[q.idx], c), P.wz) : z;
}

// (D'D f)_t + w^2 ((D'D f)_x + (D'D f)_y) + w_z^2 (D'D f)_z at q: the 7-point
// (9-point in a volume) operator R'R; fp / fn give f of the slices below /
// above (used only when the slice has them)
template <class F, class Fp, class Fn>
__device__ __forceinline__ float2 rtr(const StvSlice& P, F f, Fp fp, Fn fn, const Pos& q) {
  const int idx = q.idx, st = P.Nx * P.Ny;
  const float2 c = f(idx);
  float2 lz = make_float2(0.f, 0.f);
  if (P.zprev) lz = c_add(lz, c_sub(c, fp(idx)));
  if (P.znext) lz = c_sub(lz, c_sub(fn(idx), c));
  float2 lt = make_float2(0.f, 0.f), ls = make_float2(0.f, 0.f);
  if (q.t > 0) lt = c_add(lt, c_sub(c, f(idx - st)));
  if (q.t + 1 < P.Nt) lt = c_sub(lt, c_sub(f(idx + st), c));
  if (q.i > 0) ls = c_add(ls, c_sub(c, f(idx - P.Ny)));
  if (q.i + 1 < P.Nx) ls = c_sub(ls, c_sub(f(idx + P.Ny), c));
  if (q.j > 0) ls = c_add(ls, c_sub(c, f(idx - 1)));
  if (q.j + 1 < P.Ny) ls = c_sub(ls, c_sub(f(idx + 1), c));
  const float w2 = P.ws * P.ws, z2 = P.wz * P.wz;
  return make_float2(fmaf(z2, lz.x, fmaf(w2, ls.x, lt.x)), fmaf(z2, lz.y, fmaf(w2, ls.y, lt.y)));
}

__device__ __forceinline__ int slice_of(const StvLaunch& L) {
  int lo = 0, hi = L.nslices - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.slices[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// the slices below / above in a volume (null: none)
__device__ __forceinline__ const StvSlice* below(const StvLaunch& L, int si) {
  return L.slices[si].zprev ? &L.slices[si - 1] : nullptr;
}
__device__ __forceinline__ const StvSlice* above(const StvLaunch& L, int si) {
  return L.slices[si].znext ? &L.slices[si + 1] : nullptr;
}

// Sum of v over the slice (the volume) into *slot (deterministic order); see
// the file comment.  Takes the reduction fields by value, so a kernel's
// register copy of its descriptor never needs a memory home.
struct SliceSum {
  double* part;
  unsigned* count;
  int red0, rednblk;
};
__device__ __forceinline__ SliceSum slice_sum_of(const StvSlice& P) { return SliceSum{P.part, P.count, P.red0, P.rednblk}; }

__device__ __forceinline__ void slice_sum(SliceSum S, double v, double* slot) {
  __shared__ double red[32];
  __shared__ int last;
  const int tid = threadIdx.x, nth = (int)blockDim.x;
  const double s = group_sum(v, red, tid, nth, BlockBar());
  if (tid == 0) {
    S.part[blockIdx.x] = s;
    __threadfence();
    last = (atomicAdd(S.count, 1u) == (unsigned)(S.rednblk - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0;
  for (int b = tid; b < S.rednblk; b += nth) a += __ldcg(S.part + S.red0 + b);
  const double tot = group_sum(a, red, tid, nth, BlockBar());
  if (tid == 0) {
    *slot = tot;
    *S.count = 0u;
  }
}

__device__ __forceinline__ float rx_l1(const StvSlice& P, const float2* xz, const Pos& q) {
  float2 d[4];
  diffs(P, P.x, xz, q, d);
  return c_abs(d[0]) + c_abs(d[1]) + c_abs(d[2]) + c_abs(d[3]);
}

// e = d1 - S(R m + d1) into the padded components, with d1 = e + R m (the
// previous e, from k_stv_finish) or d1 = 0 (first = true, from k_stv_init).
// With the residual fields set (iterations K-1 and K), d1 is also kept, or
// its change ||d1_{K-1} - d1_K||^2 added to *dd1.
__device__ __forceinline__ void threshold(const StvSlice& P, const float2* mz, const Pos& q, bool first,
                                          KahanSum* dd1 = nullptr) {
  float2 rm[4];
  diffs(P, P.m, mz, q, rm);
  const int nc = (P.zprev || P.znext) ? 4 : 3;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= nc) break;
    const long long o = (long long)k * P.n + q.idx;
    const float2 dd = first ? make_float2(0.f, 0.f) : c_add(P.e[o], rm[k]);
    if (P.d1_keep) P.d1_keep[o] = dd;
    if (dd1) {
      const float2 df = c_sub(P.d1_ref ? P.d1_ref[o] : make_float2(0.f, 0.f), dd);
      dd1->add(fmaf(df.x, df.x, df.y * df.y));
    }
    P.e[o] = c_sub(dd, c_soft(c_add(rm[k], dd), P.tau1));
  }
}

__global__ void __launch_bounds__(kStvThreads) k_stv_init(StvLaunch L) {
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  if (P.stop && *P.stop) return;
  const StvSlice* Pn = above(L, si);
  const Blk b = blk_of(P);
  const float2* mz = Pn ? Pn->m : nullptr;
  for (int e = threadIdx.x; e < b.nrows * P.Ny; e += kStvThreads) threshold(P, mz, pos_of(P, b, e), true);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_prior(StvLaunch L) {
  __shared__ double red[32];
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  if (P.stop && *P.stop) return;
  const StvSlice* Pn = above(L, si);
  const Blk b = blk_of(P);
  KahanSum l1;
#pragma unroll 4
  const float2* xz = Pn ? Pn->x : nullptr;
  for (int e = threadIdx.x; e < b.nrows * P.Ny; e += kStvThreads) l1.add(rx_l1(P, xz, pos_of(P, b, e)));
  const double s = group_sum((double)l1.s, red, threadIdx.x, kStvThreads, BlockBar());
  if (threadIdx.x == 0) atomicAdd(P.prior_acc, s);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_rhs(StvLaunch L) {
  __shared__ double red[32];
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  if (P.stop && *P.stop) return;
  const StvSlice* Pp = below(L, si);
  const StvSlice* Pn = above(L, si);
  const Blk b = blk_of(P);
  const int st = P.Nx * P.Ny;
  const float2* et = P.e;
  const float2* ex = P.e + P.n;
  const float2* ey = P.e + 2 * (long long)P.n;
  const float2* m = P.m;
  const float2* mp = Pp ? Pp->m : m;
  const float2* mn = Pn ? Pn->m : m;
  const float2* ez = P.e + 3 * (long long)P.n;
  const float2* ezp = Pp ? Pp->e + 3 * (long long)Pp->n : ez;
  const float2* xz = Pn ? Pn->x : nullptr;
  KahanSum g, l1;
#pragma unroll 4
  for (int e = threadIdx.x; e < b.nrows * P.Ny; e += kStvThreads) {
    const Pos q = pos_of(P, b, e);
    const int idx = q.idx;
    l1.add(rx_l1(P, xz, q));
    // R'e (the padded components are zero past the last index)
    float2 rt = make_float2(-et[idx].x, -et[idx].y), rs = make_float2(-ex[idx].x - ey[idx].x, -ex[idx].y - ey[idx].y);
    if (q.t > 0) rt = c_add(rt, et[idx - st]);
    if (q.i > 0) rs = c_add(rs, ex[idx - P.Ny]);
    if (q.j > 0) rs = c_add(rs, ey[idx - 1]);
    float2 rte = make_float2(fmaf(P.ws, rs.x, rt.x), fmaf(P.ws, rs.y, rt.y));
    if (P.zprev || P.znext) {   // w_z D_z' e_z: e_z of the slice below minus this slice's
      float2 rz = make_float2(-ez[idx].x, -ez[idx].y);
      if (P.zprev) rz = c_add(rz, ezp[idx]);
      rte = make_float2(fmaf(P.wz, rz.x, rte.x), fmaf(P.wz, rz.y, rte.y));
    }
    const float2 xv = P.x[idx], pv = P.p[idx], mv = m[idx];
    const float2 mm = rtr(P, [m](int o) { return m[o]; }, [mp](int o) { return mp[o]; },
                          [mn](int o) { return mn[o]; }, q);
    // r = -R'e + rho (2x - p) - (rho m + R'R m)
    float2 r;
    r.x = fmaf(P.rho, 2.f * xv.x - pv.x - mv.x, -rte.x - mm.x);
    r.y = fmaf(P.rho, 2.f * xv.y - pv.y - mv.y, -rte.y - mm.y);
    P.r[idx] = r;
    g.add(fmaf(r.x, r.x, r.y * r.y));
  }
  const double s = group_sum((double)l1.s, red, threadIdx.x, kStvThreads, BlockBar());
  if (threadIdx.x == 0) atomicAdd(P.prior_acc, s);
  slice_sum(slice_sum_of(P), (double)g.s, P.red);
}

// p_j = r + beta p_{j-1} and q = M p_j, <p_j, q>.  One thread per j (the
// block is Ny_max rounded up to a warp), marching the block's image columns
// (t, i) in order: p_j of the next column (i+1) is formed once and kept for
// two steps, so a point costs the loads of r and p_{j-1} at (i+1) and at
// t -+ 1 (and z -+ 1 in a volume); the j-neighbours come through shared
// memory.  M = rho I + R'R in the grouping of rtr().
__global__ void __launch_bounds__(kStvDirMaxThreads) k_stv_dir(StvLaunch L) {
  __shared__ float2 rowbuf[2][kStvDirMaxThreads + 2];
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  if (P.stop && *P.stop) return;
  const StvSlice* Pp = below(L, si);
  const StvSlice* Pn = above(L, si);
  const int j = L.step;
  const Blk b = blk_of(P);
  double beta = 0.0;
  if (j > 0 && P.red[j - 1] > 0.0) beta = P.red[j] / P.red[j - 1];
  const float be = (float)beta;
  const float2* r = P.r;
  // the two direction buffers, picked without a dynamic index into the
  // descriptor (which would give its register copy a memory home)
  const float2* po = (j & 1) ? P.pc[0] : P.pc[1];
  float2* pn = (j & 1) ? P.pc[1] : P.pc[0];
  auto dir_of = [be, j](const float2* rr, const float2* pp, int o) {
    const float2 rv = rr[o];
    if (j == 0) return rv;
    const float2 pv = pp[o];
    return make_float2(fmaf(be, pv.x, rv.x), fmaf(be, pv.y, rv.y));
  };
  const float2* rp = Pp ? Pp->r : r;
  const float2* pop = Pp ? ((j & 1) ? Pp->pc[0] : Pp->pc[1]) : po;
  const float2* rn = Pn ? Pn->r : r;
  const float2* pon = Pn ? ((j & 1) ? Pn->pc[0] : Pn->pc[1]) : po;
  const int Nx = P.Nx, Ny = P.Ny, Nt = P.Nt, st = Nx * Ny;
  const int jj = threadIdx.x;
  const bool act = jj < Ny;
  const float2 z = make_float2(0.f, 0.f);
  const float w2 = P.ws * P.ws, z2 = P.wz * P.wz;
  if (jj == 0) {   // the zero halo of the j-neighbour exchange
    rowbuf[0][0] = rowbuf[1][0] = z;
    rowbuf[0][Ny + 1] = rowbuf[1][Ny + 1] = z;
  }
  int t = b.t0, i = b.i0;
  int idx = (t * Nx + i) * Ny + jj;
  float2 cur = z, prev = z;
  if (act) {
    cur = dir_of(r, po, idx);
    if (i > 0) prev = dir_of(r, po, idx - Ny);
  }
  KahanSum pq;
  for (int rr = 0; rr < b.nrows; ++rr) {
    float2 nxt = z, tm = z, tp = z, zm = z, zp = z;
    if (act) {
      if (i + 1 < Nx) nxt = dir_of(r, po, idx + Ny);
      if (t > 0) tm = dir_of(r, po, idx - st);
      if (t + 1 < Nt) tp = dir_of(r, po, idx + st);
      if (P.zprev) zm = dir_of(rp, pop, idx);
      if (P.znext) zp = dir_of(rn, pon, idx);
      rowbuf[rr & 1][jj + 1] = cur;
    }
    __syncthreads();
    if (act) {
      const float2 jm = rowbuf[rr & 1][jj], jp = rowbuf[rr & 1][jj + 2];
      const float2 c = cur;
      float2 lz = z;
      if (P.zprev) lz = c_add(lz, c_sub(c, zm));
      if (P.znext) lz = c_sub(lz, c_sub(zp, c));
      float2 lt = z, ls = z;
      if (t > 0) lt = c_add(lt, c_sub(c, tm));
      if (t + 1 < Nt) lt = c_sub(lt, c_sub(tp, c));
      if (i > 0) ls = c_add(ls, c_sub(c, prev));
      if (i + 1 < Nx) ls = c_sub(ls, c_sub(nxt, c));
      if (jj > 0) ls = c_add(ls, c_sub(c, jm));
      if (jj + 1 < Ny) ls = c_sub(ls, c_sub(jp, c));
      const float2 l = make_float2(fmaf(z2, lz.x, fmaf(w2, ls.x, lt.x)), fmaf(z2, lz.y, fmaf(w2, ls.y, lt.y)));
      const float2 qv = make_float2(fmaf(P.rho, c.x, l.x), fmaf(P.rho, c.y, l.y));
      pn[idx] = c;
      P.q[idx] = qv;
      pq.add(fmaf(c.x, qv.x, c.y * qv.y));
    }
    // next image column of the block: (t, i+1), or (t+1, 0) past the last i
    if (i + 1 < Nx) {
      prev = cur;
      cur = nxt;
      ++i;
      idx += Ny;
    } else {
      ++t;
      i = 0;
      idx += Ny;
      prev = z;
      cur = (act && rr + 1 < b.nrows) ? dir_of(r, po, idx) : z;
    }
  }
  slice_sum(slice_sum_of(P), (double)pq.s, P.red + P.cg + 1 + j);
}

// m += alpha p_j, r -= alpha q, gamma_{j+1} = <r, r>.  (Splitting each tile
// over 4 blocks for more warps in flight measured slower: 0.346 -> 0.396 ms a
// spatio-temporal step on the cardiac workload.)
__global__ void __launch_bounds__(kStvThreads) k_stv_update(StvLaunch L) {
  const StvSlice P = L.slices[slice_of(L)];
  if (P.stop && *P.stop) return;
  const int j = L.step;
  const Blk b = blk_of(P);
  const double gam = P.red[j], pq = P.red[P.cg + 1 + j];
  const float alpha = (pq > 0.0 && gam > 0.0) ? (float)(gam / pq) : 0.f;
  const float2* pn = (j & 1) ? P.pc[1] : P.pc[0];
  const int base = b.row0 * P.Ny;
  const int ne = b.nrows * P.Ny;
  KahanSum g;
  // element-wise: no neighbours, so no (t, i, j).  With Ny even the block's
  // elements start on a 16-byte boundary and go two per access.
  if ((P.Ny & 1) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(pn + base);
    const float4* q4 = reinterpret_cast<const float4*>(P.q + base);
    float4* m4 = reinterpret_cast<float4*>(P.m + base);
    float4* r4 = reinterpret_cast<float4*>(P.r + base);
#pragma unroll 4
    for (int e = threadIdx.x; e < ne / 2; e += kStvThreads) {
      const float4 pv = p4[e], qv = q4[e];
      float4 mv = m4[e], rv = r4[e];
      mv.x = fmaf(alpha, pv.x, mv.x); mv.y = fmaf(alpha, pv.y, mv.y);
      mv.z = fmaf(alpha, pv.z, mv.z); mv.w = fmaf(alpha, pv.w, mv.w);
      rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
      rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
      m4[e] = mv;
      r4[e] = rv;
      g.add(fmaf(rv.x, rv.x, rv.y * rv.y));
      g.add(fmaf(rv.z, rv.z, rv.w * rv.w));
    }
  } else {
#pragma unroll 4
    for (int e = threadIdx.x; e < ne; e += kStvThreads) {
      const int idx = base + e;
      const float2 pv = pn[idx], qv = P.q[idx];
      float2 mv = P.m[idx], rv = P.r[idx];
      mv.x = fmaf(alpha, pv.x, mv.x); mv.y = fmaf(alpha, pv.y, mv.y);
      rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
      P.m[idx] = mv;
      P.r[idx] = rv;
      g.add(fmaf(rv.x, rv.x, rv.y * rv.y));
    }
  }
  slice_sum(slice_sum_of(P), (double)g.s, P.red + j + 1);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_finish(StvLaunch L) {
  __shared__ double red[32];
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  if (P.stop && *P.stop) return;
  const StvSlice* Pn = above(L, si);
  const Blk b = blk_of(P);
  const float2* mz = Pn ? Pn->m : nullptr;
  KahanSum dd1;
#pragma unroll 4
  for (int e = threadIdx.x; e < b.nrows * P.Ny; e += kStvThreads) {
    const Pos q = pos_of(P, b, e);
    const int idx = q.idx;
    // e (the previous threshold's d1 - v) is read and replaced element by element
    threshold(P, mz, q, false, P.res_last ? &dd1 : nullptr);
    P.p[idx] = c_add(P.m[idx], c_sub(P.p[idx], P.x[idx]));
  }
  if (P.res_last) {   // the last iteration: v_K - R m_K = d1_{K-1} - d1_K
    const double sdd = group_sum((double)dd1.s, red, threadIdx.x, kStvThreads, BlockBar());
    if (threadIdx.x == 0) atomicAdd(P.res_acc + 1, sdd);
  }
}

// R (m_K - m_{K-1}) at q from the two fields (and the slice above's, in a volume)
__device__ __forceinline__ void diffs_dm(const StvSlice& P, const float2* mz, const float2* mpz, const Pos& q,
                                         float2 (&d)[4]) {
  const float2* m = P.m;
  const float2* mp = P.m_prev;
  auto dm = [m, mp](int o) { return c_sub(m[o], mp[o]); };
  const float2 c = dm(q.idx);
  const float2 z = make_float2(0.f, 0.f);
  d[0] = (q.t + 1 < P.Nt) ? c_sub(dm(q.idx + P.Nx * P.Ny), c) : z;
  d[1] = (q.i + 1 < P.Nx) ? c_scale(c_sub(dm(q.idx + P.Ny), c), P.ws) : z;
  d[2] = (q.j + 1 < P.Ny) ? c_scale(c_sub(dm(q.idx + 1), c), P.ws) : z;
  d[3] = mz ? c_scale(c_sub(c_sub(mz[q.idx], mpz[q.idx]), c), P.wz) : z;
}

// ADMM residual sums after the loop (final descriptor set): res_acc[0] +=
// ||m_K - x_K||^2, [2] += ||m_K - m_{K-1}||^2, [3] += ||R (m_K - m_{K-1})||^2
// ([1] came from k_stv_finish of the last iteration).
__global__ void __launch_bounds__(kStvThreads) k_stv_residuals(StvLaunch L) {
  __shared__ double red[32];
  const int si = slice_of(L);
  const StvSlice P = L.slices[si];   // a register copy: the loops store through global pointers
  const StvSlice* Pn = above(L, si);
  const Blk b = blk_of(P);
  const float2* mz = Pn ? Pn->m : nullptr;
  const float2* mpz = Pn ? Pn->m_prev : nullptr;
  KahanSum a0, a2, a3;
#pragma unroll 2
  for (int e = threadIdx.x; e < b.nrows * P.Ny; e += kStvThreads) {
    const Pos q = pos_of(P, b, e);
    const float2 mv = P.m[q.idx];
    const float2 mx = c_sub(mv, P.x[q.idx]), dm = c_sub(mv, P.m_prev[q.idx]);
    a0.add(fmaf(mx.x, mx.x, mx.y * mx.y));
    a2.add(fmaf(dm.x, dm.x, dm.y * dm.y));
    float2 d[4];
    diffs_dm(P, mz, mpz, q, d);
    float s3 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) s3 = fmaf(d[k].x, d[k].x, fmaf(d[k].y, d[k].y, s3));
    a3.add(s3);
  }
  const double s0 = group_sum((double)a0.s, red, threadIdx.x, kStvThreads, BlockBar());
  const double s2 = group_sum((double)a2.s, red, threadIdx.x, kStvThreads, BlockBar());
  const double s3 = group_sum((double)a3.s, red, threadIdx.x, kStvThreads, BlockBar());
  if (threadIdx.x == 0) {
    atomicAdd(P.res_acc + 0, s0);
    atomicAdd(P.res_acc + 2, s2);
    atomicAdd(P.res_acc + 3, s3);
  }
}

}  // namespace

#define STV_LAUNCH(kern)                                                 \
  do {                                                                   \
    if (L.nblocks < 1) return cudaSuccess;                               \
    kern<<<L.nblocks, kStvThreads, 0, s>>>(L);                           \
    note_launch();                                                       \
    return cudaGetLastError();                                           \
  } while (0)

cudaError_t launch_stv_init(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_init); }
cudaError_t launch_stv_prior(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_prior); }
cudaError_t launch_stv_rhs(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_rhs); }
cudaError_t launch_stv_dir(const StvLaunch& L, cudaStream_t s) {
  if (L.nblocks < 1) return cudaSuccess;
  if (L.dir_threads < 32 || L.dir_threads > kStvDirMaxThreads) return cudaErrorInvalidValue;
  k_stv_dir<<<L.nblocks, L.dir_threads, 0, s>>>(L);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_stv_update(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_update); }
cudaError_t launch_stv_finish(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_finish); }
cudaError_t launch_stv_residuals(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_residuals); }

}  // namespace recon
