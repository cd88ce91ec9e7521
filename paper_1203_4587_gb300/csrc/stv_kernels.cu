// Algorithm 2 with a spatio-temporal analysis operator
//   R x = (D_t x, w D_x x, w D_y x)
// (non-circular differences along t, the horizontal index i and the vertical
// index j) and an m-update by conjugate gradients, as Section IV-B suggests
// when (mu2/mu1 I + R'R)^{-1} is not used in closed form:
//
//   v   = S(R m + d1, lambda / (2 mu1))                      k_stv_prior
//   rhs = R'(v - d1) + rho (x + d2),  r = rhs - M m           k_stv_rhs
//   cg steps on M = rho I + R'R from m:                       k_stv_dir, k_stv_update
//     p_j = r_j + (gamma_j / gamma_{j-1}) p_{j-1},  q = M p_j
//     alpha = gamma_j / <p_j, q>,  m += alpha p_j,  r -= alpha q,  gamma_{j+1} = <r, r>
//   d1' = d1 - (v - R m'),  p' = m' - d2                      k_stv_finish
//
// then the inverse step forms x' = A (H'y + mu2 p') (k_col_inverse), and the
// next d2 is x' - p' (the same bookkeeping as the temporal TV step).
//
// Fields are [Nt][Nx][Ny]; element idx = (t Nx + i) Ny + j has its
// neighbours at idx +- 1 (j), +- Ny (i) and +- Nx Ny (t).  d1 and e = d1 - v
// keep the three components padded to the grid, with zeros where a
// difference leaves it; those stay zero (S(0 + 0) = 0), so the adjoint
// R'u = D_t'u_t + w D_x'u_x + w D_y'u_y needs no boundary cases beyond the
// first index of each axis.
//
// The CG inner products are sums over the whole slice: every block writes
// its partial sum, and the last block of the slice to finish (a counter
// taken with an atomic after a fence) adds the partials in block order, so
// the result does not depend on scheduling.  alpha and beta are formed in
// FP64 from those sums.
#include "kernels.h"

namespace recon {

namespace {

struct Pos {
  int t, i, j;
};

__device__ __forceinline__ Pos pos_of(const StvSlice& P, int idx) {
  const int st = P.Nx * P.Ny;
  Pos q;
  q.t = idx / st;
  const int rem = idx - q.t * st;
  q.i = rem / P.Ny;
  q.j = rem - q.i * P.Ny;
  return q;
}

// (D_t f, w D_x f, w D_y f) at idx, zero where the difference leaves the grid
__device__ __forceinline__ void diffs(const StvSlice& P, const float2* __restrict__ f, int idx, Pos q,
                                      float2& dt, float2& dx, float2& dy) {
  const float2 c = f[idx];
  const float2 z = make_float2(0.f, 0.f);
  dt = (q.t + 1 < P.Nt) ? c_sub(f[idx + P.Nx * P.Ny], c) : z;
  dx = (q.i + 1 < P.Nx) ? c_scale(c_sub(f[idx + P.Ny], c), P.ws) : z;
  dy = (q.j + 1 < P.Ny) ? c_scale(c_sub(f[idx + 1], c), P.ws) : z;
}

// (D'D f)_t + w^2 ((D'D f)_x + (D'D f)_y) at idx: the 7-point operator R'R
template <class F>
__device__ __forceinline__ float2 rtr(const StvSlice& P, F f, int idx, Pos q) {
  const float2 c = f(idx);
  const int st = P.Nx * P.Ny;
  float2 lt = make_float2(0.f, 0.f), ls = make_float2(0.f, 0.f);
  if (q.t > 0) lt = c_add(lt, c_sub(c, f(idx - st)));
  if (q.t + 1 < P.Nt) lt = c_sub(lt, c_sub(f(idx + st), c));
  if (q.i > 0) ls = c_add(ls, c_sub(c, f(idx - P.Ny)));
  if (q.i + 1 < P.Nx) ls = c_sub(ls, c_sub(f(idx + P.Ny), c));
  if (q.j > 0) ls = c_add(ls, c_sub(c, f(idx - 1)));
  if (q.j + 1 < P.Ny) ls = c_sub(ls, c_sub(f(idx + 1), c));
  const float w2 = P.ws * P.ws;
  return make_float2(fmaf(w2, ls.x, lt.x), fmaf(w2, ls.y, lt.y));
}

__device__ __forceinline__ const StvSlice& slice_of(const StvLaunch& L) {
  int lo = 0, hi = L.nslices - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.slices[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  return L.slices[lo];
}

// Sum of v over the slice into *slot (deterministic order); see the file comment.
__device__ void slice_sum(const StvSlice& P, double v, double* slot) {
  __shared__ double red[32];
  __shared__ int last;
  const int tid = threadIdx.x;
  const double s = group_sum(v, red, tid, kStvThreads, BlockBar());
  if (tid == 0) {
    P.part[blockIdx.x] = s;
    __threadfence();
    last = (atomicAdd(P.count, 1u) == (unsigned)(P.nblk - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0;
  for (int b = tid; b < P.nblk; b += kStvThreads) a += __ldcg(P.part + P.tile0 + b);
  const double tot = group_sum(a, red, tid, kStvThreads, BlockBar());
  if (tid == 0) {
    *slot = tot;
    *P.count = 0u;
  }
}

__global__ void __launch_bounds__(kStvThreads) k_stv_prior(StvLaunch L) {
  __shared__ double red[32];
  const StvSlice& P = slice_of(L);
  if (P.stop && *P.stop) return;
  const int base = ((int)blockIdx.x - P.tile0) * kStvBlockElems;
  double l1 = 0.0;
#pragma unroll
  for (int k = 0; k < kStvPerThread; ++k) {
    const int idx = base + k * kStvThreads + (int)threadIdx.x;
    if (idx >= P.n) break;
    const Pos q = pos_of(P, idx);
    float2 a, b, c;
    diffs(P, P.x, idx, q, a, b, c);
    l1 += (double)(c_abs(a) + c_abs(b) + c_abs(c));
    if (P.write_state) {
      diffs(P, P.m, idx, q, a, b, c);
      const float2 rm[3] = {a, b, c};
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const long long o = (long long)comp * P.n + idx;
        const float2 d = P.d1[o];
        P.e[o] = c_sub(d, c_soft(c_add(rm[comp], d), P.tau1));
      }
    }
  }
  const double s = group_sum(l1, red, threadIdx.x, kStvThreads, BlockBar());
  if (threadIdx.x == 0) atomicAdd(P.prior_acc, s);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_rhs(StvLaunch L) {
  const StvSlice& P = slice_of(L);
  if (P.stop && *P.stop) return;
  const int base = ((int)blockIdx.x - P.tile0) * kStvBlockElems;
  const int st = P.Nx * P.Ny;
  const float2* et = P.e;
  const float2* ex = P.e + P.n;
  const float2* ey = P.e + 2 * (long long)P.n;
  const float2* m = P.m;
  double g = 0.0;
#pragma unroll
  for (int k = 0; k < kStvPerThread; ++k) {
    const int idx = base + k * kStvThreads + (int)threadIdx.x;
    if (idx >= P.n) break;
    const Pos q = pos_of(P, idx);
    // R'e (the padded components are zero past the last index)
    float2 rt = make_float2(-et[idx].x, -et[idx].y), rs = make_float2(-ex[idx].x - ey[idx].x, -ex[idx].y - ey[idx].y);
    if (q.t > 0) rt = c_add(rt, et[idx - st]);
    if (q.i > 0) rs = c_add(rs, ex[idx - P.Ny]);
    if (q.j > 0) rs = c_add(rs, ey[idx - 1]);
    const float2 rte = make_float2(fmaf(P.ws, rs.x, rt.x), fmaf(P.ws, rs.y, rt.y));
    const float2 xv = P.x[idx], pv = P.p[idx], mv = m[idx];
    const float2 mm = rtr(P, [m](int o) { return m[o]; }, idx, q);
    // r = -R'e + rho (2x - p) - (rho m + R'R m)
    float2 r;
    r.x = fmaf(P.rho, 2.f * xv.x - pv.x - mv.x, -rte.x - mm.x);
    r.y = fmaf(P.rho, 2.f * xv.y - pv.y - mv.y, -rte.y - mm.y);
    P.r[idx] = r;
    g += (double)r.x * r.x + (double)r.y * r.y;
  }
  slice_sum(P, g, P.red);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_dir(StvLaunch L) {
  const StvSlice& P = slice_of(L);
  if (P.stop && *P.stop) return;
  const int j = L.step;
  const int base = ((int)blockIdx.x - P.tile0) * kStvBlockElems;
  double beta = 0.0;
  if (j > 0 && P.red[j - 1] > 0.0) beta = P.red[j] / P.red[j - 1];
  const float b = (float)beta;
  const float2* r = P.r;
  const float2* po = P.pc[(j + 1) & 1];
  float2* pn = P.pc[j & 1];
  auto dir = [r, po, b, j](int o) {
    const float2 rv = r[o];
    if (j == 0) return rv;
    const float2 pv = po[o];
    return make_float2(fmaf(b, pv.x, rv.x), fmaf(b, pv.y, rv.y));
  };
  double pq = 0.0;
#pragma unroll
  for (int k = 0; k < kStvPerThread; ++k) {
    const int idx = base + k * kStvThreads + (int)threadIdx.x;
    if (idx >= P.n) break;
    const Pos q = pos_of(P, idx);
    const float2 pv = dir(idx);
    const float2 l = rtr(P, dir, idx, q);
    const float2 qv = make_float2(fmaf(P.rho, pv.x, l.x), fmaf(P.rho, pv.y, l.y));
    pn[idx] = pv;
    P.q[idx] = qv;
    pq += (double)pv.x * qv.x + (double)pv.y * qv.y;
  }
  slice_sum(P, pq, P.red + P.cg + 1 + j);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_update(StvLaunch L) {
  const StvSlice& P = slice_of(L);
  if (P.stop && *P.stop) return;
  const int j = L.step;
  const int base = ((int)blockIdx.x - P.tile0) * kStvBlockElems;
  const double gam = P.red[j], pq = P.red[P.cg + 1 + j];
  const float alpha = (pq > 0.0 && gam > 0.0) ? (float)(gam / pq) : 0.f;
  const float2* pn = P.pc[j & 1];
  double g = 0.0;
#pragma unroll
  for (int k = 0; k < kStvPerThread; ++k) {
    const int idx = base + k * kStvThreads + (int)threadIdx.x;
    if (idx >= P.n) break;
    const float2 pv = pn[idx], qv = P.q[idx];
    float2 mv = P.m[idx], rv = P.r[idx];
    mv.x = fmaf(alpha, pv.x, mv.x); mv.y = fmaf(alpha, pv.y, mv.y);
    rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
    P.m[idx] = mv;
    P.r[idx] = rv;
    g += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  slice_sum(P, g, P.red + j + 1);
}

__global__ void __launch_bounds__(kStvThreads) k_stv_finish(StvLaunch L) {
  const StvSlice& P = slice_of(L);
  if (P.stop && *P.stop) return;
  const int base = ((int)blockIdx.x - P.tile0) * kStvBlockElems;
#pragma unroll
  for (int k = 0; k < kStvPerThread; ++k) {
    const int idx = base + k * kStvThreads + (int)threadIdx.x;
    if (idx >= P.n) break;
    const Pos q = pos_of(P, idx);
    float2 a, b, c;
    diffs(P, P.m, idx, q, a, b, c);
    const float2 rm[3] = {a, b, c};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const long long o = (long long)comp * P.n + idx;
      P.d1[o] = c_add(P.e[o], rm[comp]);
    }
    P.p[idx] = c_add(P.m[idx], c_sub(P.p[idx], P.x[idx]));
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

cudaError_t launch_stv_prior(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_prior); }
cudaError_t launch_stv_rhs(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_rhs); }
cudaError_t launch_stv_dir(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_dir); }
cudaError_t launch_stv_update(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_update); }
cudaError_t launch_stv_finish(const StvLaunch& L, cudaStream_t s) { STV_LAUNCH(k_stv_finish); }

}  // namespace recon
