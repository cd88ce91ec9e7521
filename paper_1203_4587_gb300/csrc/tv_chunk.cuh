// The temporal step of Algorithm 2 (R = D_t) for a chunk of kTvChunkPx
// consecutive pixels over every frame, by kTvSeg * kTvChunkPx threads with
// all values in registers:
//   v   = S(D_t m + d1, lambda/(2 mu1))
//   m'  = (rho I + D_t'D_t)^{-1} [D_t'(v - d1) + rho (x + d2)]
//   d1' = d1 - (v - D_t m')
// with d2 = x - p and p' = m' - d2 handed to the inverse step (which forms
// r = H'y + mu2 p').  Thread (seg, px) holds pixel px, frames [ta, tb) of
// segment seg (ceil(Nt / kTvSeg) frames each).  The tridiagonal solve runs
// the Thomas recurrences (forward d_t = inv_t (rhs_t + d_{t-1}), backward
// m'_t = d_t + inv_t m'_{t+1}) by segments: each composes its affine map, the
// maps are chained in order through shared memory, and each segment replays
// its frames from its incoming value.  The segmentation depends on Nt only.
// Used by the per-step temporal kernel and the persistent solve.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace recon {

constexpr int kTvChunkThreads = kTvSeg * kTvChunkPx;   // kTvSeg, kTvChunkPx: kernels.h

struct TvChunkIO {
  const float2* x;               // the incoming x ([Nt] frames of stride fstride)
  const float2* m;
  const float2* d1;              // null: d1 = 0 (the first step)
  const float2* p;               // p = m_prev - d2_prev
  float2* m_out;
  float2* d1_out;
  float2* p_out;
  const float* thomas;           // [Nt] pivots of (rho I + D'D)
  float tau1, rho;
  int Nt;
  size_t fstride;                // elements between frames
  size_t base;                   // element of the chunk's first pixel in frame 0
  int nvalid;                    // pixels of the chunk inside the image
  bool write;                    // false: only the prior term ||D_t x||_1
};

// Explicitly rounded arithmetic, so that the general and the full-chunk
// instantiations (and the persistent solve) give bit-identical results: the
// complex updates are packed FP32x2 operations, each rounded once.
__device__ __forceinline__ float2 tv_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 tv_sub(float2 a, float2 b) {   // exact -1 * b, then one rounding
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 tv_scale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 tv_fma(float2 a, float s, float2 c) { return __ffma2_rn(a, make_float2(s, s), c); }
// S(a, tau) (Section III soft threshold) as a (1 - tau / |a|) for |a|^2 > tau^2,
// with 1/|a| from the hardware reciprocal square root (relative error about
// 2^-22, far inside the FP32 path's tolerance); tau2 = tau * tau.
__device__ __forceinline__ float2 tv_soft(float2 a, float tau, float tau2) {
  const float m2 = fmaf(a.x, a.x, __fmul_rn(a.y, a.y));
  const float s = m2 > tau2 ? fmaf(-tau, rsqrtf(m2), 1.f) : 0.f;
  return tv_scale(a, s);
}
// |a| = |a|^2 / |a| with the same reciprocal square root (0 at a = 0).
__device__ __forceinline__ float tv_abs(float2 a) {
  const float m2 = fmaf(a.x, a.x, __fmul_rn(a.y, a.y));
  return m2 > 0.f ? __fmul_rn(m2, rsqrtf(m2)) : 0.f;
}

// Loads bypass L1 (__ldcg): in the persistent solve the inputs were written
// by other SMs during the same launch.  Returns this thread's FP32 share of
// ||D_t x||_1.  seg_a / seg_b / bnd: kTvChunkThreads entries of shared memory;
// bar() synchronises exactly the kTvChunkThreads threads.
//
// FULL: the chunk is known to be whole (Nt == kTvSeg * LMAX, all
// kTvChunkPx pixels inside the image, d1 present, state written), so every
// segment holds exactly LMAX frames and the bounds tests fold away at compile
// time.  The arithmetic is the same operation for operation.
template <int LMAX, bool FULL, class Bar>
__device__ __forceinline__ float tv_chunk(const TvChunkIO& P, int tid, float* seg_a, float2* seg_b, float2* bnd,
                                          Bar bar) {
  const int Nt = FULL ? kTvSeg * LMAX : P.Nt;
  const int seg = tid / kTvChunkPx, px = tid - seg * kTvChunkPx;
  const int Ls = FULL ? LMAX : (Nt + kTvSeg - 1) / kTvSeg;
  const int ta = FULL ? seg * LMAX : min(Nt, seg * Ls);
  const int tb = FULL ? ta + LMAX : min(Nt, ta + Ls);
  const int n = FULL ? LMAX : tb - ta;
  const size_t fs = P.fstride;
  const float2 z2 = make_float2(0.f, 0.f);
  const bool ok = FULL || px < P.nvalid;
  const bool write = FULL || P.write;
  const bool has_d1 = FULL || P.d1 != nullptr;
  const size_t g0 = (size_t)ta * fs + P.base + px;
  // xs: x then rhs; ms: m then d then m'; ds: d1 then e; ps: p then f
  float2 xs[LMAX], ms[LMAX], ds[LMAX], ps[LMAX];
  float2 xn = z2, mn = z2, mp = z2, dp = z2;
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    xs[u] = ms[u] = ds[u] = ps[u] = z2;
    if (ok && u < n) {
      const size_t g = g0 + (size_t)u * fs;
      xs[u] = __ldcg(P.x + g);
      if (write) {
        ms[u] = __ldcg(P.m + g);
        ps[u] = __ldcg(P.p + g);
        if (has_d1 && ta + u + 1 < Nt) ds[u] = __ldcg(P.d1 + g);
      }
    }
  }
  if (ok && n > 0 && tb < Nt) {
    xn = __ldcg(P.x + g0 + (size_t)n * fs);
    if (write) mn = __ldcg(P.m + g0 + (size_t)n * fs);
  }
  if (ok && n > 0 && ta > 0 && write) {
    mp = __ldcg(P.m + g0 - fs);
    if (has_d1) dp = __ldcg(P.d1 + g0 - fs);
  }
  float tvf = 0.f;
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (ok && u < n && ta + u + 1 < Nt) tvf += tv_abs(tv_sub(u + 1 < n ? xs[u + 1] : xn, xs[u]));
  if (!write) return tvf;
  const float tau = P.tau1, tau2 = __fmul_rn(tau, tau), rho = P.rho;
  // e_t = d1_t - S(m_{t+1} - m_t + d1_t) (t < Nt - 1; 0 at Nt - 1); e_{ta-1}
  // recomputed here from its own inputs
  float2 eprev = z2;
  if (ok && n > 0 && ta > 0) eprev = tv_sub(dp, tv_soft(tv_add(tv_sub(ms[0], mp), dp), tau, tau2));
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (u < n)
      ds[u] = (ta + u + 1 < Nt)
                  ? tv_sub(ds[u], tv_soft(tv_add(tv_sub(u + 1 < n ? ms[u + 1] : mn, ms[u]), ds[u]), tau, tau2))
                  : z2;
  // rhs_t = e_t - e_{t-1} + rho (2 x_t - p_t) into xs;  f_t = p_t - x_t into ps
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    if (u < n) {
      const float2 x_t = xs[u], p_t = ps[u];
      const float2 w = tv_sub(tv_add(x_t, x_t), p_t);
      xs[u] = tv_fma(w, rho, tv_sub(ds[u], u > 0 ? ds[u - 1] : eprev));
      ps[u] = tv_sub(p_t, x_t);
    }
  }
  // forward recurrence by segments
  {
    float A = 1.f;
    float2 B = z2;
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        const float inv = __ldg(P.thomas + ta + u);
        A = __fmul_rn(A, inv);
        B = tv_scale(tv_add(xs[u], B), inv);
      }
    seg_a[seg * kTvChunkPx + px] = A;
    seg_b[seg * kTvChunkPx + px] = B;
  }
  bar();
  {
    float2 d = z2;
#pragma unroll
    for (int q = 0; q < kTvSeg - 1; ++q)
      if (q < seg) d = tv_fma(d, seg_a[q * kTvChunkPx + px], seg_b[q * kTvChunkPx + px]);
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        d = tv_scale(tv_add(xs[u], d), __ldg(P.thomas + ta + u));
        ms[u] = d;
      }
  }
  bar();
  // backward recurrence by segments
  {
    float A = 1.f;
    float2 B = z2;
#pragma unroll
    for (int u = LMAX - 1; u >= 0; --u)
      if (u < n) {
        const float inv = __ldg(P.thomas + ta + u);
        B = tv_fma(B, inv, ms[u]);
        A = __fmul_rn(A, inv);
      }
    seg_a[seg * kTvChunkPx + px] = A;
    seg_b[seg * kTvChunkPx + px] = B;
  }
  bar();
  {
    float2 mm = z2;
#pragma unroll
    for (int q = kTvSeg - 1; q > 0; --q)
      if (q > seg) mm = tv_fma(mm, seg_a[q * kTvChunkPx + px], seg_b[q * kTvChunkPx + px]);
#pragma unroll
    for (int u = LMAX - 1; u >= 0; --u)
      if (u < n) {
        mm = tv_fma(mm, __ldg(P.thomas + ta + u), ms[u]);
        ms[u] = mm;
      }
    bnd[seg * kTvChunkPx + px] = n > 0 ? ms[0] : z2;   // m'_{ta}, read by the previous segment
  }
  bar();
  // m', d1' = e + D m', p' = m' + f
  if (ok) {
    const float2 mnext = (tb < Nt) ? bnd[(seg + 1) * kTvChunkPx + px] : z2;
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        const size_t g = g0 + (size_t)u * fs;
        P.m_out[g] = ms[u];
        P.p_out[g] = tv_add(ms[u], ps[u]);
        if (ta + u + 1 < Nt) P.d1_out[g] = tv_add(ds[u], tv_sub(u + 1 < n ? ms[u + 1] : mnext, ms[u]));
      }
  }
  return tvf;
}

}  // namespace recon
