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

namespace recon {

constexpr int kTvSeg = 8;        // Thomas segments per pixel
constexpr int kTvChunkPx = 16;   // pixels per chunk
constexpr int kTvChunkThreads = kTvSeg * kTvChunkPx;

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

// Loads bypass L1 (__ldcg): in the persistent solve the inputs were written
// by other SMs during the same launch.  Returns this thread's FP32 share of
// ||D_t x||_1.  seg_a / seg_b / bnd: kTvChunkThreads entries of shared memory;
// bar() synchronises exactly the kTvChunkThreads threads.
template <int LMAX, class Bar>
__device__ __forceinline__ float tv_chunk(const TvChunkIO& P, int tid, float* seg_a, float2* seg_b, float2* bnd,
                                          Bar bar) {
  const int Nt = P.Nt;
  const int seg = tid / kTvChunkPx, px = tid - seg * kTvChunkPx;
  const int Ls = (Nt + kTvSeg - 1) / kTvSeg;
  const int ta = min(Nt, seg * Ls), tb = min(Nt, ta + Ls), n = tb - ta;
  const size_t fs = P.fstride;
  const float2 z2 = make_float2(0.f, 0.f);
  const bool ok = px < P.nvalid;
  const size_t base = P.base + px;
  const bool write = P.write;
  // xs: x then rhs; ms: m then d then m'; ds: d1 then e; ps: p then f
  float2 xs[LMAX], ms[LMAX], ds[LMAX], ps[LMAX];
  float2 xn = z2, mn = z2, mp = z2, dp = z2;
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    xs[u] = ms[u] = ds[u] = ps[u] = z2;
    if (ok && u < n) {
      const size_t g = (size_t)(ta + u) * fs + base;
      xs[u] = __ldcg(P.x + g);
      if (write) {
        ms[u] = __ldcg(P.m + g);
        ps[u] = __ldcg(P.p + g);
        if (P.d1 && ta + u + 1 < Nt) ds[u] = __ldcg(P.d1 + g);
      }
    }
  }
  if (ok && n > 0 && tb < Nt) {
    xn = __ldcg(P.x + (size_t)tb * fs + base);
    if (write) mn = __ldcg(P.m + (size_t)tb * fs + base);
  }
  if (ok && n > 0 && ta > 0 && write) {
    mp = __ldcg(P.m + (size_t)(ta - 1) * fs + base);
    if (P.d1) dp = __ldcg(P.d1 + (size_t)(ta - 1) * fs + base);
  }
  float tvf = 0.f;
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (ok && u < n && ta + u + 1 < Nt) tvf += c_abs(c_sub(u + 1 < n ? xs[u + 1] : xn, xs[u]));
  if (!write) return tvf;
  // e_t = d1_t - S(m_{t+1} - m_t + d1_t) (t < Nt - 1; 0 at Nt - 1); e_{ta-1}
  // recomputed here from its own inputs
  float2 eprev = z2;
  if (ok && n > 0 && ta > 0) eprev = c_sub(dp, c_soft(c_add(c_sub(ms[0], mp), dp), P.tau1));
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (u < n)
      ds[u] = (ta + u + 1 < Nt) ? c_sub(ds[u], c_soft(c_add(c_sub(u + 1 < n ? ms[u + 1] : mn, ms[u]), ds[u]), P.tau1))
                                : z2;
  // rhs_t = e_t - e_{t-1} + rho (2 x_t - p_t) into xs;  f_t = p_t - x_t into ps
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    if (u < n) {
      const float2 x_t = xs[u], p_t = ps[u];
      float2 rhs = c_sub(ds[u], u > 0 ? ds[u - 1] : eprev);
      rhs.x = fmaf(P.rho, 2.f * x_t.x - p_t.x, rhs.x);
      rhs.y = fmaf(P.rho, 2.f * x_t.y - p_t.y, rhs.y);
      xs[u] = rhs;
      ps[u] = c_sub(p_t, x_t);
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
        A *= inv;
        B = c_scale(c_add(xs[u], B), inv);
      }
    seg_a[seg * kTvChunkPx + px] = A;
    seg_b[seg * kTvChunkPx + px] = B;
  }
  bar();
  {
    float2 d = z2;
    for (int q = 0; q < seg; ++q) d = c_add(c_scale(d, seg_a[q * kTvChunkPx + px]), seg_b[q * kTvChunkPx + px]);
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        d = c_scale(c_add(xs[u], d), __ldg(P.thomas + ta + u));
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
        B = make_float2(fmaf(inv, B.x, ms[u].x), fmaf(inv, B.y, ms[u].y));
        A *= inv;
      }
    seg_a[seg * kTvChunkPx + px] = A;
    seg_b[seg * kTvChunkPx + px] = B;
  }
  bar();
  {
    float2 mm = z2;
    for (int q = kTvSeg - 1; q > seg; --q) mm = c_add(c_scale(mm, seg_a[q * kTvChunkPx + px]), seg_b[q * kTvChunkPx + px]);
#pragma unroll
    for (int u = LMAX - 1; u >= 0; --u)
      if (u < n) {
        const float inv = __ldg(P.thomas + ta + u);
        mm = make_float2(fmaf(inv, mm.x, ms[u].x), fmaf(inv, mm.y, ms[u].y));
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
        const size_t g = (size_t)(ta + u) * fs + base;
        P.m_out[g] = ms[u];
        P.p_out[g] = c_add(ms[u], ps[u]);
        if (ta + u + 1 < Nt) P.d1_out[g] = c_add(ds[u], c_sub(u + 1 < n ? ms[u + 1] : mnext, ms[u]));
      }
  }
  return tvf;
}

}  // namespace recon
