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

namespace recon {

// The same step with two adjacent pixels per thread: a chunk of
// 2 * kTvChunkPx pixels by kTvChunkThreads threads (the per-step kernel).
// Thread (seg, px) holds pixels 2 px and 2 px + 1 of the chunk; their values
// move as one 16-byte access when the pair is 16-byte aligned in every frame
// (even frame stride and base).  The per-pixel state updates are those of
// tv_chunk, bit for bit, and so is each pixel's FP32 share of the prior term.
constexpr int kTvChunk2Px = 2 * kTvChunkPx;

__device__ __forceinline__ void ld_pair(const float2* p, bool vec, bool ok1, float2& a, float2& b) {
  if (vec) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  } else {
    a = __ldcg(p);
    b = ok1 ? __ldcg(p + 1) : make_float2(0.f, 0.f);
  }
}
__device__ __forceinline__ void st_pair(float2* p, bool vec, bool ok1, float2 a, float2 b) {
  if (vec) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    if (ok1) p[1] = b;
  }
}

// seg_a: 2 kTvChunkThreads floats; seg_b, bnd: 2 kTvChunkThreads float2.
// Returns this thread's share of ||D_t x||_1: each pixel's FP32 partial (as in
// tv_chunk) converted to FP64 and added.
template <int LMAX, class Bar>
__device__ __forceinline__ double tv_chunk2(const TvChunkIO& P, int tid, float* seg_a, float2* seg_b, float2* bnd,
                                            Bar bar) {
  const int Nt = P.Nt;
  const int seg = tid / kTvChunkPx, px = tid - seg * kTvChunkPx;
  const int Ls = (Nt + kTvSeg - 1) / kTvSeg;
  const int ta = min(Nt, seg * Ls), tb = min(Nt, ta + Ls), n = tb - ta;
  const size_t fs = P.fstride;
  const float2 z2 = make_float2(0.f, 0.f);
  const bool ok0 = 2 * px < P.nvalid, ok1 = 2 * px + 1 < P.nvalid;
  const size_t base = P.base + 2 * px;
  const bool vec = ok1 && ((fs | base) & 1) == 0;
  const bool write = P.write;
  float2 xs[LMAX][2], ms[LMAX][2], ds[LMAX][2], ps[LMAX][2];
  float2 xn[2] = {z2, z2}, mn[2] = {z2, z2}, mp[2] = {z2, z2}, dp[2] = {z2, z2};
  const float2* px_ = P.x + (size_t)ta * fs + base;
  const float2* pm_ = P.m + (size_t)ta * fs + base;
  const float2* pp_ = P.p + (size_t)ta * fs + base;
  const float2* pd_ = P.d1 ? P.d1 + (size_t)ta * fs + base : nullptr;
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    xs[u][0] = xs[u][1] = ms[u][0] = ms[u][1] = ds[u][0] = ds[u][1] = ps[u][0] = ps[u][1] = z2;
    if (ok0 && u < n) {
      ld_pair(px_ + (size_t)u * fs, vec, ok1, xs[u][0], xs[u][1]);
      if (write) {
        ld_pair(pm_ + (size_t)u * fs, vec, ok1, ms[u][0], ms[u][1]);
        ld_pair(pp_ + (size_t)u * fs, vec, ok1, ps[u][0], ps[u][1]);
        if (pd_ && ta + u + 1 < Nt) ld_pair(pd_ + (size_t)u * fs, vec, ok1, ds[u][0], ds[u][1]);
      }
    }
  }
  if (ok0 && n > 0 && tb < Nt) {
    ld_pair(px_ + (size_t)n * fs, vec, ok1, xn[0], xn[1]);
    if (write) ld_pair(pm_ + (size_t)n * fs, vec, ok1, mn[0], mn[1]);
  }
  if (ok0 && n > 0 && ta > 0 && write) {
    ld_pair(pm_ - fs, vec, ok1, mp[0], mp[1]);
    if (pd_) ld_pair(pd_ - fs, vec, ok1, dp[0], dp[1]);
  }
  float tvf[2] = {0.f, 0.f};
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (ok0 && u < n && ta + u + 1 < Nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) tvf[h] += c_abs(c_sub(u + 1 < n ? xs[u + 1][h] : xn[h], xs[u][h]));
  const double tvd = (double)tvf[0] + (double)tvf[1];
  if (!write) return tvd;
  float2 eprev[2] = {z2, z2};
  if (ok0 && n > 0 && ta > 0)
#pragma unroll
    for (int h = 0; h < 2; ++h) eprev[h] = c_sub(dp[h], c_soft(c_add(c_sub(ms[0][h], mp[h]), dp[h]), P.tau1));
#pragma unroll
  for (int u = 0; u < LMAX; ++u)
    if (u < n)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        ds[u][h] = (ta + u + 1 < Nt)
                       ? c_sub(ds[u][h], c_soft(c_add(c_sub(u + 1 < n ? ms[u + 1][h] : mn[h], ms[u][h]), ds[u][h]), P.tau1))
                       : z2;
#pragma unroll
  for (int u = 0; u < LMAX; ++u) {
    if (u < n) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 x_t = xs[u][h], p_t = ps[u][h];
        float2 rhs = c_sub(ds[u][h], u > 0 ? ds[u - 1][h] : eprev[h]);
        rhs.x = fmaf(P.rho, 2.f * x_t.x - p_t.x, rhs.x);
        rhs.y = fmaf(P.rho, 2.f * x_t.y - p_t.y, rhs.y);
        xs[u][h] = rhs;
        ps[u][h] = c_sub(p_t, x_t);
      }
    }
  }
  float inv[LMAX];
#pragma unroll
  for (int u = 0; u < LMAX; ++u) inv[u] = u < n ? __ldg(P.thomas + ta + u) : 0.f;
  const int s0 = seg * kTvChunk2Px + 2 * px;   // this thread's two entries of the segment arrays
  {
    float A = 1.f;
    float2 B[2] = {z2, z2};
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        A *= inv[u];
#pragma unroll
        for (int h = 0; h < 2; ++h) B[h] = c_scale(c_add(xs[u][h], B[h]), inv[u]);
      }
    seg_a[s0] = A;
    seg_a[s0 + 1] = A;
    seg_b[s0] = B[0];
    seg_b[s0 + 1] = B[1];
  }
  bar();
  {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 d = z2;
      for (int q = 0; q < seg; ++q) d = c_add(c_scale(d, seg_a[q * kTvChunk2Px + 2 * px + h]), seg_b[q * kTvChunk2Px + 2 * px + h]);
#pragma unroll
      for (int u = 0; u < LMAX; ++u)
        if (u < n) {
          d = c_scale(c_add(xs[u][h], d), inv[u]);
          ms[u][h] = d;
        }
    }
  }
  bar();
  {
    float A = 1.f;
    float2 B[2] = {z2, z2};
#pragma unroll
    for (int u = LMAX - 1; u >= 0; --u)
      if (u < n) {
#pragma unroll
        for (int h = 0; h < 2; ++h) B[h] = make_float2(fmaf(inv[u], B[h].x, ms[u][h].x), fmaf(inv[u], B[h].y, ms[u][h].y));
        A *= inv[u];
      }
    seg_a[s0] = A;
    seg_a[s0 + 1] = A;
    seg_b[s0] = B[0];
    seg_b[s0 + 1] = B[1];
  }
  bar();
  {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 mm = z2;
      for (int q = kTvSeg - 1; q > seg; --q)
        mm = c_add(c_scale(mm, seg_a[q * kTvChunk2Px + 2 * px + h]), seg_b[q * kTvChunk2Px + 2 * px + h]);
#pragma unroll
      for (int u = LMAX - 1; u >= 0; --u)
        if (u < n) {
          mm = make_float2(fmaf(inv[u], mm.x, ms[u][h].x), fmaf(inv[u], mm.y, ms[u][h].y));
          ms[u][h] = mm;
        }
      bnd[s0 + h] = n > 0 ? ms[0][h] : z2;
    }
  }
  bar();
  if (ok0) {
    float2 mnext[2] = {z2, z2};
    if (tb < Nt) {
      mnext[0] = bnd[(seg + 1) * kTvChunk2Px + 2 * px];
      mnext[1] = bnd[(seg + 1) * kTvChunk2Px + 2 * px + 1];
    }
    float2* qm = P.m_out + (size_t)ta * fs + base;
    float2* qp = P.p_out + (size_t)ta * fs + base;
    float2* qd = P.d1_out + (size_t)ta * fs + base;
#pragma unroll
    for (int u = 0; u < LMAX; ++u)
      if (u < n) {
        st_pair(qm + (size_t)u * fs, vec, ok1, ms[u][0], ms[u][1]);
        st_pair(qp + (size_t)u * fs, vec, ok1, c_add(ms[u][0], ps[u][0]), c_add(ms[u][1], ps[u][1]));
        if (ta + u + 1 < Nt) {
          const float2 e0 = c_add(ds[u][0], c_sub(u + 1 < n ? ms[u + 1][0] : mnext[0], ms[u][0]));
          const float2 e1 = c_add(ds[u][1], c_sub(u + 1 < n ? ms[u + 1][1] : mnext[1], ms[u][1]));
          st_pair(qd + (size_t)u * fs, vec, ok1, e0, e1);
        }
      }
  }
  return tvd;
}

}  // namespace recon
