// Per-iteration kernels of Algorithms 1 and 2.
//
// k_col_inverse  x_{i,t} = A_{i,t} r_{i,t} for every column (Section IV-C,
//                Eq. eigen_mu; Algorithm 2 x-update, Algorithm 1 w-update),
//                with the data term of J(k) for the new x fused into the
//                epilogue (Eq. r_ratio needs J(k)).
// k_tv_temporal  v, m and d1 updates of Algorithm 2 along t for every pixel.
// k_dft_temporal v-update, dual and Psi / Psi' of Algorithm 1 along t.
// k_objective    ||y - Hx||^2 of a given field (J(0)).
// k_finalize     J(k) = fid + lambda * prior, Delta(k) and the stop flag.
#include "kernels.h"

namespace recon {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kColThreads = kConsumers + 96;  // + producer, r loader, column manager
constexpr int kStageBytes = kRectElems * 8;   // largest unit (FP32 rect)

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// One off-diagonal 32x32 block (rows p*32.., cols q*32..): lane (lr, lc)
// holds rows lr*4..+3 and cols lc*8..+7.  Row sums are reduced over the 4
// lanes sharing lr, column sums (with conj, the lower triangle) over the 8
// lanes sharing lc, by butterfly exchanges that leave one total per lane.
template <typename E>
__device__ __forceinline__ void proc_tile(const E* __restrict__ tl, const float2* __restrict__ r,
                                          float2* __restrict__ yw, int p, int q, int lane) {
  const int lr = lane >> 2, lc = lane & 3;
  float2 rv[4], cv[8];
  {
    const float4* r4 = reinterpret_cast<const float4*>(r + p * 32 + lr * 4);
    float4 a0 = r4[0], a1 = r4[1];
    rv[0] = make_float2(a0.x, a0.y); rv[1] = make_float2(a0.z, a0.w);
    rv[2] = make_float2(a1.x, a1.y); rv[3] = make_float2(a1.z, a1.w);
    const float4* c4 = reinterpret_cast<const float4*>(r + q * 32 + lc * 8);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 c = c4[k];
      cv[2 * k] = make_float2(c.x, c.y); cv[2 * k + 1] = make_float2(c.z, c.w);
    }
  }
  float2 rowp[4], colp[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) rowp[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) colp[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int qq = 0; qq < 16; ++qq) {
    float2 e0, e1;
    Elem<E>::load2(tl + qq * 64 + lane * 2, e0, e1);
    const int ri = qq >> 2, c0 = (qq & 3) * 2;
    c_fma(rowp[ri], e0, cv[c0]);
    c_fma(rowp[ri], e1, cv[c0 + 1]);
    c_fmac(colp[c0], e0, rv[ri]);
    c_fmac(colp[c0 + 1], e1, rv[ri]);
  }
  // rows: lanes differing in bits 0,1
  const bool b1 = (lc & 2) != 0, b0 = (lc & 1) != 0;
  float2 k0 = b1 ? rowp[2] : rowp[0], s0 = b1 ? rowp[0] : rowp[2];
  float2 k1 = b1 ? rowp[3] : rowp[1], s1 = b1 ? rowp[1] : rowp[3];
  k0 = c_add(k0, shfl_xor2(s0, 2));
  k1 = c_add(k1, shfl_xor2(s1, 2));
  float2 kr = b0 ? k1 : k0, sr = b0 ? k0 : k1;
  kr = c_add(kr, shfl_xor2(sr, 1));
  // columns: lanes differing in bits 2,3,4
  const bool c2 = (lr & 4) != 0, c1 = (lr & 2) != 0, cb = (lr & 1) != 0;
  float2 h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 keep = c2 ? colp[k + 4] : colp[k], send = c2 ? colp[k] : colp[k + 4];
    h[k] = c_add(keep, shfl_xor2(send, 16));
  }
  float2 g[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float2 keep = c1 ? h[k + 2] : h[k], send = c1 ? h[k] : h[k + 2];
    g[k] = c_add(keep, shfl_xor2(send, 8));
  }
  float2 kc = cb ? g[1] : g[0], sc = cb ? g[0] : g[1];
  kc = c_add(kc, shfl_xor2(sc, 4));
  float2* yr = yw + p * 32 + lane;            // row lr*4 + lc == lane
  *yr = c_add(*yr, kr);
  float2* yc = yw + q * 32 + lc * 8 + lr;      // column lc*8 + lr
  *yc = c_add(*yc, kc);
  __syncwarp();
}

// A pair of diagonal blocks P = block p, Q = block q in one 32 x 33 cell
// array (see kernels.h).  Pass 1: lane a walks row a (row sums of P, column
// sums of Q).  Pass 2: lane l walks column l+1 (column sums of P, row sums of
// Q); column 0 (row 0 of Q) is reduced across the warp.  The skewed layout
// makes both passes free of bank conflicts.
template <typename E>
__device__ __forceinline__ void proc_rect(const E* __restrict__ tl, const float2* __restrict__ r,
                                          float2* __restrict__ yw, int p, int q, int lane) {
  const float2* rP = r + p * 32;
  const float2* rQ = r + q * 32;
  float2 rowP = make_float2(0.f, 0.f), colQ = make_float2(0.f, 0.f);
#pragma unroll 11
  for (int b = 0; b < 33; ++b) {
    float2 e = Elem<E>::load(tl + b * 32 + ((lane + b) & 31));
    if (b > lane) c_fma(rowP, e, rP[b - 1]);      // P[lane][b-1], b-1 >= lane
    else c_fmac(colQ, e, rQ[b]);                   // Q[b][lane], b <= lane
  }
  float2 colP = make_float2(0.f, 0.f), rowQ = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int a = 0; a < 32; ++a) {
    float2 e = Elem<E>::load(tl + (lane + 1) * 32 + ((a + lane + 1) & 31));
    if (a < lane) c_fmac(colP, e, rP[a]);          // P[a][lane], a < lane
    else if (a > lane + 1) c_fma(rowQ, e, rQ[a]);  // Q[lane+1][a], a > lane+1
  }
  float2 t0 = make_float2(0.f, 0.f);
  {
    float2 e = Elem<E>::load(tl + lane);           // cell (lane, 0) = Q[0][lane]
    if (lane > 0) t0 = c_mul(e, rQ[lane]);
  }
  t0 = warp_sum2(t0);
  float2* y1 = yw + p * 32 + lane;
  *y1 = c_add(*y1, c_add(rowP, colP));
  __syncwarp();
  float2 add = colQ;
  if (lane == 0) add = c_add(add, t0);
  float2* y2 = yw + q * 32 + lane;
  *y2 = c_add(*y2, add);
  __syncwarp();
  if (lane < 31) {
    float2* y3 = yw + q * 32 + lane + 1;
    *y3 = c_add(*y3, rowQ);
  }
  __syncwarp();
}

// ||y - H x||^2 of one column (i, t) whose values are in shared memory:
// for each coil, z = F_v(s_c . x) (unitary, batched FFT of `ncg` coils at a
// time) compared with the hybrid data F_h'y on the sampled rows.  By
// Parseval on F_h this is the column's share of ||y - Hx||^2.
template <class Bar>
__device__ double column_fid(const float2* xcol, int i, int t, int Nx, int Ny, int Nc, int ncg,
                             const float2* __restrict__ sens, const float2* __restrict__ yhat,
                             const int* __restrict__ rows, const int* __restrict__ rowoff, const FftPlanDev& fy,
                             float scl, float2* fa, float2* fb, int tid, int nthr, Bar bar) {
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  const int* rw = rows + r0;
  const float2* yh = yhat + (size_t)r0 * Nx * Nc + (size_t)i * Nc * mt;
  const float2* sc = sens + (size_t)i * Nc * Ny;
  double acc = 0.0;
  for (int c0 = 0; c0 < Nc; c0 += ncg) {
    const int cg = min(ncg, Nc - c0);
    for (int idx = tid; idx < cg * Ny; idx += nthr) {
      const int c = idx / Ny, j = idx - c * Ny;
      fa[idx] = c_mul(__ldg(sc + (size_t)(c0 + c) * Ny + j), xcol[j]);
    }
    bar();
    float2* res = fft_run(fa, fb, cg, Ny, 1, fy, false, tid, nthr, bar);
    for (int idx = tid; idx < cg * mt; idx += nthr) {
      const int c = idx / mt, m = idx - c * mt;
      float2 z = c_scale(res[c * Ny + rw[m]], scl);
      float2 d = c_sub(__ldg(yh + (size_t)(c0 + c) * mt + m), z);
      acc += c_abs2d(d);
    }
    bar();
  }
  return acc;
}

struct ConsumerBar {
  __device__ __forceinline__ void operator()() const { named_bar_sync(1, kConsumers); }
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kRSlots = 2;  // double-buffered r inputs / partial sums

struct ColLayout {
  size_t bars, ring, ycopy, rvec, bvec, rslot, units, total;
};
__host__ __device__ inline ColLayout col_layout(int stages, int nb, int nunits) {
  ColLayout L;
  const size_t ny32 = (size_t)(nb + 1) * 32;
  size_t o = 0;
  // full[S], empty[S], rfull[2], rempty[2], rv_full[2], yc_empty[2], col_done[2]
  L.bars = o; o += (2 * (size_t)stages + 5 * kRSlots) * 8;
  o = align_up(o, 128);
  L.ring = o; o += (size_t)stages * kStageBytes;
  o = align_up(o, 16);
  L.ycopy = o; o += (size_t)kRSlots * kConsumerWarps * ny32 * 8;   // [buf][warp][ny32]
  L.rvec = o; o += (size_t)kRSlots * ny32 * 8;
  L.bvec = o; o += (size_t)kRSlots * ny32 * 8;
  L.rslot = o; o += (size_t)kRSlots * 3 * ny32 * 8;   // [slot][base, add, b][ny32]
  L.units = o; o += (size_t)nunits * 16;
  L.total = align_up(o, 128);
  return L;
}

// Persistent column-inverse kernel, warp-specialised and free of block-wide
// barriers in the main loop (all hand-offs are bounded mbarrier waits):
//   warp 8   producer: streams the packed inverses with the TMA engine
//            (cp.async.bulk, L2 evict_first) into a ring of S stages
//   warp 9   r loader: bulk-copies each column's right-hand-side inputs
//   warp 10  column manager: r = base + coef*add into rvec[n&1]; after the
//            consumers are done, x = sum of the 8 partial y vectors, store,
//            objective dot products, clear the partials
//   warps 0-7 consumers: Hermitian matvec of each unit into their own
//            partial y vector of buffer n&1, column after column
template <typename E>
__global__ void __launch_bounds__(kColThreads, 1) k_col_inverse(ColParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (P.flags[FLAG_STOP]) return;
  const ColLayout L = col_layout(P.stages, P.nb, P.nunits);
  const int S = P.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  uint64_t* rfull = empty + S;
  uint64_t* rempty = rfull + kRSlots;
  uint64_t* rv_full = rempty + kRSlots;
  uint64_t* yc_empty = rv_full + kRSlots;
  uint64_t* col_done = yc_empty + kRSlots;
  unsigned char* ring = smem + L.ring;
  const int ny32 = (P.nb + 1) * 32;
  float2* ycopy = reinterpret_cast<float2*>(smem + L.ycopy);
  float2* rvec = reinterpret_cast<float2*>(smem + L.rvec);
  float2* bvec = reinterpret_cast<float2*>(smem + L.bvec);
  float2* rslot = reinterpret_cast<float2*>(smem + L.rslot);
  int4* units = reinterpret_cast<int4*>(smem + L.units);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int u = tid; u < P.nunits; u += blockDim.x) units[u] = P.units[u];
  for (int j = tid; j < kRSlots * kConsumerWarps * ny32; j += blockDim.x) ycopy[j] = make_float2(0.f, 0.f);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int s = 0; s < kRSlots; ++s) {
      mbar_init(&rfull[s], P.r_tma ? 1 : 32);
      mbar_init(&rempty[s], 1);
      mbar_init(&rv_full[s], 1);
      mbar_init(&yc_empty[s], 1);
      mbar_init(&col_done[s], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  constexpr int ES = Elem<E>::bytes;
  const bool sep_b = P.do_obj && P.bsrc != P.base;

  if (warp == kConsumerWarps) {
    // ---------------- producer: stream packed inverses into the ring --------
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      const unsigned char* Ab = reinterpret_cast<const unsigned char*>(P.A);
      // stage st of the ring, wraps = completed passes over the ring (no
      // divisions on the issue path)
      int st = 0, wraps = 0;
      bool ok = true;
      for (int col = blockIdx.x; col < P.ncols && ok; col += gridDim.x) {
        const unsigned char* cb = Ab + (size_t)col * (size_t)P.col_elems * ES;
        for (int u = 0; u < P.nunits; ++u) {
          if (wraps > 0 && !mbar_wait(&empty[st], (uint32_t)((wraps - 1) & 1), P.flags)) { ok = false; break; }
          const int4 un = units[u];
          const uint32_t bytes = (uint32_t)((un.x == UNIT_TILE ? kTileElems : kRectElems) * ES);
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(ring + (size_t)st * kStageBytes, cb + (size_t)un.w * ES, bytes, &full[st], pol);
          if (++st == S) { st = 0; ++wraps; }
        }
      }
      if (!ok) {
        // error path: let every copy still in flight land before the CTA exits
        const long long g = (long long)wraps * S + st;
        for (long long h = (g > S ? g - S : 0); h < g; ++h) {
          uint64_t* bb = &full[h % S];
          const uint32_t par = (uint32_t)((h / S) & 1);
          unsigned long long t0 = global_ns();
          while (!mbar_try_wait(bb, par) && global_ns() - t0 < kWaitLimitNs) {}
        }
      }
    }
    return;
  }
  if (warp == kConsumerWarps + 1) {
    // ---------------- r loader: each column's inputs into a slot -------------
    // With 16-byte aligned columns (Ny even) one lane moves them with the TMA
    // engine; otherwise all lanes load them (unrolled) and arrive.
    int n = 0;
    for (int col = blockIdx.x; col < P.ncols; col += gridDim.x, ++n) {
      const int sl = n % kRSlots;
      if (n >= kRSlots && !mbar_wait(&rempty[sl], (uint32_t)(((n / kRSlots) - 1) & 1), P.flags)) break;
      float2* d = rslot + (size_t)sl * 3 * ny32;
      const size_t cofs = (size_t)col * P.Ny;
      if (P.r_tma) {
        if (lane == 0) {
          const uint32_t bytes = (uint32_t)P.Ny * 8u;
          const uint32_t total = bytes * (1u + (P.add ? 1u : 0u) + (sep_b ? 1u : 0u));
          const uint64_t pol = policy_evict_first();
          mbar_arrive_expect_tx(&rfull[sl], total);
          bulk_g2s(d, P.base + cofs, bytes, &rfull[sl], pol);
          if (P.add) bulk_g2s(d + ny32, P.add + cofs, bytes, &rfull[sl], pol);
          if (sep_b) bulk_g2s(d + 2 * ny32, P.bsrc + cofs, bytes, &rfull[sl], pol);
        }
      } else {
        for (int j0 = 0; j0 < P.Ny; j0 += 32 * 8) {
          float2 va[8], vb[8], vc[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + q * 32 + lane;
            if (j < P.Ny) {
              va[q] = P.base[cofs + j];
              if (P.add) vb[q] = P.add[cofs + j];
              if (sep_b) vc[q] = P.bsrc[cofs + j];
            }
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + q * 32 + lane;
            if (j < P.Ny) {
              d[j] = va[q];
              if (P.add) d[ny32 + j] = vb[q];
              if (sep_b) d[2 * ny32 + j] = vc[q];
            }
          }
        }
        mbar_arrive(&rfull[sl]);
      }
    }
    if (P.r_tma && lane == 0) {
      // copies of the last slots may still be in flight if the kernel quits early
      for (int h = (n > kRSlots ? n - kRSlots : 0); h < n; ++h) {
        unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&rfull[h % kRSlots], (uint32_t)((h / kRSlots) & 1)) && global_ns() - t0 < kWaitLimitNs) {}
      }
    }
    return;
  }
  if (warp == kConsumerWarps + 2) {
    // ---------------- column manager -----------------------------------------
    // prepare(n): rvec[n&1] = base + coef*add (zero padded), bvec[n&1] = b
    auto prepare = [&](int n) -> bool {
      const int sl = n % kRSlots;
      if (!mbar_wait(&rfull[sl], (uint32_t)((n / kRSlots) & 1), P.flags)) return false;
      const float2* d = rslot + (size_t)sl * 3 * ny32;
      float2* rv = rvec + (size_t)(n & 1) * ny32;
      float2* bv = bvec + (size_t)(n & 1) * ny32;
      for (int j = lane; j < ny32; j += 32) {
        float2 v = make_float2(0.f, 0.f), bb = make_float2(0.f, 0.f);
        if (j < P.Ny) {
          v = d[j];
          bb = sep_b ? d[2 * ny32 + j] : v;
          if (P.add) {
            const float2 a = d[ny32 + j];
            v.x = fmaf(P.coef, a.x, v.x); v.y = fmaf(P.coef, a.y, v.y);
          }
        }
        rv[j] = v;
        bv[j] = bb;
      }
      __syncwarp();
      if (lane == 0) { mbar_arrive(&rempty[sl]); mbar_arrive(&rv_full[n & 1]); }
      return true;
    };
    int ncol = 0;
    for (int col = blockIdx.x; col < P.ncols; col += gridDim.x) ++ncol;
    double fid = 0.0;
    bool ok = true;
    for (int n = 0; n < ncol && n < kRSlots && ok; ++n) ok = prepare(n);
    for (int n = 0; n < ncol && ok; ++n) {
      const int bb = n & 1;
      if (!mbar_wait(&col_done[bb], (uint32_t)((n >> 1) & 1), P.flags)) break;
      const size_t cofs = (size_t)(blockIdx.x + (size_t)n * gridDim.x) * P.Ny;
      float2* yc = ycopy + (size_t)bb * kConsumerWarps * ny32;
      const float2* rv = rvec + (size_t)bb * ny32;
      const float2* bv = bvec + (size_t)bb * ny32;
      for (int j = lane; j < ny32; j += 32) {
        float2 x = yc[j];
        yc[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 1; w < kConsumerWarps; ++w) {
          x = c_add(x, yc[(size_t)w * ny32 + j]);
          yc[(size_t)w * ny32 + j] = make_float2(0.f, 0.f);
        }
        if (j < P.Ny) {
          P.xout[cofs + j] = x;
          if (P.do_obj) {
            const float2 r = rv[j], b = bv[j];
            // -2 Re<b, x> + Re<x, r> - mu |x|^2
            fid += -2.0 * ((double)b.x * x.x + (double)b.y * x.y) + ((double)x.x * r.x + (double)x.y * r.y) -
                   (double)P.mu * ((double)x.x * x.x + (double)x.y * x.y);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&yc_empty[bb]);
      if (n + kRSlots < ncol) ok = prepare(n + kRSlots);
    }
    if (P.do_obj) {
      fid = warp_sum(fid);
      if (lane == 0) atomicAdd(P.fid_acc, fid);
    }
    return;
  }

  // ---------------- consumers (8 warps) --------------------------------------
  // Unit g (counted across this CTA's columns) belongs to warp g mod 8, so a
  // warp walks g = warp, warp+8, ...: within column n that is unit index u,
  // and its ring stage advances by 8 per unit.  With S a multiple of 8 the
  // previous fill of a stage was consumed by this same warp, so every parity
  // wait is at most one phase ahead of its barrier.  Every column's rv/yc
  // barriers are waited on (and col_done arrived at) even when the warp has
  // no unit in that column, for the same reason.
  int ncol = 0;
  for (int col = blockIdx.x; col < P.ncols; col += gridDim.x) ++ncol;
  int u = warp, st = warp;
  uint32_t ph = 0;
  for (int n = 0; n < ncol; ++n) {
    const int bb = n & 1;
    if (!mbar_wait(&rv_full[bb], (uint32_t)((n >> 1) & 1), P.flags)) break;
    if (n >= 2 && !mbar_wait(&yc_empty[bb], (uint32_t)(((n >> 1) - 1) & 1), P.flags)) break;
    const float2* rv = rvec + (size_t)bb * ny32;
    float2* yw = ycopy + ((size_t)bb * kConsumerWarps + warp) * ny32;
    bool failed = false;
    for (; u < P.nunits; u += kConsumerWarps) {
      if (!mbar_wait(&full[st], ph, P.flags)) { failed = true; break; }
      const int4 un = units[u];
      const E* tl = reinterpret_cast<const E*>(ring + (size_t)st * kStageBytes);
      if (un.x == UNIT_TILE) proc_tile<E>(tl, rv, yw, un.y, un.z, lane);
      else proc_rect<E>(tl, rv, yw, un.y, un.z, lane);
      if (lane == 0) mbar_arrive(&empty[st]);
      st += kConsumerWarps;
      if (st >= S) { st -= S; ph ^= 1u; }
    }
    if (failed) break;
    u -= P.nunits;
    if (lane == 0) mbar_arrive(&col_done[bb]);
  }
}

size_t col_inverse_smem(const ColParams& p, int) { return col_layout(p.stages, p.nb, p.nunits).total; }

// Largest ring depth that fits, a multiple of the consumer warp count (the
// parity waits rely on it; see the consumer loop).
int col_inverse_max_stages(const ColParams& p, int storage) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int s = 4 * kConsumerWarps;
  while (s > kConsumerWarps) {
    ColParams q = p;
    q.stages = s;
    if (col_inverse_smem(q, storage) + 1024 <= (size_t)optin) break;
    s -= kConsumerWarps;
  }
  return s;
}

int col_inverse_stage_quantum() { return kConsumerWarps; }

template <typename E>
static cudaError_t launch_col_t(const ColParams& p, int grid, size_t smem, cudaStream_t s) {
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_col_inverse<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_col_inverse<E><<<grid, kColThreads, smem, s>>>(p); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_col_inverse(const ColParams& p, int storage, int grid, size_t smem, cudaStream_t s) {
  switch (storage) {
    case 0: return launch_col_t<float2>(p, grid, smem, s);
    case 1: return launch_col_t<__half2>(p, grid, smem, s);
    case 2: return launch_col_t<__nv_bfloat162>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Algorithm 2 temporal step, one thread per pixel over a tile of kTvPix
// pixels (column layout keeps a tile's pixels contiguous for every t):
//   v  = S(D_t m + d1, lambda/(2 mu1))
//   m' = (rho I + D_t'D_t)^{-1} [D_t'(v - d1) + rho (x + d2)]    (Thomas)
//   d1' = d1 - (v - D_t m')
// with d2 = x - p, and p' = m' - d2 handed to the inverse step, which forms
// r = H'y + mu2 (m' - d2) = b + mu2 p'.  The next d2 is then x' - p'.
// The tile's inputs are staged in shared memory with asynchronous copies
// (all in flight at once), then both sweeps run from shared memory.  Also
// accumulates ||D_t x||_1 of the incoming x (the prior term of J).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_tv_temporal(TvParams P) {
  extern __shared__ __align__(16) float2 sm_tv[];
  __shared__ double red[32];
  if (P.flags[FLAG_STOP]) return;
  const int tid = threadIdx.x, PX = blockDim.x, Nt = P.Nt;
  const long long N = P.npix;
  const long long pix0 = (long long)blockIdx.x * PX;
  const int npx = (int)min((long long)PX, N - pix0);
  // [Nt][PX] tiles: m, d1, x (later e = d1 - v), p (later f = p - x), d'
  float2* sm_m = sm_tv;
  float2* sm_d1 = sm_m + (size_t)Nt * PX;
  float2* sm_x = sm_d1 + (size_t)Nt * PX;
  float2* sm_p = sm_x + (size_t)Nt * PX;
  float2* sm_dp = sm_p + (size_t)Nt * PX;
  if (tid < npx) {
    for (int t = 0; t < Nt; ++t) {
      const long long g = t * N + pix0 + tid;
      cp_async8(&sm_x[t * PX + tid], P.x + g);
      if (P.write_state) {
        cp_async8(&sm_m[t * PX + tid], P.m + g);
        cp_async8(&sm_p[t * PX + tid], P.p + g);
        if (P.d1 && t + 1 < Nt) cp_async8(&sm_d1[t * PX + tid], P.d1 + g);
      }
    }
  }
  cp_async_wait_all();
  double tv = 0.0;
  if (tid < npx) {
    float2 x_prev = sm_x[tid];
    for (int t = 1; t < Nt; ++t) {
      const float2 x_t = sm_x[t * PX + tid];
      tv += (double)c_abs(c_sub(x_t, x_prev));
      x_prev = x_t;
    }
    if (P.write_state) {
      float2 m_t = sm_m[tid];
      float2 e_prev = make_float2(0.f, 0.f), d_prev = make_float2(0.f, 0.f);
      for (int t = 0; t < Nt; ++t) {
        const float2 x_t = sm_x[t * PX + tid], p_t = sm_p[t * PX + tid];
        float2 e_t = make_float2(0.f, 0.f), m_n = make_float2(0.f, 0.f);
        if (t + 1 < Nt) {
          m_n = sm_m[(t + 1) * PX + tid];
          const float2 d1_t = P.d1 ? sm_d1[t * PX + tid] : make_float2(0.f, 0.f);
          const float2 v = c_soft(c_add(c_sub(m_n, m_t), d1_t), P.tau1);
          e_t = c_sub(d1_t, v);
        }
        // rhs = D'(v - d1) + rho (x + d2),  (D'u)_t = u_{t-1} - u_t,  u = -e
        float2 rhs = c_sub(e_t, e_prev);
        rhs.x = fmaf(P.rho, 2.f * x_t.x - p_t.x, rhs.x);
        rhs.y = fmaf(P.rho, 2.f * x_t.y - p_t.y, rhs.y);
        const float inv = __ldg(P.thomas + t);
        const float2 dp = c_scale(c_add(rhs, d_prev), inv);
        sm_dp[t * PX + tid] = dp;
        sm_x[t * PX + tid] = e_t;               // x no longer needed: keep e
        sm_p[t * PX + tid] = c_sub(p_t, x_t);   // keep f = p - x
        d_prev = dp; e_prev = e_t; m_t = m_n;
      }
      float2 mnext = make_float2(0.f, 0.f);
      for (int t = Nt - 1; t >= 0; --t) {
        const float inv = __ldg(P.thomas + t);
        const float2 dp = sm_dp[t * PX + tid];
        const float2 mt = make_float2(fmaf(inv, mnext.x, dp.x), fmaf(inv, mnext.y, dp.y));
        const long long g = t * N + pix0 + tid;
        if (t + 1 < Nt) P.d1_out[g] = c_add(sm_x[t * PX + tid], c_sub(mnext, mt));
        P.p_out[g] = c_add(mt, sm_p[t * PX + tid]);
        P.m_out[g] = mt;
        mnext = mt;
      }
    }
  }
  const double s = group_sum(tv, red, tid, PX, BlockBar());
  if (tid == 0) atomicAdd(P.prior_acc, s);
}

cudaError_t launch_tv_temporal(const TvParams& p, cudaStream_t s) {
  // five [Nt][PX] complex tiles must fit (Nt <= 128)
  int px = 64;
  while (px > 32 && 5 * (size_t)p.Nt * px * sizeof(float2) > 200 * 1024) px >>= 1;
  const size_t smem = 5 * (size_t)p.Nt * px * sizeof(float2);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_tv_temporal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const long long grid = (p.npix + px - 1) / px;
  k_tv_temporal<<<(unsigned)grid, px, smem, s>>>(p); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1 temporal step for 64 pixels per block (tile [Nt][64] in shared
// memory, batched Stockham along t):
//   w = Psi xhat,  d = u - w  (d = 0 at k = 1),  v = S(w - d, lambda/(2 mu)),
//   u' = v + d,  r = H'y + mu Psi'(u')
// so the inverse step gives xhat' = A r and Psi xhat' is the new w.  Because
// Psi is unitary, the (I - Psi Psi') term of the w-update is zero.  Also
// accumulates ||w||_1 (the prior term of J at the incoming iterate).
// ---------------------------------------------------------------------------
constexpr int kDftPix = 64;
__global__ void __launch_bounds__(256) k_dft_temporal(DftParams P) {
  extern __shared__ float2 sm_dft[];
  __shared__ double red[32];
  if (P.flags[FLAG_STOP]) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nt = P.Nt;
  float2* A = sm_dft;
  float2* B = sm_dft + (size_t)Nt * kDftPix;
  const long long N = P.npix;
  const long long pix0 = (long long)blockIdx.x * kDftPix;
  const int npx = (int)min((long long)kDftPix, N - pix0);
  for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
    const int t = idx / kDftPix, pp = idx - t * kDftPix;
    if (pp < npx) cp_async8(&A[idx], P.xh + t * N + pix0 + pp);
    else A[idx] = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  const BlockBar bar;
  float2* W = fft_run(A, B, kDftPix, 1, kDftPix, P.ft, false, tid, nth, bar);
  float2* O = (W == A) ? B : A;
  const float sc = rsqrtf((float)Nt);
  double l1 = 0.0;
  for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
    const int t = idx / kDftPix, pp = idx - t * kDftPix;
    float2 uo = make_float2(0.f, 0.f);
    if (pp < npx) {
      const float2 w = c_scale(W[idx], sc);
      l1 += (double)c_abs(w);
      if (P.write_state) {
        const float2 d = P.first ? make_float2(0.f, 0.f) : c_sub(P.u[t * N + pix0 + pp], w);
        const float2 v = c_soft(c_sub(w, d), P.tau);
        uo = c_add(v, d);
        P.u_out[t * N + pix0 + pp] = uo;
      }
    }
    O[idx] = uo;
  }
  __syncthreads();
  if (P.write_state) {
    float2* S = fft_run(O, W, kDftPix, 1, kDftPix, P.ft, true, tid, nth, bar);
    const float ms = P.mu * sc;
    for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
      const int t = idx / kDftPix, pp = idx - t * kDftPix;
      if (pp < npx) {
        const float2 bb = P.b[t * N + pix0 + pp];
        const float2 sv = S[idx];
        P.r_out[t * N + pix0 + pp] = make_float2(fmaf(ms, sv.x, bb.x), fmaf(ms, sv.y, bb.y));
      }
    }
  }
  const double s = group_sum(l1, red, tid, nth, bar);
  if (tid == 0) atomicAdd(P.prior_acc, s);
}

cudaError_t launch_dft_temporal(const DftParams& p, cudaStream_t s) {
  const size_t smem = 2 * (size_t)p.Nt * kDftPix * sizeof(float2);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_dft_temporal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const long long grid = (p.npix + kDftPix - 1) / kDftPix;
  k_dft_temporal<<<(unsigned)grid, 256, smem, s>>>(p); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||y - H x||^2 of a whole field, one block per column.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_objective(ObjParams P) {
  extern __shared__ float2 sm_obj[];
  __shared__ double red[32];
  if (P.flags[FLAG_STOP]) return;
  const int col = blockIdx.x, tid = threadIdx.x;
  const int t = col / P.Nx, i = col - t * P.Nx;
  float2* xc = sm_obj;
  float2* fa = xc + P.Ny;
  float2* fb = fa + (size_t)P.ncg * P.Ny;
  for (int j = tid; j < P.Ny; j += blockDim.x) xc[j] = P.x[(size_t)col * P.Ny + j];
  __syncthreads();
  const double f = column_fid(xc, i, t, P.Nx, P.Ny, P.Nc, P.ncg, P.sens, P.yhat, P.rows, P.rowoff, P.fy,
                              rsqrtf((float)P.Ny), fa, fb, tid, blockDim.x, BlockBar());
  const double s = group_sum(f, red, tid, blockDim.x, BlockBar());
  if (tid == 0) atomicAdd(P.fid_acc, s);
}

cudaError_t launch_objective(const ObjParams& p, cudaStream_t s) {
  const size_t smem = ((size_t)p.Ny + 2 * (size_t)p.ncg * p.Ny) * sizeof(float2);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_objective, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_objective<<<p.Nx * p.Nt, 256, smem, s>>>(p); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// J(k) = ||y - Hx||^2 + lambda * prior, Delta(k) (Eq. r_ratio) and the stop
// flag: later launches see flags[FLAG_STOP] and return at once.
// ---------------------------------------------------------------------------
__global__ void k_finalize(const double* fid, const double* prior, const double* yy, double* J, int k, float lam,
                           double tol, int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (flags[FLAG_STOP]) return;
  const double Jk = fid[k] + (yy ? *yy : 0.0) + (double)lam * prior[k];
  J[k] = Jk;
  if (!isfinite(Jk)) atomicOr(&flags[FLAG_ERR], DEV_ERR_NONFINITE);
  if (tol > 0.0 && k >= 1) {
    const double d = (J[k - 1] - Jk) / Jk;
    if (d >= 0.0 && d < tol) {
      flags[FLAG_ITERS] = k;
      flags[FLAG_STOP] = 1;
    }
  }
}

cudaError_t launch_finalize(const double* fid, const double* prior, const double* yy, double* J, int k, float lam,
                            double tol, int* flags, cudaStream_t s) {
  k_finalize<<<1, 32, 0, s>>>(fid, prior, yy, J, k, lam, tol, flags); note_launch();
  return cudaGetLastError();
}

}  // namespace recon
