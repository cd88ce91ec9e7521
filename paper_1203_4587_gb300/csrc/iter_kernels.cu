// Per-iteration kernels of Algorithms 1 and 2.
//
// k_col_inverse  x_{i,t} = A_{i,t} r_{i,t} for every column (Section IV-C,
//                Eq. eigen_mu; Algorithm 2 x-update, Algorithm 1 w-update),
//                with the objective's data term ||y - Hx||^2 of the new x
//                fused into the epilogue (Eq. r_ratio needs J(k)).
// k_tv_temporal  v, m and d1 updates of Algorithm 2 along t for every pixel.
// k_dft_temporal v-update, dual and Psi / Psi' of Algorithm 1 along t.
// k_objective    ||y - Hx||^2 of a given field (J(0)).
// k_finalize     J(k) = fid + lambda * prior, Delta(k) and the stop flag.
#include "kernels.h"

namespace recon {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kColThreads = kConsumers + 32;  // + one producer warp
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

struct ColLayout {
  size_t bars, ring, ycopy, rvec, xcol, units, red, fa, fb, total;
};
__host__ __device__ inline ColLayout col_layout(int stages, int nb, int nunits, int ncg, int Ny, int do_obj) {
  ColLayout L;
  const size_t ny32 = (size_t)(nb + 1) * 32;
  size_t o = 0;
  L.bars = o; o += 2 * (size_t)stages * 8;
  o = align_up(o, 128);
  L.ring = o; o += (size_t)stages * kStageBytes;
  o = align_up(o, 16);
  L.ycopy = o; o += (size_t)kConsumerWarps * ny32 * 8;
  L.rvec = o; o += ny32 * 8;
  L.xcol = o; o += ny32 * 8;
  L.units = o; o += (size_t)nunits * 16;
  L.red = o; o += 32 * 8;
  L.fa = o; o += do_obj ? (size_t)ncg * Ny * 8 : 0;
  L.fb = o; o += do_obj ? (size_t)ncg * Ny * 8 : 0;
  L.total = align_up(o, 128);
  return L;
}

template <typename E>
__global__ void __launch_bounds__(kColThreads, 1) k_col_inverse(ColParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (P.flags[FLAG_STOP]) return;
  const ColLayout L = col_layout(P.stages, P.nb, P.nunits, P.ncg, P.Ny, P.do_obj);
  const int S = P.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  unsigned char* ring = smem + L.ring;
  const int ny32 = (P.nb + 1) * 32;
  float2* ycopy = reinterpret_cast<float2*>(smem + L.ycopy);
  float2* rvec = reinterpret_cast<float2*>(smem + L.rvec);
  float2* xcol = reinterpret_cast<float2*>(smem + L.xcol);
  int4* units = reinterpret_cast<int4*>(smem + L.units);
  double* red = reinterpret_cast<double*>(smem + L.red);
  float2* fa = reinterpret_cast<float2*>(smem + L.fa);
  float2* fb = reinterpret_cast<float2*>(smem + L.fb);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int u = tid; u < P.nunits; u += blockDim.x) units[u] = P.units[u];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  constexpr int ES = Elem<E>::bytes;

  if (warp == kConsumerWarps) {
    // ---------------- producer: stream packed inverses into the ring --------
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      const unsigned char* Ab = reinterpret_cast<const unsigned char*>(P.A);
      long long g = 0;
      bool ok = true;
      for (int col = blockIdx.x; col < P.ncols && ok; col += gridDim.x) {
        const unsigned char* cb = Ab + (size_t)col * (size_t)P.col_elems * ES;
        for (int u = 0; u < P.nunits; ++u) {
          const int st = (int)(g % S);
          if (g >= S && !mbar_wait(&empty[st], (uint32_t)(((g / S) - 1) & 1), P.flags)) { ok = false; break; }
          const int4 un = units[u];
          const uint32_t bytes = (uint32_t)((un.x == UNIT_TILE ? kTileElems : kRectElems) * ES);
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(ring + (size_t)st * kStageBytes, cb + (size_t)un.w * ES, bytes, &full[st], pol);
          ++g;
        }
      }
      if (!ok) {
        // error path: let every copy still in flight land before the CTA exits
        for (long long h = (g > S ? g - S : 0); h < g; ++h) {
          uint64_t* b = &full[h % S];
          const uint32_t par = (uint32_t)((h / S) & 1);
          unsigned long long t0 = global_ns();
          while (!mbar_try_wait(b, par) && global_ns() - t0 < kWaitLimitNs) {}
        }
      }
    }
    return;
  }

  // ---------------- consumers (8 warps) --------------------------------------
  const ConsumerBar cbar;
  const float scl = rsqrtf((float)P.Ny);
  float2* yw = ycopy + (size_t)warp * ny32;
  double fid = 0.0;
  long long gbase = 0;
  bool failed = false;
  for (int col = blockIdx.x; col < P.ncols; col += gridDim.x, gbase += P.nunits) {
    const size_t cofs = (size_t)col * P.Ny;
    for (int j = tid; j < ny32; j += kConsumers) {
      float2 v = make_float2(0.f, 0.f);
      if (j < P.Ny) {
        v = P.base[cofs + j];
        if (P.add) {
          float2 a = P.add[cofs + j];
          v.x = fmaf(P.coef, a.x, v.x); v.y = fmaf(P.coef, a.y, v.y);
        }
      }
      rvec[j] = v;
    }
    for (int j = tid; j < kConsumerWarps * ny32; j += kConsumers) ycopy[j] = make_float2(0.f, 0.f);
    cbar();
    for (int u = warp; u < P.nunits; u += kConsumerWarps) {
      const long long g = gbase + u;
      const int st = (int)(g % S);
      if (failed) continue;
      if (!mbar_wait(&full[st], (uint32_t)((g / S) & 1), P.flags)) { failed = true; continue; }
      const int4 un = units[u];
      const E* tl = reinterpret_cast<const E*>(ring + (size_t)st * kStageBytes);
      if (un.x == UNIT_TILE) proc_tile<E>(tl, rvec, yw, un.y, un.z, lane);
      else proc_rect<E>(tl, rvec, yw, un.y, un.z, lane);
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    cbar();
    for (int j = tid; j < P.Ny; j += kConsumers) {
      float2 s = ycopy[j];
#pragma unroll
      for (int w = 1; w < kConsumerWarps; ++w) s = c_add(s, ycopy[(size_t)w * ny32 + j]);
      xcol[j] = s;
      P.xout[cofs + j] = s;
    }
    if (P.do_obj) {
      cbar();
      const int t = col / P.Nx, i = col - t * P.Nx;
      fid += column_fid(xcol, i, t, P.Nx, P.Ny, P.Nc, P.ncg, P.sens, P.yhat, P.rows, P.rowoff, P.fy, scl, fa, fb,
                        tid, kConsumers, cbar);
    }
    cbar();
    if (tid == 0) s_abort = (*((volatile int*)&P.flags[FLAG_ERR]) != 0) || failed;
    cbar();
    if (s_abort || failed) break;
  }
  if (P.do_obj) {
    double s = group_sum(fid, red, tid, kConsumers, cbar);
    if (tid == 0) atomicAdd(P.fid_acc, s);
  }
}

size_t col_inverse_smem(const ColParams& p, int) {
  return col_layout(p.stages, p.nb, p.nunits, p.ncg, p.Ny, p.do_obj).total;
}

int col_inverse_max_stages(const ColParams& p, int storage) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int s = 32;
  while (s > 2) {
    ColParams q = p;
    q.stages = s;
    if (col_inverse_smem(q, storage) + 1024 <= (size_t)optin) break;
    --s;
  }
  return s;
}

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
// Algorithm 2 temporal step, one thread per pixel (column layout keeps the
// threads of a warp on consecutive j, so every access is coalesced):
//   v  = S(D_t m + d1, lambda/(2 mu1))
//   m' = (rho I + D_t'D_t)^{-1} [D_t'(v - d1) + rho (x + d2)]    (Thomas)
//   d1' = d1 - (v - D_t m')
// with d2 = x - p, and p' = m' - d2 handed to the inverse step, which forms
// r = H'y + mu2 (m' - d2) = b + mu2 p'.  The next d2 is then x' - p'.
// Also accumulates ||D_t x||_1 of the incoming x (the prior term of J).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_tv_temporal(TvParams P) {
  extern __shared__ float2 sm_tv[];
  __shared__ double red[32];
  if (P.flags[FLAG_STOP]) return;
  const int nth = blockDim.x, tid = threadIdx.x;
  float2* sd = sm_tv;                  // forward-sweep values d'_t
  float2* se = sm_tv + P.Nt * nth;     // e_t = d1_t - v_t
  const long long N = P.npix;
  const long long pix = (long long)blockIdx.x * nth + tid;
  double tv = 0.0;
  if (pix < N) {
    float2 x_prev = make_float2(0.f, 0.f);
    float2 m_t = P.write_state ? P.m[pix] : make_float2(0.f, 0.f);
    float2 e_prev = make_float2(0.f, 0.f), d_prev = make_float2(0.f, 0.f);
    for (int t = 0; t < P.Nt; ++t) {
      const float2 x_t = P.x[t * N + pix];
      if (t > 0) tv += (double)c_abs(c_sub(x_t, x_prev));
      x_prev = x_t;
      if (!P.write_state) continue;
      const float2 p_t = P.p[t * N + pix];
      float2 e_t = make_float2(0.f, 0.f), m_n = make_float2(0.f, 0.f);
      if (t + 1 < P.Nt) {
        m_n = P.m[(t + 1) * N + pix];
        const float2 d1_t = P.d1 ? P.d1[t * N + pix] : make_float2(0.f, 0.f);
        const float2 v = c_soft(c_add(c_sub(m_n, m_t), d1_t), P.tau1);
        e_t = c_sub(d1_t, v);
      }
      // rhs = D'(v - d1) + rho (x + d2),  (D'u)_t = u_{t-1} - u_t,  u = -e
      float2 rhs = c_sub(e_t, e_prev);
      rhs.x = fmaf(P.rho, 2.f * x_t.x - p_t.x, rhs.x);
      rhs.y = fmaf(P.rho, 2.f * x_t.y - p_t.y, rhs.y);
      const float inv = __ldg(P.thomas + t);
      const float2 dp = c_scale(c_add(rhs, d_prev), inv);
      sd[t * nth + tid] = dp;
      se[t * nth + tid] = e_t;
      d_prev = dp; e_prev = e_t; m_t = m_n;
    }
    if (P.write_state) {
      float2 mnext = make_float2(0.f, 0.f);
      for (int t = P.Nt - 1; t >= 0; --t) {
        const float inv = __ldg(P.thomas + t);
        const float2 dp = sd[t * nth + tid];
        const float2 mt = make_float2(fmaf(inv, mnext.x, dp.x), fmaf(inv, mnext.y, dp.y));
        if (t + 1 < P.Nt) P.d1_out[t * N + pix] = c_add(se[t * nth + tid], c_sub(mnext, mt));
        const float2 x_t = P.x[t * N + pix], p_t = P.p[t * N + pix];
        P.p_out[t * N + pix] = c_add(mt, c_sub(p_t, x_t));
        P.m_out[t * N + pix] = mt;
        mnext = mt;
      }
    }
  }
  const double s = group_sum(tv, red, tid, nth, BlockBar());
  if (tid == 0) atomicAdd(P.prior_acc, s);
}

cudaError_t launch_tv_temporal(const TvParams& p, cudaStream_t s) {
  // 2 x Nt x nth complex values of per-thread sweep storage must fit (Nt <= 128)
  int nth = 128;
  while (nth > 32 && 2 * (size_t)p.Nt * nth * sizeof(float2) > 160 * 1024) nth >>= 1;
  const size_t smem = p.write_state ? 2 * (size_t)p.Nt * nth * sizeof(float2) : 0;
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_tv_temporal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const long long grid = (p.npix + nth - 1) / nth;
  k_tv_temporal<<<(unsigned)grid, nth, smem, s>>>(p); note_launch();
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
    A[idx] = (pp < npx) ? P.xh[t * N + pix0 + pp] : make_float2(0.f, 0.f);
  }
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
__global__ void k_finalize(const double* fid, const double* prior, double* J, int k, float lam, double tol,
                           int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (flags[FLAG_STOP]) return;
  const double Jk = fid[k] + (double)lam * prior[k];
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

cudaError_t launch_finalize(const double* fid, const double* prior, double* J, int k, float lam, double tol,
                            int* flags, cudaStream_t s) {
  k_finalize<<<1, 32, 0, s>>>(fid, prior, J, k, lam, tol, flags); note_launch();
  return cudaGetLastError();
}

}  // namespace recon
