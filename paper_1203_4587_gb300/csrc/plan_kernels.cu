// Plan-time kernels: the exact data-consistency inverse of Section IV-C.
//
// H'H is block diagonal over frames t and columns i (Eq. HconjH):
//   G_{i,t}[j,k] = C_t[j,k] * sum_c conj(s_{j,i,c}) s_{k,i,c}
// with C_t = F~_{v,t}' F~_{v,t} = F_v' P_t F_v circulant,
//   C_t[j,k] = c_t[(j-k) mod Ny],  c_t[d] = (1/Ny) sum_{q sampled} exp(+2 pi i q d / Ny).
// (The paper prints sum_c s_c s_c'; the operator form S_c' F~' F~ S_c gives
// conj(s_j) s_k, which is used here.)  Each block is inverted exactly,
// A_{i,t} = (mu I + G_{i,t})^{-1} (Eq. eigen_mu: the eigendecomposition and a
// direct inversion give the same matrix), in double-float arithmetic
// (df64.cuh, about 48 significant bits on the FP32 pipe) by a blocked sweep
// (below), rounded once to the storage type and scattered into the packed
// stream (kernels.h).
#include "df64.cuh"
#include "kernels.h"

namespace recon {

__global__ void k_circulant(const int* __restrict__ rows, const int* __restrict__ rowoff,
                            const double2* __restrict__ w64, double2* __restrict__ circ, int Ny) {
  const int t = blockIdx.x;
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  const double inv = 1.0 / Ny;
  for (int d = threadIdx.x; d < Ny; d += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < mt; ++m) {
      const long long q = rows[r0 + m];
      const double2 w = w64[(q * d) % Ny];  // exp(+2 pi i q d / Ny)
      acc.x += w.x; acc.y += w.y;
    }
    circ[(size_t)t * Ny + d] = make_double2(acc.x * inv, acc.y * inv);
  }
}

cudaError_t launch_circulant(const int* rows, const int* rowoff, const double2* w64, double2* circ, int Ny, int Nt,
                             cudaStream_t s) {
  k_circulant<<<Nt, 256, 0, s>>>(rows, rowoff, w64, circ, Ny); note_launch();
  return cudaGetLastError();
}

// Complex position of the planar pair holding A[R][C] (R <= C, both < Nyp,
// C even) inside one column's packed stream (layout in kernels.h).
__host__ __device__ inline long long packed_pos(int R, int C, int ntiles) {
  const int bj = R >> 5, bk = C >> 5, rr = R & 31, cc = C & 31;
  const int qq = (rr & 3) * 4 + (cc & 7) / 2, lr = rr >> 2, lc = cc >> 3;
  if (bj < bk) {
    const long long u = (long long)bk * (bk - 1) / 2 + bj;
    return u * kTileElems + qq * 64 + (lr * 4 + lc) * 2;
  }
  return (long long)ntiles * kTileElems + (long long)bj * kDiagElems + qq * 2 * kDiagLanes + (lc * (lc + 1) + lr) * 2;
}

// Element (R, C), R <= C, of a packed column as planar pairs (components
// re_C, re_C+1, im_C, im_C+1); diagonal entries are stored halved.
template <typename E>
__device__ __forceinline__ void packed_store(E* Ac, int R, int C, int ntiles, double2 v) {
  using S = typename Elem<E>::S;
  S* sc = reinterpret_cast<S*>(Ac);
  if (R == C) v = make_double2(0.5 * v.x, 0.0);
  const long long b = 2 * packed_pos(R, C & ~1, ntiles);
  sc[b + (C & 1)] = Elem<E>::cvt1(v.x);
  sc[b + 2 + (C & 1)] = Elem<E>::cvt1(v.y);
}
template <typename E>
__device__ __forceinline__ float2 packed_load(const E* Ac, int R, int C, int ntiles) {
  using S = typename Elem<E>::S;
  const S* sc = reinterpret_cast<const S*>(Ac);
  const long long b = 2 * packed_pos(R, C & ~1, ntiles);
  const float2 v = make_float2(Elem<E>::widen1(sc[b + (C & 1)]), Elem<E>::widen1(sc[b + 2 + (C & 1)]));
  return R == C ? make_float2(2.f * v.x, 0.f) : v;
}

// 16 warps: a thread's double-float update chains are long and dependent, so
// the SM needs many warps in flight to hide their latency
constexpr int kPlanThreads = 512;
constexpr int kPlanRows = kPlanThreads / 16;   // rows of a 16-column tile

// The inversion runs in double-float arithmetic (df64.cuh): about 48
// significant bits on the FP32 pipe, which GB300 runs at 64 times its FP64
// rate; the result is rounded once to the storage type.  W holds one complex
// double-float per element as (re.hi, re.lo, im.hi, im.lo).
//
// M is inverted in place by the sweep operator (Goodnight 1979), blocked over
// B pivots at a time: with P the pivot block, R the other indices,
//   M[B][B] <- -P^{-1},   M[R][B] <- M[R][B] P^{-1},
//   M[R][R] <- M[R][R] - M[R][B] P^{-1} M[B][R],
// and after every pivot has been swept M holds -M^{-1}.  Sweeping the
// pivots of a Hermitian positive definite matrix in order divides by the
// diagonals of its Schur complements, which are positive, as in a Cholesky
// factorisation; it takes about n^3/2 complex multiply-adds and touches W
// once per block of B pivots.  Only the lower triangle is stored.  P^{-1} comes
// from sweeping the B x B block itself in shared memory.
__device__ __forceinline__ dc ldw(const float4* W, size_t o) { return dc_unpack(W[o]); }
__device__ __forceinline__ void stw(float4* W, size_t o, dc v) { W[o] = dc_pack(v); }
__device__ __forceinline__ dc dc_conj(dc a) { return {a.re, df_neg(a.im)}; }
__device__ __forceinline__ dc dc_neg(dc a) { return {df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ dc dc_zero() { return {df_make(0.f), df_make(0.f)}; }
// acc + a b
__device__ __forceinline__ dc dc_fma(dc acc, dc a, dc b) {
  acc.re = df_fma(df_fma(acc.re, a.re, b.re), df_neg(a.im), b.im);
  acc.im = df_fma(df_fma(acc.im, a.re, b.im), a.im, b.re);
  return acc;
}
// acc - a conj(b)
__device__ __forceinline__ dc dc_fms_conj(dc acc, dc a, dc b) {
  acc.re = df_fma(df_fma(acc.re, df_neg(a.re), b.re), df_neg(a.im), b.im);
  acc.im = df_fma(df_fma(acc.im, df_neg(a.im), b.re), a.re, b.im);
  return acc;
}
__device__ __forceinline__ dc dc_scale(dc a, df s) { return {df_mul(a.re, s), df_mul(a.im, s)}; }

template <int B>
__host__ __device__ constexpr size_t plan_smem_f4(int n, int Nc) {
  // max(sensitivities [Nc][n] float2, panel [n][B] + T [n][B] + pivot block [B][B])
  return ((size_t)Nc * n + 1) / 2 > (size_t)2 * n * B + B * B ? ((size_t)Nc * n + 1) / 2
                                                                : (size_t)2 * n * B + B * B;
}

template <typename E, int B>
__global__ void __launch_bounds__(kPlanThreads, 1) k_plan_inverse(const float2* __restrict__ sens,
                                                                  const double2* __restrict__ circ, float mu, int Nx,
                                                                  int Ny, int Nt, int Nc, E* __restrict__ A,
                                                                  long long col_elems, int ntiles,
                                                                  float4* __restrict__ scratch, int* flags) {
  static_assert(B * B <= kPlanThreads, "one pivot-block entry per thread");
  extern __shared__ float4 zs[];
  const int n = Ny, tid = threadIdx.x;
  float2* sc = reinterpret_cast<float2*>(zs);   // [Nc][n] sensitivities of column i (Gram phase only)
  float4* pan = zs;                              // [n][B]  M(i, k0 + c)
  float4* Tm = zs + (size_t)n * B;               // [n][B]  M(i, k0 + c) P^{-1}
  float4* Pq = zs + (size_t)2 * n * B;           // [B][B]  pivot block, swept to -P^{-1}
  float4* W = scratch + (size_t)blockIdx.x * n * n;  // row-major n x n, lower triangle used
  const long long nmat = (long long)Nx * Nt;
  const int ty = tid >> 4, tx = tid & 15;   // kPlanRows x 16 tiles
  bool bad = false;
  for (long long mat = blockIdx.x; mat < nmat; mat += gridDim.x) {
    const int t = (int)(mat / Nx), i = (int)(mat - (long long)t * Nx);
    for (int idx = tid; idx < Nc * n; idx += kPlanThreads) sc[idx] = sens[(size_t)i * Nc * n + idx];
    __syncthreads();
    // M = mu I + C_t (.) K_i, lower triangle; K = sum_c conj(s_j) s_k, every
    // product exact in double length
    for (long long idx = tid; idx < (long long)n * n; idx += kPlanThreads) {
      const int j = (int)(idx / n), k = (int)(idx - (long long)j * n);
      if (k > j) continue;
      df kr = df_make(0.f), ki = df_make(0.f);
      for (int c = 0; c < Nc; ++c) {
        const float2 a = sc[c * n + j], b = sc[c * n + k];
        kr = df_fma_ff(df_fma_ff(kr, a.x, b.x), a.y, b.y);     // Re conj(a) b
        ki = df_fma_ff(df_fma_ff(ki, a.x, b.y), -a.y, b.x);    // Im conj(a) b
      }
      const double2 cz = circ[(size_t)t * n + (j - k)];
      const df cr = df_from_double(cz.x), ci = df_from_double(cz.y);
      dc g;
      g.re = df_sub(df_mul(cr, kr), df_mul(ci, ki));
      g.im = df_add(df_mul(cr, ki), df_mul(ci, kr));
      if (j == k) g.re = df_add(g.re, df_make(mu));
      stw(W, (size_t)j * n + k, g);
    }
    __syncthreads();   // sc is overwritten by the panel below
    for (int k0 = 0; k0 < n; k0 += B) {
      const int bb = min(B, n - k0);
      // panel M(i, k0 + c) for every i (the upper part from the stored lower one)
      for (int idx = tid; idx < n * B; idx += kPlanThreads) {
        const int r = idx / B, c = idx - r * B;
        dc v = dc_zero();
        if (c < bb) v = (r >= k0 + c) ? ldw(W, (size_t)r * n + k0 + c) : dc_conj(ldw(W, (size_t)(k0 + c) * n + r));
        pan[idx] = dc_pack(v);
      }
      __syncthreads();
      // pivot block, swept in place: pivot k, entry (r, c)
      const int pr = tid / B, pc = tid - (tid / B) * B;
      const bool pv = tid < B * B && pr < bb && pc < bb;
      if (tid < B * B) Pq[tid] = pv ? pan[(size_t)(k0 + pr) * B + pc] : dc_pack(dc_zero());
      __syncthreads();
      for (int k = 0; k < bb; ++k) {
        df d = dc_unpack(Pq[k * B + k]).re;
        if (!(d.hi > 0.f)) { bad = true; d = df_make(1.f); }
        const df rd = df_rcp(d);
        dc rk = dc_zero(), kc = dc_zero(), old = dc_zero();
        if (pv) { rk = dc_unpack(Pq[pr * B + k]); kc = dc_unpack(Pq[k * B + pc]); old = dc_unpack(Pq[tid]); }
        __syncthreads();
        if (pv) {
          dc v;
          if (pr == k && pc == k) v = dc{df_neg(rd), df_make(0.f)};
          else if (pr == k) v = dc_scale(kc, rd);
          else if (pc == k) v = dc_scale(rk, rd);
          else v = dc_fms_conj(old, dc_scale(rk, rd), dc_conj(kc));   // old - rk kc / d
          Pq[tid] = dc_pack(v);
        }
        __syncthreads();
      }
      // T(i, c) = M(i, k0 + c) P^{-1} = -sum_d M(i, k0 + d) Pq(d, c), i outside the block
      for (int idx = tid; idx < n * B; idx += kPlanThreads) {
        const int r = idx / B, c = idx - r * B;
        if (c >= bb || (r >= k0 && r < k0 + bb)) continue;
        dc acc = dc_zero();
#pragma unroll
        for (int d = 0; d < B; ++d)
          if (d < bb) acc = dc_fma(acc, dc_unpack(pan[(size_t)r * B + d]), dc_unpack(Pq[d * B + c]));
        Tm[idx] = dc_pack(dc_neg(acc));
      }
      __syncthreads();
      // the sweep of the block over the stored lower triangle.  A thread takes
      // rows r, r + kPlanRows and columns c, c + 16 of a 64 x 32 tile: one T
      // load serves two columns, one panel load two rows, and four
      // independent double-float chains interleave
      for (int ib = 0; ib < n; ib += 2 * kPlanRows) {
        for (int jb = 0; jb < ib + 2 * kPlanRows; jb += 32) {
          const int rr[2] = {ib + ty, ib + ty + kPlanRows}, cc[2] = {jb + tx, jb + tx + 16};
          // (R, R) entries get the rank-bb update; the four run together, an
          // entry outside the triangle or in the block's rows / columns only
          // masked (its operand rows clamped in range, its result not stored)
          bool upd[2][2], any = false;
#pragma unroll
          for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
            for (int b2 = 0; b2 < 2; ++b2) {
              const int r = rr[a2], c = cc[b2];
              const bool inr = r >= k0 && r < k0 + bb, inc = c >= k0 && c < k0 + bb;
              upd[a2][b2] = r < n && c <= r && !inr && !inc;
              any = any || upd[a2][b2];
            }
          if (any) {
            const int r0 = min(rr[0], n - 1), r1 = min(rr[1], n - 1);
            const int c0 = min(cc[0], n - 1), c1 = min(cc[1], n - 1);
            dc w[2][2];
#pragma unroll
            for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
              for (int b2 = 0; b2 < 2; ++b2)
                w[a2][b2] = upd[a2][b2] ? ldw(W, (size_t)rr[a2] * n + cc[b2]) : dc_zero();
#pragma unroll
            for (int q = 0; q < B; ++q)
              if (q < bb) {
                const dc t0 = dc_unpack(Tm[(size_t)r0 * B + q]), t1 = dc_unpack(Tm[(size_t)r1 * B + q]);
                const dc p0 = dc_unpack(pan[(size_t)c0 * B + q]), p1 = dc_unpack(pan[(size_t)c1 * B + q]);
                w[0][0] = dc_fms_conj(w[0][0], t0, p0);
                w[0][1] = dc_fms_conj(w[0][1], t0, p1);
                w[1][0] = dc_fms_conj(w[1][0], t1, p0);
                w[1][1] = dc_fms_conj(w[1][1], t1, p1);
              }
#pragma unroll
            for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
              for (int b2 = 0; b2 < 2; ++b2)
                if (upd[a2][b2]) stw(W, (size_t)rr[a2] * n + cc[b2], w[a2][b2]);
          }
          // the entries of the block's rows and columns take T, its conjugate or -P^{-1}
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = rr[h >> 1], c = cc[h & 1];
            if (r >= n || c > r) continue;
            const bool rin = r >= k0 && r < k0 + bb, cin = c >= k0 && c < k0 + bb;
            if (!rin && !cin) continue;   // updated above
            const size_t o = (size_t)r * n + c;
            if (!rin) {                  // (r, c) with c in the block, r below it
              W[o] = Tm[(size_t)r * B + (c - k0)];
            } else if (!cin) {           // r in the block, c left of it: conj of (c, r)
              W[o] = dc_pack(dc_conj(dc_unpack(Tm[(size_t)c * B + (r - k0)])));
            } else {                     // inside the block
              W[o] = Pq[(r - k0) * B + (c - k0)];
            }
          }
        }
      }
      __syncthreads();
    }
    // W = -M^{-1}: A[j][k] = -conj(W[k][j]) for j <= k, rounded once
    E* Ac = A + (size_t)((long long)i * Nt + t) * col_elems;   // image-column-major (kernels.h)
    for (int jb = 0; jb < n; jb += kPlanRows) {
      for (int kb = jb / 16 * 16; kb < n; kb += 16) {
        const int j = jb + ty, k = kb + tx;
        if (j < n && k < n && j <= k) {
          const dc w = ldw(W, (size_t)k * n + j);
          // Hermitian: exact real diagonal
          packed_store(Ac, j, k, ntiles, make_double2(-df_to_double(w.re), j == k ? 0.0 : df_to_double(w.im)));
        }
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(&flags[FLAG_ERR], DEV_ERR_NOT_PD);
}

// pivot block width: 16 while the panel and T fit in shared memory, else 8 or 4
static int plan_block(int n, int Nc) {
  if (plan_smem_f4<16>(n, Nc) * sizeof(float4) <= 220 * 1024) return 16;
  if (plan_smem_f4<8>(n, Nc) * sizeof(float4) <= 220 * 1024) return 8;
  return 4;
}

template <typename E, int B>
static cudaError_t launch_plan_tb(const float2* sens, const double2* circ, double mu, int Nx, int Ny, int Nt, int Nc,
                                  void* A, const PackInfo& pk, double2* scratch, int grid, int* flags,
                                  cudaStream_t s) {
  const size_t smem = plan_smem_f4<B>(Ny, Nc) * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(k_plan_inverse<E, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_plan_inverse<E, B><<<grid, kPlanThreads, smem, s>>>(sens, circ, (float)mu, Nx, Ny, Nt, Nc, static_cast<E*>(A),
                                                        pk.col_elems, pk.ntiles, reinterpret_cast<float4*>(scratch),
                                                        flags); note_launch();
  return cudaGetLastError();
}

template <typename E>
static cudaError_t launch_plan_t(const float2* sens, const double2* circ, double mu, int Nx, int Ny, int Nt, int Nc,
                                 void* A, const PackInfo& pk, double2* scratch, int grid, int* flags,
                                 cudaStream_t s) {
  switch (plan_block(Ny, Nc)) {
    case 16: return launch_plan_tb<E, 16>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
    case 8: return launch_plan_tb<E, 8>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
    default: return launch_plan_tb<E, 4>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
  }
}

cudaError_t launch_plan_inverse(const float2* sens, const double2* circ, double mu, int Nx, int Ny, int Nt, int Nc,
                                void* A, int storage, const PackInfo& pk, double2* scratch, int grid, int* flags,
                                cudaStream_t s) {
  switch (storage) {
    case 0: return launch_plan_t<float2>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
    case 1: return launch_plan_t<__half2>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
    case 2: return launch_plan_t<__nv_bfloat162>(sens, circ, mu, Nx, Ny, Nt, Nc, A, pk, scratch, grid, flags, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename E>
__global__ void k_unpack(const E* __restrict__ A, long long col_elems, int ntiles, long long col, int Ny,
                         float2* __restrict__ dense) {
  const E* Ac = A + (size_t)col * col_elems;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)Ny * Ny;
       idx += (long long)gridDim.x * blockDim.x) {
    const int R = (int)(idx / Ny), C = (int)(idx - (long long)R * Ny);
    float2 v;
    if (R <= C) v = packed_load(Ac, R, C, ntiles);
    else v = c_conj(packed_load(Ac, C, R, ntiles));
    dense[idx] = v;
  }
}

cudaError_t launch_unpack(const void* A, int storage, const PackInfo& pk, long long col, int Ny, float2* dense,
                          cudaStream_t s) {
  const int grid = (int)(((long long)Ny * Ny + 255) / 256);
  switch (storage) {
    case 0: k_unpack<float2><<<grid, 256, 0, s>>>(static_cast<const float2*>(A), pk.col_elems, pk.ntiles, col, Ny, dense); note_launch(); break;
    case 1: k_unpack<__half2><<<grid, 256, 0, s>>>(static_cast<const __half2*>(A), pk.col_elems, pk.ntiles, col, Ny, dense); note_launch(); break;
    case 2: k_unpack<__nv_bfloat162><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat162*>(A), pk.col_elems, pk.ntiles, col, Ny, dense); note_launch(); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace recon
