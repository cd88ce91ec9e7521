// Plan-time kernels: the exact data-consistency inverse of Section IV-C.
//
// H'H is block diagonal over frames t and columns i (Eq. HconjH):
//   G_{i,t}[j,k] = C_t[j,k] * sum_c conj(s_{j,i,c}) s_{k,i,c}
// with C_t = F~_{v,t}' F~_{v,t} = F_v' P_t F_v circulant,
//   C_t[j,k] = c_t[(j-k) mod Ny],  c_t[d] = (1/Ny) sum_{q sampled} exp(+2 pi i q d / Ny).
// (The paper prints sum_c s_c s_c'; the operator form S_c' F~' F~ S_c gives
// conj(s_j) s_k, which is used here.)  Each block is inverted exactly,
// A_{i,t} = (mu I + G_{i,t})^{-1} (Eq. eigen_mu: the eigendecomposition and a
// Cholesky factorisation give the same matrix), in double-float arithmetic
// (df64.cuh, about 48 significant bits on the FP32 pipe):
//   1. M = mu I + G (lower triangle)
//   2. M = L L'                 (right-looking Cholesky)
//   3. Z = L^{-1}               (row by row)
//   4. A = Z' Z                 (upper triangle), rounded once to the storage
//      type and scattered into the packed stream (kernels.h).
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

constexpr int kPlanThreads = 256;

// The factorisation in double-float arithmetic (df64.cuh): about 48
// significant bits on the FP32 pipe, which GB300 runs at 64 times its FP64
// rate; the result is rounded once to the storage type.  W holds one complex
// double-float per element as (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ dc ldw(const float4* W, size_t o) { return dc_unpack(W[o]); }
__device__ __forceinline__ void stw(float4* W, size_t o, dc v) { W[o] = dc_pack(v); }

template <typename E>
__global__ void __launch_bounds__(kPlanThreads) k_plan_inverse(const float2* __restrict__ sens,
                                                               const double2* __restrict__ circ, float mu, int Nx,
                                                               int Ny, int Nt, int Nc, E* __restrict__ A,
                                                               long long col_elems, int ntiles,
                                                               float4* __restrict__ scratch, int* flags) {
  extern __shared__ float4 zs[];
  const int n = Ny, tid = threadIdx.x;
  float2* sc = reinterpret_cast<float2*>(zs);   // [Nc][n] sensitivities of column i (exact FP32 inputs)
  float4* cb = zs + ((size_t)Nc * n + 1) / 2;   // [n] cached column / row
  float4* W = scratch + (size_t)blockIdx.x * n * n;  // row-major n x n
  const long long nmat = (long long)Nx * Nt;
  const int ty = tid >> 4, tx = tid & 15;
  for (long long mat = blockIdx.x; mat < nmat; mat += gridDim.x) {
    const int t = (int)(mat / Nx), i = (int)(mat - (long long)t * Nx);
    for (int idx = tid; idx < Nc * n; idx += kPlanThreads) sc[idx] = sens[(size_t)i * Nc * n + idx];
    __syncthreads();
    // 1. M = mu I + C_t (.) K_i, lower triangle; K = sum_c conj(s_j) s_k, every
    //    product exact in double length
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
    __syncthreads();
    // 2. Cholesky, right-looking
    bool bad = false;
    for (int k = 0; k < n; ++k) {
      df d = ldw(W, (size_t)k * n + k).re;
      if (!(d.hi > 0.f)) { bad = true; d = df_make(1.f); }
      d = df_sqrt(d);
      const df inv = df_rcp(d);
      for (int j = k + 1 + tid; j < n; j += kPlanThreads) {
        dc v = ldw(W, (size_t)j * n + k);
        v.re = df_mul(v.re, inv);
        v.im = df_mul(v.im, inv);
        stw(W, (size_t)j * n + k, v);
        cb[j] = dc_pack(v);
      }
      __syncthreads();
      if (tid == 0) stw(W, (size_t)k * n + k, dc{d, df_make(0.f)});
      const int m = n - k - 1;
      for (int jb = 0; jb < m; jb += 16) {
        for (int lb = 0; lb <= jb; lb += 16) {
          const int jj = jb + ty, ll = lb + tx;
          if (jj < m && ll <= jj) {
            const int j = k + 1 + jj, l = k + 1 + ll;
            dc w = ldw(W, (size_t)j * n + l);
            const dc a = dc_unpack(cb[j]), b = dc_unpack(cb[l]);
            // w -= a * conj(b)
            w.re = df_fma(df_fma(w.re, df_neg(a.re), b.re), df_neg(a.im), b.im);
            w.im = df_fma(df_fma(w.im, df_neg(a.im), b.re), a.re, b.im);
            stw(W, (size_t)j * n + l, w);
          }
        }
      }
      __syncthreads();
    }
    if (bad && tid == 0) atomicOr(&flags[FLAG_ERR], DEV_ERR_NOT_PD);
    // 3. Z = L^{-1}, row j from rows < j:  Z[j][c] = -(1/L[j][j]) sum_{l=c}^{j-1} L[j][l] Z[l][c]
    for (int j = 0; j < n; ++j) {
      for (int l = tid; l <= j; l += kPlanThreads) cb[l] = W[(size_t)j * n + l];
      __syncthreads();
      const df rl = df_rcp(dc_unpack(cb[j]).re);
      for (int c = tid; c <= j; c += kPlanThreads) {
        dc z;
        if (c == j) {
          z = dc{rl, df_make(0.f)};
        } else {
          df sr = df_make(0.f), si = df_make(0.f);
          for (int l = c; l < j; ++l) {
            const dc a = dc_unpack(cb[l]), b = ldw(W, (size_t)l * n + c);
            sr = df_fma(df_fma(sr, a.re, b.re), df_neg(a.im), b.im);
            si = df_fma(df_fma(si, a.re, b.im), a.im, b.re);
          }
          z = dc{df_neg(df_mul(sr, rl)), df_neg(df_mul(si, rl))};
        }
        stw(W, (size_t)j * n + c, z);
      }
      __syncthreads();
    }
    // 4. A = Z' Z, upper triangle: A[j][k] = sum_{l >= k} conj(Z[l][j]) Z[l][k],
    //    rounded once to the storage type
    E* Ac = A + (size_t)mat * col_elems;
    for (int jb = 0; jb < n; jb += 16) {
      for (int kb = jb; kb < n; kb += 16) {
        const int j = jb + ty, k = kb + tx;
        if (j < n && k < n && j <= k) {
          df sr = df_make(0.f), si = df_make(0.f);
          for (int l = k; l < n; ++l) {
            const dc a = ldw(W, (size_t)l * n + j), b = ldw(W, (size_t)l * n + k);
            sr = df_fma(df_fma(sr, a.re, b.re), a.im, b.im);           // Re conj(a) b
            si = df_fma(df_fma(si, a.re, b.im), df_neg(a.im), b.re);   // Im conj(a) b
          }
          double2 v = make_double2(df_to_double(sr), j == k ? 0.0 : df_to_double(si));  // Hermitian: real diagonal
          packed_store(Ac, j, k, ntiles, v);
        }
      }
    }
    __syncthreads();
  }
}

template <typename E>
static cudaError_t launch_plan_t(const float2* sens, const double2* circ, double mu, int Nx, int Ny, int Nt, int Nc,
                                 void* A, const PackInfo& pk, double2* scratch, int grid, int* flags,
                                 cudaStream_t s) {
  const size_t smem = (((size_t)Nc * Ny + 1) / 2 + Ny) * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(k_plan_inverse<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_plan_inverse<E><<<grid, kPlanThreads, smem, s>>>(sens, circ, (float)mu, Nx, Ny, Nt, Nc, static_cast<E*>(A),
                                                     pk.col_elems, pk.ntiles, reinterpret_cast<float4*>(scratch),
                                                     flags); note_launch();
  return cudaGetLastError();
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
