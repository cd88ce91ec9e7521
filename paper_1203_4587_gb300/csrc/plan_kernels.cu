// Plan-time kernels: the exact data-consistency inverse of Section IV-C.
//
// H'H is block diagonal over frames t and columns i (Eq. HconjH):
//   G_{i,t}[j,k] = C_t[j,k] * sum_c conj(s_{j,i,c}) s_{k,i,c}
// with C_t = F~_{v,t}' F~_{v,t} = F_v' P_t F_v circulant,
//   C_t[j,k] = c_t[(j-k) mod Ny],  c_t[d] = (1/Ny) sum_{q sampled} exp(+2 pi i q d / Ny).
// (The paper prints sum_c s_c s_c'; the operator form S_c' F~' F~ S_c gives
// conj(s_j) s_k, which is used here.)  Each block is inverted exactly,
// A_{i,t} = (mu I + G_{i,t})^{-1} (Eq. eigen_mu: the eigendecomposition and a
// Cholesky factorisation give the same matrix), in FP64:
//   1. M = mu I + G (lower triangle)
//   2. M = L L'                 (right-looking Cholesky)
//   3. Z = L^{-1}               (row by row)
//   4. A = Z' Z                 (upper triangle), rounded once to the storage
//      type and scattered into the packed stream (kernels.h).
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

template <typename E>
__global__ void __launch_bounds__(kPlanThreads) k_plan_inverse(const float2* __restrict__ sens,
                                                               const double2* __restrict__ circ, double mu, int Nx,
                                                               int Ny, int Nt, int Nc, E* __restrict__ A,
                                                               long long col_elems, int ntiles,
                                                               double2* __restrict__ scratch, int* flags) {
  extern __shared__ double2 zs[];
  const int n = Ny, tid = threadIdx.x;
  double2* sc = zs;                  // [Nc][n] sensitivities of column i (FP64)
  double2* cb = zs + (size_t)Nc * n; // [n] cached column / row
  double2* W = scratch + (size_t)blockIdx.x * n * n;  // row-major n x n
  const long long nmat = (long long)Nx * Nt;
  const int ty = tid >> 4, tx = tid & 15;
  for (long long mat = blockIdx.x; mat < nmat; mat += gridDim.x) {
    const int t = (int)(mat / Nx), i = (int)(mat - (long long)t * Nx);
    for (int idx = tid; idx < Nc * n; idx += kPlanThreads) {
      const float2 v = sens[(size_t)i * Nc * n + idx];
      sc[idx] = make_double2(v.x, v.y);
    }
    __syncthreads();
    // 1. M = mu I + C_t (.) K_i, lower triangle
    for (long long idx = tid; idx < (long long)n * n; idx += kPlanThreads) {
      const int j = (int)(idx / n), k = (int)(idx - (long long)j * n);
      if (k > j) continue;
      double2 K = make_double2(0.0, 0.0);
      for (int c = 0; c < Nc; ++c) z_fmac(K, sc[c * n + j], sc[c * n + k]);  // conj(s_j) s_k
      double2 g = z_mul(circ[(size_t)t * n + (j - k)], K);
      if (j == k) g.x += mu;
      W[(size_t)j * n + k] = g;
    }
    __syncthreads();
    // 2. Cholesky, right-looking
    bool bad = false;
    for (int k = 0; k < n; ++k) {
      double d = W[(size_t)k * n + k].x;
      if (!(d > 0.0)) { bad = true; d = 1.0; }
      d = sqrt(d);
      const double inv = 1.0 / d;
      for (int j = k + 1 + tid; j < n; j += kPlanThreads) {
        double2 v = W[(size_t)j * n + k];
        v.x *= inv; v.y *= inv;
        W[(size_t)j * n + k] = v;
        cb[j] = v;
      }
      __syncthreads();
      if (tid == 0) W[(size_t)k * n + k] = make_double2(d, 0.0);
      const int m = n - k - 1;
      for (int jb = 0; jb < m; jb += 16) {
        for (int lb = 0; lb <= jb; lb += 16) {
          const int jj = jb + ty, ll = lb + tx;
          if (jj < m && ll <= jj) {
            const int j = k + 1 + jj, l = k + 1 + ll;
            double2 w = W[(size_t)j * n + l];
            const double2 a = cb[j], b = cb[l];
            // w -= a * conj(b)
            w.x -= fma(a.x, b.x, a.y * b.y);
            w.y -= fma(a.y, b.x, -a.x * b.y);
            W[(size_t)j * n + l] = w;
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
      const double ljj = cb[j].x;
      for (int c = tid; c <= j; c += kPlanThreads) {
        double2 z;
        if (c == j) {
          z = make_double2(1.0 / ljj, 0.0);
        } else {
          double2 s = make_double2(0.0, 0.0);
          for (int l = c; l < j; ++l) z_fma(s, cb[l], W[(size_t)l * n + c]);
          z = make_double2(-s.x / ljj, -s.y / ljj);
        }
        W[(size_t)j * n + c] = z;
      }
      __syncthreads();
    }
    // 4. A = Z' Z, upper triangle: A[j][k] = sum_{l >= k} conj(Z[l][j]) Z[l][k]
    E* Ac = A + (size_t)mat * col_elems;
    for (int jb = 0; jb < n; jb += 16) {
      for (int kb = jb; kb < n; kb += 16) {
        const int j = jb + ty, k = kb + tx;
        if (j < n && k < n && j <= k) {
          double2 s = make_double2(0.0, 0.0);
          for (int l = k; l < n; ++l) z_fmac(s, W[(size_t)l * n + j], W[(size_t)l * n + k]);
          if (j == k) s.y = 0.0;  // Hermitian: exact real diagonal
          packed_store(Ac, j, k, ntiles, s);
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
  const size_t smem = ((size_t)Nc * Ny + Ny) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_plan_inverse<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_plan_inverse<E><<<grid, kPlanThreads, smem, s>>>(sens, circ, mu, Nx, Ny, Nt, Nc, static_cast<E*>(A),
                                                     pk.col_elems, pk.ntiles, scratch, flags); note_launch();
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
