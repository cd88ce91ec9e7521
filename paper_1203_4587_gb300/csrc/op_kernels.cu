// Forward model operators (Section II-A, Eqs. mri_csmcoill, H_1, S, F).
//
//   H x  = M_{v,t} F_h F_v (s_c . x_t)
//   H' y = sum_c conj(s_c) . F_v' M' F_h' y_{t,c}
//
// F_h acts along k-space rows and F_v along image columns, so each is a batch
// of independent 1D unitary FFTs (shared-memory Stockham, fft.cuh):
//   k_hybrid_rows     yhat = F_h' y on the sampled rows only (rows [t][c][ky][:])
//   k_adjoint_combine b = sum_c conj(s_c) . F_v'(zero-filled yhat_c), per column
//   k_forward_cols    zhat = M F_v (s_c . x), per column (sampled rows only)
//   k_forward_rows    y = F_h zhat on the sampled rows
//   k_transpose       layout changes between [..][Ny][Nx] and [..][Nx][Ny]
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace recon {

constexpr int kRowGroup = 8;  // k-space rows per block in the row kernels (at most)

// Rows per block so that two [g][Nx+1] buffers of T fit in 96 KB.
template <typename T>
static int row_group(int Nx) {
  int g = kRowGroup;
  while (g > 1 && 2 * (size_t)g * (Nx + 1) * sizeof(T) > 96 * 1024) --g;
  return g;
}

// yhat = F_h' y on the sampled rows.  The k-space arrives as complex64 or as
// 16-bit pairs KIn with a per-frame scale (value = stored * kscale[t]); it is
// widened exactly and the FFT runs in T (dc: double-float, about 48 bits on
// the FP32 pipe, with the FP32 rounding also written to yhat32 for the
// objective; float2: FP32).  *yy
// accumulates ||y||^2 over the sampled entries and ymax[t] the largest
// |component| of frame t's output (float bits; both optional).
template <typename T, typename KIn>
__global__ void __launch_bounds__(256) k_hybrid_rows(const KIn* __restrict__ ksp, const float* __restrict__ kscale,
                                                     T* __restrict__ yhat, float2* __restrict__ yhat32,
                                                     double* __restrict__ yy, unsigned* __restrict__ ymax,
                                                     const int* __restrict__ rows,
                                                     const int* __restrict__ rowoff, int Nx, int Ny, int Nt, int Nc,
                                                     int G, FftPlanT<T> fx, double scl, int i0, int W) {
  __shared__ double red[32];
  extern __shared__ __align__(16) unsigned char sm_rows_raw[];
  T* sm_rows = reinterpret_cast<T*>(sm_rows_raw);
  const int t = blockIdx.z, c = blockIdx.y, m0 = blockIdx.x * G;
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  if (m0 >= mt) return;
  const int g = min(G, mt - m0);
  const int ss = Nx + 1;  // padded sequence stride: conflict-free transposed reads
  T* A = sm_rows;
  T* B = sm_rows + (size_t)G * ss;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float ks = kscale ? kscale[t] : 1.f;
  for (int idx = tid; idx < g * Nx; idx += nth) {
    const int gg = idx / Nx, kx = idx - gg * Nx;
    const int row = rows[r0 + m0 + gg];
    T v = from_f2<T>(Elem<KIn>::load(ksp + (((size_t)t * Nc + c) * Ny + row) * Nx + kx));
    if (kscale) v = c_scale(v, ks);
    A[gg * ss + kx] = v;
  }
  __syncthreads();
  const BlockBar bar;
  T* R = fft_run(A, B, g, ss, 1, fx, true, tid, nth, bar);
  // keep columns i0 .. i0+W-1 (a slab; all columns for a whole plan)
  const size_t base = (size_t)r0 * W * Nc;
  float mx = 0.f;
  double e2 = 0.0;  // ||yhat||^2 of the kept columns (= ||y||^2 of these rows for a whole plan)
  for (int idx = tid; idx < g * W; idx += nth) {
    const int i = idx / g, gg = idx - i * g;
    const size_t o = base + ((size_t)i * Nc + c) * mt + m0 + gg;
    const T v = c_scale(R[gg * ss + i0 + i], scl);
    yhat[o] = v;
    if (yhat32) yhat32[o] = to_f2(v);
    const float2 f = to_f2(v);
    mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
    e2 += c_abs2d(v);
  }
  if (yy) {
    const double s2 = group_sum(e2, red, tid, nth, bar);
    if (tid == 0) atomicAdd(yy, s2);
  }
  if (ymax) {
    const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));   // non-negative: bits order as values
    if ((tid & 31) == 0) atomicMax(ymax + t, w);
  }
}

template <typename T, typename KIn>
static cudaError_t launch_rows_t(const KIn* ksp, const float* kscale, T* yhat, float2* yhat32, double* yy,
                                 unsigned* ymax, const int* rows, const int* rowoff, int maxm, int Nx, int Ny, int Nt,
                                 int Nc, const FftPlanT<T>& fx, int G_req, int i0, int W, cudaStream_t s) {
  if (maxm <= 0) return cudaSuccess;
  const int G = G_req > 0 ? std::min(G_req, row_group<T>(Nx)) : row_group<T>(Nx);
  const size_t smem = 2 * (size_t)G * (Nx + 1) * sizeof(T);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_hybrid_rows<T, KIn>), smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((maxm + G - 1) / G, Nc, Nt);
  k_hybrid_rows<T, KIn><<<grid, 256, smem, s>>>(ksp, kscale, yhat, yhat32, yy, ymax, rows, rowoff, Nx, Ny, Nt, Nc,
                                                G, fx, 1.0 / sqrt((double)Nx), i0, W > 0 ? W : Nx);
  note_launch();
  return cudaGetLastError();
}

template <typename T, typename Plan>
static cudaError_t rows_dispatch(const void* kspace, int kstorage, const float* kscale, T* yhat, float2* yhat32,
                                 double* yy, unsigned* ymax, const int* rows, const int* rowoff, int maxm, int Nx,
                                 int Ny, int Nt, int Nc, const Plan& fx, int G, int i0, int W, cudaStream_t s) {
  switch (kstorage) {
    case 0: return launch_rows_t<T, float2>(static_cast<const float2*>(kspace), kscale, yhat, yhat32, yy, ymax,
                                            rows, rowoff, maxm, Nx, Ny, Nt, Nc, fx, G, i0, W, s);
    case 1: return launch_rows_t<T, __half2>(static_cast<const __half2*>(kspace), kscale, yhat, yhat32, yy, ymax,
                                             rows, rowoff, maxm, Nx, Ny, Nt, Nc, fx, G, i0, W, s);
    case 2: return launch_rows_t<T, __nv_bfloat162>(static_cast<const __nv_bfloat162*>(kspace), kscale, yhat,
                                                    yhat32, yy, ymax, rows, rowoff, maxm, Nx, Ny, Nt, Nc, fx, G, i0,
                                                    W, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_hybrid_rows(const void* kspace, int kstorage, const float* kscale, float2* yhat, double* yy,
                               unsigned* ymax, const int* rows, const int* rowoff, int maxm, int Nx, int Ny, int Nt,
                               int Nc, FftPlanDev fx, int G, cudaStream_t s, int i0, int W) {
  return rows_dispatch<float2>(kspace, kstorage, kscale, yhat, nullptr, yy, ymax, rows, rowoff, maxm, Nx, Ny, Nt,
                               Nc, fx, G, i0, W, s);
}

cudaError_t launch_hybrid_rows_df(const void* kspace, int kstorage, const float* kscale, dc* yhat_df,
                                  float2* yhat32, double* yy, const int* rows, const int* rowoff, int maxm, int Nx,
                                  int Ny, int Nt, int Nc, FftPlanDf fx, int G, cudaStream_t s, int i0, int W) {
  return rows_dispatch<dc>(kspace, kstorage, kscale, yhat_df, yhat32, yy, nullptr, rows, rowoff, maxm, Nx, Ny, Nt,
                           Nc, fx, G, i0, W, s);
}

constexpr int kCoilGroupMax = 8;

// b = sum_c conj(s_c) . F_v'(zero-filled yhat_c), accumulated in T and rounded
// once to FP32.  With YS != void, also writes ylp = yhat / scale_t in 16 bits
// (the stored coil data of the objective), scale_t = pow2_frame_scale(ymax[t]),
// and yscale[t] = scale_t.
template <typename T, typename YS>
__global__ void __launch_bounds__(256) k_adjoint_combine(const T* __restrict__ yhat,
                                                         const float2* __restrict__ sens, float2* __restrict__ b,
                                                         const int* __restrict__ rows,
                                                         const int* __restrict__ rowoff, int Nx, int Ny, int Nt,
                                                         int Nc, int ncg, FftPlanT<T> fy, double scl, YS* ylp,
                                                         const unsigned* __restrict__ ymax, float* yscale) {
  extern __shared__ __align__(16) unsigned char sm_adj_raw[];
  T* sm_adj = reinterpret_cast<T*>(sm_adj_raw);
  const int i = blockIdx.x, t = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  const T* yh = yhat + (size_t)r0 * Nx * Nc + (size_t)i * Nc * mt;
  const float2* sc = sens + (size_t)i * Nc * Ny;
  float yinv = 1.f;
  if constexpr (!std::is_same<YS, void>::value) {
    const float ysc = pow2_frame_scale(__uint_as_float(ymax[t]));
    yinv = 1.f / ysc;   // exact: a power of two
    if (i == 0 && tid == 0) yscale[t] = ysc;
  }
  T* A = sm_adj;
  T* B = sm_adj + (size_t)ncg * Ny;
  T acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = c_zero<T>();
  const BlockBar bar;
  for (int c0 = 0; c0 < Nc; c0 += ncg) {
    const int cg = min(ncg, Nc - c0);
    for (int idx = tid; idx < cg * Ny; idx += nth) A[idx] = c_zero<T>();
    __syncthreads();
    for (int idx = tid; idx < cg * mt; idx += nth) {
      const int c = idx / mt, m = idx - c * mt;
      const T v = yh[(size_t)(c0 + c) * mt + m];
      A[c * Ny + rows[r0 + m]] = v;
      if constexpr (!std::is_same<YS, void>::value) {
        const float2 f = to_f2(v);
        ylp[(size_t)r0 * Nx * Nc + (size_t)i * Nc * mt + (size_t)(c0 + c) * mt + m] =
            Elem<YS>::cvt(make_float2(f.x * yinv, f.y * yinv));
      }
    }
    __syncthreads();
    T* R = fft_run(A, B, cg, Ny, 1, fy, true, tid, nth, bar);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = tid + q * nth;
      if (j < Ny) {
        for (int c = 0; c < cg; ++c) c_fmac(acc[q], from_f2<T>(__ldg(sc + (size_t)(c0 + c) * Ny + j)), R[c * Ny + j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = tid + q * nth;
    if (j < Ny) b[((size_t)t * Nx + i) * Ny + j] = to_f2(c_scale(acc[q], scl));
  }
}

template <typename T>
static int coil_group(int Nc, int Ny) {
  int g = kCoilGroupMax;
  while (g > 1 && 2 * (size_t)g * Ny * sizeof(T) > 96 * 1024) --g;
  return g < Nc ? g : Nc;
}

template <typename T, typename YS>
static cudaError_t launch_combine_t(const T* yhat, const float2* sens, float2* b, const int* rows, const int* rowoff,
                                    int Nx, int Ny, int Nt, int Nc, const FftPlanT<T>& fy, YS* ylp,
                                    const unsigned* ymax, float* yscale, int ncg_req, cudaStream_t s) {
  if (Ny > 1024) return cudaErrorInvalidValue;
  const int ncg = ncg_req > 0 ? std::min(ncg_req, coil_group<T>(Nc, Ny)) : coil_group<T>(Nc, Ny);
  const size_t smem = 2 * (size_t)ncg * Ny * sizeof(T);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_adjoint_combine<T, YS>), smem);
    if (e != cudaSuccess) return e;
  }
  k_adjoint_combine<T, YS><<<dim3(Nx, Nt), 256, smem, s>>>(yhat, sens, b, rows, rowoff, Nx, Ny, Nt, Nc, ncg, fy,
                                                           1.0 / sqrt((double)Ny), ylp, ymax, yscale);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_adjoint_combine(const float2* yhat, const float2* sens, float2* b, const int* rows,
                                   const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDev fy, int ystorage,
                                   void* ylp, const unsigned* ymax, float* yscale, int ncg, cudaStream_t s) {
  switch (ystorage) {
    case 0: return launch_combine_t<float2, void>(yhat, sens, b, rows, rowoff, Nx, Ny, Nt, Nc, fy, nullptr, nullptr,
                                                  nullptr, ncg, s);
    case 1: return launch_combine_t<float2, __half2>(yhat, sens, b, rows, rowoff, Nx, Ny, Nt, Nc, fy,
                                                     static_cast<__half2*>(ylp), ymax, yscale, ncg, s);
    case 2: return launch_combine_t<float2, __nv_bfloat162>(yhat, sens, b, rows, rowoff, Nx, Ny, Nt, Nc, fy,
                                                            static_cast<__nv_bfloat162*>(ylp), ymax, yscale, ncg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adjoint_combine_df(const dc* yhat_df, const float2* sens, float2* b, const int* rows,
                                      const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDf fy, int ncg,
                                      cudaStream_t s) {
  return launch_combine_t<dc, void>(yhat_df, sens, b, rows, rowoff, Nx, Ny, Nt, Nc, fy, nullptr, nullptr, nullptr,
                                    ncg, s);
}

int row_group_max(int Nx, bool wide) { return wide ? row_group<dc>(Nx) : row_group<float2>(Nx); }
int coil_group_max(int Nc, int Ny, bool wide) { return wide ? coil_group<dc>(Nc, Ny) : coil_group<float2>(Nc, Ny); }

// ---- 16-bit k-space with per-frame scales ----------------------------------
// Three launches: the largest |component| of every frame (float bits into
// the scale array), the quantisation q = k / scale_t (one rounding: the
// scale is a power of two), and the bits replaced by the scale values.
__global__ void k_frame_absmax(const float2* __restrict__ k, long long per_frame, unsigned* mx) {
  const int t = blockIdx.y;
  const float2* kf = k + (size_t)t * per_frame;
  float m = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per_frame;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 v = kf[e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  if ((threadIdx.x & 31) == 0) atomicMax(mx + t, w);
}

template <typename E>
__global__ void k_quantize_frames(const float2* __restrict__ k, long long per_frame, const unsigned* __restrict__ mx,
                                  E* __restrict__ out) {
  const int t = blockIdx.y;
  const float inv = 1.f / pow2_frame_scale(__uint_as_float(mx[t]));
  const size_t o = (size_t)t * per_frame;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per_frame;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 v = k[o + e];
    out[o + e] = Elem<E>::cvt(make_float2(v.x * inv, v.y * inv));
  }
}

__global__ void k_bits_to_scale(float* scale, int Nt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < Nt) scale[t] = pow2_frame_scale(__uint_as_float(reinterpret_cast<unsigned*>(scale)[t]));
}

cudaError_t launch_quantize_kspace(const float2* k, long long per_frame, int Nt, int storage, void* out,
                                   float* frame_scale, cudaStream_t s) {
  if (storage != 1 && storage != 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(frame_scale, 0, (size_t)Nt * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int bx = (int)std::min<long long>(64, (per_frame + 255) / 256);
  const dim3 grid(std::max(bx, 1), Nt);
  unsigned* bits = reinterpret_cast<unsigned*>(frame_scale);
  k_frame_absmax<<<grid, 256, 0, s>>>(k, per_frame, bits); note_launch();
  if (storage == 1) k_quantize_frames<__half2><<<grid, 256, 0, s>>>(k, per_frame, bits, static_cast<__half2*>(out));
  else k_quantize_frames<__nv_bfloat162><<<grid, 256, 0, s>>>(k, per_frame, bits, static_cast<__nv_bfloat162*>(out));
  note_launch();
  k_bits_to_scale<<<(Nt + 127) / 128, 128, 0, s>>>(frame_scale, Nt); note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_forward_cols(const float2* __restrict__ x, const float2* __restrict__ sens,
                                                      float2* __restrict__ zhat, const int* __restrict__ rows,
                                                      const int* __restrict__ rowoff, int Nx, int Ny, int Nt, int Nc,
                                                      int ncg, FftPlanDev fy, float scl) {
  extern __shared__ float2 sm_fwd[];
  const int i = blockIdx.x, t = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  float2* xc = sm_fwd;
  float2* A = xc + Ny;
  float2* B = A + (size_t)ncg * Ny;
  const float2* sc = sens + (size_t)i * Nc * Ny;
  float2* zh = zhat + (size_t)r0 * Nx * Nc + (size_t)i * Nc * mt;
  for (int j = tid; j < Ny; j += nth) xc[j] = x[((size_t)t * Nx + i) * Ny + j];
  __syncthreads();
  const BlockBar bar;
  for (int c0 = 0; c0 < Nc; c0 += ncg) {
    const int cg = min(ncg, Nc - c0);
    for (int idx = tid; idx < cg * Ny; idx += nth) {
      const int c = idx / Ny, j = idx - c * Ny;
      A[idx] = c_mul(__ldg(sc + (size_t)(c0 + c) * Ny + j), xc[j]);
    }
    __syncthreads();
    float2* R = fft_run(A, B, cg, Ny, 1, fy, false, tid, nth, bar);
    for (int idx = tid; idx < cg * mt; idx += nth) {
      const int c = idx / mt, m = idx - c * mt;
      zh[(size_t)(c0 + c) * mt + m] = c_scale(R[c * Ny + rows[r0 + m]], scl);
    }
    __syncthreads();
  }
}

cudaError_t launch_forward_cols(const float2* x, const float2* sens, float2* zhat, const int* rows,
                                const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDev fy, cudaStream_t s) {
  const int ncg = coil_group<float2>(Nc, Ny);
  const size_t smem = ((size_t)Ny + 2 * (size_t)ncg * Ny) * sizeof(float2);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_forward_cols), smem);
    if (e != cudaSuccess) return e;
  }
  k_forward_cols<<<dim3(Nx, Nt), 256, smem, s>>>(x, sens, zhat, rows, rowoff, Nx, Ny, Nt, Nc, ncg, fy,
                                                 (float)(1.0 / sqrt((double)Ny))); note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_forward_rows(const float2* __restrict__ zhat, float2* __restrict__ ksp,
                                                      const int* __restrict__ rows, const int* __restrict__ rowoff,
                                                      int Nx, int Ny, int Nt, int Nc, FftPlanDev fx, float scl) {
  extern __shared__ float2 sm_frow[];
  const int t = blockIdx.z, c = blockIdx.y, m0 = blockIdx.x * kRowGroup;
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  if (m0 >= mt) return;
  const int g = min(kRowGroup, mt - m0);
  const int ss = Nx + 1;
  float2* A = sm_frow;
  float2* B = sm_frow + (size_t)kRowGroup * ss;
  const int tid = threadIdx.x, nth = blockDim.x;
  const size_t base = (size_t)r0 * Nx * Nc;
  for (int idx = tid; idx < g * Nx; idx += nth) {
    const int i = idx / g, gg = idx - i * g;
    A[gg * ss + i] = zhat[base + ((size_t)i * Nc + c) * mt + m0 + gg];
  }
  __syncthreads();
  const BlockBar bar;
  float2* R = fft_run(A, B, g, ss, 1, fx, false, tid, nth, bar);
  for (int idx = tid; idx < g * Nx; idx += nth) {
    const int gg = idx / Nx, kx = idx - gg * Nx;
    const int row = rows[r0 + m0 + gg];
    ksp[(((size_t)t * Nc + c) * Ny + row) * Nx + kx] = c_scale(R[gg * ss + kx], scl);
  }
}

cudaError_t launch_forward_rows(const float2* zhat, float2* kspace, const int* rows, const int* rowoff, int maxm,
                                int Nx, int Ny, int Nt, int Nc, FftPlanDev fx, cudaStream_t s) {
  if (maxm <= 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)kRowGroup * (Nx + 1) * sizeof(float2);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_forward_rows), smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((maxm + kRowGroup - 1) / kRowGroup, Nc, Nt);
  k_forward_rows<<<grid, 256, smem, s>>>(zhat, kspace, rows, rowoff, Nx, Ny, Nt, Nc, fx,
                                         (float)(1.0 / sqrt((double)Nx))); note_launch();
  return cudaGetLastError();
}

// out[b*obs + c*ors + r] = in[b*ibs + r*C + c]
__global__ void k_transpose(const float2* __restrict__ in, float2* __restrict__ out, int R, int C, long long ibs,
                            long long irs, long long obs, long long ors) {
  __shared__ float2 tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    if (r < R && c < C) tile[k][tx] = in[b * ibs + (long long)r * irs + c];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (r < R && c < C) out[b * obs + (long long)c * ors + r] = tile[tx][k];
  }
}

cudaError_t launch_transpose(const float2* in, float2* out, int B, int R, int C, long long ibs, long long obs,
                             long long ors, cudaStream_t s, long long irs) {
  dim3 grid((C + 31) / 32, (R + 31) / 32, B);
  k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, out, R, C, ibs, irs > 0 ? irs : C, obs, ors); note_launch();
  return cudaGetLastError();
}

}  // namespace recon
