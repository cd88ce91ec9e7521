// Allocation-free variant of the per-column inverse: recon_gram_inverse_noalloc.
//
// Some callers cannot call cudaMalloc: a real-time scanner pipeline that
// reserves all of its device memory at start-up and must not allocate while
// acquiring (an allocation can block on the device and fragment the heap), or
// code embedded in a host framework whose own allocator owns the device.
// They pass only inputs and outputs; this file keeps the FP64 factorisation
// workspace in a fixed file-scope device array instead.
//
// The array is kScratchBytes (16 MiB) per GPU that loads the library and lives
// until process exit.  It holds one Ny x Ny FP64 complex workspace per CTA
// plus a status word, so floor((16 MiB - 256) / (16 Ny^2)) blocks are
// factorised at once (Ny = 256: 15; Ny = 512: 3; Ny >= 725: one CTA, and the
// blocks then run one after another on a single SM).  In
// host code the array's name is only a host-side stand-in: the device address
// is obtained once per device with cudaGetSymbolAddress and passed to the
// kernel.  Every call shares the array, so calls that overlap on the GPU race
// on it.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/recon.h"
#include "kernels.h"

namespace recon {

constexpr size_t kScratchBytes = 16u << 20;
constexpr size_t kScratchStatusBytes = 256;  // status word area at the front
constexpr int kNoAllocThreads = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// (mu I + C (.) K)^{-1} for one block: C from the block's row mask, K from its
// coil column; same FP64 steps as the plan (Section IV-C, Eqs. HconjH,
// eigen_mu): Cholesky, triangular inverse, A = Z'Z, rounded once to FP32 and
// written as a dense Hermitian matrix.
__global__ void __launch_bounds__(kNoAllocThreads) k_gram_inverse_static(
    const uint8_t* __restrict__ mask, const float2* __restrict__ sens, int Ny, int Nc, int nblk, double mu,
    float2* __restrict__ out, unsigned char* __restrict__ scratch) {
  extern __shared__ double2 zs_na[];
  const int n = Ny, tid = threadIdx.x;
  int* status = reinterpret_cast<int*>(scratch);
  double2* W = reinterpret_cast<double2*>(scratch + kScratchStatusBytes) + (size_t)blockIdx.x * n * n;
  double2* sc = zs_na;                   // [Nc][n]
  double2* circ = zs_na + (size_t)Nc * n;  // [n]
  double2* cb = circ + n;                // [n]
  const int ty = tid >> 4, tx = tid & 15;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const uint8_t* mk = mask + (size_t)blk * n;
    for (int idx = tid; idx < Nc * n; idx += kNoAllocThreads) {
      const float2 v = sens[(size_t)blk * Nc * n + idx];
      sc[idx] = make_double2(v.x, v.y);
    }
    // c[d] = (1/n) sum_{q sampled} exp(+2 pi i q d / n)
    for (int d = tid; d < n; d += kNoAllocThreads) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < n; ++q) {
        if (!mk[q]) continue;
        double sv, cv;
        sincospi(2.0 * (double)(((long long)q * d) % n) / (double)n, &sv, &cv);
        re += cv; im += sv;
      }
      circ[d] = make_double2(re / n, im / n);
    }
    __syncthreads();
    for (long long idx = tid; idx < (long long)n * n; idx += kNoAllocThreads) {
      const int j = (int)(idx / n), k = (int)(idx - (long long)j * n);
      if (k > j) continue;
      double2 K = make_double2(0.0, 0.0);
      for (int c = 0; c < Nc; ++c) z_fmac(K, sc[c * n + j], sc[c * n + k]);  // conj(s_j) s_k
      double2 g = z_mul(circ[j - k], K);
      if (j == k) g.x += mu;
      W[(size_t)j * n + k] = g;
    }
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < n; ++k) {
      double d = W[(size_t)k * n + k].x;
      if (!(d > 0.0) || !isfinite(d)) { bad = true; d = 1.0; }   // also NaN and +Inf
      d = sqrt(d);
      const double inv = 1.0 / d;
      for (int j = k + 1 + tid; j < n; j += kNoAllocThreads) {
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
            w.x -= fma(a.x, b.x, a.y * b.y);
            w.y -= fma(a.y, b.x, -a.x * b.y);
            W[(size_t)j * n + l] = w;
          }
        }
      }
      __syncthreads();
    }
    if (bad && tid == 0) atomicOr(status, DEV_ERR_NOT_PD);
    for (int j = 0; j < n; ++j) {
      for (int l = tid; l <= j; l += kNoAllocThreads) cb[l] = W[(size_t)j * n + l];
      __syncthreads();
      const double ljj = cb[j].x;
      for (int c = tid; c <= j; c += kNoAllocThreads) {
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
    float2* Ob = out + (size_t)blk * n * n;
    for (int jb = 0; jb < n; jb += 16) {
      for (int kb = jb; kb < n; kb += 16) {
        const int j = jb + ty, k = kb + tx;
        if (j < n && k < n && j <= k) {
          double2 s = make_double2(0.0, 0.0);
          for (int l = k; l < n; ++l) z_fmac(s, W[(size_t)l * n + j], W[(size_t)l * n + k]);
          if (j == k) s.y = 0.0;
          Ob[(size_t)j * n + k] = make_float2((float)s.x, (float)s.y);
          if (j != k) Ob[(size_t)k * n + j] = make_float2((float)s.x, (float)-s.y);
        }
      }
    }
    __syncthreads();
  }
}

namespace {

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

recon_status na_fail(recon_status st, const std::string& why) {
  set_last_error(why);
  return st;
}

}  // namespace

}  // namespace recon

using namespace recon;

extern "C" recon_status recon_gram_inverse_noalloc(int Ny, int Nc, int nblk, const uint8_t* mask, const float* sens,
                                                   float mu, float* out, void* stream) {
  if (Ny < 1 || Nc < 1 || nblk < 0 || !mask || !sens || !out || !(mu > 0.f) || !std::isfinite(mu))
    return na_fail(RECON_ERR_INVALID_ARG, "bad argument");
  const size_t ws = (size_t)Ny * Ny * sizeof(double2);
  if (ws > kScratchBytes - kScratchStatusBytes)
    return na_fail(RECON_ERR_UNSUPPORTED, "Ny=" + std::to_string(Ny) + " needs a " + std::to_string(ws) +
                                              "-byte workspace; the static scratch holds " +
                                              std::to_string(kScratchBytes - kScratchStatusBytes) +
                                              " bytes (Ny <= 1023)");
  const size_t smem = ((size_t)Nc + 2) * Ny * sizeof(double2);
  if (smem > 200 * 1024) return na_fail(RECON_ERR_UNSUPPORTED, "(Nc + 2) * Ny too large for shared memory");
  if (nblk == 0) return RECON_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return na_fail(RECON_ERR_CUDA, "cudaGetDevice failed");
  void* base = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_dev[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_dev[dev] = nullptr;
        return na_fail(RECON_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_scratch_dev[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int per = (int)((kScratchBytes - kScratchStatusBytes) / ws);
  const int grid = nblk < per ? nblk : per;
  e = cudaMemsetAsync(base, 0, sizeof(int), s);  // status word of this call
  if (e == cudaSuccess)   // the dynamic shared-memory limit is a per-device attribute: cheap to set every call
    e = cudaFuncSetAttribute(k_gram_inverse_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    k_gram_inverse_static<<<grid, kNoAllocThreads, smem, s>>>(mask, reinterpret_cast<const float2*>(sens), Ny, Nc,
                                                              nblk, (double)mu, reinterpret_cast<float2*>(out),
                                                              static_cast<unsigned char*>(base));
    note_launch();
    e = cudaGetLastError();
  }
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, base, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(RECON_ERR_CUDA, cudaGetErrorString(e));
  if (status & DEV_ERR_NOT_PD) return na_fail(RECON_ERR_NONFINITE, "a block is not positive definite");
  return RECON_OK;
}
