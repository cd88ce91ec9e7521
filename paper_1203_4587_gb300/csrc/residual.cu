// ADMM residuals at the end of a solve, for recon_info, in the stacked form of
// Boyd et al. (2011, Sec. 3.3) with the paper's penalty weights.
//
// Algorithm 2 (temporal TV), splits v = D_t m (mu1, scaled dual d1) and m = x
// (mu2, d2):
//   primal = sqrt(||v_K - D_t m_K||^2 + ||m_K - x_K||^2)
//   dual   = sqrt(mu1^2 ||D_t (m_K - m_{K-1})||^2 + mu2^2 ||m_K - m_{K-1}||^2),
// where v_K - D_t m_K = d1_{K-1} - d1_K (the d1-update).  After K iterations
// the ping-pong state buffers still hold m_K, m_{K-1}, d1_K and d1_{K-1}, so one
// pass over them gives the four sums.
//
// Algorithm 1 (Psi = unitary temporal DFT), split v = w (mu, scaled dual d):
//   primal = ||w_K - v_K||,   dual = mu ||w_K - w_{K-1}||.
// The temporal step stores u = v + d (the coefficients it hands to the
// synthesis) and the inverse step xhat = Psi' w.  With d_{K-1} = u_{K-1} -
// w_{K-1} and v_K = u_K - d_{K-1},
//   w_K - v_K = Psi (xhat_K - xhat_{K-1}) - (u_K - u_{K-1})   (K >= 2),
//   w_1 - v_1 = Psi xhat_1 - u_1                               (d_0 = 0),
// and ||w_K - w_{K-1}|| = ||xhat_K - xhat_{K-1}|| as Psi is unitary (xhat_0 =
// H'y).  u_K and u_{K-1} are the two ping-pong buffers; the solve copies
// xhat_{K-1} aside before the last inverse step overwrites it.
//
// Algorithm 1 with the undecimated Haar frame (tight, Psi'Psi = I, not
// unitary): the temporal step keeps u = v + d, s = Psi'u and xhat, with
// w_k = u_k + Psi(xhat_k - s_k) and d_k = u_k - w_k = -Psi(xhat_k - s_k)
// (k >= 1; w_0 = Psi H'y, d_0 = 0).  With D = (xhat_K - s_K) - (xhat_{K-1} -
// s_{K-1}) and Psi'Psi = I,
//   ||w_K - v_K||^2 = ||d_{K-1} - d_K||^2 = ||D||^2          (K >= 2)
//   ||w_1 - v_1||^2 = ||d_1||^2 = ||xhat_1 - s_1||^2
//   ||w_K - w_{K-1}||^2 = ||du||^2 + 2 Re<Psi'du, D> + ||D||^2,  du = u_K - u_{K-1},
// Psi'du = s_K - s_{K-1}; at K = 1, u_0 = s_0 = 0 and xhat_0 - s_0 stands for
// H'y (w_0 = Psi H'y).  No transform is needed: all but ||du||^2 are sums
// over the image, ||du||^2 over the L+1 coefficient channels.
//
// Products are FP32, summed per thread in FP32 (Kahan) and across threads in
// FP64.
#include <algorithm>

#include "fft.cuh"
#include "kahan.cuh"
#include "plan.h"

namespace recon {

namespace {

constexpr int kResThreads = 256;
constexpr int kMaxResNt = 128;   // the plans' Nt limit; 2 kMaxResNt kResPix complex64 = 32 KB of shared memory

// acc[0] += ||m - x||^2, acc[1] += ||d1p - d1||^2, acc[2] += ||dm||^2,
// acc[3] += ||D_t dm||^2 (dm = m - mp); fields [Nt][npix], d1 [Nt-1][npix]
// (d1p null: zeros)
__global__ void __launch_bounds__(kResThreads) k_tv_residuals(const float2* __restrict__ x, const float2* __restrict__ m,
                                                              const float2* __restrict__ mp, const float2* __restrict__ d1,
                                                              const float2* __restrict__ d1p, long long npix, int Nt,
                                                              double* acc) {
  __shared__ double red[32];
  const long long n = npix * Nt;
  KahanSum a0, a1, a2, a3;
  for (long long idx = (long long)blockIdx.x * kResThreads + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * kResThreads) {
    const float2 mv = m[idx], xv = x[idx], pv = mp[idx];
    const float2 mx = c_sub(mv, xv), dm = c_sub(mv, pv);
    a0.add(fmaf(mx.x, mx.x, mx.y * mx.y));
    a2.add(fmaf(dm.x, dm.x, dm.y * dm.y));
    if (idx + npix < n) {   // t + 1 < Nt
      const float2 dn = c_sub(m[idx + npix], mp[idx + npix]);
      const float2 ddm = c_sub(dn, dm);
      a3.add(fmaf(ddm.x, ddm.x, ddm.y * ddm.y));
      const float2 dp = d1p ? d1p[idx] : make_float2(0.f, 0.f);
      const float2 dd = c_sub(dp, d1[idx]);
      a1.add(fmaf(dd.x, dd.x, dd.y * dd.y));
    }
  }
  const double s0 = group_sum((double)a0.s, red, threadIdx.x, kResThreads, BlockBar());
  const double s1 = group_sum((double)a1.s, red, threadIdx.x, kResThreads, BlockBar());
  const double s2 = group_sum((double)a2.s, red, threadIdx.x, kResThreads, BlockBar());
  const double s3 = group_sum((double)a3.s, red, threadIdx.x, kResThreads, BlockBar());
  if (threadIdx.x == 0) {
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, s1);
    atomicAdd(acc + 2, s2);
    atomicAdd(acc + 3, s3);
  }
}

// acc[0] += ||w_K - v_K||^2, acc[1] += ||xhat_K - xhat_{K-1}||^2 for kResPix
// pixels per block: the difference tile [Nt][kResPix] is transformed along t
// in shared memory by the same Stockham stages as the temporal step.
// xh_prev null: K = 1 (the primal transforms xhat_1 itself, u_prev = 0, and
// the dual compares with b = H'y).
constexpr int kResPix = 16;

__global__ void __launch_bounds__(kResThreads) k_dft_residuals(const float2* __restrict__ xh,
                                                               const float2* __restrict__ xh_prev,
                                                               const float2* __restrict__ b, const float2* __restrict__ u,
                                                               const float2* __restrict__ u_prev, long long npix, int Nt,
                                                               FftPlanDev ft, double* acc) {
  extern __shared__ float2 sm_res[];
  __shared__ double red[32];
  float2* A = sm_res;
  float2* B = sm_res + (size_t)Nt * kResPix;
  const int tid = threadIdx.x, nth = blockDim.x;
  const long long pix0 = (long long)blockIdx.x * kResPix;
  const int npx = (int)min((long long)kResPix, npix - pix0);
  KahanSum ad, ap;
  for (int idx = tid; idx < Nt * kResPix; idx += nth) {
    const int t = idx / kResPix, pp = idx - t * kResPix;
    float2 a = make_float2(0.f, 0.f);
    if (pp < npx) {
      const long long g = (long long)t * npix + pix0 + pp;
      const float2 xv = xh[g];
      const float2 dx = c_sub(xv, xh_prev ? xh_prev[g] : b[g]);
      ad.add(fmaf(dx.x, dx.x, dx.y * dx.y));
      a = xh_prev ? dx : xv;
    }
    A[idx] = a;
  }
  __syncthreads();
  const BlockBar bar;
  const float2* W = fft_run(A, B, kResPix, 1, kResPix, ft, false, tid, nth, bar);
  const float sc = rsqrtf((float)Nt);
  for (int idx = tid; idx < Nt * kResPix; idx += nth) {
    const int t = idx / kResPix, pp = idx - t * kResPix;
    if (pp < npx) {
      const long long g = (long long)t * npix + pix0 + pp;
      const float2 du = u_prev ? c_sub(u[g], u_prev[g]) : u[g];
      const float2 e = c_sub(c_scale(W[idx], sc), du);
      ap.add(fmaf(e.x, e.x, e.y * e.y));
    }
  }
  const double s0 = group_sum((double)ap.s, red, tid, nth, bar);
  const double s1 = group_sum((double)ad.s, red, tid, nth, bar);
  if (tid == 0) {
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, s1);
  }
}

// acc[0] += the primal sum, acc[1] += ||w_K - w_{K-1}||^2 (Haar frame, as
// above).  Image fields [Nt][npix]; u [L+1][Nt][npix].  first: K = 1 (xh_prev,
// s_prev and u_prev unused).
__global__ void __launch_bounds__(kResThreads) k_haar_residuals(const float2* __restrict__ xh,
                                                                const float2* __restrict__ xh_prev,
                                                                const float2* __restrict__ b,
                                                                const float2* __restrict__ s,
                                                                const float2* __restrict__ s_prev,
                                                                const float2* __restrict__ u,
                                                                const float2* __restrict__ u_prev, long long n,
                                                                int nch, int first, double* acc) {
  __shared__ double red[32];
  KahanSum ap, ad;
  const long long stride = (long long)gridDim.x * kResThreads;
  for (long long g = (long long)blockIdx.x * kResThreads + threadIdx.x; g < n; g += stride) {
    const float2 e = c_sub(xh[g], s[g]);
    const float2 q = first ? b[g] : c_sub(xh_prev[g], s_prev[g]);
    const float2 D = c_sub(e, q);
    const float2 dp = first ? e : D;
    ap.add(fmaf(dp.x, dp.x, dp.y * dp.y));
    const float2 ds = first ? s[g] : c_sub(s[g], s_prev[g]);
    ad.add(fmaf(2.f * ds.x, D.x, fmaf(2.f * ds.y, D.y, fmaf(D.x, D.x, D.y * D.y))));
  }
  const long long nu = n * nch;
  for (long long g = (long long)blockIdx.x * kResThreads + threadIdx.x; g < nu; g += stride) {
    const float2 du = first ? u[g] : c_sub(u[g], u_prev[g]);
    ad.add(fmaf(du.x, du.x, du.y * du.y));
  }
  const double s0 = group_sum((double)ap.s, red, threadIdx.x, kResThreads, BlockBar());
  const double s1 = group_sum((double)ad.s, red, threadIdx.x, kResThreads, BlockBar());
  if (threadIdx.x == 0) {
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, s1);
  }
}

}  // namespace

// The sums of plan p after its K iterations.  TV: the state of iteration K
// sits at index K & 1 of the ping-pong buffers, that of K-1 at (K-1) & 1 (m_0 =
// H'y and d1_0 = 0 for K = 1).  DFT and Haar: u_K (and s_K) at K & 1, u_{K-1}
// (s_{K-1}) at (K-1) & 1, xhat_{K-1} in res_prev (K >= 2).  The spatio-temporal
// prior: nothing (NaN in recon_info).
recon_status launch_residuals(recon_plan* p, cudaStream_t s) {
  const int K = p->opts.max_iters;
  if (K < 1) return RECON_OK;
  const long long npix = (long long)p->npix();
  const long long n = npix * p->Nt;
  if (p->prior == RECON_PRIOR_TV) {
    RC(cudaMemsetAsync(p->res_acc, 0, 4 * sizeof(double), s));
    const float2* mp = K == 1 ? p->b : p->s0[(K - 1) & 1];
    const float2* d1p = K == 1 ? nullptr : p->s1[(K - 1) & 1];
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + kResThreads - 1) / kResThreads,
                                                                     4LL * std::max(1, p->num_sms)));
    k_tv_residuals<<<grid, kResThreads, 0, s>>>(p->x, p->s0[K & 1], mp, p->s1[K & 1], d1p, npix, p->Nt, p->res_acc);
  } else if (p->prior == RECON_PRIOR_DFT) {
    if (p->Nt > kMaxResNt) return fail(RECON_ERR_INVALID_ARG, "residuals: Nt above the residual kernel's tile");
    RC(cudaMemsetAsync(p->res_acc, 0, 4 * sizeof(double), s));
    const int grid = (int)((npix + kResPix - 1) / kResPix);
    const size_t smem = 2 * (size_t)p->Nt * kResPix * sizeof(float2);
    k_dft_residuals<<<grid, kResThreads, smem, s>>>(p->x, K == 1 ? nullptr : p->res_prev, p->b, p->s0[K & 1],
                                                   K == 1 ? nullptr : p->s0[(K - 1) & 1], npix, p->Nt, p->ft,
                                                   p->res_acc);
  } else if (p->prior == RECON_PRIOR_HAAR) {
    RC(cudaMemsetAsync(p->res_acc, 0, 4 * sizeof(double), s));
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + kResThreads - 1) / kResThreads,
                                                                     4LL * std::max(1, p->num_sms)));
    const int first = K == 1;
    k_haar_residuals<<<grid, kResThreads, 0, s>>>(p->x, first ? nullptr : p->res_prev, p->b, p->s1[K & 1],
                                                  first ? nullptr : p->s1[(K - 1) & 1], p->s0[K & 1],
                                                  first ? nullptr : p->s0[(K - 1) & 1], n,
                                                  p->opts.frame_levels + 1, first, p->res_acc);
  } else {
    return RECON_OK;
  }
  note_launch();
  RC(cudaGetLastError());
  return RECON_OK;
}

}  // namespace recon
