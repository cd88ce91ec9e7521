// ADMM residuals of Algorithm 2 (temporal TV) at the end of a solve, for
// recon_info: with the two splits v = D_t m (penalty mu1, scaled dual d1) and
// m = x (mu2, d2), in the stacked form of Boyd et al. (2011, Sec. 3.3),
//   primal = sqrt(||v_K - D_t m_K||^2 + ||m_K - x_K||^2)
//   dual   = sqrt(mu1^2 ||D_t (m_K - m_{K-1})||^2 + mu2^2 ||m_K - m_{K-1}||^2),
// where v_K - D_t m_K = d1_{K-1} - d1_K (the d1-update).  After K iterations
// the ping-pong state buffers still hold m_K, m_{K-1}, d1_K and d1_{K-1}, so one
// pass over them gives the four sums; products are FP32, summed per thread in
// FP32 (Kahan) and across threads in FP64.
#include <algorithm>

#include "kahan.cuh"
#include "plan.h"

namespace recon {

namespace {

constexpr int kResThreads = 256;

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

}  // namespace

// The sums of plan p after its K iterations (temporal TV only): the state of
// iteration K sits at index K & 1 of the ping-pong buffers, that of K-1 at
// (K-1) & 1 (m_0 = H'y and d1_0 = 0 for K = 1).
recon_status launch_tv_residuals(recon_plan* p, cudaStream_t s) {
  const int K = p->opts.max_iters;
  if (p->prior != RECON_PRIOR_TV || K < 1) return RECON_OK;
  RC(cudaMemsetAsync(p->res_acc, 0, 4 * sizeof(double), s));
  const long long npix = (long long)p->npix();
  const long long n = npix * p->Nt;
  const float2* mp = K == 1 ? p->b : p->s0[(K - 1) & 1];
  const float2* d1p = K == 1 ? nullptr : p->s1[(K - 1) & 1];
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + kResThreads - 1) / kResThreads,
                                                                   4LL * std::max(1, p->num_sms)));
  k_tv_residuals<<<grid, kResThreads, 0, s>>>(p->x, p->s0[K & 1], mp, p->s1[K & 1], d1p, npix, p->Nt, p->res_acc);
  note_launch();
  RC(cudaGetLastError());
  return RECON_OK;
}

}  // namespace recon
