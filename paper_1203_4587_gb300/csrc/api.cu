// C ABI of the reconstruction library (include/recon.h).
//
// A plan owns every device buffer a solve needs, so recon_solve allocates
// nothing.  One ADMM iteration enqueues: the temporal kernel (Algorithm 2's
// v, m, d1 updates, or Algorithm 1's v, d and Psi/Psi' steps), the J(k-1)
// finalize kernel (when the objective is on) and the column-inverse kernel
// (x = (mu I + H'H)^{-1} r with the ||y - Hx||^2 epilogue).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "host_logic.h"
#include "plan.h"

using namespace recon;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace recon {

recon_status fail(recon_status st, const std::string& why) {
  g_last_error = why;
  return st;
}

recon_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? RECON_ERR_OOM : RECON_ERR_CUDA;
}

}  // namespace recon

namespace recon {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaError_t SmemAttrCache::ensure(const void* kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (bytes <= v[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  size_t cur = v[dev].load(std::memory_order_relaxed);
  while (cur < bytes && !v[dev].compare_exchange_weak(cur, bytes, std::memory_order_relaxed)) {}
  return cudaSuccess;
}
void set_last_error(const std::string& why) { g_last_error = why; }

void fill_twiddles_host(int n, float2* tw) {
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)n;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
}

// (re_hi, re_lo, im_hi, im_lo): each FP64 value split into its FP32 rounding
// and the FP32 rounding of the remainder
void fill_twiddles_host_df(int n, float4* tw) {
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)n;
    const double c = std::cos(a), s = std::sin(a);
    const float ch = (float)c, sh = (float)s;
    tw[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}

template <typename T>
static FftPlanT<T> fft_plan_t(int n, const T* d_tw) {
  FftPlanT<T> P{};
  P.n = n;
  P.tw = d_tw;
  P.ns = fft_factor(n, P.radix, kFftMaxStages);
  return P;
}

FftPlanDev make_fft_plan_host(int n, const float2* d_tw) { return fft_plan_t<float2>(n, d_tw); }
FftPlanDf make_fft_plan_host_df(int n, const dc* d_tw) { return fft_plan_t<dc>(n, d_tw); }

cudaError_t plan_create_events(recon_plan* p) {
  if (!p->ev_col.empty()) return cudaSuccess;
  const size_t ne = 2 * ((size_t)p->opts.max_iters + 2);
  p->ev_col.assign(ne, nullptr);
  p->ev_tmp.assign(ne, nullptr);
  for (auto& e : p->ev_col) {
    const cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) return ce;
  }
  for (auto& e : p->ev_tmp) {
    const cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) return ce;
  }
  for (auto& e : p->ev_solve) {
    const cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) return ce;
  }
  return cudaSuccess;
}

}  // namespace recon

recon_plan::~recon_plan() {
  delete eng;
  delete eng_inv;
  for (cudaEvent_t e : ev_col)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_tmp)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_solve)
    if (e) cudaEventDestroy(e);
  for (void* q : allocs) cudaFree(q);
}

namespace {
recon_status plan_invert(recon_plan* p, cudaStream_t s);   // below
}  // namespace

extern "C" {

void recon_default_opts(recon_opts* o) {
  if (!o) return;
  o->rho = 0.5f;
  o->max_iters = 50;
  o->tol = 0.0;
  o->storage = RECON_STORAGE_FP32;
  o->objective = 1;
  o->mask_full = 0;
  o->col_stages = 0;
  o->profile = 0;
  o->frame_levels = 2;
  o->spatial_weight = 1.f;
  o->cg_steps = 5;
  o->persistent = 0;
  o->overlap = 1;
}

const char* recon_status_string(recon_status s) {
  switch (s) {
    case RECON_OK: return "RECON_OK";
    case RECON_ERR_INVALID_ARG: return "RECON_ERR_INVALID_ARG";
    case RECON_ERR_MASK_NOT_CARTESIAN: return "RECON_ERR_MASK_NOT_CARTESIAN";
    case RECON_ERR_OOM: return "RECON_ERR_OOM";
    case RECON_ERR_CUDA: return "RECON_ERR_CUDA";
    case RECON_ERR_TIMEOUT: return "RECON_ERR_TIMEOUT";
    case RECON_ERR_NONFINITE: return "RECON_ERR_NONFINITE";
    case RECON_ERR_UNSUPPORTED: return "RECON_ERR_UNSUPPORTED";
  }
  return "RECON_ERR_UNKNOWN";
}

const char* recon_last_error(void) { return g_last_error.c_str(); }

size_t recon_inverse_bytes(const recon_plan* p) {
  if (!p) return 0;
  return (size_t)p->pk.col_elems * p->esize * (size_t)p->Nx * p->Nt;
}

recon_status recon_plan_set_mu(recon_plan* p, float mu, void* stream) {
  g_last_error.clear();
  if (!p) return fail(RECON_ERR_INVALID_ARG, "NULL plan");
  if (!(mu > 0.f) || !std::isfinite(mu)) return fail(RECON_ERR_INVALID_ARG, "mu must be > 0");
  cudaSetDevice(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float old = p->mu;
  p->mu = mu;
  ++p->generation;   // batches and gradient engines built on the old mu refuse to run
  recon_status st = plan_invert(p, s);
  if (st == RECON_OK) {
    // every descriptor that carries mu (thresholds, r = b + mu p, J weights)
    Engine* e = new Engine();
    st = engine_build(e, &p, 1);
    if (st == RECON_OK && p->tile_px > 0 && p->opts.max_iters > 0) st = engine_set_tile(e, p->tile_px);
    if (st == RECON_OK) {
      delete p->eng;
      p->eng = e;
      Engine* ei = new Engine();
      st = engine_build_inverse(ei, p);
      if (st == RECON_OK) {
        delete p->eng_inv;
        p->eng_inv = ei;
      } else {
        delete ei;
      }
    } else {
      delete e;
    }
  }
  if (st != RECON_OK) {   // the inverses may be half-written: the plan stays unusable
    p->mu = old;
    p->broken = true;
  }
  return st;
}

recon_status recon_destroy(recon_plan* p) {
  if (!p) return RECON_OK;
  cudaSetDevice(p->device);
  if (p->last_stream) cudaStreamSynchronize(p->last_stream);
  delete p;
  return RECON_OK;
}

}  // extern "C"

namespace {

// A_{i,t} = (mu I + G_{i,t})^{-1} for every column of the plan, from its
// device-resident sensitivities and row lists (Section IV-C), rounded once
// into the packed stream.
recon_status plan_invert(recon_plan* p, cudaStream_t s) {
  const int Nx = p->Nx, Ny = p->Ny, Nt = p->Nt, Nc = p->Nc;
  const size_t ncols = (size_t)Nx * Nt;
  std::vector<double2> w64(Ny);
  for (int k = 0; k < Ny; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)Ny;
    w64[k] = make_double2(std::cos(a), std::sin(a));
  }
  void *d_w64 = nullptr, *d_circ = nullptr, *d_scr = nullptr;
  // one CTA per SM (the sweep holds ~200 KB of shared memory): the scratch
  // triangles of all CTAs then stay in L2 up to Ny = 256
  const int grid = std::max(1, std::min<int>((int)ncols, p->num_sms));
  cudaError_t e = cudaMalloc(&d_w64, Ny * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&d_circ, (size_t)Nt * Ny * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&d_scr, (size_t)grid * Ny * Ny * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemcpy(d_w64, w64.data(), Ny * sizeof(double2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->flags, 0, FLAG_COUNT * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->A, 0, (size_t)p->pk.col_elems * p->esize * ncols, s);
  if (e == cudaSuccess)
    e = launch_circulant(p->rows, p->rowoff, static_cast<double2*>(d_w64), static_cast<double2*>(d_circ), Ny, Nt, s);
  if (e == cudaSuccess)
    e = launch_plan_inverse(p->sens, static_cast<double2*>(d_circ), (double)p->mu, Nx, Ny, Nt, Nc, p->A, p->storage,
                            p->pk, static_cast<double2*>(d_scr), grid, p->flags, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_w64); cudaFree(d_circ); cudaFree(d_scr);
  if (e != cudaSuccess) return cuda_fail(e, "plan inverse");
  int fl[FLAG_COUNT];
  RC(cudaMemcpy(fl, p->flags, sizeof(fl), cudaMemcpyDeviceToHost));
  if (fl[FLAG_ERR] & DEV_ERR_NOT_PD) return fail(RECON_ERR_NONFINITE, "a Gram block is not positive definite");
  return RECON_OK;
}

PackInfo make_pack(int Ny) {
  PackInfo pk{};
  pk.nb = (Ny + 31) / 32;
  pk.ntiles = pk.nb * (pk.nb - 1) / 2;
  pk.nunits = pk.ntiles + pk.nb;
  pk.col_elems = (long long)pk.ntiles * kTileElems + (long long)pk.nb * kDiagElems;
  return pk;
}

// Pivots of the tridiagonal (rho I + D_t'D_t) for the Thomas sweep: with
// sub/super-diagonal -1, inv_t = 1 / (b_t - inv_{t-1}), b_t = rho + deg_t.
std::vector<float> thomas_pivots(int Nt, double rho) {
  std::vector<float> out(Nt);
  double prev = 0.0;
  for (int t = 0; t < Nt; ++t) {
    const double deg = (Nt == 1) ? 0.0 : ((t == 0 || t == Nt - 1) ? 1.0 : 2.0);
    const double den = rho + deg - (t > 0 ? prev : 0.0);
    prev = 1.0 / den;
    out[t] = (float)prev;
  }
  return out;
}

int coil_group_for(int Nc, int Ny) {
  int g = 8;
  while (g > 1 && 2 * (size_t)g * Ny * 8 > 48 * 1024) --g;
  return std::min(g, Nc);
}

}  // namespace

namespace recon {
int objective_coils_max(int Nc, int Ny) { return coil_group_for(Nc, Ny); }
}  // namespace recon

namespace recon {

// ||y - H x||^2 of a field by explicit FFTs (J(0), and every J(k) in the
// exact objective mode or with 16-bit inverses, where (mu I + H'H) x = r
// holds only to the storage precision).
recon_status plan_objective(recon_plan* p, const float2* x, double* acc, cudaStream_t s) {
  if (p->tc_nitems > 0 && (x == p->x || x == p->b)) {   // on the tensor cores (objective_tc.cu)
    ObjTcParams q = p->tc_par[x == p->x ? 0 : 1];
    q.fid_acc = acc;
    RC(launch_objective_tc(q, s));
    return RECON_OK;
  }
  ObjParams o{};
  o.Nx = p->Nx; o.Ny = p->Ny; o.Nt = p->Nt; o.Nc = p->Nc;
  o.ncg = p->obj_coils > 0 ? std::min(p->obj_coils, coil_group_for(p->Nc, p->Ny)) : coil_group_for(p->Nc, p->Ny);
  o.x = x; o.sens = p->sens; o.rows = p->rows; o.rowoff = p->rowoff; o.rowidx = p->rowidx; o.fy = p->fy;
  o.grid = 8 * p->num_sms;
  o.yhat = p->storage ? p->yhat_lp : static_cast<const void*>(p->yhat);
  o.ystorage = p->storage;
  o.yscale = p->yscale;
  o.fid_acc = acc; o.flags = p->flags;
  RC(launch_objective(o, s));
  return RECON_OK;
}

// user layout [Nt][Ny][Nx_full] (the plan's columns i0 .. i0+Nx-1) -> internal [Nt][Nx][Ny]
recon_status plan_to_internal(recon_plan* p, const float2* in, float2* out, cudaStream_t s) {
  const long long uframe = (long long)p->Ny * p->Nx_full;
  RC(launch_transpose(in + p->i0, out, p->Nt, p->Ny, p->Nx, uframe, (long long)p->npix(), p->Ny, s, p->Nx_full));
  return RECON_OK;
}
recon_status plan_to_user(recon_plan* p, const float2* in, float2* out, cudaStream_t s) {
  const long long uframe = (long long)p->Ny * p->Nx_full;
  RC(launch_transpose(in, out + p->i0, p->Nt, p->Nx, p->Ny, (long long)p->npix(), uframe, p->Nx_full, s));
  return RECON_OK;
}

// H'y in double-float arithmetic (rounded once to FP32), the FP32 hybrid data for J(k) and
// ||y||^2 (into *yy, which must be zeroed first).
recon_status plan_adjoint_df(recon_plan* p, const void* kspace, int kstorage, const float* kscale,
                             float2* yhat32, float2* b, double* yy, cudaStream_t s) {
  RC(launch_hybrid_rows_df(kspace, kstorage, kscale, p->yhat_df, yhat32, yy, p->rows, p->rowoff, p->maxm,
                           p->Nx_full, p->Ny, p->Nt, p->Nc, p->fxdf, p->rows_per_block, s, p->i0, p->Nx));
  RC(launch_adjoint_combine_df(p->yhat_df, p->sens, b, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc, p->fydf,
                               p->combine_coils, s));
  return RECON_OK;
}

// FP32 storage: the double-float prologue above (the 1e-5 bar needs it).  16-bit
// storage: FP32 butterflies and accumulation, the hybrid data kept in 16 bits
// with per-frame power-of-two scales (its FP32 values pass through tmp_b).
recon_status plan_prologue(recon_plan* p, const void* kspace, int kstorage, const float* kscale, cudaStream_t s) {
  RC(cudaMemsetAsync(p->yy, 0, sizeof(double), s));
  if (p->storage == 0) return plan_adjoint_df(p, kspace, kstorage, kscale, p->yhat, p->b, p->yy, s);
  RC(cudaMemsetAsync(p->ymax, 0, (size_t)p->Nt * sizeof(unsigned), s));
  RC(launch_hybrid_rows(kspace, kstorage, kscale, p->tmp_b, p->yy, p->ymax, p->rows, p->rowoff, p->maxm, p->Nx_full,
                        p->Ny, p->Nt, p->Nc, p->fx, p->rows_per_block, s, p->i0, p->Nx));
  RC(launch_adjoint_combine(p->tmp_b, p->sens, p->b, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc, p->fy,
                            p->storage, p->yhat_lp, p->ymax, p->yscale, p->combine_coils, s));
  return RECON_OK;
}

recon_status plan_fill_info(recon_plan* p, recon_info* info, cudaStream_t s) {
  RC(cudaStreamSynchronize(s));
  int fl[FLAG_COUNT];
  RC(cudaMemcpy(fl, p->flags, sizeof(fl), cudaMemcpyDeviceToHost));
  const int K = p->opts.max_iters;
  const int iters = fl[FLAG_STOP] ? fl[FLAG_ITERS] : K;
  p->last_iters = iters;
  std::vector<double> J((size_t)K + 2);
  RC(cudaMemcpy(J.data(), p->trace_J, J.size() * sizeof(double), cudaMemcpyDeviceToHost));
  if (info) {
    info->iters = iters;
    info->stopped = fl[FLAG_STOP] ? 1 : 0;
    info->J = J[iters];
    info->J0 = J[0];
    info->delta = (iters >= 1) ? (J[iters - 1] - J[iters]) / J[iters] : NAN;
    // ADMM residuals (a solve that ran all K iterations)
    info->primal_res = info->dual_res = NAN;
    if (K >= 1 && !fl[FLAG_STOP]) {
      double a[4];
      RC(cudaMemcpy(a, p->res_acc, sizeof(a), cudaMemcpyDeviceToHost));
      if (p->prior == RECON_PRIOR_TV || p->prior == RECON_PRIOR_STV) {   // Algorithm 2
        const double mu2 = p->mu, mu1 = p->mu / p->opts.rho;
        info->primal_res = std::sqrt(a[0] + a[1]);
        info->dual_res = std::sqrt(mu1 * mu1 * a[3] + mu2 * mu2 * a[2]);
      } else {   // Algorithm 1 (DFT, Haar frame)
        info->primal_res = std::sqrt(a[0]);
        info->dual_res = (double)p->mu * std::sqrt(std::max(0.0, a[1]));
      }
    }
  }
  if (fl[FLAG_ERR] & DEV_ERR_TIMEOUT) return fail(RECON_ERR_TIMEOUT, "a bounded device-side wait timed out");
  if (fl[FLAG_ERR] & DEV_ERR_NONFINITE) return fail(RECON_ERR_NONFINITE, "non-finite objective value");
  return RECON_OK;
}

}  // namespace recon

namespace {

bool valid_ptr(const void* p) { return p != nullptr; }

// A plan over columns i0 .. i0+W-1 of an Nxf-wide problem (W = Nxf, i0 = 0
// for a whole plan).  Inside, Nx is the plan's own width W; the k-space rows
// (and the row FFTs of the prologue), the mask and the sensitivities the
// caller passes are Nxf wide.
recon_status plan_create_impl(recon_plan** out, int Nxf, int Ny, int Nt, int Nc, const uint8_t* mask,
                              const float* sens, float lambda, float mu, recon_prior prior, const recon_opts* opts,
                              int i0, int W, void* stream) {
  g_last_error.clear();
  if (!out) return fail(RECON_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const int Nx = W;
  if (Nxf < 1 || Ny < 1 || Nt < 1 || Nc < 1) return fail(RECON_ERR_INVALID_ARG, "dimensions must be >= 1");
  if (W < 1 || i0 < 0 || i0 + W > Nxf) return fail(RECON_ERR_INVALID_ARG, "slab outside the image");
  if (Ny > 1024 || Nxf > 1024 || Nt > 128 || Nc > 64 || (size_t)(Nc + 1) * Ny * 16 > 200 * 1024)
    return fail(RECON_ERR_UNSUPPORTED,
                "size beyond supported limits (Nx, Ny <= 1024, Nt <= 128, Nc <= 64, (Nc+1)*Ny <= 12800)");
  if (!valid_ptr(mask) || !valid_ptr(sens)) return fail(RECON_ERR_INVALID_ARG, "mask or sens is NULL");
  if (!(mu > 0.f) || !std::isfinite(mu)) return fail(RECON_ERR_INVALID_ARG, "mu must be > 0");
  if (!(lambda >= 0.f) || !std::isfinite(lambda)) return fail(RECON_ERR_INVALID_ARG, "lambda must be >= 0");
  if (prior != RECON_PRIOR_TV && prior != RECON_PRIOR_DFT && prior != RECON_PRIOR_HAAR && prior != RECON_PRIOR_STV)
    return fail(RECON_ERR_INVALID_ARG, "unknown prior");
  if (prior == RECON_PRIOR_STV && (i0 != 0 || W != Nxf))
    return fail(RECON_ERR_UNSUPPORTED, "the spatio-temporal prior couples columns: no slab plans");
  recon_opts o;
  recon_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rho > 0.f) || o.max_iters < 0 || !(o.tol >= 0.0) || o.storage < 0 || o.storage > 2 || o.col_stages < 0 ||
      o.persistent < 0 || o.persistent > 1 || o.overlap < 0 || o.overlap > 1 ||
      o.objective < 0 || o.objective > 2 || (prior == RECON_PRIOR_HAAR && (o.frame_levels < 1 || o.frame_levels > 6)) ||
      (prior == RECON_PRIOR_STV && (!(o.spatial_weight >= 0.f) || !std::isfinite(o.spatial_weight) ||
                                    o.cg_steps < 1 || o.cg_steps > 64)))
    return fail(RECON_ERR_INVALID_ARG, "invalid options");
  {
    // the column-inverse kernel keeps a column's vectors and its consumers'
    // partial sums in shared memory: Ny up to 768 with FP32 storage, 640 with
    // 16-bit (checked here, before any allocation, for the plan's own shape)
    int dev = 0, optin = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int es = o.storage == 0 ? 8 : 4;
    const int q = col_inverse_stage_quantum(es);
    const int work_est = (int)(((long long)Nx * Nt + std::max(sms, 1) - 1) / std::max(sms, 1)) + 2;
    auto fits = [&](int nb) { return col_inverse_smem(q, nb, 1, work_est, es) <= (size_t)optin; };
    const int nb = (Ny + 31) / 32;
    if (optin > 0 && !fits(nb)) {
      int nb_max = nb;
      while (nb_max > 1 && !fits(nb_max)) --nb_max;
      return fail(RECON_ERR_UNSUPPORTED, "Ny = " + std::to_string(Ny) +
                                             " does not fit the column-inverse kernel's shared memory; this storage "
                                             "supports Ny <= " + std::to_string(32 * nb_max));
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // mask -> sampled row lists (host)
  const size_t mcount = o.mask_full ? (size_t)Nt * Ny * Nxf : (size_t)Nt * Ny;
  std::vector<uint8_t> hm(mcount);
  {
    cudaError_t e = cudaMemcpy(hm.data(), mask, mcount, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "copy mask");
  }
  auto* p = new recon_plan();
  p->Nx = Nx; p->Ny = Ny; p->Nt = Nt; p->Nc = Nc;
  p->Nx_full = Nxf; p->i0 = i0;
  p->prior = prior; p->lam = lambda; p->mu = mu; p->opts = o;
  p->storage = o.storage;
  p->esize = (o.storage == 0) ? 8 : 4;
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  {
    int bad_t = 0, bad_j = 0;
    const int maxm = mask_rows(hm.data(), Nt, Ny, Nxf, o.mask_full != 0, p->h_rows, p->h_rowoff, &bad_t, &bad_j);
    if (maxm < 0) {
      delete p;
      return fail(RECON_ERR_MASK_NOT_CARTESIAN, "mask differs along kx (row " + std::to_string(bad_j) +
                                                    ", frame " + std::to_string(bad_t) + ")");
    }
    if (maxm == 0) {   // no data at all: nothing to reconstruct from (and no row to launch over)
      delete p;
      return fail(RECON_ERR_INVALID_ARG, "the mask samples no k-space row");
    }
    p->maxm = maxm;
  }
  p->total_rows = (int)p->h_rows.size();
  p->pk = make_pack(Ny);

  auto cleanup = [&](recon_status st) {
    delete p;
    return st;
  };
#define PC(call)                                                      \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, #call));      \
  } while (0)

  const size_t nimg = p->nimg();
  const size_t ncols = (size_t)Nx * Nt;
  PC(p->alloc(&p->A, (size_t)p->pk.col_elems * p->esize * ncols));
  PC(p->alloc((void**)&p->sens, (size_t)Nx * Nc * Ny * sizeof(float2)));
  PC(p->alloc((void**)&p->rows, std::max<size_t>(1, p->h_rows.size()) * sizeof(int)));
  PC(p->alloc((void**)&p->rowoff, (Nt + 1) * sizeof(int)));
  PC(p->alloc((void**)&p->rowidx, (size_t)Nt * Ny * sizeof(short)));
  PC(p->alloc((void**)&p->tw_x, Nxf * sizeof(float2)));
  PC(p->alloc((void**)&p->tw_y, Ny * sizeof(float2)));
  PC(p->alloc((void**)&p->tw_t, Nt * sizeof(float2)));
  PC(p->alloc((void**)&p->twdf_x, Nxf * sizeof(dc)));
  PC(p->alloc((void**)&p->twdf_y, Ny * sizeof(dc)));
  PC(p->alloc((void**)&p->yhat_df, std::max<size_t>(1, (size_t)p->total_rows * Nx * Nc) * sizeof(dc)));
  PC(p->alloc((void**)&p->thomas, Nt * sizeof(float)));
  const size_t nyhat = std::max<size_t>(1, (size_t)p->total_rows * Nx * Nc);
  if (o.storage == RECON_STORAGE_FP32) {
    PC(p->alloc((void**)&p->yhat, nyhat * sizeof(float2)));
  } else {  // 16-bit hybrid data with per-frame scales
    PC(p->alloc(&p->yhat_lp, nyhat * 4));
    PC(p->alloc((void**)&p->ymax, Nt * sizeof(unsigned)));
    PC(p->alloc((void**)&p->yscale, Nt * sizeof(float)));
  }
  PC(p->alloc((void**)&p->b, nimg * sizeof(float2)));
  // TV: m, d1, p;  DFT: u = v + d;  Haar: u ((L+1) channels) and s = Psi'u;
  // STV: m and q (s0), e = d1 - v with four components (s1[0]; z in a
  // volume), p and the CG residual (s2), the CG directions (r, cgd)
  const size_t nu = (prior == RECON_PRIOR_HAAR) ? (size_t)(o.frame_levels + 1) * nimg : nimg;
  for (int k = 0; k < 2; ++k) {
    PC(p->alloc((void**)&p->s0[k], nu * sizeof(float2)));
    if (prior == RECON_PRIOR_TV) {
      PC(p->alloc((void**)&p->s1[k], nimg * sizeof(float2)));
      PC(p->alloc((void**)&p->s2[k], nimg * sizeof(float2)));
    }
    if (prior == RECON_PRIOR_HAAR) PC(p->alloc((void**)&p->s1[k], nimg * sizeof(float2)));
    if (prior == RECON_PRIOR_STV) {
      if (k == 0) PC(p->alloc((void**)&p->s1[k], 4 * nimg * sizeof(float2)));   // t, x, y, z
      PC(p->alloc((void**)&p->s2[k], nimg * sizeof(float2)));
    }
  }
  if (prior == RECON_PRIOR_STV) PC(p->alloc((void**)&p->cgd, nimg * sizeof(float2)));
  if (prior == RECON_PRIOR_DFT || prior == RECON_PRIOR_HAAR || prior == RECON_PRIOR_STV)   // for the residuals
    PC(p->alloc((void**)&p->res_prev, nimg * sizeof(float2)));
  if (prior == RECON_PRIOR_STV) PC(p->alloc((void**)&p->res_d1, 4 * nimg * sizeof(float2)));
  PC(p->alloc((void**)&p->x, nimg * sizeof(float2)));
  if (prior != RECON_PRIOR_TV) PC(p->alloc((void**)&p->r, nimg * sizeof(float2)));
  PC(p->alloc((void**)&p->tmp_a, nimg * sizeof(float2)));
  PC(p->alloc((void**)&p->tmp_b, std::max<size_t>(nimg, (size_t)p->total_rows * Nx * Nc) * sizeof(float2)));
  const size_t nt = (size_t)o.max_iters + 2;
  PC(p->alloc((void**)&p->trace_fid, nt * sizeof(double)));
  PC(p->alloc((void**)&p->trace_prior, nt * sizeof(double)));
  PC(p->alloc((void**)&p->trace_J, nt * sizeof(double)));
  PC(p->alloc((void**)&p->flags, FLAG_COUNT * sizeof(int)));
  PC(p->alloc((void**)&p->yy, sizeof(double)));
  PC(p->alloc((void**)&p->res_acc, 4 * sizeof(double)));

  // tables
  std::vector<float2> tw(std::max(std::max(Nxf, Ny), Nt));
  fill_twiddles_host(Nxf, tw.data());
  PC(cudaMemcpy(p->tw_x, tw.data(), Nxf * sizeof(float2), cudaMemcpyHostToDevice));
  fill_twiddles_host(Ny, tw.data());
  PC(cudaMemcpy(p->tw_y, tw.data(), Ny * sizeof(float2), cudaMemcpyHostToDevice));
  fill_twiddles_host(Nt, tw.data());
  PC(cudaMemcpy(p->tw_t, tw.data(), Nt * sizeof(float2), cudaMemcpyHostToDevice));
  {
    std::vector<float4> twd(std::max(Nxf, Ny));
    fill_twiddles_host_df(Nxf, twd.data());
    PC(cudaMemcpy(p->twdf_x, twd.data(), Nxf * sizeof(float4), cudaMemcpyHostToDevice));
    fill_twiddles_host_df(Ny, twd.data());
    PC(cudaMemcpy(p->twdf_y, twd.data(), Ny * sizeof(float4), cudaMemcpyHostToDevice));
    p->fxdf = make_fft_plan_host_df(Nxf, p->twdf_x);
    p->fydf = make_fft_plan_host_df(Ny, p->twdf_y);
  }
  p->fx = make_fft_plan_host(Nxf, p->tw_x);
  p->fy = make_fft_plan_host(Ny, p->tw_y);
  p->ft = make_fft_plan_host(Nt, p->tw_t);
  std::vector<float> th = thomas_pivots(Nt, o.rho);
  PC(cudaMemcpy(p->thomas, th.data(), Nt * sizeof(float), cudaMemcpyHostToDevice));
  if (!p->h_rows.empty())
    PC(cudaMemcpy(p->rows, p->h_rows.data(), p->h_rows.size() * sizeof(int), cudaMemcpyHostToDevice));
  PC(cudaMemcpy(p->rowoff, p->h_rowoff.data(), (Nt + 1) * sizeof(int), cudaMemcpyHostToDevice));
  {
    std::vector<short> ri((size_t)Nt * Ny, (short)-1);
    for (int t = 0; t < Nt; ++t)
      for (int m = p->h_rowoff[t]; m < p->h_rowoff[t + 1]; ++m) ri[(size_t)t * Ny + p->h_rows[m]] = (short)(m - p->h_rowoff[t]);
    PC(cudaMemcpy(p->rowidx, ri.data(), ri.size() * sizeof(short), cudaMemcpyHostToDevice));
  }

  // sensitivities -> [Nx][Nc][Ny]
  {
    float2* stage = p->tmp_a;  // Nc*Ny*Nx <= nimg is not guaranteed; use a temporary
    void* tmp = nullptr;
    const size_t sbytes = (size_t)Nc * Ny * Nx * sizeof(float2);
    PC(cudaMalloc(&tmp, sbytes));
    stage = static_cast<float2*>(tmp);
    // the plan's columns i0 .. i0+Nx-1 of the caller's [Nc][Ny][Nxf] array
    cudaError_t e = cudaMemcpy2DAsync(stage, (size_t)Nx * sizeof(float2), sens + 2 * (size_t)i0,
                                      (size_t)Nxf * sizeof(float2), (size_t)Nx * sizeof(float2), (size_t)Nc * Ny,
                                      cudaMemcpyDefault, s);
    if (e == cudaSuccess)
      e = launch_transpose(stage, p->sens, Nc, Ny, Nx, (long long)Ny * Nx, (long long)Ny, (long long)Nc * Ny, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "sensitivity upload"));
  }

  // the explicit objective (16-bit storage, or objective = 2) on the tensor
  // cores: the sampled rows of every (frame, row tile), the DFT twiddles as
  // FP16 pairs, the work items, and the sensitivities' column maxima.  Even Ny only (the
  // kernel reads s and x two values at a time); odd Ny keeps the FFT kernels.
  if ((o.storage != 0 || o.objective == 2) && Ny % 2 == 0) {
    const int tiles_c = (Nx * Nc + 255) / 256;
    std::vector<int> tile0(Nt + 1, 0);
    for (int t = 0; t < Nt; ++t) {
      const int mt = p->h_rowoff[t + 1] - p->h_rowoff[t];
      tile0[t + 1] = tile0[t] + (mt + 63) / 64;
    }
    std::vector<int> hrows((size_t)std::max(tile0[Nt], 1) * 64, -1);   // sampled rows of each row tile
    std::vector<int4> items;
    for (int t = 0; t < Nt; ++t) {
      const int r0 = p->h_rowoff[t], mt = p->h_rowoff[t + 1] - r0;
      for (int rt = 0; rt * 64 < mt; ++rt) {
        for (int m = 0; m < std::min(64, mt - 64 * rt); ++m)
          hrows[(size_t)(tile0[t] + rt) * 64 + m] = p->h_rows[r0 + 64 * rt + m];
        for (int ct = 0; ct < tiles_c; ++ct) items.push_back(make_int4(t, rt, ct, tile0[t] + rt));
      }
    }
    std::vector<uint2> htw((size_t)Ny);
    objective_tc_twiddle(Ny, htw.data());
    PC(p->alloc((void**)&p->tc_rows, hrows.size() * sizeof(int)));
    PC(cudaMemcpy(p->tc_rows, hrows.data(), hrows.size() * sizeof(int), cudaMemcpyHostToDevice));
    PC(p->alloc((void**)&p->tc_twiddle, htw.size() * sizeof(uint2)));
    PC(cudaMemcpy(p->tc_twiddle, htw.data(), htw.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    PC(p->alloc((void**)&p->tc_items, std::max<size_t>(1, items.size()) * sizeof(int4)));
    if (!items.empty())
      PC(cudaMemcpy(p->tc_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    PC(p->alloc((void**)&p->tc_smax, (size_t)Nx * Nc * sizeof(float)));
    PC(p->alloc((void**)&p->tc_xmax, (size_t)Nt * Nx * sizeof(float)));
    PC(launch_col_absmax(p->sens, Nx * Nc, Ny, p->tc_smax, s));
    ObjTcParams q{};
    q.Nx = Nx; q.Ny = Ny; q.Nt = Nt; q.Nc = Nc;
    q.smax = p->tc_smax; q.xmax = p->tc_xmax;
    q.yhat = o.storage ? p->yhat_lp : static_cast<const void*>(p->yhat);
    q.ystorage = o.storage;
    q.yscale = p->yscale;
    q.rowoff = p->rowoff;
    q.tile_rows = p->tc_rows; q.twiddle = p->tc_twiddle;
    q.items = p->tc_items; q.nitems = (int)items.size();
    q.grid = std::max(1, p->num_sms);
    q.flags = p->flags; q.err = p->flags;
    p->tc_par.assign(2, q);
    // the tiles do not fit or the driver has no tensor maps: the FFT kernels stay
    if (objective_tc_prepare(p->tc_par[0], p->x, p->sens) && objective_tc_prepare(p->tc_par[1], p->b, p->sens))
      p->tc_nitems = (int)items.size();
    PC(cudaStreamSynchronize(s));
  }

  // packed inverses (double-float inversion, rounded once)
  {
    recon_status st = plan_invert(p, s);
    if (st != RECON_OK) return cleanup(st);
  }

  // the plan's own iterations (a batch of one) and the apply-inverse launch
  {
    p->eng = new Engine();
    recon_status st = engine_build(p->eng, &p, 1);
    if (st != RECON_OK) return cleanup(st);
    p->eng_inv = new Engine();
    st = engine_build_inverse(p->eng_inv, p);
    if (st != RECON_OK) return cleanup(st);
    p->col_stages = p->eng->stages;
  }
  if (o.profile) PC(plan_create_events(p));
  p->last_stream = s;
  *out = p;
  return RECON_OK;
#undef PC
}

}  // namespace

extern "C" {

recon_status recon_plan_create(recon_plan** out, int Nx, int Ny, int Nt, int Nc, const uint8_t* mask,
                               const float* sens, float lambda, float mu, recon_prior prior, const recon_opts* opts,
                               void* stream) {
  return plan_create_impl(out, Nx, Ny, Nt, Nc, mask, sens, lambda, mu, prior, opts, 0, Nx, stream);
}

recon_status recon_plan_create_slab(recon_plan** out, int Nx, int Ny, int Nt, int Nc, const uint8_t* mask,
                                    const float* sens, float lambda, float mu, recon_prior prior,
                                    const recon_opts* opts, int i0, int width, void* stream) {
  return plan_create_impl(out, Nx, Ny, Nt, Nc, mask, sens, lambda, mu, prior, opts, i0, width, stream);
}

recon_status recon_solve_slabs(int Nx, int Ny, int Nt, int Nc, const uint8_t* mask, const float* sens, float lambda,
                               float mu, recon_prior prior, const recon_opts* opts, int width, const float* kspace,
                               float* image, double* J_trace, recon_info* info, void* stream) {
  if (width < 1 || !kspace || !image) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  recon_opts o;
  recon_default_opts(&o);
  if (opts) o = *opts;
  const int K = std::max(o.max_iters, 0);
  std::vector<double> acc((size_t)K + 1, 0.0), tr((size_t)K + 1);
  recon_info tot{};
  tot.J = tot.J0 = 0.0;
  for (int i0 = 0; i0 < Nx; i0 += width) {
    const int W = std::min(width, Nx - i0);
    recon_plan* p = nullptr;
    recon_status st = plan_create_impl(&p, Nx, Ny, Nt, Nc, mask, sens, lambda, mu, prior, &o, i0, W, stream);
    if (st != RECON_OK) return st;
    recon_info si{};
    st = recon_solve(p, kspace, image, &si, stream);
    if (st == RECON_OK && J_trace) st = recon_get_trace(p, tr.data(), K + 1);
    recon_destroy(p);
    if (st != RECON_OK) return st;
    for (int k = 0; k <= K; ++k) acc[k] += tr[k];
    tot.iters = std::max(tot.iters, si.iters);
    tot.stopped |= si.stopped;
    tot.J += si.J;
    tot.J0 += si.J0;
  }
  if (J_trace)
    for (int k = 0; k <= K; ++k) J_trace[k] = acc[k];
  tot.delta = (J_trace && K >= 1) ? (acc[K - 1] - acc[K]) / acc[K] : NAN;
  if (info) *info = tot;
  return RECON_OK;
}

recon_status recon_solve_kspace(recon_plan* p, const recon_kspace* y, float* image, recon_info* info, void* stream) {
  g_last_error.clear();
  if (!p || !y || !y->data || !image) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  if (p->broken) return fail(RECON_ERR_INVALID_ARG, "the plan failed recon_plan_set_mu and is unusable");
  if (y->storage < RECON_STORAGE_FP32 || y->storage > RECON_STORAGE_BF16)
    return fail(RECON_ERR_INVALID_ARG, "k-space storage must be a recon_storage value");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->last_stream = s;
  p->n_col = p->n_tmp = 0;
  p->prof_valid = p->opts.profile != 0;
  if (p->opts.profile) cudaEventRecord(p->ev_solve[0], s);
  recon_status st = plan_prologue(p, y->data, y->storage, y->frame_scale, s);
  if (st != RECON_OK) return st;
  st = engine_iterate(p->eng, s, p->opts.profile != 0);
  if (st != RECON_OK) return st;
  st = plan_to_user(p, plan_result(p), reinterpret_cast<float2*>(image), s);
  if (st != RECON_OK) return st;
  if (p->opts.profile) cudaEventRecord(p->ev_solve[1], s);
  if (info) return plan_fill_info(p, info, s);
  return RECON_OK;
}

recon_status recon_solve(recon_plan* p, const float* kspace, float* image, recon_info* info, void* stream) {
  const recon_kspace y{kspace, RECON_STORAGE_FP32, nullptr};
  return recon_solve_kspace(p, &y, image, info, stream);
}

recon_status recon_quantize_kspace(int Nx, int Ny, int Nt, int Nc, const float* kspace, int storage, void* out,
                                   float* frame_scale, void* stream) {
  g_last_error.clear();
  if (Nx < 1 || Ny < 1 || Nt < 1 || Nc < 1 || !kspace || !out || !frame_scale)
    return fail(RECON_ERR_INVALID_ARG, "bad argument");
  if (storage != RECON_STORAGE_FP16 && storage != RECON_STORAGE_BF16)
    return fail(RECON_ERR_INVALID_ARG, "storage must be RECON_STORAGE_FP16 or RECON_STORAGE_BF16");
  RC(launch_quantize_kspace(reinterpret_cast<const float2*>(kspace), (long long)Nc * Ny * Nx, Nt, storage, out,
                            frame_scale, static_cast<cudaStream_t>(stream)));
  return RECON_OK;
}

recon_status recon_plan_set_profile(recon_plan* p, int on) {
  g_last_error.clear();
  if (!p || (on != 0 && on != 1)) return fail(RECON_ERR_INVALID_ARG, "plan must be non-NULL and on 0 or 1");
  if (on) {
    cudaSetDevice(p->device);
    RC(plan_create_events(p));
  }
  p->opts.profile = on;
  return RECON_OK;
}

recon_status recon_get_profile(recon_plan* p, recon_profile* out) {
  if (!p || !out) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (!p->prof_valid) return RECON_OK;
  if (p->last_stream) RC(cudaStreamSynchronize(p->last_stream));
  else RC(cudaDeviceSynchronize());
  auto sum = [&](std::vector<cudaEvent_t>& v, int n, double* ms) -> cudaError_t {
    double acc = 0.0;
    for (int k = 0; k < n && 2 * (size_t)k + 1 < v.size(); ++k) {
      float m = 0.f;
      cudaError_t e = cudaEventElapsedTime(&m, v[2 * k], v[2 * k + 1]);
      if (e != cudaSuccess) return e;
      acc += m;
    }
    *ms = acc;
    return cudaSuccess;
  };
  RC(sum(p->ev_col, p->n_col, &out->inverse_ms));
  out->inverse_launches = p->n_col;
  out->inverse_passes = p->eng && p->eng->persist ? p->n_col * p->eng->K : p->n_col;
  out->persistent = p->eng && p->eng->persist ? 1 : 0;
  RC(sum(p->ev_tmp, p->n_tmp, &out->temporal_ms));
  out->temporal_launches = p->n_tmp;
  float m = 0.f;
  RC(cudaEventElapsedTime(&m, p->ev_solve[0], p->ev_solve[1]));
  out->solve_ms = m;
  return RECON_OK;
}

unsigned long long recon_kernel_launches(void) { return g_launches.load(); }

recon_status recon_solve_host(recon_plan* p, const float* kspace_host, float* image_host, recon_info* info,
                              void* stream) {
  g_last_error.clear();
  if (!p || !kspace_host || !image_host) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  if (p->broken) return fail(RECON_ERR_INVALID_ARG, "the plan failed recon_plan_set_mu and is unusable");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t kbytes = (size_t)p->Nt * p->Nc * p->Ny * p->Nx_full * sizeof(float2);
  const size_t ibytes = (size_t)p->Nt * p->Ny * p->Nx_full * sizeof(float2);
  if (!p->istage) RC(p->alloc((void**)&p->istage, ibytes));
  // Page-locked host memory is mapped into the device's address space: the
  // prologue then reads only the sampled k-space rows (1/R of the array)
  // straight from it, instead of a copy of the whole array first.  Pageable
  // memory is copied to a device staging buffer.
  const void* kdev = nullptr;
  {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, kspace_host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
      kdev = at.devicePointer;
    else
      (void)cudaGetLastError();
  }
  if (!kdev) {
    if (!p->kstage) RC(p->alloc((void**)&p->kstage, kbytes));
    RC(cudaMemcpyAsync(p->kstage, kspace_host, kbytes, cudaMemcpyHostToDevice, s));
    kdev = p->kstage;
  }
  recon_status st = recon_solve(p, reinterpret_cast<const float*>(kdev), reinterpret_cast<float*>(p->istage),
                                nullptr, stream);
  if (st != RECON_OK) return st;
  if (p->Nx == p->Nx_full) {
    RC(cudaMemcpyAsync(image_host, p->istage, ibytes, cudaMemcpyDeviceToHost, s));
  } else {  // only the plan's columns of the caller's image
    const size_t pitch = (size_t)p->Nx_full * sizeof(float2);
    RC(cudaMemcpy2DAsync(reinterpret_cast<float2*>(image_host) + p->i0, pitch, p->istage + p->i0, pitch,
                         (size_t)p->Nx * sizeof(float2), (size_t)p->Nt * p->Ny, cudaMemcpyDeviceToHost, s));
  }
  return plan_fill_info(p, info, s);
}

recon_status recon_get_trace(recon_plan* p, double* J_host, int n) {
  if (!p || !J_host || n < 0) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  if (p->last_stream) RC(cudaStreamSynchronize(p->last_stream));
  const int avail = p->opts.max_iters + 2;
  std::vector<double> J(avail);
  RC(cudaMemcpy(J.data(), p->trace_J, avail * sizeof(double), cudaMemcpyDeviceToHost));
  for (int k = 0; k < n; ++k) J_host[k] = (k < avail) ? J[k] : NAN;
  return RECON_OK;
}

recon_status recon_apply_adjoint(recon_plan* p, const float* kspace, float* image, void* stream) {
  if (!p || !kspace || !image) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  if (p->Nx != p->Nx_full) return fail(RECON_ERR_UNSUPPORTED, "H' of a slab plan: use a whole plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status st = plan_adjoint_df(p, kspace, 0, nullptr, p->tmp_b, p->tmp_a, nullptr, s);
  if (st != RECON_OK) return st;
  return plan_to_user(p, p->tmp_a, reinterpret_cast<float2*>(image), s);
}

recon_status recon_apply_forward(recon_plan* p, const float* image, float* kspace, void* stream) {
  if (!p || !image || !kspace) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  if (p->Nx != p->Nx_full) return fail(RECON_ERR_UNSUPPORTED, "H of a slab plan: use a whole plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status st = plan_to_internal(p, reinterpret_cast<const float2*>(image), p->tmp_a, s);
  if (st != RECON_OK) return st;
  RC(launch_forward_cols(p->tmp_a, p->sens, p->tmp_b, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc, p->fy, s));
  RC(cudaMemsetAsync(kspace, 0, (size_t)p->Nt * p->Nc * p->Ny * p->Nx * sizeof(float2), s));
  RC(launch_forward_rows(p->tmp_b, reinterpret_cast<float2*>(kspace), p->rows, p->rowoff, p->maxm, p->Nx, p->Ny,
                         p->Nt, p->Nc, p->fx, s));
  return RECON_OK;
}

recon_status recon_apply_inverse(recon_plan* p, const float* in, float* out, void* stream) {
  if (!p || !in || !out || in == out) return fail(RECON_ERR_INVALID_ARG, "NULL or aliased argument");
  if (p->broken) return fail(RECON_ERR_INVALID_ARG, "the plan failed recon_plan_set_mu and is unusable");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status st = plan_to_internal(p, reinterpret_cast<const float2*>(in), p->tmp_a, s);
  if (st != RECON_OK) return st;
  RC(cudaMemsetAsync(p->flags, 0, FLAG_COUNT * sizeof(int), s));
  st = engine_apply_inverse(p->eng_inv, s);
  if (st != RECON_OK) return st;
  return plan_to_user(p, p->tmp_b, reinterpret_cast<float2*>(out), s);
}

recon_status recon_export_inverse(recon_plan* p, int i, int t, float* dense, void* stream) {
  if (!p || !dense || i < 0 || i >= p->Nx || t < 0 || t >= p->Nt) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  if (p->broken) return fail(RECON_ERR_INVALID_ARG, "the plan failed recon_plan_set_mu and is unusable");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RC(launch_unpack(p->A, p->storage, p->pk, (long long)i * p->Nt + t, p->Ny, reinterpret_cast<float2*>(dense), s));
  return RECON_OK;
}

}  // extern "C"
