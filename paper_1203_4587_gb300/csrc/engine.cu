// Launch engine: descriptor sets, work lists and the launch sequence of the
// ADMM iterations for one plan (a batch of one) or a batch of plans, and the
// batched C entry points (one launch per step for all slices, replayed from
// a captured CUDA graph).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "host_logic.h"
#include "plan.h"

namespace recon {

cudaError_t DevArena::alloc(void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) ptrs.push_back(*p);
  return e;
}

void DevArena::free(void* p) {
  auto it = std::find(ptrs.begin(), ptrs.end(), p);
  if (it != ptrs.end()) {
    cudaFree(p);
    ptrs.erase(it);
  }
}

void DevArena::release() {
  for (void* p : ptrs) cudaFree(p);
  ptrs.clear();
}

namespace {

template <typename T>
cudaError_t upload(DevArena& a, T** dst, const std::vector<T>& v) {
  cudaError_t e = a.alloc(reinterpret_cast<void**>(dst), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

// Column work lists of a batch: every column of every slice, by the bytes it
// streams (host_logic.h: lpt_work_lists), numbered image-column-major
// (c' = i Nt + t, the order of the packed stream) and stored as
// col = t Nx + i: a CTA's list runs through the image columns in order, and
// the CTAs of a launch read adjacent stretches of the stream.
void build_col_work(recon_plan* const* plans, int n, int grid, std::vector<unsigned>& work, std::vector<int>& off,
                    int& work_max) {
  std::vector<long long> cost(n);
  std::vector<int> ncols(n);
  for (int q = 0; q < n; ++q) {
    cost[q] = plans[q]->pk.col_elems * (long long)plans[q]->esize + 4096;
    ncols[q] = plans[q]->Nx * plans[q]->Nt;
  }
  lpt_work_lists(cost, ncols, grid, work, off, work_max);
  for (unsigned& w : work) {
    const int q = (int)(w >> 24), cp = (int)(w & 0xFFFFFFu);
    const int Nt = plans[q]->Nt, Nx = plans[q]->Nx;
    const int i = cp / Nt, t = cp - i * Nt;
    w = ((unsigned)q << 24) | (unsigned)(t * Nx + i);
  }
}

namespace {

TvSlice tv_desc(recon_plan* p, int k, int K) {
  TvSlice d{};
  d.Nt = p->Nt;
  d.npix = (long long)p->npix();
  d.tau1 = (float)(p->lam / (2.0 * (p->mu / p->opts.rho)));
  d.rho = p->opts.rho;
  d.thomas = p->thomas;
  d.stop = p->flags + FLAG_STOP;
  if (k <= K) {  // iteration k (1-based): state of k-1 -> state of k
    const int in = (k - 1) & 1, out = k & 1;
    d.m = (k == 1) ? p->b : p->s0[in];
    d.d1 = (k == 1) ? nullptr : p->s1[in];
    d.x = (k == 1) ? p->b : p->x;
    d.p = (k == 1) ? p->b : p->s2[in];
    d.m_out = p->s0[out];
    d.d1_out = p->s1[out];
    d.p_out = p->s2[out];
    d.write_state = 1;
    d.prior_acc = p->trace_prior + (k - 1);
  } else {       // final: only ||D_t x_K||_1
    d.x = (K == 0) ? p->b : p->x;
    d.write_state = 0;
    d.prior_acc = p->trace_prior + K;
  }
  return d;
}

DftSlice dft_desc(recon_plan* p, int k, int K) {
  DftSlice d{};
  d.Nt = p->Nt;
  d.npix = (long long)p->npix();
  d.b = p->b;
  d.tau = (float)(p->lam / (2.0 * p->mu));
  d.mu = p->mu;
  d.ft = p->ft;
  d.stop = p->flags + FLAG_STOP;
  if (k <= K) {
    const int in = (k - 1) & 1, out = k & 1;
    d.xh = (k == 1) ? p->b : p->x;
    d.u = (k == 1) ? nullptr : p->s0[in];
    d.first = (k == 1);
    d.u_out = p->s0[out];
    d.r_out = p->r;
    d.write_state = 1;
    d.prior_acc = p->trace_prior + (k - 1);
  } else {
    d.xh = (K == 0) ? p->b : p->x;
    d.first = 1;
    d.write_state = 0;
    d.prior_acc = p->trace_prior + K;
  }
  return d;
}

HaarSlice haar_desc(recon_plan* p, int k, int K) {
  HaarSlice d{};
  d.Nt = p->Nt;
  d.npix = (long long)p->npix();
  d.levels = p->opts.frame_levels;
  d.b = p->b;
  d.tau = (float)(p->lam / (2.0 * p->mu));
  d.mu = p->mu;
  d.stop = p->flags + FLAG_STOP;
  if (k <= K) {
    const int in = (k - 1) & 1, out = k & 1;
    d.xh = (k == 1) ? p->b : p->x;
    d.u = (k == 1) ? nullptr : p->s0[in];
    d.s = (k == 1) ? nullptr : p->s1[in];
    d.first = (k == 1);
    d.u_out = p->s0[out];
    d.s_out = p->s1[out];
    d.r_out = p->r;
    d.write_state = 1;
    d.prior_acc = p->trace_prior + (k - 1);
  } else {       // final: only ||w_K||_1 with w_K = u + Psi(xhat - Psi'u)
    const int in = K & 1;
    d.xh = (K == 0) ? p->b : p->x;
    d.u = (K == 0) ? nullptr : p->s0[in];
    d.s = (K == 0) ? nullptr : p->s1[in];
    d.first = (K == 0);
    d.write_state = 0;
    d.prior_acc = p->trace_prior + K;
  }
  return d;
}

// Iteration k (1-based) of the spatio-temporal prior; k = K+1 is the final
// prior term.  The state buffers are updated in place (m by the CG steps,
// e = d1 - v and p by the finishing kernel); a solve starts from
// m = p = x = H'y, d1 = 0.
StvSlice stv_desc(recon_plan* p, int k, int K, double* red) {
  StvSlice d{};
  d.Nx = p->Nx;
  d.Ny = p->Ny;
  d.Nt = p->Nt;
  d.n = (int)p->nimg();
  d.cg = p->opts.cg_steps;
  d.tau1 = (float)(p->lam / (2.0 * (p->mu / p->opts.rho)));
  d.rho = p->opts.rho;
  d.ws = p->opts.spatial_weight;
  d.m = p->s0[0];
  d.q = p->s0[1];
  d.e = p->s1[0];
  d.p = p->s2[0];
  d.r = p->s2[1];
  d.pc[0] = p->r;
  d.pc[1] = p->cgd;
  d.x = p->x;
  d.stop = p->flags + FLAG_STOP;
  d.red = red + (size_t)(std::min(k, std::max(K, 1)) - 1) * (2 * d.cg + 1);
  d.prior_acc = p->trace_prior + (k - 1);
  // residuals: iteration K-1 keeps d1, iteration K sums its change; the final
  // set reads m_{K-1}
  d.res_acc = p->res_acc;
  if (k == K - 1) d.d1_keep = p->res_d1;
  if (k == K) {
    d.res_last = 1;
    d.d1_ref = K >= 2 ? p->res_d1 : nullptr;
  }
  if (k == K + 1) d.m_prev = p->res_prev;
  return d;
}

ColSlice col_desc(recon_plan* p, int k, bool fused) {
  ColSlice c{};
  c.A = p->A;
  c.col_elems = p->pk.col_elems;
  c.Nx = p->Nx;
  c.Nt = p->Nt;
  c.Ny = p->Ny;
  c.nb = p->pk.nb;
  c.nunits = p->pk.nunits;
  c.r_tma = ((size_t)p->Ny * sizeof(float2)) % 16 == 0 ? 1 : 0;
  c.do_obj = fused ? 1 : 0;
  c.mu = p->mu;
  c.w_bx = -2.f;
  c.w_xr = 1.f;
  c.w_xx = -p->mu;
  c.stop = p->flags + FLAG_STOP;
  if (p->prior == RECON_PRIOR_TV) {
    c.base = p->b;
    c.add = p->s2[k & 1];
    c.coef = p->mu;
  } else if (p->prior == RECON_PRIOR_STV) {   // r = H'y + mu2 p, p = m' - d2 (in place)
    c.base = p->b;
    c.add = p->s2[0];
    c.coef = p->mu;
  } else {
    c.base = p->r;
    c.add = nullptr;
    c.coef = 0.f;
  }
  c.bsrc = p->b;
  c.xout = p->x;
  c.fid_acc = p->trace_fid + k;
  return c;
}

}  // namespace

recon_status finish_col_shape(Engine* e, recon_plan* const* plans, int n, int stages_req) {
  e->nb_max = 0;
  for (int q = 0; q < n; ++q) e->nb_max = std::max(e->nb_max, plans[q]->pk.nb);
  const int es = e->storage ? 4 : 8;
  const int maxst = col_inverse_max_stages(e->nb_max, n, e->work_max, es);
  const int qn = col_inverse_stage_quantum(es);
  int st = stages_req > 0 ? std::min(stages_req, maxst) : maxst;
  e->stages = std::max(qn, st / qn * qn);
  const size_t smem = col_inverse_smem(e->stages, e->nb_max, n, e->work_max, es);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin)
    return fail(RECON_ERR_UNSUPPORTED, "column-inverse kernel: the largest Ny and the work lists of this set of "
                                       "slices exceed shared memory");
  RC(prepare_col_inverse(e->storage, smem));
  return RECON_OK;
}

// The persistent TV solve when the engine's slices allow it: temporal TV, FP32
// inverses, a fixed iteration count, the fused objective (or none) and Nt <=
// kPersistNtMax, and every plan asks for it (opts.persistent).
recon_status engine_build_persist(Engine* e, recon_plan* const* plans, int n) {
  e->persist = false;
  if (e->prior != RECON_PRIOR_TV || e->storage != 0 || e->stop_test || (e->obj && !e->fused) || e->K < 1 ||
      e->volume)
    return RECON_OK;
  for (int q = 0; q < n; ++q)
    if (!plans[q]->opts.persistent || plans[q]->Nt > kPersistNtMax) return RECON_OK;
  // the per-step kernel's column lists (image-column-major, see build_col_work)
  std::vector<unsigned> work;
  std::vector<int> off;
  int work_max = 0;
  build_col_work(plans, n, e->grid, work, off, work_max);
  const int stages = persist_max_stages(e->nb_max, n, work_max);
  if (stages <= 0) return RECON_OK;   // the lists do not fit in shared memory: one launch per step
  size_t ncount = 0, task_sum = 0;   // task_sum: temporal chunks of one iteration
  for (int q = 0; q < n; ++q) {
    ncount += 2 * (size_t)plans[q]->Nx;
    task_sum += (size_t)plans[q]->Nx * ((plans[q]->Ny + kPersistChunkPx - 1) / kPersistChunkPx);
  }
  // colcnt and tdone of every slice, then the task queue's head and tail
  RC(e->arena.alloc(reinterpret_cast<void**>(&e->d_pcount), (ncount + 2) * sizeof(unsigned)));
  e->pcount_n = ncount + 2;
  // the temporal task ring: room for several iterations' tasks (one per image column each)
  unsigned cap = 1024;
  while (cap < 4 * task_sum) cap <<= 1;
  RC(e->arena.alloc(reinterpret_cast<void**>(&e->d_tq_ring), (size_t)cap * sizeof(int4)));
  e->tq_cap = cap;
  e->tq_total = (unsigned)((size_t)e->K * task_sum);
  std::vector<PersistSlice> ps(n);
  size_t o = 0;
  for (int q = 0; q < n; ++q) {
    recon_plan* p = plans[q];
    PersistSlice& d = ps[q];
    d.A = p->A;
    d.col_elems = p->pk.col_elems;
    d.Nx = p->Nx; d.Ny = p->Ny; d.Nt = p->Nt;
    d.nb = p->pk.nb;
    d.nunits = p->pk.nunits;
    d.nch = (p->Ny + kPersistChunkPx - 1) / kPersistChunkPx;
    d.b = p->b;
    d.x = p->x;
    for (int k = 0; k < 2; ++k) { d.m[k] = p->s0[k]; d.d1[k] = p->s1[k]; d.p[k] = p->s2[k]; }
    d.mu = p->mu;
    d.tau1 = (float)(p->lam / (2.0 * (p->mu / p->opts.rho)));
    d.rho = p->opts.rho;
    d.thomas = p->thomas;
    d.w_bx = -2.f; d.w_xr = 1.f; d.w_xx = -p->mu;
    d.do_obj = e->fused ? 1 : 0;
    d.trace_fid = p->trace_fid;
    d.trace_prior = p->trace_prior;
    d.colcnt = e->d_pcount + o;
    d.tdone = e->d_pcount + o + p->Nx;
    o += 2 * (size_t)p->Nx;
  }
  RC(upload(e->arena, &e->d_pslice, ps));
  RC(upload(e->arena, &e->d_pwork, work));
  RC(upload(e->arena, &e->d_pwork_off, off));
  e->pwork_max = work_max;
  e->pstages = stages;
  e->persist = true;
  return RECON_OK;
}

recon_status engine_build(Engine* e, recon_plan* const* plans, int n) {
  if (n < 1) return fail(RECON_ERR_INVALID_ARG, "empty batch");
  if (n > 255) return fail(RECON_ERR_UNSUPPORTED, "at most 255 slices per batch");
  recon_plan* p0 = plans[0];
  e->plans.assign(plans, plans + n);
  e->n = n;
  e->gens.resize(n);
  for (int q = 0; q < n; ++q) {
    if (plans[q]->broken) return fail(RECON_ERR_INVALID_ARG, "a plan failed recon_plan_set_mu and is unusable");
    e->gens[q] = plans[q]->generation;
  }
  e->K = p0->opts.max_iters;
  e->prior = p0->prior;
  e->tv = p0->prior == RECON_PRIOR_TV;
  e->levels = p0->opts.frame_levels;
  e->storage = p0->storage;
  e->obj = p0->opts.objective != 0 || p0->opts.tol > 0.0;
  e->stop_test = false;
  for (int q = 0; q < n; ++q) e->stop_test = e->stop_test || plans[q]->opts.tol > 0.0;
  e->overlap = true;
  for (int q = 0; q < n; ++q) e->overlap = e->overlap && plans[q]->opts.overlap != 0;
  e->fused = e->obj && p0->opts.objective != 2 && p0->storage == 0;
  for (int q = 1; q < n; ++q) {
    const recon_plan* p = plans[q];
    if (p->prior != p0->prior || p->opts.max_iters != e->K || p->storage != e->storage ||
        (p->prior == RECON_PRIOR_HAAR && p->opts.frame_levels != p0->opts.frame_levels) ||
        (p->opts.objective != 0 || p->opts.tol > 0.0) != e->obj || (p->opts.objective == 2) != (p0->opts.objective == 2))
      return fail(RECON_ERR_INVALID_ARG, "batched plans must share prior, max_iters, storage and objective mode");
    if (p->device != p0->device) return fail(RECON_ERR_INVALID_ARG, "batched plans must be on one device");
    if (p->prior == RECON_PRIOR_STV && p->opts.cg_steps != p0->opts.cg_steps)
      return fail(RECON_ERR_INVALID_ARG, "batched spatio-temporal plans must share cg_steps");
  }
  if (e->prior == RECON_PRIOR_STV) {
    e->cg = p0->opts.cg_steps;
    const size_t per = (size_t)std::max(e->K, 1) * (2 * e->cg + 1);
    e->stv_red.assign(n, nullptr);
    // a volume shares one set of slots (its sums run over every slice)
    for (int q = 0; q < (e->volume ? 1 : n); ++q)
      RC(e->arena.alloc(reinterpret_cast<void**>(&e->stv_red[q]), per * sizeof(double)));
    if (e->volume)
      for (int q = 1; q < n; ++q) e->stv_red[q] = e->stv_red[0];
    RC(e->arena.alloc(reinterpret_cast<void**>(&e->d_stv_count), (size_t)n * sizeof(unsigned)));
    RC(cudaMemset(e->d_stv_count, 0, (size_t)n * sizeof(unsigned)));
    int blocks = 0;
    for (int q = 0; q < n; ++q) blocks += (plans[q]->Nt * plans[q]->Nx + kStvRowsMin - 1) / kStvRowsMin;
    RC(e->arena.alloc(reinterpret_cast<void**>(&e->d_stv_part), (size_t)std::max(blocks, 1) * sizeof(double)));
  }
  const int K = e->K;
  // column descriptors, K sets (at least one so the layout is valid at K = 0)
  std::vector<ColSlice> cols((size_t)std::max(K, 1) * n);
  for (int k = 1; k <= std::max(K, 1); ++k)
    for (int q = 0; q < n; ++q) cols[(size_t)(k - 1) * n + q] = col_desc(plans[q], k, e->fused);
  RC(upload(e->arena, &e->d_col, cols));
  // temporal descriptors, K+1 sets
  e->Nt_max = 0;
  for (int q = 0; q < n; ++q) e->Nt_max = std::max(e->Nt_max, plans[q]->Nt);
  // a single plan uses its own tuning; a batch starts from the default (recon_batch_autotune)
  const int px = (n == 1 && p0->tile_px > 0) ? p0->tile_px : engine_default_tile(e);
  recon_status st = engine_set_tile(e, px);
  if (st != RECON_OK) return st;
  // finalize descriptors
  std::vector<FinSlice> fin(n);
  for (int q = 0; q < n; ++q) {
    recon_plan* p = plans[q];
    fin[q].fid = p->trace_fid;
    fin[q].prior = p->trace_prior;
    fin[q].yy = e->fused ? p->yy : nullptr;
    fin[q].J = p->trace_J;
    fin[q].flags = p->flags;
    fin[q].lam = p->lam;
    fin[q].tol = p->opts.tol;
  }
  RC(upload(e->arena, &e->d_fin, fin));
  // work lists and launch shape
  e->grid = std::max(1, p0->num_sms);
  std::vector<unsigned> work;
  std::vector<int> off;
  build_col_work(plans, n, e->grid, work, off, e->work_max);
  RC(upload(e->arena, &e->d_work, work));
  RC(upload(e->arena, &e->d_work_off, off));
  if (n == 1) {
    e->d_err = p0->flags;
  } else {
    RC(e->arena.alloc(reinterpret_cast<void**>(&e->d_err), FLAG_COUNT * sizeof(int)));
    RC(cudaMemset(e->d_err, 0, FLAG_COUNT * sizeof(int)));
  }
  recon_status st2 = finish_col_shape(e, plans, n,
                                      (n == 1 && p0->col_stages_tuned > 0) ? p0->col_stages_tuned : p0->opts.col_stages);
  if (st2 != RECON_OK) return st2;
  return engine_build_persist(e, plans, n);
}

int engine_tile_candidates(const Engine* e, int* out) {
  if (e->prior == RECON_PRIOR_STV) {   // image columns per block
    int nc = 0;
    for (int r : kStvRowCands) out[nc++] = r;
    return nc;
  }
  if (e->tv) return tv_tile_candidates(e->Nt_max, out);
  if (e->prior == RECON_PRIOR_HAAR) return haar_tile_candidates(e->Nt_max, e->levels, out);
  return dft_tile_candidates(e->Nt_max, out);
}

int engine_default_tile(const Engine* e) {
  if (e->prior == RECON_PRIOR_STV) return kStvRows;
  if (e->tv) return tv_tile_px(e->Nt_max);
  if (e->prior == RECON_PRIOR_HAAR) return haar_tile_px(e->Nt_max, e->levels);
  return dft_tile_px();
}

// (Re)builds the K+1 temporal descriptor sets for tiles of `px` pixels.
recon_status engine_set_tile(Engine* e, int px) {
  const int K = e->K, n = e->n;
  int cand[4];
  const int nc = engine_tile_candidates(e, cand);
  if (std::find(cand, cand + nc, px) == cand + nc) return fail(RECON_ERR_INVALID_ARG, "temporal tile width does not fit");
  std::vector<int> tile0(n);
  int blocks = 0;
  for (int q = 0; q < n; ++q) {
    tile0[q] = blocks;
    // temporal kernels tile pixels; the spatio-temporal kernels tile image columns (t, i)
    const size_t units = e->prior == RECON_PRIOR_STV ? (size_t)e->plans[q]->Nt * e->plans[q]->Nx
                                                     : e->plans[q]->npix();
    blocks += (int)((units + px - 1) / px);
  }
  void* old = e->d_tmp;
  if (e->prior == RECON_PRIOR_STV) {
    std::vector<StvSlice> t((size_t)(K + 1) * n);
    for (int k = 1; k <= K + 1; ++k)
      for (int q = 0; q < n; ++q) {
        StvSlice d = stv_desc(e->plans[q], k, K, e->stv_red[q]);
        d.tile0 = tile0[q];
        d.nblk = (e->plans[q]->Nt * e->plans[q]->Nx + px - 1) / px;
        d.rows = px;
        d.part = e->d_stv_part;
        if (e->volume) {   // neighbours at q -1 / q + 1, one sum over every slice
          d.res_acc = e->plans[0]->res_acc;   // the residuals of the volume
          d.wz = e->wz;
          d.zprev = q > 0;
          d.znext = q + 1 < n;
          d.count = e->d_stv_count;
          d.red0 = 0;
          d.rednblk = blocks;
        } else {
          d.count = e->d_stv_count + q;
          d.red0 = d.tile0;
          d.rednblk = d.nblk;
        }
        t[(size_t)(k - 1) * n + q] = d;
      }
    RC(upload(e->arena, reinterpret_cast<StvSlice**>(&e->d_tmp), t));
  } else if (e->tv) {
    std::vector<TvSlice> t((size_t)(K + 1) * n);
    e->tv_full.assign((size_t)K + 1, 0);
    const int ls = (e->Nt_max + kTvSeg - 1) / kTvSeg;
    for (int k = 1; k <= K + 1; ++k) {
      bool full = ls <= kTvFullLMax;
      for (int q = 0; q < n; ++q) {
        TvSlice d = tv_desc(e->plans[q], k, K);
        d.tile0 = tile0[q];
        t[(size_t)(k - 1) * n + q] = d;
        full = full && d.Nt == kTvSeg * ls && d.npix % kTvChunkPx == 0 && d.d1 && d.write_state;
      }
      e->tv_full[(size_t)k - 1] = full ? 1 : 0;
    }
    RC(upload(e->arena, reinterpret_cast<TvSlice**>(&e->d_tmp), t));
    RC(prepare_tv_temporal(e->Nt_max, px));
  } else if (e->prior == RECON_PRIOR_HAAR) {
    std::vector<HaarSlice> t((size_t)(K + 1) * n);
    for (int k = 1; k <= K + 1; ++k)
      for (int q = 0; q < n; ++q) {
        HaarSlice d = haar_desc(e->plans[q], k, K);
        d.tile0 = tile0[q];
        t[(size_t)(k - 1) * n + q] = d;
      }
    RC(upload(e->arena, reinterpret_cast<HaarSlice**>(&e->d_tmp), t));
    RC(prepare_haar_temporal(e->Nt_max, e->levels, px));
  } else {
    std::vector<DftSlice> t((size_t)(K + 1) * n);
    for (int k = 1; k <= K + 1; ++k)
      for (int q = 0; q < n; ++q) {
        DftSlice d = dft_desc(e->plans[q], k, K);
        d.tile0 = tile0[q];
        t[(size_t)(k - 1) * n + q] = d;
      }
    RC(upload(e->arena, reinterpret_cast<DftSlice**>(&e->d_tmp), t));
    RC(prepare_dft_temporal(e->Nt_max, px));
  }
  if (old) e->arena.free(old);
  e->tile_px = px;
  e->tmp_blocks = blocks;
  return RECON_OK;
}

recon_status engine_build_inverse(Engine* e, recon_plan* p) {
  e->plans = {p};
  e->n = 1;
  e->K = 1;
  e->storage = p->storage;
  e->obj = e->fused = false;
  ColSlice c = col_desc(p, 1, false);
  c.base = p->tmp_a;
  c.add = nullptr;
  c.coef = 0.f;
  c.bsrc = p->tmp_a;
  c.xout = p->tmp_b;
  c.fid_acc = nullptr;
  c.stop = nullptr;
  RC(upload(e->arena, &e->d_col, std::vector<ColSlice>{c}));
  e->grid = std::max(1, p->num_sms);
  std::vector<unsigned> work;
  std::vector<int> off;
  recon_plan* pl[1] = {p};
  build_col_work(pl, 1, e->grid, work, off, e->work_max);
  RC(upload(e->arena, &e->d_work, work));
  RC(upload(e->arena, &e->d_work_off, off));
  e->d_err = p->flags;
  return finish_col_shape(e, pl, 1, p->opts.col_stages);
}

recon_status launch_col_set(Engine* e, int set, cudaStream_t s, bool pdl) {
  ColLaunch L{};
  L.slices = e->d_col + (size_t)set * e->n;
  L.nslices = e->n;
  L.work = e->d_work;
  L.work_off = e->d_work_off;
  L.work_max = e->work_max;
  L.nb_max = e->nb_max;
  L.stages = e->stages;
  L.err = e->d_err;
  RC(launch_col_inverse(L, e->storage, e->grid, s, pdl));
  return RECON_OK;
}

recon_status launch_tmp_set(Engine* e, int set, cudaStream_t s, bool pdl) {
  TemporalLaunch L{};
  L.nslices = e->n;
  L.nblocks = e->tmp_blocks;
  L.Nt_max = e->Nt_max;
  L.tile_px = e->tile_px;
  if (e->prior == RECON_PRIOR_STV) {   // the prior term of set `set` (the final one in a solve)
    StvLaunch S{};
    S.slices = static_cast<StvSlice*>(e->d_tmp) + (size_t)set * e->n;
    S.nslices = e->n;
    S.nblocks = e->tmp_blocks;
    RC(launch_stv_prior(S, s));
  } else if (e->tv) {
    L.slices = static_cast<TvSlice*>(e->d_tmp) + (size_t)set * e->n;
    L.full = (size_t)set < e->tv_full.size() ? e->tv_full[(size_t)set] : 0;
    RC(launch_tv_temporal(L, s, pdl));
  } else if (e->prior == RECON_PRIOR_HAAR) {
    L.slices = static_cast<HaarSlice*>(e->d_tmp) + (size_t)set * e->n;
    RC(launch_haar_temporal(L, e->levels, s, pdl));
  } else {
    L.slices = static_cast<DftSlice*>(e->d_tmp) + (size_t)set * e->n;
    RC(launch_dft_temporal(L, s, pdl));
  }
  return RECON_OK;
}

// Spatio-temporal prior, iteration set+1 up to the inverse step: r and the
// prior term of J, the CG m-update, the d1 / p updates and the next threshold.
recon_status launch_stv_step(Engine* e, int set, cudaStream_t s) {
  StvLaunch S{};
  S.slices = static_cast<StvSlice*>(e->d_tmp) + (size_t)set * e->n;
  S.nslices = e->n;
  S.nblocks = e->tmp_blocks;
  int ny_max = 0;
  for (recon_plan* p : e->plans) ny_max = std::max(ny_max, p->Ny);
  S.dir_threads = (ny_max + 31) / 32 * 32;
  RC(launch_stv_rhs(S, s));
  for (int j = 0; j < e->cg; ++j) {
    S.step = j;
    RC(launch_stv_dir(S, s));
    RC(launch_stv_update(S, s));
  }
  RC(launch_stv_finish(S, s));
  return RECON_OK;
}

recon_status engine_iterate(Engine* e, cudaStream_t s, bool profile, bool allow_pdl) {
  const int K = e->K;
  const size_t nt = (size_t)K + 2;
  recon_plan* p0 = e->plans[0];
  const bool prof = profile && e->n == 1;
  for (recon_plan* p : e->plans) {
    RC(cudaMemsetAsync(p->res_acc, 0, 4 * sizeof(double), s));
    RC(cudaMemsetAsync(p->flags, 0, FLAG_COUNT * sizeof(int), s));
    RC(cudaMemsetAsync(p->trace_fid, 0, nt * sizeof(double), s));
    RC(cudaMemsetAsync(p->trace_prior, 0, nt * sizeof(double), s));
    RC(cudaMemsetAsync(p->trace_J, 0xff, nt * sizeof(double), s));  // NaN
  }
  if (e->n > 1) RC(cudaMemsetAsync(e->d_err, 0, FLAG_COUNT * sizeof(int), s));
  if (e->prior == RECON_PRIOR_STV) {   // m = p = x = H'y, d1 = 0
    for (recon_plan* p : e->plans) {
      const size_t bytes = p->nimg() * sizeof(float2);
      RC(cudaMemcpyAsync(p->s0[0], p->b, bytes, cudaMemcpyDeviceToDevice, s));
      RC(cudaMemcpyAsync(p->s2[0], p->b, bytes, cudaMemcpyDeviceToDevice, s));
      RC(cudaMemcpyAsync(p->x, p->b, bytes, cudaMemcpyDeviceToDevice, s));
    }
    RC(cudaMemsetAsync(e->d_stv_count, 0, (size_t)e->n * sizeof(unsigned), s));
    StvLaunch S{};   // e = -S(R m), d1 = 0
    S.slices = static_cast<StvSlice*>(e->d_tmp);
    S.nslices = e->n;
    S.nblocks = e->tmp_blocks;
    RC(launch_stv_init(S, s));
  }
  recon_status st;
  if (e->obj)
    for (recon_plan* p : e->plans)
      if ((st = plan_objective(p, p->b, p->trace_fid, s)) != RECON_OK) return st;
  if (e->persist) {
    // T_1 from x = m = p = H'y, then iterations 1..K (with T_2..T_{K+1}) in one launch
    RC(cudaMemsetAsync(e->d_pcount, 0, e->pcount_n * sizeof(unsigned), s));
    RC(cudaMemsetAsync(e->d_tq_ring, 0, (size_t)e->tq_cap * sizeof(int4), s));
    if (prof) p0->mark(p0->ev_tmp, p0->n_tmp, true, s);
    if ((st = launch_tmp_set(e, 0, s)) != RECON_OK) return st;
    if (prof) p0->mark(p0->ev_tmp, p0->n_tmp, false, s);
    PersistLaunch L{};
    L.slices = e->d_pslice;
    L.nslices = e->n;
    L.work = e->d_pwork;
    L.work_off = e->d_pwork_off;
    L.work_max = e->pwork_max;
    L.nb_max = e->nb_max;
    L.stages = e->pstages;
    L.K = K;
    L.err = e->d_err;
    L.tq_ring = e->d_tq_ring;
    L.tq_cap = e->tq_cap;
    L.tq_head = e->d_pcount + e->pcount_n - 2;
    L.tq_tail = e->d_pcount + e->pcount_n - 1;
    L.tq_total = e->tq_total;
    if (prof) p0->mark(p0->ev_col, p0->n_col, true, s);
    RC(launch_persist_tv(L, e->grid, s));
    if (prof) p0->mark(p0->ev_col, p0->n_col, false, s);
    if (e->obj) RC(launch_finalize(e->d_fin, e->n, 0, K, s));
    for (recon_plan* p : e->plans)
      if ((st = launch_residuals(p, s)) != RECON_OK) return st;
    return RECON_OK;
  }
  // Programmatic dependent launches between the temporal (TV, DFT, Haar) and
  // inverse kernels: each waits in-device for the kernel before it.  Measured
  // on the cardiac workload: TV 2791 -> 2830 iters/s.  Not used
  //   - with a stopping test (the inverse kernel reads the stop flags before
  //     its wait) or with profiling events between the launches;
  //   - for the spatio-temporal prior: its CG launches (every block of each
  //     resident at once, so the next grid's blocks wait beside them) ran 3 %
  //     slower with the dependencies;
  //   - for batches (allow_pdl false): their steady state is a graph replay,
  //     which has no launch latency to hide, and the 64-slice batch ran 1.6 %
  //     slower with the dependencies captured;
  //   - while the stream is being captured.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RC(cudaStreamIsCapturing(s, &cap));
  const bool pdl = allow_pdl && e->overlap && e->prior != RECON_PRIOR_STV && !e->stop_test && !prof &&
                   cap == cudaStreamCaptureStatusNone;
  for (int k = 1; k <= K; ++k) {
    if (k == K && e->prior == RECON_PRIOR_STV)   // m_{K-1}, before the last m-update
      for (recon_plan* p : e->plans)
        RC(cudaMemcpyAsync(p->res_prev, p->s0[0], p->nimg() * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (prof) p0->mark(p0->ev_tmp, p0->n_tmp, true, s);
    if (e->prior == RECON_PRIOR_STV) st = launch_stv_step(e, k - 1, s);
    else st = launch_tmp_set(e, k - 1, s, pdl);
    if (st != RECON_OK) return st;
    if (prof) p0->mark(p0->ev_tmp, p0->n_tmp, false, s);
    if (e->stop_test) RC(launch_finalize(e->d_fin, e->n, k - 1, k - 1, s));
    if (k == K && K >= 2 && (e->prior == RECON_PRIOR_DFT || e->prior == RECON_PRIOR_HAAR))   // xhat_{K-1}
      for (recon_plan* p : e->plans)
        RC(cudaMemcpyAsync(p->res_prev, p->x, p->nimg() * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (prof) p0->mark(p0->ev_col, p0->n_col, true, s);
    if ((st = launch_col_set(e, k - 1, s, pdl)) != RECON_OK) return st;
    if (prof) p0->mark(p0->ev_col, p0->n_col, false, s);
    if (e->obj && !e->fused)
      for (recon_plan* p : e->plans)
        if ((st = plan_objective(p, p->x, p->trace_fid + k, s)) != RECON_OK) return st;
  }
  if (e->obj) {
    if ((st = launch_tmp_set(e, K, s, pdl)) != RECON_OK) return st;
    // with a fixed iteration count J(0) .. J(K) are formed here, in one launch
    RC(launch_finalize(e->d_fin, e->n, e->stop_test ? K : 0, K, s));
  }
  if (e->prior == RECON_PRIOR_STV) {
    if (K >= 1) {   // the sums of the final set (the last iteration's d1 change is already in)
      StvLaunch S{};
      S.slices = static_cast<StvSlice*>(e->d_tmp) + (size_t)K * e->n;
      S.nslices = e->n;
      S.nblocks = e->tmp_blocks;
      RC(launch_stv_residuals(S, s));
      if (e->volume)   // every slice reports the volume's residuals
        for (int q = 1; q < e->n; ++q)
          RC(cudaMemcpyAsync(e->plans[q]->res_acc, p0->res_acc, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return RECON_OK;
  }
  for (recon_plan* p : e->plans)
    if ((st = launch_residuals(p, s)) != RECON_OK) return st;
  return RECON_OK;
}

recon_status engine_apply_inverse(Engine* e, cudaStream_t s) { return launch_col_set(e, 0, s); }

recon_status engine_check(const Engine* e) {
  for (int q = 0; q < e->n; ++q) {
    const recon_plan* p = e->plans[q];
    if (p->broken) return fail(RECON_ERR_INVALID_ARG, "a plan failed recon_plan_set_mu and is unusable");
    if (q < (int)e->gens.size() && p->generation != e->gens[q])
      return fail(RECON_ERR_INVALID_ARG, "a plan's mu changed (recon_plan_set_mu) after this batch was built: rebuild it");
  }
  return RECON_OK;
}

const float2* plan_result(const recon_plan* p) { return p->opts.max_iters == 0 ? p->b : p->x; }

}  // namespace recon

// ---------------------------------------------------------------------------
// batched entry points
// ---------------------------------------------------------------------------
using namespace recon;

recon_batch::~recon_batch() {
  if (graph) cudaGraphExecDestroy(graph);
  if (cap_stream) cudaStreamDestroy(cap_stream);
}

namespace {

recon_status batch_enqueue(recon_batch* b, const float* const* kspace, float* const* image, cudaStream_t s) {
  recon_status st;
  for (int q = 0; q < b->eng.n; ++q)
    if ((st = plan_prologue(b->eng.plans[q], kspace[q], RECON_STORAGE_FP32, nullptr, s)) != RECON_OK) return st;
  if ((st = engine_iterate(&b->eng, s, false, false)) != RECON_OK) return st;
  for (int q = 0; q < b->eng.n; ++q) {
    recon_plan* p = b->eng.plans[q];
    if ((st = plan_to_user(p, plan_result(p), reinterpret_cast<float2*>(image[q]), s)) != RECON_OK) return st;
  }
  return RECON_OK;
}

}  // namespace

extern "C" {

recon_status recon_batch_create(recon_batch** out, recon_plan* const* plans, int n) {
  if (!out || !plans || n < 1) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  for (int q = 0; q < n; ++q)
    if (!plans[q]) return fail(RECON_ERR_INVALID_ARG, "NULL plan in batch");
  auto* b = new recon_batch();
  recon_status st = engine_build(&b->eng, plans, n);
  if (st != RECON_OK) {
    delete b;
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  *out = b;
  return RECON_OK;
}

recon_status recon_volume_create(recon_batch** out, recon_plan* const* plans, int nz, float wz) {
  if (!out || !plans || nz < 1) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  if (!(wz >= 0.f) || !std::isfinite(wz)) return fail(RECON_ERR_INVALID_ARG, "wz must be >= 0");
  for (int q = 0; q < nz; ++q) {
    const recon_plan* p = plans[q];
    if (!p) return fail(RECON_ERR_INVALID_ARG, "NULL plan in volume");
    if (p->prior != RECON_PRIOR_STV) return fail(RECON_ERR_INVALID_ARG, "a volume takes spatio-temporal plans");
    if (p->Nx != plans[0]->Nx || p->Ny != plans[0]->Ny || p->Nt != plans[0]->Nt)
      return fail(RECON_ERR_INVALID_ARG, "the slices of a volume share Nx, Ny and Nt");
    if (p->opts.tol > 0.0)
      return fail(RECON_ERR_INVALID_ARG, "a volume runs a fixed number of iterations (tol = 0)");
  }
  auto* b = new recon_batch();
  b->eng.volume = true;
  b->eng.wz = wz;
  recon_status st = engine_build(&b->eng, plans, nz);
  if (st != RECON_OK) {
    delete b;
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  *out = b;
  return RECON_OK;
}

recon_status recon_batch_solve(recon_batch* b, const float* const* kspace, float* const* image, void* stream) {
  if (!b || !kspace || !image) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  {
    recon_status st = engine_check(&b->eng);
    if (st != RECON_OK) return st;
  }
  const int n = b->eng.n;
  std::vector<const void*> key;
  for (int q = 0; q < n; ++q) {
    if (!kspace[q] || !image[q]) return fail(RECON_ERR_INVALID_ARG, "NULL buffer in batch");
    key.push_back(kspace[q]);
    key.push_back(image[q]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (recon_plan* p : b->eng.plans) p->last_stream = s;
  if (b->graph && key == b->key) {
    RC(cudaGraphLaunch(b->graph, s));
    return RECON_OK;
  }
  // first call with these buffers: run directly (sets every kernel attribute),
  // then capture the same sequence for the next calls
  recon_status st = batch_enqueue(b, kspace, image, s);
  if (st != RECON_OK) return st;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (b->no_graph) return RECON_OK;
  RC(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  st = batch_enqueue(b, kspace, image, b->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
  if (st == RECON_OK && ce == cudaSuccess) {
    ce = cudaGraphInstantiate(&b->graph, g, 0);
    if (ce != cudaSuccess) b->graph = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  if (st != RECON_OK || ce != cudaSuccess) {
    // a launch this runtime cannot capture (the persistent solve is one
    // cooperative launch): later calls run the same sequence directly
    (void)cudaGetLastError();
    b->graph = nullptr;
    b->no_graph = true;
    set_last_error("");
    return RECON_OK;
  }
  b->key = key;
  return RECON_OK;
}

recon_status recon_batch_info(recon_batch* b, recon_info* info, void* stream) {
  if (!b || !info) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status worst = RECON_OK;
  for (int q = 0; q < b->eng.n; ++q) {
    recon_status st = plan_fill_info(b->eng.plans[q], &info[q], s);
    if (st != RECON_OK && worst == RECON_OK) worst = st;
  }
  int err = 0;
  if (b->eng.n > 1) RC(cudaMemcpy(&err, b->eng.d_err + FLAG_ERR, sizeof(int), cudaMemcpyDeviceToHost));
  if (err & DEV_ERR_TIMEOUT) return fail(RECON_ERR_TIMEOUT, "a bounded device-side wait timed out");
  return worst;
}

recon_status recon_batch_destroy(recon_batch* b) {
  if (!b) return RECON_OK;
  for (recon_plan* p : b->eng.plans)
    if (p && p->last_stream) cudaStreamSynchronize(p->last_stream);
  delete b;
  return RECON_OK;
}

}  // extern "C"
