// Differentiable unrolled Algorithm 2: hand-written adjoint of K ADMM steps.
//
// One step from the state (x, m, d1, d2) (d2 = x - p in the forward kernels):
//   a = D m + d1;  v = S(a, tau1);  rhs = D'(v - d1) + rho (x + d2);
//   m' = M^{-1} rhs (M = rho I + D'D);  r = b + mu (m' - d2);  x' = A(mu) r;
//   d1' = d1 - v + D m';  d2' = d2 - m' + x';   tau1 = lambda rho / (2 mu)
// Reverse of one step, given the adjoints of (x', m', d1', d2'):
//   r_bar = A (x_bar' + d2_bar')            (the column-inverse kernel; A is Hermitian)
//   mu_bar += -Re<r_bar, x'>                (dA/dmu = -A^2; dot product in its epilogue)
//   then, per pixel along t (k_tv_backward):
//   mt = m_bar' - d2_bar' + D' d1_bar' + mu r_bar;  rhs_bar = M^{-1} mt
//   b_bar += r_bar;  mu_bar += Re<r_bar, m' - d2>
//   x_bar = rho rhs_bar;  d2_bar = d2_bar' - mu r_bar + rho rhs_bar
//   u = D rhs_bar;  v_bar = -d1_bar' + u;  d1_bar = d1_bar' - u + a_bar;  m_bar = D' a_bar
//   a_bar = v_bar - (tau1/|a|)(v_bar - n Re(conj(n) v_bar)) for |a| > tau1 (else 0), n = a/|a|
//   tau_bar += -Re(conj(n) v_bar) for |a| > tau1
// At the first step b_bar also collects x_bar + m_bar (x0 = m0 = H'y), and
// finally y_bar = H b_bar.  Complex gradients use the dL/dRe + i dL/dIm
// convention.  The forward keeps the state every `seg` steps; the reverse
// recomputes each segment from its checkpoint before walking it backwards.
#include <algorithm>
#include <vector>

#include "plan.h"

namespace recon {

constexpr int kBwdThreads = 128;

__global__ void __launch_bounds__(kBwdThreads) k_tv_backward(const TvBwdSlice* sls, int nslices) {
  extern __shared__ float2 sm_bw[];  // [Nt][kBwdThreads]: Thomas sweep
  __shared__ double red[32];
  // slice of this block
  int lo = 0, hi = nslices - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sls[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const TvBwdSlice& P = sls[lo];
  const int tid = threadIdx.x, Nt = P.Nt;
  const long long N = P.npix;
  const long long pix = (long long)(blockIdx.x - P.tile0) * kBwdThreads + tid;
  double mu_part = 0.0, tau_part = 0.0;
  if (pix < N) {
    const float mu = P.mu, rho = P.rho, tau = P.tau1;
    // pass 1: mt_t and the forward Thomas sweep; b_bar += r_bar; mu term
    float2 dprev = make_float2(0.f, 0.f), d1b_prev = make_float2(0.f, 0.f);
    for (int t = 0; t < Nt; ++t) {
      const long long g = t * N + pix;
      const float2 rb = P.rb[g];
      const float2 d1b = (P.d1b && t + 1 < Nt) ? P.d1b[g] : make_float2(0.f, 0.f);
      // (D' u)_t = u_{t-1} - u_t
      float2 mt = c_sub(c_add(P.mb[g], c_sub(d1b_prev, d1b)), P.d2b[g]);
      mt.x = fmaf(mu, rb.x, mt.x);
      mt.y = fmaf(mu, rb.y, mt.y);
      dprev = c_scale(c_add(mt, dprev), __ldg(P.thomas + t));
      sm_bw[t * kBwdThreads + tid] = dprev;
      d1b_prev = d1b;
      const float2 d20 = c_sub(P.x0[g], P.p0[g]);
      const float2 w = c_sub(P.m1[g], d20);
      mu_part += (double)rb.x * w.x + (double)rb.y * w.y;
      P.bbar[g] = c_add(P.bbar[g], rb);
    }
    // pass 2: backward sweep -> rhs_bar in place
    float2 next = make_float2(0.f, 0.f);
    for (int t = Nt - 1; t >= 0; --t) {
      const float inv = __ldg(P.thomas + t);
      const float2 dp = sm_bw[t * kBwdThreads + tid];
      next = make_float2(fmaf(inv, next.x, dp.x), fmaf(inv, next.y, dp.y));
      sm_bw[t * kBwdThreads + tid] = next;
    }
    // pass 3: adjoints of the inputs
    float2 ab_prev = make_float2(0.f, 0.f);
    for (int t = 0; t < Nt; ++t) {
      const long long g = t * N + pix;
      const float2 rhsb = sm_bw[t * kBwdThreads + tid];
      const float2 rb = P.rb[g];
      const float2 xb = c_scale(rhsb, rho);
      float2 d2o = c_add(P.d2b[g], xb);
      d2o.x = fmaf(-mu, rb.x, d2o.x);
      d2o.y = fmaf(-mu, rb.y, d2o.y);
      float2 ab = make_float2(0.f, 0.f);
      if (t + 1 < Nt) {
        const float2 d1b = P.d1b ? P.d1b[g] : make_float2(0.f, 0.f);
        const float2 u = c_sub(sm_bw[(t + 1) * kBwdThreads + tid], rhsb);   // (D rhs_bar)_t
        const float2 vb = c_sub(u, d1b);
        const float2 d10 = P.d10 ? P.d10[g] : make_float2(0.f, 0.f);
        const float2 a = c_add(c_sub(P.m0[g + N], P.m0[g]), d10);
        const float mag = c_abs(a);
        if (mag > tau) {
          const float2 n = make_float2(a.x / mag, a.y / mag);
          const float proj = n.x * vb.x + n.y * vb.y;   // Re(conj(n) v_bar)
          const float sc = tau / mag;
          ab = make_float2(vb.x - sc * (vb.x - n.x * proj), vb.y - sc * (vb.y - n.y * proj));
          tau_part -= (double)proj;
        }
        P.d1b_out[g] = c_add(c_sub(d1b, u), ab);
      }
      const float2 mo = c_sub(ab_prev, ab);   // (D' a_bar)_t
      P.xb_out[g] = xb;
      P.mb_out[g] = mo;
      P.d2b_out[g] = d2o;
      if (P.first) P.bbar[g] = c_add(P.bbar[g], c_add(xb, mo));
      ab_prev = ab;
    }
  }
  const double s1 = group_sum(mu_part, red, tid, kBwdThreads, BlockBar());
  if (tid == 0) atomicAdd(P.mu_acc, s1);
  const double s2 = group_sum(tau_part, red, tid, kBwdThreads, BlockBar());
  if (tid == 0) atomicAdd(P.tau_acc, s2);
}

static cudaError_t launch_tv_backward(const TvBwdSlice* sls, int nslices, int nblocks, int Nt_max, cudaStream_t s) {
  const size_t smem = (size_t)Nt_max * kBwdThreads * sizeof(float2);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_tv_backward), smem);
    if (e != cudaSuccess) return e;
  }
  k_tv_backward<<<nblocks, kBwdThreads, smem, s>>>(sls, nslices);
  note_launch();
  return cudaGetLastError();
}

}  // namespace recon

using namespace recon;

struct GradSlice {        // per-slice buffers of the gradient engine
  struct State { float2 *m, *d1, *p, *x; };
  std::vector<State> ckpt, seg;
  State adj[2];           // adjoints (xb, mb, d1b, d2b) of a state; parity of the step index
  float2* rbar = nullptr;
  float2* bbar = nullptr;
  float2* kgrad_tmp = nullptr;   // hybrid rows of H b_bar
  double* acc = nullptr;         // [0] mu (A term), [1] mu (r term), [2] tau, [3] unused prior
};

struct recon_grad {
  Engine fwd;             // forward / recompute: temporal + inverse sets 0..K-1
  Engine bwd;             // reverse: inverse sets 0..K-1 (set k-1 = step k)
  TvBwdSlice* d_tb = nullptr;
  int tb_blocks = 0;
  int K = 0, seg = 1, n = 0, ncheck = 0;
  std::vector<GradSlice> sl;
  DevArena arena;
};

namespace {

GradSlice::State state_of(const recon_grad* g, recon_plan* p, const GradSlice& gs, int k) {
  if (k == 0) return {p->b, nullptr, p->b, p->b};
  if (k % g->seg == 0) return gs.ckpt[k / g->seg - 1];
  if (k == g->K) return gs.ckpt[g->ncheck - 1];
  return gs.seg[k % g->seg - 1];
}

}  // namespace

extern "C" {

recon_status recon_grad_create(recon_grad** out, recon_plan* const* plans, int n, int checkpoint_every) {
  if (!out || !plans || n < 1 || n > 255) return fail(RECON_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  const int K = plans[0]->opts.max_iters;
  for (int q = 0; q < n; ++q) {
    const recon_plan* p = plans[q];
    if (!p) return fail(RECON_ERR_INVALID_ARG, "NULL plan");
    if (p->prior != RECON_PRIOR_TV) return fail(RECON_ERR_UNSUPPORTED, "the adjoint is implemented for the TV prior");
    if (p->Nx != p->Nx_full) return fail(RECON_ERR_UNSUPPORTED, "the adjoint needs whole plans (dL/dy spans all columns)");
    if (p->opts.max_iters != K || p->storage != plans[0]->storage)
      return fail(RECON_ERR_INVALID_ARG, "plans must share max_iters and storage");
  }
  if (K < 1) return fail(RECON_ERR_INVALID_ARG, "max_iters must be >= 1");
  auto* g = new recon_grad();
  auto bail = [&](recon_status st) {
    delete g;
    return st;
  };
  g->K = K;
  g->n = n;
  g->seg = std::max(1, std::min(checkpoint_every > 0 ? checkpoint_every : 5, K));
  g->ncheck = (K + g->seg - 1) / g->seg;
  g->sl.resize(n);
  // buffers
  for (int q = 0; q < n; ++q) {
    recon_plan* p = plans[q];
    GradSlice& gs = g->sl[q];
    const size_t bytes = p->nimg() * sizeof(float2);
    auto make_state = [&](GradSlice::State& st) -> cudaError_t {
      cudaError_t e = g->arena.alloc((void**)&st.m, bytes);
      if (e == cudaSuccess) e = g->arena.alloc((void**)&st.d1, bytes);
      if (e == cudaSuccess) e = g->arena.alloc((void**)&st.p, bytes);
      if (e == cudaSuccess) e = g->arena.alloc((void**)&st.x, bytes);
      return e;
    };
    gs.ckpt.resize(g->ncheck);
    gs.seg.resize(g->seg - 1);
    for (auto& st : gs.ckpt)
      if (cudaError_t e = make_state(st); e != cudaSuccess) return bail(cuda_fail(e, "gradient checkpoints"));
    for (auto& st : gs.seg)
      if (cudaError_t e = make_state(st); e != cudaSuccess) return bail(cuda_fail(e, "gradient segment"));
    for (auto& st : gs.adj)
      if (cudaError_t e = make_state(st); e != cudaSuccess) return bail(cuda_fail(e, "gradient adjoints"));
    if (g->arena.alloc((void**)&gs.rbar, bytes) != cudaSuccess || g->arena.alloc((void**)&gs.bbar, bytes) != cudaSuccess ||
        g->arena.alloc((void**)&gs.kgrad_tmp, std::max<size_t>(1, (size_t)p->total_rows * p->Nx * p->Nc) * sizeof(float2)) != cudaSuccess ||
        g->arena.alloc((void**)&gs.acc, 4 * sizeof(double)) != cudaSuccess)
      return bail(fail(RECON_ERR_OOM, "gradient buffers"));
  }
  std::vector<unsigned> work;
  std::vector<int> off;
  int work_max = 0;
  const int grid = std::max(1, plans[0]->num_sms);
  build_col_work(plans, n, grid, work, off, work_max);
  for (int q = 0; q < n; ++q)
    if (plans[q]->broken) return bail(fail(RECON_ERR_INVALID_ARG, "a plan failed recon_plan_set_mu and is unusable"));
  for (Engine* e : {&g->fwd, &g->bwd}) {
    e->plans.assign(plans, plans + n);
    e->n = n;
    e->gens.resize(n);
    for (int q = 0; q < n; ++q) e->gens[q] = plans[q]->generation;
    e->K = K;
    e->tv = true;
    e->storage = plans[0]->storage;
    e->grid = grid;
    e->work_max = work_max;
    if (e->arena.alloc((void**)&e->d_work, work.size() * sizeof(unsigned)) != cudaSuccess ||
        e->arena.alloc((void**)&e->d_work_off, off.size() * sizeof(int)) != cudaSuccess ||
        e->arena.alloc((void**)&e->d_err, FLAG_COUNT * sizeof(int)) != cudaSuccess)
      return bail(fail(RECON_ERR_OOM, "gradient launch data"));
    cudaMemcpy(e->d_work, work.data(), work.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    cudaMemcpy(e->d_work_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemset(e->d_err, 0, FLAG_COUNT * sizeof(int));
  }
  // descriptors
  int Nt_max = 0;
  for (int q = 0; q < n; ++q) Nt_max = std::max(Nt_max, plans[q]->Nt);
  const int px = tv_tile_px(Nt_max);
  std::vector<int> tile0(n), tile0b(n);
  int blocks = 0, blocksb = 0;
  for (int q = 0; q < n; ++q) {
    tile0[q] = blocks;
    blocks += (int)((plans[q]->npix() + px - 1) / px);
    tile0b[q] = blocksb;
    blocksb += (int)((plans[q]->npix() + kBwdThreads - 1) / kBwdThreads);
  }
  std::vector<TvSlice> tf((size_t)K * n);
  std::vector<ColSlice> cf((size_t)K * n), cb((size_t)K * n);
  std::vector<TvBwdSlice> tb((size_t)K * n);
  for (int k = 1; k <= K; ++k) {
    for (int q = 0; q < n; ++q) {
      recon_plan* p = plans[q];
      GradSlice& gs = g->sl[q];
      const GradSlice::State s0 = state_of(g, p, gs, k - 1), s1 = state_of(g, p, gs, k);
      const size_t at = (size_t)(k - 1) * n + q;
      TvSlice& t = tf[at];
      t = TvSlice{};
      t.Nt = p->Nt;
      t.npix = (long long)p->npix();
      t.m = s0.m; t.d1 = s0.d1; t.x = s0.x; t.p = s0.p;
      t.m_out = s1.m; t.d1_out = s1.d1; t.p_out = s1.p;
      t.tau1 = (float)(p->lam / (2.0 * (p->mu / p->opts.rho)));   // as in the solve
      t.rho = p->opts.rho;
      t.thomas = p->thomas;
      t.write_state = 1;
      t.prior_acc = gs.acc + 3;
      t.stop = nullptr;
      t.tile0 = tile0[q];
      ColSlice c{};
      c.A = p->A;
      c.col_elems = p->pk.col_elems;
      c.Nx = p->Nx;
      c.Nt = p->Nt;
      c.Ny = p->Ny;
      c.nb = p->pk.nb;
      c.nunits = p->pk.nunits;
      c.r_tma = ((size_t)p->Ny * sizeof(float2)) % 16 == 0 ? 1 : 0;
      c.mu = p->mu;
      c.stop = nullptr;
      // forward: x_k = A (b + mu p_k)
      c.do_obj = 0;
      c.base = p->b; c.add = s1.p; c.coef = p->mu; c.bsrc = p->b; c.xout = s1.x; c.fid_acc = nullptr;
      cf[at] = c;
      // reverse: r_bar = A (x_bar_k + d2_bar_k), mu_bar += -Re<r_bar, x_k>
      const GradSlice::State& a1 = gs.adj[k & 1];
      c.do_obj = 1;
      c.base = a1.x; c.add = a1.p; c.coef = 1.f;   // adjoint slots: x = x_bar, p = d2_bar
      c.bsrc = s1.x; c.xout = gs.rbar;
      c.w_bx = -1.f; c.w_xr = 0.f; c.w_xx = 0.f;
      c.fid_acc = gs.acc + 0;
      cb[at] = c;
      TvBwdSlice b{};
      b.Nt = p->Nt;
      b.npix = (long long)p->npix();
      b.xb = a1.x; b.mb = a1.m; b.d1b = (k == K) ? nullptr : a1.d1; b.d2b = a1.p; b.rb = gs.rbar;
      b.x0 = s0.x; b.m0 = s0.m; b.d10 = s0.d1; b.p0 = s0.p; b.m1 = s1.m;
      const GradSlice::State& a0 = gs.adj[(k - 1) & 1];
      b.xb_out = a0.x; b.mb_out = a0.m; b.d1b_out = a0.d1; b.d2b_out = a0.p;
      b.bbar = gs.bbar;
      b.tau1 = t.tau1; b.rho = t.rho; b.mu = p->mu;
      b.thomas = p->thomas;
      b.first = (k == 1);
      b.mu_acc = gs.acc + 1;
      b.tau_acc = gs.acc + 2;
      b.tile0 = tile0b[q];
      tb[at] = b;
    }
  }
  cudaError_t e = g->arena.alloc(&g->fwd.d_tmp, tf.size() * sizeof(TvSlice));
  if (e == cudaSuccess) e = cudaMemcpy(g->fwd.d_tmp, tf.data(), tf.size() * sizeof(TvSlice), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = g->arena.alloc((void**)&g->fwd.d_col, cf.size() * sizeof(ColSlice));
  if (e == cudaSuccess) e = cudaMemcpy(g->fwd.d_col, cf.data(), cf.size() * sizeof(ColSlice), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = g->arena.alloc((void**)&g->bwd.d_col, cb.size() * sizeof(ColSlice));
  if (e == cudaSuccess) e = cudaMemcpy(g->bwd.d_col, cb.data(), cb.size() * sizeof(ColSlice), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = g->arena.alloc((void**)&g->d_tb, tb.size() * sizeof(TvBwdSlice));
  if (e == cudaSuccess) e = cudaMemcpy(g->d_tb, tb.data(), tb.size() * sizeof(TvBwdSlice), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(e, "gradient descriptors"));
  g->fwd.Nt_max = g->bwd.Nt_max = Nt_max;
  g->fwd.tile_px = px;
  g->fwd.tmp_blocks = blocks;
  g->tb_blocks = blocksb;
  recon_status st = finish_col_shape(&g->fwd, plans, n, plans[0]->opts.col_stages);
  if (st == RECON_OK) st = finish_col_shape(&g->bwd, plans, n, plans[0]->opts.col_stages);
  if (st != RECON_OK) return bail(st);
  if (prepare_tv_temporal(Nt_max, px) != cudaSuccess) return bail(fail(RECON_ERR_CUDA, "temporal kernel attributes"));
  *out = g;
  return RECON_OK;
}

recon_status recon_grad_forward(recon_grad* g, const float* const* kspace, float* const* image, void* stream) {
  if (!g || !kspace || !image) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  {
    recon_status st0 = engine_check(&g->fwd);
    if (st0 != RECON_OK) return st0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status st;
  for (recon_plan* p : g->fwd.plans) p->last_stream = s;
  for (int q = 0; q < g->n; ++q)
    if ((st = plan_prologue(g->fwd.plans[q], kspace[q], RECON_STORAGE_FP32, nullptr, s)) != RECON_OK) return st;
  for (int k = 1; k <= g->K; ++k) {
    if ((st = launch_tmp_set(&g->fwd, k - 1, s)) != RECON_OK) return st;
    if ((st = launch_col_set(&g->fwd, k - 1, s)) != RECON_OK) return st;
  }
  for (int q = 0; q < g->n; ++q) {
    recon_plan* p = g->fwd.plans[q];
    const GradSlice::State sK = state_of(g, p, g->sl[q], g->K);
    if ((st = plan_to_user(p, sK.x, reinterpret_cast<float2*>(image[q]), s)) != RECON_OK) return st;
  }
  return RECON_OK;
}

recon_status recon_grad_backward(recon_grad* g, const float* const* grad_image, float* const* grad_kspace,
                                 double* grad_lambda, double* grad_mu, void* stream) {
  if (!g || !grad_image || !grad_kspace) return fail(RECON_ERR_INVALID_ARG, "NULL argument");
  {
    recon_status st0 = engine_check(&g->fwd);
    if (st0 != RECON_OK) return st0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = g->K, n = g->n;
  recon_status st;
  for (int q = 0; q < n; ++q) {
    recon_plan* p = g->fwd.plans[q];
    GradSlice& gs = g->sl[q];
    const size_t bytes = p->nimg() * sizeof(float2);
    const GradSlice::State& aK = gs.adj[K & 1];
    if ((st = plan_to_internal(p, reinterpret_cast<const float2*>(grad_image[q]), aK.x, s)) != RECON_OK) return st;
    RC(cudaMemsetAsync(aK.m, 0, bytes, s));
    RC(cudaMemsetAsync(aK.p, 0, bytes, s));     // d2_bar
    RC(cudaMemsetAsync(gs.bbar, 0, bytes, s));
    RC(cudaMemsetAsync(gs.acc, 0, 4 * sizeof(double), s));
  }
  for (int c = g->ncheck; c >= 1; --c) {
    const int k0 = (c - 1) * g->seg, k1 = std::min(c * g->seg, K);
    // recompute the segment's inner states from its checkpoint
    for (int k = k0 + 1; k < k1; ++k) {
      if ((st = launch_tmp_set(&g->fwd, k - 1, s)) != RECON_OK) return st;
      if ((st = launch_col_set(&g->fwd, k - 1, s)) != RECON_OK) return st;
    }
    for (int k = k1; k > k0; --k) {
      if ((st = launch_col_set(&g->bwd, k - 1, s)) != RECON_OK) return st;
      RC(launch_tv_backward(g->d_tb + (size_t)(k - 1) * n, n, g->tb_blocks, g->bwd.Nt_max, s));
    }
  }
  // y_bar = H b_bar (unsampled rows 0)
  for (int q = 0; q < n; ++q) {
    recon_plan* p = g->fwd.plans[q];
    GradSlice& gs = g->sl[q];
    RC(launch_forward_cols(gs.bbar, p->sens, gs.kgrad_tmp, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc, p->fy, s));
    RC(cudaMemsetAsync(grad_kspace[q], 0, (size_t)p->Nt * p->Nc * p->Ny * p->Nx * sizeof(float2), s));
    RC(launch_forward_rows(gs.kgrad_tmp, reinterpret_cast<float2*>(grad_kspace[q]), p->rows, p->rowoff, p->maxm,
                           p->Nx, p->Ny, p->Nt, p->Nc, p->fx, s));
  }
  if (grad_lambda || grad_mu) {
    RC(cudaStreamSynchronize(s));
    for (int q = 0; q < n; ++q) {
      recon_plan* p = g->fwd.plans[q];
      double acc[4];
      RC(cudaMemcpy(acc, g->sl[q].acc, sizeof(acc), cudaMemcpyDeviceToHost));
      const double rho = p->opts.rho, mu = p->mu, lam = p->lam;
      const double tau1 = lam * rho / (2.0 * mu);
      if (grad_lambda) grad_lambda[q] = acc[2] * rho / (2.0 * mu);
      if (grad_mu) grad_mu[q] = acc[0] + acc[1] - acc[2] * tau1 / mu;
    }
    int err[2] = {0, 0};
    RC(cudaMemcpy(&err[0], g->fwd.d_err + FLAG_ERR, sizeof(int), cudaMemcpyDeviceToHost));
    RC(cudaMemcpy(&err[1], g->bwd.d_err + FLAG_ERR, sizeof(int), cudaMemcpyDeviceToHost));
    if ((err[0] | err[1]) & DEV_ERR_TIMEOUT) return fail(RECON_ERR_TIMEOUT, "a bounded device-side wait timed out");
  }
  return RECON_OK;
}

recon_status recon_grad_destroy(recon_grad* g) {
  if (!g) return RECON_OK;
  for (recon_plan* p : g->fwd.plans)
    if (p && p->last_stream) cudaStreamSynchronize(p->last_stream);
  cudaDeviceSynchronize();
  delete g;
  return RECON_OK;
}

}  // extern "C"
