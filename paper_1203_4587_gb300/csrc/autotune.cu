// Launch-shape autotuner.  For each kernel with a free tile shape it times
// every candidate on the plan's (or batch's) own device buffers with CUDA
// events and keeps the fastest:
//   temporal kernel       pixels per block (TV: 16, DFT: 16..128, Haar: 16..64)
//   column-inverse kernel ring depth (multiples of 8 that fit)
//   prologue row FFTs     k-space rows per block (1, 2, 4, 8)
//   prologue column FFTs  coils per pass of the coil combine (1, 2, 4, 8)
//   explicit objective    coils per pass (1, 2, 4, 8), when the plan uses it
// Results are cached for the process by problem shape, so plans of a shape
// already seen (the slices of a batch, repeated scans) take the cached choice.
// The buffers are filled with a deterministic pattern first; the candidates'
// results are discarded (a solve re-initialises every state it reads).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "plan.h"

namespace recon {

namespace {

__global__ void k_fill_pattern(float2* p, size_t n, unsigned seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    const float a = (float)(h & 0xFFFF) / 32768.f - 1.f, b = (float)(h >> 16) / 32768.f - 1.f;
    p[i] = make_float2(a, b);
  }
}

cudaError_t fill(void* p, size_t n_c64, unsigned seed, cudaStream_t s) {
  if (!p || n_c64 == 0) return cudaSuccess;
  k_fill_pattern<<<(unsigned)std::min<size_t>(1024, (n_c64 + 255) / 256), 256, 0, s>>>(static_cast<float2*>(p), n_c64,
                                                                                      seed);
  note_launch();
  return cudaGetLastError();
}

// Mean time of `reps` launches after one warm-up; best of three rounds.
template <class F>
recon_status time_ms(F&& launch, cudaStream_t s, float* out) {
  cudaEvent_t a = nullptr, b = nullptr;
  RC(cudaEventCreate(&a));
  cudaError_t ce = cudaEventCreate(&b);
  if (ce != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(ce, "cudaEventCreate");
  }
  recon_status st = launch();
  float best = 3.4e38f;
  constexpr int reps = 3;
  for (int round = 0; round < 3 && st == RECON_OK; ++round) {
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == RECON_OK; ++r) st = launch();
    cudaEventRecord(b, s);
    ce = cudaEventSynchronize(b);
    if (ce != cudaSuccess) {
      st = cuda_fail(ce, "cudaEventSynchronize");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms / reps);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *out = best;
  return st;
}

using Key = std::tuple<int, int, int, int, int, int, int, int, int>;   // Nx Nx_full Ny Nt Nc prior storage objective K>0
std::mutex g_mu;
std::map<Key, recon_tuning> g_cache;

Key key_of(const recon_plan* p) {
  const int objmode = (p->opts.objective != 0 || p->opts.tol > 0.0) ? (p->opts.objective == 2 ? 2 : 1) : 0;
  return Key{p->Nx, p->Nx_full, p->Ny, p->Nt, p->Nc, (int)p->prior, p->storage, objmode, p->opts.max_iters > 0 ? 1 : 0};
}

// Candidate ring depths: multiples of the quantum up to the largest that fits.
std::vector<int> stage_candidates(const Engine* e) {
  const int q = col_inverse_stage_quantum(e->storage ? 4 : 8);
  const int mx = col_inverse_max_stages(e->nb_max, e->n, e->work_max, e->storage ? 4 : 8);
  std::vector<int> out;
  for (int st = q; st <= mx; st += q) out.push_back(st);
  if (out.empty()) out.push_back(q);
  return out;
}

// Fills every state buffer of a plan (and zeroes its flags and traces).
recon_status prepare_buffers(recon_plan* p, cudaStream_t s) {
  const size_t N = p->nimg();
  RC(fill(p->b, N, 1u, s));
  for (int k = 0; k < 2; ++k) {
    RC(fill(p->s0[k], N, 2u + k, s));
    RC(fill(p->s1[k], N, 4u + k, s));
    RC(fill(p->s2[k], N, 6u + k, s));
  }
  RC(fill(p->x, N, 8u, s));
  RC(fill(p->r, N, 9u, s));
  const size_t ny = (size_t)p->total_rows * p->Nx * p->Nc;
  if (p->yhat) RC(fill(p->yhat, ny, 10u, s));
  if (p->yhat_lp) RC(cudaMemsetAsync(p->yhat_lp, 0, ny * 4, s));
  if (p->yscale) {
    std::vector<float> one(p->Nt, 1.f);
    RC(cudaMemcpyAsync(p->yscale, one.data(), p->Nt * sizeof(float), cudaMemcpyHostToDevice, s));
    RC(cudaStreamSynchronize(s));
  }
  const size_t nt = (size_t)p->opts.max_iters + 2;
  RC(cudaMemsetAsync(p->flags, 0, FLAG_COUNT * sizeof(int), s));
  RC(cudaMemsetAsync(p->trace_fid, 0, nt * sizeof(double), s));
  RC(cudaMemsetAsync(p->trace_prior, 0, nt * sizeof(double), s));
  return RECON_OK;
}

// Temporal tile width and ring depth of an engine (the plan's own, or a batch's).
recon_status tune_engine(Engine* e, cudaStream_t s, recon_tuning* t) {
  if (e->K < 1) return RECON_OK;
  int cand[4];
  const int nc = engine_tile_candidates(e, cand);
  int best_px = e->tile_px;
  float best = 3.4e38f;
  for (int i = 0; i < nc; ++i) {
    recon_status st = engine_set_tile(e, cand[i]);
    if (st != RECON_OK) return st;
    float ms = 0.f;
    // the spatio-temporal prior times its whole step (r, the CG launches, finish)
    if ((st = time_ms([&] { return e->prior == RECON_PRIOR_STV ? launch_stv_step(e, 0, s) : launch_tmp_set(e, 0, s); },
                      s, &ms)) != RECON_OK)
      return st;
    if (ms < best) { best = ms; best_px = cand[i]; }
  }
  recon_status st = engine_set_tile(e, best_px);
  if (st != RECON_OK) return st;
  t->temporal_tile_px = best_px;
  t->temporal_ms = best;
  int best_st = e->stages;
  best = 3.4e38f;
  for (int c : stage_candidates(e)) {
    if ((st = finish_col_shape(e, e->plans.data(), e->n, c)) != RECON_OK) return st;
    float ms = 0.f;
    if ((st = time_ms([&] { return launch_col_set(e, 0, s); }, s, &ms)) != RECON_OK) return st;
    if (ms < best) { best = ms; best_st = e->stages; }
  }
  if ((st = finish_col_shape(e, e->plans.data(), e->n, best_st)) != RECON_OK) return st;
  t->col_stages = best_st;
  t->col_ms = best;
  return RECON_OK;
}

// The prologue's row-FFT and coil-combine shapes and the explicit objective's
// coils per pass of one plan (its buffers already filled by prepare_buffers).
recon_status tune_prologue(recon_plan* p, cudaStream_t s, recon_tuning* t) {
  recon_status st;
  // prologue: a patterned complex64 k-space
  const size_t nk = (size_t)p->Nt * p->Nc * p->Ny * p->Nx_full;
  void* k = nullptr;
  RC(cudaMalloc(&k, nk * sizeof(float2)));
  struct Free { void* q; ~Free() { cudaFree(q); } } guard{k};
  RC(fill(k, nk, 11u, s));
  const bool wide = p->storage == 0;   // FP32 storage: the double-float prologue
  float best = 3.4e38f;
  int best_g = 0;
  for (int g : {1, 2, 4, 8}) {
    if (g > row_group_max(p->Nx_full, wide)) break;
    p->rows_per_block = g;
    float ms = 0.f;
    auto run = [&]() -> recon_status {
      if (wide) {
        RC(launch_hybrid_rows_df(k, 0, nullptr, p->yhat_df, p->yhat, nullptr, p->rows, p->rowoff, p->maxm,
                                 p->Nx_full, p->Ny, p->Nt, p->Nc, p->fxdf, g, s, p->i0, p->Nx));
      } else {
        RC(launch_hybrid_rows(k, 0, nullptr, p->tmp_b, nullptr, p->ymax, p->rows, p->rowoff, p->maxm, p->Nx_full,
                              p->Ny, p->Nt, p->Nc, p->fx, g, s, p->i0, p->Nx));
      }
      return RECON_OK;
    };
    if ((st = time_ms(run, s, &ms)) != RECON_OK) return st;
    if (ms < best) { best = ms; best_g = g; }
  }
  p->rows_per_block = t->rows_per_block = best_g;
  t->rows_ms = best;
  best = 3.4e38f;
  int best_c = 0;
  for (int c : {1, 2, 4, 8}) {
    if (c > std::max(1, std::min(p->Nc, coil_group_max(p->Nc, p->Ny, wide)))) break;
    float ms = 0.f;
    auto run = [&]() -> recon_status {
      if (wide) {
        RC(launch_adjoint_combine_df(p->yhat_df, p->sens, p->tmp_a, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc,
                                     p->fydf, c, s));
      } else {
        RC(launch_adjoint_combine(p->tmp_b, p->sens, p->tmp_a, p->rows, p->rowoff, p->Nx, p->Ny, p->Nt, p->Nc, p->fy,
                                  p->storage, p->yhat_lp, p->ymax, p->yscale, c, s));
      }
      return RECON_OK;
    };
    if ((st = time_ms(run, s, &ms)) != RECON_OK) return st;
    if (ms < best) { best = ms; best_c = c; }
  }
  p->combine_coils = t->combine_coils = best_c;
  t->combine_ms = best;
  // explicit objective (16-bit storage or objective mode 2)
  const bool objective_on = p->opts.objective != 0 || p->opts.tol > 0.0;
  const bool exact = objective_on && (p->opts.objective == 2 || p->storage != 0);
  t->objective_coils = 0;
  t->objective_ms = 0.f;
  if (exact && p->tc_nitems > 0) {   // the tensor-core form: no coil passes to choose
    float ms = 0.f;
    if ((st = time_ms([&] { return plan_objective(p, p->x, p->trace_fid, s); }, s, &ms)) != RECON_OK) return st;
    p->obj_coils = t->objective_coils = 1;
    t->objective_ms = ms;
  } else if (exact) {
    best = 3.4e38f;
    int best_o = 0;
    for (int c : {1, 2, 4, 8}) {
      if (c > objective_coils_max(p->Nc, p->Ny)) break;
      p->obj_coils = c;
      float ms = 0.f;
      if ((st = time_ms([&] { return plan_objective(p, p->x, p->trace_fid, s); }, s, &ms)) != RECON_OK) return st;
      if (ms < best) { best = ms; best_o = c; }
    }
    p->obj_coils = t->objective_coils = best_o;
    t->objective_ms = best;
  }
  return RECON_OK;
}

recon_status tune_plan(recon_plan* p, cudaStream_t s, recon_tuning* t) {
  recon_status st = prepare_buffers(p, s);
  if (st != RECON_OK) return st;
  if ((st = tune_prologue(p, s, t)) != RECON_OK) return st;
  // iteration kernels on the plan's own engine
  if ((st = tune_engine(p->eng, s, t)) != RECON_OK) return st;
  p->tile_px = t->temporal_tile_px;
  p->col_stages_tuned = t->col_stages;
  RC(cudaStreamSynchronize(s));
  return RECON_OK;
}

}  // namespace

}  // namespace recon

using namespace recon;

extern "C" {

recon_status recon_autotune(recon_plan* p, recon_tuning* out, void* stream) {
  if (!p) return fail(RECON_ERR_INVALID_ARG, "NULL plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_tuning t{};
  const Key key = key_of(p);
  bool hit = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      t = it->second;
      hit = true;
    }
  }
  if (hit) {
    p->rows_per_block = t.rows_per_block;
    p->combine_coils = t.combine_coils;
    p->obj_coils = t.objective_coils;
    p->tile_px = t.temporal_tile_px;
    p->col_stages_tuned = t.col_stages;
    if (p->opts.max_iters > 0) {
      recon_status st = engine_set_tile(p->eng, t.temporal_tile_px);
      if (st == RECON_OK) st = finish_col_shape(p->eng, &p, 1, t.col_stages);
      if (st != RECON_OK) return st;
    }
    t.from_cache = 1;
  } else {
    recon_status st = tune_plan(p, s, &t);
    if (st != RECON_OK) return st;
    t.from_cache = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = t;
  }
  if (out) *out = t;
  return RECON_OK;
}

recon_status recon_batch_autotune(recon_batch* b, recon_tuning* out, void* stream) {
  if (!b) return fail(RECON_ERR_INVALID_ARG, "NULL batch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  recon_status st;
  for (recon_plan* p : b->eng.plans)
    if ((st = prepare_buffers(p, s)) != RECON_OK) return st;
  if (b->eng.n > 1) RC(cudaMemsetAsync(b->eng.d_err, 0, FLAG_COUNT * sizeof(int), s));
  recon_tuning t{};
  // each slice's prologue shapes, once per problem shape (the plan cache's
  // entry when the plan was tuned on its own, else the batch's own); the
  // batch reports the largest slice's choice and the sum of the slices' times
  {
    std::map<Key, recon_tuning> seen;
    size_t largest = 0;
    float rows_ms = 0.f, combine_ms = 0.f, objective_ms = 0.f;
    for (recon_plan* p : b->eng.plans) {
      const Key key = key_of(p);
      recon_tuning pt{};
      bool hit = false;
      {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) { pt = it->second; hit = true; }
      }
      if (!hit) {
        auto it = seen.find(key);
        if (it != seen.end()) { pt = it->second; hit = true; }
      }
      if (hit) {
        p->rows_per_block = pt.rows_per_block;
        p->combine_coils = pt.combine_coils;
        p->obj_coils = pt.objective_coils;
      } else {
        if ((st = tune_prologue(p, s, &pt)) != RECON_OK) return st;
        seen[key] = pt;
      }
      rows_ms += pt.rows_ms;
      combine_ms += pt.combine_ms;
      objective_ms += pt.objective_ms;
      const size_t size = (size_t)p->Nt * p->Nc * p->Ny * p->Nx_full;
      if (size > largest) {
        largest = size;
        t.rows_per_block = p->rows_per_block;
        t.combine_coils = p->combine_coils;
        t.objective_coils = p->obj_coils;
      }
    }
    t.rows_ms = rows_ms;
    t.combine_ms = combine_ms;
    t.objective_ms = objective_ms;
  }
  if ((st = tune_engine(&b->eng, s, &t)) != RECON_OK) return st;
  RC(cudaStreamSynchronize(s));
  if (b->graph) {   // the captured launches used the old shapes
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->key.clear();
  }
  if (out) *out = t;
  return RECON_OK;
}

}  // extern "C"
