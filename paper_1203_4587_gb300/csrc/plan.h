// Internal host-side structures: the plan behind recon_plan*, and the
// engine that launches the ADMM iterations of one plan or of a batch.
#pragma once

#include <string>
#include <vector>

#include "../../include/recon.h"
#include "kernels.h"

namespace recon {

// Device buffers owned by one engine (freed with it).
struct DevArena {
  std::vector<void*> ptrs;
  cudaError_t alloc(void** p, size_t bytes);
  void free(void* p);
  void release();
  ~DevArena() { release(); }
};

// Launch data for the iterations of a set of plans: one descriptor set per
// iteration, built once (the buffers of a plan never move), so iteration k
// only points at set k and a whole solve can be captured as a graph.
struct Engine {
  std::vector<recon_plan*> plans;
  int n = 0;               // number of slices
  int K = 0;               // iterations (the same for every slice)
  bool tv = true;          // prior is TV (the same for every slice)
  recon_prior prior = RECON_PRIOR_TV;
  int levels = 0;          // frame levels of the Haar prior
  bool fused = false;      // objective data term inside the inverse kernel
  bool obj = false;        // objective on
  bool stop_test = false;  // some slice stops on Delta(k) < tol: J(k) is formed every iteration
  int storage = 0;
  // temporal launches: K+1 descriptor sets (k = 1..K, then the final prior term)
  void* d_tmp = nullptr;
  int tmp_blocks = 0, Nt_max = 0, tile_px = 0;
  std::vector<char> tv_full;  // per temporal set: every TV chunk whole (TemporalLaunch::full)
  bool overlap = false;       // every plan asks for programmatic dependent launches (opts.overlap)
  // column-inverse launches: K descriptor sets
  ColSlice* d_col = nullptr;
  unsigned* d_work = nullptr;
  int* d_work_off = nullptr;
  int grid = 0, nb_max = 0, stages = 0, work_max = 0;
  int* d_err = nullptr;    // flags array of the engine's launches (a single plan: its own); errors in [FLAG_ERR]
  FinSlice* d_fin = nullptr;
  // spatio-temporal prior: CG steps, per-block partial sums, per-slice block
  // counters and reduction slots (K sets of 2 cg + 1 per slice)
  int cg = 0;
  bool volume = false;     // the slices are a volume in z order, coupled by w_z D_z
  float wz = 0.f;
  double* d_stv_part = nullptr;
  unsigned* d_stv_count = nullptr;
  std::vector<double*> stv_red;
  // the persistent TV solve (persist_kernels.cu): all K iterations in one launch
  bool persist = false;
  PersistSlice* d_pslice = nullptr;
  unsigned* d_pwork = nullptr;  // per-CTA column lists, image-column-major
  int* d_pwork_off = nullptr;
  int pwork_max = 0, pstages = 0;
  unsigned* d_pcount = nullptr; // colcnt and tdone of every slice (2 sum Nx), queue head and tail; zeroed per solve
  size_t pcount_n = 0;
  int4* d_tq_ring = nullptr;    // temporal task ring (zeroed per solve)
  unsigned tq_cap = 0, tq_total = 0;
  std::vector<unsigned> gens;   // each plan's generation when this engine was built
  DevArena arena;
};

}  // namespace recon

struct recon_plan {
  int Nx = 0, Ny = 0, Nt = 0, Nc = 0;  // Nx: the plan's own columns (a slab's width)
  int Nx_full = 0, i0 = 0;             // the caller's image width and this plan's first column
  recon_prior prior = RECON_PRIOR_TV;
  float lam = 0.f, mu = 0.f;
  recon_opts opts{};
  int device = 0, num_sms = 0;
  cudaStream_t last_stream = nullptr;
  recon::PackInfo pk{};
  int storage = 0;
  size_t esize = 8;
  std::vector<int> h_rows, h_rowoff;
  int maxm = 0, total_rows = 0;
  // device memory
  std::vector<void*> allocs;
  void* A = nullptr;
  float2* sens = nullptr;
  int* rows = nullptr;
  int* rowoff = nullptr;
  short* rowidx = nullptr;             // [Nt][Ny]: position of row j among frame t's sampled rows, -1 if unsampled
  float2 *tw_x = nullptr, *tw_y = nullptr, *tw_t = nullptr;
  recon::dc *twdf_x = nullptr, *twdf_y = nullptr;   // double-float twiddles of the prologue
  recon::dc* yhat_df = nullptr;        // double-float hybrid data of the prologue
  float* thomas = nullptr;
  float2* yhat = nullptr;               // FP32 hybrid data (FP32 storage)
  void* yhat_lp = nullptr;             // 16-bit storage: hybrid data / yscale[t], 16-bit pairs
  unsigned* ymax = nullptr;            // [Nt] largest |component| of the hybrid data (float bits)
  float* yscale = nullptr;             // [Nt] power-of-two frame scales of yhat_lp
  float2* b = nullptr;
  float2* s0[2] = {nullptr, nullptr};  // TV: m;  DFT: u;  Haar: u, [L+1][Nt][Nx][Ny]
  float2* s1[2] = {nullptr, nullptr};  // TV: d1;  Haar: s = Psi'u
  float2* s2[2] = {nullptr, nullptr};  // TV: p
  float2* x = nullptr;                 // TV: x; DFT, Haar: xhat
  float2* r = nullptr;                 // DFT, Haar: r;  STV: CG direction 0
  float2* cgd = nullptr;               // STV: CG direction 1
  float2* tmp_a = nullptr;             // operator entry points
  float2* tmp_b = nullptr;
  float2* kstage = nullptr;            // host-solve staging
  float2* istage = nullptr;
  double* trace_fid = nullptr;
  double* trace_prior = nullptr;
  double* trace_J = nullptr;
  double* yy = nullptr;                // ||y||^2 over the sampled entries (FP64)
  double* res_acc = nullptr;           // [4] sums of the ADMM residuals (TV, DFT, Haar; residual.cu)
  float2* res_prev = nullptr;          // DFT, Haar: xhat_{K-1}, copied before the last inverse step;
                                       // spatio-temporal: m_{K-1}, copied before the last m-update
  float2* res_d1 = nullptr;            // spatio-temporal: d1_{K-1} (4 components), kept by that iteration
  // explicit objective on the tensor cores (16-bit storage; objective_tc.cu)
  int* tc_rows = nullptr;              // [row tiles][64] sampled rows of every (frame, row tile)
  uint2* tc_twiddle = nullptr;         // [Ny] DFT twiddles as FP16 pairs
  int4* tc_items = nullptr;
  int tc_nitems = 0;                   // 0: the FFT kernels form the explicit objective
  float* tc_smax = nullptr;            // [Nx * Nc]
  float* tc_xmax = nullptr;            // [Nt * Nx]
  std::vector<recon::ObjTcParams> tc_par;   // launch parameters for x = this->x and x = this->b
  int* flags = nullptr;
  recon::FftPlanDev fx{}, fy{}, ft{};
  recon::FftPlanDf fxdf{}, fydf{};
  int col_stages = 0;
  int last_iters = 0;
  unsigned generation = 0;             // bumped by recon_plan_set_mu: engines built before refuse to run
  bool broken = false;                 // a recon_plan_set_mu failed half-way: the inverses are not valid
  // tuned launch shapes (0 = the built-in default); see autotune.cu
  int tile_px = 0;                     // temporal kernel pixels per block
  int col_stages_tuned = 0;            // ring depth of the inverse kernel
  int obj_coils = 0;                   // coils per pass of the explicit objective
  int rows_per_block = 0;              // k-space rows per block of the prologue's row FFTs
  int combine_coils = 0;               // coils per pass of the prologue's column FFTs
  recon::Engine* eng = nullptr;        // the plan's own iterations (a batch of one)
  recon::Engine* eng_inv = nullptr;    // recon_apply_inverse (tmp_a -> tmp_b)
  // opts.profile: event pairs around every inverse / temporal launch of a solve
  std::vector<cudaEvent_t> ev_col, ev_tmp;
  cudaEvent_t ev_solve[2] = {nullptr, nullptr};
  int n_col = 0, n_tmp = 0;
  bool prof_valid = false;

  cudaError_t alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  }
  ~recon_plan();
  void mark(std::vector<cudaEvent_t>& v, int& n, bool begin, cudaStream_t s) {
    if (!opts.profile) return;
    const size_t idx = 2 * (size_t)n + (begin ? 0 : 1);
    if (idx < v.size()) cudaEventRecord(v[idx], s);
    if (!begin) ++n;
  }
  size_t npix() const { return (size_t)Nx * Ny; }
  size_t nimg() const { return (size_t)Nx * Ny * Nt; }
};

struct recon_batch {
  recon::Engine eng;
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> key;        // buffers the captured graph reads / writes
  cudaStream_t cap_stream = nullptr;
  bool no_graph = false;               // capture failed once: every call runs the launches directly
  ~recon_batch();
};

namespace recon {

recon_status fail(recon_status st, const std::string& why);
recon_status cuda_fail(cudaError_t e, const char* where);

#define RC(call)                                                \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return recon::cuda_fail(e_, #call);  \
  } while (0)

// engine.cu
void build_col_work(recon_plan* const* plans, int n, int grid, std::vector<unsigned>& work, std::vector<int>& off,
                    int& work_max);
recon_status finish_col_shape(Engine* e, recon_plan* const* plans, int n, int stages_req);
// descriptor set `set` of d_col / d_tmp; pdl: with a programmatic dependency on
// the previous kernel of `s` (TV temporal and inverse kernels only)
recon_status launch_col_set(Engine* e, int set, cudaStream_t s, bool pdl = false);
recon_status launch_tmp_set(Engine* e, int set, cudaStream_t s, bool pdl = false);
cudaError_t plan_create_events(recon_plan* p);   // the profiling events, once
// spatio-temporal prior: the step of iteration set+1 (r, CG, finish)
recon_status launch_stv_step(Engine* e, int set, cudaStream_t s);
recon_status engine_build(Engine* e, recon_plan* const* plans, int n);
recon_status engine_set_tile(Engine* e, int px);   // temporal tile width (rebuilds its descriptor sets)
int engine_tile_candidates(const Engine* e, int* out);   // temporal tile widths that fit
int engine_default_tile(const Engine* e);
recon_status engine_build_inverse(Engine* e, recon_plan* p);   // tmp_a -> tmp_b, no objective
// Resets traces/flags, J(0), K iterations and the final prior term of every
// slice (prologues must have run).  `profile` records the plan's events (n = 1).
// allow_pdl: the plan's own solve may use programmatic dependent launches
// (opts.overlap); batches run in plain stream order
recon_status engine_iterate(Engine* e, cudaStream_t s, bool profile, bool allow_pdl = true);
recon_status engine_apply_inverse(Engine* e, cudaStream_t s);
// RECON_OK while every plan of the engine is usable and unchanged since the build
recon_status engine_check(const Engine* e);
const float2* plan_result(const recon_plan* p);   // image (internal layout) after K iterations
// H'y (into p->b), the hybrid data kept for J(k) and ||y||^2.  kspace is
// complex64 (kstorage 0) or 16-bit pairs times kscale[t] (kscale may be null).
recon_status plan_prologue(recon_plan* p, const void* kspace, int kstorage, const float* kscale, cudaStream_t s);
recon_status plan_to_user(recon_plan* p, const float2* in, float2* out, cudaStream_t s);
recon_status plan_to_internal(recon_plan* p, const float2* in, float2* out, cudaStream_t s);
recon_status plan_adjoint_df(recon_plan* p, const void* kspace, int kstorage, const float* kscale, float2* yhat32,
                            float2* b, double* yy, cudaStream_t s);
recon_status plan_objective(recon_plan* p, const float2* x, double* acc, cudaStream_t s);
recon_status plan_fill_info(recon_plan* p, recon_info* info, cudaStream_t s);
// residual.cu: the sums behind recon_info's primal / dual residuals (TV, DFT, Haar)
recon_status launch_residuals(recon_plan* p, cudaStream_t s);
int objective_coils_max(int Nc, int Ny);   // largest coils-per-pass of the explicit objective

}  // namespace recon
