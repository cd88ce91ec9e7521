// Internal launch interfaces between the C-ABI layer (api.cu) and the kernels.
//
// Internal layouts (device):
//   image fields   [Nt][Nx][Ny]  column-stacked per frame (Eq. x_def: the
//                  vertical index j is fastest, so column x_{v,i,t} is
//                  contiguous)
//   sensitivities  [Nx][Nc][Ny]
//   hybrid data    yhat = F_h' y on sampled rows: frame t starts at
//                  rowoff[t]*Nx*Nc, then [Nx][Nc][m_t]
//   inverses       one packed stream of `col_elems` elements per column
//                  (i,t), stored image-column-major at i*Nt + t (see packing
//                  below); work lists and the other fields use col = t*Nx + i
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <cuda.h>   // CUtensorMap (type only; no driver library is linked)
#include <cuda_runtime.h>

#include "fft.cuh"

namespace recon {

// ---- packed Hermitian storage of A_{i,t} = (mu I + G_{i,t})^{-1} -------------
// Ny is padded to Nyp = 32*nb.  The upper triangle is cut into 32x32 blocks,
// and every block is read by one warp whose lane (lr, lc) = (lane/4, lane%4)
// owns rows 4lr..4lr+3 and columns 8lc..8lc+7 of it.  Units, in stream order:
//   * every off-diagonal block (bj < bk), bk-major: 1024 elements.  The pair
//     (R, C), (R, C+1), C even, sits at complex position
//     ((R%4)*4 + (C%8)/2)*64 + ((R/4)*4 + C/8)*2 and is stored planar,
//     components (re_C, re_C+1, im_C, im_C+1), so one 16-byte (8-byte at
//     16 bit) load gives a lane a real pair and an imaginary pair for packed
//     FP32x2 arithmetic.
//   * every diagonal block: 640 elements, the same planar pairs for the 20
//     lanes whose 4x8 patch meets the upper triangle (lr <= 2lc+1), at
//     ((R%4)*4 + (C%8)/2)*40 + (lc*(lc+1) + lr)*2.  Entries below the
//     diagonal inside those patches are zero, and the diagonal is stored
//     halved: every stored element e at (R, C) then adds e r_C to y_R and
//     conj(e) r_R to y_C, the off-diagonal rule, and the two halves of the
//     (real) diagonal make A_RR r_R.
// The diagonal blocks carry 112 padding elements each over the triangle.
enum UnitKind : int { UNIT_TILE = 0, UNIT_DIAG = 1 };
constexpr int kTileElems = 1024;
constexpr int kDiagElems = 640;
constexpr int kDiagLanes = 20;   // lanes of a diagonal block with stored elements

// Position of column col = t * Nx + i in the packed stream: image-column-major,
// so the columns a launch takes in turn (work lists run through the image
// columns, every frame of one after the other) are adjacent in memory.
__host__ __device__ inline long long packed_index(int col, int Nx, int Nt) {
  const int t = col / Nx, i = col - t * Nx;
  return (long long)i * Nt + t;
}

struct PackInfo {
  int nb;          // 32-blocks per column
  int nunits;
  int ntiles;      // off-diagonal blocks
  long long col_elems;
};

// ---- FFT plan (host side holds the device twiddle table) -------------------
FftPlanDev make_fft_plan_host(int n, const float2* d_tw);  // factorisation only
FftPlanDf make_fft_plan_host_df(int n, const dc* d_tw);
void fill_twiddles_host(int n, float2* host_tw);           // exp(-2 pi i k/n)
void fill_twiddles_host_df(int n, float4* host_tw);   // exp(-2 pi i k/n) as double-float pairs

// ---- kernel parameter blocks ----------------------------------------------
// The per-iteration kernels take arrays of per-problem ("slice") descriptors:
// a single reconstruction is a batch of one, and a batch of uneven slices
// runs in one launch per step.  The host builds one descriptor set per
// iteration once (the buffers a slice uses never move), so an iteration's
// launches only point at set k and a whole solve can be captured as a graph.

struct ColSlice {            // data-consistency inverse x = A r of one slice
  const void* A;             // packed stream base (column (i, t) at i*Nt + t)
  long long col_elems;
  int Nx, Nt;                // for the stream index of col = t*Nx + i
  int Ny, nb;
  int nunits;                // units per column (decoded from the index and nb)
  int r_tma;                 // 1: r inputs move by bulk copy (Ny*8 a multiple of 16)
  int do_obj;
  const float2* base;        // r = base + coef * add   ([Nt][Nx][Ny])
  const float2* add;         // may be null
  const float2* bsrc;        // H'y for the objective term (may equal base)
  float2* xout;
  float coef;
  float mu;
  // dot products of the new x accumulated into *fid_acc:
  //   w_bx Re<bsrc, x> + w_xr Re<x, r> + w_xx ||x||^2
  // The data term of J uses w = (-2, 1, -mu), since with (mu I + H'H) x = r
  //   ||y - Hx||^2 = ||y||^2 - 2 Re<H'y, x> + Re<x, r> - mu ||x||^2
  // (||y||^2 comes from the prologue); the adjoint pass uses w_bx = -1 for
  // the dA/dmu term of the mu gradient.
  float w_bx, w_xr, w_xx;
  double* fid_acc;
  const int* stop;           // the slice's stop flag: its columns are skipped when set
};

struct ColLaunch {
  const ColSlice* slices;
  int nslices;
  const unsigned* work;      // (slice << 24) | column, in processing order
  const int* work_off;       // [gridDim.x + 1]: CTA b processes work[work_off[b] .. work_off[b+1])
  int work_max;              // longest per-CTA list (staged in shared memory)
  int nb_max;                // largest block count of any slice (shared-memory sizing)
  int stages;                // ring depth (a multiple of the consumer warp count)
  int* err;                  // flags array of the launch: bounded waits report in err[FLAG_ERR]
};

struct TvSlice {             // temporal step of Algorithm 2 (R = D_t) of one slice
  int Nt;
  long long npix;            // Nx*Ny
  const float2* m;           // [Nt][npix]
  const float2* d1;          // [Nt-1][npix] or null (zeros)
  const float2* x;
  const float2* p;           // p = m_prev - d2_prev, so d2 = x - p
  float2* m_out;
  float2* d1_out;
  float2* p_out;
  float tau1;                // lambda / (2 mu1)
  float rho;                 // mu2 / mu1
  const float* thomas;       // [Nt] pivots of (rho I + D'D)
  int write_state;           // 0: only the prior term
  double* prior_acc;         // += ||D_t x||_1
  const int* stop;
  int tile0;                 // first block of this slice in the launch
};

struct DftSlice {            // temporal step of Algorithm 1 (Psi = temporal DFT) of one slice
  int Nt;
  long long npix;
  const float2* xh;          // xhat = A r of the previous iteration (b at k=1)
  const float2* u;           // u = v + d of the previous iteration
  const float2* b;
  float2* u_out;
  float2* r_out;             // r = b + mu Psi'(v + d)
  float tau;                 // lambda / (2 mu)
  float mu;
  int first;                 // k == 1: d = 0
  int write_state;
  FftPlanDev ft;
  double* prior_acc;         // += ||w||_1
  const int* stop;
  int tile0;
};

struct HaarSlice {           // temporal step of Algorithm 1 with the undecimated Haar frame, one slice
  int Nt;
  long long npix;
  int levels;                // L; L + 1 coefficient channels
  const float2* xh;          // xhat = A r of the previous iteration (b at k = 1)
  const float2* u;           // u = v + d of the previous iteration, [L+1][Nt][npix] (unused at k = 1)
  const float2* s;           // Psi'u of the previous iteration (unused at k = 1)
  const float2* b;
  float2* u_out;
  float2* s_out;             // Psi'u
  float2* r_out;             // r = b + mu Psi'u
  float tau;                 // lambda / (2 mu)
  float mu;
  int first;                 // k == 1: w = Psi b, d = 0
  int write_state;           // 0: only ||w||_1 of the final w
  double* prior_acc;         // += ||w||_1
  const int* stop;
  int tile0;
};

// Algorithm 2 with R = (D_t, w D_x, w D_y) (spatio-temporal differences) and a
// CG m-update, one slice.  Fields [Nt][Nx][Ny] (n elements); the difference
// components of e = d1 - v are stored padded, [4][n] (t, x, y, z), with zeros
// where a difference leaves the grid.  Reduction slots of one iteration:
// red[0..cg] = gamma_0..gamma_cg (<r, r>), red[cg+1+j] = <p_j, q_j>.
// In a volume (slices stacked along z, coupled by w_z D_z) the slices of a
// launch are in z order, the neighbours of slice q are descriptors q-1 and
// q+1, and every slice shares one reduction range, counter and slot array.
struct StvSlice {
  int Nx, Ny, Nt;
  int n;                     // Nt*Nx*Ny
  int cg;                    // CG steps per iteration
  float tau1;                // lambda / (2 mu1)
  float rho;                 // mu2 / mu1
  float ws;                  // spatial weight w
  float wz;                  // z weight w_z (volumes; 0 otherwise)
  int zprev, znext;          // 1 when the slice has a neighbour below / above in z
  float2* m;                 // m (updated in place by the CG steps)
  float2* e;                 // [4][n]: d1 - v
  float2* p;                 // p = m - d2 (so d2 = x - p); the inverse step reads r = b + mu2 p
  const float2* x;
  float2* r;                 // CG residual
  float2* pc[2];             // CG directions (alternating)
  float2* q;                 // M p
  double* red;               // this iteration's reduction slots
  double* part;              // per-block partial sums (indexed by the launch's block)
  unsigned* count;           // blocks done, for the last-block sum (reset by that block)
  int red0, rednblk;         // the blocks whose partials make one sum (the slice, or the volume)
  double* prior_acc;         // += ||R x||_1 of the incoming x
  const int* stop;
  int tile0;                 // first block of this slice in the launch
  int nblk;                  // blocks of this slice (rows image columns each)
  int rows;                  // image columns (t, i) per block, at most kStvRows
  // ADMM residuals of a solve of K iterations (k_stv_finish of iterations
  // K-1 and K, k_stv_residuals after the loop):
  float2* d1_keep;           // iteration K-1: d1 (every component) stored here
  const float2* d1_ref;      // iteration K: d1_{K-1} (null: d1_0 = 0) ...
  int res_last;              // ... and res_acc[1] += ||d1_{K-1} - d1_K||^2 when 1
  double* res_acc;           // [4] sums (the first slice's for a volume)
  const float2* m_prev;      // final set: m_{K-1}, copied before the last m-update
};

struct StvLaunch {
  const StvSlice* slices;
  int nslices;
  int nblocks;
  int step;                  // CG step j of the direction / update kernels
  int dir_threads;           // direction kernel: one thread per j, Ny_max rounded up to 32
};

// Temporal TV kernel shape (tv_chunk.cuh): chunks of kTvChunkPx pixels, the
// t-axis cut into kTvSeg segments; whole chunks with up to kTvFullLMax frames
// a segment take the specialised instantiation.
constexpr int kTvSeg = 8;
constexpr int kTvChunkPx = 16;
constexpr int kTvFullLMax = 6;

struct TemporalLaunch {      // one launch over the tiles of several slices
  const void* slices;        // TvSlice[], DftSlice[] or HaarSlice[]
  int nslices;
  int nblocks;
  int Nt_max;                // shared-memory sizing
  int tile_px;               // pixels per block (TV)
  int full;                  // TV: every slice has Nt == 8 * ceil(Nt_max / 8) <= 48, Nx*Ny a
                             // multiple of 16, d1 present and state written (whole chunks)
};

struct TvBwdSlice {          // reverse of one Algorithm 2 step (see grad.cu), one slice
  int Nt;
  long long npix;
  // adjoints of the step's outputs (x', m', d1', d2') and r_bar = A (x_bar' + d2_bar')
  const float2* xb;
  const float2* mb;
  const float2* d1b;         // null at the last step (zero)
  const float2* d2b;
  const float2* rb;
  // forward state of the step's input (x, m, d1, p with d2 = x - p) and m'
  const float2* x0;
  const float2* m0;
  const float2* d10;         // null at the first step
  const float2* p0;
  const float2* m1;
  // adjoints of the step's inputs
  float2* xb_out;
  float2* mb_out;
  float2* d1b_out;
  float2* d2b_out;
  float2* bbar;              // += r_bar (and x_bar + m_bar of the initial state when `first`)
  float tau1, rho, mu;
  const float* thomas;
  int first;                 // step 1: its input state is x = m = H'y
  double* mu_acc;            // += Re<r_bar, m' - d2>
  double* tau_acc;           // += dL/dtau1
  int tile0;
};

struct FinSlice {            // J(k), Delta(k) and the stop flag of one slice
  const double* fid;
  const double* prior;
  const double* yy;          // ||y||^2 (fused objective) or null
  double* J;
  int* flags;
  float lam;
  double tol;
};

struct ObjParams {           // ||y - H x||^2 of a given field (no inverse)
  int Nx, Ny, Nt, Nc, ncg;
  const float2* x;           // [Nt][Nx][Ny]
  const float2* sens;
  const void* yhat;          // hybrid data: complex64, or 16-bit pairs times yscale[t]
  int ystorage;              // recon_storage of yhat
  const float* yscale;       // [Nt] (16-bit yhat only)
  const int* rows;
  const int* rowoff;
  const short* rowidx;       // [Nt][Ny]: index of row j among frame t's sampled rows, or -1
  FftPlanDev fy;
  double* fid_acc;
  const int* flags;
  int grid;                  // blocks of the warp-per-(column, coil) kernel
};

// ||y - H x||^2 on the tensor cores (objective_tc.cu): per (frame, tile of 64
// sampled rows, tile of 256 columns (i, c)) item, D = A B' with A the frame's
// sampled DFT rows (formed in the kernel from a twiddle table) and B = s_c . x,
// both split into FP16 pairs.
struct ObjTcParams {        // 64-byte aligned by its tensor maps
  CUtensorMap smap;          // s as [Nx * Nc][2 Ny] floats, box 256 x 32, 128-byte swizzle
  CUtensorMap xmap;          // x as [Nt][Nx][2 Ny] floats, box 1 x ni x 32, 128-byte swizzle
  int Nx, Ny, Nt, Nc;
  int nk;                    // K chunks of 16 values of j: ceil(Ny / 16)
  int ni;                    // image columns in an x tile (a column tile of 256 (i, c) spans at most ni)
  int raw_depth;             // raw tile stages (2 or 3)
  int op_stages;             // operand (A and B) stages (2 or 3)
  int raw_bytes;             // bytes of a raw stage: the s tile, then the x tile (1024-byte multiple)
  const float2* x;           // [Nt][Nx][Ny]: the image xmap describes
  const float* smax;         // [Nx * Nc]: max_j |s_{i,c}[j]| (rounded up)
  float* xmax;               // [Nt * Nx]: max_j |x_t[i][j]| (rounded up), formed before each launch
  const void* yhat;          // hybrid data as in ObjParams
  int ystorage;
  const float* yscale;
  const int* rowoff;
  const int* tile_rows;      // [row tiles][64]: sampled row q of each (frame, row tile); -1 past its rows
  const uint2* twiddle;      // [Ny]: objective_tc_twiddle
  const int4* items;         // (t, row tile, column tile, row tile index into tile_rows)
  int nitems;
  int grid;                  // CTAs (one per SM)
  double* fid_acc;
  const int* flags;          // FLAG_STOP read
  int* err;                  // flags base: errors in [FLAG_ERR]
};
void objective_tc_twiddle(int Ny, uint2* out);   // host: [Ny] FP16-pair twiddles of the scaled DFT
// Fills the tensor maps, ni and the raw stages of q for image x and
// sensitivities sens (q.Nx, q.Ny, q.Nt, q.Nc set); false where the tiles do
// not fit in shared memory or the driver rejects a map.
bool objective_tc_prepare(ObjTcParams& q, const float2* x, const float2* sens);
cudaError_t launch_objective_tc(const ObjTcParams& p, cudaStream_t s);
cudaError_t launch_col_absmax(const float2* s, int ncols, int Ny, float* out, cudaStream_t st);

// Persistent solve of Algorithm 2 with temporal TV (persist_kernels.cu): all
// K iterations of a set of slices in one cooperative launch, FP32 inverses,
// Nt <= kPersistNtMax, Nx < 2^20.  The per-column counters colcnt and tdone ([Nx] per
// slice), the queue counters and the ring's tags must be zero at the launch.
constexpr int kPersistNtMax = 40;
constexpr int kPersistChunkPx = 16;   // pixels of an image column per temporal task
struct PersistSlice {
  const void* A;             // packed inverses
  long long col_elems;
  int Nx, Ny, Nt, nb, nunits;
  const float2* b;           // H'y   [Nt][Nx][Ny]
  float2* x;                 // x
  float2* m[2];              // state by iteration parity
  float2* d1[2];
  float2* p[2];
  float mu, tau1, rho;
  const float* thomas;       // [Nt] pivots of (rho I + D'D)
  float w_bx, w_xr, w_xx;    // objective weights (see ColSlice)
  int do_obj;
  double* trace_fid;         // [K + 2]
  double* trace_prior;
  int nch;                   // temporal chunks per image column (ceil(Ny / 16))
  unsigned* colcnt;          // [Nx] completed frames of the current iteration
  unsigned* tdone;           // [Nx] temporal chunks done in this launch
};

struct PersistLaunch {
  const PersistSlice* slices;
  int nslices;
  const unsigned* work;      // (slice << 24) | (t * Nx + i), image-column-major per CTA (build_col_work)
  const int* work_off;
  int work_max;
  int nb_max;
  int stages;
  int K;
  int* err;
  // the global queue of temporal tasks T_{k+1}(q, i): entry (q, i, k, tag),
  // tag = ticket + 1 once written, 0 when free; cap a power of two
  int4* tq_ring;
  unsigned tq_cap;
  unsigned* tq_head;         // tickets taken by the temporal warps
  unsigned* tq_tail;         // tasks produced
  unsigned tq_total;         // tasks one launch produces: K * sum over slices of Nx * nch
};

size_t persist_smem(int stages, int nb_max, int nslices, int work_max);
int persist_max_stages(int nb_max, int nslices, int work_max);   // 0: does not fit
cudaError_t launch_persist_tv(const PersistLaunch& p, int grid, cudaStream_t s);

// The dynamic shared-memory limit of a kernel is a per-device attribute.  A
// launcher keeps, per device ordinal, the largest limit it has set, and raises
// it on the current device when a launch needs more (a plan on any device of
// the process works; the first launch on a device sets its attribute).
constexpr int kMaxDevices = 64;
struct SmemAttrCache {
  std::atomic<size_t> v[kMaxDevices] = {};
  cudaError_t ensure(const void* kernel, size_t bytes);
};

// Counts kernel launches of this library (process-wide); every launcher calls it.
void note_launch();
// Sets the message recon_last_error() returns on the calling thread.
void set_last_error(const std::string& why);

// ---- launchers (return cudaGetLastError()) ---------------------------------
// pdl: launch with a programmatic dependency on the previous kernel of `s`
// (the kernel waits for it in-device; see pdl_wait in common.cuh)
cudaError_t launch_col_inverse(const ColLaunch& p, int storage, int grid, cudaStream_t s, bool pdl = false);
// esize: bytes per stored element (8 FP32, 4 FP16/BF16)
size_t col_inverse_smem(int stages, int nb_max, int nslices, int work_max, int esize);
int col_inverse_max_stages(int nb_max, int nslices, int work_max, int esize);
int col_inverse_stage_quantum(int esize);  // ring depth must be a positive multiple of this
cudaError_t prepare_tv_temporal(int Nt_max, int px);   // shared-memory attribute, outside any capture
cudaError_t prepare_dft_temporal(int Nt_max, int px);
cudaError_t prepare_col_inverse(int storage, size_t smem);
int tv_tile_px(int Nt_max);                         // default pixels per block
int dft_tile_px();
int tv_tile_candidates(int Nt_max, int* out);       // tile widths that fit (<= 4 entries)
int dft_tile_candidates(int Nt_max, int* out);
cudaError_t launch_tv_temporal(const TemporalLaunch& p, cudaStream_t s, bool pdl = false);
cudaError_t launch_dft_temporal(const TemporalLaunch& p, cudaStream_t s, bool pdl = false);
cudaError_t launch_haar_temporal(const TemporalLaunch& p, int levels, cudaStream_t s, bool pdl = false);
cudaError_t prepare_haar_temporal(int Nt_max, int levels, int px);
int haar_tile_px(int Nt_max, int levels);
int haar_tile_candidates(int Nt_max, int levels, int* out);
cudaError_t launch_objective(const ObjParams& p, cudaStream_t s);
// spatio-temporal Algorithm 2 (stv_kernels.cu): a block walks StvSlice::rows
// image columns (t, i) of Ny elements, one of kStvRowCands (picked by the
// autotuner; kStvRows by default)
constexpr int kStvThreads = 256;
constexpr int kStvDirMaxThreads = 1024;   // the direction kernel's block: Ny <= 1023
constexpr int kStvRows = 16;
constexpr int kStvRowsMin = 4;
constexpr int kStvRowCands[] = {4, 8, 16};
cudaError_t launch_stv_init(const StvLaunch& L, cudaStream_t s);     // e = -S(R m) (d1 = 0)
cudaError_t launch_stv_prior(const StvLaunch& L, cudaStream_t s);    // ||R x||_1
cudaError_t launch_stv_rhs(const StvLaunch& L, cudaStream_t s);      // r = rhs - M m, gamma_0, ||R x||_1
cudaError_t launch_stv_dir(const StvLaunch& L, cudaStream_t s);      // p_j, q = M p_j, <p_j, q>
cudaError_t launch_stv_update(const StvLaunch& L, cudaStream_t s);   // m, r, gamma_{j+1}
cudaError_t launch_stv_finish(const StvLaunch& L, cudaStream_t s);   // d1 = e + R m, p, next e
// with the final descriptor set: res_acc[0] += ||m_K - x_K||^2, [2] += ||dm||^2,
// [3] += ||R dm||^2 (dm = m_K - m_{K-1})
cudaError_t launch_stv_residuals(const StvLaunch& L, cudaStream_t s);
// per slice, for k = k0 .. k1: J(k) = fid[k] + (yy ? *yy : 0) + lambda prior[k]; Delta(k); stop flag.
cudaError_t launch_finalize(const FinSlice* fins, int nslices, int k0, int k1, cudaStream_t s);

// prologue / operators
// yhat = F_h' y (FP32 butterflies), k-space complex64 or 16-bit pairs
// (kstorage = recon_storage) times kscale[t] (may be null); ymax[t] receives
// the largest |component| of frame t's yhat (float bits, may be null).
// G (rows per block) and ncg (coils per pass) below: 0 = the largest that fits.
// Nx is the full row length of the k-space (and the FFT length); i0, W keep
// columns i0 .. i0+W-1 of the result (a slab plan), W = 0 keeps all.
cudaError_t launch_hybrid_rows(const void* kspace, int kstorage, const float* kscale, float2* yhat, double* yy,
                               unsigned* ymax, const int* rows, const int* rowoff, int maxm, int Nx, int Ny, int Nt,
                               int Nc, FftPlanDev fx, int G, cudaStream_t s, int i0 = 0, int W = 0);
// b = H'y from yhat (FP32); ystorage 1/2 also writes the 16-bit copy ylp of
// yhat with per-frame power-of-two scales yscale[t] from ymax.
cudaError_t launch_adjoint_combine(const float2* yhat, const float2* sens, float2* b, const int* rows,
                                   const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDev fy, int ystorage,
                                   void* ylp, const unsigned* ymax, float* yscale, int ncg, cudaStream_t s);
// Double-float H'y prologue: the solution of the iterations is ~100x more
// sensitive to errors in H'y than to rounding elsewhere, so H'y is formed in
// double-float arithmetic (about 48 bits, on the FP32 pipe) and rounded once.
// yhat32 receives the FP32 rounding of the hybrid data; *yy accumulates
// ||y||^2 over the sampled entries (may be null).
cudaError_t launch_hybrid_rows_df(const void* kspace, int kstorage, const float* kscale, dc* yhat_df,
                                  float2* yhat32, double* yy, const int* rows, const int* rowoff, int maxm, int Nx,
                                  int Ny, int Nt, int Nc, FftPlanDf fx, int G, cudaStream_t s, int i0 = 0,
                                  int W = 0);
cudaError_t launch_adjoint_combine_df(const dc* yhat_df, const float2* sens, float2* b, const int* rows,
                                      const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDf fy, int ncg,
                                      cudaStream_t s);
int row_group_max(int Nx, bool wide);              // largest rows-per-block of the row FFTs (wide: double-float)
int coil_group_max(int Nc, int Ny, bool wide);     // largest coils-per-pass of the combine
// 16-bit k-space (storage 1 = FP16, 2 = BF16 pairs) with per-frame
// power-of-two scales: out = k / frame_scale[t], one rounding.
cudaError_t launch_quantize_kspace(const float2* k, long long per_frame, int Nt, int storage, void* out,
                                  float* frame_scale, cudaStream_t s);
cudaError_t launch_forward_cols(const float2* x, const float2* sens, float2* zhat, const int* rows,
                                const int* rowoff, int Nx, int Ny, int Nt, int Nc, FftPlanDev fy, cudaStream_t s);
cudaError_t launch_forward_rows(const float2* zhat, float2* kspace, const int* rows, const int* rowoff, int maxm,
                                int Nx, int Ny, int Nt, int Nc, FftPlanDev fx, cudaStream_t s);
// out[b*obs + c*ors + r] = in[b*ibs + r*irs + c], for r < R, c < C, b < B (irs = 0: C)
cudaError_t launch_transpose(const float2* in, float2* out, int B, int R, int C, long long ibs, long long obs,
                             long long ors, cudaStream_t s, long long irs = 0);

// plan
cudaError_t launch_circulant(const int* rows, const int* rowoff, const double2* w64, double2* circ, int Ny, int Nt,
                             cudaStream_t s);
cudaError_t launch_plan_inverse(const float2* sens, const double2* circ, double mu, int Nx, int Ny, int Nt, int Nc,
                                void* A, int storage, const PackInfo& pk, double2* scratch, int grid,
                                int* flags, cudaStream_t s);
cudaError_t launch_unpack(const void* A, int storage, const PackInfo& pk, long long col, int Ny, float2* dense,
                          cudaStream_t s);

}  // namespace recon
