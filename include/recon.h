/*
 * recon.h - C ABI of the GB300 dynamic-SENSE ADMM reconstruction library.
 *
 * Method: Bilen, Wang & Selesnick, "High Speed Compressed Sensing
 * Reconstruction in Dynamic Parallel MRI Using Augmented Lagrangian and
 * Parallel Processing".  The library solves
 *
 *   analysis prior   (Eq. L1an_pri, Algorithm 2)
 *       min_x  lambda ||R x||_1 + ||y - H x||^2,
 *       R = D_t (temporal TV), or R = (D_t, w D_x, w D_y) with a
 *       conjugate-gradient m-update (RECON_PRIOR_STV; plus w_z D_z across the
 *       slices of a 3D volume, recon_volume_create)
 *   synthesis prior  (Eq. L1unconst, Algorithm 1)
 *       min_w  lambda ||w||_1 + ||y - H Psi' w||^2,   x = Psi' w,
 *       Psi = unitary temporal DFT, or an undecimated temporal Haar frame
 *
 * for Cartesian ky-t undersampled multi-coil data, y_{t,c} = M_{v,t} F_h F_v
 * (s_c . x_t) + n (Eqs. mri_csmcoill, H_1, S, F).  The data-consistency
 * inverse (mu I + H'H)^{-1} is applied exactly, one dense Hermitian
 * Ny x Ny block per image column and frame (Section IV-C, Eqs. HconjH,
 * eigen_mu).
 *
 * Conventions shared by every entry point
 *   - Complex arrays are interleaved complex64: element k is (re, im) at
 *     float offsets 2k, 2k+1.  Row-major, last index fastest:
 *       mask    uint8  [Nt][Ny]          (or [Nt][Ny][Nx], see opts.mask_full)
 *       sens    c64    [Nc][Ny][Nx]
 *       kspace  c64    [Nt][Nc][Ny][Nx]  (ky rows; unsampled rows are ignored)
 *       image   c64    [Nt][Ny][Nx]
 *     Index j (0..Ny-1) is the vertical / ky axis, i (0..Nx-1) the horizontal
 *     / kx axis.  ky indices are in FFT order (row 0 is ky = 0).
 *   - All Fourier transforms are unitary: forward exp(-2 pi i k n / N) / sqrt(N).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls are stream-ordered; unless stated otherwise they return
 *     after enqueueing the work.
 *   - Pointers marked "device" must be device (or managed) memory of the
 *     current device.  The caller owns every buffer it passes; the library
 *     only reads inputs during the call and keeps no reference to them.
 *   - Buffers must hold at least the elements their stated layout implies:
 *     the library receives bare pointers and cannot check their sizes (the
 *     Python binding checks every tensor's shape, dtype and device first).
 *   - Every function returns a recon_status; no function throws or aborts.
 *     recon_last_error() gives a human-readable reason for the last failure
 *     of the calling thread.
 *   - Devices: a plan lives on the device that was current at its creation,
 *     and every call on it (or on a batch, volume or gradient engine built on
 *     it) must be made with that device current.  Plans on several devices
 *     of one process are fine: each kernel's raised shared-memory limit is
 *     set on the current device at its first launch there and remembered per
 *     device ordinal.
 *   - Host threads: calls on different plans may come from different threads;
 *     calls that use one plan (or a batch, volume or gradient engine built
 *     on it) must not overlap.  The per-device limits above are kept in
 *     atomics (two first launches racing both set the attribute, which is
 *     harmless); the autotuner's cache and the allocation-free workspace are
 *     locked.
 */
#ifndef RECON_H
#define RECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct recon_plan recon_plan; /* opaque, owned by the library */

typedef enum {
  RECON_PRIOR_TV = 0,   /* Algorithm 2: analysis prior, R = D_t (non-circular temporal differences) */
  RECON_PRIOR_DFT = 1,  /* Algorithm 1: synthesis prior, Psi = unitary temporal DFT */
  RECON_PRIOR_HAAR = 2, /* Algorithm 1: synthesis prior, Psi = undecimated temporal Haar frame of
                           opts.frame_levels levels with circular shifts: a_0 = x and for level j
                           (shift s = 2^(j-1) mod Nt) a_j[t] = (a_{j-1}[t] + a_{j-1}[t+s]) / 2,
                           d_j[t] = (a_{j-1}[t] - a_{j-1}[t+s]) / 2; coefficients d_1..d_L, a_L.
                           A redundant tight frame (Psi'Psi = I, Psi Psi' != I): the w-update
                           keeps the (1/mu)(I - Psi Psi') term of the lemma in Section IV-A,
                           w = u + Psi (A (H'y + mu Psi'u) - Psi'u) with u = v + d. */
  RECON_PRIOR_STV = 3   /* Algorithm 2: analysis prior, R x = (D_t x, w D_x x, w D_y x): non-circular
                           differences along t, the horizontal and the vertical axis, spatial weight
                           w = opts.spatial_weight; l1 over all three components (anisotropic).  The
                           m-update (mu2/mu1 I + R'R) m = R'(v - d1) + mu2/mu1 (x + d2) takes
                           opts.cg_steps conjugate-gradient steps from the previous m (Section IV-B:
                           CG where no closed form is used).  Couples columns: no slab plans. */
} recon_prior;

typedef enum {
  RECON_OK = 0,
  RECON_ERR_INVALID_ARG = 1,        /* bad size, pointer or parameter */
  RECON_ERR_MASK_NOT_CARTESIAN = 2, /* a full [Nt][Ny][Nx] mask that differs along kx */
  RECON_ERR_OOM = 3,                /* device allocation failed */
  RECON_ERR_CUDA = 4,               /* a CUDA call failed (see recon_last_error) */
  RECON_ERR_TIMEOUT = 5,            /* a bounded device-side wait gave up */
  RECON_ERR_NONFINITE = 6,          /* a non-finite objective or a non-positive-definite block */
  RECON_ERR_UNSUPPORTED = 7         /* valid request the library does not support */
} recon_status;

/* Storage of the data a solve keeps in device memory.  For a plan (opts.storage):
 *   FP32  packed inverses and hybrid coil data F_h'y in complex64; the H'y
 *         prologue in double-float arithmetic (about 48 bits), rounded once.
 *   FP16 / BF16  packed inverses (double-float inversion rounded once) and the
 *         hybrid coil data (per-frame power-of-two scales) as 16-bit (re, im)
 *         pairs; FFT butterflies, products and accumulation in FP32; the
 *         objective and the stopping test reduce in FP64.
 * For k-space (recon_kspace.storage): complex64, or 16-bit pairs with
 * per-frame scales (recon_quantize_kspace).  Any k-space storage goes with
 * any plan storage. */
typedef enum {
  RECON_STORAGE_FP32 = 0,
  RECON_STORAGE_FP16 = 1,
  RECON_STORAGE_BF16 = 2
} recon_storage;

typedef struct {
  float rho;        /* mu2 / mu1 for Algorithm 2 (default 0.5, Section V); ignored for DFT */
  int max_iters;    /* iterations K (default 50); 0 returns H'y */
  double tol;       /* stop when 0 <= Delta(k) < tol (Eq. r_ratio); 0 = run K iterations */
  int storage;      /* recon_storage of the inverses and hybrid coil data (default FP32) */
  int objective;    /* J(k) every iteration: 0 = off (tol must be 0), 1 = fused (default), 2 = exact.
                       Fused: the data term ||y - Hx||^2 = ||y||^2 - 2Re<H'y,x> + Re<x,r> - mu||x||^2
                       uses (mu I + H'H) x = r of the inverse step, in the inverse kernel; its absolute
                       error is <x, e>, e the FP32 residual of that system, at most about
                       2 (1 + mu) sqrt(Ny) eps ||x||^2 (eps = 2^-24), adequate for Delta(k) (Eq. r_ratio).
                       Exact: ||y - Hx||^2 formed explicitly after each inverse step: for even Ny
                       on the tensor cores (the sampled DFT rows times s_c . x, operands split into
                       FP16 pairs, three products accumulated in FP32: about 22 bits), else by FFTs.
                       16-bit storage always uses the exact form. */
  int mask_full;    /* 1 = mask is [Nt][Ny][Nx] and must be constant along kx (default 0) */
  int col_stages;   /* ring depth of the inverse kernel, rounded down to a multiple of its consumer
                       warp count (8 at FP32 storage, 12 at 16 bit; at least that count) and
                       capped by shared memory; 0 = deepest that fits (default) */
  int profile;      /* 1 = time every kernel of a solve with CUDA events (default 0) */
  int frame_levels; /* levels L of RECON_PRIOR_HAAR, 1..6 (default 2); the frame has L+1 channels */
  float spatial_weight; /* w of RECON_PRIOR_STV, >= 0 (default 1) */
  int cg_steps;     /* CG steps per iteration of RECON_PRIOR_STV, 1..64 (default 5) */
  int persistent;   /* 0 (default): one launch per step.  1: a temporal-TV solve with FP32 storage,
                       a fixed K (tol = 0), the fused or no objective and Nt <= 40 runs its K
                       iterations as one persistent cooperative launch (Section IV-C: columns are
                       independent, so each column waits only for its own image column's temporal
                       step, never for a grid barrier); other solves ignore it.  Both give the same
                       iterates up to FP32 rounding order. */
  int overlap;      /* 1 (default): in a plan's own one-launch-per-step solve with the TV, DFT or
                       Haar prior, each inverse and temporal launch carries a programmatic dependency
                       on the kernel before it, so its launch and set-up (and the inverse kernel's
                       stream of the packed inverses, which no step writes) overlap the end of that
                       kernel; the kernel waits in-device before it touches the iteration's state.
                       Not used with a stopping test, with profile = 1, for the spatio-temporal prior,
                       or in batches (replayed graphs).  0: plain stream order.  Results are identical
                       either way. */
} recon_opts;

typedef struct {
  int iters;        /* iterations performed */
  double J;         /* J(iters), NaN when the objective was off */
  double J0;        /* J(0) at the initial point x = H'y */
  double delta;     /* Delta(iters) = (J(iters-1) - J(iters)) / J(iters), NaN if undefined */
  int stopped;      /* 1 when the tolerance test ended the run */
  double primal_res; /* ADMM residuals of the last iteration of a solve of all K iterations
                        (Boyd et al. 2011, Sec. 3.3, the paper's penalty weights).
                        RECON_PRIOR_TV and RECON_PRIOR_STV (R = D_t, or the stacked
                        spatio-temporal R), splits v = R m (mu1) and m = x (mu2):
                        sqrt(||v - R m||^2 + ||m - x||^2); a volume's slices all report the
                        volume's.  RECON_PRIOR_DFT and RECON_PRIOR_HAAR, split v = w (mu):
                        ||w - v|| (w the frame coefficients) */
  double dual_res;  /* TV, STV: sqrt(mu1^2 ||R (m_K - m_{K-1})||^2 + mu2^2 ||m_K - m_{K-1}||^2);
                        DFT, Haar: mu ||w_K - w_{K-1}||.  Both NaN after an early stop.
                        Summed in FP64. */
} recon_info;

/* Fills `opts` with the defaults listed above.  NULL-safe. */
void recon_default_opts(recon_opts* opts);

/* Builds a plan: validates the mask, copies sensitivities and the sampled row
 * lists into plan-owned device memory and computes every packed inverse
 * A_{i,t} = (mu2 I + G_{i,t})^{-1}, G_{i,t} = C_t (.) sum_c conj(s_{.,i,c}) s_{.,i,c}^T
 * (Section IV-C; C_t = F_v' P_t F_v is circulant).  The inversion runs on
 * the GPU in double-float arithmetic (pairs of FP32 numbers, about 48
 * significant bits; a blocked Hermitian sweep) and is rounded once to the
 * storage type.
 *   out     receives the plan (set to NULL on failure)
 *   Nx, Ny, Nt, Nc >= 1
 *   mask    host or device uint8, nonzero = sampled row (see opts.mask_full); at least one
 *           row sampled in some frame (a frame may have none: its inverses are I / mu2)
 *   sens    host or device complex64 [Nc][Ny][Nx]
 *   lambda  >= 0;  mu > 0: mu of Algorithm 1, mu2 of Algorithm 2 (mu1 = mu / rho)
 *   opts    NULL for defaults
 * Blocks until the plan is built (the factorisation is done once, outside
 * the timed iterations, as in Section V).  Size limits (UNSUPPORTED beyond
 * them): Nx <= 1024, Nt <= 128, Nc <= 64, (Nc + 1) Ny <= 12800, and Ny <= 768
 * with FP32 storage, 640 with 16-bit storage (the column-inverse kernel keeps
 * a column's vectors and partial sums in shared memory).  Errors: INVALID_ARG,
 * MASK_NOT_CARTESIAN, OOM, CUDA, UNSUPPORTED, NONFINITE (a block not positive
 * definite). */
recon_status recon_plan_create(recon_plan** out, int Nx, int Ny, int Nt, int Nc, const uint8_t* mask,
                               const float* sens, float lambda, float mu, recon_prior prior,
                               const recon_opts* opts, void* stream);

/* Changes mu (mu2 of Algorithm 2) of an existing plan: recomputes every packed
 * inverse (mu I + G_{i,t})^{-1} from the plan's device-resident sensitivities
 * and row lists (Eq. eigen_mu with the new mu) and every launch descriptor
 * that carries mu, keeping the allocations and the tuned launch shapes.
 * Blocks until done.  Batches and gradient engines built from the plan
 * before the call refuse to run afterwards (INVALID_ARG): build them again.
 * If the recomputation fails, the plan keeps its old mu but is unusable
 * (every later call on it returns INVALID_ARG) and must be destroyed.
 * Errors: INVALID_ARG (NULL plan, mu <= 0 or not finite), OOM, CUDA,
 * NONFINITE. */
recon_status recon_plan_set_mu(recon_plan* plan, float mu, void* stream);

/* ---- sequential reconstruction along the horizontal axis ---------------------
 * Every step of the method is separable over the image columns i once the
 * k-space rows are inverse-transformed along x (Section IV-C), so a problem
 * can be solved a slab of columns at a time with the memory of one slab's
 * inverses (Section V notes this remedy for the memory of the inverses).
 *
 * A slab plan covers columns i0 .. i0+width-1 of an Nx-wide problem.  It
 * takes the same arguments as recon_plan_create (mask, sens and, at solve
 * time, kspace and image are the whole Nx-wide arrays) and builds only its
 * columns' inverses.  Its solve reads the whole k-space rows (row IFFTs over
 * the full width, its columns kept), iterates on its columns and writes only
 * those columns of `image`.  J(k) and the stopping test are the slab's own:
 * J of the whole problem is the sum over slabs.  recon_apply_adjoint /
 * recon_apply_forward and recon_grad_* need whole plans (UNSUPPORTED);
 * recon_apply_inverse and recon_export_inverse use the slab's columns (the
 * column index of recon_export_inverse is relative to i0).  Errors: as
 * recon_plan_create; INVALID_ARG when the slab leaves the image. */
recon_status recon_plan_create_slab(recon_plan** out, int Nx, int Ny, int Nt, int Nc, const uint8_t* mask,
                                    const float* sens, float lambda, float mu, recon_prior prior,
                                    const recon_opts* opts, int i0, int width, void* stream);

/* Solves the whole problem slab after slab (slabs of `width` columns, the last
 * one narrower), holding one slab plan at a time: peak memory is one slab's
 * inverses plus the k-space and image.  kspace and image are device arrays as
 * for recon_solve.  J_trace (host, max_iters + 1 entries, may be NULL)
 * receives the sum over slabs of J(k) (meaningful with tol = 0: with a
 * tolerance each slab stops on its own); info (host, may be NULL) gets the
 * largest iteration count and the summed J, J0.  Synchronises `stream`.  Each
 * slab's plan (its factorisation) is built inside the call. */
recon_status recon_solve_slabs(int Nx, int Ny, int Nt, int Nc, const uint8_t* mask, const float* sens, float lambda,
                               float mu, recon_prior prior, const recon_opts* opts, int width, const float* kspace,
                               float* image, double* J_trace, recon_info* info, void* stream);

/* Runs the reconstruction: H'y prologue (batched row/column IFFTs and coil
 * combine), K ADMM iterations, and writes the image.
 *   kspace  device complex64 [Nt][Nc][Ny][Nx]; entries on unsampled rows are ignored
 *   image   device complex64 [Nt][Ny][Nx], written (x of Algorithm 2, Psi'w of Algorithm 1)
 *   info    host, may be NULL.  When non-NULL the call synchronises `stream`
 *           and fills it; otherwise it returns after enqueueing.
 * Errors: INVALID_ARG, CUDA, TIMEOUT, NONFINITE (only reported when info != NULL). */
recon_status recon_solve(recon_plan* plan, const float* kspace, float* image, recon_info* info, void* stream);

/* Same as recon_solve with HOST buffers: solves, copies the image
 * device->host and synchronises `stream`.  Page-locked (pinned) k-space is
 * read in place by the prologue through its device mapping, only the sampled
 * rows (1/R of the array); pageable k-space is first copied whole to a device
 * staging buffer.  The caller must not write kspace_host until the call
 * returns.
 *   kspace_host  complex64 [Nt][Nc][Ny][Nx];  image_host complex64 [Nt][Ny][Nx] */
recon_status recon_solve_host(recon_plan* plan, const float* kspace_host, float* image_host, recon_info* info,
                              void* stream);

/* Copies J(0..n-1) of the last solve to `J_host` (synchronises the plan's
 * last stream).  Entries past the last iteration are NaN. */
recon_status recon_get_trace(recon_plan* plan, double* J_host, int n);

/* Turns the per-kernel CUDA-event timing of later solves on (1) or off (0),
 * as opts.profile at creation; creates the events on first use.  Errors:
 * INVALID_ARG (NULL plan, on not 0 or 1), CUDA. */
recon_status recon_plan_set_profile(recon_plan* plan, int on);

/* Device time of the kernels of the last solve, from CUDA events recorded on
 * the solve's stream when opts.profile == 1 (synchronises that stream).
 * Fields are zero when profiling was off. */
typedef struct {
  double inverse_ms;      /* column-inverse kernel (x = A r + data-term epilogue), summed */
  int inverse_launches;
  double temporal_ms;     /* temporal kernel (prior step along t), summed */
  int temporal_launches;
  double solve_ms;        /* whole solve: prologue, iterations, output */
  int inverse_passes;     /* passes over every column those launches made (iterations) */
  int persistent;         /* 1: the iterations ran as one persistent launch, whose time (in
                             inverse_ms) includes the temporal steps of iterations 2..K */
} recon_profile;
recon_status recon_get_profile(recon_plan* plan, recon_profile* out);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long recon_kernel_launches(void);

/* Self-test of the failure path of the bounded device-side waits (no fault
 * involved): one CTA waits, through the same bounded mbarrier wait the
 * persistent kernels use, on a barrier phase that nothing completes, with a
 * wall-clock limit of limit_us microseconds (1..2000000; the kernels' own
 * limit is 2 s).  The wait gives up, records DEV_ERR_TIMEOUT in the launch's
 * error word and returns, and the call reports RECON_ERR_TIMEOUT, the status
 * a solve returns when one of its waits gives up; the CUDA context stays
 * usable.  *waited_ms (may be NULL) receives the host-measured time of the
 * launch.  Any other status means the path is broken: RECON_ERR_CUDA when the
 * wait came back without reporting, INVALID_ARG for a bad limit. */
recon_status recon_selftest_wait_timeout(int limit_us, double* waited_ms, void* stream);

/* ---- batched solves --------------------------------------------------------
 * Many independent slices (plans of uneven Nx, Ny, Nt, Nc) solved together:
 * every ADMM step is one launch over all slices (the column-inverse kernel
 * takes a work list of (slice, column) pairs balanced by bytes across the
 * SMs; the temporal kernel covers every slice's pixel tiles), and the whole
 * batched solve is captured once as a CUDA graph and replayed.  Columns and
 * slices are independent (Section IV-C), so each slice's result equals its
 * own recon_solve. */
typedef struct recon_batch recon_batch; /* opaque, owned by the library */

/* Prepares a batch over `n` plans (borrowed: they must outlive the batch).
 * The plans must share prior, max_iters, storage and objective mode and live
 * on one device.  Errors: INVALID_ARG, OOM, CUDA. */
recon_status recon_batch_create(recon_batch** out, recon_plan* const* plans, int n);

/* A 3D volume as a batch: slices stacked along z, after an inverse FFT
 * along a fully sampled kz, each with its own ky-t mask, coil profiles and
 * per-column inverses (Section II-A: the model extends to volumes; Section
 * IV-C holds slice by slice).  The plans must be RECON_PRIOR_STV with equal
 * Nx, Ny, Nt, cg_steps, max_iters, storage and objective mode, and tol = 0.
 * plans[0..nz-1] are in z order.  R gains a z-difference,
 * R x = (D_t x, w D_x x, w D_y x, w_z D_z x), non-circular along z, and the
 * m-update's CG runs over the whole volume (its inner products sum every
 * slice).  The result is a recon_batch: solve, info and destroy as for a
 * batch.  Each slice's J(k) carries the z-differences to the slice above it;
 * the volume's J is the sum over slices.  A volume of one slice is the 2D
 * solve.  Errors: INVALID_ARG (NULL, wz < 0 or not finite, mixed plans),
 * OOM, CUDA. */
recon_status recon_volume_create(recon_batch** out, recon_plan* const* plans, int nz, float wz);

/* Solves every slice: kspace[q] and image[q] are device buffers laid out as
 * for recon_solve.  The first call with a given set of buffers runs the
 * launches directly and captures them into a graph; later calls with the same
 * buffers replay that graph.  Returns after enqueueing on `stream`. */
recon_status recon_batch_solve(recon_batch* b, const float* const* kspace, float* const* image, void* stream);

/* Synchronises `stream` and fills info[q] for every slice (n entries). */
recon_status recon_batch_info(recon_batch* b, recon_info* info, void* stream);

/* Frees the batch (not its plans).  NULL-safe. */
recon_status recon_batch_destroy(recon_batch* b);

/* ---- differentiable unrolled Algorithm 2 -----------------------------------
 * Reverse mode of K = max_iters steps of Algorithm 2 (temporal TV), so that
 * the reconstruction can sit inside a learned pipeline.  The paper gives no
 * derivative; the adjoint of each step is written out by hand:
 *   x' = (mu I + H'H)^{-1} r (Eq. eigen_mu) is self-adjoint and
 *   d/dmu (mu I + H'H)^{-1} = -(mu I + H'H)^{-2};
 *   the Thomas solve with the symmetric (rho I + D_t'D_t) is self-adjoint;
 *   the complex soft threshold S(a, tau) has, for |a| > tau, the Jacobian
 *   (1 - tau/|a|) I + (tau/|a|) n n^T (n = a/|a| as a real 2-vector), and
 *   dS/dtau = -n; for |a| <= tau both are 0.
 * Parameters: mu2 = mu (the plan's mu), mu1 = mu / rho with rho fixed, so
 * the threshold is lambda rho / (2 mu).  Gradients of the complex inputs
 * follow dL/dRe + i dL/dIm (a real loss L of the image).  The forward keeps
 * the state (x, m, d1, d2) every `checkpoint_every` steps (and the last);
 * the backward recomputes each segment from its checkpoint and then walks it
 * backwards: memory is (K / checkpoint_every + checkpoint_every + 3) states of
 * 4 image fields per slice. */
typedef struct recon_grad recon_grad; /* opaque, owned by the library */

/* Prepares the forward/backward pair over `n` plans (borrowed, 1 <= n <= 255;
 * TV prior, equal max_iters >= 1 and storage).  checkpoint_every <= 0 means 5.
 * The plans' H'y buffers hold the forward's input until the backward ran:
 * do not solve with these plans in between.  Errors: INVALID_ARG,
 * UNSUPPORTED, OOM, CUDA. */
recon_status recon_grad_create(recon_grad** out, recon_plan* const* plans, int n, int checkpoint_every);

/* image[q] = x_K of slice q from kspace[q] (device buffers laid out as for
 * recon_solve; no objective, no early stop).  Enqueues on `stream`. */
recon_status recon_grad_forward(recon_grad* g, const float* const* kspace, float* const* image, void* stream);

/* Given grad_image[q] = dL/dx_K (device complex64 [Nt][Ny][Nx]), writes
 * grad_kspace[q] = dL/dy (device complex64 [Nt][Nc][Ny][Nx], 0 on unsampled
 * rows) and, when the pointers are non-NULL, grad_lambda[q] = dL/dlambda and
 * grad_mu[q] = dL/dmu (host double arrays of n entries; filling them
 * synchronises `stream`).  Must follow recon_grad_forward with the same
 * plans; may be called again for another grad_image.  Errors: INVALID_ARG,
 * TIMEOUT (a bounded device-side wait expired), CUDA. */
recon_status recon_grad_backward(recon_grad* g, const float* const* grad_image, float* const* grad_kspace,
                                 double* grad_lambda, double* grad_mu, void* stream);

/* Frees the gradient state (not its plans).  NULL-safe. */
recon_status recon_grad_destroy(recon_grad* g);

/* ---- reduced-precision k-space ----------------------------------------------
 * k-space in device memory as complex64, or as 16-bit (re, im) pairs scaled
 * per frame: entry (t, c, ky, kx) is data[t][c][ky][kx] * frame_scale[t]. */
typedef struct {
  const void* data;          /* device [Nt][Nc][Ny][Nx]: complex64, or 2 x fp16 / 2 x bf16 */
  int storage;               /* recon_storage of `data` */
  const float* frame_scale;  /* device [Nt]; NULL = all 1 */
} recon_kspace;

/* recon_solve with a recon_kspace input (same behaviour otherwise). */
recon_status recon_solve_kspace(recon_plan* plan, const recon_kspace* kspace, float* image, recon_info* info,
                                void* stream);

/* Quantises complex64 k-space (device [Nt][Nc][Ny][Nx]) to 16-bit pairs
 * (storage FP16 or BF16) with per-frame power-of-two scales: frame_scale[t]
 * (device [Nt], written) = 2^e with max_component_t / 2^e in [2^14, 2^15)
 * (1 for an all-zero frame), out[t] = k[t] / frame_scale[t] rounded once
 * to nearest.  FP16 then holds every frame's values with an 11-bit
 * significand down to 2^-29 of the frame's largest component.  `out` is
 * device memory of Nt*Nc*Ny*Nx*4 bytes.  Enqueued on `stream`.
 * Errors: INVALID_ARG, CUDA. */
recon_status recon_quantize_kspace(int Nx, int Ny, int Nt, int Nc, const float* kspace, int storage, void* out,
                                   float* frame_scale, void* stream);

/* ---- launch-shape autotuner ---------------------------------------------------
 * Times every candidate tile shape of the kernels below on the plan's (or
 * batch's) own device buffers with CUDA events and keeps the fastest.  The
 * buffers are overwritten with a pattern (a later solve re-initialises every
 * state it reads).  Results are cached per problem shape for the process, so
 * a plan of a shape already tuned takes the cached choice at once.  Not part
 * of the paper; it only picks launch shapes, never the arithmetic (for
 * RECON_PRIOR_STV the block rows also move the CG inner products' partial
 * sums, so the image may change in rounding). */
typedef struct {
  int temporal_tile_px;   /* pixels per block of the temporal kernel (TV 16, DFT 16..128, Haar 16..64);
                             for RECON_PRIOR_STV the image columns per block of its kernels (4, 8, 16) */
  int col_stages;         /* ring depth of the column-inverse kernel */
  int rows_per_block;     /* k-space rows per block of the prologue's row FFTs (1..8) */
  int combine_coils;      /* coils per pass of the prologue's column FFTs and coil combine (1..8) */
  int objective_coils;    /* coils per pass of the explicit objective; 0 when the plan does not use it,
                             1 for its tensor-core form (all coils of 256 columns (i, c) in one item) */
  float temporal_ms, col_ms, rows_ms, combine_ms, objective_ms;   /* time per launch of the chosen shape */
  int from_cache;         /* 1 when the plan took a cached result */
} recon_tuning;

/* Tunes every kernel of a plan (synchronises `stream`).  out may be NULL.
 * Errors: INVALID_ARG, CUDA, OOM. */
recon_status recon_autotune(recon_plan* plan, recon_tuning* out, void* stream);

/* Tunes the batch's temporal tile width and ring depth over all of its slices,
 * and each slice's prologue shapes (rows per block, coils per pass, the
 * explicit objective's coils per pass), once per problem shape (synchronises
 * `stream`; drops a captured graph, which is re-captured at the next
 * recon_batch_solve).  Fills temporal_tile_px, col_stages and their times,
 * the largest slice's prologue shapes and the sum of the slices' prologue
 * times.  Errors: INVALID_ARG, CUDA, OOM. */
recon_status recon_batch_autotune(recon_batch* batch, recon_tuning* out, void* stream);

/* Frees the plan and all its device memory.  NULL-safe. */
recon_status recon_destroy(recon_plan* plan);

/* ---- operators of the forward model (used by solves, exposed for tests and
 *      for callers that compose their own iterations) ---------------------- */

/* image = H' kspace = sum_c conj(s_c) . F_v' M_t' F_h' y_{t,c}  (adjoint of Eq. mri_csmcoill).
 *   kspace device complex64 [Nt][Nc][Ny][Nx];  image device complex64 [Nt][Ny][Nx] */
recon_status recon_apply_adjoint(recon_plan* plan, const float* kspace, float* image, void* stream);

/* kspace = H image = M_t F_h F_v (s_c . x_t); unsampled rows are written as 0.
 *   image device complex64 [Nt][Ny][Nx];  kspace device complex64 [Nt][Nc][Ny][Nx] */
recon_status recon_apply_forward(recon_plan* plan, const float* image, float* kspace, void* stream);

/* out = (mu I + H'H)^{-1} in, column by column with the packed inverses
 * (Eq. eigen_mu).  in, out device complex64 [Nt][Ny][Nx]; may not alias. */
recon_status recon_apply_inverse(recon_plan* plan, const float* in, float* out, void* stream);

/* Unpacks A_{i,t} into a dense row-major Ny x Ny complex64 matrix (device
 * `dense`), for inspection and tests.  0 <= i < Nx, 0 <= t < Nt. */
recon_status recon_export_inverse(recon_plan* plan, int i, int t, float* dense, void* stream);

/* Allocation-free computation of per-column inverses, for callers that
 * cannot call cudaMalloc: for example a real-time scanner pipeline that
 * reserves all of its device memory at start-up and must not allocate while
 * acquiring (an allocation can block and fragment the heap), or code embedded
 * in a host framework whose own allocator owns the device.  The paper has no
 * counterpart; it is the plan's factorisation offered without a plan.
 *
 * For each of `nblk` blocks b it writes A_b = (mu I + C_b (.) K_b)^{-1}, with
 * C_b = F_v' P_b F_v from the row mask of the block and
 * K_b[j][k] = sum_c conj(s_{b,c,j}) s_{b,c,k}, computed in FP64 and rounded
 * once to FP32.
 *   mask  device uint8 [nblk][Ny] (nonzero = sampled row)
 *   sens  device complex64 [nblk][Nc][Ny] (the coil profiles of the block's column)
 *   out   device complex64 [nblk][Ny][Ny], dense Hermitian, written
 * Allocates nothing: the FP64 workspace is a fixed 16 MiB static device array
 * that every GPU loading this library holds until exit.  It holds
 * floor((16 MiB - 256) / (16 Ny^2)) workspaces, and that many blocks are
 * factorised at once, one CTA each (15 at Ny = 256, 3 at Ny = 512); from
 * Ny = 725 on only one fits, so all blocks run one after another on a single
 * SM: large Ny is far slower here than in recon_plan_create.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU race; the call
 * synchronises `stream` before returning.
 * Errors: INVALID_ARG (also a non-finite mu); UNSUPPORTED when Ny > 1023 (one
 * Ny x Ny FP64 workspace must fit in the array) or (Nc + 2) * Ny > 12800;
 * NONFINITE for a block that is not positive definite or meets a non-finite
 * pivot (a non-finite coil profile); CUDA. */
recon_status recon_gram_inverse_noalloc(int Ny, int Nc, int nblk, const uint8_t* mask, const float* sens, float mu,
                                        float* out, void* stream);

/* Bytes of the packed inverses streamed per ADMM iteration. */
size_t recon_inverse_bytes(const recon_plan* plan);

/* Human-readable status name; never NULL. */
const char* recon_status_string(recon_status s);

/* Reason for the last failure on the calling thread ("" if none); never NULL. */
const char* recon_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H */
