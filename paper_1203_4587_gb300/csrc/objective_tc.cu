// The explicit data term ||y - H x||^2 of J(k) (Sec. V, Eq. r_ratio) on the
// tensor cores.
//
// For frame t the sampled rows of the vertical DFT of u_c = s_c . x are a
// dense contraction: C_t = F_t U_t with F_t the m_t x Ny rows of the unitary
// DFT (F[q][j] = exp(-2 pi i q j / Ny) / sqrt(Ny)) at the sampled rows q and
// U_t the Ny x (Nx Nc) matrix of every column (i, c).  Written over the reals
// with the real and imaginary parts interleaved along K (k = 2j, 2j + 1),
//   D = A B',  A = [Re F, -Im F; Im F, Re F] (rows: 64 real, then 64 imaginary
//   parts of one tile of 64 sampled rows),  B[n][2j] = Re u_n[j], B[n][2j+1] = Im u_n[j],
// so D's rows 0..63 hold Re C and rows 64..127 Im C.  The operands are split
// into FP16 pairs (hi = fp16(v), lo = fp16(v - hi), about 22 bits together)
// and D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (tcgen05.mma
// kind::f16, M = 128, N = 256, the accumulator in tensor memory).  A is
// scaled by 2^12 and each column n of B by a power of two that puts
// max |u_n| in [2^13, 2^14), so both halves stay in FP16's normal range; the
// epilogue undoes the scales exactly.
//
// Work item = (frame, tile of 64 sampled rows, tile of 256 columns (i, c)).
// A CTA per SM (1 CTA/SM by shared memory) loops over items; per item the K
// range 2 Ny_pad is walked in chunks of 32 (16 values of j).  The CTA's warps
// have two roles, synchronised by mbarriers (and a named barrier among the
// converters once per item):
//   issuer (1 warp, one thread): copies the raw tiles of each chunk (s of
//   the 256 columns and x of the image columns they span, 16 values of j
//   each) by TMA tensor copies into a ring of 2-3 stages, 2-3 chunks ahead
//   (out-of-range columns and j >= Ny read as zeros), and issues the 6 MMAs
//   of a chunk (3 products x 2 K-steps of 16) once its operands are formed,
//   committing them to the operand stage's mbarrier and, after an item's last
//   chunk, to its accumulator's;
//   converters (16 warps): form each chunk's operands in one of two stages.
//   A (hi and lo, 16 KB): a lane writes one K pair of a real row [Re F, -Im F]
//   and of its imaginary row [Im F, Re F] for two values j, from a table of
//   the Ny twiddles exp(-2 pi i d / Ny) as FP16 pairs in shared memory (index
//   q j mod Ny, stepped by 16 q a chunk).  B (hi and lo, 32 KB): a lane holds
//   two columns (i, c), (i, c + 1) at two adjacent values j, j + 1 of the raw
//   tiles, reads them with 16-byte shared loads and writes 8 bytes of a core
//   row per column and half.  They also run each item's epilogue (D read from
//   tensor memory, |y_hat - C|^2 summed over the valid rows and columns)
//   during the next item's first chunks, 8 columns a chunk, the loads of y_hat
//   in flight while the chunk is formed.
// Two accumulators of 256 columns in tensor memory alternate between items.
// The per-column scales come from max_j |x_t[i][j]| (k_col_absmax over x
// before the launch) and max_j |s_c[i][j]| (at plan time).
//
// Operand layout in shared memory (tcgen05 K-major, no swizzle): 8 x 8
// core matrices of 8 rows x 16 bytes; core (row8, k8) of a chunk at
// (k8 * rows/8 + row8) * 128 bytes; the descriptors' leading-dimension offset
// is the K-neighbour's distance (rows/8 * 128), the stride offset the row
// neighbour's (128).  The raw tiles are rows of 128 bytes (16 complex
// values) in the TMA's 128-byte swizzle: 16-byte unit u of row r sits at unit
// u ^ (r mod 8), so that the lanes' 16-byte loads fall in distinct banks.
// Every wait is bounded (DEV_ERR_TIMEOUT); on a timeout the kernel lets its
// copies and MMAs in flight finish (bounded) and frees its tensor memory
// before it returns.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kTcM = 128;              // D rows: 64 real + 64 imaginary
constexpr int kTcRows = 64;            // sampled rows per tile
constexpr int kTcN = 256;              // columns (i, c) per tile
constexpr int kTcJc = 16;              // values of j per chunk
constexpr int kTcKc = 2 * kTcJc;       // real K per chunk
constexpr int kTcConv = 512;           // 16 converter warps (B chunks, epilogues)
constexpr int kTcWarpIss = kTcConv / 32;   // the issuer warp (copies, MMAs)
constexpr int kTcThreads = kTcConv + 32;
constexpr int kTcEpCols = kTcN / (kTcConv / 128);   // accumulator columns a converter warp reads: 64
constexpr int kTcEB = 8;                            // of them a batch
constexpr int kTcENB = kTcEpCols / kTcEB;
constexpr int kTcAHalf = kTcM * kTcKc * 2;    // bytes of one FP16 half (hi or lo) of an A chunk: 8 KB
constexpr int kTcBHalf = kTcN * kTcKc * 2;    // 16 KB
constexpr int kTcStage = 2 * kTcAHalf + 2 * kTcBHalf;   // 48 KB: A hi, A lo, B hi, B lo of a chunk
constexpr int kTcRawS = kTcN * kTcJc * 8;     // 32 KB: s of 256 columns x 16 values
constexpr int kTcRawRow = kTcJc * 8;          // 128 bytes: one column's 16 values
constexpr int kTcTmemCols = 2 * kTcN;   // two accumulators: an item's epilogue overlaps the next item
constexpr int kTcSmemMax = 227 * 1024;
static_assert(kTcN / 8 == 2 * (kTcConv / 32), "a warp forms the cores of two row groups n8");
static_assert(kTcRawRow == 128, "raw rows are one 128-byte swizzle row");

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  return d;                 // base offset 0, no swizzle
}
// kind::f16 instruction descriptor: D FP32, A and B FP16, both K-major
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d_tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMA tile copies global -> shared, completion counted on bar
__device__ __forceinline__ void tma_tile_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
               :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_tile_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
               :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
               : "memory");
}

// 16-byte unit u of row r of a raw tile (128-byte swizzle)
__device__ __forceinline__ uint32_t raw_off(int r, int u) { return (uint32_t)(r * kTcRawRow + ((u ^ (r & 7)) << 4)); }

// component im (0: real, 1: imaginary) of the sampled-data value at p
__device__ __forceinline__ float y_component(const float2* p, int im) { return __ldg(reinterpret_cast<const float*>(p) + im); }
__device__ __forceinline__ float y_component(const __half2* p, int im) {
  return __half2float(__ldg(reinterpret_cast<const __half*>(p) + im));
}
__device__ __forceinline__ float y_component(const __nv_bfloat162* p, int im) {
  return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p) + im));
}

// exponent e of column col's power-of-two scale for frame t: |Re u|, |Im u|
// <= |s| |x| <= smax xmax, and 2^e puts that bound below 2^14 (0 outside the image)
__device__ __forceinline__ int tc_col_exp(const ObjTcParams& P, int t, int col, int ncols) {
  if (col >= ncols) return 0;
  const float bound = P.smax[col] * P.xmax[(size_t)t * P.Nx + col / P.Nc];
  if (!(bound > 0.f && bound < 3.0e38f)) return 0;
  int ex;
  frexpf(bound, &ex);   // bound in [2^(ex-1), 2^ex)
  return min(100, max(-100, 14 - ex));
}

// named barrier of the 16 converter warps (the issuer warp does not take part)
__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, %0;" :: "n"(kTcConv) : "memory"); }


template <class YE>
__global__ void __launch_bounds__(kTcThreads, 1) k_objective_tc(const __grid_constant__ ObjTcParams P) {
  extern __shared__ unsigned char sm_dyn[];
  __shared__ __align__(8) uint64_t mma_bar[3], raw_bar[3], bfull[3], acc_full[2], acc_empty[2];
  __shared__ uint32_t tslot;
  __shared__ double red[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (P.flags[FLAG_STOP]) return;
  // 1024-byte aligned base: the swizzle of the raw tiles repeats every 1024 bytes
  const uint32_t s0 = smem_u32(sm_dyn);
  const uint32_t pad = ((s0 + 1023u) & ~1023u) - s0;
  unsigned char* sm = sm_dyn + pad;
  const int D = P.raw_depth;
  const int S = P.op_stages;   // operand stages (2 or 3): chunk g in stage g mod S
  const int raw_bytes = P.raw_bytes;
  unsigned char* raw0 = sm + S * kTcStage;   // raw ring after the operand stages
  float* escale = reinterpret_cast<float*>(raw0 + D * raw_bytes);   // [kTcN] 2^e of column n
  float* unscale = escale + kTcN;                                   // [2][kTcN] 2^-(e + 12), by item parity
  uint2* twid = reinterpret_cast<uint2*>(unscale + 2 * kTcN);       // [Ny] DFT twiddles, FP16 pairs
  if (tid == 0) {
    for (int b = 0; b < S; ++b) { mbar_init(&mma_bar[b], 1); mbar_init(&bfull[b], kTcConv / 32); }
    for (int b = 0; b < D; ++b) mbar_init(&raw_bar[b], 1);
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kTcConv / 32); }
    fence_mbar_init();
  }
  if (warp == kTcWarpIss) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tslot)), "r"(kTcTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const int Nx = P.Nx, Nc = P.Nc, nk = P.nk;
  const int ncols = Nx * Nc;
  int* err = P.err;
  const int nmine = P.nitems > (int)blockIdx.x ? (P.nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int G = nmine * nk;   // chunks of this CTA
  double acc = 0.0;

  if (warp == kTcWarpIss) {
    // ---- issuer warp: lane 0 issues every copy and MMA of this CTA ----
    // (32-bit counters stepped by one: no integer division on this serial path)
    if (lane == 0) {
      uint32_t pend_m = 0u, pend_r = 0u;   // MMA groups / copies in flight, by stage
      uint32_t par_m = 0u, par_r = 0u;
      // raw-tile cursor over this CTA's chunks: item li, K chunk kc, ring stage st, phase parity
      int cli = 0, ckc = 0, cst = 0;
      uint32_t cph = 0u;
      int4 cit = G > 0 ? P.items[blockIdx.x] : make_int4(0, 0, 0, 0);
      // raw tiles of the cursor's chunk into its stage
      auto issue_raw = [&]() {
        const int n0 = cit.z * kTcN;
        const uint32_t dst = smem_u32(raw0) + (uint32_t)(cst * raw_bytes);
        mbar_arrive_expect_tx(&raw_bar[cst], (uint32_t)(kTcRawS + P.ni * kTcRawRow));
        tma_tile_2d(dst, &P.smap, ckc * 2 * kTcJc, n0, &raw_bar[cst]);
        tma_tile_3d(dst + kTcRawS, &P.xmap, ckc * 2 * kTcJc, n0 / Nc, cit.x, &raw_bar[cst]);
        pend_r |= 1u << cst;
        par_r = (par_r & ~(1u << cst)) | (cph << cst);
        if (++ckc == nk) {
          ckc = 0;
          if (++cli < nmine) cit = P.items[(int)blockIdx.x + cli * (int)gridDim.x];
        }
        if (++cst == D) { cst = 0; cph ^= 1u; }
      };
      for (int c = 0; c < G && c < D; ++c) issue_raw();
      bool ok = true;
      int kc = 0, li = 0, st = 0;      // chunk g: K chunk, item, raw stage
      int b = 0;                       // its operand stage (g mod S)
      uint32_t ph = 0u;                // and that stage's phase parity ((g / S) mod 2)
      for (int g = 0; g < G && ok; ++g) {
        if (kc == 0 && li >= 2) {   // the epilogue of item li - 2 has read accumulator li mod 2
          if (!mbar_wait(&acc_empty[li & 1], (uint32_t)(((li - 2) >> 1) & 1), err)) { ok = false; break; }
        }
        // A and B of chunk g formed (after the MMAs of chunk g - S left the stage), raw stage read
        if (!mbar_wait(&bfull[b], ph, err)) { ok = false; break; }
        pend_m &= ~(1u << b);   // the converters saw the MMAs of chunk g - S complete
        pend_r &= ~(1u << st);  // and the raw tiles of chunk g land
        if (g + D < G) issue_raw();
        tc_fence_after();
        const uint32_t a_hi = smem_u32(sm) + (uint32_t)(b * kTcStage), a_lo = a_hi + kTcAHalf;
        const uint32_t b_hi = a_hi + 2 * kTcAHalf, b_lo = b_hi + kTcBHalf;
        const uint32_t lboA = (kTcM / 8) * 128, lboB = (kTcN / 8) * 128;
        const uint32_t pa[3] = {a_hi, a_hi, a_lo}, pb[3] = {b_hi, b_lo, b_hi};
#pragma unroll
        for (int pr = 0; pr < 3; ++pr)
#pragma unroll
          for (int kk = 0; kk < kTcKc / 16; ++kk)
            tc_mma(tmem + (uint32_t)((li & 1) * kTcN), tc_sdesc(pa[pr] + kk * 2 * lboA, lboA, 128),
                   tc_sdesc(pb[pr] + kk * 2 * lboB, lboB, 128), (kc > 0 || pr > 0 || kk > 0) ? 1u : 0u);
        tc_commit(&mma_bar[b]);
        if (kc == nk - 1) tc_commit(&acc_full[li & 1]);   // the item's accumulator is complete
        pend_m |= 1u << b;
        par_m = (par_m & ~(1u << b)) | (ph << b);
        if (++kc == nk) { kc = 0; ++li; }
        if (++st == D) st = 0;
        if (++b == S) { b = 0; ph ^= 1u; }
      }
      if (!ok) {   // let the copies and MMAs in flight land before the memory is released
        for (int b = 0; b < 3; ++b) {
          unsigned long long t0 = global_ns();
          if ((pend_m >> b) & 1u)
            while (!mbar_try_wait(&mma_bar[b], (par_m >> b) & 1u) && global_ns() - t0 < kWaitLimitNs) {}
          t0 = global_ns();
          if ((pend_r >> b) & 1u)
            while (!mbar_try_wait(&raw_bar[b], (par_r >> b) & 1u) && global_ns() - t0 < kWaitLimitNs) {}
        }
      } else if (nmine > 0) {   // the last MMAs (committed to the last item's accumulator) complete
        mbar_wait(&acc_full[(nmine - 1) & 1], (uint32_t)(((nmine - 1) >> 1) & 1), err);
      }
    }
    __syncwarp();
  } else {
    // ---- converter warps: B chunks from the raw tiles; the epilogue of each
    // item (|y_hat - C|^2 from its accumulator) runs during the first chunks
    // of the next one, 8 columns a chunk, its loads of y_hat issued before
    // the chunk's conversion ----
    // this lane's share of a B chunk: column pair cp of row group n8 = warp +
    // 16 pp, values j = 2 jq, 2 jq + 1 of the chunk (jq = 2 k8 + hf); the pair's
    // columns are taken in the order 2 cp + e, 2 cp + 1 - e, which puts the 16
    // lanes of each half warp on 16 distinct 8-byte bank slots of a core row
    const int cp = lane & 3, e = (lane >> 2) & 1, hf = (lane >> 3) & 1, k8 = 2 * e + (lane >> 4);
    const int jq = 2 * k8 + hf;
    uint32_t offs[2][2], ob[2][2];
#pragma unroll
    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int n8 = warp + 16 * pp, n = 8 * n8 + 2 * cp + (cc ^ e);
        offs[pp][cc] = raw_off(n, jq);
        ob[pp][cc] = (uint32_t)((k8 * (kTcN / 8) + n8) * 128 + (n & 7) * 16 + hf * 8);
      }
    // epilogue share: lane quarter q of the accumulator (D row r), columns h * 64 ..
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;
    const int im = r >= kTcRows ? 1 : 0;   // D rows 64..127: imaginary parts
    // the pending epilogue (item li - 1): y_hat of row m at column h * 64 + c: ey[c mt]
    const YE* ey = nullptr;
    int emt = 0, encv = 0;                 // its mt and the lane's valid columns
    float eys = 1.f;
    float part = 0.f;
    auto load_y = [&](float (&y)[kTcEB], int eb) {
#pragma unroll
      for (int e2 = 0; e2 < kTcEB; ++e2) {
        const int c = eb * kTcEB + e2;
        y[e2] = c < encv ? y_component(ey + (size_t)c * emt, im) * eys : 0.f;
      }
    };
    auto use_acc = [&](const float (&y)[kTcEB], int eb, int li_prev) {   // batch eb of item li_prev
      const int ab = li_prev & 1;
      uint32_t v[kTcEB];
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * kTcN + h * kTcEpCols + eb * kTcEB);
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const float* us = unscale + ab * kTcN + h * kTcEpCols + eb * kTcEB;
#pragma unroll
      for (int e2 = 0; e2 < kTcEB; ++e2) {
        if (eb * kTcEB + e2 < encv) {
          const float d = y[e2] - __uint_as_float(v[e2]) * us[e2];
          part = fmaf(d, d, part);
        }
      }
    };
    auto release_acc = [&](int li_prev) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[li_prev & 1]);   // this warp has read the accumulator
    };
    const int per = (kTcENB + nk - 1) / nk;   // epilogue batches a chunk
    // A share: sampled row m = 4 warp + lane / 8 of the tile (real part in D row m,
    // imaginary in row m + 64), values j = jj, jj + 8 of each chunk; 4 bytes (a
    // K pair) of a core row each, for hi and lo
    const int am = 4 * warp + (lane >> 3), ajj = lane & 7;
    uint32_t aoff[2];
#pragma unroll
    for (int pa = 0; pa < 2; ++pa) {
      const int j = ajj + 8 * pa;
      aoff[pa] = (uint32_t)(((j >> 2) * (kTcM / 8) + (am >> 3)) * 128 + (am & 7) * 16 + (j & 3) * 4);
    }
    for (int d = tid; d < P.Ny; d += kTcConv) twid[d] = P.twiddle[d];   // ordered by the first conv_sync
    bool ok = true;
    int g = 0;                 // chunks of this CTA seen
    int st = 0;                // their raw stage (g mod D)
    uint32_t ph_r = 0u;        // and its phase parity ((g / D) mod 2)
    int b = 0;                 // their operand stage (g mod S)
    uint32_t ph_b = 0u;        // and its phase parity ((g / S) mod 2)
    // every converter warp takes both named barriers of every item, also after
    // a failed wait (ok = false then skips the work), so that none waits forever
    for (int li = 0; li < nmine; ++li) {
      const int item = (int)blockIdx.x + li * (int)gridDim.x;
      const int4 it = P.items[item];   // (t, row tile, column tile, A tile index)
      const int t = it.x, n0 = it.z * kTcN, ilo = n0 / Nc;
      conv_sync();   // every converter has read the previous item's scales (and item li - 2's epilogue is done)
      if (tid < kTcN) {
        const int ex = tc_col_exp(P, t, n0 + tid, ncols);
        escale[tid] = ldexpf(1.f, ex);
        unscale[(li & 1) * kTcN + tid] = ldexpf(1.f, -(ex + 12));
      }
      conv_sync();
      if (!ok) continue;
      // this lane's sampled row q (-1: none) and its twiddle indices q j mod Ny
      const int aq = P.tile_rows[(size_t)it.w * kTcRows + am];
      const int aq16 = aq >= 0 ? (aq * kTcJc) % P.Ny : 0;   // q < Ny <= 768: no overflow
      int ad[2];
#pragma unroll
      for (int pa = 0; pa < 2; ++pa) ad[pa] = aq >= 0 ? (aq * (ajj + 8 * pa)) % P.Ny : 0;
      float esv[2][2];
      uint32_t offx[2][2];
#pragma unroll
      for (int pp = 0; pp < 2; ++pp)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int n = 8 * (warp + 16 * pp) + 2 * cp + (cc ^ e), col = n0 + n;
          esv[pp][cc] = escale[n];
          const int xr = col < ncols ? min(col / Nc - ilo, P.ni - 1) : 0;   // a column outside: s reads 0
          offx[pp][cc] = (uint32_t)kTcRawS + raw_off(xr, jq);
        }
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int eb0 = li > 0 ? min(kTcENB, kc * per) : kTcENB, eb1 = min(kTcENB, eb0 + per);
        float yb[kTcEB];
        if (eb0 < eb1) load_y(yb, eb0);   // in flight during the conversion
        // the MMAs of chunk g - S have read operand stage b
        if (g >= S && !mbar_wait(&mma_bar[b], ph_b ^ 1u, err)) { ok = false; break; }
        if (!mbar_wait(&raw_bar[st], ph_r, err)) { ok = false; break; }
        const unsigned char* rs = raw0 + st * raw_bytes;
        unsigned char* Ah = sm + b * kTcStage;
        unsigned char* Bh = Ah + 2 * kTcAHalf;
        // A: rows [Re F, -Im F] and [Im F, Re F] of the twiddle exp(-2 pi i q j / Ny) (scaled)
#pragma unroll
        for (int pa = 0; pa < 2; ++pa) {
          uint2 w = make_uint2(0u, 0u);   // (hi re, hi im), (lo re, lo im) as FP16 pairs
          if (aq >= 0 && kc * kTcJc + ajj + 8 * pa < P.Ny) w = twid[ad[pa]];
          const uint32_t o = aoff[pa];
          *reinterpret_cast<uint32_t*>(Ah + o) = w.x ^ 0x80000000u;                            // (Re, -Im) hi
          *reinterpret_cast<uint32_t*>(Ah + o + 1024) = __funnelshift_l(w.x, w.x, 16);        // (Im, Re) hi
          *reinterpret_cast<uint32_t*>(Ah + kTcAHalf + o) = w.y ^ 0x80000000u;                 // lo
          *reinterpret_cast<uint32_t*>(Ah + kTcAHalf + o + 1024) = __funnelshift_l(w.y, w.y, 16);
          ad[pa] += aq16;
          if (ad[pa] >= P.Ny) ad[pa] -= P.Ny;
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const float4 sv = *reinterpret_cast<const float4*>(rs + offs[pp][cc]);
            const float4 xv = *reinterpret_cast<const float4*>(rs + offx[pp][cc]);
            const float es = esv[pp][cc];
            const float2 w0 = c_scale(c_mul(make_float2(sv.x, sv.y), make_float2(xv.x, xv.y)), es);
            const float2 w1 = c_scale(c_mul(make_float2(sv.z, sv.w), make_float2(xv.z, xv.w)), es);
            const __half2 h0 = __floats2half2_rn(w0.x, w0.y), h1 = __floats2half2_rn(w1.x, w1.y);
            const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
            const __half2 l0 = __floats2half2_rn(w0.x - f0.x, w0.y - f0.y);
            const __half2 l1 = __floats2half2_rn(w1.x - f1.x, w1.y - f1.y);
            *reinterpret_cast<uint2*>(Bh + ob[pp][cc]) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
            *reinterpret_cast<uint2*>(Bh + kTcBHalf + ob[pp][cc]) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&l0), *reinterpret_cast<const uint32_t*>(&l1));
          }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bfull[b]);
        if (++st == D) { st = 0; ph_r ^= 1u; }
        if (++b == S) { b = 0; ph_b ^= 1u; }
        // the epilogue batches of item li - 1 that fall on this chunk
        if (eb0 < eb1) {
          if (eb0 == 0) {
            if (!mbar_wait(&acc_full[(li - 1) & 1], (uint32_t)(((li - 1) >> 1) & 1), err)) { ok = false; break; }
            tc_fence_after();
          }
          use_acc(yb, eb0, li - 1);
          for (int eb = eb0 + 1; eb < eb1; ++eb) {
            load_y(yb, eb);
            use_acc(yb, eb, li - 1);
          }
          if (eb1 == kTcENB) release_acc(li - 1);
        }
      }
      if (!ok) continue;
      // item li's epilogue, for the next item's chunks (or below, after the last item)
      {
        const int rt = it.y;
        const int r0 = P.rowoff[t], mt = P.rowoff[t + 1] - r0;
        const int m = rt * kTcRows + (r & (kTcRows - 1));
        ey = static_cast<const YE*>(P.yhat) + (size_t)r0 * ncols + (size_t)(n0 + h * kTcEpCols) * mt + m;
        emt = mt;
        encv = m < mt ? min(kTcEpCols, ncols - (n0 + h * kTcEpCols)) : 0;
        eys = P.yscale ? P.yscale[t] : 1.f;
      }
    }
    // the last item's epilogue
    if (ok && nmine > 0) {
      const int lp = nmine - 1;
      float ya[kTcEB], yb2[kTcEB];
      load_y(ya, 0);
      if (mbar_wait(&acc_full[lp & 1], (uint32_t)((lp >> 1) & 1), err)) {
        tc_fence_after();
        for (int eb = 0; eb < kTcENB; eb += 2) {
          load_y(yb2, eb + 1);
          use_acc(ya, eb, lp);
          if (eb + 2 < kTcENB) load_y(ya, eb + 2);
          use_acc(yb2, eb + 1, lp);
        }
        release_acc(lp);
      }
    }
    acc = (double)part;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTcWarpIss)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcTmemCols) : "memory");
  const double sum = group_sum(acc, red, tid, kTcThreads, BlockBar());
  if (tid == 0 && sum != 0.0) atomicAdd(P.fid_acc, sum);
}

// shared memory of a launch: 1 KB alignment slack, two operand stages, the
// raw ring, the column scales, the twiddle table
size_t tc_smem_bytes(int op_stages, int raw_depth, int raw_bytes, int Ny) {
  return 1024 + (size_t)op_stages * kTcStage + (size_t)raw_depth * raw_bytes + 3 * kTcN * sizeof(float) +
         (size_t)((Ny + 1) / 2) * 2 * sizeof(uint2);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

}  // namespace

// max_j |s[col][j]| of each column (i, c): one warp a column
__global__ void k_col_absmax(const float2* __restrict__ s, int ncols, int Ny, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); col < ncols; col += gridDim.x * (blockDim.x >> 5)) {
    float mx = 0.f;
    for (int j = lane; j < Ny; j += 32) {
      const float2 v = s[(size_t)col * Ny + j];
      mx = fmaxf(mx, sqrtf(fmaf(v.x, v.x, v.y * v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) out[col] = mx * 1.0001f;   // above the rounding of the magnitude
  }
}

cudaError_t launch_col_absmax(const float2* s, int ncols, int Ny, float* out, cudaStream_t st) {
  if (ncols < 1) return cudaSuccess;
  k_col_absmax<<<(ncols + 7) / 8, 256, 0, st>>>(s, ncols, Ny, out);
  note_launch();
  return cudaGetLastError();
}

// The twiddles exp(-2 pi i d / Ny) 2^12 / sqrt(Ny), d = 0..Ny-1, each part split
// into an FP16 pair from FP64: x = (hi re, hi im), y = (lo re, lo im), the
// low half of each word the real part.
void objective_tc_twiddle(int Ny, uint2* out) {
  const double scl = 4096.0 / std::sqrt((double)Ny);
  auto bits = [](__half h) { return (uint32_t)__half_as_ushort(h); };
  for (int d = 0; d < Ny; ++d) {
    const double a = -2.0 * M_PI * (double)d / (double)Ny;
    const double fr = std::cos(a) * scl, fi = std::sin(a) * scl;
    const __half hr = __double2half(fr), hi = __double2half(fi);
    const __half lr = __double2half(fr - (double)__half2float(hr)), li = __double2half(fi - (double)__half2float(hi));
    out[d] = make_uint2(bits(hr) | (bits(hi) << 16), bits(lr) | (bits(li) << 16));
  }
}

bool objective_tc_prepare(ObjTcParams& q, const float2* x, const float2* sens) {
  const int Nx = q.Nx, Ny = q.Ny, Nt = q.Nt, Nc = q.Nc;
  if (Ny % 2 != 0 || Nx < 1 || Nc < 1 || Nt < 1) return false;   // rows of 8 Ny bytes: a multiple of 16
  // image columns spanned by a tile of 256 columns (i, c)
  q.ni = std::min(Nx, std::min(256, (kTcN - 1) / Nc + 2));
  q.raw_bytes = kTcRawS + ((q.ni * kTcRawRow + 1023) / 1024) * 1024;
  // the deepest rings that fit: three operand stages first (they hide the MMAs' completion
  // latency), then a third raw stage
  const size_t cap = (size_t)kTcSmemMax - 1024;   // the static shared memory's share
  q.op_stages = 0;
  for (int S : {3, 2})
    for (int D : {3, 2})
      if (!q.op_stages && tc_smem_bytes(S, D, q.raw_bytes, Ny) <= cap) { q.op_stages = S; q.raw_depth = D; }
  if (!q.op_stages) return false;
  q.nk = (Ny + kTcJc - 1) / kTcJc;
  q.x = x;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)2 * Ny, (cuuint64_t)Nx * Nc};
    const cuuint64_t strides[1] = {(cuuint64_t)Ny * 8};
    const cuuint32_t box[2] = {(cuuint32_t)2 * kTcJc, (cuuint32_t)kTcN};
    if (enc(&q.smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(sens), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)2 * Ny, (cuuint64_t)Nx, (cuuint64_t)Nt};
    const cuuint64_t strides[2] = {(cuuint64_t)Ny * 8, (cuuint64_t)Ny * 8 * Nx};
    const cuuint32_t box[3] = {(cuuint32_t)2 * kTcJc, (cuuint32_t)q.ni, 1};
    if (enc(&q.xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(x), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

cudaError_t launch_objective_tc(const ObjTcParams& p, cudaStream_t s) {
  static SmemAttrCache cache[3];
  const void* fn[3] = {reinterpret_cast<const void*>(k_objective_tc<float2>),
                       reinterpret_cast<const void*>(k_objective_tc<__half2>),
                       reinterpret_cast<const void*>(k_objective_tc<__nv_bfloat162>)};
  if (p.ystorage < 0 || p.ystorage > 2 || p.raw_depth < 2 || p.raw_depth > 3 || p.op_stages < 2 || p.op_stages > 3)
    return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes(p.op_stages, p.raw_depth, p.raw_bytes, p.Ny);
  cudaError_t e = cache[p.ystorage].ensure(fn[p.ystorage], smem);
  if (e != cudaSuccess) return e;
  if ((e = launch_col_absmax(p.x, p.Nt * p.Nx, p.Ny, p.xmax, s)) != cudaSuccess) return e;
  if (p.nitems < 1) return cudaSuccess;
  const int grid = std::min(p.nitems, p.grid);
  ObjTcParams q = p;
  void* args[] = {&q};
  const cudaError_t el = cudaLaunchKernel(fn[p.ystorage], dim3(grid), dim3(kTcThreads), args, smem, s);
  note_launch();
  return el != cudaSuccess ? el : cudaGetLastError();
}

}  // namespace recon
