// Persistent solve of Algorithm 2 with temporal TV: every ADMM iteration of
// one or many slices in one cooperative launch.
//
// Every step of the iteration separates along the horizontal axis (Section
// IV-C; Section V: "separated along the horizontal axis"), so the iteration is
// a dataflow over image columns (slice q, column i):
//   T_k(q, i)     the v-, m- and d1-updates of iteration k for the Ny x Nt
//                 pixels of column i (they couple the frames t), giving
//                 p_k = m_k - d2_{k-1};
//   I_k(q, i, t)  the x-update x = A_{i,t} (H'y + mu2 p_k) of one column, with
//                 the data term of J(k) (the d2-update is implicit: d2 = x - p).
// I_k(q, i, t) needs T_k(q, i); T_{k+1}(q, i) needs I_k(q, i, t) for every t.
// No grid barrier is needed: each CTA streams its list of columns (the
// column-inverse pipeline of colinv.cuh) for k = 1..K in turn, and
//   * the CTA whose column completes the last frame of (q, i) in iteration k
//     (a per-column atomic counter) appends T_{k+1}(q, i) to a global task
//     queue; the four temporal warps of every CTA take tasks from it by
//     ticket (which CTA completes a column's last frame is systematic, so
//     running the task there would pile the temporal work onto a few SMs),
//     and count each finished chunk (kPersistPx pixels of the column, every
//     frame; a task is one chunk) in tdone[q][i];
//   * the r loader waits (bounded) for tdone[q][i] >= (k - 1) * chunks before
//     it reads p_k of a column of iteration k.
// Every dependency points to an earlier iteration, so with all CTAs resident
// (a cooperative launch) every wait ends; each still has a wall-clock limit
// after which the kernel sets DEV_ERR_TIMEOUT and leaves.  State buffers
// alternate by iteration parity as in the per-iteration launches, so the
// ADMM residuals and the final image read the same buffers.  T_1 (from
// x = m = p = H'y) runs before the launch; T_{K+1} only forms ||D_t x_K||_1.
#include "colinv.cuh"
#include "tv_chunk.cuh"
#include "plan.h"

namespace recon {

constexpr int kPersistTWarps = 4;                 // temporal warps
constexpr int kPersistTThreads = 32 * kPersistTWarps;
constexpr int kPersistSeg = kTvSeg;               // Thomas segments (tv_chunk.cuh)
constexpr int kPersistPx = kTvChunkPx;            // pixels per temporal chunk
static_assert(kPersistTThreads == kTvChunkThreads && kPersistPx == kPersistChunkPx, "temporal chunk shape");
constexpr int kPersistLMax = kPersistNtMax / kPersistSeg;   // frames per segment
constexpr int kPersistRSlots = 4;                 // the r loader's lookahead (columns)

__host__ __device__ constexpr int persist_threads() { return col_threads(8) + kPersistTThreads; }

struct PersistLayout {
  ColLayout c;   // the column-inverse regions; c.slices holds PersistSlice entries
  size_t rbars, rslot, segA, segB, bnd, red, total;
};

__host__ __device__ inline PersistLayout persist_layout(int stages, int nb, int nslices, int work_max) {
  PersistLayout L;
  // the column-inverse layout without its slice table, then a table of
  // PersistSlice entries, the work list and the temporal warps' regions
  L.c = col_layout(stages, nb, 0, 0, 8);   // its 2-slot r ring and barriers are left unused
  size_t o = align_up(L.c.slices, 16);
  L.c.slices = o; o += (size_t)nslices * sizeof(PersistSlice);
  o = align_up(o, 16);
  L.c.skip = o;
  L.c.work = o; o += (size_t)work_max * 4;
  o = align_up(o, 16);
  L.rbars = o; o += 2 * kPersistRSlots * 8;              // rfull, rempty of the deeper slot ring
  o = align_up(o, 16);
  L.rslot = o; o += (size_t)kPersistRSlots * 2 * (size_t)nb * 32 * sizeof(float2);   // [slot][b, p][ny32]
  L.segA = o; o += kPersistSeg * kPersistPx * sizeof(float);
  o = align_up(o, 16);
  L.segB = o; o += kPersistSeg * kPersistPx * sizeof(float2);
  L.bnd = o; o += kPersistSeg * kPersistPx * sizeof(float2);
  L.red = o; o += 32 * sizeof(double);
  L.total = align_up(o, 128);
  return L;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= want (acquire).  False on timeout (DEV_ERR_TIMEOUT
// set) or when another CTA has reported an error.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned want, int* flags) {
  if (ld_acquire_u32(p) >= want) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    __nanosleep(64);
    if (ld_acquire_u32(p) >= want) return true;
    if ((it & 63u) == 0) {
      if (*((volatile int*)&flags[FLAG_ERR]) != 0) return false;
      if (global_ns() - t0 > kWaitLimitNs) { atomicOr(&flags[FLAG_ERR], DEV_ERR_TIMEOUT); return false; }
    }
  }
}

// Bounded wait until *p == 0 (acquire).
__device__ __forceinline__ bool wait_zero(const unsigned* p, int* flags) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (ld_acquire_u32(p) == 0u) return true;
    __nanosleep(64);
    if ((it & 63u) == 0) {
      if (*((volatile int*)&flags[FLAG_ERR]) != 0) return false;
      if (global_ns() - t0 > kWaitLimitNs) { atomicOr(&flags[FLAG_ERR], DEV_ERR_TIMEOUT); return false; }
    }
  }
}

__device__ __forceinline__ void tbar() { named_bar_sync(1, kPersistTThreads); }

// One chunk of T_{k+1}(q, i) -- pixels j = chunk * kPersistPx + px of image
// column i, every frame -- by the temporal warps (thread tid of
// kPersistTThreads), the arithmetic of tv_chunk.cuh.  k == K: only
// ||D_t x_K||_1.  A column's chunks are independent tasks, so tdone[i] counts
// chunks.
__device__ void persist_temporal(const PersistSlice& S, int i, int chunk, int k, int K, int tid, float* segA,
                                 float2* segB, float2* bnd, double* red) {
  const bool write = k < K;
  const int in = k & 1, out = (k + 1) & 1;
  TvChunkIO io;
  io.x = S.x;
  io.m = S.m[in];
  io.d1 = S.d1[in];
  io.p = S.p[in];
  io.m_out = S.m[out];
  io.d1_out = S.d1[out];
  io.p_out = S.p[out];
  io.thomas = S.thomas;
  io.tau1 = S.tau1;
  io.rho = S.rho;
  io.Nt = S.Nt;
  io.fstride = (size_t)S.Nx * S.Ny;
  io.base = (size_t)i * S.Ny + (size_t)chunk * kPersistPx;
  io.nvalid = min(kPersistPx, S.Ny - chunk * kPersistPx);
  io.write = write;
  struct TBar {
    __device__ void operator()() const { tbar(); }
  };
  const float tvf = tv_chunk<kPersistLMax, false>(io, tid, segA, segB, bnd, TBar());
  // the prior term of J at x_k
  double v = warp_sum((double)tvf);
  const int w = tid >> 5, lane = tid & 31;
  if (lane == 0) red[w] = v;
  tbar();
  if (tid == 0) {
    double s = 0.0;
    for (int q = 0; q < kPersistTWarps; ++q) s += red[q];
    atomicAdd(S.trace_prior + k, s);
  }
  if (write) {
    // publish this chunk of T_{k+1}(q, i): the new state before the count
    __threadfence();
    tbar();
    if (tid == 0) {
      __threadfence();
      atomicAdd(S.tdone + i, 1u);
    }
  } else {
    tbar();
  }
}

__global__ void __launch_bounds__(persist_threads(), 1) k_persist_tv(PersistLaunch P) {
  extern __shared__ __align__(128) unsigned char smem[];
  using E = float2;
  constexpr int kProducers = col_producers(8);
  constexpr int kConsumerWarps = col_consumer_warps(8);
  constexpr int kStage = stage_bytes(8);
  constexpr int kLoader = kConsumerWarps + kProducers;
  constexpr int kManager = kLoader + 1;
  constexpr int kTWarp0 = kManager + 1;
  const PersistLayout PL = persist_layout(P.stages, P.nb_max, P.nslices, P.work_max);
  const ColLayout& L = PL.c;
  const int S = P.stages, K = P.K;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  uint64_t* rv_full = empty + S + 2 * kRSlots;   // after the unused rfull / rempty of colinv.cuh
  uint64_t* yc_empty = rv_full + kRSlots;
  uint64_t* col_done = yc_empty + kRSlots;
  unsigned char* ring = smem + L.ring;
  const int ny32m = P.nb_max * 32;
  float2* ycopy = reinterpret_cast<float2*>(smem + L.ycopy);
  float2* rvec = reinterpret_cast<float2*>(smem + L.rvec);
  float2* bvec = reinterpret_cast<float2*>(smem + L.bvec);
  uint64_t* rfull = reinterpret_cast<uint64_t*>(smem + PL.rbars);
  uint64_t* rempty = rfull + kPersistRSlots;
  float2* rslot = reinterpret_cast<float2*>(smem + PL.rslot);
  PersistSlice* sl = reinterpret_cast<PersistSlice*>(smem + L.slices);
  int* tiles = reinterpret_cast<int*>(smem + L.tiles);
  unsigned* wl = reinterpret_cast<unsigned*>(smem + L.work);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int m = tid; m < P.nb_max * (P.nb_max - 1) / 2; m += blockDim.x) tiles[m] = tile_pq(m);
  for (int q = tid; q < P.nslices; q += blockDim.x) sl[q] = P.slices[q];
  for (int j = tid; j < kRSlots * kConsumerWarps * ny32m; j += blockDim.x) ycopy[j] = make_float2(0.f, 0.f);
  const int w0 = P.work_off[blockIdx.x], w1 = P.work_off[blockIdx.x + 1];
  for (int w = w0 + tid; w < w1; w += blockDim.x) wl[w - w0] = P.work[w];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int s = 0; s < kPersistRSlots; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], 1);
    }
    for (int s = 0; s < kRSlots; ++s) {
      mbar_init(&rv_full[s], 1);
      mbar_init(&yc_empty[s], 1);
      mbar_init(&col_done[s], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int nw = w1 - w0;            // columns per iteration
  const int ncol = nw * K;           // columns over the whole solve
#define WSL(w) ((int)(wl[w] >> 24))
#define WCOL(w) ((int)(wl[w] & 0xFFFFFFu))

  if (warp >= kConsumerWarps && warp < kLoader) {
    // ---------------- producers: the packed inverses, K passes over the list ----
    if (lane == 0) {
      const int p = warp - kConsumerWarps;
      const uint64_t pol = policy_evict_first();
      int st = p, wraps = 0, gu = 0, issued = 0, ncolumn = 0;
      bool ok = true;
      for (int n = 0; n < ncol && ok; ++n) {
        const int w = n % nw;
        const PersistSlice& c = sl[WSL(w)];
        const unsigned char* cb = reinterpret_cast<const unsigned char*>(c.A) +
                                  (size_t)packed_index(WCOL(w), c.Nx, c.Nt) * (size_t)c.col_elems * 8;
        const int rot = unit_rotation(ncolumn++, c.nunits);
        int u = p - gu % kProducers;
        if (u < 0) u += kProducers;
        for (; u < c.nunits; u += kProducers) {
          if (wraps > 0 && !mbar_wait(&empty[st], (uint32_t)((wraps - 1) & 1), P.err)) { ok = false; break; }
          const int4 un = decode_unit(rotated_unit(u, rot, c.nunits), c.nb, tiles);
          const uint32_t bytes = (uint32_t)((un.x == UNIT_TILE ? kTileElems : kDiagElems) * 8);
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(ring + (size_t)st * kStage, cb + (size_t)un.w * 8, bytes, &full[st], pol);
          ++issued;
          st += kProducers;
          if (st >= S) { st -= S; ++wraps; }
        }
        gu += c.nunits;
      }
      if (!ok) {
        const int per = S / kProducers;
        for (int q = (issued > per ? issued - per : 0); q < issued; ++q) {
          const long long gi = p + (long long)q * kProducers;
          uint64_t* bb = &full[gi % S];
          const uint32_t par = (uint32_t)((gi / S) & 1);
          const unsigned long long t0 = global_ns();
          while (!mbar_try_wait(bb, par) && global_ns() - t0 < kWaitLimitNs) {}
        }
      }
    }
    return;
  }
  if (warp == kLoader) {
    // ---------------- r loader: b and p_k of each column, once T_k is published --
    const uint64_t pol_first = policy_evict_first();
    int issued = 0;   // columns whose bulk copies lane 0 issued (for the error path)
    for (int n = 0; n < ncol; ++n) {
      const int w = n % nw, k = n / nw + 1;
      const PersistSlice& c = sl[WSL(w)];
      const int col = WCOL(w), i = col % c.Nx;
      const int slt = n % kPersistRSlots;
      // lane 0 waits (the slot, then T_k of this image column) and shares the outcome
      int ok = 1;
      if (lane == 0) {
        if (n >= kPersistRSlots) ok = mbar_wait(&rempty[slt], (uint32_t)(((n / kPersistRSlots) - 1) & 1), P.err) ? 1 : 0;
        if (ok && k >= 2) ok = wait_at_least(c.tdone + i, (unsigned)(k - 1) * (unsigned)c.nch, P.err) ? 1 : 0;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      float2* d = rslot + (size_t)slt * 2 * ny32m;
      const size_t cofs = (size_t)col * c.Ny;
      const float2* pk = c.p[k & 1];
      if ((c.Ny & 1) == 0) {
        // 16-byte aligned columns: two bulk copies, completion counted on the
        // slot's barrier, so the loader moves on to the next column at once.
        // p_k was written by other CTAs' generic stores, published by tdone
        // (acquired above); the proxy fence orders those writes before this
        // thread's async-proxy reads.
        if (lane == 0) {
          const uint32_t bytes = (uint32_t)c.Ny * 8u;
          asm volatile("fence.proxy.async.global;" ::: "memory");
          mbar_arrive_expect_tx(&rfull[slt], 2u * bytes);
          bulk_g2s(d, c.b + cofs, bytes, &rfull[slt], pol_first);
          bulk_g2s(d + ny32m, pk + cofs, bytes, &rfull[slt], pol_first);
        }
        issued = n + 1;
        continue;
      } else {
        for (int j = lane; j < c.Ny; j += 32) {
          d[j] = __ldcg(c.b + cofs + j);
          d[ny32m + j] = __ldcg(pk + cofs + j);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&rfull[slt]);
    }
    if (lane == 0) {
      // bulk copies of the last slots may still be in flight if the kernel quits early
      for (int h = (issued > kPersistRSlots ? issued - kPersistRSlots : 0); h < issued; ++h) {
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&rfull[h % kPersistRSlots], (uint32_t)((h / kPersistRSlots) & 1)) &&
               global_ns() - t0 < kWaitLimitNs) {}
      }
    }
    return;
  }
  if (warp == kManager) {
    // ---------------- column manager ------------------------------------------
    // It prepares r = H'y + mu2 p_k of column n (once its inputs are in a slot)
    // and runs the epilogue of column n (once the consumers are done), in
    // whichever order they become ready: column n + 1 may be the same image
    // column one iteration later, whose p needs this column's epilogue first.
    auto prepare = [&](int n) {   // rfull of column n has completed
      const int w = n % nw;
      const PersistSlice& c = sl[WSL(w)];
      const int ny32 = c.nb * 32;
      const int slt = n % kPersistRSlots;
      const float2* d = rslot + (size_t)slt * 2 * ny32m;
      float2* rv = rvec + (size_t)(n & 1) * ny32m;
      float2* bv = bvec + (size_t)(n & 1) * ny32m;
      for (int j = 2 * lane; j < ny32; j += 64) {
        float4 v = *reinterpret_cast<const float4*>(d + j);
        const float4 bb0 = v;
        float4 bb = bb0;
        const float4 a = *reinterpret_cast<const float4*>(d + ny32m + j);
        v.x = fmaf(c.mu, a.x, v.x); v.y = fmaf(c.mu, a.y, v.y);
        v.z = fmaf(c.mu, a.z, v.z); v.w = fmaf(c.mu, a.w, v.w);
        if (j >= c.Ny) { v.x = v.y = 0.f; bb.x = bb.y = 0.f; }
        if (j + 1 >= c.Ny) { v.z = v.w = 0.f; bb.z = bb.w = 0.f; }
        *reinterpret_cast<float4*>(rv + j) = v;
        *reinterpret_cast<float4*>(bv + j) = bb;
      }
      __syncwarp();
      if (lane == 0) { mbar_arrive(&rempty[slt]); mbar_arrive(&rv_full[n & 1]); }
    };
    // T_{k+1}(q, i) into the global queue (lane 0): entry h = the h-th task
    // produced; its tag h + 1, stored last with release, marks it written
    // every chunk of T_{k+1}(q, i) as its own task, lanes in parallel
    auto push = [&](int q, int i, int k) -> bool {
      const int nch = sl[q].nch;
      unsigned h0 = 0;
      if (lane == 0) h0 = atomicAdd(P.tq_tail, (unsigned)nch);
      h0 = __shfl_sync(0xffffffffu, h0, 0);
      int ok = 1;
      for (int ch = lane; ch < nch && ok; ch += 32) {
        const unsigned h = h0 + (unsigned)ch;
        int4* e = P.tq_ring + (h & (P.tq_cap - 1));
        unsigned* tag = reinterpret_cast<unsigned*>(&e->w);
        // the slot's previous task (h - cap) must have been taken: never in
        // practice (the ring holds several iterations of tasks), still bounded
        if (ld_acquire_u32(tag) != 0u) ok = wait_zero(tag, P.err) ? 1 : 0;
        if (ok) {
          e->x = q; e->y = i | (ch << 20); e->z = k;
          __threadfence();
          st_release_u32(tag, h + 1u);
        }
      }
      return __all_sync(0xffffffffu, ok) != 0;
    };
    double fid = 0.0;
    int fid_slice = -1, fid_k = -1;
    auto epilogue = [&](int n) -> bool {   // col_done of column n has completed
      const int bb = n & 1;
      const int w = n % nw, k = n / nw + 1;
      const int q = WSL(w);
      const PersistSlice& c = sl[q];
      if (q != fid_slice || k != fid_k) {
        if (fid_slice >= 0 && sl[fid_slice].do_obj) {
          const double f = warp_sum(fid);
          if (lane == 0) atomicAdd(sl[fid_slice].trace_fid + fid_k, f);
        }
        fid = 0.0;
        fid_slice = q;
        fid_k = k;
      }
      const int ny32 = c.nb * 32;
      const int col = WCOL(w);
      const size_t cofs = (size_t)col * c.Ny;
      float2* yc = ycopy + (size_t)bb * kConsumerWarps * ny32m;
      const float2* rv = rvec + (size_t)bb * ny32m;
      const float2* bv = bvec + (size_t)bb * ny32m;
      float fcol = 0.f;
      const bool vec_out = ((cofs & 1) == 0);
      for (int j = 2 * lane; j < ny32; j += 64) {
        float4 x = *reinterpret_cast<const float4*>(yc + j);
        *reinterpret_cast<float4*>(yc + j) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int ww = 1; ww < kConsumerWarps; ++ww) {
          float4* pw = reinterpret_cast<float4*>(yc + (size_t)ww * ny32m + j);
          const float4 t = *pw;
          x.x += t.x; x.y += t.y; x.z += t.z; x.w += t.w;
          *pw = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (j + 1 < c.Ny && vec_out) {
          *reinterpret_cast<float4*>(c.x + cofs + j) = x;
        } else {
          if (j < c.Ny) c.x[cofs + j] = make_float2(x.x, x.y);
          if (j + 1 < c.Ny) c.x[cofs + j + 1] = make_float2(x.z, x.w);
        }
        if (c.do_obj) {
          if (j >= c.Ny) x.x = x.y = 0.f;
          if (j + 1 >= c.Ny) x.z = x.w = 0.f;
          const float4 r = *reinterpret_cast<const float4*>(rv + j), b = *reinterpret_cast<const float4*>(bv + j);
          float f = c.w_bx * fmaf(b.x, x.x, fmaf(b.y, x.y, fmaf(b.z, x.z, b.w * x.w)));
          f = fmaf(c.w_xr, fmaf(x.x, r.x, fmaf(x.y, r.y, fmaf(x.z, r.z, x.w * r.w))), f);
          f = fmaf(c.w_xx, fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, x.w * x.w))), f);
          fcol += f;
        }
      }
      fid += (double)fcol;
      // x of this column is stored: count the frame; the last frame of (q, i)
      // in iteration k queues T_{k+1}(q, i) (the prior term alone at k = K)
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        const int i = col % c.Nx;
        const unsigned old = atomicAdd(c.colcnt + i, 1u);
        if (old + 1 == (unsigned)c.Nt) {
          atomicExch(c.colcnt + i, 0u);
          __threadfence();
          last = 1;
        }
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (lane == 0) mbar_arrive(&yc_empty[bb]);
      return !last || push(q, col % c.Nx, k);
    };
    // np: next column to prepare (at most kRSlots ahead of the epilogues, the
    // r / b buffers being double-buffered); ne: next epilogue.  Lane 0 polls
    // both barriers; a wall-clock limit on idle time ends the loop with
    // DEV_ERR_TIMEOUT.
    int np = 0, ne = 0;
    unsigned long long idle0 = 0;
    unsigned spins = 0;
    while (ne < ncol) {
      int act = 0;
      if (lane == 0) {
        // test_wait never suspends: a suspended try_wait on one barrier could
        // hold back the other, which may be the one its phase depends on
        if (np < ncol && np < ne + kRSlots &&
            mbar_test_wait(&rfull[np % kPersistRSlots], (uint32_t)((np / kPersistRSlots) & 1)))
          act = 1;
        else if (ne < np && mbar_test_wait(&col_done[ne & 1], (uint32_t)((ne >> 1) & 1)))
          act = 2;
        else {
          __nanosleep(32);
          if ((++spins & 255u) == 0) {
            if (*((volatile int*)&P.err[FLAG_ERR]) != 0) act = 3;
            const unsigned long long now = global_ns();
            if (idle0 == 0) idle0 = now;
            else if (now - idle0 > kWaitLimitNs) { atomicOr(&P.err[FLAG_ERR], DEV_ERR_TIMEOUT); act = 3; }
          }
        }
        if (act == 1 || act == 2) { idle0 = 0; spins = 0; }
      }
      act = __shfl_sync(0xffffffffu, act, 0);
      if (act == 1) {
        prepare(np++);
      } else if (act == 2) {
        if (!epilogue(ne++)) break;
      } else if (act == 3) {
        break;
      }
    }
    if (fid_slice >= 0 && sl[fid_slice].do_obj) {
      fid = warp_sum(fid);
      if (lane == 0) atomicAdd(sl[fid_slice].trace_fid + fid_k, fid);
    }
    return;
  }
  if (warp >= kTWarp0) {
    // ---------------- temporal warps: T_{k+1} of the columns this CTA completed --
    const int ttid = tid - 32 * kTWarp0;
    float* segA = reinterpret_cast<float*>(smem + PL.segA);
    float2* segB = reinterpret_cast<float2*>(smem + PL.segB);
    float2* bnd = reinterpret_cast<float2*>(smem + PL.bnd);
    double* red = reinterpret_cast<double*>(smem + PL.red);
    volatile int4* task_sm = reinterpret_cast<volatile int4*>(red + 28);   // the task, shared by the 128 threads
    for (;;) {
      // thread 0 takes a ticket and waits for its entry; the outcome is shared
      // so all temporal threads take the same path through the named
      // barriers.  Exactly tq_total tasks are produced in a launch; a ticket
      // beyond that ends this CTA's temporal work.  A wait can legitimately
      // last long in a long solve, so its limit runs from the last task
      // produced anywhere (the queue tail), not from the start of the wait.
      if (ttid == 0) {
        int4 task = make_int4(-1, 0, 0, 0);
        const unsigned h = atomicAdd(P.tq_head, 1u);
        if (h < P.tq_total) {
          int4* e = P.tq_ring + (h & (P.tq_cap - 1));
          unsigned* tag = reinterpret_cast<unsigned*>(&e->w);
          unsigned seen = ld_acquire_u32(P.tq_tail);
          unsigned long long t0 = global_ns();
          bool got = false;
          for (unsigned it = 0;; ++it) {
            if (ld_acquire_u32(tag) == h + 1u) { got = true; break; }
            __nanosleep(128);
            if ((it & 63u) == 63u) {
              if (*((volatile int*)&P.err[FLAG_ERR]) != 0) break;
              const unsigned tail = ld_acquire_u32(P.tq_tail);
              const unsigned long long now = global_ns();
              if (tail != seen) { seen = tail; t0 = now; }
              else if (now - t0 > kWaitLimitNs) { atomicOr(&P.err[FLAG_ERR], DEV_ERR_TIMEOUT); break; }
            }
          }
          if (got) {
            task = make_int4(__ldcg(&e->x), __ldcg(&e->y), __ldcg(&e->z), 0);
            st_release_u32(tag, 0u);   // the slot is free for entry h + cap
          }
        }
        task_sm->x = task.x; task_sm->y = task.y; task_sm->z = task.z;
      }
      tbar();
      const int4 task = make_int4(task_sm->x, task_sm->y, task_sm->z, 0);
      tbar();
      if (task.x < 0) break;
      __threadfence();   // order this thread's reads of x, m, d1, p after the task's acquire
      persist_temporal(sl[task.x], task.y & 0xFFFFF, task.y >> 20, task.z, K, ttid, segA, segB, bnd, red);
    }
    return;
  }

  // ---------------- consumers (as in k_col_inverse) --------------------------
  const int dlr = lane >> 2, dlc = lane & 3;
  const bool diag_has = dlr <= 2 * dlc + 1;
  const int diag_off = diag_has ? (dlc * (dlc + 1) + dlr) * 2 : 0;
  int u = warp, st = warp;
  uint32_t ph = 0;
  for (int n = 0; n < ncol; ++n) {
    const PersistSlice& c = sl[WSL(n % nw)];
    const int bb = n & 1;
    if (!mbar_wait(&rv_full[bb], (uint32_t)((n >> 1) & 1), P.err)) break;
    if (n >= 2 && !mbar_wait(&yc_empty[bb], (uint32_t)(((n >> 1) - 1) & 1), P.err)) break;
    const float2* rv = rvec + (size_t)bb * ny32m;
    float2* yw = ycopy + ((size_t)bb * kConsumerWarps + warp) * ny32m;
    bool failed = false;
    const int rot = unit_rotation(n, c.nunits);
    for (; u < c.nunits; u += kConsumerWarps) {
      if (!mbar_wait(&full[st], ph, P.err)) { failed = true; break; }
      const int4 un = decode_unit(rotated_unit(u, rot, c.nunits), c.nb, tiles);
      const E* tl = reinterpret_cast<const E*>(ring + (size_t)st * kStage);
      if (un.x == UNIT_TILE) proc_tile<E>(tl, rv, yw, un.y, un.z, lane, &empty[st], 64, lane * 2, true);
      else proc_tile<E>(tl, rv, yw, un.y, un.z, lane, &empty[st], 2 * kDiagLanes, diag_off, diag_has);
      st += kConsumerWarps;
      if (st >= S) { st -= S; ph ^= 1u; }
    }
    if (failed) break;
    u -= c.nunits;
    if (lane == 0) mbar_arrive(&col_done[bb]);
  }
#undef WSL
#undef WCOL
}

size_t persist_smem(int stages, int nb_max, int nslices, int work_max) {
  return persist_layout(stages, nb_max, nslices, work_max).total;
}

int persist_max_stages(int nb_max, int nslices, int work_max) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int qn = col_consumer_warps(8);
  int s = 8 * qn;
  while (s > qn) {
    if (persist_smem(s, nb_max, nslices, work_max) + 1024 <= (size_t)optin) break;
    s -= qn;
  }
  return (persist_smem(s, nb_max, nslices, work_max) + 1024 <= (size_t)optin) ? s : 0;
}

cudaError_t launch_persist_tv(const PersistLaunch& p, int grid, cudaStream_t s) {
  const size_t smem = persist_smem(p.stages, p.nb_max, p.nslices, p.work_max);
  static SmemAttrCache smem_attr;
  {
    const cudaError_t e = smem_attr.ensure(reinterpret_cast<const void*>(k_persist_tv), smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(persist_threads());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: the dataflow waits all end
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_persist_tv, p);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace recon
