// Per-iteration kernels of Algorithms 1 and 2.
//
// k_col_inverse  x_{i,t} = A_{i,t} r_{i,t} for every column (Section IV-C,
//                Eq. eigen_mu; Algorithm 2 x-update, Algorithm 1 w-update),
//                with the data term of J(k) for the new x fused into the
//                epilogue (Eq. r_ratio needs J(k)).
// k_tv_temporal  v, m and d1 updates of Algorithm 2 along t for every pixel.
// k_dft_temporal v-update, dual and Psi / Psi' of Algorithm 1 along t.
// k_objective    ||y - Hx||^2 of a given field (J(0)).
// k_finalize     J(k) = fid + lambda * prior, Delta(k) and the stop flag.
#include "colinv.cuh"
#include "tv_chunk.cuh"

namespace recon {

// ||y - H x||^2 of one column (i, t) whose values are in shared memory:
// for each coil, z = F_v(s_c . x) (unitary, batched FFT of `ncg` coils at a
// time) compared with the hybrid data F_h'y on the sampled rows.  By
// Parseval on F_h this is the column's share of ||y - Hx||^2.
template <class YE, class Bar>
__device__ double column_fid(const float2* xcol, int i, int t, int Nx, int Ny, int Nc, int ncg,
                             const float2* __restrict__ sens, const YE* __restrict__ yhat, const float* yscale,
                             const int* __restrict__ rows, const int* __restrict__ rowoff, const FftPlanDev& fy,
                             float scl, float2* fa, float2* fb, int tid, int nthr, Bar bar) {
  const int r0 = rowoff[t], mt = rowoff[t + 1] - r0;
  const int* rw = rows + r0;
  const YE* yh = yhat + (size_t)r0 * Nx * Nc + (size_t)i * Nc * mt;
  const float2* sc = sens + (size_t)i * Nc * Ny;
  const float ys = yscale ? yscale[t] : 1.f;
  double acc = 0.0;
  for (int c0 = 0; c0 < Nc; c0 += ncg) {
    const int cg = min(ncg, Nc - c0);
    for (int idx = tid; idx < cg * Ny; idx += nthr) {
      const int c = idx / Ny, j = idx - c * Ny;
      fa[idx] = c_mul(__ldg(sc + (size_t)(c0 + c) * Ny + j), xcol[j]);
    }
    bar();
    float2* res = fft_run(fa, fb, cg, Ny, 1, fy, false, tid, nthr, bar);
    for (int idx = tid; idx < cg * mt; idx += nthr) {
      const int c = idx / mt, m = idx - c * mt;
      float2 z = c_scale(res[c * Ny + rw[m]], scl);
      float2 d = c_sub(c_scale(Elem<YE>::load(yh + (size_t)(c0 + c) * mt + m), ys), z);
      acc += c_abs2d(d);
    }
    bar();
  }
  return acc;
}

// Persistent column-inverse kernel over a work list of (slice, column) pairs,
// warp-specialised and free of block-wide barriers in the main loop (all
// hand-offs are bounded mbarrier waits):
//   warps 0..C-1  consumers (C = 8 at FP32, 12 at 16 bit): Hermitian matvec
//            of each unit into their own partial y vector of buffer n&1,
//            column after column
//   warps C..C+P-1  producers (P = 2 at FP32, 4 at 16 bit): stream the
//            packed inverses with the TMA engine (cp.async.bulk, L2
//            evict_first) into a ring of S stages
//   warp C+P  r loader: bulk-copies each column's right-hand-side inputs
//   warp C+P+1  column manager: r = base + coef*add into rvec[n&1]; after
//            the consumers are done, x = sum of the C partial y vectors,
//            store, objective dot products, clear the partials
// Columns of slices whose stop flag is set are dropped from the work list
// (every role reads the same snapshot of the flags).
template <typename E>
__global__ void __launch_bounds__(col_threads(Elem<E>::bytes), 1) k_col_inverse(ColLaunch P) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kProducers = col_producers(Elem<E>::bytes);
  constexpr int kConsumerWarps = col_consumer_warps(Elem<E>::bytes);
  constexpr int kStage = stage_bytes(Elem<E>::bytes);
  const ColLayout L = col_layout(P.stages, P.nb_max, P.nslices, P.work_max, Elem<E>::bytes);
  const int S = P.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + S;
  uint64_t* rfull = empty + S;
  uint64_t* rempty = rfull + kRSlots;
  uint64_t* rv_full = rempty + kRSlots;
  uint64_t* yc_empty = rv_full + kRSlots;
  uint64_t* col_done = yc_empty + kRSlots;
  unsigned char* ring = smem + L.ring;
  const int ny32m = P.nb_max * 32;   // buffer stride (largest slice)
  float2* ycopy = reinterpret_cast<float2*>(smem + L.ycopy);
  float2* rvec = reinterpret_cast<float2*>(smem + L.rvec);
  float2* bvec = reinterpret_cast<float2*>(smem + L.bvec);
  float2* rslot = reinterpret_cast<float2*>(smem + L.rslot);
  ColSlice* sl = reinterpret_cast<ColSlice*>(smem + L.slices);
  int* tiles = reinterpret_cast<int*>(smem + L.tiles);
  int* skip = reinterpret_cast<int*>(smem + L.skip);
  unsigned* wl = reinterpret_cast<unsigned*>(smem + L.work);   // this CTA's work list

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int m = tid; m < P.nb_max * (P.nb_max - 1) / 2; m += blockDim.x) tiles[m] = tile_pq(m);
  for (int q = tid; q < P.nslices; q += blockDim.x) {
    sl[q] = P.slices[q];
    skip[q] = P.slices[q].stop ? *P.slices[q].stop : 0;
  }
  for (int j = tid; j < kRSlots * kConsumerWarps * ny32m; j += blockDim.x) ycopy[j] = make_float2(0.f, 0.f);
  {
    const int a = P.work_off[blockIdx.x], b = P.work_off[blockIdx.x + 1];
    for (int w = a + tid; w < b; w += blockDim.x) wl[w - a] = P.work[w];
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int s = 0; s < kRSlots; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], 1);
      mbar_init(&rv_full[s], 1);
      mbar_init(&yc_empty[s], 1);
      mbar_init(&col_done[s], kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  // Launched after the temporal step with a programmatic dependency, the
  // producers start streaming the packed inverses (which no earlier kernel
  // writes) at once; every other role waits for the previous kernel before it
  // reads or writes the iteration's state.  The stop flags read above change
  // only with a stopping test, where the engine launches without the
  // dependency.  The next kernel may be scheduled as soon as every CTA runs.
  pdl_trigger();
  constexpr int ES = Elem<E>::bytes;
  const int w0 = 0, w1 = P.work_off[blockIdx.x + 1] - P.work_off[blockIdx.x];
  // work entry: slice in the high byte, column in the low 24 bits
#define WSL(w) ((int)(wl[w] >> 24))
#define WCOL(w) ((int)(wl[w] & 0xFFFFFFu))

  if (warp >= kConsumerWarps && warp < kConsumerWarps + kProducers) {
    // ---------------- producers: stream packed inverses into the ring -------
    // Producer p issues the units whose index (counted across this CTA's
    // columns) is p mod kProducers, into stage (index mod S): one issuing
    // thread streams a bulk copy every ~150 ns at best, which would limit
    // the 2.5-4 KB units of 16-bit storage, so the issue work is split.  S is
    // a multiple of kProducers, so each producer owns a fixed set of stages.
    if (lane == 0) {
      const int p = warp - kConsumerWarps;
      const uint64_t pol = policy_evict_first();
      // stage st of the ring, wraps = completed passes over the ring (no
      // divisions on the issue path)
      int st = p, wraps = 0, gu = 0, issued = 0, ncolumn = 0;
      bool ok = true;
      for (int w = w0; w < w1 && ok; ++w) {
        if (skip[WSL(w)]) continue;
        const ColSlice& c = sl[WSL(w)];
        const unsigned char* cb = reinterpret_cast<const unsigned char*>(c.A) +
                                  (size_t)packed_index(WCOL(w), c.Nx, c.Nt) * (size_t)c.col_elems * ES;
        const int rot = unit_rotation(ncolumn++, c.nunits);
        // first position of this column whose global index is p mod kProducers
        int u = p - gu % kProducers;
        if (u < 0) u += kProducers;
        for (; u < c.nunits; u += kProducers) {
          if (wraps > 0 && !mbar_wait(&empty[st], (uint32_t)((wraps - 1) & 1), P.err)) { ok = false; break; }
          const int4 un = decode_unit(rotated_unit(u, rot, c.nunits), c.nb, tiles);
          const uint32_t bytes = (uint32_t)((un.x == UNIT_TILE ? kTileElems : kDiagElems) * ES);
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(ring + (size_t)st * kStage, cb + (size_t)un.w * ES, bytes, &full[st], pol);
          ++issued;
          st += kProducers;
          if (st >= S) { st -= S; ++wraps; }
        }
        gu += c.nunits;
      }
      if (!ok) {
        // error path: let this producer's copies still in flight land before
        // the CTA exits (its k-th copy filled stage (p + k*P) mod S for the
        // ((p + k*P) / S)-th time)
        const int per = S / kProducers;
        for (int k = (issued > per ? issued - per : 0); k < issued; ++k) {
          const long long gi = p + (long long)k * kProducers;
          uint64_t* bb = &full[gi % S];
          const uint32_t par = (uint32_t)((gi / S) & 1);
          unsigned long long t0 = global_ns();
          while (!mbar_try_wait(bb, par) && global_ns() - t0 < kWaitLimitNs) {}
        }
      }
    }
    return;
  }
  pdl_wait();
  if (warp == kConsumerWarps + kProducers) {
    // ---------------- r loader: each column's inputs into a slot -------------
    // With 16-byte aligned columns (Ny even) lane 0 moves them with the TMA
    // engine; otherwise all lanes load them and lane 0 arrives after a warp
    // sync (the slot barrier always expects one arrival).
    int n = 0;
    for (int w = w0; w < w1; ++w) {
      if (skip[WSL(w)]) continue;
      const ColSlice& c = sl[WSL(w)];
      const bool sep_b = c.do_obj && c.bsrc != c.base;
      const int slt = n % kRSlots;
      if (n >= kRSlots && !mbar_wait(&rempty[slt], (uint32_t)(((n / kRSlots) - 1) & 1), P.err)) break;
      float2* d = rslot + (size_t)slt * 3 * ny32m;
      const size_t cofs = (size_t)WCOL(w) * c.Ny;
      if (c.r_tma) {
        if (lane == 0) {
          const uint32_t bytes = (uint32_t)c.Ny * 8u;
          const uint32_t total = bytes * (1u + (c.add ? 1u : 0u) + (sep_b ? 1u : 0u));
          const uint64_t pol = policy_evict_first();
          mbar_arrive_expect_tx(&rfull[slt], total);
          bulk_g2s(d, c.base + cofs, bytes, &rfull[slt], pol);
          if (c.add) bulk_g2s(d + ny32m, c.add + cofs, bytes, &rfull[slt], pol);
          if (sep_b) bulk_g2s(d + 2 * ny32m, c.bsrc + cofs, bytes, &rfull[slt], pol);
        }
      } else {
        for (int j0 = 0; j0 < c.Ny; j0 += 32 * 8) {
          float2 va[8], vb[8], vc[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + q * 32 + lane;
            if (j < c.Ny) {
              va[q] = c.base[cofs + j];
              if (c.add) vb[q] = c.add[cofs + j];
              if (sep_b) vc[q] = c.bsrc[cofs + j];
            }
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + q * 32 + lane;
            if (j < c.Ny) {
              d[j] = va[q];
              if (c.add) d[ny32m + j] = vb[q];
              if (sep_b) d[2 * ny32m + j] = vc[q];
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rfull[slt]);
      }
      ++n;
    }
    if (lane == 0) {
      // copies of the last slots may still be in flight if the kernel quits early
      for (int h = (n > kRSlots ? n - kRSlots : 0); h < n; ++h) {
        unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&rfull[h % kRSlots], (uint32_t)((h / kRSlots) & 1)) && global_ns() - t0 < kWaitLimitNs) {}
      }
    }
    return;
  }

  // the columns this CTA processes (after dropping stopped slices)
  int ncol = 0;
  for (int w = w0; w < w1; ++w) ncol += skip[WSL(w)] ? 0 : 1;

  if (warp == kConsumerWarps + kProducers + 1) {
    // ---------------- column manager -----------------------------------------
    // walks the work list twice, in step: `wp` for prepare(n), `we` for the epilogue
    int wp = w0, we = w0;
    auto next_col = [&](int& w) -> int2 {
      while (skip[WSL(w)]) ++w;
      const int2 r = make_int2(WSL(w), WCOL(w));
      ++w;
      return r;
    };
    // prepare(n): rvec[n&1] = base + coef*add (zero padded), bvec[n&1] = b
    auto prepare = [&](int n) -> bool {
      const int2 wk = next_col(wp);
      const ColSlice& c = sl[wk.x];
      const bool sep_b = c.do_obj && c.bsrc != c.base;
      const int ny32 = c.nb * 32;
      const int slt = n % kRSlots;
      if (!mbar_wait(&rfull[slt], (uint32_t)((n / kRSlots) & 1), P.err)) return false;
      const float2* d = rslot + (size_t)slt * 3 * ny32m;
      float2* rv = rvec + (size_t)(n & 1) * ny32m;
      float2* bv = bvec + (size_t)(n & 1) * ny32m;
      // two elements per lane and 16-byte accesses (all buffers are 16-byte
      // aligned and ny32 is even); elements past Ny are zero padding
      for (int j = 2 * lane; j < ny32; j += 64) {
        float4 v = *reinterpret_cast<const float4*>(d + j);
        float4 bb = sep_b ? *reinterpret_cast<const float4*>(d + 2 * ny32m + j) : v;
        if (c.add) {
          const float4 a = *reinterpret_cast<const float4*>(d + ny32m + j);
          v.x = fmaf(c.coef, a.x, v.x); v.y = fmaf(c.coef, a.y, v.y);
          v.z = fmaf(c.coef, a.z, v.z); v.w = fmaf(c.coef, a.w, v.w);
        }
        if (j >= c.Ny) { v.x = v.y = 0.f; bb.x = bb.y = 0.f; }
        if (j + 1 >= c.Ny) { v.z = v.w = 0.f; bb.z = bb.w = 0.f; }
        *reinterpret_cast<float4*>(rv + j) = v;
        *reinterpret_cast<float4*>(bv + j) = bb;
      }
      __syncwarp();
      if (lane == 0) { mbar_arrive(&rempty[slt]); mbar_arrive(&rv_full[n & 1]); }
      return true;
    };
    double fid = 0.0;
    int fid_slice = -1;
    bool ok = true;
    for (int n = 0; n < ncol && n < kRSlots && ok; ++n) ok = prepare(n);
    for (int n = 0; n < ncol && ok; ++n) {
      const int bb = n & 1;
      const int2 wk = next_col(we);
      const ColSlice& c = sl[wk.x];
      if (!mbar_wait(&col_done[bb], (uint32_t)((n >> 1) & 1), P.err)) break;
      if (wk.x != fid_slice) {
        // results of one slice go to that slice's accumulator
        if (fid_slice >= 0 && sl[fid_slice].do_obj) {
          const double f = warp_sum(fid);
          if (lane == 0) atomicAdd(sl[fid_slice].fid_acc, f);
        }
        fid = 0.0;
        fid_slice = wk.x;
      }
      const int ny32 = c.nb * 32;
      const size_t cofs = (size_t)wk.y * c.Ny;
      float2* yc = ycopy + (size_t)bb * kConsumerWarps * ny32m;
      const float2* rv = rvec + (size_t)bb * ny32m;
      const float2* bv = bvec + (size_t)bb * ny32m;
      // per element in FP32 (GB300's FP64 rate is a small fraction of FP32),
      // summed per lane over the column in FP32 and added once to the FP64
      // accumulator: w_bx Re<b, x> + w_xr Re<x, r> + w_xx |x|^2
      float fcol = 0.f;
      const bool vec_out = ((cofs & 1) == 0);   // 16-byte aligned pairs of x
      for (int j = 2 * lane; j < ny32; j += 64) {
        float4 x = *reinterpret_cast<const float4*>(yc + j);
        *reinterpret_cast<float4*>(yc + j) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 1; w < kConsumerWarps; ++w) {
          float4* pw = reinterpret_cast<float4*>(yc + (size_t)w * ny32m + j);
          const float4 t = *pw;
          x.x += t.x; x.y += t.y; x.z += t.z; x.w += t.w;
          *pw = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (j + 1 < c.Ny && vec_out) {
          *reinterpret_cast<float4*>(c.xout + cofs + j) = x;
        } else {
          if (j < c.Ny) c.xout[cofs + j] = make_float2(x.x, x.y);
          if (j + 1 < c.Ny) c.xout[cofs + j + 1] = make_float2(x.z, x.w);
        }
        if (c.do_obj) {   // only elements < Ny (r and b are zero past Ny; x need not be)
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
      __syncwarp();
      if (lane == 0) mbar_arrive(&yc_empty[bb]);
      if (n + kRSlots < ncol) ok = prepare(n + kRSlots);
    }
    if (fid_slice >= 0 && sl[fid_slice].do_obj) {
      fid = warp_sum(fid);
      if (lane == 0) atomicAdd(sl[fid_slice].fid_acc, fid);
    }
    return;
  }

  // ---------------- consumers (C warps) --------------------------------------
  // Unit g (counted across this CTA's columns) belongs to warp g mod C, so a
  // warp walks g = warp, warp+C, ...: within column n that is unit index u,
  // and its ring stage advances by C per unit.  With S a multiple of C the
  // previous fill of a stage was consumed by this same warp, so every parity
  // wait is at most one phase ahead of its barrier.  Every column's rv/yc
  // barriers are waited on (and col_done arrived at) even when the warp has
  // no unit in that column, for the same reason.
  // this lane's place in a diagonal unit: patch (lr, lc) is stored when it
  // meets the upper triangle
  const int dlr = lane >> 2, dlc = lane & 3;
  const bool diag_has = dlr <= 2 * dlc + 1;
  const int diag_off = diag_has ? (dlc * (dlc + 1) + dlr) * 2 : 0;
  int u = warp, st = warp;
  uint32_t ph = 0;
  int w = w0;
  for (int n = 0; n < ncol; ++n) {
    while (skip[WSL(w)]) ++w;
    const ColSlice& c = sl[WSL(w)];
    ++w;
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

size_t col_inverse_smem(int stages, int nb_max, int nslices, int work_max, int esize) {
  return col_layout(stages, nb_max, nslices, work_max, esize).total;
}

// Largest ring depth that fits, a multiple of the consumer warp count (the
// parity waits rely on it; see the consumer loop).
int col_inverse_max_stages(int nb_max, int nslices, int work_max, int esize) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int q = col_consumer_warps(esize);
  int s = 8 * q;
  while (s > q) {
    if (col_inverse_smem(s, nb_max, nslices, work_max, esize) + 1024 <= (size_t)optin) break;
    s -= q;
  }
  return s;
}

int col_inverse_stage_quantum(int esize) { return col_consumer_warps(esize); }

cudaError_t prepare_col_inverse(int storage, size_t smem) {
  static SmemAttrCache c32, c16, cb16;
  switch (storage) {
    case 0: return c32.ensure(reinterpret_cast<const void*>(k_col_inverse<float2>), smem);
    case 1: return c16.ensure(reinterpret_cast<const void*>(k_col_inverse<__half2>), smem);
    case 2: return cb16.ensure(reinterpret_cast<const void*>(k_col_inverse<__nv_bfloat162>), smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col_inverse(const ColLaunch& p, int storage, int grid, cudaStream_t s, bool pdl) {
  const size_t smem = col_inverse_smem(p.stages, p.nb_max, p.nslices, p.work_max, storage ? 4 : 8);
  cudaError_t e = prepare_col_inverse(storage, smem);
  if (e != cudaSuccess) return e;
  switch (storage) {
    case 0: e = launch_ex(k_col_inverse<float2>, grid, col_threads(8), smem, s, pdl, p); break;
    case 1: e = launch_ex(k_col_inverse<__half2>, grid, col_threads(4), smem, s, pdl, p); break;
    case 2: e = launch_ex(k_col_inverse<__nv_bfloat162>, grid, col_threads(4), smem, s, pdl, p); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// Slice of a temporal launch's block (binary search over the slices' first blocks).
template <typename SliceT>
__device__ __forceinline__ int find_slice(const SliceT* sl, int n, int blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sl[mid].tile0 <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Algorithm 2 temporal step (v-, m- and d1-updates along t) for every pixel:
// one block of kTvChunkThreads threads per chunk of kTvChunkPx consecutive
// pixels (the column layout keeps them contiguous in every frame), all values
// in registers (tv_chunk.cuh).  LMAX >= ceil(Nt / kTvSeg) frames per
// segment.  Also accumulates ||D_t x||_1 of the incoming x (the prior term of
// J): FP32 per thread and across each warp, one FP64 value per warp (GB300's
// FP64 pipe is too narrow for a conversion per thread).
// ---------------------------------------------------------------------------
// Blocks an SM by frames a segment: up to 4 frames, 8 blocks (64 registers)
// hide the load latency best; 5 frames keep 6 blocks (80 registers), 6 frames
// 5 (96); more frames need the registers.
constexpr int tv_min_blocks(int lmax) { return lmax <= 4 ? 8 : lmax == 5 ? 6 : lmax == 6 ? 5 : 1; }
template <int LMAX, bool FULL>
__global__ void __launch_bounds__(kTvChunkThreads, tv_min_blocks(LMAX)) k_tv_temporal(TemporalLaunch L) {
  __shared__ float seg_a[kTvChunkThreads];
  __shared__ float2 seg_b[kTvChunkThreads];
  __shared__ float2 bnd[kTvChunkThreads];
  __shared__ double red[kTvChunkThreads / 32];
  // launched after the inverse step with a programmatic dependency: wait for
  // it (x, and the stop flag), then let the next inverse step be scheduled
  pdl_wait();
  pdl_trigger();
  const TvSlice* sls = static_cast<const TvSlice*>(L.slices);
  const TvSlice& P = sls[find_slice(sls, L.nslices, (int)blockIdx.x)];
  if (P.stop && *P.stop) return;
  const long long pix0 = (long long)(blockIdx.x - P.tile0) * kTvChunkPx;
  TvChunkIO io;
  io.x = P.x;
  io.m = P.m;
  io.d1 = P.d1;
  io.p = P.p;
  io.m_out = P.m_out;
  io.d1_out = P.d1_out;
  io.p_out = P.p_out;
  io.thomas = P.thomas;
  io.tau1 = P.tau1;
  io.rho = P.rho;
  io.Nt = P.Nt;
  io.fstride = (size_t)P.npix;
  io.base = (size_t)pix0;
  io.nvalid = (int)min((long long)kTvChunkPx, P.npix - pix0);
  io.write = P.write_state != 0;
  float tvf;
  if (FULL) {
    tvf = tv_chunk<LMAX, true>(io, (int)threadIdx.x, seg_a, seg_b, bnd, BlockBar());
  } else {
    // a launch over slices of several Nt (a batch): a whole chunk of a slice
    // with Nt = 8 l takes the whole-chunk code for its own l (the same
    // arithmetic), the rest the general code
    const int l = (P.Nt % kTvSeg == 0) ? P.Nt / kTvSeg : 0;
    const bool whole = io.nvalid == kTvChunkPx && io.d1 != nullptr && io.write;
    const int tid = (int)threadIdx.x;
    if (whole && l == LMAX && LMAX <= kTvFullLMax) tvf = tv_chunk<LMAX, true>(io, tid, seg_a, seg_b, bnd, BlockBar());
    else if (whole && l == LMAX - 1 && LMAX - 1 >= 1 && LMAX <= kTvFullLMax)
      tvf = tv_chunk<(LMAX > 1 ? LMAX - 1 : 1), true>(io, tid, seg_a, seg_b, bnd, BlockBar());
    else if (whole && l == LMAX - 2 && LMAX - 2 >= 1 && LMAX <= kTvFullLMax)
      tvf = tv_chunk<(LMAX > 2 ? LMAX - 2 : 1), true>(io, tid, seg_a, seg_b, bnd, BlockBar());
    else if (whole && l == LMAX - 3 && LMAX - 3 >= 1 && LMAX <= kTvFullLMax)
      tvf = tv_chunk<(LMAX > 3 ? LMAX - 3 : 1), true>(io, tid, seg_a, seg_b, bnd, BlockBar());
    else tvf = tv_chunk<LMAX, false>(io, tid, seg_a, seg_b, bnd, BlockBar());
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tvf += __shfl_down_sync(0xffffffffu, tvf, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)tvf;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kTvChunkThreads / 32; ++w) s += red[w];
    atomicAdd(P.prior_acc, s);
  }
}

constexpr size_t kSmemOptin = 227 * 1024;
// one chunk width; the frames-per-segment array covers Nt <= 128
int tv_tile_candidates(int Nt_max, int* out) {
  (void)Nt_max;
  out[0] = kTvChunkPx;
  return 1;
}
int tv_tile_px(int Nt_max) {
  (void)Nt_max;
  return kTvChunkPx;
}
cudaError_t prepare_tv_temporal(int Nt_max, int px) {   // static shared memory only
  return (px == kTvChunkPx && Nt_max <= 16 * kTvSeg) ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tv_temporal(const TemporalLaunch& p, cudaStream_t s, bool pdl) {
  cudaError_t e = prepare_tv_temporal(p.Nt_max, p.tile_px);
  if (e != cudaSuccess) return e;
  const int ls = (p.Nt_max + kTvSeg - 1) / kTvSeg;
  const int nb = p.nblocks, nt = kTvChunkThreads;
  if (p.full) {   // every chunk whole (set by the engine): the specialised instantiation
    switch (ls) {
      case 1: e = launch_ex(k_tv_temporal<1, true>, nb, nt, 0, s, pdl, p); break;
      case 2: e = launch_ex(k_tv_temporal<2, true>, nb, nt, 0, s, pdl, p); break;
      case 3: e = launch_ex(k_tv_temporal<3, true>, nb, nt, 0, s, pdl, p); break;
      case 4: e = launch_ex(k_tv_temporal<4, true>, nb, nt, 0, s, pdl, p); break;
      case 5: e = launch_ex(k_tv_temporal<5, true>, nb, nt, 0, s, pdl, p); break;
      case 6: e = launch_ex(k_tv_temporal<6, true>, nb, nt, 0, s, pdl, p); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (ls <= 1) e = launch_ex(k_tv_temporal<1, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 2) e = launch_ex(k_tv_temporal<2, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 3) e = launch_ex(k_tv_temporal<3, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 4) e = launch_ex(k_tv_temporal<4, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 5) e = launch_ex(k_tv_temporal<5, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 6) e = launch_ex(k_tv_temporal<6, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 8) e = launch_ex(k_tv_temporal<8, false>, nb, nt, 0, s, pdl, p);
  else if (ls <= 12) e = launch_ex(k_tv_temporal<12, false>, nb, nt, 0, s, pdl, p);
  else e = launch_ex(k_tv_temporal<16, false>, nb, nt, 0, s, pdl, p);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1 temporal step for 64 pixels per block (tile [Nt][64] in shared
// memory, batched Stockham along t):
//   w = Psi xhat,  d = u - w  (d = 0 at k = 1),  v = S(w - d, lambda/(2 mu)),
//   u' = v + d,  r = H'y + mu Psi'(u')
// so the inverse step gives xhat' = A r and Psi xhat' is the new w.  Because
// Psi is unitary, the (I - Psi Psi') term of the w-update is zero.  Also
// accumulates ||w||_1 (the prior term of J at the incoming iterate).
// ---------------------------------------------------------------------------
static size_t dft_smem(int Nt_max, int px) { return 2 * (size_t)Nt_max * px * sizeof(float2); }
int dft_tile_px() { return 64; }
int dft_tile_candidates(int Nt_max, int* out) {
  int n = 0;
  for (int px : {16, 32, 64, 128})
    if (dft_smem(Nt_max, px) + 1024 <= kSmemOptin) out[n++] = px;
  return n;
}

template <int kDftPix>
__global__ void __launch_bounds__(256) k_dft_temporal(TemporalLaunch L) {
  extern __shared__ float2 sm_dft[];
  __shared__ double red[32];
  pdl_wait();      // launched with a programmatic dependency on the inverse step
  pdl_trigger();
  const DftSlice* sls = static_cast<const DftSlice*>(L.slices);
  const DftSlice& P = sls[find_slice(sls, L.nslices, (int)blockIdx.x)];
  if (P.stop && *P.stop) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nt = P.Nt;
  float2* A = sm_dft;
  float2* B = sm_dft + (size_t)Nt * kDftPix;
  const long long N = P.npix;
  const long long pix0 = (long long)(blockIdx.x - P.tile0) * kDftPix;
  const int npx = (int)min((long long)kDftPix, N - pix0);
  for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
    const int t = idx / kDftPix, pp = idx - t * kDftPix;
    if (pp < npx) cp_async8(&A[idx], P.xh + t * N + pix0 + pp);
    else A[idx] = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  const BlockBar bar;
  float2* W = fft_run(A, B, kDftPix, 1, kDftPix, P.ft, false, tid, nth, bar);
  float2* O = (W == A) ? B : A;
  const float sc = rsqrtf((float)Nt);
  double l1 = 0.0;   // per element in FP64: the sum does not depend on the tile width
  for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
    const int t = idx / kDftPix, pp = idx - t * kDftPix;
    float2 uo = make_float2(0.f, 0.f);
    if (pp < npx) {
      const float2 w = c_scale(W[idx], sc);
      l1 += (double)c_abs(w);
      if (P.write_state) {
        const float2 d = P.first ? make_float2(0.f, 0.f) : c_sub(P.u[t * N + pix0 + pp], w);
        const float2 v = c_soft(c_sub(w, d), P.tau);
        uo = c_add(v, d);
        P.u_out[t * N + pix0 + pp] = uo;
      }
    }
    O[idx] = uo;
  }
  __syncthreads();
  if (P.write_state) {
    float2* S = fft_run(O, W, kDftPix, 1, kDftPix, P.ft, true, tid, nth, bar);
    const float ms = P.mu * sc;
    for (int idx = tid; idx < Nt * kDftPix; idx += nth) {
      const int t = idx / kDftPix, pp = idx - t * kDftPix;
      if (pp < npx) {
        const float2 bb = P.b[t * N + pix0 + pp];
        const float2 sv = S[idx];
        P.r_out[t * N + pix0 + pp] = make_float2(fmaf(ms, sv.x, bb.x), fmaf(ms, sv.y, bb.y));
      }
    }
  }
  const double s = group_sum(l1, red, tid, nth, bar);
  if (tid == 0) atomicAdd(P.prior_acc, s);
}

cudaError_t prepare_dft_temporal(int Nt_max, int px) {
  static SmemAttrCache c[4];
  const size_t smem = dft_smem(Nt_max, px);
  switch (px) {
    case 16: return c[0].ensure(reinterpret_cast<const void*>(k_dft_temporal<16>), smem);
    case 32: return c[1].ensure(reinterpret_cast<const void*>(k_dft_temporal<32>), smem);
    case 64: return c[2].ensure(reinterpret_cast<const void*>(k_dft_temporal<64>), smem);
    case 128: return c[3].ensure(reinterpret_cast<const void*>(k_dft_temporal<128>), smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_dft_temporal(const TemporalLaunch& p, cudaStream_t s, bool pdl) {
  cudaError_t e = prepare_dft_temporal(p.Nt_max, p.tile_px);
  if (e != cudaSuccess) return e;
  const size_t smem = dft_smem(p.Nt_max, p.tile_px);
  switch (p.tile_px) {
    case 16: e = launch_ex(k_dft_temporal<16>, p.nblocks, 256, smem, s, pdl, p); break;
    case 32: e = launch_ex(k_dft_temporal<32>, p.nblocks, 256, smem, s, pdl, p); break;
    case 64: e = launch_ex(k_dft_temporal<64>, p.nblocks, 256, smem, s, pdl, p); break;
    default: e = launch_ex(k_dft_temporal<128>, p.nblocks, 256, smem, s, pdl, p); break;
  }
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1 with the undecimated temporal Haar frame (a redundant tight
// frame; Section IV-A's lemma with its (1/mu)(I - Psi Psi') term), on a tile
// of PX pixels x Nt frames held in shared memory:
//   w = u_prev + Psi (xhat - Psi'u_prev)   (w = Psi b at k = 1)
//   d = u_prev - w (0 at k = 1);  v = S(w - d, lambda/(2 mu));  u = v + d
//   s = Psi'u;  r = b + mu s  (the inverse step then gives xhat = A r)
// Psi: a_0 = z, a_j[t] = (a_{j-1}[t] + a_{j-1}[t+s]) / 2,
//      d_j[t] = (a_{j-1}[t] - a_{j-1}[t+s]) / 2 with s = 2^(j-1) mod Nt;
// Psi': a_{j-1}[t] = (a_j[t] + a_j[t-s]) / 2 + (d_j[t] - d_j[t-s]) / 2.
// Also accumulates ||w||_1 (the prior term of J).
// ---------------------------------------------------------------------------
static size_t haar_smem(int Nt_max, int levels, int px) {
  return (size_t)(levels + 3) * Nt_max * px * sizeof(float2);   // L+1 channels, two approximations
}
int haar_tile_candidates(int Nt_max, int levels, int* out) {
  int n = 0;
  for (int px : {16, 32, 64})
    if (haar_smem(Nt_max, levels, px) + 1024 <= kSmemOptin) out[n++] = px;
  return n;
}
int haar_tile_px(int Nt_max, int levels) {
  int c[4];
  const int n = haar_tile_candidates(Nt_max, levels, c);
  for (int i = n - 1; i >= 0; --i)
    if (c[i] <= 32) return c[i];
  return n ? c[0] : 16;
}

template <int PX>
__global__ void __launch_bounds__(256) k_haar_temporal(TemporalLaunch L, int levels) {
  extern __shared__ __align__(16) float2 sm_h[];
  __shared__ double red[32];
  pdl_wait();      // launched with a programmatic dependency on the inverse step
  pdl_trigger();
  const HaarSlice* sls = static_cast<const HaarSlice*>(L.slices);
  const HaarSlice& P = sls[find_slice(sls, L.nslices, (int)blockIdx.x)];
  if (P.stop && *P.stop) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nt = P.Nt, T = Nt * PX, nch = levels + 1;
  const long long N = P.npix;
  const long long pix0 = (long long)(blockIdx.x - P.tile0) * PX;
  const int npx = (int)min((long long)PX, N - pix0);
  float2* W = sm_h;                          // [L+1][Nt][PX] channels
  float2* A0 = W + (size_t)nch * T;          // approximations (ping-pong)
  float2* A1 = A0 + T;
  const BlockBar bar;
  // z = xhat - Psi'u_prev (b at k = 1)
  for (int idx = tid; idx < T; idx += nth) {
    const int t = idx / PX, pp = idx - t * PX;
    float2 z = make_float2(0.f, 0.f);
    if (pp < npx) {
      const long long g = t * N + pix0 + pp;
      z = P.first ? P.b[g] : c_sub(P.xh[g], P.s[g]);
    }
    A0[idx] = z;
  }
  bar();
  // analysis into W
  float2* a = A0;
  float2* an = A1;
  int sh = 1 % Nt;
  for (int j = 1; j <= levels; ++j) {
    for (int idx = tid; idx < T; idx += nth) {
      const int t = idx / PX, pp = idx - t * PX;
      int tn = t + sh;
      if (tn >= Nt) tn -= Nt;
      const float2 cur = a[idx], nxt = a[tn * PX + pp];
      W[(size_t)(j - 1) * T + idx] = c_scale(c_sub(cur, nxt), 0.5f);
      an[idx] = c_scale(c_add(cur, nxt), 0.5f);
    }
    bar();
    float2* tmp = a; a = an; an = tmp;
    sh = (2 * sh) % Nt;
  }
  for (int idx = tid; idx < T; idx += nth) W[(size_t)levels * T + idx] = a[idx];
  bar();
  // w, ||w||_1 (per element in FP64: independent of the tile width), the v- and d-updates
  double l1 = 0.0;
  const size_t NU = (size_t)Nt * N;          // one channel of u in global memory
  for (int idx = tid; idx < nch * T; idx += nth) {
    const int c = idx / T, rem = idx - c * T;
    const int t = rem / PX, pp = rem - t * PX;
    float2 uo = make_float2(0.f, 0.f);
    if (pp < npx) {
      const size_t g = (size_t)c * NU + (size_t)t * N + pix0 + pp;
      const float2 up = P.first ? make_float2(0.f, 0.f) : P.u[g];
      const float2 w = c_add(up, W[idx]);
      l1 += (double)c_abs(w);
      if (P.write_state) {
        const float2 d = P.first ? make_float2(0.f, 0.f) : c_sub(up, w);
        const float2 v = c_soft(c_sub(w, d), P.tau);
        uo = c_add(v, d);
        P.u_out[g] = uo;
      }
    }
    W[idx] = uo;
  }
  bar();
  if (P.write_state) {
    // synthesis s = Psi'u from the channels now holding u
    a = A0;
    an = A1;
    for (int idx = tid; idx < T; idx += nth) a[idx] = W[(size_t)levels * T + idx];
    int shl = 1 % Nt;
    for (int j = 1; j < levels; ++j) shl = (2 * shl) % Nt;   // shift of level L
    bar();
    for (int j = levels; j >= 1; --j) {
      const float2* dj = W + (size_t)(j - 1) * T;
      for (int idx = tid; idx < T; idx += nth) {
        const int t = idx / PX, pp = idx - t * PX;
        int tp = t - shl;
        if (tp < 0) tp += Nt;
        const int jdx = tp * PX + pp;
        const float2 lo = c_scale(c_add(a[idx], a[jdx]), 0.5f);
        const float2 hi = c_scale(c_sub(dj[idx], dj[jdx]), 0.5f);
        an[idx] = c_add(lo, hi);
      }
      bar();
      float2* tmp = a; a = an; an = tmp;
      // shift of level j-1 (2^(j-2) mod Nt), recomputed from 1 to stay exact mod Nt
      shl = 1 % Nt;
      for (int k = 1; k < j - 1; ++k) shl = (2 * shl) % Nt;
    }
    const float ms = P.mu;
    for (int idx = tid; idx < T; idx += nth) {
      const int t = idx / PX, pp = idx - t * PX;
      if (pp < npx) {
        const long long g = t * N + pix0 + pp;
        const float2 sv = a[idx], bb = P.b[g];
        P.s_out[g] = sv;
        P.r_out[g] = make_float2(fmaf(ms, sv.x, bb.x), fmaf(ms, sv.y, bb.y));
      }
    }
  }
  const double sum = group_sum(l1, red, tid, nth, bar);
  if (tid == 0) atomicAdd(P.prior_acc, sum);
}

cudaError_t prepare_haar_temporal(int Nt_max, int levels, int px) {
  static SmemAttrCache c[3];
  const size_t smem = haar_smem(Nt_max, levels, px);
  if (smem + 1024 > kSmemOptin) return cudaErrorInvalidValue;
  switch (px) {
    case 16: return c[0].ensure(reinterpret_cast<const void*>(k_haar_temporal<16>), smem);
    case 32: return c[1].ensure(reinterpret_cast<const void*>(k_haar_temporal<32>), smem);
    case 64: return c[2].ensure(reinterpret_cast<const void*>(k_haar_temporal<64>), smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_haar_temporal(const TemporalLaunch& p, int levels, cudaStream_t s, bool pdl) {
  cudaError_t e = prepare_haar_temporal(p.Nt_max, levels, p.tile_px);
  if (e != cudaSuccess) return e;
  const size_t smem = haar_smem(p.Nt_max, levels, p.tile_px);
  switch (p.tile_px) {
    case 16: e = launch_ex(k_haar_temporal<16>, p.nblocks, 256, smem, s, pdl, p, levels); break;
    case 32: e = launch_ex(k_haar_temporal<32>, p.nblocks, 256, smem, s, pdl, p, levels); break;
    default: e = launch_ex(k_haar_temporal<64>, p.nblocks, 256, smem, s, pdl, p, levels); break;
  }
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||y - H x||^2 of a whole field, one block per column.
// ---------------------------------------------------------------------------
template <class YE>
__global__ void __launch_bounds__(256) k_objective(ObjParams P) {
  extern __shared__ float2 sm_obj[];
  __shared__ double red[32];
  if (P.flags[FLAG_STOP]) return;
  const int col = blockIdx.x, tid = threadIdx.x;
  const int t = col / P.Nx, i = col - t * P.Nx;
  float2* xc = sm_obj;
  float2* fa = xc + P.Ny;
  float2* fb = fa + (size_t)P.ncg * P.Ny;
  for (int j = tid; j < P.Ny; j += blockDim.x) xc[j] = P.x[(size_t)col * P.Ny + j];
  __syncthreads();
  const double f = column_fid(xc, i, t, P.Nx, P.Ny, P.Nc, P.ncg, P.sens, static_cast<const YE*>(P.yhat), P.yscale,
                              P.rows, P.rowoff, P.fy, rsqrtf((float)P.Ny), fa, fb, tid, blockDim.x, BlockBar());
  const double s = group_sum(f, red, tid, blockDim.x, BlockBar());
  if (tid == 0) atomicAdd(P.fid_acc, s);
}

// ---------------------------------------------------------------------------
// ||y - H x||^2 of a whole field with one warp per (column, coil): the
// vertical FFT z = F_v(s_c . x_col) of length Ny = 32 E runs in the warp's
// registers as a four-step transform, with no shared-memory passes and no
// block barriers.  Input n = l + 32 k (lane l holds k = 0..E-1), output
// f = q + E m:
//   1. an E-point DFT over k in each lane's registers;
//   2. the twiddle w_Ny^(l q);
//   3. a 32-point DFT over the lanes for every q (five radix-2
//      decimation-in-frequency stages with shuffles), after which lane l holds
//      m = bitrev5(l).
// Each output on a sampled row is compared with the hybrid data F_h'y.
// Twiddles w_Ny^j come from the FP64-computed table, staged in shared memory.
// ---------------------------------------------------------------------------
template <int N>
struct SmallestFactor {
  static constexpr int value = N % 2 == 0 ? 2 : N % 3 == 0 ? 3 : N % 5 == 0 ? 5 : N;
};

// In-register forward DFT of N values, x[f] = sum_n x[n] w_N^(n f), by
// recursive decimation in time over the smallest prime factor; w_N^j is
// tw[j * ts] (tw a table of a length that N divides, ts = length / N).
template <int N>
__device__ __forceinline__ void reg_dft(float2 (&x)[N], const float2* __restrict__ tw, int ts) {
  if constexpr (N > 1) {
    constexpr int R = SmallestFactor<N>::value, M = N / R;
    float2 s[R][M];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int m = 0; m < M; ++m) s[r][m] = x[m * R + r];
#pragma unroll
    for (int r = 0; r < R; ++r) reg_dft<M>(s[r], tw, ts * R);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = (r == 0 || k == 0) ? s[r][k] : c_mul(s[r][k], tw[r * k * ts]);
      if constexpr (R == 2) {
        x[k] = c_add(v[0], v[1]);
        x[k + M] = c_sub(v[0], v[1]);
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
          float2 acc = v[0];
#pragma unroll
          for (int r = 1; r < R; ++r) c_fma(acc, v[r], tw[((q * r) % R) * M * ts]);
          x[k + q * M] = acc;
        }
      }
    }
  }
}

__device__ __forceinline__ float2 shfl_xor_c(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <int E, class YE>
__global__ void __launch_bounds__(256) k_objective_warp(ObjParams P) {
  constexpr int Ny = 32 * E;
  __shared__ float2 tw[Ny];
  if (P.flags[FLAG_STOP]) return;
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) tw[j] = __ldg(P.fy.tw + j);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wglob = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int Nc = P.Nc, Nx = P.Nx;
  const long long ntask = (long long)P.Nt * Nx * Nc;
  const float scl = rsqrtf((float)Ny);
  const int mrow = (int)(__brev((unsigned)lane) >> 27);   // this lane's m after the lane DFT
  double acc = 0.0;
  for (long long task = wglob; task < ntask; task += nwarps) {
    const int c = (int)(task % Nc);
    const long long col = task / Nc;               // t * Nx + i
    const int t = (int)(col / Nx), i = (int)(col - (long long)t * Nx);
    const float2* xc = P.x + col * Ny;
    const float2* sc = P.sens + ((size_t)i * Nc + c) * Ny;
    float2 v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = c_mul(__ldg(sc + lane + 32 * k), __ldg(xc + lane + 32 * k));
    reg_dft<E>(v, tw, 32);
#pragma unroll
    for (int q = 1; q < E; ++q) v[q] = c_mul(v[q], tw[lane * q]);
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
      const bool hi = (lane & h) != 0;
      const float2 w = tw[(lane & (h - 1)) * (Ny / (2 * h))];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const float2 o = shfl_xor_c(v[q], h);
        v[q] = hi ? c_mul(c_sub(o, v[q]), w) : c_add(v[q], o);
      }
    }
    const int r0 = P.rowoff[t], mt = P.rowoff[t + 1] - r0;
    const YE* yh = static_cast<const YE*>(P.yhat) + (size_t)r0 * Nx * Nc + ((size_t)i * Nc + c) * mt;
    const float ys = P.yscale ? P.yscale[t] : 1.f;
    const short* ri = P.rowidx + (size_t)t * Ny;
    float part = 0.f;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int mi = ri[q + E * mrow];
      if (mi >= 0) {
        const float2 y = c_scale(Elem<YE>::load(yh + mi), ys);
        const float dx = y.x - v[q].x * scl, dy = y.y - v[q].y * scl;
        part = fmaf(dx, dx, fmaf(dy, dy, part));
      }
    }
    acc += (double)part;
  }
  acc = warp_sum(acc);
  if (lane == 0 && acc != 0.0) atomicAdd(P.fid_acc, acc);
}

// Ny = 32 E with E in this list: the warp kernel; other lengths: the block kernel
#define RECON_OBJ_WARP_SIZES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(16) X(20) X(24) X(32)

template <class YE>
static cudaError_t launch_objective_warp(const ObjParams& p, cudaStream_t s, bool* done) {
  *done = false;
  if (p.Ny % 32 != 0) return cudaSuccess;
  const int E = p.Ny / 32;
  const int grid = p.grid > 0 ? p.grid : 1024;
  switch (E) {
#define RECON_OBJ_CASE(e) \
    case e: k_objective_warp<e, YE><<<grid, 256, 0, s>>>(p); *done = true; break;
    RECON_OBJ_WARP_SIZES(RECON_OBJ_CASE)
#undef RECON_OBJ_CASE
    default: return cudaSuccess;
  }
  note_launch();
  return cudaGetLastError();
}

template <class YE>
static cudaError_t launch_objective_t(const ObjParams& p, cudaStream_t s) {
  {
    bool done = false;
    const cudaError_t e = launch_objective_warp<YE>(p, s, &done);
    if (e != cudaSuccess || done) return e;
  }
  const size_t smem = ((size_t)p.Ny + 2 * (size_t)p.ncg * p.Ny) * sizeof(float2);
  static SmemAttrCache attr;
  {
    const cudaError_t e = attr.ensure(reinterpret_cast<const void*>(k_objective<YE>), smem);
    if (e != cudaSuccess) return e;
  }
  k_objective<YE><<<p.Nx * p.Nt, 256, smem, s>>>(p); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_objective(const ObjParams& p, cudaStream_t s) {
  switch (p.ystorage) {
    case 0: return launch_objective_t<float2>(p, s);
    case 1: return launch_objective_t<__half2>(p, s);
    case 2: return launch_objective_t<__nv_bfloat162>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Per slice: J(k) = ||y - Hx||^2 + lambda * prior, Delta(k) (Eq. r_ratio) and
// the stop flag, for k = k0 .. k1 in order; later launches see the flag and
// skip that slice.  With the stop test on, the engine calls it once per
// iteration (k0 = k1); with a fixed iteration count, once after the loop.
// ---------------------------------------------------------------------------
__global__ void k_finalize(const FinSlice* fins, int n, int k0, int k1) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const FinSlice f = fins[q];
  int* flags = f.flags;
  for (int k = k0; k <= k1; ++k) {
    if (flags[FLAG_STOP]) return;
    const double Jk = f.fid[k] + ((f.yy && k > 0) ? *f.yy : 0.0) + (double)f.lam * f.prior[k];
    f.J[k] = Jk;
    if (!isfinite(Jk)) atomicOr(&flags[FLAG_ERR], DEV_ERR_NONFINITE);
    if (f.tol > 0.0 && k >= 1) {
      const double d = (f.J[k - 1] - Jk) / Jk;
      if (d >= 0.0 && d < f.tol) {
        flags[FLAG_ITERS] = k;
        flags[FLAG_STOP] = 1;
      }
    }
  }
}

cudaError_t launch_finalize(const FinSlice* fins, int nslices, int k0, int k1, cudaStream_t s) {
  k_finalize<<<(nslices + 127) / 128, 128, 0, s>>>(fins, nslices, k0, k1); note_launch();
  return cudaGetLastError();
}

}  // namespace recon
