// Pieces of the column-inverse kernels (x = A r per column, Section IV-C,
// Eq. eigen_mu) shared by the per-iteration kernel (iter_kernels.cu) and the
// persistent solve (persist_kernels.cu): warp roles, the packed-unit decoder,
// the Hermitian block product of one 32x32 unit and the shared-memory layout.
#pragma once

#include "kernels.h"

namespace recon {

// consumer warps: 8 at FP32; 12 for the 16-bit streams, whose consumers do
// the same arithmetic per element on half the bytes and need more warps in
// flight to hide their latency (the smaller ring leaves the shared memory)
__host__ __device__ constexpr int col_consumer_warps(int esize) { return esize == 8 ? 8 : 12; }
// producer warps (one issuing thread each): 2 for 8-byte elements, 4 for
// the half-size units of 16-bit storage (more copies per byte)
__host__ __device__ constexpr int col_producers(int esize) { return esize == 8 ? 2 : 4; }
// consumers + producers + r loader + column manager
__host__ __device__ constexpr int col_threads(int esize) {
  return 32 * (col_consumer_warps(esize) + col_producers(esize) + 2);
}
// A ring stage holds the largest unit of the storage type: kTileElems
// elements of esize bytes (8 FP32, 4 FP16/BF16; both multiples of 16 bytes).
__host__ __device__ constexpr int stage_bytes(int esize) { return kTileElems * esize; }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// One 32x32 block (rows p*32.., cols q*32..): lane (lr, lc) holds rows
// lr*4..+3 and cols lc*8..+7, and each element e at (R, C) adds e r_C to
// y_R and conj(e) r_R to y_C.  For an off-diagonal block (p < q) that is its
// product and the product of its conjugate transpose (the lower triangle);
// for a diagonal block (p == q, zeros below the diagonal, the diagonal
// halved, 12 lanes without elements) it is the block's Hermitian product.
// Row sums are reduced over the 4 lanes sharing lr, column sums over the 8
// lanes sharing lc, by butterfly exchanges that leave one total per lane.
// Lane data of pair qq sit at qq*qstride + loff (kernels.h).
template <typename E>
__device__ __forceinline__ void proc_tile(const E* __restrict__ tl, const float2* __restrict__ r,
                                          float2* __restrict__ yw, int p, int q, int lane, uint64_t* release,
                                          int qstride, int loff, bool has) {
  const int lr = lane >> 2, lc = lane & 3;
  // the whole unit into registers first, then the ring stage goes back to the
  // producer while this warp computes
  E el[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) el[k] = Elem<E>::zero();
  if (has) {
#pragma unroll
    for (int qq = 0; qq < 16; ++qq) Elem<E>::load2raw(tl + qq * qstride + loff, el[2 * qq], el[2 * qq + 1]);
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(release);
  float2 rv[4], cv[8];
  {
    const float4* r4 = reinterpret_cast<const float4*>(r + p * 32 + lr * 4);
    float4 a0 = r4[0], a1 = r4[1];
    rv[0] = make_float2(a0.x, a0.y); rv[1] = make_float2(a0.z, a0.w);
    rv[2] = make_float2(a1.x, a1.y); rv[3] = make_float2(a1.z, a1.w);
    const float4* c4 = reinterpret_cast<const float4*>(r + q * 32 + lc * 8);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 c = c4[k];
      cv[2 * k] = make_float2(c.x, c.y); cv[2 * k + 1] = make_float2(c.z, c.w);
    }
  }
  // Planar pairs: el[2qq] = (re_c, re_c+1), el[2qq+1] = (im_c, im_c+1) of row
  // ri = qq/4, columns c = 2(qq%4), c+1.  Packed FP32x2 FMAs accumulate
  //   row ri:         e_c cv_c over the two columns  (Re = re cx - im cy, Im = re cy + im cx)
  //   columns c, c+1: conj(e_c) rv_ri                (Re = re rv.x + im rv.y, Im = re rv.y - im rv.x)
  // with the subtracted products in their own accumulators.
  f32x2 cx[4], cy[4], rx[4], ry[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cx[k] = pack2(cv[2 * k].x, cv[2 * k + 1].x);
    cy[k] = pack2(cv[2 * k].y, cv[2 * k + 1].y);
    rx[k] = pack2(rv[k].x, rv[k].x);
    ry[k] = pack2(rv[k].y, rv[k].y);
  }
  const f32x2 z2 = pack2(0.f, 0.f);
  f32x2 rre[4], rren[4], rim[4], cre[4], cim[4], cimn[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { rre[k] = rren[k] = rim[k] = cre[k] = cim[k] = cimn[k] = z2; }
#pragma unroll
  for (int qq = 0; qq < 16; ++qq) {
    const float2 ref = Elem<E>::widen(el[2 * qq]), imf = Elem<E>::widen(el[2 * qq + 1]);
    const f32x2 re = pack2(ref.x, ref.y), im = pack2(imf.x, imf.y);
    const int ri = qq >> 2, cp = qq & 3;
    rre[ri] = ffma2(re, cx[cp], rre[ri]);
    rren[ri] = ffma2(im, cy[cp], rren[ri]);
    rim[ri] = ffma2(re, cy[cp], rim[ri]);
    rim[ri] = ffma2(im, cx[cp], rim[ri]);
    cre[cp] = ffma2(re, rx[ri], cre[cp]);
    cre[cp] = ffma2(im, ry[ri], cre[cp]);
    cim[cp] = ffma2(re, ry[ri], cim[cp]);
    cimn[cp] = ffma2(im, rx[ri], cimn[cp]);
  }
  float2 rowp[4], colp[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 a = unpack2(rre[k]), an = unpack2(rren[k]), b = unpack2(rim[k]);
    rowp[k] = make_float2((a.x - an.x) + (a.y - an.y), b.x + b.y);
    const float2 c = unpack2(cre[k]), d = unpack2(cim[k]), dn = unpack2(cimn[k]);
    colp[2 * k] = make_float2(c.x, d.x - dn.x);
    colp[2 * k + 1] = make_float2(c.y, d.y - dn.y);
  }
  // rows: lanes differing in bits 0,1
  const bool b1 = (lc & 2) != 0, b0 = (lc & 1) != 0;
  float2 k0 = b1 ? rowp[2] : rowp[0], s0 = b1 ? rowp[0] : rowp[2];
  float2 k1 = b1 ? rowp[3] : rowp[1], s1 = b1 ? rowp[1] : rowp[3];
  k0 = c_add(k0, shfl_xor2(s0, 2));
  k1 = c_add(k1, shfl_xor2(s1, 2));
  float2 kr = b0 ? k1 : k0, sr = b0 ? k0 : k1;
  kr = c_add(kr, shfl_xor2(sr, 1));
  // columns: lanes differing in bits 2,3,4
  const bool c2 = (lr & 4) != 0, c1 = (lr & 2) != 0, cb = (lr & 1) != 0;
  float2 h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 keep = c2 ? colp[k + 4] : colp[k], send = c2 ? colp[k] : colp[k + 4];
    h[k] = c_add(keep, shfl_xor2(send, 16));
  }
  float2 g[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float2 keep = c1 ? h[k + 2] : h[k], send = c1 ? h[k] : h[k + 2];
    g[k] = c_add(keep, shfl_xor2(send, 8));
  }
  float2 kc = cb ? g[1] : g[0], sc = cb ? g[0] : g[1];
  kc = c_add(kc, shfl_xor2(sc, 4));
  float2* yr = yw + p * 32 + lane;            // row lr*4 + lc == lane
  *yr = c_add(*yr, kr);
  float2* yc = yw + q * 32 + lc * 8 + lr;      // column lc*8 + lr
  *yc = c_add(*yc, kc);
  __syncwarp();
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kRSlots = 2;  // double-buffered r inputs / partial sums

// Units of the n-th column a CTA processes are taken in an order rotated by
// 3n: with few units per column the diagonal units (the smaller ones, at the
// end of a column's stream) would otherwise fall on the same consumer warps
// in every column.  Producers and consumers agree on the order; the unit ->
// warp / stage mapping by position is unchanged.
__device__ __forceinline__ int unit_rotation(int n, int nunits) { return (int)((3ll * n) % nunits); }

// Unit m of a column with nb blocks, in stream order: {kind, p, q, element
// offset}.  Off-diagonal tiles (bj, bk), bj < bk, bk-major (an order that
// does not depend on nb, so one table of (bj | bk << 8) for the largest nb
// of a launch serves every slice), then the diagonal blocks (the packed
// layout of kernels.h).
__device__ __forceinline__ int tile_pq(int m) {   // the table's entry m, computed once per launch
  int bk = (int)((1.f + sqrtf(1.f + 8.f * (float)m)) * 0.5f);   // bk(bk-1)/2 <= m < bk(bk+1)/2
  while (bk * (bk - 1) / 2 > m) --bk;
  while ((bk + 1) * bk / 2 <= m) ++bk;
  return (m - bk * (bk - 1) / 2) | (bk << 8);
}
__device__ __forceinline__ int4 decode_unit(int m, int nb, const int* tiles) {
  const int ntiles = nb * (nb - 1) / 2;
  if (m < ntiles) {
    const int pq = tiles[m];
    return make_int4(UNIT_TILE, pq & 0xff, pq >> 8, m * kTileElems);
  }
  const int d = m - ntiles;
  return make_int4(UNIT_DIAG, d, d, ntiles * kTileElems + d * kDiagElems);
}

__device__ __forceinline__ int rotated_unit(int pos, int rot, int nunits) {
  const int u = pos + rot;
  return u >= nunits ? u - nunits : u;
}

struct ColLayout {
  size_t bars, ring, ycopy, rvec, bvec, rslot, tiles, slices, skip, work, total;
};
__host__ __device__ inline ColLayout col_layout(int stages, int nb, int nslices, int work_max, int esize) {
  ColLayout L;
  const size_t ny32 = (size_t)nb * 32;
  size_t o = 0;
  // full[S], empty[S], rfull[2], rempty[2], rv_full[2], yc_empty[2], col_done[2]
  L.bars = o; o += (2 * (size_t)stages + 5 * kRSlots) * 8;
  o = align_up(o, 128);
  L.ring = o; o += (size_t)stages * stage_bytes(esize);
  o = align_up(o, 16);
  L.ycopy = o; o += (size_t)kRSlots * col_consumer_warps(esize) * ny32 * 8;   // [buf][warp][ny32]
  L.rvec = o; o += (size_t)kRSlots * ny32 * 8;
  L.bvec = o; o += (size_t)kRSlots * ny32 * 8;
  L.rslot = o; o += (size_t)kRSlots * 3 * ny32 * 8;   // [slot][base, add, b][ny32]
  L.tiles = o; o += (size_t)(nb * (nb - 1) / 2) * 4;   // (bj | bk << 8) of the off-diagonal tiles
  o = align_up(o, 16);
  L.slices = o; o += (size_t)nslices * sizeof(ColSlice);
  o = align_up(o, 16);
  L.skip = o; o += (size_t)nslices * 4;
  L.work = o; o += (size_t)work_max * 4;
  L.total = align_up(o, 128);
  return L;
}

}  // namespace recon
