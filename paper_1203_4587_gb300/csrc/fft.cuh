// Batched mixed-radix Stockham FFT in shared memory.
//
// Unitary DFTs appear in every step of the method: F_h and F_v of the forward
// model (Section II-A) and the temporal DFT Psi of Algorithm 1.  This header
// computes the unnormalised transform  X[q] = sum_n x[n] exp(-+2 pi i q n / N)
// for `cnt` sequences held in shared memory; callers apply 1/sqrt(N).
//
// Stockham autosort, decimation in time: with N = R_1 R_2 ... R_s and
// Ns = R_1...R_{k-1} before stage k, butterfly j (0 <= j < N/R) reads
// x[j + r N/R] (r < R), multiplies input r by w^(r (j mod Ns) N/(Ns R)),
// takes an R-point DFT and writes X[(j/Ns) Ns R + (j mod Ns) + q Ns].  The
// result is in natural order after the last stage (out of place, ping-pong).
// Radices 2 and 4 are hand-written; 3, 5, 7, 8 use a register DFT; any other
// factor (a large prime) uses a direct O(R^2) stage, so every length works.
//
// Twiddles come from one table per length, tw[k] = exp(-2 pi i k / N),
// computed on the host in FP64 (stored as FP32 for float2 transforms, as a
// double-float pair for dc).  The transform is templated on the complex type:
// float2 for the per-iteration work, dc (double-float, df64.cuh) for the
// once-per-solve H'y prologue, double2 where FP64 is wanted.
#pragma once

#include "common.cuh"
#include "df64.cuh"

namespace recon {

constexpr int kFftMaxStages = 24;

template <typename T>
struct FftPlanT {
  int n;
  int ns;
  int radix[kFftMaxStages];
  const T* tw;  // [n], exp(-2 pi i k / n)
};
using FftPlanDev = FftPlanT<float2>;
using FftPlanDev64 = FftPlanT<double2>;
using FftPlanDf = FftPlanT<dc>;

__device__ __forceinline__ float2 tw_get(const float2* tw, int k, bool inv) {
  float2 w = __ldg(tw + k);
  return inv ? make_float2(w.x, -w.y) : w;
}
__device__ __forceinline__ double2 tw_get(const double2* tw, int k, bool inv) {
  double2 w = __ldg(tw + k);
  return inv ? make_double2(w.x, -w.y) : w;
}
__device__ __forceinline__ dc tw_get(const dc* tw, int k, bool inv) {
  dc w = dc_unpack(__ldg(reinterpret_cast<const float4*>(tw) + k));
  if (inv) w.im = df_neg(w.im);
  return w;
}

// d * (-i) (forward) or d * (+i) (inverse): a swap and a sign, exact
__device__ __forceinline__ float2 mul_mi(float2 d, bool inv) {
  return inv ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
}
__device__ __forceinline__ double2 mul_mi(double2 d, bool inv) {
  return inv ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);
}
__device__ __forceinline__ dc mul_mi(dc d, bool inv) {
  return inv ? dc{df_neg(d.im), d.re} : dc{d.im, df_neg(d.re)};
}

template <int R, typename T>
__device__ __forceinline__ void bfly_reg(const T* __restrict__ in, T* __restrict__ out, int j, int nR,
                                         int Ns, int tws, int ks, const T* tw, int n, bool inv) {
  T v[R];
  const int k = j % Ns;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[(j + r * nR) * ks];
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw_get(tw, k * r * tws, inv));
  const int od = (j / Ns) * Ns * R + k;
  if (R == 2) {
    out[od * ks] = c_add(v[0], v[1]);
    out[(od + Ns) * ks] = c_sub(v[0], v[1]);
  } else if (R == 4) {
    T a = c_add(v[0], v[2]), b = c_sub(v[0], v[2]);
    T c = c_add(v[1], v[3]), d = c_sub(v[1], v[3]);
    const T di = mul_mi(d, inv);   // forward: d * (-i); inverse: d * (+i)
    out[od * ks] = c_add(a, c);
    out[(od + Ns) * ks] = c_add(b, di);
    out[(od + 2 * Ns) * ks] = c_sub(a, c);
    out[(od + 3 * Ns) * ks] = c_sub(b, di);
  } else {
    const int step = n / R;  // exp(-2 pi i / R) = tw[n / R]
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) c_fma(acc, v[r], tw_get(tw, ((q * r) % R) * step, inv));
      out[(od + q * Ns) * ks] = acc;
    }
  }
}

// Any radix, straight from shared memory (used for large prime factors).
template <typename T>
__device__ __forceinline__ void bfly_direct(const T* __restrict__ in, T* __restrict__ out, int R, int j,
                                            int nR, int Ns, int tws, int ks, const T* tw, int n, bool inv) {
  const int k = j % Ns;
  const int od = (j / Ns) * Ns * R + k;
  const int step = n / R;
  for (int q = 0; q < R; ++q) {
    T acc = c_zero<T>();
    for (int r = 0; r < R; ++r) {
      T x = in[(j + r * nR) * ks];
      if (r) x = c_mul(x, tw_get(tw, k * r * tws, inv));
      c_fma(acc, x, tw_get(tw, ((q * r) % R) * step, inv));
    }
    out[(od + q * Ns) * ks] = acc;
  }
}

// Runs the whole transform on `cnt` sequences: sequence s, element m lives at
// a[s * ss + m * ks].  `b` is scratch of the same shape.  `bar()` must
// synchronise exactly the `nthr` participating threads.  Returns the buffer
// that holds the result (a or b).
template <typename T, class Bar>
__device__ T* fft_run(T* a, T* b, int cnt, int ss, int ks, const FftPlanT<T>& P, bool inv, int tid, int nthr,
                      Bar bar) {
  const int n = P.n;
  int Ns = 1;
  for (int st = 0; st < P.ns; ++st) {
    const int R = P.radix[st];
    const int nR = n / R;
    const int tws = n / (Ns * R);
    const int total = cnt * nR;
    for (int idx = tid; idx < total; idx += nthr) {
      const int s = idx / nR;
      const int j = idx - s * nR;
      const T* in = a + s * ss;
      T* out = b + s * ss;
      switch (R) {
        case 2: bfly_reg<2>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        case 3: bfly_reg<3>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        case 4: bfly_reg<4>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        case 5: bfly_reg<5>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        case 7: bfly_reg<7>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        case 8: bfly_reg<8>(in, out, j, nR, Ns, tws, ks, P.tw, n, inv); break;
        default: bfly_direct(in, out, R, j, nR, Ns, tws, ks, P.tw, n, inv); break;
      }
    }
    bar();
    T* t = a; a = b; b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace recon
