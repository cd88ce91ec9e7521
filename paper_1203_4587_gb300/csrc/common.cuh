// Device-side helpers shared by the reconstruction kernels (sm_103a).
//
// Complex numbers are float2 {re, im} in FP32 (double2 in the FP64 plan).
// The mbarrier / bulk-copy wrappers are inline PTX; every wait is bounded by a
// wall-clock limit read from %globaltimer and reports RECON_DEV_ERR_TIMEOUT in
// a device status word instead of hanging.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace recon {

// ---- device status word bits (flags[1]) -----------------------------------
enum : int {
  DEV_ERR_TIMEOUT = 1,      // a bounded wait gave up
  DEV_ERR_NOT_PD = 2,       // plan: a Gram block was not positive definite
  DEV_ERR_NONFINITE = 4,    // non-finite value met in a reduction
  DEV_ERR_BOUNDS = 8,       // an index check failed (skipped the access)
};
// flags[] layout: [0] stop, [1] error bits, [2] iterations done at stop
enum : int { FLAG_STOP = 0, FLAG_ERR = 1, FLAG_ITERS = 2, FLAG_COUNT = 4 };

// 2 s: far above any legitimate wait inside one launch.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---- complex helpers --------------------------------------------------------
__host__ __device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void c_fma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void c_fmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
// |a| as the correctly rounded sqrt of the FP32 sum of squares (no overflow
// or underflow concerns at the magnitudes of the reconstruction)
__device__ __forceinline__ float c_abs(float2 a) { return __fsqrt_rn(fmaf(a.x, a.x, a.y * a.y)); }
__device__ __forceinline__ double c_abs2d(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }

// Complex soft threshold S(a, tau) = (|a| - tau) a / |a| if |a| > tau, else 0.
__device__ __forceinline__ float2 c_soft(float2 a, float tau) {
  float mag = __fsqrt_rn(fmaf(a.x, a.x, a.y * a.y));
  if (!(mag > tau)) return make_float2(0.f, 0.f);
  float s = (mag - tau) / mag;
  return make_float2(a.x * s, a.y * s);
}

// double2 helpers (plan)
__device__ __forceinline__ double2 z_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 z_mulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ void z_fma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void z_fmac(double2& acc, double2 a, double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// double2 overloads with the float2 names, so templated code (the FFT) works
// on either precision.
__host__ __device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 c_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) { return z_mul(a, b); }
__device__ __forceinline__ void c_fma(double2& acc, double2 a, double2 b) { z_fma(acc, a, b); }
__device__ __forceinline__ void c_fmac(double2& acc, double2 a, double2 b) { z_fmac(acc, a, b); }
template <typename T> __device__ __forceinline__ T c_zero();
template <> __device__ __forceinline__ float2 c_zero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 c_zero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 to_f2(double2 z) { return make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ float2 to_f2(float2 z) { return z; }
template <typename T> __device__ __forceinline__ T from_f2(float2 v);
template <> __device__ __forceinline__ float2 from_f2<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 from_f2<double2>(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double c_abs2d(double2 a) { return a.x * a.x + a.y * a.y; }

// Per-frame scale of 16-bit storage: the power of two 2^e with
// maxabs / 2^e in [2^14, 2^15), so the largest component keeps the full FP16
// mantissa and cannot overflow (FP16 max 65504), and dividing by the scale is
// exact.  maxabs <= 0 or non-finite gives 1.
__host__ __device__ inline float pow2_frame_scale(float maxabs) {
  if (!(maxabs > 0.f) || !(maxabs < 3.0e38f)) return 1.f;
  int e = 0;
  frexpf(maxabs, &e);          // maxabs = f 2^e, f in [0.5, 1)
  if (e < -100) e = -100;
  return ldexpf(1.f, e - 15);
}

// ---- storage element types (FP32 complex, or 16-bit complex pairs) --------
struct c32 { float2 v; };
struct c16h { __half2 v; };
struct c16b { __nv_bfloat162 v; };

template <typename E> struct Elem;
template <> struct Elem<float2> {
  static constexpr int bytes = 8;
  using S = float;   // one component
  __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static S cvt1(double v) { return (float)v; }
  __device__ __forceinline__ static float widen1(S v) { return v; }
  // two adjacent elements in one 16-byte load (p 16-byte aligned), not widened
  __device__ __forceinline__ static void load2raw(const float2* p, float2& a, float2& b) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    a = make_float2(q.x, q.y); b = make_float2(q.z, q.w);
  }
  __device__ __forceinline__ static float2 widen(float2 v) { return v; }
  __device__ __forceinline__ static float2 load(const float2* p) { return *p; }
  __device__ __forceinline__ static void load2(const float2* p, float2& a, float2& b) {
    float4 q = *reinterpret_cast<const float4*>(p);
    a = make_float2(q.x, q.y); b = make_float2(q.z, q.w);
  }
  __device__ __forceinline__ static float2 cvt(double2 z) { return make_float2((float)z.x, (float)z.y); }
  __device__ __forceinline__ static float2 cvt(float2 z) { return z; }
};
template <> struct Elem<__half2> {
  static constexpr int bytes = 4;
  using S = __half;
  __device__ __forceinline__ static __half2 zero() { return __float2half2_rn(0.f); }
  __device__ __forceinline__ static S cvt1(double v) { return __double2half(v); }
  __device__ __forceinline__ static float widen1(S v) { return __half2float(v); }
  __device__ __forceinline__ static void load2raw(const __half2* p, __half2& a, __half2& b) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    a = *reinterpret_cast<const __half2*>(&q.x); b = *reinterpret_cast<const __half2*>(&q.y);
  }
  __device__ __forceinline__ static float2 widen(__half2 v) { return __half22float2(v); }
  __device__ __forceinline__ static float2 load(const __half2* p) { return __half22float2(*p); }
  __device__ __forceinline__ static void load2(const __half2* p, float2& a, float2& b) {
    uint2 q = *reinterpret_cast<const uint2*>(p);
    __half2 h0 = *reinterpret_cast<__half2*>(&q.x), h1 = *reinterpret_cast<__half2*>(&q.y);
    a = __half22float2(h0); b = __half22float2(h1);
  }
  __device__ __forceinline__ static __half2 cvt(double2 z) {   // one rounding from FP64
    return __halves2half2(__double2half(z.x), __double2half(z.y));
  }
  __device__ __forceinline__ static __half2 cvt(float2 z) { return __floats2half2_rn(z.x, z.y); }
};
template <> struct Elem<__nv_bfloat162> {
  static constexpr int bytes = 4;
  using S = __nv_bfloat16;
  __device__ __forceinline__ static __nv_bfloat162 zero() { return __float2bfloat162_rn(0.f); }
  __device__ __forceinline__ static S cvt1(double v) { return __double2bfloat16(v); }
  __device__ __forceinline__ static float widen1(S v) { return __bfloat162float(v); }
  __device__ __forceinline__ static void load2raw(const __nv_bfloat162* p, __nv_bfloat162& a, __nv_bfloat162& b) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    a = *reinterpret_cast<const __nv_bfloat162*>(&q.x); b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
  }
  __device__ __forceinline__ static float2 widen(__nv_bfloat162 v) { return __bfloat1622float2(v); }
  __device__ __forceinline__ static float2 load(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
  __device__ __forceinline__ static void load2(const __nv_bfloat162* p, float2& a, float2& b) {
    uint2 q = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 h0 = *reinterpret_cast<__nv_bfloat162*>(&q.x), h1 = *reinterpret_cast<__nv_bfloat162*>(&q.y);
    a = __bfloat1622float2(h0); b = __bfloat1622float2(h1);
  }
  __device__ __forceinline__ static __nv_bfloat162 cvt(double2 z) {   // one rounding from FP64
    return __halves2bfloat162(__double2bfloat16(z.x), __double2bfloat16(z.y));
  }
  __device__ __forceinline__ static __nv_bfloat162 cvt(float2 z) { return __floats2bfloat162_rn(z.x, z.y); }
};

// Packed FP32x2 arithmetic on pairs held in one 64-bit register (two
// independent round-to-nearest operations per instruction).
struct f32x2 { unsigned long long v; };
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
  return r;
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {   // a * b + c
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}

// ---- programmatic dependent launch ------------------------------------------
// A grid launched with cudaLaunchAttributeProgrammaticStreamSerialization may
// start while the previous kernel of its stream is still running.
// pdl_wait(): the calling thread waits until the grids this one depends on
// have completed and their memory operations are visible (returns at once
// for a grid launched without the attribute).  pdl_trigger(): this CTA lets
// the next such grid be scheduled once every CTA has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// cudaLaunchKernelEx with the programmatic-dependency attribute when `pdl`.
template <typename... Args>
inline cudaError_t launch_ex(void (*kern)(Args...), int grid, int threads, size_t smem, cudaStream_t s, bool pdl,
                             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- timers, barriers ------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Non-blocking test of an mbarrier phase (never suspends the thread), for a
// thread that polls several barriers in turn.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and sets DEV_ERR_TIMEOUT)
// when the wall-clock limit passes, or false when another CTA already
// reported an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flags,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*((volatile int*)&flags[FLAG_ERR]) != 0) return false;
      if (global_ns() - t0 > limit_ns) { atomicOr(&flags[FLAG_ERR], DEV_ERR_TIMEOUT); return false; }
    }
  }
}

// L2 policy for data read exactly once per pass (the packed inverses).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 1D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}

// 8-byte asynchronous global -> shared copy (LDGSTS); completes at cp_async_wait().
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

struct BlockBar {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// ---- reductions --------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum2(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}
// Sum `v` over `nthreads` threads (a multiple of 32) that all call this with
// the same `scratch` (>= 32 doubles of shared memory).  The result is valid
// in thread 0 of the group.  `sync` synchronises exactly those threads.
template <class Sync>
__device__ double group_sum(double v, double* scratch, int tid, int nthreads, Sync sync) {
  v = warp_sum(v);
  int w = tid >> 5, lane = tid & 31;
  if (lane == 0) scratch[w] = v;
  sync();
  double s = 0.0;
  if (tid < 32) {
    s = (tid < (nthreads >> 5)) ? scratch[tid] : 0.0;
    s = warp_sum(s);
  }
  sync();
  return s;
}

}  // namespace recon
