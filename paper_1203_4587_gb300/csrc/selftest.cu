// Self-test of the failure path of the bounded device-side waits.
//
// Every hand-off inside the persistent kernels is an mbarrier phase wait with
// a wall-clock limit (mbar_wait, common.cuh): when the limit passes the wait
// sets DEV_ERR_TIMEOUT in the launch's error word and returns, the kernel
// winds down, and the host reports RECON_ERR_TIMEOUT with the context still
// usable.  recon_selftest_wait_timeout exercises exactly that path without a
// fault: one CTA waits, through the same mbar_wait, on a phase of a
// shared-memory barrier that nothing ever arrives at, with a short limit.
#include <chrono>

#include "plan.h"

namespace recon {

namespace {

__global__ void k_wait_selftest(int* flags, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);   // one arrival would complete phase 0; none comes
    fence_mbar_init();
  }
  __syncthreads();
  // flags[FLAG_COUNT]: the wait returned without its phase (the kernel's own record)
  if (!mbar_wait(&bar, 0u, flags, limit_ns) && threadIdx.x == 0) atomicOr(&flags[FLAG_COUNT], 1);
}

}  // namespace

}  // namespace recon

using namespace recon;

extern "C" {

recon_status recon_selftest_wait_timeout(int limit_us, double* waited_ms, void* stream) {
  if (limit_us < 1 || limit_us > 2000000) return fail(RECON_ERR_INVALID_ARG, "limit_us must be in 1..2000000");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* flags = nullptr;   // the error words of a launch, plus the kernel's record
  RC(cudaMalloc(&flags, (FLAG_COUNT + 1) * sizeof(int)));
  cudaError_t e = cudaMemsetAsync(flags, 0, (FLAG_COUNT + 1) * sizeof(int), s);
  const auto t0 = std::chrono::steady_clock::now();
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(flags, (unsigned long long)limit_us * 1000ull);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const auto t1 = std::chrono::steady_clock::now();
  int h[FLAG_COUNT + 1] = {};
  if (e == cudaSuccess) e = cudaMemcpy(h, flags, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(flags);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (waited_ms) *waited_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if ((h[FLAG_ERR] & DEV_ERR_TIMEOUT) && h[FLAG_COUNT]) return fail(RECON_ERR_TIMEOUT, "a bounded device-side wait timed out");
  return fail(RECON_ERR_CUDA, "the self-test wait did not report a timeout");
}

}  // extern "C"
