// Kahan's compensated summation of FP32 terms: the error of a sum of n terms
// is about 2 eps instead of n eps.  Per-thread partial sums of the reductions
// use it before the FP64 sum across threads.
#pragma once

namespace recon {

struct KahanSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float y) {
    const float t = y - c;
    const float u = s + t;
    c = (u - s) - t;
    s = u;
  }
};

}  // namespace recon
