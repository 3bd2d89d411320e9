// Device helpers shared by the all-pairs kernels (force and force-VJP).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody_internal.h"

namespace nbody {

// Hardware approximate reciprocal square root (MUFU), flush-to-zero input.
// rsqrt.approx.ftz.f32(+0) = +inf, which the self-pair mask turns into 0.
__device__ __forceinline__ float rsq_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Hardware approximate reciprocal (MUFU), flush-to-zero input; rcp(+0) = +inf.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Knuth's TwoSum: hi + lo absorbs t, with the rounding error of hi + t carried
// into lo (Knuth, TAOCP vol. 2, 4.2.2). Six float32 additions, no branches.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float t) {
  const float s = hi + t;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (t - bp);
  hi = s;
  lo += err;
}

// Persistent-kernel work distribution: CTAs take items from counter[0]; the
// last CTA to finish zeroes both counters for the next launch. No CTA waits
// on another, so no wait can hang.
__device__ __forceinline__ int next_item(unsigned* counter, int* s_item) {
  __syncthreads();  // everyone is done with the previous item and s_item
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(&counter[0], 1u);
  __syncthreads();
  return *s_item;
}

__device__ __forceinline__ void retire_cta(unsigned* counter) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&counter[1], 1u);
    if (done == gridDim.x - 1) {
      counter[0] = 0u;
      counter[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace nbody
