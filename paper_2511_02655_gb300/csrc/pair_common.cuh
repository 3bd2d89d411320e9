// Device helpers shared by the all-pairs kernels (force, force-VJP and the
// allocation-free entry point).
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

// d of a near pair from the staged float32 parts x - c = hi + lo (lo is the
// float32 remainder of the float64 value): the hi difference is exact for close
// pairs (Sterbenz) and the lo difference restores the bits the staging dropped,
// so d is good to a rounding of |d| itself, in float32 arithmetic only.
__device__ __forceinline__ void refine_pair(const float4* __restrict__ lo, const int i, const int j, const float dhx,
                                            const float dhy, const float dhz, const float eps2, float& dx, float& dy,
                                            float& dz, float& r2) {
  const float4 lj = lo[j], li = lo[i];
  dx = dhx + (lj.x - li.x);
  dy = dhy + (lj.y - li.y);
  dz = dhz + (lj.z - li.z);
  r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
}

// Second look at one pair (j-body q at global index jg, i-body at ig) of a
// flagged sub-block: if it is near and not the self pair, replace its
// unrefined contribution in (ax, ay, az, pp) by the refined one. The
// unrefined terms are recomputed with exactly the first pass's operations.
// LAW 0: softened gravity (q.w = m_j); LAW 1: Lennard-Jones (s2 = sigma^2 in the
// staged length unit, i.e. 1 on the mixed path).
template <int LAW = 0>
__device__ __forceinline__ void correct_pair(const float4 q, const int jg, const int ig, const int i_end,
                                             const float xi, const float yi, const float zi, const float eps2,
                                             const float r2c, const float4* __restrict__ lo, float& ax, float& ay,
                                             float& az, float& pp, const float s2 = 0.f) {
  const float dx = q.x - xi;
  const float dy = q.y - yi;
  const float dz = q.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  if (!(r2 < r2c) || ig >= i_end || jg < 0 || ig == jg) return;
  float rx, ry, rz, rr2;
  refine_pair(lo, ig, jg, dx, dy, dz, eps2, rx, ry, rz, rr2);
  if (LAW == 0) {
    const float iu = rsq_approx(r2);
    const float msu = q.w * iu;
    const float wu = msu * (iu * iu);
    const float ir = rsq_approx(rr2);
    const float msr = q.w * ir;
    const float wr = msr * (ir * ir);
    ax += fmaf(rx, wr, -(dx * wu));
    ay += fmaf(ry, wr, -(dy * wu));
    az += fmaf(rz, wr, -(dz * wu));
    pp += msr - msu;
  } else {
    const float iu = rcp_approx(r2);
    const float su2 = s2 * iu, su6 = su2 * (su2 * su2), su12 = su6 * su6;
    const float wu = fmaf(su12, -2.f, su6) * iu;
    const float ir = rcp_approx(rr2);
    const float sr2 = s2 * ir, sr6 = sr2 * (sr2 * sr2), sr12 = sr6 * sr6;
    const float wr = fmaf(sr12, -2.f, sr6) * ir;
    ax += fmaf(rx, wr, -(dx * wu));
    ay += fmaf(ry, wr, -(dy * wu));
    az += fmaf(rz, wr, -(dz * wu));
    pp += fmaf(sr6, -1.f, sr12) - fmaf(su6, -1.f, su12);
  }
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
