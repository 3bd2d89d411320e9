// Device helpers of the O(N) kernels around the all-pairs passes
// (post_kernels.cu): the per-body combine / kick / drift / staging / energy
// terms of one body, the fixed-order CTA and per-system float64 sums, and the
// last-arrival ticket.
#pragma once

#include <math.h>

#include "nbody_internal.h"

namespace nbody {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA sum of NV values per thread; result valid in thread 0.
// The sum is transposed so that every thread adds: the CTA's NV x THREADS
// values go to shared memory, then a group of TPV lanes per value adds its
// row in a fixed interleaved order and a TPV-lane xor shuffle finishes it.
// For NV = 8 and 128 threads that is 11 float64 additions per thread instead
// of the 40 of a per-value warp butterfly (float64 adds are GB300's scarce
// resource in these kernels).
template <int NV, int THREADS>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  constexpr int NVP = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : 16;
  constexpr int TPV0 = THREADS / NVP;
  constexpr int TPV = TPV0 > 32 ? 32 : TPV0;  // lanes per value: one aligned group inside a warp
  constexpr int EPT = THREADS / TPV;          // entries each of those lanes adds
  static_assert(TPV >= 1 && THREADS % 32 == 0 && NV <= 16, "block_sum layout");
  __shared__ double red[NV][THREADS];
  __shared__ double res[NV];
  __syncthreads();  // an earlier block_sum of the same shape may still be reading
#pragma unroll
  for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  const int k = (int)threadIdx.x / TPV, p = (int)threadIdx.x % TPV;
  double s = 0.0;
  if (k < NV) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) s += red[k][p + e * TPV];
  }
#pragma unroll
  for (int o = TPV / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (k < NV && p == 0) res[k] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = res[q];
  }
}

// Reflecting walls of [0, box] ("boundary checking"): a coordinate that left
// the box is mirrored back across the wall and its velocity component flips;
// repeated (bounded) for steps that cross the box more than once.
__device__ __forceinline__ void reflect(double& x, double& v, const double box) {
  for (int k = 0; k < 64; ++k) {
    if (x < 0.0) {
      x = -x, v = -v;
    } else if (x > box) {
      x = 2.0 * box - x, v = -v;
    } else {
      return;
    }
  }
}

// Staging entry of body i. Mixed: float4 ((x - c) * scale, m) rounded to
// float32 and, when lo is given, the float32 remainders of the scaled
// coordinates used by the near-pair refinement of the force kernels (scale is
// 1, or 1 / sigma for Lennard-Jones). FP64: double4 (x, m).
__device__ __forceinline__ void stage_store(int precision, void* stage, int i, double x, double y, double z,
                                            double m, const double* c, void* lo = nullptr, double scale = 1.0) {
  if (precision == 1) {
    const double X = (x - c[0]) * scale, Y = (y - c[1]) * scale, Z = (z - c[2]) * scale;
    const float hx = (float)X, hy = (float)Y, hz = (float)Z;
    static_cast<float4*>(stage)[i] = make_float4(hx, hy, hz, (float)m);
    if (lo)
      static_cast<float4*>(lo)[i] =
          make_float4((float)(X - (double)hx), (float)(Y - (double)hy), (float)(Z - (double)hz), 0.f);
  } else {
    static_cast<double4_32a*>(stage)[i] = make_double4_32a(x, y, z, m);
  }
}

// Final per-system sums of partials [n_parts][kEnergyVals] (one per chunk of
// an O(N) kernel), in a fixed order whichever CTA runs it. The partials were
// written by other CTAs of the same launch, so they are read from L2
// (ld.global.cg). Up to four systems: the whole CTA adds each system's
// partials (thread t takes partials t, t + THREADS, ...), then block_sum; more
// systems: one warp per system, lanes striding over its range, then a warp
// butterfly. Every thread of the CTA must call it.
template <int NV, int THREADS, typename Emit>
__device__ __forceinline__ void systems_final(const int32_t* sys_part, const int n_sys, const double* part,
                                              const int n_parts, unsigned* status, Emit emit) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (n_sys <= 4) {
    for (int sy = 0; sy < n_sys; ++sy) {
      double v[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = 0.0;
      // NBODY_DEBUG builds: the system's range lies inside the partials
      const bool ok = nb_debug_ok(sys_part[sy] >= 0 && sys_part[sy] <= sys_part[sy + 1] &&
                                      sys_part[sy + 1] <= n_parts,
                                  threadIdx.x == 0 ? status : nullptr);
#pragma unroll 4
      for (int c = sys_part[sy] + (int)threadIdx.x; ok && c < sys_part[sy + 1]; c += THREADS) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + (int64_t)c * kEnergyVals + k);
      }
      block_sum<NV, THREADS>(v);
      if (threadIdx.x == 0) emit(sy, v);
    }
    return;
  }
  for (int sy = wid; sy < n_sys; sy += THREADS / 32) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    const bool ok = nb_debug_ok(sys_part[sy] >= 0 && sys_part[sy] <= sys_part[sy + 1] && sys_part[sy + 1] <= n_parts,
                                lane == 0 ? status : nullptr);
    for (int c = sys_part[sy] + lane; ok && c < sys_part[sy + 1]; c += 32) {
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + (int64_t)c * kEnergyVals + k);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) emit(sy, v);
  }
}

// True in every thread of the CTA that arrives last of `expected` arrivals at
// the ticket `done` (its results were published with a fence before the
// ticket); that CTA resets the ticket for the next launch. No CTA waits.
__device__ __forceinline__ bool last_of(unsigned* done, const unsigned expected) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1u) == expected - 1u;
    if (s_last) *done = 0u;
  }
  __syncthreads();
  return s_last;
}

__device__ __forceinline__ void emit_energy(double* out, const int sy, const double (&v)[kEnergyVals]) {
  double* o = out + 9 * (int64_t)sy;
  o[0] = v[0] + v[1];
  o[1] = v[0];
  o[2] = v[1];
#pragma unroll
  for (int k = 2; k < kEnergyVals; ++k) o[k + 1] = v[k];
}

// The O(N) work of one body i in the PostMode bits of `mode`: with kCombine its
// summed partials (sx, sy, sz, sp) become a = G S (or the Lennard-Jones
// scaling) and phi; then the closing half-kick, the energy or virial terms
// (accumulated into e), the opening half-kick and drift of the next step (with
// the walls), and the staging entry of the new position. cen is the system's
// staging origin. Returns true if a combined value is not finite.
__device__ __forceinline__ bool post_body(const PostLaunch& P, const unsigned mode, const int i, const double* cen,
                                          const double sx, const double sy, const double sz, const double sp,
                                          double (&e)[kEnergyVals]) {
  bool bad = false;
  // every load of the body first, so that they are in flight together (x, v, m
  // and a are distinct arrays; nothing below is stored before it is read)
  const bool need_x = mode & (kKickEnd | kEnergy | kDrift | kStage | kVirial);
  const bool need_v = mode & (kKickEnd | kEnergy | kDrift | kVirial);
  const bool need_m = need_x || (mode & kCombine && P.law != 0);
  double x0 = 0.0, x1 = 0.0, x2 = 0.0, v0 = 0.0, v1 = 0.0, v2 = 0.0, m = 0.0;
  if (need_x) x0 = P.x[3 * i + 0], x1 = P.x[3 * i + 1], x2 = P.x[3 * i + 2];
  if (need_v) v0 = P.v[3 * i + 0], v1 = P.v[3 * i + 1], v2 = P.v[3 * i + 2];
  if (need_m) m = P.m[i];
  double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
  if (mode & kCombine) {
    if (P.law == 0) {  // softened gravity
      ax = P.G * sx, ay = P.G * sy, az = P.G * sz, ph = -P.G * sp;
    } else {  // Lennard-Jones: per unit mass of body i (sums over staged coordinates in units of sigma
              // carry one factor sigma: S = sigma * sum (u^3 - 2 u^6) d / r^2, hence the stage_scale)
      const double im = 1.0 / m, ca = 24.0 * P.lj_eps * P.stage_scale * im, cp = 4.0 * P.lj_eps * im;
      ax = ca * sx, ay = ca * sy, az = ca * sz, ph = cp * sp;
    }
    P.a[3 * i + 0] = ax, P.a[3 * i + 1] = ay, P.a[3 * i + 2] = az;
    if (P.phi) P.phi[i] = ph;
    bad = !(isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(ph));
  } else if (mode & (kKickEnd | kDrift)) {
    ax = P.a[3 * i + 0], ay = P.a[3 * i + 1], az = P.a[3 * i + 2];
  }
  if (mode & kVirial) {
    e[0] += 0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2);
    e[1] += m * (x0 * ax + x1 * ay + x2 * az);
  }
  if (!(mode & (kKickEnd | kEnergy | kDrift | kStage))) return bad;
  if (mode & (kKickEnd | kEnergy | kDrift)) {
    if (mode & kKickEnd) {
      v0 += P.half_dt * ax, v1 += P.half_dt * ay, v2 += P.half_dt * az;
    }
    if (mode & kEnergy) {
      e[0] += 0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2);
      e[1] += 0.5 * m * ph;
      e[2] += m * v0, e[3] += m * v1, e[4] += m * v2;
      e[5] += m * (x1 * v2 - x2 * v1);
      e[6] += m * (x2 * v0 - x0 * v2);
      e[7] += m * (x0 * v1 - x1 * v0);
    }
    if (mode & kDrift) {
      v0 += P.half_dt * ax, v1 += P.half_dt * ay, v2 += P.half_dt * az;
      x0 += P.dt * v0, x1 += P.dt * v1, x2 += P.dt * v2;
      if (P.box > 0.0) {
        reflect(x0, v0, P.box);
        reflect(x1, v1, P.box);
        reflect(x2, v2, P.box);
      }
      P.x[3 * i + 0] = x0, P.x[3 * i + 1] = x1, P.x[3 * i + 2] = x2;
      if (P.x_copy) P.x_copy[3 * i + 0] = x0, P.x_copy[3 * i + 1] = x1, P.x_copy[3 * i + 2] = x2;
    }
    if (mode & (kKickEnd | kDrift)) P.v[3 * i + 0] = v0, P.v[3 * i + 1] = v1, P.v[3 * i + 2] = v2;
  }
  if (mode & kStage) stage_store(P.precision, P.stage, i, x0, x1, x2, m, cen, P.stage_lo, P.stage_scale);
  return bad;
}

}  // namespace nbody
