// O(N) kernels around the all-pairs passes: staging, slice combination, the
// leapfrog kicks and drift (Verlet half-stepping, Sec. II-A), the fixed-order
// float64 reductions of energy and momenta (Sec. VI) and of the virial, the
// reverse-sweep update of the adjoint (with its G and eps sums), and the copy
// kernel of the host-buffer step. One CTA handles one chunk of one system, so chunk
// partials never mix systems and every sum has a fixed order.
#include <math.h>

#include <algorithm>

#include "nbody_internal.h"
#include "post_common.cuh"

namespace nbody {
namespace {

__global__ void __launch_bounds__(kPostThreads) k_post(const PostLaunch P) {
  pdl_wait();     // the force kernel before it has finished writing the partials
  pdl_trigger();  // the next force kernel may be scheduled once every CTA has started
  if ((int)blockIdx.x == P.n_chunks) {
    // the extra CTA: the previous step's energy record from its chunk partials
    systems_final<kEnergyVals, kPostThreads>(P.sys_chunk, P.n_sys, P.eprev, P.n_chunks, P.status,
                                             [&](int sy, const double (&v)[kEnergyVals]) {
                                               emit_energy(P.eprev_out, sy, v);
                                             });
    return;
  }
  Chunk c = P.chunks[blockIdx.x];
  if (!chunk_ok(c, P.n_total, P.n_sys, (P.mode & kCombine) ? P.part_slices : 0, P.status))
    c.begin = c.end = 0;  // NBODY_DEBUG builds only: processed as an empty chunk
  const double4_32a* part = reinterpret_cast<const double4_32a*>(P.part);
  const double* cen = P.centre + 3 * c.sys;
  double e[kEnergyVals];
#pragma unroll
  for (int k = 0; k < kEnergyVals; ++k) e[k] = 0.0;
  bool bad = false;
  const unsigned mode = P.mode;

  for (int i = c.begin + (int)threadIdx.x; i < c.end; i += kPostThreads) {
    double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
    if ((mode & kCombine) && P.precision == 1) {
      // compensated float32 pairs, added as pairs on the FP32 pipe: TwoSum of
      // the hi parts, the lo parts and rounding errors summed alongside
      const fpair4* fp = reinterpret_cast<const fpair4*>(P.part);
      float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f, hz = 0.f, lz = 0.f, hp = 0.f, lp = 0.f;
#pragma unroll 8
      for (int s = 0; s < c.n_slices; ++s) {
        const fpair4 q = fp[(int64_t)s * P.n_total + i];
        two_sum_acc(hx, lx, q.xy.x), lx += q.xy.y;
        two_sum_acc(hy, ly, q.xy.z), ly += q.xy.w;
        two_sum_acc(hz, lz, q.zp.x), lz += q.zp.y;
        two_sum_acc(hp, lp, q.zp.z), lp += q.zp.w;
      }
      sx = (double)hx + (double)lx, sy = (double)hy + (double)ly;
      sz = (double)hz + (double)lz, sp = (double)hp + (double)lp;
    } else if (mode & kCombine) {
#pragma unroll 8
      for (int s = 0; s < c.n_slices; ++s) {
        const double4_32a q = part[(int64_t)s * P.n_total + i];
        sx += q.x, sy += q.y, sz += q.z, sp += q.w;
      }
    }
    bad |= post_body(P, mode, i, cen, sx, sy, sz, sp, e);
  }
  if (bad) atomicOr(P.status, kFlagNonFinite);
  if (mode & kVirial) {
    double kw[2] = {e[0], e[1]};
    block_sum<2, kPostThreads>(kw);
    if (threadIdx.x == 0) P.epart[(int64_t)blockIdx.x * kEnergyVals + 0] = kw[0],
                          P.epart[(int64_t)blockIdx.x * kEnergyVals + 1] = kw[1];
    if (last_of(P.done, (unsigned)P.n_chunks)) {
      __threadfence();
      systems_final<2, kPostThreads>(P.sys_chunk, P.n_sys, P.epart, P.n_chunks, P.status,
                                     [&](int sy, const double (&v)[2]) {
                                       double* o = P.vout + 3 * (int64_t)sy;
                                       o[0] = v[0];
                                       o[1] = v[1];
                                       o[2] = v[1] != 0.0 ? -2.0 * v[0] / v[1] : 0.0;
                                     });
    }
    return;
  }
  if (mode & kEnergy) {
    block_sum<kEnergyVals, kPostThreads>(e);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < kEnergyVals; ++k) P.epart[(int64_t)blockIdx.x * kEnergyVals + k] = e[k];
    }
    // the last chunk CTA to finish forms the per-system records (no separate launch); with
    // eout null the partials wait for the next step's k_post
    if (P.eout && last_of(P.done, (unsigned)P.n_chunks)) {
      __threadfence();
      systems_final<kEnergyVals, kPostThreads>(P.sys_chunk, P.n_sys, P.epart, P.n_chunks, P.status,
                                               [&](int sy, const double (&v)[kEnergyVals]) {
                                                 emit_energy(P.eout, sy, v);
                                               });
    }
  }
}

// Staging origin: per chunk, sum m x (3), sum m, sum x (3) into cpart[chunk][8];
// the last CTA then forms, per system in a fixed order, the mass-weighted mean
// position (plain mean if the mass is not positive; 0 for an empty system).
__global__ void __launch_bounds__(kPostThreads) k_centre(const Chunk* chunks, const int32_t* sys_chunk,
                                                         const int64_t* off, const int n_sys, const double* x,
                                                         const double* m, double* cpart, double* centre,
                                                         unsigned* done, const int64_t n_total, unsigned* status) {
  Chunk c = chunks[blockIdx.x];
  if (!chunk_ok(c, n_total, n_sys, 0, status)) c.begin = c.end = 0;  // NBODY_DEBUG builds only
  double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = c.begin + (int)threadIdx.x; i < c.end; i += kPostThreads) {
    const double mi = m[i];
    const double x0 = x[3 * i + 0], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
    v[0] += mi * x0, v[1] += mi * x1, v[2] += mi * x2, v[3] += mi;
    v[4] += x0, v[5] += x1, v[6] += x2;
  }
  block_sum<7, kPostThreads>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 7; ++k) cpart[(int64_t)blockIdx.x * kEnergyVals + k] = v[k];
  }
  if (!last_of(done, gridDim.x)) return;
  __threadfence();
  systems_final<7, kPostThreads>(sys_chunk, n_sys, cpart, gridDim.x, status, [&](int sy, const double (&w)[7]) {
    const int64_t n = off[sy + 1] - off[sy];
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    if (w[3] > 0.0 && isfinite(w[3])) {
      c0 = w[0] / w[3], c1 = w[1] / w[3], c2 = w[2] / w[3];
    } else if (n > 0) {
      c0 = w[4] / (double)n, c1 = w[5] / (double)n, c2 = w[6] / (double)n;
    }
    if (!(isfinite(c0) && isfinite(c1) && isfinite(c2))) c0 = c1 = c2 = 0.0;
    centre[3 * sy + 0] = c0, centre[3 * sy + 1] = c1, centre[3 * sy + 2] = c2;
  });
}

__global__ void __launch_bounds__(kPostThreads) k_adj_update(const AdjLaunch A) {
  Chunk c = A.chunks[blockIdx.x];
  if (!chunk_ok(c, A.n_total, A.n_sys, A.part_slices, A.status)) c.begin = c.end = 0;  // NBODY_DEBUG builds only
  const double4_32a* part = reinterpret_cast<const double4_32a*>(A.part);
  const double* cen = A.centre + 3 * c.sys;
  const int kw = A.g_params ? 3 : 2;  // partials (fpair4 / double4_32a) per body and slice
  double pv[2] = {0.0, 0.0};          // this thread's w.da/dG and sum m (d.w) / s^5
  bool bad = false;
  for (int i = c.begin + (int)threadIdx.x; i < c.end; i += kPostThreads) {
    double a1x = 0, a1y = 0, a1z = 0, a2 = 0, gbx = 0, gby = 0, gbz = 0, gm = 0;
    if (A.precision == 1) {
      // compensated float32 pairs (fpair4), added as pairs on the FP32 pipe
      const fpair4* fp = reinterpret_cast<const fpair4*>(A.part);
      float h[10], l[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) h[q] = l[q] = 0.f;
      auto add = [&](const int q, const float hv, const float lv) {
        two_sum_acc(h[q], l[q], hv);
        l[q] += lv;
      };
#pragma unroll 4
      for (int s = 0; s < c.n_slices; ++s) {
        const int64_t k = kw * ((int64_t)s * A.n_total + i);
        const fpair4 p = fp[k], q = fp[k + 1];
        add(0, p.xy.x, p.xy.y), add(1, p.xy.z, p.xy.w), add(2, p.zp.x, p.zp.y), add(3, p.zp.z, p.zp.w);
        add(4, q.xy.x, q.xy.y), add(5, q.xy.z, q.xy.w), add(6, q.zp.x, q.zp.y), add(7, q.zp.z, q.zp.w);
        if (A.g_params) {
          const fpair4 r = fp[k + 2];
          add(8, r.xy.x, r.xy.y), add(9, r.xy.z, r.xy.w);
        }
      }
      auto d = [&](const int q) { return (double)h[q] + (double)l[q]; };
      a1x = d(0), a1y = d(1), a1z = d(2), a2 = d(3), gbx = d(4), gby = d(5), gbz = d(6), gm = d(7);
      if (A.g_params) pv[0] += d(8), pv[1] += d(9);
    } else {
#pragma unroll 4
      for (int s = 0; s < c.n_slices; ++s) {
        const int64_t k = kw * ((int64_t)s * A.n_total + i);
        const double4_32a p = part[k], q = part[k + 1];
        a1x += p.x, a1y += p.y, a1z += p.z, a2 += p.w;
        gbx += q.x, gby += q.y, gbz += q.z, gm += q.w;
        if (A.g_params) {
          const double4_32a r = part[k + 2];
          pv[0] += r.x, pv[1] += r.y;
        }
      }
    }
    const double mi = A.m[i];
    double w0 = A.lam_v[3 * i + 0], w1 = A.lam_v[3 * i + 1], w2 = A.lam_v[3 * i + 2];
    const double gx0 = A.G * (mi * a1x - a2 * w0 - 3.0 * gbx);
    const double gx1 = A.G * (mi * a1y - a2 * w1 - 3.0 * gby);
    const double gx2 = A.G * (mi * a1z - a2 * w2 - 3.0 * gbz);
    const double gmi = -A.G * gm;
    bad |= !(isfinite(gx0) && isfinite(gx1) && isfinite(gx2) && isfinite(gmi));
    const double l0 = A.lam_x[3 * i + 0] + A.coef * gx0;
    const double l1 = A.lam_x[3 * i + 1] + A.coef * gx1;
    const double l2 = A.lam_x[3 * i + 2] + A.coef * gx2;
    A.lam_x[3 * i + 0] = l0, A.lam_x[3 * i + 1] = l1, A.lam_x[3 * i + 2] = l2;
    A.g_m[i] += A.coef * gmi;
    if (A.drift_rev) {
      w0 += A.dt * l0, w1 += A.dt * l1, w2 += A.dt * l2;
      A.lam_v[3 * i + 0] = w0, A.lam_v[3 * i + 1] = w1, A.lam_v[3 * i + 2] = w2;
      if (A.precision == 1)
        static_cast<float4*>(A.stage_w)[i] = make_float4((float)w0, (float)w1, (float)w2, 0.f);
      else
        static_cast<double4_32a*>(A.stage_w)[i] = make_double4_32a(w0, w1, w2, 0.0);
    }
    if (A.x_next)
      stage_store(A.precision, A.stage_x, i, A.x_next[3 * i + 0], A.x_next[3 * i + 1], A.x_next[3 * i + 2], mi,
                  cen, A.stage_lo);
  }
  if (bad) atomicOr(A.status, kFlagNonFinite);
  if (!A.g_params) return;
  // dL/dG += coef sum_k w_k . da_k/dG; dL/deps += coef (-3 G eps) sum_k sum_j m_j (d.w_k) / s^5,
  // per system in a fixed order (chunk partials, then the last CTA)
  block_sum<2, kPostThreads>(pv);
  if (threadIdx.x == 0) A.cpart[(int64_t)blockIdx.x * kEnergyVals + 0] = pv[0],
                        A.cpart[(int64_t)blockIdx.x * kEnergyVals + 1] = pv[1];
  if (!last_of(A.done, gridDim.x)) return;
  __threadfence();
  systems_final<2, kPostThreads>(A.sys_chunk, A.n_sys, A.cpart, gridDim.x, A.status, [&](int sy, const double (&v)[2]) {
    const double dG = A.coef * v[0], de = A.coef * (-3.0 * A.G * A.eps) * v[1];
    if (!(isfinite(dG) && isfinite(de))) atomicOr(A.status, kFlagNonFinite);
    A.g_params[2 * sy + 0] += dG;
    A.g_params[2 * sy + 1] += de;
  });
}

__global__ void __launch_bounds__(kPostThreads) k_stage_vec(const Chunk* chunks, int precision, const double* vec,
                                                            const double* m, const double* centre, void* stage,
                                                            void* stage_lo, int as_position, const int64_t n_total,
                                                            const int n_sys, unsigned* status) {
  Chunk c = chunks[blockIdx.x];
  if (!chunk_ok(c, n_total, n_sys, 0, status)) c.begin = c.end = 0;  // NBODY_DEBUG builds only
  const double* cen = centre + 3 * c.sys;
  for (int i = c.begin + (int)threadIdx.x; i < c.end; i += kPostThreads) {
    const double v0 = vec[3 * i + 0], v1 = vec[3 * i + 1], v2 = vec[3 * i + 2];
    if (as_position) {
      stage_store(precision, stage, i, v0, v1, v2, m[i], cen, stage_lo);
    } else if (precision == 1) {
      static_cast<float4*>(stage)[i] = make_float4((float)v0, (float)v1, (float)v2, 0.f);
    } else {
      static_cast<double4_32a*>(stage)[i] = make_double4_32a(v0, v1, v2, 0.0);
    }
  }
}

// Up to four plain copies of float64 arrays in one launch (the host-buffer
// step's transfers through mapped pinned host memory).
__global__ void __launch_bounds__(256) k_copy4(const Copy4 C) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double* __restrict__ src = C.src[k];
    double* __restrict__ dst = C.dst[k];
    const int64_t n = (src && dst) ? C.n[k] : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
  }
}

}  // namespace

cudaError_t launch_copy4(const Copy4& C, int n_sms, cudaStream_t st) {
  int64_t most = 0;
  for (int k = 0; k < 4; ++k) most = std::max<int64_t>(most, C.src[k] && C.dst[k] ? C.n[k] : 0);
  if (most == 0) return cudaSuccess;
  const int64_t want = (most + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)std::max(1, n_sms) * 8);
  k_copy4<<<grid, 256, 0, st>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_post(const PostLaunch& P, cudaStream_t st) {
  if (P.n_chunks <= 0) return cudaSuccess;
  return launch_pdl(k_post, (unsigned)P.n_chunks + (P.eprev_out ? 1u : 0u), kPostThreads, st, P);
}

cudaError_t launch_centre(const Chunk* chunks, int n_chunks, const int32_t* sys_chunk, const int64_t* off, int n_sys,
                          const double* x, const double* m, double* cpart, double* centre, unsigned* done,
                          int64_t n_total, unsigned* status, cudaStream_t st) {
  if (n_sys <= 0 || n_chunks <= 0) return cudaSuccess;
  k_centre<<<n_chunks, kPostThreads, 0, st>>>(chunks, sys_chunk, off, n_sys, x, m, cpart, centre, done, n_total,
                                              status);
  return cudaGetLastError();
}

cudaError_t launch_adj_update(const AdjLaunch& A, cudaStream_t st) {
  if (A.n_chunks <= 0) return cudaSuccess;
  k_adj_update<<<A.n_chunks, kPostThreads, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_stage_vec(const Chunk* chunks, int n_chunks, int precision, const double* vec, const double* m,
                             const double* centre, void* stage, void* stage_lo, int as_position, int64_t n_total,
                             int n_sys, unsigned* status, cudaStream_t st) {
  if (n_chunks <= 0) return cudaSuccess;
  k_stage_vec<<<n_chunks, kPostThreads, 0, st>>>(chunks, precision, vec, m, centre, stage, stage_lo, as_position,
                                                 n_total, n_sys, status);
  return cudaGetLastError();
}

}  // namespace nbody
