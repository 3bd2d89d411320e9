// All-pairs softened-gravity force kernels (the paper's force calculation over
// "N_p^2 operations", Sec. V-B, with the energy term fused into the same loop,
// Sec. VI). Two precisions:
//
//   mixed : staged j-bodies are float4 (x - c, y - c, z - c, m) with c the
//           system's staging origin; each interaction is 3 FADD + 3 FFMA +
//           1 MUFU.RSQ + 3 FMUL + 3 FFMA + 1 FADD in float32; per j-tile the
//           float32 partial sums are folded into a compensated (hi, lo) float32
//           pair per body (TwoSum), converted to float64 per work item.
//   fp64  : staged double4_32a (x, y, z, m), every operation in float64.
//
// Both are persistent kernels over a work list of (i-tile, j-slice) items.
// i-bodies live in registers (R per thread, strided by the CTA size so loads
// and stores coalesce), j-bodies stream through a shared-memory tile that
// every thread reads with broadcast loads; the next tile is prefetched into
// registers while the current one is consumed. Each item writes one float64
// partial (sum m d / s^3, sum m / s) per i-body to its slice; the O(N) post
// kernel adds the slices in a fixed order, so results are deterministic.
// Self pairs are masked in the tiles that overlap the item's own i-range.
#include "nbody_internal.h"
#include "pair_common.cuh"

namespace nbody {
namespace {

template <bool MASK>
__device__ __forceinline__ void pair_f32(const float4 q, const float xi, const float yi, const float zi,
                                         const float eps2, float& ax, float& ay, float& az, float& pp,
                                         const bool self) {
  const float dx = q.x - xi;
  const float dy = q.y - yi;
  const float dz = q.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float inv = rsq_approx(r2);
  if (MASK) inv = self ? 0.f : inv;
  const float ms = q.w * inv;         // m_j / s
  const float w = ms * (inv * inv);   // m_j / s^3
  ax = fmaf(dx, w, ax);
  ay = fmaf(dy, w, ay);
  az = fmaf(dz, w, az);
  pp += ms;
}

template <bool MASK>
__device__ __forceinline__ void pair_f64(const double4_32a q, const double xi, const double yi, const double zi,
                                         const double eps2, double& ax, double& ay, double& az, double& pp,
                                         const bool self) {
  const double dx = q.x - xi;
  const double dy = q.y - yi;
  const double dz = q.z - zi;
  const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  double inv = rsqrt(r2);
  if (MASK) inv = self ? 0.0 : inv;
  const double ms = q.w * inv;
  const double w = ms * (inv * inv);
  ax = fma(dx, w, ax);
  ay = fma(dy, w, ay);
  az = fma(dz, w, az);
  pp += ms;
}

template <int BLOCK, int R, int J>
__global__ void __launch_bounds__(BLOCK) k_force_mixed(const PairLaunch L) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;  // tile entries loaded per thread
  __shared__ __align__(16) float4 tile[J];
  __shared__ int s_item;
  const float4* __restrict__ st = static_cast<const float4*>(L.stage_x);
  double4_32a* __restrict__ part = reinterpret_cast<double4_32a*>(L.part);
  const float eps2 = (float)L.eps2;

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];

    float xi[R], yi[R], zi[R];
    float hx[R], hy[R], hz[R], hp[R], lx[R], ly[R], lz[R], lp[R];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const float4 q = ig[r] < w.i_end ? st[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      xi[r] = q.x, yi[r] = q.y, zi[r] = q.z;
      hx[r] = hy[r] = hz[r] = hp[r] = 0.f;
      lx[r] = ly[r] = lz[r] = lp[r] = 0.f;
    }

    float4 pre[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int jj = w.j_begin + (int)threadIdx.x + k * BLOCK;
      if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) pre[k] = st[jj];
    }

    for (int jt = w.j_begin; jt < w.j_end; jt += J) {
      const int nj = min(J, w.j_end - jt);
      __syncthreads();  // all threads are done reading the previous tile
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj) tile[t] = pre[k];
      }
      __syncthreads();
      if (jt + J < w.j_end) {  // prefetch the next tile while this one is consumed
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) pre[k] = st[jj];
        }
      }

      float ax[R], ay[R], az[R], pp[R];
#pragma unroll
      for (int r = 0; r < R; ++r) ax[r] = ay[r] = az[r] = pp[r] = 0.f;

      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      if (diag) {
        for (int j = 0; j < nj; ++j) {
          const float4 q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f32<true>(q, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], jt + j == ig[r]);
        }
      } else if (nj == J) {
#pragma unroll 8
        for (int j = 0; j < J; ++j) {
          const float4 q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f32<false>(q, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], false);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
          const float4 q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f32<false>(q, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], false);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        two_sum_acc(hx[r], lx[r], ax[r]);
        two_sum_acc(hy[r], ly[r], ay[r]);
        two_sum_acc(hz[r], lz[r], az[r]);
        two_sum_acc(hp[r], lp[r], pp[r]);
      }
    }

    double4_32a* out = part + (int64_t)w.slice * L.n_total;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end)
        out[ig[r]] = make_double4_32a((double)hx[r] + (double)lx[r], (double)hy[r] + (double)ly[r],
                                  (double)hz[r] + (double)lz[r], (double)hp[r] + (double)lp[r]);
    }
  }
  retire_cta(L.counter);
}

template <int BLOCK, int R, int J>
__global__ void __launch_bounds__(BLOCK) k_force_fp64(const PairLaunch L) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  __shared__ __align__(32) double4_32a tile[J];
  __shared__ int s_item;
  const double4_32a* __restrict__ st = static_cast<const double4_32a*>(L.stage_x);
  double4_32a* __restrict__ part = reinterpret_cast<double4_32a*>(L.part);
  const double eps2 = L.eps2;

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];

    double xi[R], yi[R], zi[R], ax[R], ay[R], az[R], pp[R];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const double4_32a q = ig[r] < w.i_end ? st[ig[r]] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
      xi[r] = q.x, yi[r] = q.y, zi[r] = q.z;
      ax[r] = ay[r] = az[r] = pp[r] = 0.0;
    }

    double4_32a pre[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int jj = w.j_begin + (int)threadIdx.x + k * BLOCK;
      if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) pre[k] = st[jj];
    }

    for (int jt = w.j_begin; jt < w.j_end; jt += J) {
      const int nj = min(J, w.j_end - jt);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj) tile[t] = pre[k];
      }
      __syncthreads();
      if (jt + J < w.j_end) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) pre[k] = st[jj];
        }
      }
      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      if (diag) {
        for (int j = 0; j < nj; ++j) {
          const double4_32a q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f64<true>(q, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], jt + j == ig[r]);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
          const double4_32a q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f64<false>(q, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], false);
        }
      }
    }

    double4_32a* out = part + (int64_t)w.slice * L.n_total;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (ig[r] < w.i_end) out[ig[r]] = make_double4_32a(ax[r], ay[r], az[r], pp[r]);
  }
  retire_cta(L.counter);
}

template <typename K>
int occupancy_of(K kern, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, 0) != cudaSuccess) return 0;
  return n;
}

// Tilings compiled: BLOCK in {128, 256}, R in {1, 2, 4}, J in {128, 256}.
#define NBODY_FORCE_TILINGS(X) \
  X(128, 1, 128) X(128, 2, 128) X(128, 4, 128) X(128, 1, 256) X(128, 2, 256) X(128, 4, 256) \
  X(256, 1, 128) X(256, 2, 128) X(256, 4, 128) X(256, 1, 256) X(256, 2, 256) X(256, 4, 256)

}  // namespace

cudaError_t launch_force(int precision, const PairLaunch& L, cudaStream_t st) {
  if (L.n_ctas <= 0) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                                                     \
  if (L.block == B && L.ipt == R && L.jtile == J) {                                          \
    if (precision == 1)                                                                      \
      k_force_mixed<B, R, J><<<L.n_ctas, B, 0, st>>>(L);                                     \
    else                                                                                     \
      k_force_fp64<B, R, J><<<L.n_ctas, B, 0, st>>>(L);                                      \
    return cudaGetLastError();                                                               \
  }
  NBODY_FORCE_TILINGS(NBODY_X)
#undef NBODY_X
  return cudaErrorInvalidConfiguration;
}

int force_ctas_per_sm(int precision, int block, int ipt, int jtile) {
#define NBODY_X(B, R, J)                                                                     \
  if (block == B && ipt == R && jtile == J)                                                  \
    return precision == 1 ? occupancy_of(k_force_mixed<B, R, J>, B) : occupancy_of(k_force_fp64<B, R, J>, B);
  NBODY_FORCE_TILINGS(NBODY_X)
#undef NBODY_X
  return 0;
}

}  // namespace nbody
