// All-pairs vector-Jacobian product of the force map a(x, m), the inner kernel
// of the adjoint (reverse) leapfrog. For weights w (w_k = dL/da_k):
//
//   g_x,k = G sum_{j != k} J(d_kj) (m_k w_j - m_j w_k),  J(d) = I / s^3 - 3 d d^T / s^5
//   g_m,k = -G sum_{j != k} (w_j . d_kj) / s_kj^3          (d_kj = x_j - x_k)
//
// Expanding u = m_k w_j - m_j w_k lets every pair update four per-body sums:
//   A1 = sum w_j / s^3,  A2 = sum m_j / s^3,
//   Gb = sum (m_k (d.w_j) - m_j (d.w_k)) d / s^5,  Gm = sum (d.w_j) / s^3,
// so that g_x,k = G (m_k A1 - A2 w_k - 3 Gb) and g_m,k = -G Gm (formed by the
// O(N) update kernel). The pair costs 26 float32 operations plus one MUFU.RSQ.
// With P (the gradients with respect to G and eps requested) two more sums,
//   Pg = sum m_j (d.w_k) / s^3   (w_k . da_k/dG),
//   Pe = sum m_j (d.w_k) / s^5   (w_k . da_k/deps = -3 G eps Pe),
// cost two float32 operations more per pair and a third double4 per body and slice.
// Tiling, work distribution, self-pair masking and the compensated per-tile
// fold are those of the force kernels.
#include <algorithm>

#include "nbody_internal.h"
#include "pair_common.cuh"

namespace nbody {
namespace {

struct Acc8f {
  float a1x, a1y, a1z, a2, gbx, gby, gbz, gm, pg, pe;
};

template <bool MASK, bool P>
__device__ __forceinline__ void vjp_pair_f32(const float4 q, const float4 wj, const float xk, const float yk,
                                             const float zk, const float mk, const float wkx, const float wky,
                                             const float wkz, const float eps2, Acc8f& s, const bool self) {
  const float dx = q.x - xk;
  const float dy = q.y - yk;
  const float dz = q.z - zk;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float inv = rsq_approx(r2);
  if (MASK) inv = self ? 0.f : inv;
  const float inv2 = inv * inv;
  const float inv3 = inv2 * inv;
  const float dwj = fmaf(dx, wj.x, fmaf(dy, wj.y, dz * wj.z));
  const float dwk = fmaf(dx, wkx, fmaf(dy, wky, dz * wkz));
  s.gm = fmaf(dwj, inv3, s.gm);
  const float pk = q.w * dwk;
  const float du = fmaf(mk, dwj, -pk);
  const float inv5 = inv3 * inv2;
  const float t = du * inv5;
  if (P) {
    s.pg = fmaf(pk, inv3, s.pg);
    s.pe = fmaf(pk, inv5, s.pe);
  }
  s.gbx = fmaf(t, dx, s.gbx);
  s.gby = fmaf(t, dy, s.gby);
  s.gbz = fmaf(t, dz, s.gbz);
  s.a1x = fmaf(inv3, wj.x, s.a1x);
  s.a1y = fmaf(inv3, wj.y, s.a1y);
  s.a1z = fmaf(inv3, wj.z, s.a1z);
  s.a2 = fmaf(q.w, inv3, s.a2);
}

struct Acc8d {
  double a1x, a1y, a1z, a2, gbx, gby, gbz, gm, pg, pe;
};

template <bool MASK, bool P>
__device__ __forceinline__ void vjp_pair_f64(const double4_32a q, const double4_32a wj, const double xk, const double yk,
                                             const double zk, const double mk, const double wkx, const double wky,
                                             const double wkz, const double eps2, Acc8d& s, const bool self) {
  const double dx = q.x - xk;
  const double dy = q.y - yk;
  const double dz = q.z - zk;
  const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  double inv = rsqrt(r2);
  if (MASK) inv = self ? 0.0 : inv;
  const double inv2 = inv * inv;
  const double inv3 = inv2 * inv;
  const double dwj = fma(dx, wj.x, fma(dy, wj.y, dz * wj.z));
  const double dwk = fma(dx, wkx, fma(dy, wky, dz * wkz));
  s.gm = fma(dwj, inv3, s.gm);
  const double pk = q.w * dwk;
  const double du = fma(mk, dwj, -pk);
  const double inv5 = inv3 * inv2;
  const double t = du * inv5;
  if (P) {
    s.pg = fma(pk, inv3, s.pg);
    s.pe = fma(pk, inv5, s.pe);
  }
  s.gbx = fma(t, dx, s.gbx);
  s.gby = fma(t, dy, s.gby);
  s.gbz = fma(t, dz, s.gbz);
  s.a1x = fma(inv3, wj.x, s.a1x);
  s.a1y = fma(inv3, wj.y, s.a1y);
  s.a1z = fma(inv3, wj.z, s.a1z);
  s.a2 = fma(q.w, inv3, s.a2);
}

template <int BLOCK, int R, int J, bool P>
__global__ void __launch_bounds__(BLOCK) k_vjp_mixed(const PairLaunch L) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  __shared__ __align__(16) float4 tx[J];
  __shared__ __align__(16) float4 tw[J];
  __shared__ int s_item;
  const float4* __restrict__ sx = static_cast<const float4*>(L.stage_x);
  const float4* __restrict__ sw = static_cast<const float4*>(L.stage_w);
  double4_32a* __restrict__ part = reinterpret_cast<double4_32a*>(L.part);
  const float eps2 = (float)L.eps2;

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];

    float xk[R], yk[R], zk[R], mk[R], wkx[R], wky[R], wkz[R];
    Acc8f hi[R], lo[R];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const bool ok = ig[r] < w.i_end;
      const float4 q = ok ? sx[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 u = ok ? sw[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      xk[r] = q.x, yk[r] = q.y, zk[r] = q.z, mk[r] = q.w;
      wkx[r] = u.x, wky[r] = u.y, wkz[r] = u.z;
      hi[r] = Acc8f{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      lo[r] = hi[r];
    }

    float4 px[LPT], pw[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int jj = w.j_begin + (int)threadIdx.x + k * BLOCK;
      if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) px[k] = sx[jj], pw[k] = sw[jj];
    }

    for (int jt = w.j_begin; jt < w.j_end; jt += J) {
      const int nj = min(J, w.j_end - jt);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj) tx[t] = px[k], tw[t] = pw[k];
      }
      __syncthreads();
      if (jt + J < w.j_end) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) px[k] = sx[jj], pw[k] = sw[jj];
        }
      }
      Acc8f s[R];
#pragma unroll
      for (int r = 0; r < R; ++r) s[r] = Acc8f{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      if (diag) {
        for (int j = 0; j < nj; ++j) {
          const float4 q = tx[j], u = tw[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            vjp_pair_f32<true, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r],
                               jt + j == ig[r]);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
          const float4 q = tx[j], u = tw[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            vjp_pair_f32<false, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r], false);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        two_sum_acc(hi[r].a1x, lo[r].a1x, s[r].a1x);
        two_sum_acc(hi[r].a1y, lo[r].a1y, s[r].a1y);
        two_sum_acc(hi[r].a1z, lo[r].a1z, s[r].a1z);
        two_sum_acc(hi[r].a2, lo[r].a2, s[r].a2);
        two_sum_acc(hi[r].gbx, lo[r].gbx, s[r].gbx);
        two_sum_acc(hi[r].gby, lo[r].gby, s[r].gby);
        two_sum_acc(hi[r].gbz, lo[r].gbz, s[r].gbz);
        two_sum_acc(hi[r].gm, lo[r].gm, s[r].gm);
        if (P) {
          two_sum_acc(hi[r].pg, lo[r].pg, s[r].pg);
          two_sum_acc(hi[r].pe, lo[r].pe, s[r].pe);
        }
      }
    }

    constexpr int kW = P ? 3 : 2;  // double4 per body and slice
    double4_32a* out = part + kW * ((int64_t)w.slice * L.n_total);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end) {
        out[kW * (int64_t)ig[r]] =
            make_double4_32a((double)hi[r].a1x + lo[r].a1x, (double)hi[r].a1y + lo[r].a1y,
                         (double)hi[r].a1z + lo[r].a1z, (double)hi[r].a2 + lo[r].a2);
        out[kW * (int64_t)ig[r] + 1] =
            make_double4_32a((double)hi[r].gbx + lo[r].gbx, (double)hi[r].gby + lo[r].gby,
                         (double)hi[r].gbz + lo[r].gbz, (double)hi[r].gm + lo[r].gm);
        if (P)
          out[kW * (int64_t)ig[r] + 2] =
              make_double4_32a((double)hi[r].pg + lo[r].pg, (double)hi[r].pe + lo[r].pe, 0.0, 0.0);
      }
    }
  }
  retire_cta(L.counter);
}

template <int BLOCK, int R, int J, bool P>
__global__ void __launch_bounds__(BLOCK) k_vjp_fp64(const PairLaunch L) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  __shared__ __align__(32) double4_32a tx[J];
  __shared__ __align__(32) double4_32a tw[J];
  __shared__ int s_item;
  const double4_32a* __restrict__ sx = static_cast<const double4_32a*>(L.stage_x);
  const double4_32a* __restrict__ sw = static_cast<const double4_32a*>(L.stage_w);
  double4_32a* __restrict__ part = reinterpret_cast<double4_32a*>(L.part);
  const double eps2 = L.eps2;

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];

    double xk[R], yk[R], zk[R], mk[R], wkx[R], wky[R], wkz[R];
    Acc8d s[R];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const bool ok = ig[r] < w.i_end;
      const double4_32a q = ok ? sx[ig[r]] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
      const double4_32a u = ok ? sw[ig[r]] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
      xk[r] = q.x, yk[r] = q.y, zk[r] = q.z, mk[r] = q.w;
      wkx[r] = u.x, wky[r] = u.y, wkz[r] = u.z;
      s[r] = Acc8d{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    }

    double4_32a px[LPT], pw[LPT];
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int jj = w.j_begin + (int)threadIdx.x + k * BLOCK;
      if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) px[k] = sx[jj], pw[k] = sw[jj];
    }

    for (int jt = w.j_begin; jt < w.j_end; jt += J) {
      const int nj = min(J, w.j_end - jt);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj) tx[t] = px[k], tw[t] = pw[k];
      }
      __syncthreads();
      if (jt + J < w.j_end) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) px[k] = sx[jj], pw[k] = sw[jj];
        }
      }
      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      if (diag) {
        for (int j = 0; j < nj; ++j) {
          const double4_32a q = tx[j], u = tw[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            vjp_pair_f64<true, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r],
                               jt + j == ig[r]);
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < nj; ++j) {
          const double4_32a q = tx[j], u = tw[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            vjp_pair_f64<false, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r], false);
        }
      }
    }

    constexpr int kW = P ? 3 : 2;  // double4 per body and slice
    double4_32a* out = part + kW * ((int64_t)w.slice * L.n_total);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end) {
        out[kW * (int64_t)ig[r]] = make_double4_32a(s[r].a1x, s[r].a1y, s[r].a1z, s[r].a2);
        out[kW * (int64_t)ig[r] + 1] = make_double4_32a(s[r].gbx, s[r].gby, s[r].gbz, s[r].gm);
        if (P) out[kW * (int64_t)ig[r] + 2] = make_double4_32a(s[r].pg, s[r].pe, 0.0, 0.0);
      }
    }
  }
  retire_cta(L.counter);
}

template <typename K>
int occupancy_of(K kern, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, 0) != cudaSuccess) return 0;
  return n;
}

// Tilings compiled for the VJP: BLOCK in {128, 256}, R in {1, 2}, J = 128.
#define NBODY_VJP_TILINGS(X) X(128, 1, 128) X(128, 2, 128) X(256, 1, 128) X(256, 2, 128)

}  // namespace

cudaError_t launch_vjp(int precision, const PairLaunch& L, cudaStream_t st) {
  if (L.n_ctas <= 0) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                                 \
  if (L.block == B && L.ipt == R && L.jtile == J) {                      \
    if (precision == 1 && L.params)                                      \
      k_vjp_mixed<B, R, J, true><<<L.n_ctas, B, 0, st>>>(L);             \
    else if (precision == 1)                                             \
      k_vjp_mixed<B, R, J, false><<<L.n_ctas, B, 0, st>>>(L);            \
    else if (L.params)                                                   \
      k_vjp_fp64<B, R, J, true><<<L.n_ctas, B, 0, st>>>(L);              \
    else                                                                 \
      k_vjp_fp64<B, R, J, false><<<L.n_ctas, B, 0, st>>>(L);             \
    return cudaGetLastError();                                           \
  }
  NBODY_VJP_TILINGS(NBODY_X)
#undef NBODY_X
  return cudaErrorInvalidConfiguration;
}

int vjp_ctas_per_sm(int precision, int block, int ipt, int jtile) {
#define NBODY_X(B, R, J)                                                                              \
  if (block == B && ipt == R && jtile == J)                                                           \
    return precision == 1                                                                             \
               ? std::min(occupancy_of(k_vjp_mixed<B, R, J, false>, B), occupancy_of(k_vjp_mixed<B, R, J, true>, B)) \
               : std::min(occupancy_of(k_vjp_fp64<B, R, J, false>, B), occupancy_of(k_vjp_fp64<B, R, J, true>, B));
  NBODY_VJP_TILINGS(NBODY_X)
#undef NBODY_X
  return 0;
}

}  // namespace nbody
