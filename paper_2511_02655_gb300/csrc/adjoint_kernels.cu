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
// cost two float32 operations more per pair and a third partial per body and slice.
// Partials are written per work item and slice: on the mixed path as the
// compensated float32 sums themselves (fpair4), float64 on the FP64 path.
// Tiling, work distribution, self-pair masking, the compensated per-tile fold
// and the near-pair refinement (pairs with s^2 below r2_near recomputed from the
// staged float32 remainders, found through a running minimum of s^2 per
// sub-block of kSubV j-bodies) are those of the force kernels.
#include <algorithm>
#include <type_traits>

#include "nbody_internal.h"
#include "pair_common.cuh"

namespace nbody {
namespace {

constexpr int kSubV = 32;  // j-bodies per near-pair check

struct Acc8f {
  float a1x, a1y, a1z, a2, gbx, gby, gbz, gm, pg, pe;
};

template <bool MASK, bool P>
__device__ __forceinline__ void vjp_pair_f32(const float4 q, const float4 wj, const float xk, const float yk,
                                             const float zk, const float mk, const float wkx, const float wky,
                                             const float wkz, const float eps2, Acc8f& s, const bool self,
                                             float& mn) {
  const float dx = q.x - xk;
  const float dy = q.y - yk;
  const float dz = q.z - zk;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  mn = fminf(mn, r2);
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

// The VJP terms of one pair with separation d and s^2 = r2, scaled by sg
// (+1 adds them, -1 removes them): the same operations as vjp_pair_f32 and
// vjp_pair2, so that a removed unrefined term matches the one accumulated.
template <bool P>
__device__ __forceinline__ void vjp_terms_f32(const float dx, const float dy, const float dz, const float r2,
                                              const float mj, const float wjx, const float wjy, const float wjz,
                                              const float mk, const float wkx, const float wky, const float wkz,
                                              const float sg, Acc8f& s) {
  const float inv = rsq_approx(r2);
  const float inv2 = inv * inv;
  const float inv3 = inv2 * inv;
  const float dwj = fmaf(dx, wjx, fmaf(dy, wjy, dz * wjz));
  const float dwk = fmaf(dx, wkx, fmaf(dy, wky, dz * wkz));
  const float pk = mj * dwk;
  const float du = fmaf(mk, dwj, -pk);
  const float inv5 = inv3 * inv2;
  const float t = (du * inv5) * sg;
  const float i3 = inv3 * sg;
  s.gm = fmaf(dwj, i3, s.gm);
  if (P) {
    s.pg = fmaf(pk, i3, s.pg);
    s.pe = fmaf(pk, inv5 * sg, s.pe);
  }
  s.gbx = fmaf(t, dx, s.gbx);
  s.gby = fmaf(t, dy, s.gby);
  s.gbz = fmaf(t, dz, s.gbz);
  s.a1x = fmaf(i3, wjx, s.a1x);
  s.a1y = fmaf(i3, wjy, s.a1y);
  s.a1z = fmaf(i3, wjz, s.a1z);
  s.a2 = fmaf(mj, i3, s.a2);
}

// Second look at one pair of a flagged sub-block (j-body at global index jg
// with staged (q, m_j) and weight w_j, i-body k at ig): if it is near and not
// the self pair, its unrefined terms in s are replaced by those of the
// separation refined with the staged remainders (refine_pair).
template <bool P>
__device__ __forceinline__ void vjp_correct_f32(const float qx, const float qy, const float qz, const float mj,
                                                const float wjx, const float wjy, const float wjz, const int jg,
                                                const int ig, const int i_end, const float xk, const float yk,
                                                const float zk, const float mk, const float wkx, const float wky,
                                                const float wkz, const float eps2, const float r2c,
                                                const float4* __restrict__ lo, Acc8f& s) {
  const float dx = qx - xk;
  const float dy = qy - yk;
  const float dz = qz - zk;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  if (!(r2 < r2c) || ig >= i_end || jg < 0 || ig == jg) return;
  float rx, ry, rz, rr2;
  refine_pair(lo, ig, jg, dx, dy, dz, eps2, rx, ry, rz, rr2);
  vjp_terms_f32<P>(dx, dy, dz, r2, mj, wjx, wjy, wjz, mk, wkx, wky, wkz, -1.f, s);
  vjp_terms_f32<P>(rx, ry, rz, rr2, mj, wjx, wjy, wjz, mk, wkx, wky, wkz, 1.f, s);
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
  fpair4* __restrict__ part = reinterpret_cast<fpair4*>(L.part);
  const float eps2 = (float)L.eps2;
  const float r2c = L.r2_near;
  const float4* __restrict__ slo = L.stage_lo;

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

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
      for (int jb = 0; jb < nj; jb += kSubV) {
        const int je = min(nj, jb + kSubV);
        float mn = 3.0e38f;
        if (diag) {
          for (int j = jb; j < je; ++j) {
            const float4 q = tx[j], u = tw[j];
#pragma unroll
            for (int r = 0; r < R; ++r)
              vjp_pair_f32<true, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r],
                                    jt + j == ig[r], mn);
          }
        } else {
#pragma unroll 4
          for (int j = jb; j < je; ++j) {
            const float4 q = tx[j], u = tw[j];
#pragma unroll
            for (int r = 0; r < R; ++r)
              vjp_pair_f32<false, P>(q, u, xk[r], yk[r], zk[r], mk[r], wkx[r], wky[r], wkz[r], eps2, s[r], false,
                                     mn);
          }
        }
        if (mn < r2c) {
          for (int j = jb; j < je; ++j) {
            const float4 q = tx[j], u = tw[j];
#pragma unroll
            for (int r = 0; r < R; ++r)
              vjp_correct_f32<P>(q.x, q.y, q.z, q.w, u.x, u.y, u.z, jt + j, ig[r], w.i_end, xk[r], yk[r], zk[r],
                                 mk[r], wkx[r], wky[r], wkz[r], eps2, r2c, slo, s[r]);
          }
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

    constexpr int kW = P ? 3 : 2;  // fpair4 per body and slice
    fpair4* out = part + kW * ((int64_t)w.slice * L.n_total);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end) {
        out[kW * (int64_t)ig[r]] = fpair4{make_float4(hi[r].a1x, lo[r].a1x, hi[r].a1y, lo[r].a1y),
                                          make_float4(hi[r].a1z, lo[r].a1z, hi[r].a2, lo[r].a2)};
        out[kW * (int64_t)ig[r] + 1] = fpair4{make_float4(hi[r].gbx, lo[r].gbx, hi[r].gby, lo[r].gby),
                                              make_float4(hi[r].gbz, lo[r].gbz, hi[r].gm, lo[r].gm)};
        if (P)
          out[kW * (int64_t)ig[r] + 2] =
              fpair4{make_float4(hi[r].pg, lo[r].pg, hi[r].pe, lo[r].pe), make_float4(0.f, 0.f, 0.f, 0.f)};
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
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

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

// ---- packed float32x2 form: two j-bodies per instruction (j-pairs from a
// structure-of-arrays tile, the i-body duplicated in both lanes), 13 packed
// FMA-pipe operations and two MUFU.RSQ per pair of interactions. The tile holds
// -m_j, so that the one subtraction of the pair (m_k (d.w_j) - m_j (d.w_k))
// needs no negation: A2, Pg and Pe are accumulated negated and flipped at the end.

struct Acc2 {
  float2 a1x, a1y, a1z, a2n, gbx, gby, gbz, gm, pgn, pen;
};

template <bool MASK, bool P>
__device__ __forceinline__ void vjp_pair2(const float2 xj, const float2 yj, const float2 zj, const float2 mjn,
                                          const float2 wxj, const float2 wyj, const float2 wzj, const int jg0,
                                          const int ig, const float2 nx, const float2 ny, const float2 nz,
                                          const float2 mk, const float2 wkx, const float2 wky, const float2 wkz,
                                          const float2 e2, Acc2& s, float& mn) {
  const float2 dx = __fadd2_rn(xj, nx);
  const float2 dy = __fadd2_rn(yj, ny);
  const float2 dz = __fadd2_rn(zj, nz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
  mn = fminf(mn, fminf(r2.x, r2.y));
  float2 inv = make_float2(rsq_approx(r2.x), rsq_approx(r2.y));
  if (MASK) {
    inv.x = (jg0 == ig) ? 0.f : inv.x;
    inv.y = (jg0 + 1 == ig) ? 0.f : inv.y;
  }
  const float2 inv2 = __fmul2_rn(inv, inv);
  const float2 inv3 = __fmul2_rn(inv2, inv);
  const float2 dwj = __ffma2_rn(dx, wxj, __ffma2_rn(dy, wyj, __fmul2_rn(dz, wzj)));
  const float2 dwk = __ffma2_rn(dx, wkx, __ffma2_rn(dy, wky, __fmul2_rn(dz, wkz)));
  s.gm = __ffma2_rn(dwj, inv3, s.gm);
  const float2 pkn = __fmul2_rn(mjn, dwk);      // -m_j (d.w_k)
  const float2 du = __ffma2_rn(mk, dwj, pkn);   // m_k (d.w_j) - m_j (d.w_k)
  const float2 inv5 = __fmul2_rn(inv3, inv2);
  const float2 t = __fmul2_rn(du, inv5);
  s.gbx = __ffma2_rn(t, dx, s.gbx);
  s.gby = __ffma2_rn(t, dy, s.gby);
  s.gbz = __ffma2_rn(t, dz, s.gbz);
  s.a1x = __ffma2_rn(inv3, wxj, s.a1x);
  s.a1y = __ffma2_rn(inv3, wyj, s.a1y);
  s.a1z = __ffma2_rn(inv3, wzj, s.a1z);
  s.a2n = __ffma2_rn(mjn, inv3, s.a2n);
  if (P) {
    s.pgn = __ffma2_rn(pkn, inv3, s.pgn);
    s.pen = __ffma2_rn(pkn, inv5, s.pen);
  }
}

// far, massless, weightless padding of a tile to whole quads
constexpr float kFarAwayV = 1.0e18f;

template <int BLOCK, int R, int J, bool P>
__global__ void __launch_bounds__(BLOCK) k_vjp_mixed2(const PairLaunch L) {
  static_assert(J % 4 == 0, "tiles hold whole quads of j-bodies");
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  constexpr int NC = P ? 10 : 8;  // compensated components per i-body
  __shared__ __align__(16) float tx[2][J], ty[2][J], tz[2][J], tmn[2][J];
  __shared__ __align__(16) float twx[2][J], twy[2][J], twz[2][J];
  __shared__ int s_item;
  const float4* __restrict__ sx = static_cast<const float4*>(L.stage_x);
  const float4* __restrict__ sw = static_cast<const float4*>(L.stage_w);
  fpair4* __restrict__ part = reinterpret_cast<fpair4*>(L.part);
  const float eps2 = (float)L.eps2;
  const float2 e2 = make_float2(eps2, eps2);
  const float r2c = L.r2_near;
  const float4* __restrict__ slo = L.stage_lo;

  auto put = [&](const int b, const int t, const float4 q, const float4 u) {
    tx[b][t] = q.x, ty[b][t] = q.y, tz[b][t] = q.z, tmn[b][t] = -q.w;
    twx[b][t] = u.x, twy[b][t] = u.y, twz[b][t] = u.z;
  };
  auto pad = [&](const int b, const int t) {
    tx[b][t] = kFarAwayV, ty[b][t] = kFarAwayV, tz[b][t] = kFarAwayV, tmn[b][t] = 0.f;
    twx[b][t] = 0.f, twy[b][t] = 0.f, twz[b][t] = 0.f;
  };

  for (;;) {
    const int it = next_item(L.counter, &s_item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

    float2 nx[R], ny[R], nz[R], mk[R], wkx[R], wky[R], wkz[R];
    float hi[R][NC], lo[R][NC];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const bool ok = ig[r] < w.i_end;
      const float4 q = ok ? sx[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 u = ok ? sw[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      nx[r] = make_float2(-q.x, -q.x), ny[r] = make_float2(-q.y, -q.y), nz[r] = make_float2(-q.z, -q.z);
      mk[r] = make_float2(q.w, q.w);
      wkx[r] = make_float2(u.x, u.x), wky[r] = make_float2(u.y, u.y), wkz[r] = make_float2(u.z, u.z);
#pragma unroll
      for (int c = 0; c < NC; ++c) hi[r][c] = lo[r][c] = 0.f;
    }

    {
      const int nj = min(J, w.j_end - w.j_begin), nj4 = (nj + 3) & ~3;
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj)
          put(0, t, sx[w.j_begin + t], sw[w.j_begin + t]);
        else if (t < nj4)
          pad(0, t);
      }
    }
    __syncthreads();

    int buf = 0;
    for (int jt = w.j_begin; jt < w.j_end; jt += J, buf ^= 1) {
      const int nj = min(J, w.j_end - jt), nj4 = (nj + 3) & ~3;
      const bool more = jt + J < w.j_end;
      float4 px[LPT], pw[LPT];
      if (more) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) px[k] = sx[jj], pw[k] = sw[jj];
        }
      }
      Acc2 s[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 z = make_float2(0.f, 0.f);
        s[r] = Acc2{z, z, z, z, z, z, z, z, z, z};
      }
      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      const float *cx = tx[buf], *cy = ty[buf], *cz = tz[buf], *cm = tmn[buf];
      const float *cwx = twx[buf], *cwy = twy[buf], *cwz = twz[buf];
      auto quad = [&](const int j, auto mask, float& mn) {
        constexpr bool M = decltype(mask)::value;
        const float4 X = *reinterpret_cast<const float4*>(cx + j);
        const float4 Y = *reinterpret_cast<const float4*>(cy + j);
        const float4 Z = *reinterpret_cast<const float4*>(cz + j);
        const float4 Mn = *reinterpret_cast<const float4*>(cm + j);
        const float4 WX = *reinterpret_cast<const float4*>(cwx + j);
        const float4 WY = *reinterpret_cast<const float4*>(cwy + j);
        const float4 WZ = *reinterpret_cast<const float4*>(cwz + j);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          vjp_pair2<M, P>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                          make_float2(Mn.x, Mn.y), make_float2(WX.x, WX.y), make_float2(WY.x, WY.y),
                          make_float2(WZ.x, WZ.y), jt + j, ig[r], nx[r], ny[r], nz[r], mk[r], wkx[r], wky[r],
                          wkz[r], e2, s[r], mn);
          vjp_pair2<M, P>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                          make_float2(Mn.z, Mn.w), make_float2(WX.z, WX.w), make_float2(WY.z, WY.w),
                          make_float2(WZ.z, WZ.w), jt + j + 2, ig[r], nx[r], ny[r], nz[r], mk[r], wkx[r], wky[r],
                          wkz[r], e2, s[r], mn);
        }
      };
      // near-pair corrections of one j-body of the tile for every i-body of the thread,
      // added to lane 0 of the packed sums (the lanes are added at the fold; A2, Pg, Pe
      // are held negated)
      auto correct = [&](const int j) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          Acc8f d{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          vjp_correct_f32<P>(cx[j], cy[j], cz[j], -cm[j], cwx[j], cwy[j], cwz[j], jt + j, ig[r], w.i_end, -nx[r].x,
                             -ny[r].x, -nz[r].x, mk[r].x, wkx[r].x, wky[r].x, wkz[r].x, eps2, r2c, slo, d);
          s[r].a1x.x += d.a1x, s[r].a1y.x += d.a1y, s[r].a1z.x += d.a1z, s[r].a2n.x -= d.a2;
          s[r].gbx.x += d.gbx, s[r].gby.x += d.gby, s[r].gbz.x += d.gbz, s[r].gm.x += d.gm;
          if (P) s[r].pgn.x -= d.pg, s[r].pen.x -= d.pe;
        }
      };
      // first pass: one bit per sub-block whose minimum s^2 fell below the radius; the
      // flagged sub-blocks are revisited after the whole tile (fewer live registers in
      // the pair loop than a rescan inside it)
      static_assert(J / kSubV <= 32, "one flag bit per sub-block of a tile");
      unsigned flagged = 0u;
      for (int jb = 0; jb < nj4; jb += kSubV) {
        const int je = min(nj4, jb + kSubV);
        float mn = 3.0e38f;
        if (diag) {
          for (int j = jb; j < je; j += 4) quad(j, std::true_type{}, mn);
        } else {
#pragma unroll 2
          for (int j = jb; j < je; j += 4) quad(j, std::false_type{}, mn);
        }
        if (mn < r2c) flagged |= 1u << (jb / kSubV);
      }
      while (flagged) {
        const int jb = (__ffs(flagged) - 1) * kSubV;
        flagged &= flagged - 1u;
        for (int j = jb; j < min(jb + kSubV, nj); ++j) correct(j);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float v[10] = {s[r].a1x.x + s[r].a1x.y, s[r].a1y.x + s[r].a1y.y, s[r].a1z.x + s[r].a1z.y,
                             -(s[r].a2n.x + s[r].a2n.y), s[r].gbx.x + s[r].gbx.y, s[r].gby.x + s[r].gby.y,
                             s[r].gbz.x + s[r].gbz.y, s[r].gm.x + s[r].gm.y, -(s[r].pgn.x + s[r].pgn.y),
                             -(s[r].pen.x + s[r].pen.y)};
#pragma unroll
        for (int c = 0; c < NC; ++c) two_sum_acc(hi[r][c], lo[r][c], v[c]);
      }
      if (more) {
        const int nn = min(J, w.j_end - jt - J), nn4 = (nn + 3) & ~3;
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int t = (int)threadIdx.x + k * BLOCK;
          if (t < nn)
            put(buf ^ 1, t, px[k], pw[k]);
          else if (t < nn4)
            pad(buf ^ 1, t);
        }
      }
      __syncthreads();
    }

    constexpr int kW = P ? 3 : 2;  // fpair4 per body and slice
    fpair4* out = part + kW * ((int64_t)w.slice * L.n_total);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end) {
        const float(&h)[NC] = hi[r];
        const float(&l)[NC] = lo[r];
        out[kW * (int64_t)ig[r]] =
            fpair4{make_float4(h[0], l[0], h[1], l[1]), make_float4(h[2], l[2], h[3], l[3])};
        out[kW * (int64_t)ig[r] + 1] =
            fpair4{make_float4(h[4], l[4], h[5], l[5]), make_float4(h[6], l[6], h[7], l[7])};
        if constexpr (P)
          out[kW * (int64_t)ig[r] + 2] = fpair4{make_float4(h[8], l[8], h[9], l[9]), make_float4(0.f, 0.f, 0.f, 0.f)};
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

// Tilings compiled for the VJP: BLOCK in {128, 256}, R in {1, 2}, J in {128, 256}.
#define NBODY_VJP_TILINGS(X) \
  X(128, 1, 128) X(128, 2, 128) X(256, 1, 128) X(256, 2, 128) X(128, 1, 256) X(128, 2, 256) X(256, 1, 256) X(256, 2, 256)

}  // namespace

cudaError_t launch_vjp(int precision, const PairLaunch& L, cudaStream_t st) {
  if (L.n_ctas <= 0) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                                 \
  if (L.block == B && L.ipt == R && L.jtile == J) {                      \
    if (precision == 1 && L.variant == 1 && L.params)                    \
      k_vjp_mixed2<B, R, J, true><<<L.n_ctas, B, 0, st>>>(L);            \
    else if (precision == 1 && L.variant == 1)                           \
      k_vjp_mixed2<B, R, J, false><<<L.n_ctas, B, 0, st>>>(L);           \
    else if (precision == 1 && L.params)                                 \
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

int vjp_ctas_per_sm(int precision, int variant, int block, int ipt, int jtile) {
  if (variant != 0 && (variant != 1 || precision != 1)) return 0;
#define NBODY_X(B, R, J)                                                                                     \
  if (block == B && ipt == R && jtile == J) {                                                                \
    if (precision == 1 && variant == 1)                                                                      \
      return std::min(occupancy_of(k_vjp_mixed2<B, R, J, false>, B), occupancy_of(k_vjp_mixed2<B, R, J, true>, B)); \
    return precision == 1                                                                                    \
               ? std::min(occupancy_of(k_vjp_mixed<B, R, J, false>, B), occupancy_of(k_vjp_mixed<B, R, J, true>, B)) \
               : std::min(occupancy_of(k_vjp_fp64<B, R, J, false>, B), occupancy_of(k_vjp_fp64<B, R, J, true>, B)); \
  }
  NBODY_VJP_TILINGS(NBODY_X)
#undef NBODY_X
  return 0;
}

}  // namespace nbody
