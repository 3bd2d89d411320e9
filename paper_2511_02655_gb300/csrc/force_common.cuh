// All-pairs force passes of the force kernels (force_kernels.cu): the
// pair arithmetic of the mixed (scalar and packed float32x2) and FP64 paths for
// softened gravity and the Lennard-Jones law (the paper's Eq. 1), and the loops
// over work items, each taking items from an atomic counter until the list is
// exhausted. The design is described in force_kernels.cu.
#pragma once

#include "nbody_internal.h"
#include "pair_common.cuh"

namespace nbody {
namespace fc {


// Near-pair refinement. The float32 staging coordinates carry an absolute
// rounding error of about |x - c| 2^-24, harmless for distant pairs but
// dominant for pairs closer than a few softening lengths. Pairs with s^2 below
// the refinement radius get d recomputed with the staged remainders
// (refine_pair, correct_pair in pair_common.cuh).
// For gravity such pairs are rare, so they are found without a branch per
// pair: every pair folds its s^2 into a running minimum (one FMNMX), and after
// each sub-block of kSub j-bodies a thread whose minimum fell below the radius
// rescans that sub-block (s^2 only) and, for each near pair, adds the refined
// contribution minus the unrefined one it accumulated in the first pass. The
// Lennard-Jones kernel marks near pairs in a bit mask instead (see there).
//
// Compile-time tuning of the mixed kernels. The defaults won a sweep on GB300
// (Plummer N = 65 536 and two spheres N = 1 048 576): 32-body sub-blocks were
// 2-5% faster than 16 or 8; unroll depth 2 vs 4 within 1%; requesting a minimum
// number of resident CTAs did not help; folding both s^2 of a packed pair with one
// three-input min (min.f32 d, a, b, c) instead of two FMNMX was within noise.
//   NBODY_SUB          j-bodies per near-pair check (sub-block)
//   NBODY_QUAD_UNROLL  quads of j-bodies unrolled per packed sub-block loop
//   NBODY_MIN_CTAS     minimum resident CTAs per SM requested in __launch_bounds__ (0: none)
#ifndef NBODY_SUB
#define NBODY_SUB 32
#endif
#ifndef NBODY_QUAD_UNROLL
#define NBODY_QUAD_UNROLL 2
#endif
#ifndef NBODY_MIN_CTAS
#define NBODY_MIN_CTAS 0
#endif
constexpr int kSub = NBODY_SUB;  // j-bodies per near-pair check
constexpr int kQuadUnroll = NBODY_QUAD_UNROLL;

// ---- scalar kernel: one j-body against the thread's R i-bodies per step

template <bool MASK>
__device__ __forceinline__ void pair_f32(const float4 q, const int jg, const int ig, const float xi, const float yi,
                                         const float zi, const float eps2, float& ax, float& ay, float& az, float& pp,
                                         float& mn) {
  const float dx = q.x - xi;
  const float dy = q.y - yi;
  const float dz = q.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  mn = fminf(mn, r2);
  float inv = rsq_approx(r2);
  if (MASK) inv = (jg == ig) ? 0.f : inv;
  const float ms = q.w * inv;        // m_j / s
  const float w = ms * (inv * inv);  // m_j / s^3
  ax = fmaf(dx, w, ax);
  ay = fmaf(dy, w, ay);
  az = fmaf(dz, w, az);
  pp += ms;
}

template <int R, bool MASK>
__device__ __forceinline__ void tile_pass_f32(const float4* tile, const int jt, const int nj, const float (&xi)[R],
                                              const float (&yi)[R], const float (&zi)[R], const int (&ig)[R],
                                              const int i_end, const float eps2, const float r2c,
                                              const float4* __restrict__ lo, float (&ax)[R], float (&ay)[R],
                                              float (&az)[R], float (&pp)[R]) {
  for (int jb = 0; jb < nj; jb += kSub) {
    const int nb = min(kSub, nj - jb);
    float mn = 3.0e38f;
    if (nb == kSub) {
#pragma unroll 8
      for (int j = jb; j < jb + kSub; ++j) {
        const float4 q = tile[j];
#pragma unroll
        for (int r = 0; r < R; ++r)
          pair_f32<MASK>(q, jt + j, ig[r], xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], mn);
      }
    } else {
      for (int j = jb; j < jb + nb; ++j) {
        const float4 q = tile[j];
#pragma unroll
        for (int r = 0; r < R; ++r)
          pair_f32<MASK>(q, jt + j, ig[r], xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], mn);
      }
    }
    if (mn < r2c) {
      for (int j = jb; j < jb + nb; ++j) {
        const float4 q = tile[j];
#pragma unroll
        for (int r = 0; r < R; ++r)
          correct_pair(q, jt + j, ig[r], i_end, xi[r], yi[r], zi[r], eps2, r2c, lo, ax[r], ay[r], az[r], pp[r]);
      }
    }
  }
}

template <int J>
struct SmemMixed {
  float4 tile[2][J];  // double buffer: one barrier per tile
  int item;
};

// Work items of the scalar mixed kernel, taken from `counter` until none is left;
// each writes its slice's compensated float32 sums (fpair4) per i-body.
template <int BLOCK, int R, int J>
__device__ __forceinline__ void items_mixed(const PairLaunch& L, unsigned* counter, SmemMixed<J>& sm) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;  // tile entries loaded per thread
  auto& tile = sm.tile;
  const float4* __restrict__ st = static_cast<const float4*>(L.stage_x);
  fpair4* __restrict__ part = reinterpret_cast<fpair4*>(L.part);
  const float eps2 = (float)L.eps2;
  const float r2c = L.r2_near;
  const float4* __restrict__ lo = L.stage_lo;

  for (;;) {
    const int it = next_item(counter, &sm.item);  // also a barrier: the buffers are free
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

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

    // first tile straight into buffer 0
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int t = (int)threadIdx.x + k * BLOCK;
      if (t < J && w.j_begin + t < w.j_end) tile[0][t] = st[w.j_begin + t];
    }
    __syncthreads();

    int buf = 0;
    for (int jt = w.j_begin; jt < w.j_end; jt += J, buf ^= 1) {
      const int nj = min(J, w.j_end - jt);
      const bool more = jt + J < w.j_end;
      float4 pre[LPT];
      if (more) {  // next tile's loads are in flight while this one is consumed
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
      if (diag)
        tile_pass_f32<R, true>(tile[buf], jt, nj, xi, yi, zi, ig, w.i_end, eps2, r2c, lo, ax, ay, az, pp);
      else
        tile_pass_f32<R, false>(tile[buf], jt, nj, xi, yi, zi, ig, w.i_end, eps2, r2c, lo, ax, ay, az, pp);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        two_sum_acc(hx[r], lx[r], ax[r]);
        two_sum_acc(hy[r], ly[r], ay[r]);
        two_sum_acc(hz[r], lz[r], az[r]);
        two_sum_acc(hp[r], lp[r], pp[r]);
      }
      if (more) {  // the other buffer was last read before the previous barrier
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int t = (int)threadIdx.x + k * BLOCK;
          if (t < J && jt + J + t < w.j_end) tile[buf ^ 1][t] = pre[k];
        }
      }
      __syncthreads();
    }

    fpair4* out = part + (int64_t)w.slice * L.n_total;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end)
        out[ig[r]] = fpair4{make_float4(hx[r], lx[r], hy[r], ly[r]), make_float4(hz[r], lz[r], hp[r], lp[r])};
    }
  }
}

// ---- packed kernel: two j-bodies per float32x2 instruction
//
// The j-tile is kept as structure of arrays (x[], y[], z[], m[]), so one
// 16-byte shared load yields the coordinates of four j-bodies, i.e. two
// float32x2 operands, and each i-body is held once as a duplicated pair
// (-x_i, -x_i). Lane 0 of every float32x2 accumulator sums the even j-bodies
// of a tile, lane 1 the odd ones; the lanes are added when the tile is folded.
// FADD2 / FFMA2 / FMUL2 halve the issue slots of the FMA-pipe work, which
// leaves issue bandwidth for the MUFU, shared-load and minimum instructions.
// Tail tiles are padded to a multiple of four with massless bodies far away.

constexpr float kFarAway = 1.0e18f;

template <bool MASK, bool PHI>
__device__ __forceinline__ void pair2_f32x2(const float2 xj, const float2 yj, const float2 zj, const float2 mj,
                                            const int jg0, const int ig, const float2 nx, const float2 ny,
                                            const float2 nz, const float2 e2, float2& ax, float2& ay, float2& az,
                                            float2& pp, float& mn0, float& mn1) {
  const float2 dx = __fadd2_rn(xj, nx);
  const float2 dy = __fadd2_rn(yj, ny);
  const float2 dz = __fadd2_rn(zj, nz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
  mn0 = fminf(mn0, r2.x);
  mn1 = fminf(mn1, r2.y);
  float2 inv = make_float2(rsq_approx(r2.x), rsq_approx(r2.y));
  if (MASK) {
    inv.x = (jg0 == ig) ? 0.f : inv.x;
    inv.y = (jg0 + 1 == ig) ? 0.f : inv.y;
  }
  const float2 ms = __fmul2_rn(mj, inv);
  const float2 w = __fmul2_rn(ms, __fmul2_rn(inv, inv));
  ax = __ffma2_rn(dx, w, ax);
  ay = __ffma2_rn(dy, w, ay);
  az = __ffma2_rn(dz, w, az);
  if (PHI) pp = __fadd2_rn(pp, ms);
}

// Lennard-Jones pair (Eq. 1) on two j-bodies. The mixed path stages positions
// in units of sigma, so u = sigma^2 / r^2 is the reciprocal of the staged s^2
// itself (eps is scaled alike) and the kernel sums
//   sum (u^3 - 2 u^6) u d'    (a_i = 24 eps / (m_i sigma) times this)
//   sum (u^6 - u^3)           (phi_i = 4 eps / m_i times this),
// 16 float32 operations (8 packed) and one MUFU.RCP per interaction.
// Near pairs are common in a gas (a dozen neighbours inside the 4 sigma
// refinement radius per particle), so instead of a running minimum each pair
// sets its bit in the sub-block's near mask (bit0 for the first j-body, the
// next bit for the second) and the second look visits exactly those pairs.
template <bool MASK, bool PHI>
__device__ __forceinline__ void pair2_lj_f32x2(const float2 xj, const float2 yj, const float2 zj, const int jg0,
                                               const int ig, const float2 nx, const float2 ny, const float2 nz,
                                               const float2 e2, float2& ax, float2& ay, float2& az, float2& pp,
                                               unsigned& near, const unsigned bit0, const float r2c) {
  const float2 dx = __fadd2_rn(xj, nx);
  const float2 dy = __fadd2_rn(yj, ny);
  const float2 dz = __fadd2_rn(zj, nz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
  if (r2.x < r2c) near |= bit0;
  if (r2.y < r2c) near |= bit0 << 1;
  float2 u = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));  // sigma^2 / r^2
  if (MASK) {
    u.x = (jg0 == ig) ? 0.f : u.x;
    u.y = (jg0 + 1 == ig) ? 0.f : u.y;
  }
  const float2 u3 = __fmul2_rn(u, __fmul2_rn(u, u));
  const float2 u6 = __fmul2_rn(u3, u3);
  const float2 w = __fmul2_rn(__ffma2_rn(u6, make_float2(-2.f, -2.f), u3), u);
  ax = __ffma2_rn(dx, w, ax);
  ay = __ffma2_rn(dy, w, ay);
  az = __ffma2_rn(dz, w, az);
  if (PHI) pp = __fadd2_rn(pp, __ffma2_rn(u3, make_float2(-1.f, -1.f), u6));
}

// Four j-bodies (tile entries j..j+3) against the thread's R i-bodies.
template <int LAW, int R, bool MASK, bool PHI>
__device__ __forceinline__ void quad_f32x2(const float* tx, const float* ty, const float* tz, const float* tm,
                                           const int j, const int jg, const int (&ig)[R], const float2 (&nx)[R],
                                           const float2 (&ny)[R], const float2 (&nz)[R], const float2 e2,
                                           const float2 s2, float2 (&ax)[R], float2 (&ay)[R], float2 (&az)[R],
                                           float2 (&pp)[R], float& mn0, float& mn1, unsigned (&near)[R],
                                           const unsigned qbit, const float r2c) {
  const float4 X = *reinterpret_cast<const float4*>(tx + j);
  const float4 Y = *reinterpret_cast<const float4*>(ty + j);
  const float4 Z = *reinterpret_cast<const float4*>(tz + j);
  if (LAW == 0) {
    const float4 M = *reinterpret_cast<const float4*>(tm + j);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      pair2_f32x2<MASK, PHI>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                        make_float2(M.x, M.y), jg, ig[r], nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], pp[r], mn0,
                        mn1);
      pair2_f32x2<MASK, PHI>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                        make_float2(M.z, M.w), jg + 2, ig[r], nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], pp[r],
                        mn0, mn1);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      pair2_lj_f32x2<MASK, PHI>(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y), jg, ig[r], nx[r],
                                ny[r], nz[r], e2, ax[r], ay[r], az[r], pp[r], near[r], qbit, r2c);
      pair2_lj_f32x2<MASK, PHI>(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w), jg + 2, ig[r],
                                nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], pp[r], near[r], qbit << 2, r2c);
    }
  }
}

template <int LAW, int R, bool MASK, bool PHI>
__device__ __forceinline__ void tile_pass_f32x2(const float* tx, const float* ty, const float* tz, const float* tm,
                                                const int jt, const int nj, const int (&ig)[R], const float2 (&nx)[R],
                                                const float2 (&ny)[R], const float2 (&nz)[R], const int i_end,
                                                const float2 e2, const float2 s2, const float r2c,
                                                const float4* __restrict__ lo, float2 (&ax)[R], float2 (&ay)[R],
                                                float2 (&az)[R], float2 (&pp)[R]) {
  static_assert(kSub <= 32, "one near-mask bit per j-body of a sub-block");
  const int nj4 = (nj + 3) & ~3;  // the tile is padded to a multiple of four
  for (int jb = 0; jb < nj4; jb += kSub) {
    const int nb = min(kSub, nj4 - jb);
    float mn0 = 3.0e38f, mn1 = 3.0e38f;
    unsigned near[R];
#pragma unroll
    for (int r = 0; r < R; ++r) near[r] = 0u;
    if (nb == kSub) {
#pragma unroll(kQuadUnroll)
      for (int j = jb; j < jb + kSub; j += 4)
        quad_f32x2<LAW, R, MASK, PHI>(tx, ty, tz, tm, j, jt + j, ig, nx, ny, nz, e2, s2, ax, ay, az, pp, mn0, mn1, near,
                                 1u << (j - jb), r2c);
    } else {
      for (int j = jb; j < jb + nb; j += 4)
        quad_f32x2<LAW, R, MASK, PHI>(tx, ty, tz, tm, j, jt + j, ig, nx, ny, nz, e2, s2, ax, ay, az, pp, mn0, mn1, near,
                                 1u << (j - jb), r2c);
    }
    if (LAW == 1) {
      // Lennard-Jones: correct exactly the flagged pairs (any lane of the partial will do)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        unsigned b = near[r];
        while (b) {
          const int j = jb + __ffs(b) - 1;
          b &= b - 1u;
          if (j < nj)
            correct_pair<LAW>(make_float4(tx[j], ty[j], tz[j], tm[j]), jt + j, ig[r], i_end, -nx[r].x, -ny[r].x,
                              -nz[r].x, e2.x, r2c, lo, ax[r].x, ay[r].x, az[r].x, pp[r].x, s2.x);
        }
      }
    } else if (fminf(mn0, mn1) < r2c) {
      // rescan two j-bodies at a time: packed s^2, scalar correction of the near ones
      for (int j = jb; j < jb + nb; j += 2) {
        const float2 xj = *reinterpret_cast<const float2*>(tx + j);
        const float2 yj = *reinterpret_cast<const float2*>(ty + j);
        const float2 zj = *reinterpret_cast<const float2*>(tz + j);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float2 dx = __fadd2_rn(xj, nx[r]);
          const float2 dy = __fadd2_rn(yj, ny[r]);
          const float2 dz = __fadd2_rn(zj, nz[r]);
          const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
          if (r2.x < r2c && j < nj)
            correct_pair<LAW>(make_float4(tx[j], ty[j], tz[j], tm[j]), jt + j, ig[r], i_end, -nx[r].x, -ny[r].x,
                              -nz[r].x, e2.x, r2c, lo, ax[r].x, ay[r].x, az[r].x, pp[r].x, s2.x);
          if (r2.y < r2c && j + 1 < nj)
            correct_pair<LAW>(make_float4(tx[j + 1], ty[j + 1], tz[j + 1], tm[j + 1]), jt + j + 1, ig[r], i_end,
                              -nx[r].x, -ny[r].x, -nz[r].x, e2.x, r2c, lo, ax[r].y, ay[r].y, az[r].y, pp[r].y,
                              s2.x);
        }
      }
    }
  }
}

// PHI = false skips the potential (one packed operation per pair of interactions
// for gravity, two for Lennard-Jones) when no caller needs it; the partials'
// fourth component is then 0.
template <int J>
struct SmemMixed2 {
  __align__(16) float tx[2][J];  // double buffer: one barrier per tile
  __align__(16) float ty[2][J];
  __align__(16) float tz[2][J];
  __align__(16) float tm[2][J];
  int item;
};

// Work items of the packed mixed kernel, taken from `counter` until none is left;
// each writes its slice's compensated float32 sums (fpair4) per i-body.
template <int LAW, int BLOCK, int R, int J, bool PHI>
__device__ __forceinline__ void items_mixed2(const PairLaunch& L, unsigned* counter, SmemMixed2<J>& sm) {
  static_assert(J % 4 == 0, "tiles hold whole quads of j-bodies");
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  auto& tx = sm.tx;
  auto& ty = sm.ty;
  auto& tz = sm.tz;
  auto& tm = sm.tm;
  const float4* __restrict__ st = static_cast<const float4*>(L.stage_x);
  fpair4* __restrict__ part = reinterpret_cast<fpair4*>(L.part);
  const float eps2 = (float)L.eps2;
  const float2 e2 = make_float2(eps2, eps2);
  const float2 s2 = make_float2((float)L.sigma2, (float)L.sigma2);
  const float r2c = L.r2_near;
  const float4* __restrict__ lo = L.stage_lo;

  for (;;) {
    const int it = next_item(counter, &sm.item);  // also a barrier: the buffers are free
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

    float2 nx[R], ny[R], nz[R];
    float hx[R], hy[R], hz[R], hp[R], lx[R], ly[R], lz[R], lp[R];
    int ig[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ig[r] = w.i_begin + (int)threadIdx.x + r * BLOCK;
      const float4 q = ig[r] < w.i_end ? st[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
      nx[r] = make_float2(-q.x, -q.x);
      ny[r] = make_float2(-q.y, -q.y);
      nz[r] = make_float2(-q.z, -q.z);
      hx[r] = hy[r] = hz[r] = hp[r] = 0.f;
      lx[r] = ly[r] = lz[r] = lp[r] = 0.f;
    }

    // first tile straight into buffer 0 (padded to a whole quad with far, massless bodies)
    {
      const int nj = min(J, w.j_end - w.j_begin), nj4 = (nj + 3) & ~3;
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int t = (int)threadIdx.x + k * BLOCK;
        if (t < nj) {
          const float4 q = st[w.j_begin + t];
          tx[0][t] = q.x, ty[0][t] = q.y, tz[0][t] = q.z, tm[0][t] = q.w;
        } else if (t < nj4) {
          tx[0][t] = kFarAway, ty[0][t] = kFarAway, tz[0][t] = kFarAway, tm[0][t] = 0.f;
        }
      }
    }
    __syncthreads();

    int buf = 0;
    for (int jt = w.j_begin; jt < w.j_end; jt += J, buf ^= 1) {
      const int nj = min(J, w.j_end - jt);
      const bool more = jt + J < w.j_end;
      float4 pre[LPT];
      if (more) {
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int jj = jt + J + (int)threadIdx.x + k * BLOCK;
          if ((int)threadIdx.x + k * BLOCK < J && jj < w.j_end) pre[k] = st[jj];
        }
      }

      float2 ax[R], ay[R], az[R], pp[R];
#pragma unroll
      for (int r = 0; r < R; ++r) ax[r] = ay[r] = az[r] = pp[r] = make_float2(0.f, 0.f);
      const bool diag = (jt < w.i_end) && (w.i_begin < jt + nj);
      if (diag)
        tile_pass_f32x2<LAW, R, true, PHI>(tx[buf], ty[buf], tz[buf], tm[buf], jt, nj, ig, nx, ny, nz, w.i_end, e2, s2,
                                      r2c, lo, ax, ay, az, pp);
      else
        tile_pass_f32x2<LAW, R, false, PHI>(tx[buf], ty[buf], tz[buf], tm[buf], jt, nj, ig, nx, ny, nz, w.i_end, e2, s2,
                                       r2c, lo, ax, ay, az, pp);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        two_sum_acc(hx[r], lx[r], ax[r].x + ax[r].y);
        two_sum_acc(hy[r], ly[r], ay[r].x + ay[r].y);
        two_sum_acc(hz[r], lz[r], az[r].x + az[r].y);
        two_sum_acc(hp[r], lp[r], pp[r].x + pp[r].y);
      }
      if (more) {  // the other buffer was last read before the previous barrier
        const int nn = min(J, w.j_end - jt - J), nn4 = (nn + 3) & ~3;
        const int b = buf ^ 1;
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
          const int t = (int)threadIdx.x + k * BLOCK;
          if (t < nn) {
            tx[b][t] = pre[k].x, ty[b][t] = pre[k].y, tz[b][t] = pre[k].z, tm[b][t] = pre[k].w;
          } else if (t < nn4) {
            tx[b][t] = kFarAway, ty[b][t] = kFarAway, tz[b][t] = kFarAway, tm[b][t] = 0.f;
          }
        }
      }
      __syncthreads();
    }

    fpair4* out = part + (int64_t)w.slice * L.n_total;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ig[r] < w.i_end)
        out[ig[r]] = fpair4{make_float4(hx[r], lx[r], hy[r], ly[r]), make_float4(hz[r], lz[r], hp[r], lp[r])};
    }
  }
}

template <int LAW, bool MASK>
__device__ __forceinline__ void pair_f64(const double4_32a q, const double xi, const double yi, const double zi,
                                         const double eps2, const double s2, double& ax, double& ay, double& az,
                                         double& pp, const bool self) {
  const double dx = q.x - xi;
  const double dy = q.y - yi;
  const double dz = q.z - zi;
  const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  if (LAW == 0) {
    double inv = rsqrt(r2);
    if (MASK) inv = self ? 0.0 : inv;
    const double ms = q.w * inv;
    const double w = ms * (inv * inv);
    ax = fma(dx, w, ax);
    ay = fma(dy, w, ay);
    az = fma(dz, w, az);
    pp += ms;
  } else {  // Lennard-Jones, u = sigma^2 / r^2
    double inv2 = 1.0 / r2;
    if (MASK) inv2 = self ? 0.0 : inv2;
    const double u = s2 * inv2, u3 = u * u * u, u6 = u3 * u3;
    const double w = (u3 - 2.0 * u6) * inv2;
    ax = fma(dx, w, ax);
    ay = fma(dy, w, ay);
    az = fma(dz, w, az);
    pp += u6 - u3;
  }
}

template <int J>
struct SmemFp64 {
  double4_32a tile[J];
  int item;
};

// Work items of the FP64 kernel, taken from `counter` until none is left.
template <int LAW, int BLOCK, int R, int J>
__device__ __forceinline__ void items_fp64(const PairLaunch& L, unsigned* counter, SmemFp64<J>& sm) {
  constexpr int LPT = (J + BLOCK - 1) / BLOCK;
  auto& tile = sm.tile;
  const double4_32a* __restrict__ st = static_cast<const double4_32a*>(L.stage_x);
  double4_32a* __restrict__ part = reinterpret_cast<double4_32a*>(L.part);
  const double eps2 = L.eps2;
  const double s2 = L.sigma2;

  for (;;) {
    const int it = next_item(counter, &sm.item);
    if (it >= L.n_items) break;
    const WorkItem w = L.items[it];
    if (!item_ok(w, L)) continue;  // NBODY_DEBUG builds only

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
            pair_f64<LAW, true>(q, xi[r], yi[r], zi[r], eps2, s2, ax[r], ay[r], az[r], pp[r], jt + j == ig[r]);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
          const double4_32a q = tile[j];
#pragma unroll
          for (int r = 0; r < R; ++r)
            pair_f64<LAW, false>(q, xi[r], yi[r], zi[r], eps2, s2, ax[r], ay[r], az[r], pp[r], false);
        }
      }
    }

    double4_32a* out = part + (int64_t)w.slice * L.n_total;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (ig[r] < w.i_end) out[ig[r]] = make_double4_32a(ax[r], ay[r], az[r], pp[r]);
  }
}


}  // namespace fc
}  // namespace nbody

// Tilings compiled. Softened gravity: BLOCK in {128, 256}, R in {1, 2, 4},
// J in {128, 256} for every kernel, and J = 512 for the two mixed kernels.
// Lennard-Jones: the packed mixed kernel and the FP64 kernel on the subsets below.
#define NBODY_FORCE_TILINGS(X) \
  X(128, 1, 128) X(128, 2, 128) X(128, 4, 128) X(128, 1, 256) X(128, 2, 256) X(128, 4, 256) \
  X(256, 1, 128) X(256, 2, 128) X(256, 4, 128) X(256, 1, 256) X(256, 2, 256) X(256, 4, 256)
#define NBODY_MIXED_TILINGS(X) \
  NBODY_FORCE_TILINGS(X) X(128, 1, 512) X(128, 2, 512) X(128, 4, 512) X(256, 1, 512) X(256, 2, 512) X(256, 4, 512)
// The register-capped packed variant (4 CTAs per SM): softened gravity only.
#define NBODY_CAPPED_TILINGS(X) X(128, 2, 256)
// The register-capped Lennard-Jones variant (6 CTAs per SM, <= 85 registers).
#define NBODY_LJ_CAPPED_TILINGS(X) X(128, 1, 256) X(128, 1, 512)
#define NBODY_LJ_MIXED_TILINGS(X) \
  X(128, 1, 256) X(256, 1, 256) X(128, 2, 256) X(128, 1, 512) X(256, 1, 512) X(256, 2, 512)
#define NBODY_LJ_FP64_TILINGS(X) X(128, 1, 128) X(256, 1, 128) X(128, 2, 128) X(256, 2, 128)
