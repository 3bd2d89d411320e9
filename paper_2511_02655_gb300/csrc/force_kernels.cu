// All-pairs force kernels (the paper's force calculation over "N_p^2
// operations", Sec. V-B, with the energy term fused into the same loop,
// Sec. VI) for softened gravity and for the paper's Lennard-Jones law (Eq. 1).
// Two precisions:
//
//   mixed : staged j-bodies are float4 (x - c, y - c, z - c, m) with c the
//           system's staging origin; each interaction is 3 FADD + 3 FFMA +
//           1 MUFU.RSQ + 3 FMUL + 3 FFMA + 1 FADD in float32; per j-tile the
//           float32 partial sums are folded into a compensated (hi, lo) float32
//           pair per body (TwoSum), written per work item as it is (fpair4).
//   fp64  : staged double4_32a (x, y, z, m), every operation in float64.
//
// The mixed path has a scalar kernel and a packed one (two j-bodies per
// float32x2 instruction); the autotuner picks. The packed kernel also comes
// without the potential term, for passes that need no energy.
// Both precisions are persistent kernels over a work list of (i-tile, j-slice) items.
// i-bodies live in registers (R per thread, strided by the CTA size so loads
// and stores coalesce), j-bodies stream through a shared-memory tile that
// every thread reads with broadcast loads; the next tile is prefetched into
// registers while the current one is consumed. Each item writes one partial
// (sum m d / s^3, sum m / s) per i-body to its slice, float64 on the FP64 path
// and compensated float32 pairs on the mixed path; the O(N) post kernel adds
// the slices in a fixed order, so results are deterministic.
// Self pairs are masked in the tiles that overlap the item's own i-range.
#include <algorithm>

#include "force_common.cuh"
#include "nbody_internal.h"

namespace nbody {
namespace {

// Standalone force kernels: one pass over the work list, then the last CTA to
// retire resets the item counter for the next launch. They are launched as
// programmatic dependents (launch_pdl): pdl_wait() holds every CTA until the
// kernel before them on the stream has completed, so only the launch latency
// overlaps with that kernel's tail.
template <int BLOCK, int R, int J>
__global__ void __launch_bounds__(BLOCK) k_force_mixed(const PairLaunch L) {
  __shared__ fc::SmemMixed<J> sm;
  pdl_wait();
  fc::items_mixed<BLOCK, R, J>(L, L.counter, sm);
  pdl_trigger();
  retire_cta(L.counter);
}

// Resident CTAs per SM each packed tiling is compiled for (a register bound of
// 65 536 / (BLOCK x CTAs)): the occupancy its register use gives anyway, pinned
// down so that small code changes cannot push a tiling over an allocation edge
// (the 128 x 2 x 512 kernel once grew from 162 to 170 registers and fell from 3
// to 2 CTAs per SM, 3% slower).
constexpr int packed_min_ctas(int block, int r) {
  return block == 128 ? (r == 1 ? 4 : r == 2 ? 3 : 2) : (r == 1 ? 2 : 1);
}

// MINB > 0 asks for MINB resident CTAs instead (a tighter register cap): the
// 128 x 2 x 256 tiling at 4 CTAs per SM is ~1% faster at N = 65 536 but ~4%
// slower at N = 262 144 than at 3, so the tuner gets both (variant 3 of
// nbody_config). (The same cap on the 512-body tile timed well on the tuner's
// synthetic sphere but 3% slower on real inputs.)
template <int LAW, int BLOCK, int R, int J, bool PHI, int MINB = 0>
__global__ void __launch_bounds__(BLOCK, (MINB > 0 ? MINB
                                                  : (NBODY_MIN_CTAS > 0 ? NBODY_MIN_CTAS : packed_min_ctas(BLOCK, R))))
    k_force_mixed2(const PairLaunch L) {
  __shared__ fc::SmemMixed2<J> sm;
  pdl_wait();
  fc::items_mixed2<LAW, BLOCK, R, J, PHI>(L, L.counter, sm);
  pdl_trigger();
  retire_cta(L.counter);
}

template <int LAW, int BLOCK, int R, int J>
__global__ void __launch_bounds__(BLOCK) k_force_fp64(const PairLaunch L) {
  __shared__ fc::SmemFp64<J> sm;
  pdl_wait();
  fc::items_fp64<LAW, BLOCK, R, J>(L, L.counter, sm);
  pdl_trigger();
  retire_cta(L.counter);
}

template <typename K>
int occupancy_of(K kern, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, 0) != cudaSuccess) return 0;
  return n;
}

}  // namespace

cudaError_t launch_force(int precision, const PairLaunch& L, cudaStream_t st) {
  if (L.n_ctas <= 0) return cudaErrorInvalidConfiguration;
  if (L.law == 1) {
    if (precision == 1 && L.variant == 2) {  // register-capped: 6 CTAs per SM
#define NBODY_X(B, R, J)                                               \
  if (L.block == B && L.ipt == R && L.jtile == J) {                    \
    if (L.phi)                                                         \
      return launch_pdl(k_force_mixed2<1, B, R, J, true, 6>, L.n_ctas, B, st, L);  \
    else                                                               \
      return launch_pdl(k_force_mixed2<1, B, R, J, false, 6>, L.n_ctas, B, st, L); \
  }
      NBODY_LJ_CAPPED_TILINGS(NBODY_X)
#undef NBODY_X
      return cudaErrorInvalidConfiguration;
    }
    if (precision == 1) {
      if (L.variant != 1) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                               \
  if (L.block == B && L.ipt == R && L.jtile == J) {                    \
    if (L.phi)                                                         \
      return launch_pdl(k_force_mixed2<1, B, R, J, true>, L.n_ctas, B, st, L);     \
    else                                                               \
      return launch_pdl(k_force_mixed2<1, B, R, J, false>, L.n_ctas, B, st, L);    \
  }
      NBODY_LJ_MIXED_TILINGS(NBODY_X)
#undef NBODY_X
      return cudaErrorInvalidConfiguration;
    }
#define NBODY_X(B, R, J)                                               \
  if (L.block == B && L.ipt == R && L.jtile == J) {                    \
    return launch_pdl(k_force_fp64<1, B, R, J>, L.n_ctas, B, st, L);               \
  }
    if (L.variant != 0) return cudaErrorInvalidConfiguration;
    NBODY_LJ_FP64_TILINGS(NBODY_X)
#undef NBODY_X
    return cudaErrorInvalidConfiguration;
  }
  if (L.law != 0) return cudaErrorInvalidConfiguration;
  if (precision == 1) {
    if (L.variant == 2) {
#define NBODY_X(B, R, J)                                                \
  if (L.block == B && L.ipt == R && L.jtile == J) {                     \
    if (L.phi)                                                          \
      return launch_pdl(k_force_mixed2<0, B, R, J, true, 4>, L.n_ctas, B, st, L);   \
    else                                                                \
      return launch_pdl(k_force_mixed2<0, B, R, J, false, 4>, L.n_ctas, B, st, L);  \
  }
      NBODY_CAPPED_TILINGS(NBODY_X)
#undef NBODY_X
      return cudaErrorInvalidConfiguration;
    }
    if (L.variant != 0 && L.variant != 1) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                               \
  if (L.block == B && L.ipt == R && L.jtile == J) {                    \
    if (L.variant == 1 && L.phi)                                       \
      return launch_pdl(k_force_mixed2<0, B, R, J, true>, L.n_ctas, B, st, L);     \
    else if (L.variant == 1)                                           \
      return launch_pdl(k_force_mixed2<0, B, R, J, false>, L.n_ctas, B, st, L);    \
    else                                                               \
      return launch_pdl(k_force_mixed<B, R, J>, L.n_ctas, B, st, L);               \
  }
    NBODY_MIXED_TILINGS(NBODY_X)
#undef NBODY_X
    return cudaErrorInvalidConfiguration;
  }
  if (L.variant != 0) return cudaErrorInvalidConfiguration;
#define NBODY_X(B, R, J)                                               \
  if (L.block == B && L.ipt == R && L.jtile == J) {                    \
    return launch_pdl(k_force_fp64<0, B, R, J>, L.n_ctas, B, st, L);               \
  }
  NBODY_FORCE_TILINGS(NBODY_X)
#undef NBODY_X
  return cudaErrorInvalidConfiguration;
}

int force_ctas_per_sm(int precision, int variant, int block, int ipt, int jtile, int law) {
  if (law == 1) {
    if (precision == 1 && variant == 2) {
#define NBODY_X(B, R, J)                                                                                     \
  if (block == B && ipt == R && jtile == J)                                                                  \
    return std::min(occupancy_of(k_force_mixed2<1, B, R, J, true, 6>, B), occupancy_of(k_force_mixed2<1, B, R, J, false, 6>, B));
      NBODY_LJ_CAPPED_TILINGS(NBODY_X)
#undef NBODY_X
      return 0;
    }
    if (precision == 1) {
      if (variant != 1) return 0;
#define NBODY_X(B, R, J) \
  if (block == B && ipt == R && jtile == J)                                                          \
    return std::min(occupancy_of(k_force_mixed2<1, B, R, J, true>, B), occupancy_of(k_force_mixed2<1, B, R, J, false>, B));
      NBODY_LJ_MIXED_TILINGS(NBODY_X)
#undef NBODY_X
      return 0;
    }
    if (variant != 0) return 0;
#define NBODY_X(B, R, J) \
  if (block == B && ipt == R && jtile == J) return occupancy_of(k_force_fp64<1, B, R, J>, B);
    NBODY_LJ_FP64_TILINGS(NBODY_X)
#undef NBODY_X
    return 0;
  }
  if (law != 0) return 0;
  if (precision == 1 && variant == 2) {
#define NBODY_X(B, R, J)                                                                                    \
  if (block == B && ipt == R && jtile == J)                                                                 \
    return std::min(occupancy_of(k_force_mixed2<0, B, R, J, true, 4>, B), occupancy_of(k_force_mixed2<0, B, R, J, false, 4>, B));
    NBODY_CAPPED_TILINGS(NBODY_X)
#undef NBODY_X
    return 0;
  }
  if (precision == 1) {
    if (variant != 0 && variant != 1) return 0;
#define NBODY_X(B, R, J)                                                                             \
  if (block == B && ipt == R && jtile == J)                                                          \
    return variant == 1 ? std::min(occupancy_of(k_force_mixed2<0, B, R, J, true>, B),                  \
                                   occupancy_of(k_force_mixed2<0, B, R, J, false>, B))                 \
                        : occupancy_of(k_force_mixed<B, R, J>, B);
    NBODY_MIXED_TILINGS(NBODY_X)
#undef NBODY_X
    return 0;
  }
  if (variant != 0) return 0;
#define NBODY_X(B, R, J) \
  if (block == B && ipt == R && jtile == J) return occupancy_of(k_force_fp64<0, B, R, J>, B);
  NBODY_FORCE_TILINGS(NBODY_X)
#undef NBODY_X
  return 0;
}

}  // namespace nbody
