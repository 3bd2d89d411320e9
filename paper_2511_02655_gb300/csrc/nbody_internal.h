// Internal declarations shared by the CUDA translation units of libnbody.
// Nothing here is part of the C ABI (include/nbody.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nbody {

// One unit of all-pairs work: i-bodies [i_begin, i_end) of one system against
// its j-bodies [j_begin, j_end), partial sums written to slice `slice` of the
// system's n_slices. Indices are global body indices (rows of the caller's
// arrays).
struct WorkItem {
  int32_t sys;
  int32_t i_begin, i_end;
  int32_t j_begin, j_end;
  int32_t slice;
  int32_t n_slices;
};

// A contiguous run of bodies of one system, the unit of the O(N) kernels and
// of the fixed-order energy reduction.
struct Chunk {
  int32_t sys;
  int32_t begin, end;
  int32_t n_slices;  // force/VJP slices of this system (partials to combine)
};

// The O(N) kernels do their float64 work on GB300's FP64 pipe (about 1/75 of
// the FP32 rate), so their time is the float64 operations per SM: chunks of 128
// bodies spread even small systems (10 000 bodies: 79 CTAs) over many SMs.
constexpr int kChunk = 128;         // bodies per chunk (one per thread of an O(N) CTA)
constexpr int kPostThreads = 128;   // threads per O(N) kernel CTA
constexpr int kEnergyVals = 8;      // K, U, Px, Py, Pz, Lx, Ly, Lz per chunk
constexpr int kAdjVals = 8;         // VJP partial values per body per slice

// Force partial of one body and slice on the mixed path: the four compensated
// float32 sums (hi, lo) of the force kernels (sum m d / s^3 per axis and
// sum m / s), stored as they are: (hx, lx, hy, ly), (hz, lz, hp, lp). The
// O(N) kernel adds the slices as float32 pairs (TwoSum) and converts the total
// once, instead of converting each slice and adding on the FP64 pipe.
struct __align__(32) fpair4 {
  float4 xy;
  float4 zp;
};

// Knuth's TwoSum: hi + lo absorbs t, with the rounding error of hi + t carried
// into lo (Knuth, TAOCP vol. 2, 4.2.2). Six float32 additions, no branches.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float t) {
  const float s = hi + t;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (t - bp);
  hi = s;
  lo += err;
}

// Programmatic dependent launch (sm_90 and later) between the kernels of a
// step: a kernel launched with launch_pdl may be scheduled while the kernel
// before it on the stream is still finishing; pdl_wait(), its first
// statement, waits (in hardware) until that grid has completed and its memory
// is visible, so data dependences are exactly those of plain stream order and
// only the launch latency overlaps. pdl_trigger() lets the next such kernel be
// scheduled once every CTA of this one has passed it. Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Device status word bits (latched, read by nbody_sync).
constexpr unsigned kFlagNonFinite = 1u;
constexpr unsigned kFlagTimeout = 2u;
constexpr unsigned kFlagIndex = 4u;  // NBODY_DEBUG builds: an index check failed, the access was skipped

// Index checks of NBODY_DEBUG builds: nb_debug_ok(cond, status) is true when
// cond holds; otherwise it latches kFlagIndex in *status and returns false, and
// the caller skips the access. Release builds compile it to `true`.
#ifdef NBODY_DEBUG
__device__ __forceinline__ bool nb_debug_ok(const bool cond, unsigned* status) {
  if (!cond && status) atomicOr(status, kFlagIndex);
  return cond;
}
#else
__device__ __forceinline__ constexpr bool nb_debug_ok(const bool, unsigned*) { return true; }
#endif

// Host-side argument check (capi.cu): false when the driver reports that the
// device allocation holding p ends before p + bytes (cuMemGetAddressRange);
// *avail then holds the bytes left from p. True when the driver does not
// expose the query or does not know p.
bool allocation_holds(const void* p, size_t bytes, size_t* avail);

// ---------------------------------------------------------------------------
// all-pairs kernels (force_kernels.cu, adjoint_kernels.cu)

struct PairLaunch {
  const void* stage_x;   // float4 (x-c, m) [mixed] or double4_32a (x, m) [fp64], [N]
  const void* stage_w;   // VJP only: float4 / double4_32a (w, 0), [N]
  const WorkItem* items;
  int32_t n_items;
  unsigned* counter;     // [2]: next item, CTAs done (zero between launches)
  double* part;          // [slices][N] x (force: 1, VJP: 2, or 3 with params) of fpair4 (mixed) or double4_32a (FP64)
  int64_t n_total;
  double eps2;
  const float4* stage_lo;  // mixed: float32 remainders (x - c) - hi [N], near-pair refinement
  float r2_near;         // mixed: refine pairs with s^2 below this (0 = never)
  int variant;           // mixed kernels: 0 scalar float32, 1 packed float32x2
  int law;               // 0 softened gravity, 1 Lennard-Jones
  double sigma2;         // Lennard-Jones sigma^2
  int block, ipt, jtile; // tiling
  int n_ctas;            // persistent grid size
  int params;            // VJP: also the sums for the G and eps gradients (third double4)
  int phi;               // force (mixed packed): accumulate the potential (0: skip it, partial .w = 0)
  int32_t part_slices;   // slices the partial buffer holds (index checks of NBODY_DEBUG builds)
  int32_t block_bodies;  // debug checks: i-bodies a work item may hold (block x ipt)
  unsigned* status;      // device status word (index checks of NBODY_DEBUG builds)
};

#ifdef NBODY_DEBUG
// NBODY_DEBUG check of a work item against the buffers it indexes: its body
// ranges inside the rows, its i-range inside one CTA's tile, its slice inside
// the partial-sum buffer. The kernel skips an item that fails.
__device__ __forceinline__ bool item_ok(const WorkItem& w, const PairLaunch& L) {
  return nb_debug_ok(w.i_begin >= 0 && w.i_begin < w.i_end && w.i_end <= L.n_total && w.j_begin >= 0 &&
                         w.j_begin < w.j_end && w.j_end <= L.n_total && w.i_end - w.i_begin <= L.block_bodies &&
                         w.slice >= 0 && w.slice < w.n_slices && w.n_slices <= L.part_slices,
                     L.status);
}

// NBODY_DEBUG check of a chunk of an O(N) kernel: rows, system index and (when
// part_slices > 0) its slice count against the partial-sum buffer. A chunk that
// fails is processed as an empty one.
__device__ __forceinline__ bool chunk_ok(const Chunk& c, const int64_t n_total, const int n_sys, const int part_slices,
                                         unsigned* status) {
  return nb_debug_ok(c.begin >= 0 && c.begin < c.end && c.end <= n_total && c.end - c.begin <= kChunk && c.sys >= 0 &&
                         c.sys < n_sys && (part_slices <= 0 || (c.n_slices >= 1 && c.n_slices <= part_slices)),
                     status);
}
#else
__device__ __forceinline__ constexpr bool item_ok(const WorkItem&, const PairLaunch&) { return true; }
__device__ __forceinline__ constexpr bool chunk_ok(const Chunk&, int64_t, int, int, unsigned*) { return true; }
#endif

// Returns cudaErrorInvalidConfiguration for an unsupported tiling.
cudaError_t launch_force(int precision, const PairLaunch& L, cudaStream_t st);
cudaError_t launch_vjp(int precision, const PairLaunch& L, cudaStream_t st);
// CTAs of the force kernel that fit on one SM for the tiling (0 if unsupported).
int force_ctas_per_sm(int precision, int variant, int block, int ipt, int jtile, int law);
int vjp_ctas_per_sm(int precision, int variant, int block, int ipt, int jtile);

// ---------------------------------------------------------------------------
// O(N) kernels (post_kernels.cu)

enum PostMode : unsigned {
  kCombine = 1u,   // a, phi <- G * sum over slices of the partials
  kKickEnd = 2u,   // v += dt/2 a           (closing half-kick of a step)
  kEnergy = 4u,    // per-chunk partial energies / momenta at (x, v)
  kDrift = 8u,     // v += dt/2 a; x += dt v (opening half-kick + drift of the next step)
  kStage = 16u,    // staging tile entry from x (after the drift, if any)
  kVirial = 32u,   // per-chunk partial K and Clausius virial W = sum m x.a (not with kEnergy)
};

struct PostLaunch {
  const Chunk* chunks;
  int32_t n_chunks;
  const double* part;      // [slices][N] of fpair4 (mixed) or double4_32a (FP64)
  int64_t n_total;
  double G, half_dt, dt;
  double* x;
  double* v;
  const double* m;
  double* a;
  double* phi;             // nullable
  double* x_copy;          // nullable: copy of x after the drift
  unsigned mode;
  int precision;
  int law;                 // 0 gravity: a = G S, phi = -G S_phi; 1 Lennard-Jones: a = 24 eps S / m, phi = 4 eps S_phi / m
  double lj_eps;
  double stage_scale;      // mixed: staged positions are (x - c) * stage_scale (1 / sigma for Lennard-Jones)
  double box;              // > 0: reflecting walls of [0, box]^3 applied after the drift
  void* stage;             // float4 / double4_32a [N]
  void* stage_lo;          // mixed: float4 remainders of the staged coordinates [N] (nullable)
  const double* centre;    // [n_sys][3] staging origin (mixed)
  double* epart;           // [n_chunks][kEnergyVals]
  unsigned* status;        // device status word
  double* eout;            // kEnergy: nullable [n_sys][9] record formed by the last CTA (null: partials only)
  const double* eprev;     // nullable: chunk partials [n_chunks][kEnergyVals] of the previous step's record,
  double* eprev_out;       //   finished into eprev_out [n_sys][9] by one extra CTA (blockIdx.x == n_chunks)
  double* vout;            // kVirial: [n_sys][3] record {K, W, -2K/W} formed by the last CTA
  const int32_t* sys_chunk;  // [n_sys + 1] chunk range of each system
  int n_sys;
  unsigned* done;          // last-CTA ticket (zero between launches)
  int32_t part_slices;     // slices the partial buffer holds (index checks of NBODY_DEBUG builds)
};
cudaError_t launch_post(const PostLaunch& P, cudaStream_t st);

// centre[s] = mass-weighted mean position of system s (plain mean if the mass is 0):
// per-chunk sums into cpart [n_chunks][kEnergyVals], then per system in a fixed
// order by the last CTA (ticket `done`, zero between launches).
cudaError_t launch_centre(const Chunk* chunks, int n_chunks, const int32_t* sys_chunk, const int64_t* off, int n_sys,
                          const double* x, const double* m, double* cpart, double* centre, unsigned* done,
                          int64_t n_total, unsigned* status, cudaStream_t st);

struct AdjLaunch {
  const Chunk* chunks;
  int32_t n_chunks;
  const double* part;      // 2 (3 with g_params) x fpair4 (mixed) or double4_32a (FP64) [slices][N]
  int64_t n_total;
  double G, coef, dt;      // lam_x += coef * gx ; g_m += coef * gm ; lam_v += dt lam_x
  const double* m;
  double* lam_x;
  double* lam_v;
  double* g_m;
  int drift_rev;           // apply lam_v += dt lam_x and restage w = lam_v
  const double* x_next;    // nullable: positions to stage for the next VJP
  int precision;
  void* stage_x;
  void* stage_w;
  void* stage_lo;          // mixed: float4 remainders of the staged positions (nullable)
  const double* centre;
  unsigned* status;
  double* g_params;        // nullable [n_sys][2]: += coef (w.da/dG, w.da/deps), formed by the last CTA
  double eps;
  double* cpart;           // [n_chunks][kEnergyVals] chunk partials (g_params only)
  const int32_t* sys_chunk;
  int n_sys;
  unsigned* done;          // last-CTA ticket (zero between launches)
  int32_t part_slices;     // slices the partial buffer holds (index checks of NBODY_DEBUG builds)
};
cudaError_t launch_adj_update(const AdjLaunch& A, cudaStream_t st);

// dst[k][0 .. n[k]) = src[k][...] for k = 0..3 in one launch (entries with a
// null pointer or n = 0 are skipped); grid at most 8 CTAs per SM.
struct Copy4 {
  const double* src[4];
  double* dst[4];
  int64_t n[4];
};
cudaError_t launch_copy4(const Copy4& C, int n_sms, cudaStream_t st);

// stage w = lam (float4 / double4_32a) or positions x (as_position; with their
// float32 remainders into stage_lo when given) for a VJP without an update
cudaError_t launch_stage_vec(const Chunk* chunks, int n_chunks, int precision, const double* vec, const double* m,
                             const double* centre, void* stage, void* stage_lo, int as_position, int64_t n_total,
                             int n_sys, unsigned* status, cudaStream_t st);

}  // namespace nbody
