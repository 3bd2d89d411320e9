// Internal declarations shared by the CUDA translation units of libnbody.
// Nothing here is part of the C ABI (include/nbody.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nbody {

// One unit of all-pairs work: i-bodies [i_begin, i_end) of one system against
// its j-bodies [j_begin, j_end), partial sums written to slice `slice`.
// Indices are global body indices (rows of the caller's arrays).
struct WorkItem {
  int32_t sys;
  int32_t i_begin, i_end;
  int32_t j_begin, j_end;
  int32_t slice;
};

// A contiguous run of bodies of one system, the unit of the O(N) kernels and
// of the fixed-order energy reduction.
struct Chunk {
  int32_t sys;
  int32_t begin, end;
  int32_t n_slices;  // force/VJP slices of this system (partials to combine)
};

constexpr int kChunk = 256;         // bodies per chunk (one per thread of an O(N) CTA)
constexpr int kPostThreads = 256;   // threads per O(N) kernel CTA
constexpr int kEnergyVals = 8;      // K, U, Px, Py, Pz, Lx, Ly, Lz per chunk
constexpr int kAdjVals = 8;         // VJP partial values per body per slice

// Device status word bits (latched, read by nbody_sync).
constexpr unsigned kFlagNonFinite = 1u;
constexpr unsigned kFlagTimeout = 2u;

// ---------------------------------------------------------------------------
// all-pairs kernels (force_kernels.cu, adjoint_kernels.cu)

struct PairLaunch {
  const void* stage_x;   // float4 (x-c, m) [mixed] or double4_32a (x, m) [fp64], [N]
  const void* stage_w;   // VJP only: float4 / double4_32a (w, 0), [N]
  const WorkItem* items;
  int32_t n_items;
  unsigned* counter;     // [2]: next item, CTAs done (zero between launches)
  double* part;          // force: double4_32a [slices][N]; VJP: (2 or 3 with params) x double4_32a [slices][N]
  int64_t n_total;
  double eps2;
  const float4* stage_lo;  // force (mixed): float32 remainders (x - c) - hi [N], near-pair refinement
  float r2_near;         // force (mixed): refine pairs with s^2 below this (0 = never)
  int variant;           // mixed kernels: 0 scalar float32, 1 packed float32x2
  int law;               // 0 softened gravity, 1 Lennard-Jones
  double sigma2;         // Lennard-Jones sigma^2
  int block, ipt, jtile; // tiling
  int n_ctas;            // persistent grid size
  int params;            // VJP: also the sums for the G and eps gradients (third double4)
  int phi;               // force (mixed packed): accumulate the potential (0: skip it, partial .w = 0)
};

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
  const double* part;      // double4_32a [slices][N]
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
  double box;              // > 0: reflecting walls of [0, box]^3 applied after the drift
  void* stage;             // float4 / double4_32a [N]
  void* stage_lo;          // mixed: float4 remainders of the staged coordinates [N] (nullable)
  const double* centre;    // [n_sys][3] staging origin (mixed)
  double* epart;           // [n_chunks][kEnergyVals]
  unsigned* status;        // device status word
  double* eout;            // kEnergy: nullable [n_sys][9] record formed by the last CTA
  double* vout;            // kVirial: [n_sys][3] record {K, W, -2K/W} formed by the last CTA
  const int32_t* sys_chunk;  // [n_sys + 1] chunk range of each system
  int n_sys;
  unsigned* done;          // last-CTA ticket (zero between launches)
};
cudaError_t launch_post(const PostLaunch& P, cudaStream_t st);

// centre[s] = mass-weighted mean position of system s (plain mean if the mass is 0):
// per-chunk sums into cpart [n_chunks][kEnergyVals], then per system in a fixed
// order by the last CTA (ticket `done`, zero between launches).
cudaError_t launch_centre(const Chunk* chunks, int n_chunks, const int32_t* sys_chunk, const int64_t* off, int n_sys,
                          const double* x, const double* m, double* cpart, double* centre, unsigned* done,
                          cudaStream_t st);

struct AdjLaunch {
  const Chunk* chunks;
  int32_t n_chunks;
  const double* part;      // 2 (3 with g_params) x double4_32a [slices][N]
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
  const double* centre;
  unsigned* status;
  double* g_params;        // nullable [n_sys][2]: += coef (w.da/dG, w.da/deps), formed by the last CTA
  double eps;
  double* cpart;           // [n_chunks][kEnergyVals] chunk partials (g_params only)
  const int32_t* sys_chunk;
  int n_sys;
  unsigned* done;          // last-CTA ticket (zero between launches)
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

// stage w = lam (float4 / double4_32a) and/or x for a VJP without an update
cudaError_t launch_stage_vec(const Chunk* chunks, int n_chunks, int precision, const double* vec, const double* m,
                             const double* centre, void* stage, int as_position, cudaStream_t st);

}  // namespace nbody
