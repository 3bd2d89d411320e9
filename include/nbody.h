/*
 * nbody.h -- C ABI of the GB300 (sm_103a) softened-gravity N-body hot path.
 *
 * The operations follow the N-body miniapp of "Implementing Multi-GPU
 * Scientific Computing Miniapps Across Performance Portable Frameworks"
 * (arXiv 2511.02655): an all-pairs force evaluation over every pair of
 * particles (Sec. V-B, "N_p^2 operations"), Verlet half-step time integration
 * (Sec. II-A) and a total-energy reduction fused with the force calculation
 * (Sec. VI). Two pair laws:
 *
 *   softened gravity (default):
 *     d_ij = x_j - x_i,   s_ij = sqrt(|d_ij|^2 + eps^2)
 *     a_i   =  G sum_{j != i} m_j d_ij / s_ij^3
 *     phi_i = -G sum_{j != i} m_j / s_ij
 *   Lennard-Jones, the paper's Eq. 1 (law = NBODY_LAW_LJ), with u = sigma^2 / s_ij^2:
 *     a_i   =  (24 epsilon / m_i) sum_{j != i} (u^3 - 2 u^6) d_ij / s_ij^2   (= F_i / m_i)
 *     phi_i =  ( 4 epsilon / m_i) sum_{j != i} (u^6 - u^3)                   (= sum_j V(r_ij) / m_i)
 * so that U = 1/2 sum m_i phi_i in both cases. No cutoff: every pair counts.
 *
 * Conventions shared by every call:
 *   - All array arguments are DEVICE pointers (CUDA global memory of the
 *     context's device), caller-owned, C-contiguous float64, 8-byte aligned:
 *     positions/velocities/accelerations are [N, 3] row-major (x0 y0 z0 x1 ...),
 *     masses and potentials [N]. N is the total body count of all systems.
 *     The *_host variants take host pointers instead (see there).
 *   - Several independent systems may share one context: system s owns rows
 *     offsets[s] .. offsets[s+1]-1; bodies of different systems never interact.
 *   - Every call is asynchronous on the context's stream and returns a status.
 *     Argument errors (NBODY_EINVAL) are detected on the host before anything
 *     is launched. Device-side conditions (non-finite results, a bounded wait
 *     that gave up) are latched in the context and reported by nbody_sync().
 *   - Results are deterministic: the same inputs on the same device and tuning
 *     give bit-identical outputs (no floating-point atomics).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbody_ctx nbody_ctx; /* opaque, library-owned */

typedef enum {
  NBODY_OK = 0,
  NBODY_EINVAL = 1,     /* invalid argument; nothing was launched */
  NBODY_ENOMEM = 2,     /* a device or host allocation failed */
  NBODY_ECUDA = 3,      /* a CUDA runtime call failed (text in nbody_last_error) */
  NBODY_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
  NBODY_ENONFINITE = 5, /* a non-finite acceleration or energy was produced */
  NBODY_EUNSUPPORTED = 6, /* no sm_103a device / operation not available */
  NBODY_EINTERNAL = 7     /* NBODY_DEBUG builds: a device-side index check failed (the access was skipped) */
} nbody_status;

typedef enum {
  NBODY_FP64 = 0, /* all pair arithmetic and sums in float64 (plain GPU path) */
  NBODY_MIXED = 1 /* float32 pair arithmetic; per-tile float32 partials folded into a
                     compensated float32 pair, then summed across slices in float64;
                     state and reductions float64 */
} nbody_precision;

typedef enum {
  NBODY_LAW_GRAVITY = 0, /* softened Newtonian gravity (G, eps) */
  NBODY_LAW_LJ = 1       /* Lennard-Jones, the paper's Eq. 1 (lj_epsilon, lj_sigma; eps softens r^2) */
} nbody_law;

/* Flags for nbody_config.flags */
#define NBODY_FLAG_GRAPH 1u   /* replay nbody_step as a captured CUDA graph (same pointers) */
#define NBODY_FLAG_NOCHECK 2u /* skip the non-finite scan in nbody_sync */

typedef struct {
  double G;             /* gravitational constant (finite) */
  double eps;           /* Plummer softening length, >= 0 (0: unsoftened, coincident bodies give inf) */
  double dt;            /* KDK time step; must be finite and > 0 for nbody_step / nbody_adjoint */
  int32_t precision;    /* nbody_precision */
  int32_t energy_every; /* nbody_step records energies after every k-th step (0 = never) */
  int32_t block;        /* force kernel: threads per CTA, 128 or 256 (0 = autotune) */
  int32_t i_per_thread; /* force kernel: i-bodies kept in registers per thread, 1, 2 or 4 (0 = autotune) */
  int32_t j_tile;       /* force kernel: j-bodies per shared-memory tile, 128 or 256 (512 too for
                           NBODY_MIXED) (0 = autotune) */
  int32_t slice;        /* force kernel: j-bodies per work item, multiple of j_tile (0 = autotune) */
  uint32_t flags;       /* NBODY_FLAG_* */
  int32_t variant;      /* mixed force and adjoint-VJP kernels: 1 = scalar float32, 2 = packed
                           float32x2, 3 = packed force kernel under a register cap (softened
                           gravity: 4 CTAs per SM, tiling 128 x 2 x 256; Lennard-Jones: 6 CTAs
                           per SM, tilings 128 x 1 x 256 and 128 x 1 x 512; the VJP then uses
                           2), 0 = autotune (each kernel separately); must be 0 or 1 for
                           NBODY_FP64; NBODY_LAW_LJ with NBODY_MIXED takes 0, 2 or 3 */
  int32_t law;          /* nbody_law */
  int32_t reserved;     /* must be 0 */
  double lj_epsilon;    /* Lennard-Jones well depth (finite; law = NBODY_LAW_LJ) */
  double lj_sigma;      /* Lennard-Jones length scale (> 0; law = NBODY_LAW_LJ) */
  double box;           /* > 0: reflecting walls of the cube [0, box]^3 applied after each drift
                           ("boundary checking"); 0: open space. Finite, >= 0. */
} nbody_config;

/*
 * Creates a context for n_systems independent systems with host array
 * offsets[n_systems + 1] (offsets[0] = 0, non-decreasing; empty systems allowed;
 * total N = offsets[n_systems] < 2^29). The context allocates its own
 * device scratch (staging tiles, per-slice partial sums, reduction partials,
 * work lists) on the current device and binds `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream). When any tile parameter is 0 the autotuner
 * times candidate tilings of the force kernel on synthetic positions of this
 * layout during init (this synchronises the device). The context keeps a copy
 * of *cfg. On failure *ctx is NULL.
 *
 * Environment: NBODY_TUNE_CACHE=<file> keeps the tuner's choices (force and
 * VJP) across runs, keyed by device, configuration and layout;
 * NBODY_TUNE_VERBOSE=1 prints the candidates' costs on stderr;
 * NBODY_FAULT_ALLOC=k makes the k-th scratch allocation of the context report
 * NBODY_ENOMEM (for testing failure paths); NBODY_NVTX=1 wraps the context's
 * API calls (and the adjoint's forward and reverse phases) in NVTX ranges.
 */
nbody_status nbody_init(nbody_ctx** ctx, const nbody_config* cfg, int64_t n_systems, const int64_t* offsets,
                        void* cuda_stream);

/* Rebinds the context's stream (a cudaStream_t; NULL = legacy default stream). */
nbody_status nbody_set_stream(nbody_ctx* ctx, void* cuda_stream);

/*
 * All-pairs force evaluation (Sec. V-B): a [N,3] = accelerations, phi [N] =
 * potentials (phi may be NULL). x [N,3], m [N] are read only. Self pairs are
 * excluded from both sums. In NBODY_MIXED, pairs closer than 4 eps (4 sigma for
 * Lennard-Jones) take their separation from the float32 staging copy plus its
 * staged float32 remainder, (hi_j - hi_i) + (lo_j - lo_i), so that the staging
 * rounding of |x - c| 2^-24 does not dominate close-pair forces.
 */
nbody_status nbody_forces(nbody_ctx* ctx, const double* x, const double* m, double* a, double* phi);

/*
 * n_steps kick-drift-kick leapfrog steps (Verlet half-stepping, Sec. II-A),
 * one force evaluation per step:
 *     v += dt/2 a(x);  x += dt v;  a = a(x);  v += dt/2 a
 * x, v [N,3] are updated in place; a [N,3] must hold a(x) on entry when
 * a_valid != 0 (else it is computed first) and holds a(x_final) on exit.
 * energy_log (device, nullable): if cfg.energy_every = k > 0, after every k-th
 * step the record [n_systems][9] = {E, K, U, Px, Py, Pz, Lx, Ly, Lz} is
 * written to energy_log + r * n_systems * 9 for record r = 0, 1, ...
 * (n_steps / k records). n_steps = 0 only computes a when a_valid == 0.
 */
nbody_status nbody_step(nbody_ctx* ctx, double* x, double* v, const double* m, double* a, int32_t a_valid,
                        int32_t n_steps, double* energy_log);

/*
 * Global reductions (Sec. VI) at the state (x, v): out [n_systems][9] (device)
 * = {E, K, U, Px, Py, Pz, Lx, Ly, Lz} with K = 1/2 sum m|v|^2,
 * U = 1/2 sum m phi (phi from a force evaluation in the context's precision),
 * E = K + U, P = sum m v, L = sum m x cross v. Sums run in float64 in a fixed order.
 */
nbody_status nbody_energy(nbody_ctx* ctx, const double* x, const double* v, const double* m, double* out);

/*
 * Virial diagnostics at the state (x, v): out [n_systems][3] (device) =
 * {K, W, Q} with K = 1/2 sum m|v|^2, the Clausius virial W = sum m x . a
 * (a from a force evaluation in the context's precision, either pair law; for
 * softened gravity W = -G sum_{i<j} m_i m_j r_ij^2 / s_ij^3, equal to U when
 * eps = 0) and the virial ratio Q = -2K/W (0 if W = 0; Q = 1 in virial
 * equilibrium). Sums run in float64 in a fixed order.
 */
nbody_status nbody_virial(nbody_ctx* ctx, const double* x, const double* v, const double* m, double* out);

/*
 * Reverse-mode gradient through n_steps KDK steps from (x0, v0) with masses m:
 * given lam_xT = dL/dx_T and lam_vT = dL/dv_T [N,3] (device), writes
 * g_x0 = dL/dx0, g_v0 = dL/dv0 [N,3] and g_m = dL/dm [N]. The forward
 * trajectory is recomputed from checkpoints of (x, v, a) taken every
 * checkpoint_every steps (1 <= checkpoint_every; device memory about
 * (72 * ceil(n_steps / checkpoint_every) + 24 * (checkpoint_every + 1)) * N
 * bytes, allocated by the context on first use and kept). Each reverse step applies the
 * vector-Jacobian product of a(x, m),
 *     g_x,k = G sum_{j != k} J(d_kj) (m_k w_j - m_j w_k),  J(d) = I/s^3 - 3 d d^T / s^5
 *     g_m,j = G sum_{i != j} w_i . d_ij / s_ij^3
 * in the context's precision. x0/v0/m are not modified. Softened gravity
 * without walls only (NBODY_EUNSUPPORTED otherwise).
 */
nbody_status nbody_adjoint(nbody_ctx* ctx, const double* x0, const double* v0, const double* m, int32_t n_steps,
                           int32_t checkpoint_every, const double* lam_xT, const double* lam_vT, double* g_x0,
                           double* g_v0, double* g_m);

/*
 * nbody_adjoint plus the gradients with respect to the two model parameters of
 * softened gravity, per system: g_params [n_systems][2] (device, overwritten)
 * = {dL/dG, dL/deps}. The acceleration depends on G linearly and on eps through
 * s^2 = |d|^2 + eps^2, so every half-kick with weight w (= coef * lam_v) adds
 *     dL/dG   += sum_k w_k . sum_{j != k} m_j d_kj / s_kj^3
 *     dL/deps += sum_k w_k . (-3 G eps) sum_{j != k} m_j d_kj / s_kj^5
 * (summed per system in a fixed order). G and eps are shared by all systems of
 * the context, so the gradient of a loss summed over systems is the sum of the
 * rows. Costs two more float32 (or float64) operations per pair of each VJP
 * and 32 bytes more partial memory per body and slice. Same arguments, errors
 * and restrictions as nbody_adjoint; g_params NULL is NBODY_EINVAL.
 */
nbody_status nbody_adjoint_params(nbody_ctx* ctx, const double* x0, const double* v0, const double* m,
                                  int32_t n_steps, int32_t checkpoint_every, const double* lam_xT,
                                  const double* lam_vT, double* g_x0, double* g_v0, double* g_m, double* g_params);

/*
 * Host-memory variant of nbody_step: x, v, a (in/out), m (in) and energy_log
 * (out, nullable) are HOST pointers. The context copies them to its own device
 * buffers, runs nbody_step, copies x, v, a and the energy records back, and
 * synchronises the stream before returning. When every buffer is mapped
 * page-locked memory (cudaHostAlloc / cudaHostRegister, e.g. torch pinned
 * tensors) one copy kernel moves the inputs and one the results across the
 * host link; otherwise cudaMemcpyAsync is used.
 */
nbody_status nbody_step_host(nbody_ctx* ctx, double* x, double* v, const double* m, double* a, int32_t a_valid,
                             int32_t n_steps, double* energy_log);

/*
 * Waits for all work queued on the context's stream, then reports latched
 * device-side conditions: NBODY_ENONFINITE if the last force evaluation
 * produced a non-finite acceleration (unless NBODY_FLAG_NOCHECK),
 * NBODY_ETIMEOUT if a bounded wait gave up, NBODY_ECUDA on a CUDA error.
 * Clears the latched flags.
 */
nbody_status nbody_sync(nbody_ctx* ctx);

/*
 * Tiling in use (after init / autotune): block, i_per_thread, j_tile, slice,
 * the number of persistent CTAs the force kernel launches, and the force
 * kernel variant (as in nbody_config.variant: 1 scalar, 2 packed, 3 packed capped). Any pointer
 * may be NULL.
 */
nbody_status nbody_get_tuning(const nbody_ctx* ctx, int32_t* block, int32_t* i_per_thread, int32_t* j_tile,
                              int32_t* slice, int32_t* n_ctas, int32_t* variant);

/*
 * Work-list shape of the force pass (after init / autotune): tail = 0 when
 * each system's j-range is cut into equal slices, 1 when it ends in a tail of
 * halving slices; the number of work items and the largest slice count of any
 * system. Any pointer may be NULL.
 */
nbody_status nbody_get_slicing(const nbody_ctx* ctx, int32_t* tail, int32_t* n_items, int32_t* max_slices);

/*
 * Kernel timing. nbody_profile(ctx, 1) clears the counters and makes the
 * context record a CUDA event pair on its stream around every launch of the
 * all-pairs kernels (eagerly issued calls only; graph replays are not timed);
 * nbody_profile(ctx, 0) stops recording. nbody_kernel_time synchronises the
 * stream and returns, for which = 0 (force kernel) or 1 (force-VJP kernel),
 * the summed device milliseconds and the number of timed launches.
 */
nbody_status nbody_profile(nbody_ctx* ctx, int32_t enable);
nbody_status nbody_kernel_time(nbody_ctx* ctx, int32_t which, double* ms_total, int64_t* launches);

/*
 * Number of kernels the context launched since creation (counted on the host
 * at each launch or graph replay node); for launch accounting.
 */
int64_t nbody_launch_count(const nbody_ctx* ctx);

/*
 * Largest body count nbody_forces_noalloc accepts. Its scratch is a fixed
 * 32 MiB + 256 B __device__ array (32 bytes per body: the float32 staging
 * entry and the float32 remainders of the near-pair refinement), held on every
 * GPU that loads the library's device code, for the life of the process.
 */
#define NBODY_NOALLOC_MAX_BODIES 1048576

/*
 * Mixed-precision forces of ONE system without allocating anything: no
 * context, no cudaMalloc/cudaFree, no allocating library call. For callers
 * that cannot allocate device memory where they need forces (a fixed memory
 * budget owned by a host framework, a plugin handed only ready-made buffers,
 * code that must not hit the allocator or its implicit synchronisation).
 * The paper has no counterpart; this is a deployment convenience.
 *
 * x [n,3], m [n] (read), a [n,3] (written), phi [n] (written, nullable) are
 * float64 device pointers on the current device, each holding at least that
 * many elements (checked where the driver reports the allocation's extent);
 * the work is queued on cuda_stream (NULL = legacy default stream) and is
 * asynchronous. Same pair arithmetic as nbody_forces with NBODY_MIXED:
 * float32 pairs with the near-pair refinement (pairs closer than 4 eps
 * recomputed from the staged float32 remainders), compensated float32 tile
 * sums, float64 result; the same error bounds against the float64 direct sum
 * (median <= 1e-6, max <= 1e-4 relative per body). One CTA per i-tile and no
 * j-slices, so results agree with nbody_forces to rounding, not bit for bit.
 *
 * Scratch is a static __device__ array shared by every call in the process:
 * calls that overlap on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller. Each call overwrites
 * everything it reads, so no state carries over from an earlier call.
 *
 * The first call on a device is a warm-up: it looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, which makes the
 * CUDA runtime load the library's device code on that device if it has not
 * yet, and loading reserves the 32 MiB array and the kernels' code there (it
 * can fail with NBODY_ECUDA when the device is out of memory, and may
 * synchronise). Make that first call before the region that must not
 * allocate, and before any stream capture; later calls on that device
 * allocate nothing. The looked-up address belongs to the device's current
 * CUDA context: do not use the library across a cudaDeviceReset (which ends
 * that context and invalidates every nbody_ctx as well).
 *
 * Returns NBODY_EINVAL for n > NBODY_NOALLOC_MAX_BODIES, n < 0, bad or short
 * pointers or bad parameters (message in nbody_last_error(NULL)).
 */
nbody_status nbody_forces_noalloc(const double* x, const double* m, int64_t n, double G, double eps, double* a,
                                  double* phi, void* cuda_stream);

/* Last error text for ctx (or a process-wide message when ctx is NULL). Never NULL. */
const char* nbody_last_error(const nbody_ctx* ctx);

/* Frees the context and its device memory (after synchronising its stream). NULL is ignored. */
void nbody_destroy(nbody_ctx* ctx);

/* ABI version: (major << 16) | minor. */
int32_t nbody_version(void);

/*
 * Build options of the loaded library, as bits: 1 = NBODY_DEBUG, a build
 * whose kernels check every work item, chunk and per-system range they read
 * against the buffers it indexes (body rows, partial-sum slices, chunk and
 * system tables) before using it. A failed check skips the access and latches
 * a device status bit that the next nbody_sync reports as NBODY_EINTERNAL. It
 * stands in for a device memory checker; release builds return 0.
 */
int32_t nbody_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
