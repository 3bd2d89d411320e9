// C ABI of libnbody (include/nbody.h): context, argument validation, work
// lists, autotuner (with its optional cache), the KDK step sequence (with
// optional CUDA-graph replay), the host-buffer step, the energy and virial
// reductions and the checkpointed adjoint driver.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nbody.h"
#include "nbody_internal.h"

using namespace nbody;

namespace {

constexpr int64_t kMaxBodies = int64_t(1) << 29;      // 3 * N fits in int32 index arithmetic
constexpr size_t kMaxPartialBytes = size_t(1) << 30;  // cap on per-slice partial-sum memory
constexpr int kMinTilesPerSlice = 1;  // shortest slice in j-tiles (small systems need many items)
constexpr double kTuneLargePairs = 4.0e10;  // above this many pairs per force pass, tune on short slices
constexpr int kTuneSlice = 8192;
constexpr int kSliceQuantum = 4;  // slice lengths are multiples of this many bodies
constexpr int64_t kTailMin = 64;   // shortest slice of a halving tail

struct Tiling {
  int block = 0, ipt = 0, jtile = 0, slice = 0, n_ctas = 0;
  int variant = 0;  // mixed kernels: 0 scalar, 1 packed float32x2, 2 packed with a 4-CTA register cap (force)
  int tail = 0;     // slicing of a system's j-range: 0 equal slices, 1 full slices and a halving tail
};

// Near-pair refinement radius of the mixed force kernels: 4 softening lengths
// for gravity, 4 sigma for Lennard-Jones (the neighbour shells that carry its
// force in a dilute gas).
constexpr double kNearRadiusEps = 4.0;
constexpr double kNearRadiusSigma = 4.0;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// NVTX range for profilers (nsys, ncu --nvtx), pushed only when the context asks for it.
struct NvtxRange {
  bool on;
  NvtxRange(bool enable, const char* name) : on(enable) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
};

std::mutex g_err_mu;
std::string g_err = "no error";

void set_global_error(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = s;
}

PFN_cuMemGetAddressRange_v3020 g_addr_range = nullptr;
std::once_flag g_addr_once;

void load_addr_range() {
  std::call_once(g_addr_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_addr_range = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(fn);
  });
}

}  // namespace

namespace nbody {
// Error text reported by nbody_last_error(NULL), for entry points without a context.
void set_global_error_text(const char* msg) { set_global_error(msg); }

bool allocation_holds(const void* p, size_t bytes, size_t* avail) {
  load_addr_range();
  if (!g_addr_range) return true;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (g_addr_range(&base, &size, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS) return true;
  const uintptr_t end = static_cast<uintptr_t>(base) + size, at = reinterpret_cast<uintptr_t>(p);
  if (avail) *avail = end > at ? static_cast<size_t>(end - at) : 0;
  return at + bytes <= end;
}
}  // namespace nbody

struct nbody_ctx {
  nbody_config cfg{};
  // mixed Lennard-Jones: positions are staged in units of sigma, (x - c) / sigma,
  // so that u = sigma^2 / r^2 is the reciprocal itself; 1 everywhere else
  double stage_scale = 1.0;
  int device = 0;
  int sm_count = 0;
  std::string dev_name;  // cudaDeviceProp::name, part of the tuning-cache key
  int dev_cc = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  int64_t n_total = 0;
  int n_sys = 0;
  std::vector<int64_t> offsets;
  std::string err = "no error";
  int64_t launches = 0;

  // layout
  std::vector<Chunk> chunks;  // force tiling's slices
  std::vector<int32_t> sys_chunk;
  Chunk* d_chunks = nullptr;
  Chunk* d_vchunks = nullptr;  // same chunks, VJP tiling's slice counts
  int32_t* d_sys_chunk = nullptr;
  int64_t* d_off = nullptr;

  // force work list
  Tiling ft;
  WorkItem* d_items = nullptr;
  int n_items = 0;
  int max_slices = 1;
  // VJP work list (built on first adjoint)
  Tiling vt;
  WorkItem* d_vitems = nullptr;
  int n_vitems = 0;
  int vmax_slices = 1;
  bool vjp_ready = false;
  int64_t fault_alloc = 0;  // > 0: the fault_alloc-th scratch allocation fails (NBODY_FAULT_ALLOC, tests)
  bool nvtx = false;        // NBODY_NVTX=1: NVTX ranges around the API calls and the adjoint's phases
  bool vjp_params = false;  // VJP launches also form the G and eps gradient sums

  // scratch
  DevBuf stage, stage_lo, stage_w, part, centre, epart, status_counter, a_scratch;
  unsigned* counter = nullptr;  // [2]
  unsigned* status = nullptr;   // [1]

  // adjoint scratch
  DevBuf xw, vw, aw, ckpt, traj;

  // host-memory entry point scratch
  DevBuf hx, hv, hm, ha, hlog;
  unsigned* h_status = nullptr;  // pinned host word the status is copied into by nbody_sync

  // kernel timing (nbody_profile)
  bool profiling = false;
  bool capturing = false;  // enqueueing into a graph capture (no timing events then)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;  // (which, (start, end))

  // graph cache for nbody_step
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int32_t gkey_valid = -1, gkey_steps = -1;
  int64_t glaunches = 0;
};

namespace {

nbody_status fail(nbody_ctx* c, nbody_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    set_global_error(buf);
  return s;
}

#define NB_CUDA(ctx, call)                                                                         \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail((ctx), NBODY_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                       \
  } while (0)

// Drops the cached nbody_step graph: it holds raw pointers into the
// context's buffers, so it must not outlive any reallocation.
void invalidate_graph(nbody_ctx* c) {
  if (c->gexec) {
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
}

nbody_status ensure(nbody_ctx* c, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return NBODY_OK;
  invalidate_graph(c);
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  if (c->fault_alloc > 0 && --c->fault_alloc == 0)
    return fail(c, NBODY_ENOMEM, "injected allocation failure (NBODY_FAULT_ALLOC) for %zu bytes", bytes);
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(c, NBODY_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return NBODY_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool finite(double v) { return std::isfinite(v); }

// Checks that [p, p + bytes) is device-accessible memory of the context's device
// and lies inside one allocation. Catches host pointers and gross overruns
// before a kernel could fault on them.
nbody_status check_dev(nbody_ctx* c, const void* p, size_t bytes, const char* name, bool nullable = false) {
  if (bytes == 0) return NBODY_OK;
  if (!p) {
    if (nullable) return NBODY_OK;
    return fail(c, NBODY_EINVAL, "%s is NULL", name);
  }
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0) return fail(c, NBODY_EINVAL, "%s is not 8-byte aligned", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, NBODY_EINVAL, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(c, NBODY_EINVAL, "%s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != c->device)
    return fail(c, NBODY_EINVAL, "%s lives on device %d, context on device %d", name, at.device, c->device);
  size_t avail = 0;
  if (!allocation_holds(p, bytes, &avail))
    return fail(c, NBODY_EINVAL, "%s: %zu bytes needed, allocation holds %zu from that address", name, bytes, avail);
  return NBODY_OK;
}

// ---------------------------------------------------------------------------
// work lists

int ctas_per_sm(int prec, const Tiling& t, bool vjp, int law) {
  return vjp ? vjp_ctas_per_sm(prec, t.variant, t.block, t.ipt, t.jtile)
             : force_ctas_per_sm(prec, t.variant, t.block, t.ipt, t.jtile, law);
}

// Slice length for tiling t: the largest power-of-two multiple of jtile that
// still yields >= 4 items per persistent CTA (fewer, larger partial buffers),
// within the partial-memory cap.
int auto_slice(const nbody_ctx* c, const Tiling& t, int n_ctas) {
  int64_t nmax = 1;
  for (int s = 0; s < c->n_sys; ++s) nmax = std::max<int64_t>(nmax, c->offsets[s + 1] - c->offsets[s]);
  const int64_t itile = (int64_t)t.block * t.ipt;
  const int64_t lmin = (int64_t)t.jtile * kMinTilesPerSlice;
  int64_t best = lmin;
  for (int64_t L = lmin; L < 2 * nmax + lmin; L *= 2) {
    int64_t items = 0, max_sl = 1;
    for (int s = 0; s < c->n_sys; ++s) {
      const int64_t n = c->offsets[s + 1] - c->offsets[s];
      if (n <= 0) continue;
      const int64_t sl = (n + L - 1) / L;
      items += ((n + itile - 1) / itile) * sl;
      max_sl = std::max(max_sl, sl);
    }
    if ((size_t)max_sl * (size_t)c->n_total * 32 > kMaxPartialBytes) continue;
    if (items >= 4 * (int64_t)n_ctas) best = L;
  }
  return (int)std::min<int64_t>(best, INT32_MAX / 2);
}

// Work items of tiling t with slice length L (the count build_items produces).
// Slice lengths of a system of n bodies for slice length L. tail 0: equal
// slices, each a multiple of kSliceQuantum bodies. tail 1: full slices of L
// while more than 2 L bodies remain, then a tail of halving slices (half of
// what remains each, down to kTailMin bodies): the work list, sorted longest
// first, then ends in ever shorter items, so the CTAs of the persistent grid
// run out of work at nearly the same time instead of one long item apart.
void slice_lengths(int64_t n, int64_t L, int tail, std::vector<int64_t>& lens) {
  lens.clear();
  auto up = [](int64_t v) { return ((v + kSliceQuantum - 1) / kSliceQuantum) * kSliceQuantum; };
  if (!tail || n <= 2 * L) {
    int64_t ns = (n + L - 1) / L;
    const int64_t len = up((n + ns - 1) / ns);
    ns = (n + len - 1) / len;
    for (int64_t k = 0; k < ns; ++k) lens.push_back(std::min(len, n - k * len));
    return;
  }
  int64_t pos = 0;
  while (n - pos > 2 * L) lens.push_back(L), pos += L;
  while (pos < n) {
    const int64_t r = n - pos;
    const int64_t len = r <= 2 * kTailMin ? r : std::min<int64_t>(L, up(r / 2));
    lens.push_back(len);
    pos += len;
  }
}

int64_t count_items(const nbody_ctx* c, const Tiling& t, int64_t L) {
  const int64_t itile = (int64_t)t.block * t.ipt;
  int64_t items = 0;
  std::vector<int64_t> lens;
  for (int s = 0; s < c->n_sys; ++s) {
    const int64_t n = c->offsets[s + 1] - c->offsets[s];
    if (n <= 0) continue;
    slice_lengths(n, L, t.tail, lens);
    items += ((n + itile - 1) / itile) * (int64_t)lens.size();
  }
  return items;
}

void build_items(const nbody_ctx* c, const Tiling& t, std::vector<WorkItem>& items, std::vector<int>& sys_slices,
                 int& max_slices) {
  items.clear();
  sys_slices.assign(c->n_sys, 1);
  max_slices = 1;
  const int64_t itile = (int64_t)t.block * t.ipt;
  std::vector<int64_t> lens;
  for (int s = 0; s < c->n_sys; ++s) {
    const int64_t b = c->offsets[s], n = c->offsets[s + 1] - b;
    if (n <= 0) continue;
    // slice lengths a multiple of four (whole quads of the packed kernels' tiles;
    // a slice's last j-tile may be partial), equal or with a halving tail
    slice_lengths(n, t.slice, t.tail, lens);
    const int64_t ns = (int64_t)lens.size();
    sys_slices[s] = (int)ns;
    max_slices = std::max(max_slices, (int)ns);
    for (int64_t i0 = 0; i0 < n; i0 += itile) {
      int64_t j0 = 0;
      for (int64_t k = 0; k < ns; j0 += lens[k], ++k) {
        WorkItem w;
        w.sys = s;
        w.i_begin = (int32_t)(b + i0);
        w.i_end = (int32_t)(b + std::min(n, i0 + itile));
        w.j_begin = (int32_t)(b + j0);
        w.j_end = (int32_t)(b + j0 + lens[k]);
        w.slice = (int32_t)k;
        w.n_slices = (int32_t)ns;
        items.push_back(w);
      }
    }
  }
  // longest-processing-time-first order for the dynamic persistent schedule
  std::stable_sort(items.begin(), items.end(), [](const WorkItem& a, const WorkItem& b) {
    const int64_t ca = (int64_t)(a.i_end - a.i_begin) * (a.j_end - a.j_begin);
    const int64_t cb = (int64_t)(b.i_end - b.i_begin) * (b.j_end - b.j_begin);
    return ca > cb;
  });
}

nbody_status upload_items(nbody_ctx* c, const std::vector<WorkItem>& items, WorkItem** dst) {
  invalidate_graph(c);
  if (*dst) {
    cudaStreamSynchronize(c->stream);
    cudaFree(*dst);
    *dst = nullptr;
  }
  const size_t bytes = std::max<size_t>(1, items.size()) * sizeof(WorkItem);
  if (cudaMalloc(dst, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, NBODY_ENOMEM, "cudaMalloc of the work list failed");
  }
  if (!items.empty()) NB_CUDA(c, cudaMemcpy(*dst, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  // a pageable-memory cudaMemcpy may return before its DMA lands; the context
  // stream can be non-blocking, so wait for the device before any launch
  NB_CUDA(c, cudaDeviceSynchronize());
  return NBODY_OK;
}

nbody_status upload_chunks(nbody_ctx* c, const std::vector<int>& sys_slices, Chunk** dst) {
  std::vector<Chunk> ch = c->chunks;
  for (auto& k : ch) k.n_slices = sys_slices[k.sys];
  if (!*dst) {
    if (cudaMalloc(dst, std::max<size_t>(1, ch.size()) * sizeof(Chunk)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, NBODY_ENOMEM, "cudaMalloc of the chunk list failed");
    }
  }
  if (!ch.empty()) NB_CUDA(c, cudaMemcpy(*dst, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
  NB_CUDA(c, cudaDeviceSynchronize());
  return NBODY_OK;
}

// Installs tiling t for the force (vjp=false) or VJP (vjp=true) pass.
nbody_status install_tiling(nbody_ctx* c, Tiling t, bool vjp) {
  const int prec = c->cfg.precision;
  const int occ = ctas_per_sm(prec, t, vjp, c->cfg.law);
  if (occ <= 0)
    return fail(c, NBODY_EINVAL, "unsupported tiling block=%d ipt=%d jtile=%d variant=%d", t.block, t.ipt, t.jtile,
                t.variant);
  if (t.slice <= 0) t.slice = auto_slice(c, t, occ * c->sm_count);
  t.slice = std::max(kSliceQuantum, (t.slice / kSliceQuantum) * kSliceQuantum);
  std::vector<WorkItem> items;
  std::vector<int> sys_slices;
  int max_slices = 1;
  build_items(c, t, items, sys_slices, max_slices);
  t.n_ctas = std::max(1, std::min<int>(occ * c->sm_count, (int)std::max<size_t>(1, items.size())));
  nbody_status s = upload_items(c, items, vjp ? &c->d_vitems : &c->d_items);
  if (s) return s;
  s = upload_chunks(c, sys_slices, vjp ? &c->d_vchunks : &c->d_chunks);
  if (s) return s;
  const size_t per = vjp ? 64 : 32;
  s = ensure(c, c->part, (size_t)max_slices * (size_t)c->n_total * per);
  if (s) return s;
  if (vjp) {
    c->vt = t, c->n_vitems = (int)items.size(), c->vmax_slices = max_slices, c->vjp_ready = true;
  } else {
    c->ft = t, c->n_items = (int)items.size(), c->max_slices = max_slices;
  }
  return NBODY_OK;
}

// refine: the mixed force and VJP kernels may use the staged remainders (near pairs).
PairLaunch pair_launch(nbody_ctx* c, bool vjp, bool refine = true, bool phi = true) {
  PairLaunch L{};
  const bool lo = refine && c->cfg.precision == NBODY_MIXED && c->stage_lo.p;
  L.stage_lo = lo ? static_cast<const float4*>(c->stage_lo.p) : nullptr;
  L.law = vjp ? 0 : c->cfg.law;
  const double sc2 = c->stage_scale * c->stage_scale;  // staged length units: sigma (mixed LJ) or 1
  L.sigma2 = c->cfg.lj_sigma * c->cfg.lj_sigma * sc2;   // 1 for mixed Lennard-Jones
  L.r2_near = 0.f;
  if (lo)
    L.r2_near = c->cfg.law == NBODY_LAW_LJ
                    ? (float)(kNearRadiusSigma * kNearRadiusSigma * L.sigma2 + c->cfg.eps * c->cfg.eps * sc2)
                    : (float)(kNearRadiusEps * kNearRadiusEps * c->cfg.eps * c->cfg.eps);
  L.stage_x = c->stage.p;
  L.stage_w = c->stage_w.p;
  L.items = vjp ? c->d_vitems : c->d_items;
  L.n_items = vjp ? c->n_vitems : c->n_items;
  L.counter = c->counter;
  L.part = static_cast<double*>(c->part.p);
  L.n_total = c->n_total;
  L.eps2 = c->cfg.eps * c->cfg.eps * sc2;
  const Tiling& t = vjp ? c->vt : c->ft;
  L.block = t.block, L.ipt = t.ipt, L.jtile = t.jtile, L.n_ctas = t.n_ctas;
  L.variant = t.variant;
  L.params = vjp && c->vjp_params ? 1 : 0;
  L.phi = phi ? 1 : 0;
  L.status = c->status;
  L.block_bodies = t.block * t.ipt;
  const size_t per = vjp ? (L.params ? 96 : 64) : 32;  // partial-sum bytes per body and slice
  L.part_slices = c->n_total > 0 ? (int32_t)std::min<size_t>(INT32_MAX, c->part.bytes / ((size_t)c->n_total * per)) : 0;
  return L;
}

// Slices of partials (bytes_per_body each) the partial-sum buffer holds.
int32_t part_slices(const nbody_ctx* c, size_t bytes_per_body) {
  if (c->n_total <= 0) return 0;
  return (int32_t)std::min<size_t>(INT32_MAX, c->part.bytes / ((size_t)c->n_total * bytes_per_body));
}

cudaEvent_t pooled_event(nbody_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Launches an all-pairs kernel, bracketed by an event pair when profiling an
// eager (non-capturing) stream.
nbody_status run_pair(nbody_ctx* c, cudaStream_t st, bool vjp, bool phi = true) {
  if (c->n_total == 0) return NBODY_OK;
  PairLaunch L = pair_launch(c, vjp, true, phi);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profiling && !c->capturing) {
    e0 = pooled_event(c);
    e1 = pooled_event(c);
    if (e0 && e1) NB_CUDA(c, cudaEventRecord(e0, st));
  }
  NB_CUDA(c, vjp ? launch_vjp(c->cfg.precision, L, st) : launch_force(c->cfg.precision, L, st));
  if (e0 && e1) {
    NB_CUDA(c, cudaEventRecord(e1, st));
    c->ev_used.push_back({vjp ? 1 : 0, {e0, e1}});
  }
  ++c->launches;
  return NBODY_OK;
}

// phi: whether the potential is needed (an energy record, a phi output); only
// the packed mixed kernel can skip it, the others always form it.
nbody_status run_force(nbody_ctx* c, cudaStream_t st, bool phi) { return run_pair(c, st, false, phi); }
nbody_status run_vjp(nbody_ctx* c, cudaStream_t st) { return run_pair(c, st, true); }


PostLaunch post_launch(nbody_ctx* c, unsigned mode, double* x, double* v, const double* m, double* a, double* phi) {
  PostLaunch P{};
  P.chunks = c->d_chunks;
  P.n_chunks = (int32_t)c->chunks.size();
  P.part = static_cast<const double*>(c->part.p);
  P.n_total = c->n_total;
  P.G = c->cfg.G;
  P.half_dt = 0.5 * c->cfg.dt;
  P.dt = c->cfg.dt;
  P.x = x, P.v = v, P.m = m, P.a = a, P.phi = phi;
  P.x_copy = nullptr;
  P.mode = mode;
  P.precision = c->cfg.precision;
  P.law = c->cfg.law;
  P.lj_eps = c->cfg.lj_epsilon;
  P.stage_scale = c->stage_scale;
  P.box = c->cfg.box;
  P.stage = c->stage.p;
  P.stage_lo = c->stage_lo.p;
  P.centre = static_cast<const double*>(c->centre.p);
  P.epart = static_cast<double*>(c->epart.p);
  P.status = c->status;
  P.eout = nullptr;
  P.sys_chunk = c->d_sys_chunk;
  P.n_sys = c->n_sys;
  P.done = c->counter + 4;
  P.part_slices = part_slices(c, 32);
  return P;
}

nbody_status run_post(nbody_ctx* c, const PostLaunch& P, cudaStream_t st) {
  if (P.n_chunks == 0) return NBODY_OK;
  NB_CUDA(c, launch_post(P, st));
  ++c->launches;
  return NBODY_OK;
}

nbody_status run_centre(nbody_ctx* c, const double* x, const double* m, cudaStream_t st) {
  if (c->cfg.precision != NBODY_MIXED || c->n_total == 0) return NBODY_OK;
  NB_CUDA(c, launch_centre(c->d_chunks, (int)c->chunks.size(), c->d_sys_chunk, c->d_off, c->n_sys, x, m,
                           static_cast<double*>(c->epart.p), static_cast<double*>(c->centre.p), c->counter + 5,
                           c->n_total, c->status, st));
  c->launches += c->chunks.empty() ? 0 : 1;
  return NBODY_OK;
}


// The KDK sequence of nbody_step, enqueued on st (eager or under capture).
nbody_status enqueue_step(nbody_ctx* c, double* x, double* v, const double* m, double* a, int a_valid, int n_steps,
                          double* elog, cudaStream_t st) {
  nbody_status s;
  if ((s = run_centre(c, x, m, st))) return s;
  if (!a_valid) {
    if ((s = run_post(c, post_launch(c, kStage, x, v, m, a, nullptr), st))) return s;
    if ((s = run_force(c, st, false))) return s;
    if ((s = run_post(c, post_launch(c, kCombine, x, v, m, a, nullptr), st))) return s;
  }
  if (n_steps == 0) return NBODY_OK;
  if ((s = run_post(c, post_launch(c, kDrift | kStage, x, v, m, a, nullptr), st))) return s;
  const int every = c->cfg.energy_every;
  // With up to four systems a step's energy record, except the call's last, is
  // finished by one extra CTA of the next step's k_post (same fixed-order sum)
  // instead of by the last CTA of its own: the ticket and the serial per-system
  // sum leave the step's critical path. The chunk partials alternate between two
  // sets so that the pending set survives the next step's own record.
  const bool defer = c->n_sys <= 4;
  const size_t eset = std::max<size_t>(1, c->chunks.size()) * kEnergyVals;
  const double* pend_part = nullptr;
  double* pend_out = nullptr;
  int rec = 0;
  for (int k = 0; k < n_steps; ++k) {
    const bool rec_now = elog && every > 0 && (k + 1) % every == 0;
    if ((s = run_force(c, st, rec_now))) return s;
    unsigned mode = kCombine | kKickEnd;
    if (rec_now) mode |= kEnergy;
    if (k + 1 < n_steps) mode |= kDrift | kStage;
    PostLaunch P = post_launch(c, mode, x, v, m, a, nullptr);
    P.eprev = pend_part, P.eprev_out = pend_out;
    pend_part = nullptr, pend_out = nullptr;
    if (rec_now) {
      double* out = elog + (int64_t)rec * c->n_sys * 9;
      P.epart = static_cast<double*>(c->epart.p) + (size_t)(rec % 2) * eset;
      ++rec;
      if (defer && k + 1 < n_steps)
        pend_part = P.epart, pend_out = out;  // the next k_post finishes it
      else
        P.eout = out;
    }
    if ((s = run_post(c, P, st))) return s;
  }
  return NBODY_OK;
}

// ---------------------------------------------------------------------------
// autotuner

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Fills the staging buffers with synthetic bodies so that candidate tilings
// can be timed before any user data exists: for gravity each system is a
// Plummer sphere (scale radius 1, total mass 1, radii truncated at 20), for
// Lennard-Jones a gas on a jittered lattice, the distributions these kernels
// are typically run on, which also set how often the near-pair correction of
// the mixed kernels fires.
nbody_status fill_synthetic(nbody_ctx* c, bool with_w) {
  const int64_t n = c->n_total;
  uint64_t seed = 12345;
  auto u01 = [&] { return ((double)(splitmix(seed) >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  std::vector<double> pos(3 * (size_t)n), mass((size_t)n);
  for (int s = 0; s < c->n_sys; ++s) {
    const int64_t b = c->offsets[s], e = c->offsets[s + 1];
    if (c->cfg.law == NBODY_LAW_LJ) {
      // a Lennard-Jones gas: jittered cubic lattice at the box's density (0.05 / sigma^3 without walls)
      const double sig = c->cfg.lj_sigma, nn = (double)(e - b);
      const double side = c->cfg.box > 0 ? c->cfg.box : std::cbrt(nn / 0.05) * sig;
      const int64_t k = std::max<int64_t>(1, (int64_t)std::ceil(std::cbrt(nn) - 1e-9));
      const double h = side / (double)k;
      for (int64_t i = b; i < e; ++i) {
        const int64_t q = i - b;
        const int64_t lat[3] = {q % k, (q / k) % k, q / (k * k)};
        for (int d = 0; d < 3; ++d) pos[3 * i + d] = ((double)lat[d] + 0.5 + 0.2 * (u01() - 0.5)) * h - 0.5 * side;
        mass[i] = 1.0;
      }
      continue;
    }
    for (int64_t i = b; i < e; ++i) {
      double r;
      do {
        r = 1.0 / std::sqrt(std::pow(u01(), -2.0 / 3.0) - 1.0);
      } while (!(r <= 20.0));
      const double z = 2.0 * u01() - 1.0, ph = 6.283185307179586 * u01();
      const double rho = std::sqrt(std::max(0.0, 1.0 - z * z));
      pos[3 * i + 0] = r * rho * std::cos(ph);
      pos[3 * i + 1] = r * rho * std::sin(ph);
      pos[3 * i + 2] = r * z;
      mass[i] = 1.0 / (double)(e - b);
    }
  }
  if (c->cfg.precision == NBODY_MIXED) {
    std::vector<float4> h(n), hl(n);
    for (int64_t i = 0; i < n; ++i) {
      const double X = pos[3 * i] * c->stage_scale, Y = pos[3 * i + 1] * c->stage_scale,
                   Z = pos[3 * i + 2] * c->stage_scale;
      const float hx = (float)X, hy = (float)Y, hz = (float)Z;
      h[i] = make_float4(hx, hy, hz, (float)mass[i]);
      hl[i] = make_float4((float)(X - hx), (float)(Y - hy), (float)(Z - hz), 0.f);
    }
    NB_CUDA(c, cudaMemcpy(c->stage.p, h.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    if (c->stage_lo.p) NB_CUDA(c, cudaMemcpy(c->stage_lo.p, hl.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    if (with_w) {
      for (int64_t i = 0; i < n; ++i) h[i] = make_float4((float)u01(), (float)u01(), (float)u01(), 0.f);
      NB_CUDA(c, cudaMemcpy(c->stage_w.p, h.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    }
  } else {
    std::vector<double4_32a> h(n);
    for (int64_t i = 0; i < n; ++i) h[i] = make_double4_32a(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
    NB_CUDA(c, cudaMemcpy(c->stage.p, h.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
    if (with_w) {
      for (int64_t i = 0; i < n; ++i) h[i] = make_double4_32a(u01(), u01(), u01(), 0.0);
      NB_CUDA(c, cudaMemcpy(c->stage_w.p, h.data(), n * sizeof(double4_32a), cudaMemcpyHostToDevice));
    }
  }
  NB_CUDA(c, cudaDeviceSynchronize());
  return NBODY_OK;
}

// Times the installed tiling; returns seconds per interaction slot (lower is
// better), the best of three timed launches. Short work lists are timed whole,
// together with the O(N) pass that adds the slices, so that lists of shorter
// slices pay for their partial-sum traffic and the tail of the schedule
// counts; long lists are timed on a prefix of two items per persistent CTA.
nbody_status time_tiling(nbody_ctx* c, bool vjp, double* cost) {
  PairLaunch L = pair_launch(c, vjp);
  const Tiling& t = vjp ? c->vt : c->ft;
  auto launch = [&](const PairLaunch& P) {
    return vjp ? launch_vjp(c->cfg.precision, P, c->stream) : launch_force(c->cfg.precision, P, c->stream);
  };
  PostLaunch C{};
  C.chunks = vjp ? c->d_vchunks : c->d_chunks;
  C.n_chunks = (int32_t)c->chunks.size();
  C.part = static_cast<const double*>(c->part.p);
  C.n_total = c->n_total;
  C.G = 1.0;
  C.a = static_cast<double*>(c->a_scratch.p);
  C.mode = kCombine;
  C.status = c->status;
  C.n_sys = c->n_sys;
  C.part_slices = part_slices(c, vjp ? 64 : 32);
  cudaEvent_t ev[4];
  for (auto& e : ev) NB_CUDA(c, cudaEventCreate(&e));
  auto timed = [&](const PairLaunch& P, bool combine, float* best_ms) -> cudaError_t {
    cudaError_t err = launch(P);  // warm-up; also writes every partial the combine reads
    if (err == cudaSuccess && combine) err = launch_post(C, c->stream);
    *best_ms = 1e30f;
    // best of 3 launches, or of as many as fill ~2 ms (at most 20) for short ones
    int reps = 3;
    for (int rep = 0; rep < reps && err == cudaSuccess; ++rep) {
      err = cudaEventRecord(ev[0], c->stream);
      if (err == cudaSuccess) err = launch(P);
      if (err == cudaSuccess && combine) err = launch_post(C, c->stream);
      if (err == cudaSuccess) err = cudaEventRecord(ev[1], c->stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (err == cudaSuccess) *best_ms = std::min(*best_ms, ms);
      if (rep == 0 && err == cudaSuccess) reps = std::max(3, std::min(20, (int)std::ceil(2.0 / std::max(ms, 1e-3f))));
    }
    c->launches += (reps + 1) * (combine ? 2 : 1);
    return err;
  };
  PairLaunch P = L;
  P.n_items = std::min(L.n_items, 2 * t.n_ctas);
  float ms = 0.f;
  cudaError_t err = cudaSuccess;
  if (P.n_items < L.n_items) err = timed(P, false, &ms);
  if (err == cudaSuccess && (P.n_items == L.n_items || ms * (double)L.n_items / std::max(1, P.n_items) < 60.0)) {
    P = L;
    err = timed(P, !vjp, &ms);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return fail(c, NBODY_ECUDA, "autotune launch failed: %s", cudaGetErrorString(err));
  // interaction slots covered by the timed items (the list is longest-first)
  double slots = 0.0;
  {
    std::vector<WorkItem> h(P.n_items);
    NB_CUDA(c, cudaMemcpy(h.data(), L.items, h.size() * sizeof(WorkItem), cudaMemcpyDeviceToHost));
    for (const auto& w : h) slots += (double)(w.i_end - w.i_begin) * (double)(w.j_end - w.j_begin);
  }
  *cost = slots > 0 ? (ms * 1e-3) / slots : 1e30;
  return NBODY_OK;
}

// ---------------------------------------------------------------------------
// tuning cache: NBODY_TUNE_CACHE=<file> keeps the tuner's choices across runs.
// One line per choice, "<key>\t<block> <ipt> <jtile> <slice> <variant> <tail>"; the key
// holds the device, the kernel (force or VJP), every configuration field the
// choice depends on and a hash of the system layout, so an entry is reused only
// for the same setup. A cached tiling that no longer installs is re-tuned.

std::string tune_key(const nbody_ctx* c, bool vjp) {
  const nbody_config& g = c->cfg;
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the offsets
  for (int s = 0; s <= c->n_sys; ++s) {
    uint64_t v = (uint64_t)c->offsets[s];
    for (int k = 0; k < 8; ++k, v >>= 8) h = (h ^ (v & 0xff)) * 1099511628211ull;
  }
  char buf[512];
  snprintf(buf, sizeof(buf),
           "v2|%s|cc%d|sm%d|%s|prec%d|law%d|var%d|b%d|r%d|j%d|s%d|nsys%d|n%lld|lay%016llx|eps%.17g|sig%.17g|box%.17g",
           c->dev_name.c_str(), c->dev_cc, c->sm_count, vjp ? "vjp" : "force", g.precision, g.law, g.variant,
           vjp ? 0 : g.block, vjp ? 0 : g.i_per_thread, vjp ? 0 : g.j_tile, vjp ? 0 : g.slice, c->n_sys,
           (long long)c->n_total, (unsigned long long)h, g.eps, g.lj_sigma, g.box);
  for (char* p = buf; *p; ++p)
    if (*p == '\t' || *p == '\n') *p = ' ';
  return buf;
}

bool tune_cache_lookup(const nbody_ctx* c, bool vjp, Tiling* t) {
  const char* path = getenv("NBODY_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  const std::string key = tune_key(c, vjp);
  bool found = false;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = '\0';
    if (key != line) continue;
    Tiling u;
    if (sscanf(tab + 1, "%d %d %d %d %d %d", &u.block, &u.ipt, &u.jtile, &u.slice, &u.variant, &u.tail) == 6)
      *t = u, found = true;
  }
  fclose(f);
  return found;
}

void tune_cache_store(const nbody_ctx* c, bool vjp, const Tiling& t) {
  const char* path = getenv("NBODY_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d %d %d %d %d %d\n", tune_key(c, vjp).c_str(), t.block, t.ipt, t.jtile, t.slice, t.variant, t.tail);
  fclose(f);
}

nbody_status autotune(nbody_ctx* c, bool vjp) {
  NvtxRange range(c->nvtx, vjp ? "nbody_autotune_vjp" : "nbody_autotune");
  {
    Tiling t;
    if (tune_cache_lookup(c, vjp, &t)) {
      t.n_ctas = 0;
      if (install_tiling(c, t, vjp) == NBODY_OK) return NBODY_OK;
      cudaGetLastError();
    }
  }
  const nbody_config& g = c->cfg;
  std::vector<Tiling> cands;
  const int blocks[] = {128, 256};
  const int ipts_f[] = {1, 2, 4}, ipts_v[] = {1, 2};
  const int jts_v[] = {128, 256};
  // j-tiles: 128 and 256 for every kernel, 512 for the mixed kernels
  const std::vector<int> jts_f = g.precision == NBODY_MIXED ? std::vector<int>{128, 256, 512} : std::vector<int>{128, 256};
  std::vector<int> variants = {0};
  if (g.precision == NBODY_MIXED) {
    // a variant fixed by the caller applies to the force and the VJP kernels (the
    // register-capped packed force kernel pairs with the packed VJP)
    if (vjp)
      variants = g.variant ? std::vector<int>{std::min(g.variant - 1, 1)} : std::vector<int>{0, 1};
    else
      variants = g.variant ? std::vector<int>{g.variant - 1} : std::vector<int>{0, 1, 2};
    // Lennard-Jones: the packed kernel, uncapped and capped (6 CTAs per SM)
    if (!vjp && g.law == NBODY_LAW_LJ) variants = g.variant ? std::vector<int>{g.variant - 1} : std::vector<int>{1, 2};
  }
  for (int var : variants)
    for (int b : blocks) {
      if (!vjp && g.block && g.block != b) continue;
      for (int r : (vjp ? std::vector<int>(ipts_v, ipts_v + 2) : std::vector<int>(ipts_f, ipts_f + 3))) {
        if (!vjp && g.i_per_thread && g.i_per_thread != r) continue;
        for (int j : (vjp ? std::vector<int>(jts_v, jts_v + 2) : jts_f)) {
          if (!vjp && g.j_tile && g.j_tile != j) continue;
          Tiling t;
          t.block = b, t.ipt = r, t.jtile = j, t.slice = vjp ? 0 : g.slice, t.variant = var;
          cands.push_back(t);
        }
      }
    }
  if (cands.empty()) return fail(c, NBODY_EINVAL, "no compiled tiling matches the requested parameters");
  nbody_status s = fill_synthetic(c, vjp);
  if (s) return s;
  if ((s = ensure(c, c->a_scratch, (size_t)c->n_total * 3 * sizeof(double)))) return s;
  // Large layouts are compared on work lists of short slices (the cost per
  // interaction no longer depends on the slice length there), which keeps the
  // timed prefix short; their final slice is the automatic choice.
  double pairs = 0.0;
  for (int k = 0; k < c->n_sys; ++k) {
    const double n = (double)(c->offsets[k + 1] - c->offsets[k]);
    pairs += n * n;
  }
  const bool large = pairs > kTuneLargePairs;
  const char* verbose_env = getenv("NBODY_TUNE_VERBOSE");  // tuning log on stderr when set to 1
  const bool verbose = verbose_env && verbose_env[0] == '1';
  // one timed measurement of candidate t0 (large layouts: short slices, scaled by the
  // wave quantisation of the final work list, which the prefix cannot see)
  auto measure = [&](const Tiling& t0, double* cost) -> nbody_status {
    Tiling t = t0;
    if (large && t.slice == 0) t.slice = kTuneSlice;
    nbody_status r;
    if ((r = install_tiling(c, t, vjp))) return r;
    if ((r = time_tiling(c, vjp, cost))) return r;
    if (large && t0.slice == 0) {
      const int ctas = (vjp ? c->vt : c->ft).n_ctas;
      const int64_t items = count_items(c, t0, auto_slice(c, t0, ctas));
      const double waves = (double)items / std::max(1, ctas);
      if (waves > 0) *cost *= std::ceil(waves) / waves;
    }
    if (verbose)
      fprintf(stderr, "nbody tune %s: variant=%d block=%d ipt=%d jtile=%d slice=%d ctas=%d items=%d -> %.4g ps/pair\n",
              vjp ? "vjp" : "force", (vjp ? c->vt : c->ft).variant, t.block, t.ipt, t.jtile,
              (vjp ? c->vt : c->ft).slice, (vjp ? c->vt : c->ft).n_ctas, vjp ? c->n_vitems : c->n_items, *cost * 1e12);
    return NBODY_OK;
  };
  std::vector<std::pair<double, Tiling>> timed;
  // one untimed pass first, so that the GPU has left its idle clocks before the first candidate is timed
  for (const Tiling& t0 : cands) {
    if (ctas_per_sm(g.precision, t0, vjp, g.law) <= 0) continue;
    double cost = 0;
    if ((s = measure(t0, &cost))) return s;
    break;
  }
  for (const Tiling& t0 : cands) {
    if (ctas_per_sm(g.precision, t0, vjp, g.law) <= 0) continue;
    double cost = 0;
    if ((s = measure(t0, &cost))) return s;
    timed.push_back({cost, t0});
  }
  if (timed.empty()) return fail(c, NBODY_EINVAL, "no compiled tiling matches the requested parameters");
  // the candidates within 8% of the best (at most five) are timed twice more, interleaved, and
  // keep their best time: single timings differ by 1-3% from run to run
  std::stable_sort(timed.begin(), timed.end(),
                   [](const std::pair<double, Tiling>& a, const std::pair<double, Tiling>& b) { return a.first < b.first; });
  size_t top = 1;
  while (top < timed.size() && top < 5 && timed[top].first <= 1.08 * timed[0].first) ++top;
  for (int round = 0; round < 2 && top > 1; ++round)
    for (size_t k = 0; k < top; ++k) {
      double cost = 0;
      if ((s = measure(timed[k].second, &cost))) return s;
      timed[k].first = std::min(timed[k].first, cost);
    }
  // order the re-timed candidates; the first is the choice unless the slice refinement finds better
  std::stable_sort(timed.begin(), timed.begin() + top,
                   [](const std::pair<double, Tiling>& a, const std::pair<double, Tiling>& b) { return a.first < b.first; });
  Tiling bt = timed[0].second;
  // slice-length refinement of all those tilings (up to five): the automatic
  // choice, half and twice it, and (one system) the lengths whose work list
  // fills a whole number of waves of the persistent grid (equal items, a
  // multiple of the CTA count, leave no CTA idle at the end of the launch),
  // each with equal slices and with a halving tail. Tilings are refined
  // together because the tail helps some more than others (it changes how the
  // last wave ends): with equal slices several tilings often lie within 0.2%
  // of each other, and the one the tail favours must not be cut by that noise.
  // Every setting is timed twice, interleaved, the best kept.
  if (!vjp && g.slice == 0 && !large) {
    std::vector<Tiling> settings;
    for (size_t f = 0; f < top; ++f) {
      Tiling base = timed[f].second;
      base.slice = 0;
      base.tail = 0;
      if ((s = install_tiling(c, base, vjp))) return s;
      const int L0 = c->ft.slice;
      const int64_t n_ctas = c->ft.n_ctas;
      std::vector<int> ls = {L0 / 2, L0, L0 * 2};
      if (c->n_sys == 1) {
        const int64_t n = c->offsets[1], tiles = (n + (int64_t)base.block * base.ipt - 1) / ((int64_t)base.block * base.ipt);
        for (int64_t W = 1; W <= 64 && ls.size() < 7; ++W) {
          const int64_t ns = W * n_ctas / tiles;  // slices per tile with tiles x ns <= W x CTAs
          if (ns < 1 || (double)(tiles * ns) < 0.98 * (double)(W * n_ctas)) continue;
          int64_t len = (n + ns - 1) / ns;
          len = ((len + kSliceQuantum - 1) / kSliceQuantum) * kSliceQuantum;
          if ((n + len - 1) / len != ns || len < L0 / 4 || len > 4 * (int64_t)L0) continue;
          if (std::find(ls.begin(), ls.end(), (int)len) == ls.end()) ls.push_back((int)len);
        }
      }
      for (int len : ls) {
        if (len < kSliceQuantum) continue;
        for (int tail = 0; tail < 2; ++tail) {
          Tiling t = base;
          t.slice = len;
          t.tail = tail;
          settings.push_back(t);
        }
      }
    }
    std::vector<double> lc(settings.size(), 1e300);
    for (int round = 0; round < 2; ++round)
      for (size_t k = 0; k < settings.size(); ++k) {
        if ((s = install_tiling(c, settings[k], vjp))) return s;
        double cost = 0;
        if ((s = time_tiling(c, vjp, &cost))) return s;
        if (verbose)
          fprintf(stderr, "nbody tune variant=%d block=%d ipt=%d jtile=%d slice=%d tail=%d items=%d -> %.4g ps/pair\n",
                  settings[k].variant, settings[k].block, settings[k].ipt, settings[k].jtile, settings[k].slice,
                  settings[k].tail, c->n_items, cost * 1e12);
        lc[k] = std::min(lc[k], cost);
      }
    double bc = 1e300;
    for (size_t k = 0; k < settings.size(); ++k)
      if (lc[k] < bc) bc = lc[k], bt = settings[k];
  }
  bt.n_ctas = 0;
  if ((s = install_tiling(c, bt, vjp))) return s;
  // synthetic data must not leave a latched device condition behind
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  NB_CUDA(c, cudaMemset(c->status, 0, sizeof(unsigned)));
  Tiling chosen = vjp ? c->vt : c->ft;
  tune_cache_store(c, vjp, chosen);
  return NBODY_OK;
}

nbody_status validate_cfg(const nbody_config* g) {
  if (!g) return NBODY_EINVAL;
  if (!finite(g->G) || !finite(g->eps) || g->eps < 0 || !finite(g->dt)) return NBODY_EINVAL;
  if (g->precision != NBODY_FP64 && g->precision != NBODY_MIXED) return NBODY_EINVAL;
  if (g->energy_every < 0 || g->variant < 0 || g->variant > 3) return NBODY_EINVAL;
  if (g->precision == NBODY_FP64 && g->variant > 1) return NBODY_EINVAL;
  if (g->block && g->block != 128 && g->block != 256) return NBODY_EINVAL;
  if (g->i_per_thread && g->i_per_thread != 1 && g->i_per_thread != 2 && g->i_per_thread != 4) return NBODY_EINVAL;
  if (g->j_tile && g->j_tile != 128 && g->j_tile != 256 && g->j_tile != 512) return NBODY_EINVAL;
  if (g->j_tile == 512 && g->precision != NBODY_MIXED) return NBODY_EINVAL;
  if (g->slice < 0) return NBODY_EINVAL;
  if (g->flags & ~(NBODY_FLAG_GRAPH | NBODY_FLAG_NOCHECK)) return NBODY_EINVAL;
  if (g->law != NBODY_LAW_GRAVITY && g->law != NBODY_LAW_LJ) return NBODY_EINVAL;
  if (g->reserved != 0) return NBODY_EINVAL;
  if (!finite(g->box) || g->box < 0) return NBODY_EINVAL;
  if (g->law == NBODY_LAW_LJ) {
    if (!finite(g->lj_epsilon) || !finite(g->lj_sigma) || !(g->lj_sigma > 0)) return NBODY_EINVAL;
    if (g->precision == NBODY_MIXED && g->variant == 1) return NBODY_EINVAL;  // no scalar Lennard-Jones kernel
  }
  return NBODY_OK;
}

void free_ctx(nbody_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& u : c->ev_used) cudaEventDestroy(u.second.first), cudaEventDestroy(u.second.second);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (DevBuf* b : {&c->stage, &c->stage_lo, &c->stage_w, &c->part, &c->centre, &c->epart, &c->status_counter, &c->a_scratch,
                    &c->xw, &c->vw, &c->aw, &c->ckpt, &c->traj, &c->hx, &c->hv, &c->hm, &c->ha, &c->hlog})
    release(*b);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->d_chunks) cudaFree(c->d_chunks);
  if (c->d_vchunks) cudaFree(c->d_vchunks);
  if (c->d_sys_chunk) cudaFree(c->d_sys_chunk);
  if (c->d_off) cudaFree(c->d_off);
  if (c->d_items) cudaFree(c->d_items);
  if (c->d_vitems) cudaFree(c->d_vitems);
  delete c;
}

nbody_status check_state_args(nbody_ctx* c, const double* x, const double* v, const double* m, const double* a,
                              bool need_v, bool need_a) {
  const size_t n3 = (size_t)c->n_total * 3 * sizeof(double), n1 = (size_t)c->n_total * sizeof(double);
  nbody_status s;
  if ((s = check_dev(c, x, n3, "x"))) return s;
  if (need_v && (s = check_dev(c, v, n3, "v"))) return s;
  if ((s = check_dev(c, m, n1, "m"))) return s;
  if (need_a && (s = check_dev(c, a, n3, "a"))) return s;
  return NBODY_OK;
}

// RAII switch of the VJP launches to the parameter-gradient variant.
struct ParamsScope {
  nbody_ctx* c;
  ParamsScope(nbody_ctx* ctx, bool on) : c(ctx) { c->vjp_params = on; }
  ~ParamsScope() { c->vjp_params = false; }
};

nbody_status adjoint_sweep(nbody_ctx* c, const double* x0, const double* v0, const double* m, int32_t T, int32_t K,
                           const double* lam_xT, const double* lam_vT, double* g_x0, double* g_v0, double* g_m,
                           double* g_params) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_adjoint");
  if (T < 0 || K < 1) return fail(c, NBODY_EINVAL, "need n_steps >= 0 and checkpoint_every >= 1");
  if (c->cfg.law != NBODY_LAW_GRAVITY || c->cfg.box > 0)
    return fail(c, NBODY_EUNSUPPORTED, "nbody_adjoint supports softened gravity without walls only");
  if (T > 0 && !(c->cfg.dt > 0)) return fail(c, NBODY_EINVAL, "dt must be > 0");
  if (c->n_total == 0) return NBODY_OK;
  const size_t n = (size_t)c->n_total, n3b = n * 3 * sizeof(double);
  nbody_status s;
  if ((s = check_state_args(c, x0, v0, m, nullptr, true, false))) return s;
  if ((s = check_dev(c, lam_xT, n3b, "lam_xT"))) return s;
  if ((s = check_dev(c, lam_vT, n3b, "lam_vT"))) return s;
  if ((s = check_dev(c, g_x0, n3b, "g_x0"))) return s;
  if ((s = check_dev(c, g_v0, n3b, "g_v0"))) return s;
  if ((s = check_dev(c, g_m, n * sizeof(double), "g_m"))) return s;
  if (g_params && (s = check_dev(c, g_params, (size_t)c->n_sys * 2 * sizeof(double), "g_params"))) return s;
  cudaStream_t st = c->stream;

  const size_t stage_bytes = n * (c->cfg.precision == NBODY_MIXED ? sizeof(float4) : sizeof(double4_32a));
  if ((s = ensure(c, c->stage_w, stage_bytes))) return s;
  if (!c->vjp_ready) {
    // VJP tiling: tuned once per context (synchronises the stream)
    NB_CUDA(c, cudaStreamSynchronize(st));
    if ((s = autotune(c, true))) return s;
  }
  const int vjp_bytes = g_params ? 96 : 64;  // per body and slice: 2 or 3 double4
  if ((s = ensure(c, c->part, (size_t)std::max(c->max_slices * 32, c->vmax_slices * vjp_bytes) * n))) return s;

  NB_CUDA(c, cudaMemcpyAsync(g_x0, lam_xT, n3b, cudaMemcpyDeviceToDevice, st));
  NB_CUDA(c, cudaMemcpyAsync(g_v0, lam_vT, n3b, cudaMemcpyDeviceToDevice, st));
  NB_CUDA(c, cudaMemsetAsync(g_m, 0, n * sizeof(double), st));
  if (g_params) NB_CUDA(c, cudaMemsetAsync(g_params, 0, (size_t)c->n_sys * 2 * sizeof(double), st));
  if (T == 0) return NBODY_OK;
  ParamsScope scope(c, g_params != nullptr);

  const int nseg = (T + K - 1) / K;
  if ((s = ensure(c, c->xw, n3b)) || (s = ensure(c, c->vw, n3b)) || (s = ensure(c, c->aw, n3b))) return s;
  if ((s = ensure(c, c->ckpt, (size_t)nseg * 3 * n3b))) return s;
  if ((s = ensure(c, c->traj, (size_t)(K + 1) * n3b))) return s;
  double* xw = static_cast<double*>(c->xw.p);
  double* vw = static_cast<double*>(c->vw.p);
  double* aw = static_cast<double*>(c->aw.p);
  double* ck = static_cast<double*>(c->ckpt.p);
  double* X = static_cast<double*>(c->traj.p);
  const size_t n3 = n * 3;

  // staging origin for the whole call, from x0 (the same as nbody_step uses)
  if ((s = run_centre(c, x0, m, st))) return s;
  NB_CUDA(c, cudaMemcpyAsync(xw, x0, n3b, cudaMemcpyDeviceToDevice, st));
  NB_CUDA(c, cudaMemcpyAsync(vw, v0, n3b, cudaMemcpyDeviceToDevice, st));
  if ((s = run_post(c, post_launch(c, kStage, xw, vw, m, aw, nullptr), st))) return s;
  if ((s = run_force(c, st, false))) return s;
  if ((s = run_post(c, post_launch(c, kCombine, xw, vw, m, aw, nullptr), st))) return s;

  // one KDK step on (xw, vw, aw), optionally copying x after the drift
  auto step = [&](double* xcopy) -> nbody_status {
    nbody_status r;
    PostLaunch P = post_launch(c, kDrift | kStage, xw, vw, m, aw, nullptr);
    P.x_copy = xcopy;
    if ((r = run_post(c, P, st))) return r;
    if ((r = run_force(c, st, false))) return r;
    return run_post(c, post_launch(c, kCombine | kKickEnd, xw, vw, m, aw, nullptr), st);
  };

  // forward pass: checkpoints (x, v, a) at the start of every segment; it stops at
  // the last checkpoint, since the reverse sweep recomputes the last segment anyway
  std::unique_ptr<NvtxRange> fwd(new NvtxRange(c->nvtx, "forward"));
  const int last_ckpt = (nseg - 1) * K;
  for (int t = 0; t <= last_ckpt; ++t) {
    if (t % K == 0) {
      double* cp = ck + (size_t)(t / K) * 3 * n3;
      NB_CUDA(c, cudaMemcpyAsync(cp, xw, n3b, cudaMemcpyDeviceToDevice, st));
      NB_CUDA(c, cudaMemcpyAsync(cp + n3, vw, n3b, cudaMemcpyDeviceToDevice, st));
      NB_CUDA(c, cudaMemcpyAsync(cp + 2 * n3, aw, n3b, cudaMemcpyDeviceToDevice, st));
    }
    if (t < last_ckpt && (s = step(nullptr))) return s;
  }

  fwd.reset();
  NvtxRange rev(c->nvtx, "reverse");
  // reverse sweep. VJPs at x_T (coef dt/2), x_s for 0 < s < T (coef dt: the
  // closing half-kick of step s-1 and the opening half-kick of step s share
  // x_s and the same weights), x_0 (coef dt/2).
  AdjLaunch A{};
  A.chunks = c->d_vchunks;
  A.n_chunks = (int32_t)c->chunks.size();
  A.part = static_cast<const double*>(c->part.p);
  A.n_total = c->n_total;
  A.G = c->cfg.G;
  A.dt = c->cfg.dt;
  A.m = m;
  A.lam_x = g_x0;
  A.lam_v = g_v0;
  A.g_m = g_m;
  A.precision = c->cfg.precision;
  A.stage_x = c->stage.p;
  A.stage_w = c->stage_w.p;
  A.stage_lo = c->stage_lo.p;
  A.centre = static_cast<const double*>(c->centre.p);
  A.status = c->status;
  A.g_params = g_params;
  A.eps = c->cfg.eps;
  A.cpart = static_cast<double*>(c->epart.p);
  A.sys_chunk = c->d_sys_chunk;
  A.n_sys = c->n_sys;
  A.done = c->counter + 6;
  A.part_slices = part_slices(c, g_params ? 96 : 64);
  const Chunk* vch = c->d_vchunks;
  const int nch = (int)c->chunks.size();
  for (int k = nseg - 1; k >= 0; --k) {
    const int s0 = k * K, s1 = std::min(T, s0 + K), len = s1 - s0;
    double* cp = ck + (size_t)k * 3 * n3;
    NB_CUDA(c, cudaMemcpyAsync(xw, cp, n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(c, cudaMemcpyAsync(vw, cp + n3, n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(c, cudaMemcpyAsync(aw, cp + 2 * n3, n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(c, cudaMemcpyAsync(X, xw, n3b, cudaMemcpyDeviceToDevice, st));
    // positions s0 .. top; a segment's end state is the next segment's start, whose
    // VJP that segment has already taken, so only the last segment steps to its end
    const int top = (k == nseg - 1) ? s1 : s1 - 1;
    for (int t = 0; t < top - s0; ++t)
      if ((s = step(X + (size_t)(t + 1) * n3))) return s;
    NB_CUDA(c, launch_stage_vec(vch, nch, c->cfg.precision, X + (size_t)(top - s0) * n3, m,
                                static_cast<const double*>(c->centre.p), c->stage.p, c->stage_lo.p, 1, c->n_total,
                                c->n_sys, c->status, st));
    ++c->launches;
    if (k == nseg - 1) {
      NB_CUDA(c, launch_stage_vec(vch, nch, c->cfg.precision, g_v0, m, static_cast<const double*>(c->centre.p),
                                  c->stage_w.p, nullptr, 0, c->n_total, c->n_sys, c->status, st));
      ++c->launches;
    }
    for (int t = top; t >= s0; --t) {
      if ((s = run_vjp(c, st))) return s;
      A.coef = (t == T || t == 0) ? 0.5 * c->cfg.dt : c->cfg.dt;
      A.drift_rev = t > 0;
      A.x_next = (t - 1 >= s0) ? X + (size_t)(t - 1 - s0) * n3 : nullptr;
      NB_CUDA(c, launch_adj_update(A, st));
      ++c->launches;
    }
  }
  return NBODY_OK;
}

// Device address of a mapped, page-locked host buffer (cudaHostAlloc /
// cudaHostRegister under unified addressing), or NULL for any other pointer.
double* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, const_cast<void*>(p), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<double*>(d);
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" {

int32_t nbody_version(void) { return (1 << 16) | 1; }

int32_t nbody_build_flags(void) {
#ifdef NBODY_DEBUG
  return 1;
#else
  return 0;
#endif
}

const char* nbody_last_error(const nbody_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  static thread_local std::string copy;
  std::lock_guard<std::mutex> lk(g_err_mu);
  copy = g_err;
  return copy.c_str();
}

int64_t nbody_launch_count(const nbody_ctx* ctx) { return ctx ? ctx->launches : 0; }

nbody_status nbody_init(nbody_ctx** out, const nbody_config* cfg, int64_t n_systems, const int64_t* offsets,
                        void* cuda_stream) {
  if (!out) return fail(nullptr, NBODY_EINVAL, "ctx out-pointer is NULL");
  *out = nullptr;
  if (validate_cfg(cfg) != NBODY_OK) return fail(nullptr, NBODY_EINVAL, "invalid nbody_config");
  if (n_systems < 1 || n_systems > (1 << 24) || !offsets)
    return fail(nullptr, NBODY_EINVAL, "n_systems must be in [1, 2^24] with a host offsets array");
  if (offsets[0] != 0) return fail(nullptr, NBODY_EINVAL, "offsets[0] must be 0");
  for (int64_t s = 0; s < n_systems; ++s)
    if (offsets[s + 1] < offsets[s]) return fail(nullptr, NBODY_EINVAL, "offsets must be non-decreasing");
  if (offsets[n_systems] >= kMaxBodies) return fail(nullptr, NBODY_EINVAL, "total body count must be < 2^29");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, NBODY_EUNSUPPORTED, "no CUDA device");
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, NBODY_EUNSUPPORTED, "cudaGetDeviceProperties failed");
  }
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, NBODY_EUNSUPPORTED, "libnbody is built for sm_103a; device %s is sm_%d%d", prop.name,
                prop.major, prop.minor);

  nbody_ctx* c = new (std::nothrow) nbody_ctx();
  if (!c) return fail(nullptr, NBODY_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  if (cfg->precision == NBODY_MIXED && cfg->law == NBODY_LAW_LJ) c->stage_scale = 1.0 / cfg->lj_sigma;
  c->device = dev;
  c->sm_count = prop.multiProcessorCount;
  c->dev_name = prop.name;
  c->dev_cc = prop.major * 10 + prop.minor;
  // host-side fault injection for tests: NBODY_FAULT_ALLOC=k makes the k-th scratch
  // allocation of this context report NBODY_ENOMEM (no device fault is involved)
  if (const char* fa = getenv("NBODY_FAULT_ALLOC")) c->fault_alloc = std::max<int64_t>(0, atoll(fa));
  if (const char* nv = getenv("NBODY_NVTX")) c->nvtx = nv[0] == '1';
  NvtxRange range_init(c->nvtx, "nbody_init");
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->n_sys = (int)n_systems;
  c->offsets.assign(offsets, offsets + n_systems + 1);
  c->n_total = offsets[n_systems];

  // chunks: runs of <= kChunk bodies inside one system
  c->sys_chunk.assign(c->n_sys + 1, 0);
  for (int s = 0; s < c->n_sys; ++s) {
    c->sys_chunk[s] = (int32_t)c->chunks.size();
    for (int64_t b = offsets[s]; b < offsets[s + 1]; b += kChunk)
      c->chunks.push_back(Chunk{s, (int32_t)b, (int32_t)std::min<int64_t>(offsets[s + 1], b + kChunk), 1});
  }
  c->sys_chunk[c->n_sys] = (int32_t)c->chunks.size();

  nbody_status s;
  auto bail = [&](nbody_status st) {
    set_global_error(c->err);
    free_ctx(c);
    return st;
  };
  const size_t n = (size_t)c->n_total;
  const size_t stage_bytes = n * (cfg->precision == NBODY_MIXED ? sizeof(float4) : sizeof(double4_32a));
  if ((s = ensure(c, c->stage, stage_bytes))) return bail(s);
  if (cfg->precision == NBODY_MIXED && (s = ensure(c, c->stage_lo, n * sizeof(float4)))) return bail(s);
  if ((s = ensure(c, c->centre, (size_t)c->n_sys * 3 * sizeof(double)))) return bail(s);
  // two sets of chunk partials: a step's energy record may be finished by the next step's k_post
  if ((s = ensure(c, c->epart, 2 * std::max<size_t>(1, c->chunks.size()) * kEnergyVals * sizeof(double)))) return bail(s);
  // [0..1] work counter, [2] status word, [4] energy ticket, [5] centre ticket, [6] adjoint-parameter ticket
  if ((s = ensure(c, c->status_counter, 8 * sizeof(unsigned)))) return bail(s);
  c->counter = static_cast<unsigned*>(c->status_counter.p);
  c->status = c->counter + 2;
  if (cudaMemset(c->status_counter.p, 0, 8 * sizeof(unsigned)) != cudaSuccess) return bail(fail(c, NBODY_ECUDA, "memset failed"));
  if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_status), sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    c->h_status = nullptr;
    return bail(fail(c, NBODY_ENOMEM, "cudaHostAlloc of the status word failed"));
  }
  *c->h_status = 0u;
  if (cudaMemset(c->centre.p, 0, (size_t)c->n_sys * 3 * sizeof(double)) != cudaSuccess)
    return bail(fail(c, NBODY_ECUDA, "memset failed"));
  if (cudaMalloc(&c->d_off, (n_systems + 1) * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&c->d_sys_chunk, (n_systems + 1) * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(c, NBODY_ENOMEM, "cudaMalloc of layout tables failed"));
  }
  if (cudaMemcpy(c->d_off, offsets, (n_systems + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_sys_chunk, c->sys_chunk.data(), (n_systems + 1) * sizeof(int32_t), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return bail(fail(c, NBODY_ECUDA, "upload of layout tables failed"));

  const bool fixed_variant = cfg->precision == NBODY_FP64 || cfg->variant != 0 || cfg->law == NBODY_LAW_LJ;
  if (c->n_total > 0 && (cfg->block == 0 || cfg->i_per_thread == 0 || cfg->j_tile == 0 || !fixed_variant)) {
    if ((s = autotune(c, false))) return bail(s);
  } else {
    Tiling t;
    t.block = cfg->block ? cfg->block : 256;
    t.ipt = cfg->i_per_thread ? cfg->i_per_thread : 2;
    t.jtile = cfg->j_tile ? cfg->j_tile : 128;
    t.slice = cfg->slice;
    t.variant = cfg->precision != NBODY_MIXED ? 0 : cfg->law == NBODY_LAW_LJ ? (cfg->variant == 3 ? 2 : 1) : cfg->variant == 3 ? 2 : cfg->variant == 2 ? 1 : 0;
    if ((s = install_tiling(c, t, false))) return bail(s);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(c, NBODY_ECUDA, "init synchronisation failed"));
  *out = c;
  return NBODY_OK;
}

nbody_status nbody_set_stream(nbody_ctx* c, void* stream) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  c->stream = static_cast<cudaStream_t>(stream);
  return NBODY_OK;
}

nbody_status nbody_forces(nbody_ctx* c, const double* x, const double* m, double* a, double* phi) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_forces");
  if (c->n_total == 0) return NBODY_OK;
  nbody_status s;
  if ((s = check_state_args(c, x, nullptr, m, a, false, true))) return s;
  if ((s = check_dev(c, phi, (size_t)c->n_total * sizeof(double), "phi", true))) return s;
  double* xm = const_cast<double*>(x);
  if ((s = run_centre(c, x, m, c->stream))) return s;
  if ((s = run_post(c, post_launch(c, kStage, xm, nullptr, m, a, nullptr), c->stream))) return s;
  if ((s = run_force(c, c->stream, phi != nullptr))) return s;
  return run_post(c, post_launch(c, kCombine, xm, nullptr, m, a, phi), c->stream);
}

namespace {
nbody_status step_validated(nbody_ctx* c, double* x, double* v, const double* m, double* a, int32_t a_valid,
                            int32_t n_steps, double* energy_log);
}  // namespace

nbody_status nbody_step(nbody_ctx* c, double* x, double* v, const double* m, double* a, int32_t a_valid,
                        int32_t n_steps, double* energy_log) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_step");
  if (n_steps < 0) return fail(c, NBODY_EINVAL, "n_steps < 0");
  if (n_steps > 0 && !(c->cfg.dt > 0)) return fail(c, NBODY_EINVAL, "dt must be > 0");
  if (c->n_total == 0) return NBODY_OK;
  nbody_status s;
  if ((s = check_state_args(c, x, v, m, a, true, true))) return s;
  const int every = c->cfg.energy_every;
  const int nrec = every > 0 ? n_steps / every : 0;
  if (energy_log && (s = check_dev(c, energy_log, (size_t)nrec * c->n_sys * 9 * sizeof(double), "energy_log")))
    return s;
  return step_validated(c, x, v, m, a, a_valid, n_steps, energy_log);
}

namespace {

// nbody_step after its argument checks (also the host-buffer step's path, whose
// device buffers are the context's own).
nbody_status step_validated(nbody_ctx* c, double* x, double* v, const double* m, double* a, int32_t a_valid,
                            int32_t n_steps, double* energy_log) {
  nbody_status s;
  if (!(c->cfg.flags & NBODY_FLAG_GRAPH)) return enqueue_step(c, x, v, m, a, a_valid, n_steps, energy_log, c->stream);

  // CUDA-graph replay: capture the whole call once per argument set, replay afterwards.
  const void* key[5] = {x, v, m, a, energy_log};
  const bool hit = c->gexec && c->gkey_valid == (a_valid ? 1 : 0) && c->gkey_steps == n_steps &&
                   std::equal(key, key + 5, c->gkey);
  if (!hit) {
    invalidate_graph(c);
    if (!c->cap_stream) NB_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int64_t before = c->launches;
    NB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    s = enqueue_step(c, x, v, m, a, a_valid, n_steps, energy_log, c->cap_stream);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
    c->glaunches = c->launches - before;
    c->launches = before;
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (ce != cudaSuccess) return fail(c, NBODY_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      c->gexec = nullptr;
      return fail(c, NBODY_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    }
    std::copy(key, key + 5, c->gkey);
    c->gkey_valid = a_valid ? 1 : 0;
    c->gkey_steps = n_steps;
  }
  NB_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
  c->launches += c->glaunches;
  return NBODY_OK;
}

}  // namespace

nbody_status nbody_energy(nbody_ctx* c, const double* x, const double* v, const double* m, double* out) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_energy");
  nbody_status s;
  if ((s = check_dev(c, out, (size_t)c->n_sys * 9 * sizeof(double), "out"))) return s;
  if (c->n_total == 0) {
    NB_CUDA(c, cudaMemsetAsync(out, 0, (size_t)c->n_sys * 9 * sizeof(double), c->stream));
    return NBODY_OK;
  }
  if ((s = check_state_args(c, x, v, m, nullptr, true, false))) return s;
  if ((s = ensure(c, c->a_scratch, (size_t)c->n_total * 3 * sizeof(double)))) return s;
  double* xm = const_cast<double*>(x);
  double* vm = const_cast<double*>(v);
  double* as = static_cast<double*>(c->a_scratch.p);
  if ((s = run_centre(c, x, m, c->stream))) return s;
  if ((s = run_post(c, post_launch(c, kStage, xm, vm, m, as, nullptr), c->stream))) return s;
  if ((s = run_force(c, c->stream, true))) return s;
  // the last CTA writes every system's record (systems without bodies get zeros)
  PostLaunch P = post_launch(c, kCombine | kEnergy, xm, vm, m, as, nullptr);
  P.eout = out;
  return run_post(c, P, c->stream);
}

nbody_status nbody_virial(nbody_ctx* c, const double* x, const double* v, const double* m, double* out) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_virial");
  nbody_status s;
  if ((s = check_dev(c, out, (size_t)c->n_sys * 3 * sizeof(double), "out"))) return s;
  if (c->n_total == 0) {
    NB_CUDA(c, cudaMemsetAsync(out, 0, (size_t)c->n_sys * 3 * sizeof(double), c->stream));
    return NBODY_OK;
  }
  if ((s = check_state_args(c, x, v, m, nullptr, true, false))) return s;
  if ((s = ensure(c, c->a_scratch, (size_t)c->n_total * 3 * sizeof(double)))) return s;
  double* xm = const_cast<double*>(x);
  double* vm = const_cast<double*>(v);
  double* as = static_cast<double*>(c->a_scratch.p);
  if ((s = run_centre(c, x, m, c->stream))) return s;
  if ((s = run_post(c, post_launch(c, kStage, xm, vm, m, as, nullptr), c->stream))) return s;
  if ((s = run_force(c, c->stream, false))) return s;
  PostLaunch P = post_launch(c, kCombine | kVirial, xm, vm, m, as, nullptr);
  P.vout = out;
  return run_post(c, P, c->stream);
}

nbody_status nbody_adjoint(nbody_ctx* c, const double* x0, const double* v0, const double* m, int32_t T,
                           int32_t K, const double* lam_xT, const double* lam_vT, double* g_x0, double* g_v0,
                           double* g_m) {
  return adjoint_sweep(c, x0, v0, m, T, K, lam_xT, lam_vT, g_x0, g_v0, g_m, nullptr);
}

nbody_status nbody_adjoint_params(nbody_ctx* c, const double* x0, const double* v0, const double* m, int32_t T,
                                  int32_t K, const double* lam_xT, const double* lam_vT, double* g_x0,
                                  double* g_v0, double* g_m, double* g_params) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  if (!g_params) return fail(c, NBODY_EINVAL, "g_params must be a device pointer to n_systems x 2 doubles");
  return adjoint_sweep(c, x0, v0, m, T, K, lam_xT, lam_vT, g_x0, g_v0, g_m, g_params);
}

nbody_status nbody_step_host(nbody_ctx* c, double* x, double* v, const double* m, double* a, int32_t a_valid,
                             int32_t n_steps, double* energy_log) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  NvtxRange range(c->nvtx, "nbody_step_host");
  if (c->n_total == 0) return NBODY_OK;
  if (!x || !v || !m || !a) return fail(c, NBODY_EINVAL, "x, v, m and a must be non-NULL host pointers");
  if (n_steps < 0) return fail(c, NBODY_EINVAL, "n_steps < 0");
  if (n_steps > 0 && !(c->cfg.dt > 0)) return fail(c, NBODY_EINVAL, "dt must be > 0");
  const size_t n = (size_t)c->n_total, n3b = n * 3 * sizeof(double);
  const int every = c->cfg.energy_every;
  const int nrec = (every > 0 && n_steps > 0) ? n_steps / every : 0;
  const size_t logb = (size_t)nrec * c->n_sys * 9 * sizeof(double);
  nbody_status s;
  if ((s = ensure(c, c->hx, n3b)) || (s = ensure(c, c->hv, n3b)) || (s = ensure(c, c->hm, n * sizeof(double))) ||
      (s = ensure(c, c->ha, n3b)))
    return s;
  if (energy_log && logb && (s = ensure(c, c->hlog, logb))) return s;
  cudaStream_t st = c->stream;
  double* hx = static_cast<double*>(c->hx.p);
  double* hv = static_cast<double*>(c->hv.p);
  double* hm = static_cast<double*>(c->hm.p);
  double* ha = static_cast<double*>(c->ha.p);
  double* hlog = (energy_log && logb) ? static_cast<double*>(c->hlog.p) : nullptr;
  // Mapped pinned buffers move in one copy kernel each way, read and written by
  // the GPU across the host link; any other host memory takes cudaMemcpyAsync.
  double* mx = mapped_host(x);
  double* mv = mapped_host(v);
  double* mm = mapped_host(m);
  double* ma = mapped_host(a);
  double* mlog = hlog ? mapped_host(energy_log) : nullptr;
  const bool zero_copy = mx && mv && mm && ma && (!hlog || mlog);
  const int64_t n3 = (int64_t)n * 3;
  if (zero_copy) {
    const Copy4 in{{mx, mv, mm, a_valid ? ma : nullptr}, {hx, hv, hm, ha}, {n3, n3, (int64_t)n, a_valid ? n3 : 0}};
    NB_CUDA(c, launch_copy4(in, c->sm_count, st));
    ++c->launches;
  } else {
    NB_CUDA(c, cudaMemcpyAsync(hx, x, n3b, cudaMemcpyHostToDevice, st));
    NB_CUDA(c, cudaMemcpyAsync(hv, v, n3b, cudaMemcpyHostToDevice, st));
    NB_CUDA(c, cudaMemcpyAsync(hm, m, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (a_valid) NB_CUDA(c, cudaMemcpyAsync(ha, a, n3b, cudaMemcpyHostToDevice, st));
  }
  s = step_validated(c, hx, hv, hm, ha, a_valid, n_steps, hlog);  // the context's own buffers
  if (s) return s;
  if (zero_copy) {
    const Copy4 out{{hx, hv, ha, hlog}, {mx, mv, ma, mlog}, {n3, n3, n3, hlog ? (int64_t)(logb / sizeof(double)) : 0}};
    NB_CUDA(c, launch_copy4(out, c->sm_count, st));
    ++c->launches;
  } else {
    NB_CUDA(c, cudaMemcpyAsync(x, hx, n3b, cudaMemcpyDeviceToHost, st));
    NB_CUDA(c, cudaMemcpyAsync(v, hv, n3b, cudaMemcpyDeviceToHost, st));
    NB_CUDA(c, cudaMemcpyAsync(a, ha, n3b, cudaMemcpyDeviceToHost, st));
    if (hlog) NB_CUDA(c, cudaMemcpyAsync(energy_log, hlog, logb, cudaMemcpyDeviceToHost, st));
  }
  return nbody_sync(c);
}

nbody_status nbody_sync(nbody_ctx* c) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  // the status word rides on the stream into pinned memory: one wait, no second round trip
  NB_CUDA(c, cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  const unsigned st = *c->h_status;
  if (st) NB_CUDA(c, cudaMemset(c->status, 0, sizeof(unsigned)));
  if (st & kFlagIndex) return fail(c, NBODY_EINTERNAL, "a device-side index check failed (NBODY_DEBUG build)");
  if (st & kFlagTimeout) return fail(c, NBODY_ETIMEOUT, "a bounded device-side wait gave up");
  if ((st & kFlagNonFinite) && !(c->cfg.flags & NBODY_FLAG_NOCHECK))
    return fail(c, NBODY_ENONFINITE, "non-finite acceleration, potential or gradient produced");
  return NBODY_OK;
}

nbody_status nbody_get_tuning(const nbody_ctx* c, int32_t* block, int32_t* ipt, int32_t* jtile, int32_t* slice,
                              int32_t* n_ctas, int32_t* variant) {
  if (!c) return NBODY_EINVAL;
  if (block) *block = c->ft.block;
  if (ipt) *ipt = c->ft.ipt;
  if (jtile) *jtile = c->ft.jtile;
  if (slice) *slice = c->ft.slice;
  if (n_ctas) *n_ctas = c->ft.n_ctas;
  if (variant) *variant = c->ft.variant + 1;
  return NBODY_OK;
}

nbody_status nbody_get_slicing(const nbody_ctx* c, int32_t* tail, int32_t* n_items, int32_t* max_slices) {
  if (!c) return NBODY_EINVAL;
  if (tail) *tail = c->ft.tail;
  if (n_items) *n_items = c->n_items;
  if (max_slices) *max_slices = c->max_slices;
  return NBODY_OK;
}

nbody_status nbody_profile(nbody_ctx* c, int32_t enable) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  if (enable) {
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& u : c->ev_used) c->ev_pool.push_back(u.second.first), c->ev_pool.push_back(u.second.second);
    c->ev_used.clear();
  }
  c->profiling = enable != 0;
  return NBODY_OK;
}

nbody_status nbody_kernel_time(nbody_ctx* c, int32_t which, double* ms_total, int64_t* launches) {
  if (!c) return fail(nullptr, NBODY_EINVAL, "ctx is NULL");
  if (which != 0 && which != 1) return fail(c, NBODY_EINVAL, "which must be 0 (force) or 1 (VJP)");
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  int64_t k = 0;
  for (auto& u : c->ev_used) {
    if (u.first != which) continue;
    float ms = 0.f;
    NB_CUDA(c, cudaEventElapsedTime(&ms, u.second.first, u.second.second));
    tot += ms, ++k;
  }
  if (ms_total) *ms_total = tot;
  if (launches) *launches = k;
  return NBODY_OK;
}

void nbody_destroy(nbody_ctx* c) { free_ctx(c); }

}  // extern "C"
