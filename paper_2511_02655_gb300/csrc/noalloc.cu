// nbody_forces_noalloc: an entry point that computes the mixed-precision
// all-pairs forces of one system without allocating any memory.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// forces, e.g. a host program that runs under a fixed device-memory budget
// handed out by a surrounding framework, a plugin whose host only passes it
// ready-made device buffers, or a caller that must not trigger the allocator
// (and its implicit synchronisation) in the middle of its own work. The
// regular path needs an nbody_ctx, and creating one allocates the context's
// staging, partial-sum and work-list buffers; this entry point takes no
// context and allocates nothing.
//
// Its scratch (the float32 staging copy of the bodies, the float32 remainders
// the near-pair refinement reads, and the staging origin) lives in one
// file-scope __device__ array of fixed size, held on every GPU that loads the
// library's module until the process exits. Host code cannot use the array's
// name as a device address (on the host it names a host-side stand-in), so
// the device address is looked up with cudaGetSymbolAddress once per device,
// on the first call made with that device current, and passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/nbody.h"
#include "nbody_internal.h"
#include "pair_common.cuh"

namespace nbody {
void set_global_error_text(const char* msg);  // capi.cu
}

namespace {

constexpr int64_t kMaxBodies = NBODY_NOALLOC_MAX_BODIES;
constexpr int kThreads = 256;  // threads per CTA of the force kernel
constexpr int kIpt = 2;        // i-bodies per thread
constexpr int kTile = 256;     // j-bodies per shared-memory tile
constexpr int kSub = 32;       // j-bodies per near-pair check
constexpr int kHeaderBytes = 256;
constexpr size_t kStageBytes = sizeof(float4) * (size_t)kMaxBodies;
constexpr size_t kScratchBytes = kHeaderBytes + 2 * kStageBytes;
// Near-pair refinement radius: 4 softening lengths, as in the context path.
constexpr double kNearRadiusEps = 4.0;

// Layout: [0, 256) header (staging origin, 3 doubles); then float4 staging
// entries (x - c, m) [kMaxBodies]; then float4 remainders (x - c) - hi [kMaxBodies].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

nbody_status fail(nbody_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  nbody::set_global_error_text(buf);
  return s;
}

// Device memory of the current device holding at least `bytes` from p
// (the extent is checked where the driver can report the allocation's range).
nbody_status check_dev_ptr(const void* p, size_t bytes, int dev, const char* name, bool nullable) {
  if (!p) return nullable ? NBODY_OK : fail(NBODY_EINVAL, "nbody_forces_noalloc: %s is NULL", name);
  if (reinterpret_cast<uintptr_t>(p) % 8 != 0)
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: %s is not 8-byte aligned", name);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: %s is not a CUDA pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: %s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: %s is on device %d, current device is %d", name, at.device, dev);
  size_t avail = 0;
  if (!nbody::allocation_holds(p, bytes, &avail))
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: %s needs %zu bytes, its allocation holds %zu from that address",
                name, bytes, avail);
  return NBODY_OK;
}

// Staging origin = mass-weighted mean position (plain mean if the total mass is
// not positive), written to the scratch header. One CTA: this entry point
// trades speed for needing no reduction buffers.
__global__ void __launch_bounds__(256) k_na_centre(const double* x, const double* m, int n, unsigned char* scratch) {
  __shared__ double red[8][7];
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n; i += 256) {
    const double mi = m[i];
    const double x0 = x[3 * (int64_t)i], x1 = x[3 * (int64_t)i + 1], x2 = x[3 * (int64_t)i + 2];
    v[0] += mi * x0, v[1] += mi * x1, v[2] += mi * x2, v[3] += mi, v[4] += x0, v[5] += x1, v[6] += x2;
  }
#pragma unroll
  for (int k = 0; k < 7; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 7; ++k) red[threadIdx.x >> 5][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int w = 0; w < 8; ++w)
      for (int k = 0; k < 7; ++k) s[k] += red[w][k];
    double c0 = 0, c1 = 0, c2 = 0;
    if (s[3] > 0 && isfinite(s[3])) {
      c0 = s[0] / s[3], c1 = s[1] / s[3], c2 = s[2] / s[3];
    } else if (n > 0) {
      c0 = s[4] / n, c1 = s[5] / n, c2 = s[6] / n;
    }
    if (!(isfinite(c0) && isfinite(c1) && isfinite(c2))) c0 = c1 = c2 = 0;
    double* c = reinterpret_cast<double*>(scratch);
    c[0] = c0, c[1] = c1, c[2] = c2;
  }
}

__global__ void __launch_bounds__(256) k_na_stage(const double* x, const double* m, int n, unsigned char* scratch) {
  const double* c = reinterpret_cast<const double*>(scratch);
  float4* st = reinterpret_cast<float4*>(scratch + kHeaderBytes);
  float4* lo = reinterpret_cast<float4*>(scratch + kHeaderBytes + kStageBytes);
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
    const double X = x[3 * (int64_t)i] - c[0], Y = x[3 * (int64_t)i + 1] - c[1], Z = x[3 * (int64_t)i + 2] - c[2];
    const float hx = (float)X, hy = (float)Y, hz = (float)Z;
    st[i] = make_float4(hx, hy, hz, (float)m[i]);
    lo[i] = make_float4((float)(X - (double)hx), (float)(Y - (double)hy), (float)(Z - (double)hz), 0.f);
  }
}

template <bool MASK>
__device__ __forceinline__ void na_pair(const float4 q, const float xi, const float yi, const float zi,
                                        const float eps2, float& ax, float& ay, float& az, float& pp, float& mn,
                                        const bool self) {
  const float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  mn = fminf(mn, r2);
  float inv = nbody::rsq_approx(r2);
  if (MASK) inv = self ? 0.f : inv;
  const float ms = q.w * inv;
  const float w = ms * (inv * inv);
  ax = fmaf(dx, w, ax), ay = fmaf(dy, w, ay), az = fmaf(dz, w, az);
  pp += ms;
}

// One CTA per i-tile of kThreads * kIpt bodies, each against all n j-bodies;
// writes a and phi directly (no partial-sum buffer). The pair arithmetic is
// that of the context path's scalar mixed kernel, near-pair refinement
// included: every pair folds s^2 into a running minimum, and a sub-block of
// kSub j-bodies whose minimum fell below r2c is rescanned, each near pair's
// contribution replaced by the one from the separation refined with the
// staged remainders.
__global__ void __launch_bounds__(kThreads) k_na_force(const unsigned char* scratch, int n, float eps2, float r2c,
                                                       double G, double* a, double* phi) {
  __shared__ __align__(16) float4 tile[kTile];
  const float4* st = reinterpret_cast<const float4*>(scratch + kHeaderBytes);
  const float4* lo = reinterpret_cast<const float4*>(scratch + kHeaderBytes + kStageBytes);
  const int i0 = blockIdx.x * kThreads * kIpt;
  float xi[kIpt], yi[kIpt], zi[kIpt], hx[kIpt], hy[kIpt], hz[kIpt], hp[kIpt], lx[kIpt], ly[kIpt], lz[kIpt],
      lp[kIpt];
  int ig[kIpt];
#pragma unroll
  for (int r = 0; r < kIpt; ++r) {
    ig[r] = i0 + (int)threadIdx.x + r * kThreads;
    const float4 q = ig[r] < n ? st[ig[r]] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = q.x, yi[r] = q.y, zi[r] = q.z;
    hx[r] = hy[r] = hz[r] = hp[r] = lx[r] = ly[r] = lz[r] = lp[r] = 0.f;
  }
  const int i_end = min(n, i0 + kThreads * kIpt);
  for (int jt = 0; jt < n; jt += kTile) {
    const int nj = min(kTile, n - jt);
    __syncthreads();
    if ((int)threadIdx.x < nj) tile[threadIdx.x] = st[jt + threadIdx.x];
    __syncthreads();
    float ax[kIpt], ay[kIpt], az[kIpt], pp[kIpt];
#pragma unroll
    for (int r = 0; r < kIpt; ++r) ax[r] = ay[r] = az[r] = pp[r] = 0.f;
    const bool diag = jt < i_end && i0 < jt + nj;
    for (int jb = 0; jb < nj; jb += kSub) {
      const int je = min(nj, jb + kSub);
      float mn = 3.0e38f;
      if (diag) {
        for (int j = jb; j < je; ++j)
#pragma unroll
          for (int r = 0; r < kIpt; ++r)
            na_pair<true>(tile[j], xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], mn, jt + j == ig[r]);
      } else {
#pragma unroll 8
        for (int j = jb; j < je; ++j)
#pragma unroll
          for (int r = 0; r < kIpt; ++r)
            na_pair<false>(tile[j], xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pp[r], mn, false);
      }
      if (mn < r2c) {
        for (int j = jb; j < je; ++j)
#pragma unroll
          for (int r = 0; r < kIpt; ++r)
            nbody::correct_pair<0>(tile[j], jt + j, ig[r], n, xi[r], yi[r], zi[r], eps2, r2c, lo, ax[r], ay[r],
                                   az[r], pp[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kIpt; ++r) {
      nbody::two_sum_acc(hx[r], lx[r], ax[r]);
      nbody::two_sum_acc(hy[r], ly[r], ay[r]);
      nbody::two_sum_acc(hz[r], lz[r], az[r]);
      nbody::two_sum_acc(hp[r], lp[r], pp[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < kIpt; ++r) {
    if (ig[r] >= n) continue;
    a[3 * (int64_t)ig[r] + 0] = G * ((double)hx[r] + (double)lx[r]);
    a[3 * (int64_t)ig[r] + 1] = G * ((double)hy[r] + (double)ly[r]);
    a[3 * (int64_t)ig[r] + 2] = G * ((double)hz[r] + (double)lz[r]);
    if (phi) phi[ig[r]] = -G * ((double)hp[r] + (double)lp[r]);
  }
}

}  // namespace

extern "C" nbody_status nbody_forces_noalloc(const double* x, const double* m, int64_t n, double G, double eps,
                                             double* a, double* phi, void* cuda_stream) {
  if (n < 0 || n > kMaxBodies)
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: n = %lld is outside [0, %lld] (NBODY_NOALLOC_MAX_BODIES)",
                (long long)n, (long long)kMaxBodies);
  if (!std::isfinite(G) || !std::isfinite(eps) || eps < 0)
    return fail(NBODY_EINVAL, "nbody_forces_noalloc: G must be finite and eps finite and >= 0");
  if (n == 0) return NBODY_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(NBODY_EUNSUPPORTED, "nbody_forces_noalloc: no usable current CUDA device");
  }
  nbody_status s;
  const size_t n3b = (size_t)n * 3 * sizeof(double), n1b = (size_t)n * sizeof(double);
  if ((s = check_dev_ptr(x, n3b, dev, "x", false)) || (s = check_dev_ptr(m, n1b, dev, "m", false)) ||
      (s = check_dev_ptr(a, n3b, dev, "a", false)) || (s = check_dev_ptr(phi, n1b, dev, "phi", true)))
    return s;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(NBODY_ECUDA, "nbody_forces_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                    cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  const int ni = (int)n;
  k_na_centre<<<1, 256, 0, st>>>(x, m, ni, sp);
  k_na_stage<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(x, m, ni, sp);
  const float r2c = (float)(kNearRadiusEps * kNearRadiusEps * eps * eps);  // 0 for eps = 0: no refinement
  k_na_force<<<(unsigned)((n + kThreads * kIpt - 1) / (kThreads * kIpt)), kThreads, 0, st>>>(
      sp, ni, (float)(eps * eps), r2c, G, a, phi);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NBODY_ECUDA, "nbody_forces_noalloc: launch failed: %s", cudaGetErrorString(e));
  return NBODY_OK;
}
