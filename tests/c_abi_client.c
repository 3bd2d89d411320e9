/*
 * A plain C client of the libnbody C ABI, used by tests/test_gpu_c_abi.py.
 * It allocates device memory with the CUDA runtime, runs forces, KDK steps
 * and the energy reduction through include/nbody.h, checks every status code,
 * and writes the inputs and results to a binary file for the test to compare
 * against the CPU oracle.
 *
 * usage: c_abi_client <n> <precision 0|1> <out-file>
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "nbody.h"

#define CHECK_NB(call)                                                                     \
  do {                                                                                     \
    nbody_status s_ = (call);                                                              \
    if (s_ != NBODY_OK) {                                                                  \
      fprintf(stderr, "%s -> %d: %s\n", #call, (int)s_, nbody_last_error(ctx));            \
      return 2;                                                                            \
    }                                                                                      \
  } while (0)
#define CHECK_CU(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      fprintf(stderr, "%s -> %s\n", #call, cudaGetErrorString(e_));                        \
      return 3;                                                                            \
    }                                                                                      \
  } while (0)

/* deterministic pseudo-random numbers in [0, 1) (64-bit LCG, top 53 bits) */
static uint64_t lcg = 0x2545F4914F6CDD1Dull;
static double u01(void) {
  lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(lcg >> 11) * (1.0 / 9007199254740992.0);
}

int main(int argc, char** argv) {
  nbody_ctx* ctx = NULL;
  if (argc != 4) return 1;
  const int64_t n = atoll(argv[1]);
  const int prec = atoi(argv[2]);
  const size_t n3 = (size_t)n * 3;
  double* x = (double*)malloc(n3 * sizeof(double));
  double* v = (double*)malloc(n3 * sizeof(double));
  double* m = (double*)malloc((size_t)n * sizeof(double));
  double* a = (double*)malloc(n3 * sizeof(double));
  double* a1 = (double*)malloc(n3 * sizeof(double));
  double* x1 = (double*)malloc(n3 * sizeof(double));
  double e[9];
  if (!x || !v || !m || !a || !a1 || !x1) return 4;
  for (size_t k = 0; k < n3; ++k) x[k] = 2.0 * u01() - 1.0, v[k] = 0.2 * (2.0 * u01() - 1.0);
  for (int64_t i = 0; i < n; ++i) m[i] = (0.5 + u01()) / (double)n;

  nbody_config cfg = {0};
  cfg.G = 1.0;
  cfg.eps = 0.02;
  cfg.dt = 1e-3;
  cfg.precision = prec;
  cfg.energy_every = 0;
  cfg.lj_epsilon = 1.0;
  cfg.lj_sigma = 1.0;
  const int64_t offsets[2] = {0, n};
  CHECK_NB(nbody_init(&ctx, &cfg, 1, offsets, NULL));

  double *dx, *dv, *dm, *da, *de, *dphi;
  CHECK_CU(cudaMalloc((void**)&dx, n3 * sizeof(double)));
  CHECK_CU(cudaMalloc((void**)&dv, n3 * sizeof(double)));
  CHECK_CU(cudaMalloc((void**)&dm, (size_t)n * sizeof(double)));
  CHECK_CU(cudaMalloc((void**)&da, n3 * sizeof(double)));
  CHECK_CU(cudaMalloc((void**)&dphi, (size_t)n * sizeof(double)));
  CHECK_CU(cudaMalloc((void**)&de, 9 * sizeof(double)));
  CHECK_CU(cudaMemcpy(dx, x, n3 * sizeof(double), cudaMemcpyHostToDevice));
  CHECK_CU(cudaMemcpy(dv, v, n3 * sizeof(double), cudaMemcpyHostToDevice));
  CHECK_CU(cudaMemcpy(dm, m, (size_t)n * sizeof(double), cudaMemcpyHostToDevice));

  /* a host pointer must be refused before anything is launched */
  if (nbody_forces(ctx, x, dm, da, NULL) != NBODY_EINVAL) {
    fprintf(stderr, "host pointer was not rejected\n");
    return 5;
  }
  CHECK_NB(nbody_forces(ctx, dx, dm, da, dphi));
  CHECK_NB(nbody_sync(ctx));
  CHECK_CU(cudaMemcpy(a, da, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  CHECK_NB(nbody_energy(ctx, dx, dv, dm, de));
  CHECK_NB(nbody_step(ctx, dx, dv, dm, da, 1, 5, NULL));
  CHECK_NB(nbody_sync(ctx));
  CHECK_CU(cudaMemcpy(x1, dx, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  CHECK_CU(cudaMemcpy(a1, da, n3 * sizeof(double), cudaMemcpyDeviceToHost));
  CHECK_CU(cudaMemcpy(e, de, 9 * sizeof(double), cudaMemcpyDeviceToHost));
  int32_t block = 0, ipt = 0, jtile = 0, slice = 0, ctas = 0, variant = 0;
  CHECK_NB(nbody_get_tuning(ctx, &block, &ipt, &jtile, &slice, &ctas, &variant));
  const int64_t launches = nbody_launch_count(ctx);
  nbody_destroy(ctx);
  ctx = NULL;

  /* the allocation-free entry point on the original positions */
  double* ana = (double*)malloc(n3 * sizeof(double));
  CHECK_CU(cudaMemcpy(dx, x, n3 * sizeof(double), cudaMemcpyHostToDevice));
  CHECK_NB(nbody_forces_noalloc(dx, dm, n, 1.0, 0.02, da, NULL, NULL));
  CHECK_CU(cudaDeviceSynchronize());
  CHECK_CU(cudaMemcpy(ana, da, n3 * sizeof(double), cudaMemcpyDeviceToHost));

  FILE* f = fopen(argv[3], "wb");
  if (!f) return 6;
  fwrite(x, sizeof(double), n3, f);
  fwrite(v, sizeof(double), n3, f);
  fwrite(m, sizeof(double), (size_t)n, f);
  fwrite(a, sizeof(double), n3, f);
  fwrite(x1, sizeof(double), n3, f);
  fwrite(a1, sizeof(double), n3, f);
  fwrite(e, sizeof(double), 9, f);
  fwrite(ana, sizeof(double), n3, f);
  fclose(f);
  printf("ok n=%lld prec=%d tuning=%d,%d,%d,%d,%d,%d launches=%lld version=%d\n", (long long)n, prec, block, ipt,
         jtile, slice, ctas, variant, (long long)launches, nbody_version());
  cudaFree(dx), cudaFree(dv), cudaFree(dm), cudaFree(da), cudaFree(dphi), cudaFree(de);
  free(x), free(v), free(m), free(a), free(a1), free(x1), free(ana);
  return 0;
}
