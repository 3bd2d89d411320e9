/*
 * CPU ORACLE for the softened-gravity N-body hot path -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. The GPU library shares no code with it.
 *
 * Everything here is plain FP64 C with straightforward loops, written from
 * the method's definition so that it can be checked by eye:
 *
 *   d_ij   = x_j - x_i,  s_ij^2 = |d_ij|^2 + eps^2          (Plummer softening)
 *   a_i    =  G sum_{j != i} m_j d_ij / s_ij^3              (all-pairs force,
 *   phi_i  = -G sum_{j != i} m_j / s_ij                      "N_p^2 operations", Sec. V-B)
 *
 *   KDK leapfrog ("Verlet half-stepping", Sec. II-A), one force evaluation per
 *   step, the end-of-step force reused as the next step's start force:
 *     v <- v + dt/2 a(x);  x <- x + dt v;  a <- a(x);  v <- v + dt/2 a
 *
 *   Global reductions (the system's total energy, Sec. VI):
 *     K = 1/2 sum m |v|^2,  U = -G sum_{i<j} m_i m_j / s_ij,  E = K + U,
 *     P = sum m v,          L = sum m x cross v
 *
 *   Adjoint of the KDK map (reverse-mode, no approximation): with w_k = dL/da_k,
 *     J(d)   = I / s^3 - 3 d d^T / s^5               (derivative of d / s^3)
 *     gx_k   = G sum_{j != k} J(d_kj) (m_k w_j - m_j w_k)
 *     gm_j   = G sum_{i != j} w_i . d_ij / s_ij^3
 *   and for the two model parameters (a depends on G linearly and on eps
 *   through s^2 = |d|^2 + eps^2):
 *     dL/dG   = sum_k w_k . sum_{j != k} m_j d_kj / s_kj^3
 *     dL/deps = sum_k w_k . (-3 G eps) sum_{j != k} m_j d_kj / s_kj^5
 *
 * The pair law (softened Newtonian gravity) replaces the paper's Lennard-Jones
 * law (Eq. 1); the all-pairs structure, the Verlet half-step integrator and the
 * energy reduction are the paper's.
 *
 * Summation order: j = 0 .. N-1 for every body; pair sums for U and the
 * reductions use Neumaier compensated summation so that the oracle is the
 * accuracy anchor. Row loops may run on several threads (each body's sum is
 * still evaluated in the order above). Compile with -ffp-contract=off so that
 * no multiply-add is fused, on any host.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* threading helper: run fn(lo, hi, arg) over [0, n) split in contiguous rows */

typedef void (*row_fn)(int64_t lo, int64_t hi, void* arg);

typedef struct {
  row_fn fn;
  void* arg;
  int64_t lo, hi;
} row_job;

static void* row_job_main(void* p) {
  row_job* j = (row_job*)p;
  j->fn(j->lo, j->hi, j->arg);
  return NULL;
}

int oracle_default_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void parallel_rows(int64_t n, int nthreads, row_fn fn, void* arg) {
  if (nthreads <= 0) nthreads = oracle_default_threads();
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads <= 1) {
    fn(0, n, arg);
    return;
  }
  pthread_t th[256];
  row_job jobs[256];
  int started[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].arg = arg;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    started[t] = pthread_create(&th[t], NULL, row_job_main, &jobs[t]) == 0;
    if (!started[t]) row_job_main(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(th[t], NULL);
}

/* Neumaier (improved Kahan-Babuska) compensated sum */
typedef struct {
  double s, c;
} csum;

static void csum_add(csum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

static double csum_get(const csum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* forces: the direct sum, one body at a time                                */

static void body_force(int64_t n, const double* x, const double* m, double G, double eps, int64_t i,
                       double* ai, double* phii) {
  double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
  const double e2 = eps * eps;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double dx = x[3 * j + 0] - x[3 * i + 0];
    double dy = x[3 * j + 1] - x[3 * i + 1];
    double dz = x[3 * j + 2] - x[3 * i + 2];
    double s2 = dx * dx + dy * dy + dz * dz + e2;
    double inv_s = 1.0 / sqrt(s2);
    double inv_s3 = inv_s * inv_s * inv_s;
    ax += m[j] * dx * inv_s3;
    ay += m[j] * dy * inv_s3;
    az += m[j] * dz * inv_s3;
    p -= m[j] * inv_s;
  }
  ai[0] = G * ax;
  ai[1] = G * ay;
  ai[2] = G * az;
  if (phii) *phii = G * p;
}

typedef struct {
  int64_t n;
  const double *x, *m;
  double G, eps;
  const int64_t* idx; /* NULL: all bodies */
  double *a, *phi;
} force_args;

static void force_rows(int64_t lo, int64_t hi, void* p) {
  force_args* f = (force_args*)p;
  for (int64_t r = lo; r < hi; ++r) {
    int64_t i = f->idx ? f->idx[r] : r;
    body_force(f->n, f->x, f->m, f->G, f->eps, i, f->a + 3 * r, f->phi ? f->phi + r : NULL);
  }
}

/* a [n,3] and phi [n] (phi may be NULL) for all bodies. */
int oracle_forces(int64_t n, const double* x, const double* m, double G, double eps, double* a, double* phi,
                  int nthreads) {
  if (n < 0 || (n > 0 && (!x || !m || !a))) return 1;
  force_args f = {n, x, m, G, eps, NULL, a, phi};
  parallel_rows(n, nthreads, force_rows, &f);
  return 0;
}

/* a [k,3] and phi [k] for the bodies idx[0..k-1] only, each against all n. */
int oracle_forces_at(int64_t n, const double* x, const double* m, double G, double eps, const int64_t* idx,
                     int64_t k, double* a, double* phi, int nthreads) {
  if (n < 0 || k < 0 || (k > 0 && (!x || !m || !a || !idx))) return 1;
  for (int64_t r = 0; r < k; ++r)
    if (idx[r] < 0 || idx[r] >= n) return 1;
  force_args f = {n, x, m, G, eps, idx, a, phi};
  parallel_rows(k, nthreads, force_rows, &f);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* global reductions                                                          */

typedef struct {
  int64_t n;
  const double *x, *m;
  double G, eps;
  double* row_u; /* per-row pair sums, U_i = -G sum_{j>i} m_i m_j / s_ij */
} pot_args;

static void pot_rows(int64_t lo, int64_t hi, void* p) {
  pot_args* f = (pot_args*)p;
  const double e2 = f->eps * f->eps;
  for (int64_t i = lo; i < hi; ++i) {
    csum u = {0.0, 0.0};
    for (int64_t j = i + 1; j < f->n; ++j) {
      double dx = f->x[3 * j + 0] - f->x[3 * i + 0];
      double dy = f->x[3 * j + 1] - f->x[3 * i + 1];
      double dz = f->x[3 * j + 2] - f->x[3 * i + 2];
      double s = sqrt(dx * dx + dy * dy + dz * dz + e2);
      csum_add(&u, -f->G * f->m[i] * f->m[j] / s);
    }
    f->row_u[i] = csum_get(&u);
  }
}

/* out[9] = {E, K, U, Px, Py, Pz, Lx, Ly, Lz}; U from the pair sum over i < j. */
int oracle_energy(int64_t n, const double* x, const double* v, const double* m, double G, double eps, double* out,
                  int nthreads) {
  if (n < 0 || !out || (n > 0 && (!x || !v || !m))) return 1;
  double* row_u = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!row_u) return 2;
  pot_args f = {n, x, m, G, eps, row_u};
  parallel_rows(n, nthreads, pot_rows, &f);
  csum K = {0, 0}, U = {0, 0}, P[3] = {{0, 0}, {0, 0}, {0, 0}}, L[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + 3 * i;
    const double* vi = v + 3 * i;
    csum_add(&K, 0.5 * m[i] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
    csum_add(&U, row_u[i]);
    for (int c = 0; c < 3; ++c) csum_add(&P[c], m[i] * vi[c]);
    csum_add(&L[0], m[i] * (xi[1] * vi[2] - xi[2] * vi[1]));
    csum_add(&L[1], m[i] * (xi[2] * vi[0] - xi[0] * vi[2]));
    csum_add(&L[2], m[i] * (xi[0] * vi[1] - xi[1] * vi[0]));
  }
  free(row_u);
  out[1] = csum_get(&K);
  out[2] = csum_get(&U);
  out[0] = out[1] + out[2];
  for (int c = 0; c < 3; ++c) {
    out[3 + c] = csum_get(&P[c]);
    out[6 + c] = csum_get(&L[c]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* KDK leapfrog                                                               */

/*
 * Advances (x, v) by n_steps KDK steps in place. a [n,3] holds a(x) on entry
 * when a_valid != 0 (else it is computed first) and a(x_final) on exit.
 * If energy_every > 0 and energy_log != NULL, after every energy_every-th step
 * the 9 reductions of oracle_energy are appended to energy_log.
 */
int oracle_kdk(int64_t n, double* x, double* v, const double* m, double G, double eps, double dt, int n_steps,
               double* a, int a_valid, int energy_every, double* energy_log, int nthreads) {
  if (n < 0 || n_steps < 0 || (n > 0 && (!x || !v || !m || !a))) return 1;
  if (!a_valid) oracle_forces(n, x, m, G, eps, a, NULL, nthreads);
  int rec = 0;
  for (int s = 0; s < n_steps; ++s) {
    for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * a[k];
    for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];
    oracle_forces(n, x, m, G, eps, a, NULL, nthreads);
    for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * a[k];
    if (energy_every > 0 && energy_log && (s + 1) % energy_every == 0) {
      int rc = oracle_energy(n, x, v, m, G, eps, energy_log + 9 * rec, nthreads);
      if (rc) return rc;
      ++rec;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* adjoint                                                                    */

typedef struct {
  int64_t n;
  const double *x, *m, *w;
  double G, eps;
  double *gx, *gm;
} vjp_args;

static void vjp_rows(int64_t lo, int64_t hi, void* p) {
  vjp_args* f = (vjp_args*)p;
  const double e2 = f->eps * f->eps;
  for (int64_t k = lo; k < hi; ++k) {
    double g[3] = {0.0, 0.0, 0.0};
    double gm = 0.0;
    for (int64_t j = 0; j < f->n; ++j) {
      if (j == k) continue;
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = f->x[3 * j + c] - f->x[3 * k + c]; /* d_kj = x_j - x_k */
      double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + e2;
      double inv_s = 1.0 / sqrt(s2);
      double inv_s3 = inv_s * inv_s * inv_s;
      double inv_s5 = inv_s3 * inv_s * inv_s;
      /* u = m_k w_j - m_j w_k ; J(d) u = u / s^3 - 3 d (d . u) / s^5 */
      double u[3];
      for (int c = 0; c < 3; ++c) u[c] = f->m[k] * f->w[3 * j + c] - f->m[j] * f->w[3 * k + c];
      double du = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
      for (int c = 0; c < 3; ++c) g[c] += u[c] * inv_s3 - 3.0 * d[c] * du * inv_s5;
      /* gm_k = sum_{i != k} w_i . d_ik / s^3 with d_ik = x_k - x_i = -d_kj (i = j) */
      double wd = f->w[3 * j + 0] * d[0] + f->w[3 * j + 1] * d[1] + f->w[3 * j + 2] * d[2];
      gm -= wd * inv_s3;
    }
    for (int c = 0; c < 3; ++c) f->gx[3 * k + c] = f->G * g[c];
    f->gm[k] = f->G * gm;
  }
}

/* Vector-Jacobian product of the force map a(x, m) with w [n,3]: gx [n,3], gm [n]. */
int oracle_force_vjp(int64_t n, const double* x, const double* m, const double* w, double G, double eps, double* gx,
                     double* gm, int nthreads) {
  if (n < 0 || (n > 0 && (!x || !m || !w || !gx || !gm))) return 1;
  vjp_args f = {n, x, m, w, G, eps, gx, gm};
  parallel_rows(n, nthreads, vjp_rows, &f);
  return 0;
}

typedef struct {
  int64_t n;
  const double *x, *m, *w;
  double G, eps;
  double* rows; /* [n][2]: per-body terms of dL/dG and dL/deps */
} pvjp_args;

static void param_vjp_rows(int64_t lo, int64_t hi, void* p) {
  pvjp_args* f = (pvjp_args*)p;
  const double e2 = f->eps * f->eps;
  for (int64_t k = lo; k < hi; ++k) {
    double da_dG[3] = {0.0, 0.0, 0.0}, da_deps[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < f->n; ++j) {
      if (j == k) continue;
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = f->x[3 * j + c] - f->x[3 * k + c];
      double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + e2;
      double inv_s = 1.0 / sqrt(s2);
      double inv_s3 = inv_s * inv_s * inv_s;
      double inv_s5 = inv_s3 * inv_s * inv_s;
      for (int c = 0; c < 3; ++c) {
        da_dG[c] += f->m[j] * d[c] * inv_s3;                          /* d a_k / dG */
        da_deps[c] += -3.0 * f->G * f->eps * f->m[j] * d[c] * inv_s5; /* d a_k / d eps */
      }
    }
    const double* wk = f->w + 3 * k;
    f->rows[2 * k + 0] = wk[0] * da_dG[0] + wk[1] * da_dG[1] + wk[2] * da_dG[2];
    f->rows[2 * k + 1] = wk[0] * da_deps[0] + wk[1] * da_deps[1] + wk[2] * da_deps[2];
  }
}

/* out[0] = sum_k w_k . d a_k / dG, out[1] = sum_k w_k . d a_k / d eps. */
int oracle_param_vjp(int64_t n, const double* x, const double* m, const double* w, double G, double eps, double* out,
                     int nthreads) {
  if (n < 0 || !out || (n > 0 && (!x || !m || !w))) return 1;
  out[0] = out[1] = 0.0;
  if (n == 0) return 0;
  double* rows = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  if (!rows) return 2;
  pvjp_args f = {n, x, m, w, G, eps, rows};
  parallel_rows(n, nthreads, param_vjp_rows, &f);
  csum acc[2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t k = 0; k < n; ++k)
    for (int c = 0; c < 2; ++c) csum_add(&acc[c], rows[2 * k + c]);
  out[0] = csum_get(&acc[0]);
  out[1] = csum_get(&acc[1]);
  free(rows);
  return 0;
}

/*
 * Gradients of a loss L(x_T, v_T) with respect to x0, v0 and m through n_steps
 * KDK steps, given lam_xT = dL/dx_T and lam_vT = dL/dv_T. The forward
 * trajectory is stored in full (no checkpointing) and each step is reversed in
 * the order kick(x') -> drift -> kick(x):
 *   lam_vh  = lam_v';  lam_x' += dt/2 gx(x'; lam_v');  g_m += dt/2 gm(x'; lam_v')
 *   lam_vh += dt lam_x'
 *   lam_v   = lam_vh;  lam_x   = lam_x' + dt/2 gx(x; lam_vh);  g_m += dt/2 gm(x; lam_vh)
 */
static int adjoint_sweep(int64_t n, const double* x0, const double* v0, const double* m, double G, double eps,
                         double dt, int n_steps, const double* lam_xT, const double* lam_vT, double* g_x0,
                         double* g_v0, double* g_m, double* g_params, int nthreads) {
  if (n < 0 || n_steps < 0) return 1;
  if (n == 0) return 0;
  if (!x0 || !v0 || !m || !lam_xT || !lam_vT || !g_x0 || !g_v0 || !g_m) return 1;
  const size_t sz = (size_t)(3 * n);
  double* traj = (double*)malloc(sizeof(double) * sz * (size_t)(n_steps + 1));
  double* v = (double*)malloc(sizeof(double) * sz);
  double* a = (double*)malloc(sizeof(double) * sz);
  double* gx = (double*)malloc(sizeof(double) * sz);
  double* gmv = (double*)malloc(sizeof(double) * (size_t)n);
  double* lam_vh = (double*)malloc(sizeof(double) * sz);
  if (!traj || !v || !a || !gx || !gmv || !lam_vh) {
    free(traj), free(v), free(a), free(gx), free(gmv), free(lam_vh);
    return 2;
  }
  memcpy(traj, x0, sizeof(double) * sz);
  memcpy(v, v0, sizeof(double) * sz);
  oracle_forces(n, traj, m, G, eps, a, NULL, nthreads);
  for (int s = 0; s < n_steps; ++s) {
    double* xs = traj + sz * (size_t)(s + 1);
    memcpy(xs, traj + sz * (size_t)s, sizeof(double) * sz);
    if (oracle_kdk(n, xs, v, m, G, eps, dt, 1, a, 1, 0, NULL, nthreads)) break;
  }
  /* reverse sweep; g_x0 holds lam_x and g_v0 holds lam_v while running */
  memcpy(g_x0, lam_xT, sizeof(double) * sz);
  memcpy(g_v0, lam_vT, sizeof(double) * sz);
  for (int64_t k = 0; k < n; ++k) g_m[k] = 0.0;
  for (int s = n_steps - 1; s >= 0; --s) {
    const double* x_new = traj + sz * (size_t)(s + 1);
    const double* x_old = traj + sz * (size_t)s;
    double pg[2];
    memcpy(lam_vh, g_v0, sizeof(double) * sz);
    oracle_force_vjp(n, x_new, m, g_v0, G, eps, gx, gmv, nthreads);
    if (g_params) {
      oracle_param_vjp(n, x_new, m, g_v0, G, eps, pg, nthreads);
      g_params[0] += 0.5 * dt * pg[0], g_params[1] += 0.5 * dt * pg[1];
    }
    for (size_t k = 0; k < sz; ++k) g_x0[k] += 0.5 * dt * gx[k];
    for (int64_t k = 0; k < n; ++k) g_m[k] += 0.5 * dt * gmv[k];
    for (size_t k = 0; k < sz; ++k) lam_vh[k] += dt * g_x0[k];
    oracle_force_vjp(n, x_old, m, lam_vh, G, eps, gx, gmv, nthreads);
    if (g_params) {
      oracle_param_vjp(n, x_old, m, lam_vh, G, eps, pg, nthreads);
      g_params[0] += 0.5 * dt * pg[0], g_params[1] += 0.5 * dt * pg[1];
    }
    for (size_t k = 0; k < sz; ++k) g_x0[k] += 0.5 * dt * gx[k];
    for (int64_t k = 0; k < n; ++k) g_m[k] += 0.5 * dt * gmv[k];
    memcpy(g_v0, lam_vh, sizeof(double) * sz);
  }
  free(traj), free(v), free(a), free(gx), free(gmv), free(lam_vh);
  return 0;
}

int oracle_adjoint(int64_t n, const double* x0, const double* v0, const double* m, double G, double eps, double dt,
                   int n_steps, const double* lam_xT, const double* lam_vT, double* g_x0, double* g_v0, double* g_m,
                   int nthreads) {
  return adjoint_sweep(n, x0, v0, m, G, eps, dt, n_steps, lam_xT, lam_vT, g_x0, g_v0, g_m, NULL, nthreads);
}

/* oracle_adjoint plus g_params[0] = dL/dG and g_params[1] = dL/deps. */
int oracle_adjoint_params(int64_t n, const double* x0, const double* v0, const double* m, double G, double eps,
                          double dt, int n_steps, const double* lam_xT, const double* lam_vT, double* g_x0,
                          double* g_v0, double* g_m, double* g_params, int nthreads) {
  if (!g_params) return 1;
  g_params[0] = g_params[1] = 0.0;
  return adjoint_sweep(n, x0, v0, m, G, eps, dt, n_steps, lam_xT, lam_vT, g_x0, g_v0, g_m, g_params, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones gas (the paper's pair law, Eq. 1)                            */
/*
 *   V(r) = 4 eps_lj [ (sigma / r)^12 - (sigma / r)^6 ]
 *   F_i  = -dV/dx_i = 24 eps_lj [ 2 sigma^12 / r^14 - sigma^6 / r^8 ] (x_i - x_j)
 * summed over every j != i (no cutoff: all N^2 pairs, Sec. V-B). Accelerations
 * are F_i / m_i; phi_i = sum_{j != i} V(r_ij) / m_i (potential energy per unit
 * mass of body i, so that U = 1/2 sum m_i phi_i = sum_{i<j} V(r_ij)).
 * r^2 may be softened as r^2 + soft^2 (soft = 0 gives the plain law).
 */
static void body_force_lj(int64_t n, const double* x, const double* m, double eps_lj, double sigma, double soft,
                          int64_t i, double* ai, double* phii) {
  double fx = 0.0, fy = 0.0, fz = 0.0, v = 0.0;
  const double s2 = sigma * sigma;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double dx = x[3 * i + 0] - x[3 * j + 0]; /* x_i - x_j */
    double dy = x[3 * i + 1] - x[3 * j + 1];
    double dz = x[3 * i + 2] - x[3 * j + 2];
    double r2 = dx * dx + dy * dy + dz * dz + soft * soft;
    double sr2 = s2 / r2;
    double sr6 = sr2 * sr2 * sr2;
    double sr12 = sr6 * sr6;
    double coef = 24.0 * eps_lj * (2.0 * sr12 - sr6) / r2; /* 24 eps [2 s^12/r^14 - s^6/r^8] */
    fx += coef * dx;
    fy += coef * dy;
    fz += coef * dz;
    v += 4.0 * eps_lj * (sr12 - sr6);
  }
  ai[0] = fx / m[i];
  ai[1] = fy / m[i];
  ai[2] = fz / m[i];
  if (phii) *phii = v / m[i];
}

typedef struct {
  int64_t n;
  const double *x, *m;
  double eps_lj, sigma, soft;
  const int64_t* idx;
  double *a, *phi;
} lj_args;

static void lj_rows(int64_t lo, int64_t hi, void* p) {
  lj_args* f = (lj_args*)p;
  for (int64_t r = lo; r < hi; ++r) {
    int64_t i = f->idx ? f->idx[r] : r;
    body_force_lj(f->n, f->x, f->m, f->eps_lj, f->sigma, f->soft, i, f->a + 3 * r, f->phi ? f->phi + r : NULL);
  }
}

int oracle_lj_forces(int64_t n, const double* x, const double* m, double eps_lj, double sigma, double soft,
                     double* a, double* phi, int nthreads) {
  if (n < 0 || (n > 0 && (!x || !m || !a))) return 1;
  lj_args f = {n, x, m, eps_lj, sigma, soft, NULL, a, phi};
  parallel_rows(n, nthreads, lj_rows, &f);
  return 0;
}

int oracle_lj_forces_at(int64_t n, const double* x, const double* m, double eps_lj, double sigma, double soft,
                        const int64_t* idx, int64_t k, double* a, double* phi, int nthreads) {
  if (n < 0 || k < 0 || (k > 0 && (!x || !m || !a || !idx))) return 1;
  for (int64_t r = 0; r < k; ++r)
    if (idx[r] < 0 || idx[r] >= n) return 1;
  lj_args f = {n, x, m, eps_lj, sigma, soft, idx, a, phi};
  parallel_rows(k, nthreads, lj_rows, &f);
  return 0;
}

typedef struct {
  int64_t n;
  const double* x;
  double eps_lj, sigma, soft;
  double* row_u;
} lj_pot_args;

static void lj_pot_rows(int64_t lo, int64_t hi, void* p) {
  lj_pot_args* f = (lj_pot_args*)p;
  const double s2 = f->sigma * f->sigma;
  for (int64_t i = lo; i < hi; ++i) {
    csum u = {0.0, 0.0};
    for (int64_t j = i + 1; j < f->n; ++j) {
      double dx = f->x[3 * j + 0] - f->x[3 * i + 0];
      double dy = f->x[3 * j + 1] - f->x[3 * i + 1];
      double dz = f->x[3 * j + 2] - f->x[3 * i + 2];
      double sr2 = s2 / (dx * dx + dy * dy + dz * dz + f->soft * f->soft);
      double sr6 = sr2 * sr2 * sr2;
      csum_add(&u, 4.0 * f->eps_lj * (sr6 * sr6 - sr6));
    }
    f->row_u[i] = csum_get(&u);
  }
}

/* out[9] = {E, K, U, Px, Py, Pz, Lx, Ly, Lz} with U = sum_{i<j} V(r_ij). */
int oracle_lj_energy(int64_t n, const double* x, const double* v, const double* m, double eps_lj, double sigma,
                     double soft, double* out, int nthreads) {
  if (n < 0 || !out || (n > 0 && (!x || !v || !m))) return 1;
  double* row_u = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!row_u) return 2;
  lj_pot_args f = {n, x, eps_lj, sigma, soft, row_u};
  parallel_rows(n, nthreads, lj_pot_rows, &f);
  csum K = {0, 0}, U = {0, 0}, P[3] = {{0, 0}, {0, 0}, {0, 0}}, L[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + 3 * i;
    const double* vi = v + 3 * i;
    csum_add(&K, 0.5 * m[i] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
    csum_add(&U, row_u[i]);
    for (int c = 0; c < 3; ++c) csum_add(&P[c], m[i] * vi[c]);
    csum_add(&L[0], m[i] * (xi[1] * vi[2] - xi[2] * vi[1]));
    csum_add(&L[1], m[i] * (xi[2] * vi[0] - xi[0] * vi[2]));
    csum_add(&L[2], m[i] * (xi[0] * vi[1] - xi[1] * vi[0]));
  }
  free(row_u);
  out[1] = csum_get(&K);
  out[2] = csum_get(&U);
  out[0] = out[1] + out[2];
  for (int c = 0; c < 3; ++c) {
    out[3 + c] = csum_get(&P[c]);
    out[6 + c] = csum_get(&L[c]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* virial diagnostics                                                         */
/*
 * Clausius virial W = sum_i x_i . F_i (F_i = m_i a_i) in its pair form: the
 * pair (i, j) contributes (x_i - x_j) . F_ij, F_ij the force of j on i, i.e.
 *   gravity:        -G m_i m_j |d|^2 / s^3,                 s^2 = |d|^2 + eps^2
 *   Lennard-Jones:  24 eps_lj (2 sigma^12 / s^14 - sigma^6 / s^8) |d|^2,  s^2 = |d|^2 + soft^2
 * so that the sum over i < j is independent of the origin and of any per-body
 * route. out[3] = {K, W, Q = -2K/W (0 if W = 0)}.
 */
typedef struct {
  int64_t n;
  const double *x, *m;
  int law;
  double G, eps, eps_lj, sigma, soft;
  double* row_w;
} vir_args;

static void virial_rows(int64_t lo, int64_t hi, void* p) {
  vir_args* f = (vir_args*)p;
  for (int64_t i = lo; i < hi; ++i) {
    csum w = {0.0, 0.0};
    for (int64_t j = i + 1; j < f->n; ++j) {
      double dx = f->x[3 * j + 0] - f->x[3 * i + 0];
      double dy = f->x[3 * j + 1] - f->x[3 * i + 1];
      double dz = f->x[3 * j + 2] - f->x[3 * i + 2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (f->law == 0) {
        double s2 = r2 + f->eps * f->eps;
        double s = sqrt(s2);
        csum_add(&w, -f->G * f->m[i] * f->m[j] * r2 / (s2 * s));
      } else {
        double s2 = r2 + f->soft * f->soft;
        double u = f->sigma * f->sigma / s2; /* sigma^2 / s^2 */
        double u3 = u * u * u;
        csum_add(&w, 24.0 * f->eps_lj * (2.0 * u3 * u3 - u3) * r2 / s2);
      }
    }
    f->row_w[i] = csum_get(&w);
  }
}

int oracle_virial(int64_t n, const double* x, const double* v, const double* m, int law, double G, double eps,
                  double eps_lj, double sigma, double soft, double* out, int nthreads) {
  if (n < 0 || !out || (law != 0 && law != 1) || (n > 0 && (!x || !v || !m))) return 1;
  double* row_w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!row_w) return 2;
  vir_args f = {n, x, m, law, G, eps, eps_lj, sigma, soft, row_w};
  parallel_rows(n, nthreads, virial_rows, &f);
  csum K = {0, 0}, W = {0, 0};
  for (int64_t i = 0; i < n; ++i) {
    const double* vi = v + 3 * i;
    csum_add(&K, 0.5 * m[i] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
    csum_add(&W, row_w[i]);
  }
  free(row_w);
  out[0] = csum_get(&K);
  out[1] = csum_get(&W);
  out[2] = out[1] != 0.0 ? -2.0 * out[0] / out[1] : 0.0;
  return 0;
}

/*
 * Reflecting walls of the box [0, box]^3 ("boundary checking", Fig. 3/4
 * captions): after the drift, a coordinate that left the box is mirrored back
 * across the wall it crossed and that velocity component changes sign
 * (specular reflection; repeated while it is still outside, for large steps).
 */
static void reflect(double* xc, double* vc, double box) {
  for (int guard = 0; guard < 64; ++guard) {
    if (*xc < 0.0) {
      *xc = -*xc;
      *vc = -*vc;
    } else if (*xc > box) {
      *xc = 2.0 * box - *xc;
      *vc = -*vc;
    } else {
      return;
    }
  }
}

/* KDK leapfrog for the Lennard-Jones gas, with reflecting walls when box > 0. */
int oracle_lj_kdk(int64_t n, double* x, double* v, const double* m, double eps_lj, double sigma, double soft,
                  double box, double dt, int n_steps, double* a, int a_valid, int energy_every, double* energy_log,
                  int nthreads) {
  if (n < 0 || n_steps < 0 || (n > 0 && (!x || !v || !m || !a))) return 1;
  if (!a_valid) oracle_lj_forces(n, x, m, eps_lj, sigma, soft, a, NULL, nthreads);
  int rec = 0;
  for (int s = 0; s < n_steps; ++s) {
    for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * a[k];
    for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];
    if (box > 0.0)
      for (int64_t k = 0; k < 3 * n; ++k) reflect(&x[k], &v[k], box);
    oracle_lj_forces(n, x, m, eps_lj, sigma, soft, a, NULL, nthreads);
    for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * a[k];
    if (energy_every > 0 && energy_log && (s + 1) % energy_every == 0) {
      int rc = oracle_lj_energy(n, x, v, m, eps_lj, sigma, soft, energy_log + 9 * rec, nthreads);
      if (rc) return rc;
      ++rec;
    }
  }
  return 0;
}
