/*
 * hbe_oracle.c -- CPU oracle for the 3D Higgs boson equation (HBE) in de Sitter
 * spacetime, discretised as in Sec. 2.1 of Balogh, Banda & Yagdjian,
 * "Computational Results for the Higgs Boson Equation in the de Sitter
 * Spacetime" (arXiv:1803.01291).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct FP64
 * restatement that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * library never links or calls it.  It shares no code with the CUDA path.
 *
 * What it computes (all in double precision, plain loops):
 *   - Eq. (higgs-boson-rescalled) on a box of side L with the unknowns on the
 *     N^3 interior nodes (zero-Dirichlet: h = L/(N+1); periodic: h = L/N);
 *   - the FD4 second derivative of Sec. 2.1 per axis,
 *       d2u/dx2 ~ (-1/12 u[i-2] + 4/3 u[i-1] - 5/2 u[i] + 4/3 u[i+1] - 1/12 u[i+2]) / h^2,
 *     with the symmetric neighbours paired first, axes summed in x, y, z order;
 *     neighbours outside the box read 0 (Dirichlet, both ghost layers) or wrap
 *     (periodic);
 *   - the first-order system Eq. (rhs): f1 = v2,
 *       f2 = -3 v2 + e^{-2t} Lap(v1) + mu^2 v1 - lambda v1^3
 *     (the physical-coordinate form of e^{-2t} L^{-2} Delta on the unit box);
 *   - the classic RK4 step of Sec. 2.1 in its textbook form with four full
 *     k arrays (not the storage-reuse variant), stage times t, t+dt/2,
 *     t+dt/2, t+dt, and t_n = t0 + n dt;
 *   - the sign/bubble diagnostics (bubble = maximal connected set where the
 *     solution changes sign, Sec. 1): components of {phi > eps} and
 *     {phi < -eps} under 6-connectivity (wrapping when periodic), found by
 *     breadth-first search; bubble count = max(0, n_pos + n_neg - 1).
 *
 * Parity pins: see tests/test_oracle_pins.py (Duffing ODE, vacua, lambda = 0
 * plane wave against the Bessel closed form, radial u = r phi solver, octant
 * symmetry, 4th-order convergence, FD4 polynomial exactness, RK4 stability
 * polynomial, superposition and shift invariance, BFS against a library
 * labelling).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_DIRICHLET 0
#define ORACLE_PERIODIC 1

/* A box of nx * ny * nz unknowns (the paper's grid is the cube nx = ny = nz;
 * boxes serve the one-point window evaluation of the tests). */
typedef struct {
  int nx, ny, nz;
  int bc;
  double h;
  double mu2;
  double lambda;
} grid_t;

double oracle_grid_spacing(int N, double L, int bc) {
  return bc == ORACLE_PERIODIC ? L / (double)N : L / (double)(N + 1);
}

static inline size_t idx3(int N, int i, int j, int k) {
  return ((size_t)k * (size_t)N + (size_t)j) * (size_t)N + (size_t)i;
}

static inline size_t gidx(const grid_t *g, int i, int j, int k) {
  return ((size_t)k * (size_t)g->ny + (size_t)j) * (size_t)g->nx + (size_t)i;
}

static inline size_t gsize(const grid_t *g) { return (size_t)g->nx * g->ny * g->nz; }

/* Value of u at node (i, j, k) with the boundary rule applied. */
static inline double node(const double *u, const grid_t *g, int i, int j, int k) {
  if (g->bc == ORACLE_PERIODIC) {
    i = ((i % g->nx) + g->nx) % g->nx;
    j = ((j % g->ny) + g->ny) % g->ny;
    k = ((k % g->nz) + g->nz) % g->nz;
    return u[gidx(g, i, j, k)];
  }
  if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) return 0.0;
  return u[gidx(g, i, j, k)];
}

/* FD4 Laplacian, Sec. 2.1: one 5-point second difference per axis, divided by h^2. */
static void laplacian(const double *u, double *out, const grid_t *g) {
  const double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        const double c = node(u, g, i, j, k);
        const double dxx = (-1.0 / 12.0 * (node(u, g, i - 2, j, k) + node(u, g, i + 2, j, k)) +
                            4.0 / 3.0 * (node(u, g, i - 1, j, k) + node(u, g, i + 1, j, k)) -
                            5.0 / 2.0 * c) * ih2;
        const double dyy = (-1.0 / 12.0 * (node(u, g, i, j - 2, k) + node(u, g, i, j + 2, k)) +
                            4.0 / 3.0 * (node(u, g, i, j - 1, k) + node(u, g, i, j + 1, k)) -
                            5.0 / 2.0 * c) * ih2;
        const double dzz = (-1.0 / 12.0 * (node(u, g, i, j, k - 2) + node(u, g, i, j, k + 2)) +
                            4.0 / 3.0 * (node(u, g, i, j, k - 1) + node(u, g, i, j, k + 1)) -
                            5.0 / 2.0 * c) * ih2;
        out[gidx(g, i, j, k)] = dxx + dyy + dzz;
      }
}

/* Right-hand side f(t, v) of Eq. (rhs). lap is caller scratch of N^3 doubles. */
static void rhs(double t, const double *v1, const double *v2, double *f1, double *f2,
                double *lap, const grid_t *g) {
  const size_t n3 = gsize(g);
  const double e = exp(-2.0 * t);
  laplacian(v1, lap, g);
#pragma omp parallel for schedule(static)
  for (size_t p = 0; p < n3; ++p) {
    const double u = v1[p];
    f1[p] = v2[p];
    f2[p] = -3.0 * v2[p] + e * lap[p] + g->mu2 * u - g->lambda * u * u * u;
  }
}

/* out = v + a * k  (both components) */
static void axpy2(const double *v1, const double *v2, double a, const double *k1, const double *k2,
                  double *o1, double *o2, size_t n3) {
#pragma omp parallel for schedule(static)
  for (size_t p = 0; p < n3; ++p) {
    o1[p] = v1[p] + a * k1[p];
    o2[p] = v2[p] + a * k2[p];
  }
}

typedef struct {
  double *k1a, *k1b, *k2a, *k2b, *k3a, *k3b, *k4a, *k4b, *ta, *tb, *lap;
} work_t;

static int work_alloc(work_t *w, size_t n3) {
  double **f[] = {&w->k1a, &w->k1b, &w->k2a, &w->k2b, &w->k3a, &w->k3b,
                  &w->k4a, &w->k4b, &w->ta,  &w->tb,  &w->lap};
  for (size_t i = 0; i < sizeof(f) / sizeof(f[0]); ++i) {
    *f[i] = (double *)malloc(n3 * sizeof(double));
    if (!*f[i]) return -1;
  }
  return 0;
}

static void work_free(work_t *w) {
  free(w->k1a); free(w->k1b); free(w->k2a); free(w->k2b); free(w->k3a); free(w->k3b);
  free(w->k4a); free(w->k4b); free(w->ta);  free(w->tb);  free(w->lap);
}

/* One classic RK4 step (Sec. 2.1), textbook form. */
static void rk4_step(double t, double dt, double *v1, double *v2, work_t *w, const grid_t *g) {
  const size_t n3 = gsize(g);
  rhs(t, v1, v2, w->k1a, w->k1b, w->lap, g);
  axpy2(v1, v2, dt / 2.0, w->k1a, w->k1b, w->ta, w->tb, n3);
  rhs(t + dt / 2.0, w->ta, w->tb, w->k2a, w->k2b, w->lap, g);
  axpy2(v1, v2, dt / 2.0, w->k2a, w->k2b, w->ta, w->tb, n3);
  rhs(t + dt / 2.0, w->ta, w->tb, w->k3a, w->k3b, w->lap, g);
  axpy2(v1, v2, dt, w->k3a, w->k3b, w->ta, w->tb, n3);
  rhs(t + dt, w->ta, w->tb, w->k4a, w->k4b, w->lap, g);
#pragma omp parallel for schedule(static)
  for (size_t p = 0; p < n3; ++p) {
    v1[p] = v1[p] + dt * (w->k1a[p] + 2.0 * w->k2a[p] + 2.0 * w->k3a[p] + w->k4a[p]) / 6.0;
    v2[p] = v2[p] + dt * (w->k1b[p] + 2.0 * w->k2b[p] + 2.0 * w->k3b[p] + w->k4b[p]) / 6.0;
  }
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* max |phi| over n values; *finite = 0 if any value is NaN or infinite. */
static double max_abs_n(const double *phi, size_t n3, int *finite) {
  double m = 0.0;
  int fin = 1;
  for (size_t p = 0; p < n3; ++p) {
    const double a = fabs(phi[p]);
    if (!(a <= 1.79769313486231570815e308)) fin = 0;
    else if (a > m) m = a;
  }
  if (finite) *finite = fin;
  return m;
}

/* max |phi| over the N^3 unknowns; *finite = 0 if any value is NaN or infinite. */
double oracle_max_abs(const double *phi, int N, int *finite) {
  return max_abs_n(phi, (size_t)N * N * N, finite);
}

/*
 * Advance (phi, psi) in place on an nx * ny * nz box with spacing h by up to
 * nsteps RK4 steps of size dt from t0.  If stop_threshold > 0, stop after the
 * first completed step whose max|phi| exceeds it or is non-finite.  Returns the
 * number of steps taken, or -1 on allocation failure.
 */
int64_t oracle_run_box(double *phi, double *psi, int nx, int ny, int nz, double h, double mu,
                       double lambda, int bc, double t0, double dt, int64_t nsteps,
                       double stop_threshold, int nthreads) {
  grid_t g = {nx, ny, nz, bc, h, mu * mu, lambda};
  work_t w;
  memset(&w, 0, sizeof(w));
  set_threads(nthreads);
  if (work_alloc(&w, gsize(&g)) != 0) {
    work_free(&w);
    return -1;
  }
  int64_t n = 0;
  for (; n < nsteps; ++n) {
    rk4_step(t0 + (double)n * dt, dt, phi, psi, &w, &g);
    if (stop_threshold > 0.0) {
      int fin;
      const double m = max_abs_n(phi, gsize(&g), &fin);
      if (!fin || m > stop_threshold) {
        ++n;
        break;
      }
    }
  }
  work_free(&w);
  return n;
}

/* The cubic grid of the paper: N^3 unknowns on a box of side L. */
int64_t oracle_run(double *phi, double *psi, int N, double L, double mu, double lambda, int bc,
                   double t0, double dt, int64_t nsteps, double stop_threshold, int nthreads) {
  return oracle_run_box(phi, psi, N, N, N, oracle_grid_spacing(N, L, bc), mu, lambda, bc, t0, dt,
                        nsteps, stop_threshold, nthreads);
}

/* The FD4 Laplacian alone (for the polynomial-exactness pin). */
void oracle_laplacian(const double *u, double *out, int N, double h, int bc, int nthreads) {
  grid_t g = {N, N, N, bc, h, 0.0, 0.0};
  set_threads(nthreads);
  laplacian(u, out, &g);
}

/* f(t, v) alone (both components). */
int oracle_rhs(double t, const double *v1, const double *v2, double *f1, double *f2, int N,
               double L, double mu, double lambda, int bc) {
  grid_t g = {N, N, N, bc, oracle_grid_spacing(N, L, bc), mu * mu, lambda};
  double *lap = (double *)malloc((size_t)N * N * N * sizeof(double));
  if (!lap) return -1;
  rhs(t, v1, v2, f1, f2, lap, &g);
  free(lap);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Sign masks and connected components (bubbles, Sec. 1).
 * Masks: bit (x % 32) of word ((z * N + y) * W + x / 32), W = ceil(N / 32).
 * ------------------------------------------------------------------------- */

static int64_t count_components(const unsigned char *in, int N, int bc, int32_t *queue,
                                unsigned char *seen) {
  const size_t n3 = (size_t)N * N * N;
  memset(seen, 0, n3);
  int64_t comps = 0;
  for (size_t s = 0; s < n3; ++s) {
    if (!in[s] || seen[s]) continue;
    ++comps;
    size_t head = 0, tail = 0;
    queue[tail++] = (int32_t)s;
    seen[s] = 1;
    while (head < tail) {
      const size_t p = (size_t)queue[head++];
      const int i = (int)(p % N), j = (int)((p / N) % N), k = (int)(p / ((size_t)N * N));
      const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                            {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
      for (int d = 0; d < 6; ++d) {
        int a = nb[d][0], b = nb[d][1], c = nb[d][2];
        if (bc == ORACLE_PERIODIC) {
          a = (a + N) % N;
          b = (b + N) % N;
          c = (c + N) % N;
        } else if (a < 0 || a >= N || b < 0 || b >= N || c < 0 || c >= N) {
          continue;
        }
        const size_t q = idx3(N, a, b, c);
        if (in[q] && !seen[q]) {
          seen[q] = 1;
          queue[tail++] = (int32_t)q;
        }
      }
    }
  }
  return comps;
}

/*
 * Diagnostics of one field: max|phi|, finiteness, sign masks (optional) and
 * the component counts.  Returns 0, or -1 on allocation failure.
 */
int oracle_diag(const double *phi, int N, int bc, double eps, double *max_abs, int *finite,
                int64_t *n_pos, int64_t *n_neg, int64_t *bubbles, uint32_t *pos_mask,
                uint32_t *neg_mask) {
  const size_t n3 = (size_t)N * N * N;
  const int W = (N + 31) / 32;
  unsigned char *pos = (unsigned char *)calloc(n3, 1);
  unsigned char *neg = (unsigned char *)calloc(n3, 1);
  unsigned char *seen = (unsigned char *)malloc(n3);
  int32_t *queue = (int32_t *)malloc(n3 * sizeof(int32_t));
  if (!pos || !neg || !seen || !queue) {
    free(pos); free(neg); free(seen); free(queue);
    return -1;
  }
  *max_abs = oracle_max_abs(phi, N, finite);
  for (size_t p = 0; p < n3; ++p) {
    pos[p] = phi[p] > eps;
    neg[p] = phi[p] < -eps;
  }
  if (pos_mask) memset(pos_mask, 0, (size_t)N * N * W * sizeof(uint32_t));
  if (neg_mask) memset(neg_mask, 0, (size_t)N * N * W * sizeof(uint32_t));
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const size_t p = idx3(N, i, j, k);
        const size_t w = ((size_t)k * N + j) * W + (size_t)(i / 32);
        if (pos_mask && pos[p]) pos_mask[w] |= 1u << (i % 32);
        if (neg_mask && neg[p]) neg_mask[w] |= 1u << (i % 32);
      }
  *n_pos = count_components(pos, N, bc, queue, seen);
  *n_neg = count_components(neg, N, bc, queue, seen);
  const int64_t b = *n_pos + *n_neg - 1;
  *bubbles = b > 0 ? b : 0;
  free(pos); free(neg); free(seen); free(queue);
  return 0;
}
