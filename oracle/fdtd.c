/*
 * FP64 CPU oracle for the photoacoustic forward map K and its adjoint K*.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code with the GPU path.
 *
 * What it computes (paper Sec. 2, the wave IVP of Eq. (wave_equation) and the
 * measurement map K of Sec. 2.2):
 *
 *   p_tt = c(x)^2 lap p,  p(0) = x,  p_t(0) = 0,   density 1,
 *
 * discretised *literally* as the staggered pressure/velocity leapfrog of order
 * 2M on a uniform grid of spacing h (cell i at coordinate i*h), with p = 0
 * outside the grid:
 *
 *   v^{1/2}     = -(dt/2h) G P^0                    (symmetric start, p_t(0)=0)
 *   P^{n}       = P^{n-1} + (c^2 dt/h) (G^T v^{n-1/2})  on interior cells
 *   v^{n+1/2}   = v^{n-1/2} - (dt/h) G P^n
 *
 * G is the staggered difference along each axis,
 *   (G P)_{i+1/2} = sum_{k=1..M} c_k (P_{i+k} - P_{i+1-k}),
 * with the standard staggered Fornberg weights c_k; -G^T is the matching
 * divergence.  Faces exist wherever they can touch an interior cell.
 *
 * Absorbing layer (optional; this implementation's reading of the paper's PML, which the
 * paper takes from k-Wave): a damping rate sigma(x) >= 0 [1/s] enters the
 * pressure equation, p_t + sigma p = -c^2 div v, with sigma p averaged over
 * the two time levels (trapezoidal rule):
 *
 *   P^{n} = alpha .* P^{n-1} + beta .* (c^2 dt/h) (G^T v^{n-1/2}),
 *   alpha = (1 - sigma dt/2) / (1 + sigma dt/2),  beta = 1 / (1 + sigma dt/2),
 *
 * which reduces to the undamped program for sigma = 0.
 *
 * Sampling (the point-sensor trace of Sec. 2.2): y[s, n] = sum of the
 * bilinear (2D) / trilinear (3D) interpolation weights of sensor s times
 * P^n at the 2^d surrounding cells, for n = 0 .. nt-1 (P^0 included).
 * y is stored sensor-major: y[s*nt + n].
 *
 * The adjoint is the reverse sweep of exactly this program (each assignment
 * transposed in reverse order); it is NOT time reversal of the PDE.  Inner
 * products are plain Euclidean sums on both spaces, so adjoint == transpose.
 *
 * Layout: cells row-major with x fastest: idx = (z*ny + y)*nx + x.  2D grids
 * use dim = 2 and n[2] = 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Staggered first-derivative weights c_k of order 2M (Fornberg), k = 1..M. */
static const double STAG[4][4] = {
    {1.0, 0, 0, 0},
    {9.0 / 8.0, -1.0 / 24.0, 0, 0},
    {75.0 / 64.0, -25.0 / 384.0, 3.0 / 640.0, 0},
    {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0},
};

/* Padded geometry: every axis in use carries PAD zero cells on each side, so
 * the stencils below never test bounds.  PAD = 2M covers every index that the
 * gradient at the outermost face can reach. */
typedef struct {
  int dim, M, pad;
  int n[3];   /* interior extent */
  int np[3];  /* padded extent */
  long st[3]; /* padded strides */
  long total; /* padded element count */
} geom;

static void geom_init(geom* g, int dim, const int* n, int M) {
  g->dim = dim;
  g->M = M;
  g->pad = 2 * M;
  for (int a = 0; a < 3; ++a) {
    g->n[a] = (a < dim) ? n[a] : 1;
    g->np[a] = (a < dim) ? n[a] + 2 * g->pad : 1;
  }
  g->st[0] = 1;
  g->st[1] = g->np[0];
  g->st[2] = (long)g->np[0] * g->np[1];
  g->total = g->st[2] * g->np[2];
}

/* padded index of interior coordinate (x, y, z) */
static long pidx(const geom* g, int x, int y, int z) {
  long off = (long)(x + g->pad);
  off += (long)(y + g->pad) * g->st[1];
  if (g->dim == 3) off += (long)(z + g->pad) * g->st[2];
  return off;
}

/* Face storage: the face at position p+1/2 along axis a lives at the padded
 * slot of coordinate p along a.  Valid faces: p in [-M, n_a + M - 2]. */

/* V_a[faces] (op)= scale * (G_a F)  for F given on padded cells (zero pad). */
static void grad_axis(const geom* g, int a, const double* F, double* V, double scale) {
  const int M = g->M;
  const double* c = STAG[M - 1];
  const long s = g->st[a];
  int lo[3] = {0, 0, 0}, hi[3] = {g->n[0], g->n[1], g->n[2]};
  lo[a] = -M;
  hi[a] = g->n[a] + M - 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = lo[2]; z < hi[2]; ++z)
    for (int y = lo[1]; y < hi[1]; ++y)
      for (int x = lo[0]; x < hi[0]; ++x) {
        const long p = pidx(g, x, y, z);
        double acc = 0.0;
        for (int k = 1; k <= M; ++k) acc += c[k - 1] * (F[p + k * s] - F[p + (1 - k) * s]);
        V[p] += scale * acc;
      }
}

/* out[interior] += scale * (G_a^T V) */
static void gradT_axis(const geom* g, int a, const double* V, double* out, double scale) {
  const int M = g->M;
  const double* c = STAG[M - 1];
  const long s = g->st[a];
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < g->n[2]; ++z)
    for (int y = 0; y < g->n[1]; ++y)
      for (int x = 0; x < g->n[0]; ++x) {
        const long p = pidx(g, x, y, z);
        double acc = 0.0;
        for (int k = 1; k <= M; ++k) acc += c[k - 1] * (V[p - k * s] - V[p + (k - 1) * s]);
        out[p] += scale * acc;
      }
}

/* Interpolation stencil of one sensor: 2^dim cells and weights. */
typedef struct {
  long cell[8];
  double w[8];
  int cnt;
} sensor_t;

static int sensor_setup(const geom* g, const double* pos, double h, sensor_t* s) {
  int i0[3] = {0, 0, 0};
  double f[3] = {0, 0, 0};
  for (int a = 0; a < g->dim; ++a) {
    const double u = pos[a] / h;
    if (!(u >= 0.0 && u <= (double)(g->n[a] - 1))) return -1;
    int i = (int)floor(u);
    if (i > g->n[a] - 2) i = g->n[a] - 2;
    i0[a] = i;
    f[a] = u - (double)i;
  }
  s->cnt = 1 << g->dim;
  for (int corner = 0; corner < s->cnt; ++corner) {
    int c3[3] = {0, 0, 0};
    double w = 1.0;
    for (int a = 0; a < g->dim; ++a) {
      const int bit = (corner >> a) & 1;
      c3[a] = i0[a] + bit;
      w *= bit ? f[a] : (1.0 - f[a]);
    }
    s->cell[corner] = pidx(g, c3[0], c3[1], c3[2]);
    s->w[corner] = w;
  }
  return 0;
}

typedef struct {
  geom g;
  int nt, ns;
  double dt, h;
  double* b;  /* c^2 dt / h on padded cells (0 in the pad) */
  double* alpha;  /* damping of P (NULL: none) */
  double* beta;   /* damping of the update (NULL: none) */
  sensor_t* sens;
} problem;

static int problem_init(problem* pb, int dim, const int* n, double h, double dt, int nt, int order,
                        const double* c, int ns, const double* sensors) {
  memset(pb, 0, sizeof(*pb));
  if (dim != 2 && dim != 3) return -1;
  if (order != 2 && order != 4 && order != 6 && order != 8) return -1;
  if (nt < 1 || ns < 0) return -1;
  for (int a = 0; a < dim; ++a)
    if (n[a] < 2) return -1;
  geom_init(&pb->g, dim, n, order / 2);
  pb->nt = nt;
  pb->ns = ns;
  pb->dt = dt;
  pb->h = h;
  pb->b = (double*)calloc((size_t)pb->g.total, sizeof(double));
  pb->sens = (sensor_t*)calloc((size_t)(ns > 0 ? ns : 1), sizeof(sensor_t));
  if (!pb->b || !pb->sens) return -2;
  const geom* g = &pb->g;
  for (int z = 0; z < g->n[2]; ++z)
    for (int y = 0; y < g->n[1]; ++y)
      for (int x = 0; x < g->n[0]; ++x) {
        const double cc = c[((long)z * g->n[1] + y) * g->n[0] + x];
        pb->b[pidx(g, x, y, z)] = cc * cc * dt / h;
      }
  for (int s = 0; s < ns; ++s)
    if (sensor_setup(g, sensors + (long)s * dim, h, &pb->sens[s]) != 0) return -3;
  return 0;
}

static void problem_free(problem* pb) {
  free(pb->b);
  free(pb->alpha);
  free(pb->beta);
  free(pb->sens);
}

/* alpha, beta from the damping rate sigma (N cells, 1/s); NULL leaves the program undamped. */
static int set_damping(problem* pb, const double* sigma) {
  if (!sigma) return 0;
  const geom* g = &pb->g;
  pb->alpha = (double*)calloc((size_t)g->total, sizeof(double));
  pb->beta = (double*)calloc((size_t)g->total, sizeof(double));
  if (!pb->alpha || !pb->beta) return -2;
  for (long i = 0; i < g->total; ++i) pb->alpha[i] = pb->beta[i] = 1.0;
  for (int z = 0; z < g->n[2]; ++z)
    for (int y = 0; y < g->n[1]; ++y)
      for (int x = 0; x < g->n[0]; ++x) {
        const double sg = sigma[((long)z * g->n[1] + y) * g->n[0] + x];
        if (!(sg >= 0.0)) return -4;
        const double q = 0.5 * sg * pb->dt;
        pb->alpha[pidx(g, x, y, z)] = (1.0 - q) / (1.0 + q);
        pb->beta[pidx(g, x, y, z)] = 1.0 / (1.0 + q);
      }
  return 0;
}

static void sample(const problem* pb, const double* P, double* y, int n) {
  for (int s = 0; s < pb->ns; ++s) {
    double acc = 0.0;
    for (int k = 0; k < pb->sens[s].cnt; ++k) acc += pb->sens[s].w[k] * P[pb->sens[s].cell[k]];
    y[(long)s * pb->nt + n] = acc;
  }
}

static void inject(const problem* pb, const double* r, double* P, int n) {
  for (int s = 0; s < pb->ns; ++s) {
    const double rv = r[(long)s * pb->nt + n];
    for (int k = 0; k < pb->sens[s].cnt; ++k) P[pb->sens[s].cell[k]] += pb->sens[s].w[k] * rv;
  }
}

static void to_padded(const geom* g, const double* x, double* P) {
  for (int z = 0; z < g->n[2]; ++z)
    for (int y = 0; y < g->n[1]; ++y)
      memcpy(P + pidx(g, 0, y, z), x + ((long)z * g->n[1] + y) * g->n[0], sizeof(double) * g->n[0]);
}

static void from_padded(const geom* g, const double* P, double* x) {
  for (int z = 0; z < g->n[2]; ++z)
    for (int y = 0; y < g->n[1]; ++y)
      memcpy(x + ((long)z * g->n[1] + y) * g->n[0], P + pidx(g, 0, y, z), sizeof(double) * g->n[0]);
}

/* P[interior] = alpha .* P + beta .* b .* (sum_a G_a^T V_a)   (alpha = beta = 1 without damping) */
static void pressure_update(const problem* pb, double* const* V, double* P, double* tmp) {
  const geom* g = &pb->g;
  memset(tmp, 0, sizeof(double) * g->total);
  for (int a = 0; a < g->dim; ++a) gradT_axis(g, a, V[a], tmp, 1.0);
  if (pb->alpha) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < g->total; ++i) P[i] = pb->alpha[i] * P[i] + pb->beta[i] * pb->b[i] * tmp[i];
  } else {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < g->total; ++i) P[i] += pb->b[i] * tmp[i];
  }
}

void oracle_set_threads(int nthreads) {
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

/* y = K x with the damping rate sigma (N cells, or NULL).  x: N cells; y: ns*nt (sensor-major).
 * Returns 0 on success. */
int oracle_forward_damped(int dim, const int* n, double h, double dt, int nt, int order, const double* c, int ns,
                          const double* sensors, const double* sigma, const double* x, double* y) {
  problem pb;
  int rc = problem_init(&pb, dim, n, h, dt, nt, order, c, ns, sensors);
  if (!rc) rc = set_damping(&pb, sigma);
  if (rc) {
    problem_free(&pb);
    return rc;
  }
  const geom* g = &pb.g;
  double* P = (double*)calloc((size_t)g->total, sizeof(double));
  double* tmp = (double*)calloc((size_t)g->total, sizeof(double));
  double* V[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) V[a] = (double*)calloc((size_t)g->total, sizeof(double));
  to_padded(g, x, P);
  for (int a = 0; a < dim; ++a) grad_axis(g, a, P, V[a], -0.5 * dt / h);
  sample(&pb, P, y, 0);
  for (int step = 1; step < nt; ++step) {
    pressure_update(&pb, V, P, tmp);
    sample(&pb, P, y, step);
    if (step < nt - 1)
      for (int a = 0; a < dim; ++a) grad_axis(g, a, P, V[a], -dt / h);
  }
  for (int a = 0; a < dim; ++a) free(V[a]);
  free(P);
  free(tmp);
  problem_free(&pb);
  return 0;
}

int oracle_forward(int dim, const int* n, double h, double dt, int nt, int order, const double* c, int ns,
                   const double* sensors, const double* x, double* y) {
  return oracle_forward_damped(dim, n, h, dt, nt, order, c, ns, sensors, NULL, x, y);
}

/* x = K* y, the reverse sweep of oracle_forward_damped. */
int oracle_adjoint_damped(int dim, const int* n, double h, double dt, int nt, int order, const double* c, int ns,
                          const double* sensors, const double* sigma, const double* y, double* x) {
  problem pb;
  int rc = problem_init(&pb, dim, n, h, dt, nt, order, c, ns, sensors);
  if (!rc) rc = set_damping(&pb, sigma);
  if (rc) {
    problem_free(&pb);
    return rc;
  }
  const geom* g = &pb.g;
  double* Pb = (double*)calloc((size_t)g->total, sizeof(double));
  double* bP = (double*)calloc((size_t)g->total, sizeof(double));
  double* tmp = (double*)calloc((size_t)g->total, sizeof(double));
  double* Vb[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) Vb[a] = (double*)calloc((size_t)g->total, sizeof(double));
  for (int step = nt - 1; step >= 1; --step) {
    /* transpose of  v -= (dt/h) G P^step  (present when step < nt-1) */
    if (step < nt - 1) {
      memset(tmp, 0, sizeof(double) * g->total);
      for (int a = 0; a < dim; ++a) gradT_axis(g, a, Vb[a], tmp, 1.0);
#pragma omp parallel for schedule(static)
      for (long i = 0; i < g->total; ++i) Pb[i] -= (dt / h) * tmp[i];
    }
    /* transpose of  y_step = S P^step */
    inject(&pb, y, Pb, step);
    /* transpose of  P^step = alpha .* P^{step-1} + beta .* b .* G^T v :
     * v_bar += G (beta .* b .* P_bar), then P_bar <- alpha .* P_bar */
    if (pb.alpha) {
#pragma omp parallel for schedule(static)
      for (long i = 0; i < g->total; ++i) {
        bP[i] = pb.beta[i] * pb.b[i] * Pb[i];
        Pb[i] *= pb.alpha[i];
      }
    } else {
#pragma omp parallel for schedule(static)
      for (long i = 0; i < g->total; ++i) bP[i] = pb.b[i] * Pb[i];
    }
    for (int a = 0; a < dim; ++a) grad_axis(g, a, bP, Vb[a], 1.0);
  }
  inject(&pb, y, Pb, 0);
  /* transpose of  v^{1/2} = -(dt/2h) G P^0 */
  memset(tmp, 0, sizeof(double) * g->total);
  for (int a = 0; a < dim; ++a) gradT_axis(g, a, Vb[a], tmp, 1.0);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < g->total; ++i) Pb[i] -= 0.5 * (dt / h) * tmp[i];
  from_padded(g, Pb, x);
  for (int a = 0; a < dim; ++a) free(Vb[a]);
  free(Pb);
  free(bP);
  free(tmp);
  problem_free(&pb);
  return 0;
}

int oracle_adjoint(int dim, const int* n, double h, double dt, int nt, int order, const double* c, int ns,
                   const double* sensors, const double* y, double* x) {
  return oracle_adjoint_damped(dim, n, h, dt, nt, order, c, ns, sensors, NULL, y, x);
}

/* Medium gradient: g = d<r, K x>/d kappa per cell, kappa = (c dt/h)^2 (undamped program).
 *
 * kappa enters the program only through b = c^2 dt / h = kappa h / dt in
 * P^n = P^{n-1} + b .* (G^T v^{n-1/2}).  Reversing the program as in
 * oracle_adjoint while also collecting the explicit dependence on b gives
 *   d<r, y>/db = sum_{n=1}^{nt-1} Pbar^n .* (G^T v^{n-1/2}),
 * with Pbar^n the adjoint of P^n at the point of that update; then
 * d/dkappa = (h/dt) d/db.  The velocities v^{n-1/2} of the forward run are
 * kept in memory (small problems only). */
int oracle_kappa_grad(int dim, const int* n, double h, double dt, int nt, int order, const double* c, int ns,
                      const double* sensors, const double* x, const double* r, double* g) {
  problem pb;
  int rc = problem_init(&pb, dim, n, h, dt, nt, order, c, ns, sensors);
  if (rc) {
    problem_free(&pb);
    return rc;
  }
  const geom* gm = &pb.g;
  const long total = gm->total;
  /* forward run, storing G^T v^{n-1/2} (on cells) for n = 1..nt-1 */
  double* P = (double*)calloc((size_t)total, sizeof(double));
  double* V[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) V[a] = (double*)calloc((size_t)total, sizeof(double));
  double* GTv = (double*)calloc((size_t)total * (nt > 1 ? nt : 1), sizeof(double));
  to_padded(gm, x, P);
  for (int a = 0; a < dim; ++a) grad_axis(gm, a, P, V[a], -0.5 * dt / h);
  for (int step = 1; step < nt; ++step) {
    double* gtv = GTv + (long)step * total;
    for (int a = 0; a < dim; ++a) gradT_axis(gm, a, V[a], gtv, 1.0);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < total; ++i) P[i] += pb.b[i] * gtv[i];
    if (step < nt - 1)
      for (int a = 0; a < dim; ++a) grad_axis(gm, a, P, V[a], -dt / h);
  }
  /* reverse sweep (as oracle_adjoint) with the explicit b-derivative */
  double* Pb = (double*)calloc((size_t)total, sizeof(double));
  double* bP = (double*)calloc((size_t)total, sizeof(double));
  double* tmp = (double*)calloc((size_t)total, sizeof(double));
  double* gb = (double*)calloc((size_t)total, sizeof(double));
  double* Vb[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) Vb[a] = (double*)calloc((size_t)total, sizeof(double));
  for (int step = nt - 1; step >= 1; --step) {
    if (step < nt - 1) {
      memset(tmp, 0, sizeof(double) * total);
      for (int a = 0; a < dim; ++a) gradT_axis(gm, a, Vb[a], tmp, 1.0);
#pragma omp parallel for schedule(static)
      for (long i = 0; i < total; ++i) Pb[i] -= (dt / h) * tmp[i];
    }
    inject(&pb, r, Pb, step);
    const double* gtv = GTv + (long)step * total;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < total; ++i) {
      gb[i] += Pb[i] * gtv[i];
      bP[i] = pb.b[i] * Pb[i];
    }
    for (int a = 0; a < dim; ++a) grad_axis(gm, a, bP, Vb[a], 1.0);
  }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < total; ++i) gb[i] *= h / dt;
  from_padded(gm, gb, g);
  for (int a = 0; a < dim; ++a) {
    free(V[a]);
    free(Vb[a]);
  }
  free(P);
  free(GTv);
  free(Pb);
  free(bP);
  free(tmp);
  free(gb);
  problem_free(&pb);
  return 0;
}

/* Full wavefield history for small problems: P^n for n = 0..nt-1 into
 * hist[n*N + cell], with the damping rate sigma (or NULL).  Used by the
 * energy and closed-form checks. */
int oracle_forward_history_damped(int dim, const int* n, double h, double dt, int nt, int order, const double* c,
                                  const double* sigma, const double* x, double* hist) {
  problem pb;
  int rc = problem_init(&pb, dim, n, h, dt, nt, order, c, 0, NULL);
  if (!rc) rc = set_damping(&pb, sigma);
  if (rc) {
    problem_free(&pb);
    return rc;
  }
  const geom* g = &pb.g;
  const long N = (long)g->n[0] * g->n[1] * g->n[2];
  double* P = (double*)calloc((size_t)g->total, sizeof(double));
  double* tmp = (double*)calloc((size_t)g->total, sizeof(double));
  double* V[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) V[a] = (double*)calloc((size_t)g->total, sizeof(double));
  to_padded(g, x, P);
  for (int a = 0; a < dim; ++a) grad_axis(g, a, P, V[a], -0.5 * dt / h);
  from_padded(g, P, hist);
  for (int step = 1; step < nt; ++step) {
    pressure_update(&pb, V, P, tmp);
    from_padded(g, P, hist + (long)step * N);
    if (step < nt - 1)
      for (int a = 0; a < dim; ++a) grad_axis(g, a, P, V[a], -dt / h);
  }
  for (int a = 0; a < dim; ++a) free(V[a]);
  free(P);
  free(tmp);
  problem_free(&pb);
  return 0;
}

int oracle_forward_history(int dim, const int* n, double h, double dt, int nt, int order, const double* c,
                           const double* x, double* hist) {
  return oracle_forward_history_damped(dim, n, h, dt, nt, order, c, NULL, x, hist);
}
