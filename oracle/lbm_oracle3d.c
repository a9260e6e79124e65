/*
 * lbm_oracle3d.c -- plain, slow FP64 CPU oracle of the N-phase phase-field
 * lattice Boltzmann model (Yuan, Liang, Chai, Shi, arXiv:1904.12553) on the
 * D3Q15 lattice that the paper lists for three dimensions (Section 3.1).
 *
 * TEST INFRASTRUCTURE, like lbm_oracle.c: only the tests, the smoke check
 * and the benchmark's CPU-baseline leg use it; it shares nothing with the
 * CUDA library. The time step follows the paper's order exactly as the 2-D
 * oracle does (same readings of the paper), with every lattice sum running
 * over the 15 D3Q15 velocities and the stencils of Eq. N31 over their 14
 * neighbours. Grids are nx x ny x nz, periodic in x and z; y is periodic or
 * bounded by halfway bounce-back walls (ghost layers repeat the adjacent
 * fluid layer). Arrays are [field][z][y][x].
 *
 * "parity unpinned": none; the pins are in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O3_MAXN 5
#define O3_Q 15

/* D3Q15 velocities and weights (Section 3.1). */
static const int CX[O3_Q] = {0, 1, 0, 0, -1, 0, 0, 1, 1, 1, -1, -1, -1, -1, 1};
static const int CY[O3_Q] = {0, 0, 1, 0, 0, -1, 0, 1, 1, -1, 1, -1, -1, 1, -1};
static const int CZ[O3_Q] = {0, 0, 0, 1, 0, 0, -1, 1, -1, 1, 1, -1, 1, -1, -1};
static const double W[O3_Q] = {2.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                               1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 72.0,
                               1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
                               1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0};
static const double CS2 = 1.0 / 3.0;

/* Model parameters (Sections 2-4); nz is the third grid dimension. */
typedef struct {
  int32_t N, nx, ny, nz;
  int32_t wall_y;
  int32_t pad_;
  double rho_t[O3_MAXN];
  double sigma[O3_MAXN][O3_MAXN];
  double eta, beta, tau_g;
  double tau[O3_MAXN - 1], mob[O3_MAXN - 1];
  double grav[3];
  double rho0;
} o3_params;

typedef struct {
  o3_params p;
  double gam[O3_MAXN], Gam, beta;
  double lam[O3_MAXN - 1][O3_MAXN - 1];
  double a[O3_MAXN - 1], bulk, kap[O3_MAXN - 1];
} o3_model;

static int opp(int k) {
  for (int j = 0; j < O3_Q; ++j)
    if (CX[j] == -CX[k] && CY[j] == -CY[k] && CZ[j] == -CZ[k]) return j;
  return -1;
}

/* Eqs. N14-N16 by Gaussian elimination (as the 2-D oracle). */
static double L_coef(const o3_params *p, int i, int k, int l) {
  int n = p->N - 1;
  double rN = p->rho_t[n];
  if (l == n) return i == k ? 1.0 : rN / (p->rho_t[i] + rN);
  if (i == k) return p->rho_t[k] / (p->rho_t[k] + rN);
  if (i == l) return -p->rho_t[l] / (p->rho_t[l] + rN);
  return 0.0;
}

static double beta_of(const o3_params *p) {
  if (p->beta > 0.0) return p->beta;
  double smin = INFINITY;
  for (int k = 0; k < p->N; ++k)
    for (int l = k + 1; l < p->N; ++l)
      if (p->sigma[k][l] < smin) smin = p->sigma[k][l];
  return sqrt(3.0 * sqrt(2.0) * smin * p->eta); /* Eq. N36 */
}

static int solve_lambda(const o3_params *p, double beta, double lam[4][4]) {
  int n = p->N - 1, M = p->N * (p->N - 1) / 2, ui[10], uj[10], u = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) { ui[u] = i; uj[u] = j; ++u; }
  double A[10][10], b[10], x[10];
  int row = 0;
  for (int k = 0; k < p->N; ++k)
    for (int l = k + 1; l < p->N; ++l) {
      for (int c = 0; c < M; ++c) {
        double Li = L_coef(p, ui[c], k, l), Lj = L_coef(p, uj[c], k, l);
        A[row][c] = ui[c] == uj[c] ? Li * Li : 2.0 * Li * Lj;
      }
      b[row] = 4.5 * p->eta * p->eta / (beta * beta) * p->sigma[k][l] *
               p->sigma[k][l];
      ++row;
    }
  for (int col = 0; col < M; ++col) {
    int piv = col;
    for (int r = col + 1; r < M; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (fabs(A[piv][col]) < 1e-300) return -1;
    for (int c = 0; c < M; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
    { double t = b[col]; b[col] = b[piv]; b[piv] = t; }
    for (int r = col + 1; r < M; ++r) {
      double f = A[r][col] / A[col][col];
      for (int c = col; c < M; ++c) A[r][c] -= f * A[col][c];
      b[r] -= f * b[col];
    }
  }
  for (int r = M - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < M; ++c) s -= A[r][c] * x[c];
    x[r] = s / A[r][r];
  }
  for (int c = 0; c < M; ++c) { lam[ui[c]][uj[c]] = x[c]; lam[uj[c]][ui[c]] = x[c]; }
  return 0;
}

static int setup(o3_model *m, const o3_params *p) {
  memset(m, 0, sizeof(*m));
  m->p = *p;
  int N = p->N, n = N - 1;
  if (N < 2 || N > O3_MAXN) return -1;
  for (int k = 0; k < N; ++k) { m->gam[k] = 1.0 / p->rho_t[k]; m->Gam += m->gam[k]; }
  m->beta = beta_of(p);
  if (solve_lambda(p, m->beta, m->lam) != 0) return -2;
  for (int i = 0; i < n; ++i) {
    m->a[i] = p->mob[i] / (CS2 * (p->tau[i] - 0.5)); /* Eq. N30 */
    m->kap[i] = (1.0 - N * m->gam[i] / m->Gam) * (p->rho_t[i] + p->rho_t[n]) / 2.0;
  }
  m->bulk = m->beta * m->beta / (p->eta * p->eta);
  return 0;
}

/* Eqs. N12, N18, N29 and N17 (as printed). */
static void fractions(const o3_model *m, const double *phi, double *c,
                      double *rho, double *hf) {
  const o3_params *p = &m->p;
  int N = p->N, n = N - 1;
  double vp[O3_MAXN];
  for (int j = 0; j < n; ++j)
    vp[j] = 0.5 * (p->rho_t[j] - p->rho_t[n]) + 0.5 * (p->rho_t[j] + p->rho_t[n]) * phi[j];
  for (int k = 0; k < N; ++k) {
    double s = m->gam[k] / m->Gam;
    for (int j = 0; j < n; ++j)
      s += (m->gam[k] * (k == j ? 1.0 : 0.0) - m->gam[k] * m->gam[j] / m->Gam) * vp[j];
    c[k] = s;
  }
  double r = N / m->Gam;
  for (int i = 0; i < n; ++i) r += (1.0 - N * m->gam[i] / m->Gam) * vp[i];
  *rho = r;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < N; ++k)
      s += (m->gam[k] * (k == i ? 1.0 : 0.0) - m->gam[k] * m->gam[i] / m->Gam) *
           c[k] * (1.0 - c[k]) * (1.0 - 2.0 * c[k]);
    hf[i] = (p->rho_t[i] + p->rho_t[n]) / 2.0 * s;
  }
}

static double s_k(int k, const double *u) {
  double cu = CX[k] * u[0] + CY[k] * u[1] + CZ[k] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return W[k] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 25 on D3Q15. */
void o3_geq(double rho0, double pr, double rho, const double *u, double *geq) {
  for (int k = 0; k < O3_Q; ++k)
    geq[k] = (k == 0 ? rho0 + pr / CS2 * (W[0] - 1.0) : pr / CS2 * W[k]) + rho * s_k(k, u);
}

/* Eq. N20_1 on D3Q15 (J~u contracted as the tensor J~_a u_b). */
void o3_force_dist(double tau_g, const double *u, const double *F,
                   const double *gr, const double *J, double *G) {
  double T[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      T[a][b] = u[a] * F[b] + F[a] * u[b] + CS2 * u[a] * gr[b] + CS2 * gr[a] * u[b] +
                J[a] * u[b] / (tau_g - 0.5);
  double ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
  for (int k = 0; k < O3_Q; ++k) {
    double c[3] = {(double)CX[k], (double)CY[k], (double)CZ[k]};
    double cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2], QT = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) QT += (c[a] * c[b] - (a == b ? CS2 : 0.0)) * T[a][b];
    G[k] = W[k] * (ugr + cF / CS2 + QT / (2.0 * CS2 * CS2));
  }
}

/* Eq. N25 on D3Q15. */
void o3_heq(double a_i, double phi, double C, const double *u, double *heq) {
  for (int k = 0; k < O3_Q; ++k)
    heq[k] = k == 0 ? phi + (W[0] - 1.0) * a_i * C
                    : W[k] * a_i * C +
                          W[k] * (CX[k] * phi * u[0] + CY[k] * phi * u[1] + CZ[k] * phi * u[2]) / CS2;
}

/* Eqs. N26, N27 on D3Q15. */
void o3_source(double tau_i, double phi, const double *u, double phi_prev,
               const double *u_prev, double *R) {
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = phi * u[a] - phi_prev * u_prev[a];
  for (int k = 0; k < O3_Q; ++k)
    R[k] = (1.0 - 1.0 / (2.0 * tau_i)) * W[k] * (CX[k] * d[0] + CY[k] * d[1] + CZ[k] * d[2]) / CS2;
}

typedef struct {
  o3_model m;
  int nx, ny, nz;
  long V;
  double *h, *g, *hn, *gn, *phi_prev, *u_prev;
  double *phi, *c, *rho, *hf, *gphi, *lphi, *C, *gC, *J, *grho, *F, *u, *p;
} o3_state;

static long node(const o3_state *s, int x, int y, int z) {
  return ((long)z * s->ny + y) * s->nx + x;
}

/* Neighbour (x+dx, y+dy, z+dz) with the boundary rules of the grid. */
static long nb(const o3_state *s, int x, int y, int z, int dx, int dy, int dz) {
  int xx = ((x + dx) % s->nx + s->nx) % s->nx;
  int zz = ((z + dz) % s->nz + s->nz) % s->nz;
  int yy = y + dy;
  if (s->m.p.wall_y) {
    if (yy < 0) yy = 0;
    if (yy > s->ny - 1) yy = s->ny - 1;
  } else {
    yy = (yy % s->ny + s->ny) % s->ny;
  }
  return node(s, xx, yy, zz);
}

/* Eq. N31a (out[3][V]) and Eq. N31b (out[V]) with the D3Q15 stencil. */
static void gradient(const o3_state *s, const double *zf, double *out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        double g[3] = {0, 0, 0};
        for (int k = 1; k < O3_Q; ++k) {
          double d = (zf[nb(s, x, y, z, CX[k], CY[k], CZ[k])] -
                      zf[nb(s, x, y, z, -CX[k], -CY[k], -CZ[k])]) / (2.0 * CS2);
          g[0] += W[k] * CX[k] * d;
          g[1] += W[k] * CY[k] * d;
          g[2] += W[k] * CZ[k] * d;
        }
        long q = node(s, x, y, z);
        for (int a = 0; a < 3; ++a) out[a * s->V + q] = g[a];
      }
}

static void laplacian(const o3_state *s, const double *zf, double *out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        long q = node(s, x, y, z);
        double l = 0.0;
        for (int k = 1; k < O3_Q; ++k)
          l += W[k] * (zf[nb(s, x, y, z, CX[k], CY[k], CZ[k])] - 2.0 * zf[q] +
                       zf[nb(s, x, y, z, -CX[k], -CY[k], -CZ[k])]) / CS2;
        out[q] = l;
      }
}

static double *za(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

void o3_destroy(o3_state *s) {
  if (!s) return;
  double *b[] = {s->h, s->g, s->hn, s->gn, s->phi_prev, s->u_prev, s->phi, s->c,
                 s->rho, s->hf, s->gphi, s->lphi, s->C, s->gC, s->J, s->grho,
                 s->F, s->u, s->p};
  for (size_t i = 0; i < sizeof(b) / sizeof(b[0]); ++i) free(b[i]);
  free(s);
}

o3_state *o3_create(const o3_params *p) {
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
  o3_state *s = (o3_state *)calloc(1, sizeof(o3_state));
  if (!s) return NULL;
  if (setup(&s->m, p) != 0) { free(s); return NULL; }
  s->nx = p->nx; s->ny = p->ny; s->nz = p->nz;
  long V = s->V = (long)p->nx * p->ny * p->nz;
  int N = p->N, n = N - 1;
  s->h = za(n * O3_Q * V); s->hn = za(n * O3_Q * V);
  s->g = za(O3_Q * V); s->gn = za(O3_Q * V);
  s->phi_prev = za(n * V); s->u_prev = za(3 * V);
  s->phi = za(n * V); s->c = za(N * V); s->rho = za(V); s->hf = za(n * V);
  s->gphi = za(3 * n * V); s->lphi = za(n * V); s->C = za(n * V);
  s->gC = za(3 * n * V); s->J = za(3 * V); s->grho = za(3 * V);
  s->F = za(3 * V); s->u = za(3 * V); s->p = za(V);
  if (!s->h || !s->hn || !s->g || !s->gn || !s->phi_prev || !s->u_prev || !s->phi ||
      !s->c || !s->rho || !s->hf || !s->gphi || !s->lphi || !s->C || !s->gC || !s->J ||
      !s->grho || !s->F || !s->u || !s->p) {
    o3_destroy(s);
    return NULL;
  }
  return s;
}

static void zeroth_moment(o3_state *s) {
  int n = s->m.p.N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q)
    for (int i = 0; i < n; ++i) {
      double f = 0.0;
      for (int k = 0; k < O3_Q; ++k) f += s->h[(i * O3_Q + k) * V + q];
      s->phi[i * V + q] = f; /* Eq. N28 */
    }
}

/* c, rho, h_i, stencils, C_i (Eq. N18), grad C_i, J~, grad rho. */
static void chemical_potentials(o3_state *s) {
  const o3_model *m = &s->m;
  int N = m->p.N, n = N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q) {
    double ph[O3_MAXN], cc[O3_MAXN], hf[O3_MAXN], r;
    for (int i = 0; i < n; ++i) ph[i] = s->phi[i * V + q];
    fractions(m, ph, cc, &r, hf);
    for (int k = 0; k < N; ++k) s->c[k * V + q] = cc[k];
    s->rho[q] = r;
    for (int i = 0; i < n; ++i) s->hf[i * V + q] = hf[i];
  }
  for (int i = 0; i < n; ++i) {
    gradient(s, s->phi + i * V, s->gphi + 3 * i * V);
    laplacian(s, s->phi + i * V, s->lphi + i * V);
  }
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q)
    for (int i = 0; i < n; ++i) {
      double Ci = 0.0;
      for (int j = 0; j < n; ++j) Ci -= m->lam[i][j] * s->lphi[j * V + q];
      s->C[i * V + q] = Ci + m->bulk * s->hf[i * V + q];
    }
  for (int i = 0; i < n; ++i) gradient(s, s->C + i * V, s->gC + 3 * i * V);
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q)
    for (int a = 0; a < 3; ++a) {
      double J = 0.0, gr = 0.0;
      for (int i = 0; i < n; ++i) {
        J -= m->kap[i] * m->p.mob[i] * s->gC[(3 * i + a) * V + q];
        gr += m->kap[i] * s->gphi[(3 * i + a) * V + q];
      }
      s->J[a * V + q] = J;
      s->grho[a * V + q] = gr;
    }
}

/* F, u (Eq. N22_1), p (Eq. N23). */
static void hydrodynamics(o3_state *s) {
  const o3_model *m = &s->m;
  int n = m->p.N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q) {
    double F[3], mo[3] = {0, 0, 0}, sg = 0.0, r = s->rho[q];
    for (int a = 0; a < 3; ++a) {
      F[a] = r * m->p.grav[a];
      for (int i = 0; i < n; ++i) F[a] += s->C[i * V + q] * s->gphi[(3 * i + a) * V + q];
    }
    for (int k = 0; k < O3_Q; ++k) {
      double gk = s->g[k * V + q];
      mo[0] += CX[k] * gk; mo[1] += CY[k] * gk; mo[2] += CZ[k] * gk;
      if (k != 0) sg += gk;
    }
    double u[3], ugr = 0.0;
    for (int a = 0; a < 3; ++a) {
      u[a] = (mo[a] + 0.5 * F[a]) / r;
      ugr += u[a] * s->grho[a * V + q];
      s->F[a * V + q] = F[a];
      s->u[a * V + q] = u[a];
    }
    s->p[q] = CS2 / (1.0 - W[0]) * (sg + 0.5 * ugr + r * s_k(0, u));
  }
}

static void target(const o3_state *s, int x, int y, int z, int k, long *q, int *kk) {
  int yy = y + CY[k];
  if (s->m.p.wall_y && (yy < 0 || yy >= s->ny)) {
    *q = node(s, x, y, z);
    *kk = opp(k);
    return;
  }
  *q = nb(s, x, y, z, CX[k], CY[k], CZ[k]);
  *kk = k;
}

static void step_once(o3_state *s) {
  const o3_model *m = &s->m;
  int n = m->p.N - 1;
  long V = s->V;
  double tg = m->p.tau_g;
  zeroth_moment(s);
  chemical_potentials(s);
  hydrodynamics(s);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        long q = node(s, x, y, z);
        double u[3], F[3], gr[3], J[3], up[3];
        for (int a = 0; a < 3; ++a) {
          u[a] = s->u[a * V + q]; F[a] = s->F[a * V + q];
          gr[a] = s->grho[a * V + q]; J[a] = s->J[a * V + q];
          up[a] = s->u_prev[a * V + q];
        }
        double geq[O3_Q], G[O3_Q];
        o3_geq(m->p.rho0, s->p[q], s->rho[q], u, geq);
        o3_force_dist(tg, u, F, gr, J, G);
        for (int k = 0; k < O3_Q; ++k) {
          double gk = s->g[k * V + q];
          long t; int kk;
          target(s, x, y, z, k, &t, &kk);
          s->gn[kk * V + t] = gk - (gk - geq[k]) / tg + (1.0 - 1.0 / (2.0 * tg)) * G[k];
        }
        for (int i = 0; i < n; ++i) {
          double heq[O3_Q], R[O3_Q], ph = s->phi[i * V + q];
          o3_heq(m->a[i], ph, s->C[i * V + q], u, heq);
          o3_source(m->p.tau[i], ph, u, s->phi_prev[i * V + q], up, R);
          for (int k = 0; k < O3_Q; ++k) {
            double hk = s->h[(i * O3_Q + k) * V + q];
            long t; int kk;
            target(s, x, y, z, k, &t, &kk);
            s->hn[(i * O3_Q + kk) * V + t] = hk - (hk - heq[k]) / m->p.tau[i] + R[k];
          }
        }
      }
  memcpy(s->phi_prev, s->phi, sizeof(double) * n * V);
  memcpy(s->u_prev, s->u, sizeof(double) * 3 * V);
  double *t;
  t = s->h; s->h = s->hn; s->hn = t;
  t = s->g; s->g = s->gn; s->gn = t;
}

int o3_init(o3_state *s, const double *c0, const double *u0, double p0) {
  const o3_model *m = &s->m;
  int N = m->p.N, n = N - 1;
  long V = s->V;
  for (long q = 0; q < V; ++q)
    for (int i = 0; i < n; ++i) {
      double ci = c0[i * V + q], cN = c0[n * V + q];
      s->phi[i * V + q] =
          (2.0 * (m->p.rho_t[i] * ci - m->p.rho_t[n] * cN) - (m->p.rho_t[i] - m->p.rho_t[n])) /
          (m->p.rho_t[i] + m->p.rho_t[n]);
    }
  chemical_potentials(s);
  for (long q = 0; q < V; ++q) {
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = u0 ? u0[a * V + q] : 0.0;
    double geq[O3_Q];
    o3_geq(m->p.rho0, p0, s->rho[q], u, geq);
    for (int k = 0; k < O3_Q; ++k) s->g[k * V + q] = geq[k];
    for (int i = 0; i < n; ++i) {
      double heq[O3_Q];
      o3_heq(m->a[i], s->phi[i * V + q], s->C[i * V + q], u, heq);
      for (int k = 0; k < O3_Q; ++k) s->h[(i * O3_Q + k) * V + q] = heq[k];
      s->phi_prev[i * V + q] = s->phi[i * V + q];
    }
    for (int a = 0; a < 3; ++a) s->u_prev[a * V + q] = u[a];
  }
  return 0;
}

void o3_step(o3_state *s, long nsteps) {
  for (long t = 0; t < nsteps; ++t) step_once(s);
}

void o3_moments(o3_state *s, double *phi, double *c, double *u, double *p, double *rho) {
  int N = s->m.p.N, n = N - 1;
  long V = s->V;
  zeroth_moment(s);
  chemical_potentials(s);
  hydrodynamics(s);
  if (phi) memcpy(phi, s->phi, sizeof(double) * n * V);
  if (c) memcpy(c, s->c, sizeof(double) * N * V);
  if (u) memcpy(u, s->u, sizeof(double) * 3 * V);
  if (p) memcpy(p, s->p, sizeof(double) * V);
  if (rho) memcpy(rho, s->rho, sizeof(double) * V);
}

/* The populations h[N-1][15][V] and g[15][V] of the current state (for
 * tests; reads only). */
void o3_populations(const o3_state *s, double *h, double *g) {
  long V = s->V;
  memcpy(h, s->h, sizeof(double) * (s->m.p.N - 1) * O3_Q * V);
  memcpy(g, s->g, sizeof(double) * O3_Q * V);
}

/* C_i, J~ and grad(rho) (Eq. N18) of the current state (for tests; reads
 * only): C[N-1][V], J[3][V], grho[3][V]. */
void o3_fluxes(o3_state *s, double *C, double *J, double *grho) {
  int n = s->m.p.N - 1;
  long V = s->V;
  zeroth_moment(s);
  chemical_potentials(s);
  memcpy(C, s->C, sizeof(double) * n * V);
  memcpy(J, s->J, sizeof(double) * 3 * V);
  memcpy(grho, s->grho, sizeof(double) * 3 * V);
}

void o3_stencils(o3_state *s, const double *zf, double *grad, double *lap) {
  if (grad) gradient(s, zf, grad);
  if (lap) laplacian(s, zf, lap);
}

int o3_sizeof_params(void) { return (int)sizeof(o3_params); }
