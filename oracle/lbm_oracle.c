/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the phase-field lattice
 * Boltzmann model for immiscible incompressible N-phase flow
 * (Yuan, Liang, Chai, Shi, arXiv:1904.12553).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this file. It states what one time
 * step of the model computes, node by node, in the order of the paper, and it
 * shares no code, header, table or helper with the CUDA library.
 *
 * Notation follows the paper: phi_i (i = 1..N-1) order parameters, c_k
 * (k = 1..N) volume fractions, rho~_k pure-phase densities, gamma~_k =
 * 1/rho~_k, Gamma = sum gamma~_k, lambda_ij mixing energy coefficients,
 * C_i chemical potentials, g_k (NS) and h^i_k (CH) distributions on D2Q9
 * with c_s^2 = 1/3 and dx = dt = 1. The CH mobility-tuning constant that
 * the paper calls eta_i is named a_i here, so that it does not clash with
 * the interface thickness eta. Indices are 0-based in code (phase 0 is the
 * paper's phase 1, phase N-1 the paper's phase N).
 *
 * Readings of the paper that the text leaves open (all are listed in the
 * design notes of the repository):
 *  - h_i(phi) is Eq. N17 exactly as printed, with the factor
 *    (rho~_i + rho~_N)/2.
 *  - In Eqs. N18 and N29 the phi_j inside the sum over i is read as phi_i.
 *  - Eq. N26 uses phi_i u for equation i; Eq. N23 sums g over k = 1..8.
 *  - The J~u term of Eq. N20_1 is contracted literally as J~_a u_b.
 *  - rho_0 in g_0^eq (Eq. 25) is a free constant; g_0 enters nothing else.
 *  - c -> phi is the inverse of Eqs. N2 and N12.
 *  - grad(rho) is the linear combination of grad(phi_i) implied by Eq. N29.
 *  - Start: h = h^eq(phi, C, u0), g = g^eq(p0, u0), (phi u)_prev = phi u0.
 *  - Walls (wall_y = 1): halfway bounce-back at y = -1/2 and y = ny - 1/2;
 *    stencil ghost rows repeat the adjacent fluid row.
 *  - Eq. N40 is read with -zeta(x + 2c_i): the mean of the central and the
 *    second-order upwind directional differences. As printed (+zeta) the
 *    scheme returns twice the gradient of a linear field.
 *
 * "parity unpinned": none of the functions below; the pins are in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 5
#define ORC_Q 9

/* D2Q9 velocities and weights (Section 3.1, D2Q9 model). */
static const int CX[ORC_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[ORC_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[ORC_Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Opposite direction: c_opp(k) = -c_k. */
static const int OPP[ORC_Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;

/* Model parameters as the paper states them (Sections 2-4). */
typedef struct {
  int32_t N, nx, ny;
  int32_t wall_y;      /* 0 periodic in y, 1 halfway bounce-back walls */
  int32_t grad_scheme; /* 0 central Eq. N31a, 1 mixed Eq. N40 */
  int32_t pad_;
  double rho_t[ORC_MAXN];            /* rho~_k */
  double sigma[ORC_MAXN][ORC_MAXN];  /* sigma_kl */
  double eta;                        /* interface thickness */
  double beta;                       /* <= 0: Eq. N36 */
  double tau_g;                      /* NS relaxation time */
  double tau[ORC_MAXN - 1];          /* CH relaxation times */
  double mob[ORC_MAXN - 1];          /* mobilities m_i */
  double grav[2];                    /* G = rho * grav */
  double rho0;                       /* constant of g_0^eq */
} orc_params;

/* Constants derived once from the parameters. */
typedef struct {
  orc_params p;
  double gam[ORC_MAXN], Gam;             /* Eq. N1 */
  double beta;                           /* Eq. N36 or given */
  double lam[ORC_MAXN - 1][ORC_MAXN - 1];/* Eq. N14-N16 */
  double a[ORC_MAXN - 1];                /* Eq. N30: m_i = a_i cs2 (tau_i-1/2) */
  double bulk;                           /* beta^2 / eta^2 */
  double kap[ORC_MAXN - 1];              /* (1 - N gam_i/Gam)(rho~_i+rho~_N)/2 */
} orc_model;

/* ------------------------------------------------------------------------ */
/* Mixing energy coefficients, Eqs. N14-N16.                                */
/* ------------------------------------------------------------------------ */

/* Coefficient L_i^{kl} of Eq. N15 (l = N) and Eq. N16 (l < N). */
static double L_coef(const orc_params *p, int i, int k, int l) {
  int n = p->N - 1; /* index of phase N */
  double rN = p->rho_t[n];
  if (l == n) {
    if (i == k) return 1.0;
    return rN / (p->rho_t[i] + rN);
  }
  if (i == k) return p->rho_t[k] / (p->rho_t[k] + rN);
  if (i == l) return -p->rho_t[l] / (p->rho_t[l] + rN);
  return 0.0;
}

/* Solve A x = b (n <= 10) by Gaussian elimination with partial pivoting.
 * Returns 0 on success, -1 if a pivot vanishes. */
static int gauss_solve(int n, double A[10][10], double b[10], double x[10]) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (fabs(A[piv][col]) < 1e-300) return -1;
    if (piv != col) {
      for (int c = 0; c < n; ++c) {
        double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t;
      }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      double f = A[r][col] / A[col][col];
      for (int c = col; c < n; ++c) A[r][c] -= f * A[col][c];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < n; ++c) s -= A[r][c] * x[c];
    x[r] = s / A[r][r];
  }
  return 0;
}

/* beta from Eq. N36 unless the caller fixed it. */
double orc_beta(const orc_params *p) {
  if (p->beta > 0.0) return p->beta;
  double smin = INFINITY;
  for (int k = 0; k < p->N; ++k)
    for (int l = k + 1; l < p->N; ++l)
      if (p->sigma[k][l] < smin) smin = p->sigma[k][l];
  return sqrt(3.0 * sqrt(2.0) * smin * p->eta);
}

/* lambda_ij from Eq. N14: one equation per pair k < l, unknowns lambda_ij
 * with i <= j. Writes the full symmetric (N-1)x(N-1) matrix, row-major.
 * Returns 0 on success. */
int orc_lambda(const orc_params *p, double *lam_out) {
  int n = p->N - 1;
  int M = p->N * (p->N - 1) / 2;
  int ui[10], uj[10];
  int u = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) { ui[u] = i; uj[u] = j; ++u; }
  double beta = orc_beta(p);
  double A[10][10], b[10], x[10];
  int row = 0;
  for (int k = 0; k < p->N; ++k)
    for (int l = k + 1; l < p->N; ++l) {
      for (int c = 0; c < M; ++c) {
        double Li = L_coef(p, ui[c], k, l), Lj = L_coef(p, uj[c], k, l);
        A[row][c] = (ui[c] == uj[c]) ? Li * Li : 2.0 * Li * Lj;
      }
      b[row] = 4.5 * p->eta * p->eta / (beta * beta) * p->sigma[k][l] *
               p->sigma[k][l];
      ++row;
    }
  if (gauss_solve(M, A, b, x) != 0) return -1;
  for (int c = 0; c < M; ++c) {
    lam_out[ui[c] * n + uj[c]] = x[c];
    lam_out[uj[c] * n + ui[c]] = x[c];
  }
  return 0;
}

static int model_setup(orc_model *m, const orc_params *p) {
  memset(m, 0, sizeof(*m));
  m->p = *p;
  int N = p->N, n = N - 1;
  if (N < 2 || N > ORC_MAXN) return -1;
  m->Gam = 0.0;
  for (int k = 0; k < N; ++k) {
    m->gam[k] = 1.0 / p->rho_t[k]; /* Eq. N1 */
    m->Gam += m->gam[k];
  }
  m->beta = orc_beta(p);
  double lam[16];
  if (orc_lambda(p, lam) != 0) return -2;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) m->lam[i][j] = lam[i * n + j];
  for (int i = 0; i < n; ++i) {
    m->a[i] = p->mob[i] / (CS2 * (p->tau[i] - 0.5)); /* Eq. N30 */
    m->kap[i] = (1.0 - N * m->gam[i] / m->Gam) *
                (p->rho_t[i] + p->rho_t[n]) / 2.0;
  }
  m->bulk = m->beta * m->beta / (p->eta * p->eta);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Local algebra, Eqs. N12, N17, N18, N29.                                  */
/* ------------------------------------------------------------------------ */

/* Eq. N18 (c_k) and Eq. N29 (rho) from the N-1 order parameters. */
static void volume_fractions(const orc_model *m, const double *phi,
                             double *c, double *rho) {
  const orc_params *p = &m->p;
  int N = p->N, n = N - 1;
  double vp[ORC_MAXN]; /* varphi_j of Eq. N12 */
  for (int j = 0; j < n; ++j)
    vp[j] = 0.5 * (p->rho_t[j] - p->rho_t[n]) +
            0.5 * (p->rho_t[j] + p->rho_t[n]) * phi[j];
  for (int k = 0; k < N; ++k) {
    double s = m->gam[k] / m->Gam;
    for (int j = 0; j < n; ++j)
      s += (m->gam[k] * (k == j ? 1.0 : 0.0) - m->gam[k] * m->gam[j] / m->Gam) *
           vp[j];
    c[k] = s;
  }
  double r = N / m->Gam;
  for (int i = 0; i < n; ++i) r += (1.0 - N * m->gam[i] / m->Gam) * vp[i];
  *rho = r;
}

/* Eq. N17 as printed. */
static void hfun(const orc_model *m, const double *c, double *hf) {
  const orc_params *p = &m->p;
  int N = p->N, n = N - 1;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < N; ++k)
      s += (m->gam[k] * (k == i ? 1.0 : 0.0) - m->gam[k] * m->gam[i] / m->Gam) *
           c[k] * (1.0 - c[k]) * (1.0 - 2.0 * c[k]);
    hf[i] = (p->rho_t[i] + p->rho_t[n]) / 2.0 * s;
  }
}

/* Inverse of Eqs. N2 and N12: phi_i from the volume fractions. */
static void phi_from_c(const orc_params *p, const double *c, double *phi) {
  int n = p->N - 1;
  for (int i = 0; i < n; ++i)
    phi[i] = (2.0 * (p->rho_t[i] * c[i] - p->rho_t[n] * c[n]) -
              (p->rho_t[i] - p->rho_t[n])) /
             (p->rho_t[i] + p->rho_t[n]);
}

/* ------------------------------------------------------------------------ */
/* Equilibria and sources, Eqs. 25, N20_1, N25, N26.                        */
/* ------------------------------------------------------------------------ */

/* s_k(u) of Eq. 25. */
static double s_k(int k, double ux, double uy) {
  double cu = CX[k] * ux + CY[k] * uy;
  double uu = ux * ux + uy * uy;
  return W[k] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* g_k^eq of Eq. 25, k = 0..8. */
void orc_geq(const orc_params *p, double pr, double rho, double ux, double uy,
             double *geq) {
  for (int k = 0; k < ORC_Q; ++k) {
    if (k == 0)
      geq[k] = p->rho0 + pr / CS2 * (W[0] - 1.0) + rho * s_k(0, ux, uy);
    else
      geq[k] = pr / CS2 * W[k] + rho * s_k(k, ux, uy);
  }
}

/* Total-force distribution G_k of Eq. N20_1. T is the tensor in square
 * brackets; the J~u term is the tensor J~_a u_b, contracted as printed. */
void orc_force_dist(double tau_g, double ux, double uy, double Fx, double Fy,
                    double grx, double gry, double Jx, double Jy, double *G) {
  double u[2] = {ux, uy}, F[2] = {Fx, Fy}, gr[2] = {grx, gry}, J[2] = {Jx, Jy};
  double T[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      T[a][b] = u[a] * F[b] + F[a] * u[b] + CS2 * u[a] * gr[b] +
                CS2 * gr[a] * u[b] + J[a] * u[b] / (tau_g - 0.5);
  double ugr = ux * grx + uy * gry;
  for (int k = 0; k < ORC_Q; ++k) {
    double c[2] = {(double)CX[k], (double)CY[k]};
    double cF = c[0] * Fx + c[1] * Fy;
    double QT = 0.0; /* (c c - cs2 I) : T */
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        QT += (c[a] * c[b] - (a == b ? CS2 : 0.0)) * T[a][b];
    G[k] = W[k] * (ugr + cF / CS2 + QT / (2.0 * CS2 * CS2));
  }
}

/* h_k^{i,eq} of Eq. N25 for one phase. */
void orc_heq(double a_i, double phi, double C, double ux, double uy,
             double *heq) {
  for (int k = 0; k < ORC_Q; ++k) {
    if (k == 0)
      heq[k] = phi + (W[0] - 1.0) * a_i * C;
    else
      heq[k] = W[k] * a_i * C +
               W[k] * (CX[k] * phi * ux + CY[k] * phi * uy) / CS2;
  }
}

/* Source R_k of Eq. N26 with the Euler difference of Eq. N27 (dt = 1). */
void orc_source(double tau_i, double phi, double ux, double uy,
                double phi_prev, double ux_prev, double uy_prev, double *R) {
  double dx = phi * ux - phi_prev * ux_prev;
  double dy = phi * uy - phi_prev * uy_prev;
  for (int k = 0; k < ORC_Q; ++k)
    R[k] = (1.0 - 1.0 / (2.0 * tau_i)) * W[k] * (CX[k] * dx + CY[k] * dy) / CS2;
}

/* ------------------------------------------------------------------------ */
/* Field state and the finite-difference stencils, Eqs. N31a, N31b, N40.     */
/* ------------------------------------------------------------------------ */

typedef struct {
  orc_model m;
  int nx, ny;
  long V;
  double *h;        /* h[i][k][y][x], post-stream populations at time t */
  double *g;        /* g[k][y][x], k = 0..8 */
  double *hn, *gn;  /* streaming targets */
  double *phi_prev; /* phi_i at t-1 */
  double *u_prev;   /* u at t-1, [2][y][x] */
  /* per-step work fields */
  double *phi, *c, *rho, *hf, *gphi, *lphi, *C, *gC, *J, *grho, *F, *u, *p;
} orc_state;

/* Neighbour (x+dx, y+dy): periodic in x; in y periodic, or, with walls, the
 * ghost rows repeat the adjacent fluid row. */
static long nb(const orc_state *s, int x, int y, int dx, int dy) {
  int xx = ((x + dx) % s->nx + s->nx) % s->nx;
  int yy = y + dy;
  if (s->m.p.wall_y) {
    if (yy < 0) yy = 0;
    if (yy > s->ny - 1) yy = s->ny - 1;
  } else {
    yy = (yy % s->ny + s->ny) % s->ny;
  }
  return (long)yy * s->nx + xx;
}

/* grad(zeta): Eq. N31a (central) or Eq. N40 (mixed). out[2][V]. */
static void gradient(const orc_state *s, const double *z, double *out) {
  int nx = s->nx, ny = s->ny;
  long V = s->V;
  int mixed = s->m.p.grad_scheme == 1;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      double gx = 0.0, gy = 0.0;
      for (int k = 1; k < ORC_Q; ++k) {
        double d;
        if (!mixed)
          d = (z[nb(s, x, y, CX[k], CY[k])] - z[nb(s, x, y, -CX[k], -CY[k])]) /
              (2.0 * CS2);
        else
          d = (-z[nb(s, x, y, 2 * CX[k], 2 * CY[k])] +
               5.0 * z[nb(s, x, y, CX[k], CY[k])] - 3.0 * z[n] -
               z[nb(s, x, y, -CX[k], -CY[k])]) /
              (4.0 * CS2);
        gx += W[k] * CX[k] * d;
        gy += W[k] * CY[k] * d;
      }
      out[n] = gx;
      out[V + n] = gy;
    }
}

/* laplacian(zeta): Eq. N31b. */
static void laplacian(const orc_state *s, const double *z, double *out) {
  int nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      double l = 0.0;
      for (int k = 1; k < ORC_Q; ++k)
        l += W[k] * (z[nb(s, x, y, CX[k], CY[k])] - 2.0 * z[n] +
                     z[nb(s, x, y, -CX[k], -CY[k])]) /
             CS2;
      out[n] = l;
    }
}

static double *zalloc(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

void orc_destroy(orc_state *s) {
  if (!s) return;
  double *bufs[] = {s->h,  s->g,  s->hn,   s->gn,   s->phi_prev, s->u_prev,
                    s->phi, s->c, s->rho,  s->hf,   s->gphi, s->lphi,
                    s->C,  s->gC, s->J,    s->grho, s->F,    s->u,  s->p};
  for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b) free(bufs[b]);
  free(s);
}

orc_state *orc_create(const orc_params *p) {
  if (p->nx < 1 || p->ny < 1) return NULL;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  if (model_setup(&s->m, p) != 0) { free(s); return NULL; }
  s->nx = p->nx; s->ny = p->ny;
  s->V = (long)p->nx * p->ny;
  int N = p->N, n = N - 1;
  long V = s->V;
  s->h = zalloc(n * ORC_Q * V);  s->hn = zalloc(n * ORC_Q * V);
  s->g = zalloc(ORC_Q * V);      s->gn = zalloc(ORC_Q * V);
  s->phi_prev = zalloc(n * V);   s->u_prev = zalloc(2 * V);
  s->phi = zalloc(n * V);        s->c = zalloc(N * V);
  s->rho = zalloc(V);            s->hf = zalloc(n * V);
  s->gphi = zalloc(2 * n * V);   s->lphi = zalloc(n * V);
  s->C = zalloc(n * V);          s->gC = zalloc(2 * n * V);
  s->J = zalloc(2 * V);          s->grho = zalloc(2 * V);
  s->F = zalloc(2 * V);          s->u = zalloc(2 * V);
  s->p = zalloc(V);
  if (!s->h || !s->hn || !s->g || !s->gn || !s->phi_prev || !s->u_prev ||
      !s->phi || !s->c || !s->rho || !s->hf || !s->gphi || !s->lphi ||
      !s->C || !s->gC || !s->J || !s->grho || !s->F || !s->u || !s->p) {
    orc_destroy(s);
    return NULL;
  }
  return s;
}

/* Copy the derived constants out (for tests): lam[(N-1)^2], a[N-1],
 * beta, Gamma. */
void orc_constants(const orc_state *s, double *lam, double *a, double *beta,
                   double *Gam) {
  int n = s->m.p.N - 1;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) lam[i * n + j] = s->m.lam[i][j];
    a[i] = s->m.a[i];
  }
  *beta = s->m.beta;
  *Gam = s->m.Gam;
}

/* From phi (already in s->phi): c, rho, h_i(c), grad/lap of phi, C_i,
 * grad C_i, J~, grad rho. Steps 2-4 of one time step. */
static void chemical_potentials(orc_state *s) {
  const orc_model *m = &s->m;
  int N = m->p.N, n = N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q) {
    double ph[ORC_MAXN], cc[ORC_MAXN], hf[ORC_MAXN], r;
    for (int i = 0; i < n; ++i) ph[i] = s->phi[i * V + q];
    volume_fractions(m, ph, cc, &r);
    hfun(m, cc, hf);
    for (int k = 0; k < N; ++k) s->c[k * V + q] = cc[k];
    s->rho[q] = r;
    for (int i = 0; i < n; ++i) s->hf[i * V + q] = hf[i];
  }
  for (int i = 0; i < n; ++i) {
    gradient(s, s->phi + i * V, s->gphi + 2 * i * V);
    laplacian(s, s->phi + i * V, s->lphi + i * V);
  }
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q)
    for (int i = 0; i < n; ++i) {
      double Ci = 0.0;
      for (int j = 0; j < n; ++j) Ci -= m->lam[i][j] * s->lphi[j * V + q];
      Ci += m->bulk * s->hf[i * V + q];
      s->C[i * V + q] = Ci;
    }
  for (int i = 0; i < n; ++i) gradient(s, s->C + i * V, s->gC + 2 * i * V);
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q) {
    double Jx = 0.0, Jy = 0.0, rx = 0.0, ry = 0.0;
    for (int i = 0; i < n; ++i) {
      Jx -= m->kap[i] * m->p.mob[i] * s->gC[2 * i * V + q];
      Jy -= m->kap[i] * m->p.mob[i] * s->gC[(2 * i + 1) * V + q];
      rx += m->kap[i] * s->gphi[2 * i * V + q];
      ry += m->kap[i] * s->gphi[(2 * i + 1) * V + q];
    }
    s->J[q] = Jx; s->J[V + q] = Jy;
    s->grho[q] = rx; s->grho[V + q] = ry;
  }
}

/* Step 5: F_s, F, u (Eq. N22_1), p (Eq. N23). */
static void hydrodynamics(orc_state *s) {
  const orc_model *m = &s->m;
  int n = m->p.N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q) {
    double Fx = 0.0, Fy = 0.0;
    for (int i = 0; i < n; ++i) {
      Fx += s->C[i * V + q] * s->gphi[2 * i * V + q];
      Fy += s->C[i * V + q] * s->gphi[(2 * i + 1) * V + q];
    }
    double r = s->rho[q];
    Fx += r * m->p.grav[0];
    Fy += r * m->p.grav[1];
    double mx = 0.0, my = 0.0, sg = 0.0;
    for (int k = 0; k < ORC_Q; ++k) {
      double gk = s->g[k * V + q];
      mx += CX[k] * gk;
      my += CY[k] * gk;
      if (k != 0) sg += gk;
    }
    double ux = (mx + 0.5 * Fx) / r, uy = (my + 0.5 * Fy) / r;
    double ugr = ux * s->grho[q] + uy * s->grho[V + q];
    double pr = CS2 / (1.0 - W[0]) * (sg + 0.5 * ugr + r * s_k(0, ux, uy));
    s->F[q] = Fx; s->F[V + q] = Fy;
    s->u[q] = ux; s->u[V + q] = uy;
    s->p[q] = pr;
  }
}

static void zeroth_moment(orc_state *s) {
  int n = s->m.p.N - 1;
  long V = s->V;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < V; ++q)
    for (int i = 0; i < n; ++i) {
      double f = 0.0;
      for (int k = 0; k < ORC_Q; ++k) f += s->h[(i * ORC_Q + k) * V + q];
      s->phi[i * V + q] = f; /* Eq. N28 */
    }
}

/* Destination of population k leaving node (x, y): periodic in x; in y
 * periodic or halfway bounce-back (same node, opposite direction). */
static void stream_target(const orc_state *s, int x, int y, int k, long *q,
                          int *kk) {
  int xx = ((x + CX[k]) % s->nx + s->nx) % s->nx;
  int yy = y + CY[k];
  if (s->m.p.wall_y && (yy < 0 || yy >= s->ny)) {
    *q = (long)y * s->nx + x;
    *kk = OPP[k];
    return;
  }
  yy = (yy % s->ny + s->ny) % s->ny;
  *q = (long)yy * s->nx + xx;
  *kk = k;
}

/* One time step t -> t+1, in the order of the paper. */
static void step_once(orc_state *s) {
  const orc_model *m = &s->m;
  int n = m->p.N - 1;
  int nx = s->nx, ny = s->ny;
  long V = s->V;
  double tg = m->p.tau_g;
  zeroth_moment(s);        /* 1. phi_i = sum_k h_k^i (Eq. N28) */
  chemical_potentials(s);  /* 2-4. c, rho, C_i, J~, grad rho */
  hydrodynamics(s);        /* 5. F, u, p */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long q = (long)y * nx + x;
      double ux = s->u[q], uy = s->u[V + q];
      /* 6. NS: Eq. 24 with Eq. 25 and Eq. N20_1 */
      double geq[ORC_Q], G[ORC_Q];
      orc_geq(&m->p, s->p[q], s->rho[q], ux, uy, geq);
      orc_force_dist(tg, ux, uy, s->F[q], s->F[V + q], s->grho[q],
                     s->grho[V + q], s->J[q], s->J[V + q], G);
      for (int k = 0; k < ORC_Q; ++k) {
        double gk = s->g[k * V + q];
        double gs = gk - (gk - geq[k]) / tg + (1.0 - 1.0 / (2.0 * tg)) * G[k];
        long t; int kk;
        stream_target(s, x, y, k, &t, &kk); /* 8. streaming */
        s->gn[kk * V + t] = gs;
      }
      /* 7. CH: Eq. N24 with Eq. N25 and Eq. N26 */
      for (int i = 0; i < n; ++i) {
        double heq[ORC_Q], R[ORC_Q];
        double ph = s->phi[i * V + q];
        orc_heq(m->a[i], ph, s->C[i * V + q], ux, uy, heq);
        orc_source(m->p.tau[i], ph, ux, uy, s->phi_prev[i * V + q],
                   s->u_prev[q], s->u_prev[V + q], R);
        for (int k = 0; k < ORC_Q; ++k) {
          double hk = s->h[(i * ORC_Q + k) * V + q];
          double hs = hk - (hk - heq[k]) / m->p.tau[i] + R[k];
          long t; int kk;
          stream_target(s, x, y, k, &t, &kk);
          s->hn[(i * ORC_Q + kk) * V + t] = hs;
        }
      }
    }
  /* 9. (phi u)_prev <- (phi u)(t) */
  memcpy(s->phi_prev, s->phi, sizeof(double) * n * V);
  memcpy(s->u_prev, s->u, sizeof(double) * 2 * V);
  double *t;
  t = s->h; s->h = s->hn; s->hn = t;
  t = s->g; s->g = s->gn; s->gn = t;
}

/* Start from volume fractions c0[N][y][x], velocity u0[2][y][x] (may be
 * NULL = rest) and uniform pressure p0. */
int orc_init(orc_state *s, const double *c0, const double *u0, double p0) {
  const orc_model *m = &s->m;
  int N = m->p.N, n = N - 1;
  long V = s->V;
  for (long q = 0; q < V; ++q) {
    double cc[ORC_MAXN], ph[ORC_MAXN];
    for (int k = 0; k < N; ++k) cc[k] = c0[k * V + q];
    phi_from_c(&m->p, cc, ph);
    for (int i = 0; i < n; ++i) s->phi[i * V + q] = ph[i];
  }
  chemical_potentials(s);
  for (long q = 0; q < V; ++q) {
    double ux = u0 ? u0[q] : 0.0, uy = u0 ? u0[V + q] : 0.0;
    double geq[ORC_Q];
    orc_geq(&m->p, p0, s->rho[q], ux, uy, geq);
    for (int k = 0; k < ORC_Q; ++k) s->g[k * V + q] = geq[k];
    for (int i = 0; i < n; ++i) {
      double heq[ORC_Q];
      orc_heq(m->a[i], s->phi[i * V + q], s->C[i * V + q], ux, uy, heq);
      for (int k = 0; k < ORC_Q; ++k) s->h[(i * ORC_Q + k) * V + q] = heq[k];
      s->phi_prev[i * V + q] = s->phi[i * V + q];
    }
    s->u_prev[q] = ux;
    s->u_prev[V + q] = uy;
  }
  return 0;
}

void orc_step(orc_state *s, long nsteps) {
  for (long t = 0; t < nsteps; ++t) step_once(s);
}

/* Macroscopic fields at the current time: phi[N-1], c[N], u[2], p, rho
 * (each [..][y][x]); any pointer may be NULL. */
void orc_moments(orc_state *s, double *phi, double *c, double *u, double *p,
                 double *rho) {
  int N = s->m.p.N, n = N - 1;
  long V = s->V;
  zeroth_moment(s);
  chemical_potentials(s);
  hydrodynamics(s);
  if (phi) memcpy(phi, s->phi, sizeof(double) * n * V);
  if (c) memcpy(c, s->c, sizeof(double) * N * V);
  if (u) memcpy(u, s->u, sizeof(double) * 2 * V);
  if (p) memcpy(p, s->p, sizeof(double) * V);
  if (rho) memcpy(rho, s->rho, sizeof(double) * V);
}

/* Chemical potentials C_i at the current time, [N-1][y][x]. */
void orc_chemical_potential(orc_state *s, double *C) {
  zeroth_moment(s);
  chemical_potentials(s);
  memcpy(C, s->C, sizeof(double) * (s->m.p.N - 1) * s->V);
}

/* J~ and grad(rho) (Eq. N18) of the current state, [2][y][x] each (for
 * tests; reads only). */
void orc_fluxes(orc_state *s, double *J, double *grho) {
  zeroth_moment(s);
  chemical_potentials(s);
  memcpy(J, s->J, sizeof(double) * 2 * s->V);
  memcpy(grho, s->grho, sizeof(double) * 2 * s->V);
}

/* Per-phase mass sum_x c_k, kinetic energy 1/2 sum rho |u|^2, max |u|,
 * summed serially in node order. */
void orc_diagnostics(orc_state *s, double *mass, double *ke, double *umax) {
  int N = s->m.p.N;
  long V = s->V;
  orc_moments(s, NULL, NULL, NULL, NULL, NULL);
  for (int k = 0; k < N; ++k) {
    double a = 0.0;
    for (long q = 0; q < V; ++q) a += s->c[k * V + q];
    mass[k] = a;
  }
  double e = 0.0, um = 0.0;
  for (long q = 0; q < V; ++q) {
    double u2 = s->u[q] * s->u[q] + s->u[V + q] * s->u[V + q];
    e += 0.5 * s->rho[q] * u2;
    if (sqrt(u2) > um) um = sqrt(u2);
  }
  *ke = e;
  *umax = um;
}

/* Raw state access for tests: h[N-1][9][V], g[9][V], phi_prev, u_prev. */
void orc_get_state(const orc_state *s, double *h, double *g, double *phi_prev,
                   double *u_prev) {
  int n = s->m.p.N - 1;
  long V = s->V;
  if (h) memcpy(h, s->h, sizeof(double) * n * ORC_Q * V);
  if (g) memcpy(g, s->g, sizeof(double) * ORC_Q * V);
  if (phi_prev) memcpy(phi_prev, s->phi_prev, sizeof(double) * n * V);
  if (u_prev) memcpy(u_prev, s->u_prev, sizeof(double) * 2 * V);
}

void orc_set_state(orc_state *s, const double *h, const double *g,
                   const double *phi_prev, const double *u_prev) {
  int n = s->m.p.N - 1;
  long V = s->V;
  memcpy(s->h, h, sizeof(double) * n * ORC_Q * V);
  memcpy(s->g, g, sizeof(double) * ORC_Q * V);
  memcpy(s->phi_prev, phi_prev, sizeof(double) * n * V);
  memcpy(s->u_prev, u_prev, sizeof(double) * 2 * V);
}

/* Stencils on one field (for tests): grad -> out[2][V], lap -> out[V]. */
void orc_stencils(orc_state *s, const double *z, double *grad, double *lap) {
  if (grad) gradient(s, z, grad);
  if (lap) laplacian(s, z, lap);
}

/* Local algebra on one node (for tests). */
void orc_local_fractions(orc_state *s, const double *phi, double *c,
                         double *rho, double *hf) {
  volume_fractions(&s->m, phi, c, rho);
  if (hf) hfun(&s->m, c, hf);
}

void orc_local_phi_from_c(const orc_params *p, const double *c, double *phi) {
  phi_from_c(p, c, phi);
}

int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
