/*
 * lbm_nphase.h -- C ABI of the GB300 (sm_103a) phase-field lattice Boltzmann
 * solver for immiscible incompressible N-phase flow, after Yuan, Liang, Chai
 * and Shi, "Phase-field-based lattice Boltzmann model for immiscible
 * incompressible N-phase flows" (arXiv:1904.12553).
 *
 * One handle owns one D2Q9 grid of nx x ny nodes with N phases (2 <= N <= 5):
 * N-1 Cahn-Hilliard distributions h^i_k (Eq. N24) and one Navier-Stokes
 * distribution g_k (Eq. 24) per node. A time step computes the chemical
 * potentials C_i from the isotropic stencils of Eq. N31, the total force
 * F = sum_i C_i grad(phi_i) + G, the moments u (Eq. N22_1) and p (Eq. N23),
 * the collisions with the equilibria of Eqs. 25 and N25, the total-force
 * distribution of Eq. N20_1 and the source of Eqs. N26-N27, and streams the
 * populations. Lattice units: dx = dt = 1, c_s^2 = 1/3.
 *
 * Conventions for every function below:
 *  - Arrays are row-major [field][y][x] (D2Q9) or [field][z][y][x] (D3Q15)
 *    with x fastest, FP64, nodes at integer coordinates. Field order: phases
 *    1..N (the paper's indices); velocity fields have D = 2 or 3 components.
 *  - Device work is ordered on the CUDA stream given to lbm_nphase_create
 *    (NULL = the legacy default stream). lbm_nphase_step is asynchronous;
 *    lbm_nphase_init, lbm_nphase_moments and lbm_nphase_diagnostics return
 *    after their results are complete (they synchronise the stream).
 *  - A handle is not thread safe. The library never frees caller memory; the
 *    workspace must outlive the handle.
 *  - Functions never abort or exit; they return an lbm_status. After
 *    LBM_EUNSTABLE the handle refuses lbm_nphase_step (LBM_ESTATE) until
 *    lbm_nphase_init is called again.
 */
#ifndef LBM_NPHASE_H
#define LBM_NPHASE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_N 5

typedef struct lbm_nphase_t lbm_nphase_t; /* opaque; owns all device state */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* invalid argument or parameter set */
  LBM_ENOMEM = 2,    /* workspace too small */
  LBM_ECUDA = 3,     /* a CUDA call failed (see lbm_nphase_cuda_error) */
  LBM_ETIMEOUT = 4,  /* a bounded device wait gave up (reported by the next
                        lbm_nphase_moments or lbm_nphase_diagnostics) */
  LBM_EUNSTABLE = 5, /* non-finite mass or kinetic energy detected */
  LBM_ESTATE = 6     /* call not valid in the handle's current state */
} lbm_status;

typedef enum {
  LBM_FP64 = 0,     /* FP64 storage and arithmetic */
  LBM_FP32 = 1,     /* FP32 storage and arithmetic */
  LBM_MIX_BF16 = 2, /* moving populations stored as BF16 s (h_k/w_k - 3 c_k.u phi_i)
                       and s (g_k/w_k - 3 p - rho~ (3 c_k.u + 4.5 (c_k.u)^2
                       - 1.5 |u|^2)), rho~ = N/Gamma, with u, p and phi_i at
                       t - 1 of the node the population was streamed from
                       (D2Q9 and D3Q15); FP32 math */
  LBM_MIX_FP16 = 3  /* the same with FP16 storage; FP32 math */
} lbm_precision;

/* Model parameters, as the paper states them (Sections 2-4). */
typedef struct {
  int32_t N;           /* number of phases, 2..5 */
  int32_t nx, ny;      /* grid size, >= 1 each; nx <= 2^20; D2Q9:
                          ny <= 524280, D3Q15: ny <= 262140 (the generic
                          kernels' launch grid); nx*ny*nz <= 2^34 */
  int32_t nz;          /* third dimension of a D3Q15 grid (1..131070); D2Q9:
                          0 or 1 */
  int32_t lattice;     /* 0: D2Q9 (two dimensions); 1: D3Q15 (three; Section
                          3.1), central scheme only */
  int32_t wall_y;      /* 0: periodic in y; 1: halfway bounce-back walls at
                          y = -1/2 and y = ny - 1/2 (Section 4.2). x (and z)
                          are always periodic. */
  int32_t precision;   /* lbm_precision */
  int32_t grad_scheme; /* first derivatives: 0 isotropic central scheme,
                          Eq. N31a; 1 isotropic mixed scheme, Eq. N40, read
                          with -zeta(x + 2c_i) (the Laplacian is Eq. N31b
                          either way). 1 runs on the generic kernel. */
  double rho[LBM_MAX_N];              /* pure-phase densities rho~_k > 0 */
  double sigma[LBM_MAX_N][LBM_MAX_N]; /* pairwise surface tensions sigma_kl
                                         > 0, symmetric; diagonal ignored */
  double eta;          /* interface thickness; tanh profile width sqrt(2) eta */
  double beta;         /* <= 0: beta = sqrt(3 sqrt(2) sigma_min eta), Eq. N36 */
  double tau_g;        /* NS relaxation time > 1/2; nu = (tau_g - 1/2)/3, Eq. N21_1 */
  double tau[LBM_MAX_N - 1];      /* CH relaxation times tau_i > 1/2 */
  double mobility[LBM_MAX_N - 1]; /* m_i > 0; a_i = m_i / (c_s^2 (tau_i - 1/2)), Eq. N30 */
  double gravity[3];   /* body force G = rho * gravity (x, y, z) */
  double rho0;         /* constant of g_0^eq (Eq. 25); it affects no output */
} lbm_nphase_params;

/* Constants derived on the host from the parameters. */
typedef struct {
  double lambda[LBM_MAX_N - 1][LBM_MAX_N - 1]; /* lambda_ij, Eqs. N14-N16 */
  double lambda_eig_min, lambda_eig_max;       /* extreme eigenvalues */
  double beta;                                 /* Eq. N36 or given */
  double a[LBM_MAX_N - 1];                     /* a_i of Eq. N30 */
  double Gamma;                                /* sum 1/rho~_k, Eq. N1 */
  double nu;                                   /* Eq. N21_1 */
  int32_t uniform_density;                     /* 1 if all rho~_k are equal */
  int32_t pad_;
} lbm_nphase_model;

/* Validate a parameter set and derive its constants on the host (no GPU
 * needed). lambda comes from the N(N-1)/2 equations of Eq. N14 with the
 * coefficients of Eqs. N15/N16. Returns LBM_EINVAL if a parameter is out of
 * range, sigma is not symmetric, or lambda is singular or not positive
 * definite. `out` may be NULL (validation only). */
lbm_status lbm_nphase_derive(const lbm_nphase_params *params,
                             lbm_nphase_model *out);

/* Bytes of device workspace a handle with these parameters needs (0 if the
 * parameters are invalid). */
size_t lbm_nphase_workspace_bytes(const lbm_nphase_params *params);

/* Create a handle on the current CUDA device. `d_workspace` is caller-owned
 * device memory of at least lbm_nphase_workspace_bytes() bytes, 256-byte
 * aligned; `cuda_stream` is a cudaStream_t (NULL: default stream). No device
 * computation happens here. Errors: LBM_EINVAL (parameters, NULL arguments,
 * misaligned workspace), LBM_ENOMEM (workspace too small), LBM_ECUDA. */
lbm_status lbm_nphase_create(const lbm_nphase_params *params,
                             void *d_workspace, size_t workspace_bytes,
                             void *cuda_stream, lbm_nphase_t **out);

/* Initial state from volume fractions c[N][(nz)][ny][nx] (Eq. N2,
 * sum_k c_k = 1) and velocity u[D][(nz)][ny][nx] (NULL: fluid at rest),
 * uniform pressure p0.
 * Pointers may be host or device memory. The order parameters follow from
 * the inverse of Eqs. N2 and N12; the distributions start at equilibrium,
 * h = h^eq(phi, C, u) (Eq. N25) and g = g^eq(p0, u) (Eq. 25), and the
 * previous-step product of Eq. N27 starts at phi u. Synchronises. */
lbm_status lbm_nphase_init(lbm_nphase_t *h, const double *c, const double *u,
                           double p0);

/* Advance nsteps >= 0 time steps (asynchronous on the handle's stream). Each
 * step is one fused kernel: zeroth moments (Eq. N28), chemical potentials
 * (Eqs. N17, N18, N31), forces, u and p (Eqs. N22_1, N23), both
 * collisions (Eqs. 24, N24) and streaming. From nsteps >= 4 on, pairs of
 * steps are replayed from a CUDA graph captured on the handle's first such
 * call (on a private stream; call it outside any capture of your own).
 * Errors: LBM_ESTATE before init or after LBM_EUNSTABLE, LBM_ECUDA. */
lbm_status lbm_nphase_step(lbm_nphase_t *h, int64_t nsteps);

/* Macroscopic fields at the current time: phi[N-1], c[N], u[D], p, rho,
 * each field [(nz)][ny][nx] (Eqs. N28, N18, N22_1, N23, N29).
 * Any pointer may be NULL; non-NULL pointers may be host or device memory.
 * Synchronises. */
lbm_status lbm_nphase_moments(lbm_nphase_t *h, double *phi, double *c,
                              double *u, double *p, double *rho);

/* FP64 conservation diagnostics at the current time, reduced on the GPU in a
 * fixed order: mass[k] = sum_x c_k (N values), ke = 1/2 sum_x rho |u|^2,
 * umax = max_x |u|. Host pointers; any may be NULL. Returns LBM_EUNSTABLE
 * (and marks the handle) if a result is not finite. Synchronises. */
lbm_status lbm_nphase_diagnostics(lbm_nphase_t *h, double *mass, double *ke,
                                  double *umax);

/* The same diagnostics as lbm_nphase_diagnostics, for callers that cannot
 * allocate device memory at this point (for example code running where a
 * cudaMalloc would synchronise the device or is forbidden by an allocator
 * policy). It allocates nothing: its scratch (the per-tile partial sums and
 * the reduced values) is a 1 MiB static device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * The paper has no counterpart; this is a library convenience.
 *  - Limit: at most 16384 partial sums, one per tile of the grid: tiles of
 *    32 x 8 nodes on D2Q9 (e.g. 2048 x 2048) and of 32 x 4 x 2 nodes on
 *    D3Q15 (e.g. 128 x 128 x 256). Larger grids return LBM_EINVAL.
 *  - The handle's device must be current. The first call on a device looks
 *    up the array's device address; make that first call before any stream
 *    capture.
 *  - All calls in the process share the array and it keeps the last call's
 *    contents: calls that overlap on the GPU (other streams, other handles
 *    on the same device) race. Each call writes every slot it reads, so
 *    nothing needs clearing between calls.
 * Returns and synchronises like lbm_nphase_diagnostics. */
lbm_status lbm_nphase_diagnostics_static(lbm_nphase_t *h, double *mass,
                                         double *ke, double *umax);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent grids advanced together.
 *
 * Cases may differ in size, N, walls and parameters; all use FP32 storage
 * and equal pure-phase densities (J~ = 0). Each time step of the whole batch
 * is one persistent kernel launch that walks a list of (case, tile) work
 * items; steps are replayed from a CUDA graph captured at schedule time.
 * ------------------------------------------------------------------------ */
typedef struct lbm_nphase_batch_t lbm_nphase_batch_t;

typedef struct {
  int32_t tile_height; /* 4 or 8 rows of 32 nodes per work item */
  int32_t schedule;    /* 0: CTA b takes items b, b + ctas, ... of the
                          cost-ordered list; 1: per-CTA contiguous runs of
                          equal cost; 2: items taken from an atomic counter */
  int32_t ctas;        /* persistent CTAs (0: all that are resident) */
  int32_t pipelined;   /* 1: TMA-pipelined tile body (32 x 8 tiles, the next
                          item's populations loaded while the current one is
                          computed; tile_height is then 8); needs every case
                          to satisfy the pipelined kernel's conditions
                          (nx a multiple of 8, lbm_nphase_uses_pipelined_kernel
                          true for it), else LBM_EINVAL */
  int32_t chunk;       /* dynamic schedule: consecutive items taken per
                          atomic grab (0 means 1); ignored otherwise */
} lbm_nphase_batch_schedule;

/* Workspace for `ncases` grids described by params[0..ncases-1] (0 if a
 * parameter set is invalid, not FP32, or has unequal densities). */
size_t lbm_nphase_batch_workspace_bytes(const lbm_nphase_params *params,
                                        int ncases);

/* Create the batch in caller-owned device memory (256-byte aligned) on the
 * current device; work is ordered on `cuda_stream`. The initial schedule is
 * {8, 2, 0, 0, 1}. Errors as lbm_nphase_create. */
lbm_status lbm_nphase_batch_create(const lbm_nphase_params *params, int ncases,
                                   void *d_workspace, size_t workspace_bytes,
                                   void *cuda_stream, lbm_nphase_batch_t **out);

/* Initial state of case `c`, as lbm_nphase_init. Every case must be
 * initialised before lbm_nphase_batch_step. */
lbm_status lbm_nphase_batch_init(lbm_nphase_batch_t *b, int c, const double *c0,
                                 const double *u, double p0);

/* Advance every case by nsteps time steps (asynchronous): one persistent
 * launch per step, two steps per graph replay. */
lbm_status lbm_nphase_batch_step(lbm_nphase_batch_t *b, int64_t nsteps);

/* Handle of case `c` (owned by the batch; do not destroy). Use it with
 * lbm_nphase_moments and lbm_nphase_diagnostics. Stepping it alone with
 * lbm_nphase_step takes it out of step with the batch (lbm_nphase_batch_step
 * then returns LBM_ESTATE until the case is re-initialised). */
lbm_nphase_t *lbm_nphase_batch_case(lbm_nphase_batch_t *b, int c);

/* Macroscopic fields and diagnostics of case `c`: lbm_nphase_moments and
 * lbm_nphase_diagnostics on its handle (same arguments, layout and errors;
 * LBM_EINVAL for a case index outside 0..size-1). */
lbm_status lbm_nphase_batch_moments(lbm_nphase_batch_t *b, int c, double *phi,
                                    double *cfrac, double *u, double *p,
                                    double *rho);
lbm_status lbm_nphase_batch_diagnostics(lbm_nphase_batch_t *b, int c,
                                        double *mass, double *ke,
                                        double *umax);

/* Time every kernel variant (generic at tile heights 4 and 8, and the
 * pipelined kernel when every case allows it) x schedule (strided, lists,
 * dynamic with chunks of 1, 4 and 16), with all resident CTAs, over
 * 2 * trial_steps steps each and keep the fastest; its time per step goes to
 * *best_ms_per_step (may be NULL). The trials advance the cases' state by
 * 2 * (trial_steps + 1) steps per candidate (10 or 15 candidates):
 * re-initialise afterwards for a clean run. */
lbm_status lbm_nphase_batch_autotune(lbm_nphase_batch_t *b, int trial_steps,
                                     double *best_ms_per_step);

/* Set or read the schedule explicitly (rebuilds the work lists and graphs). */
lbm_status lbm_nphase_batch_set_schedule(lbm_nphase_batch_t *b,
                                         const lbm_nphase_batch_schedule *s);
lbm_status lbm_nphase_batch_get_schedule(const lbm_nphase_batch_t *b,
                                         lbm_nphase_batch_schedule *s);

/* Number of cases. */
int lbm_nphase_batch_size(const lbm_nphase_batch_t *b);

/* Release the batch and its case handles (not the workspace). NULL ok. */
lbm_status lbm_nphase_batch_destroy(lbm_nphase_batch_t *b);

/* Checkpoint / resume. The state at the current time (distributions,
 * phi(t-1), u(t-1) and a 64-byte header with N, nx, ny, precision and the
 * step count) as one blob of lbm_nphase_state_bytes() bytes, in host or
 * device memory. lbm_nphase_set_state accepts a blob of a handle with the
 * same N, grid, lattice, precision, walls and gradient scheme (else
 * LBM_EINVAL) and leaves the handle
 * initialised at that state; continuing from it reproduces the uninterrupted
 * run bit for bit. Both synchronise. Not part of the paper. */
size_t lbm_nphase_state_bytes(const lbm_nphase_t *h);
lbm_status lbm_nphase_get_state(lbm_nphase_t *h, void *dst, size_t bytes);
lbm_status lbm_nphase_set_state(lbm_nphase_t *h, const void *src, size_t bytes);

/* Number of time steps taken since the last init. */
int64_t lbm_nphase_steps_taken(const lbm_nphase_t *h);

/* Which kernel lbm_nphase_step runs for this handle: 1 the TMA-pipelined
 * D2Q9 kernel (FP32 and 16-bit forms, equal pure-phase densities, nx a
 * multiple of 8), 2 the z-marching D3Q15 kernel (equal densities, every
 * storage form), 3 the z-marching D3Q15 kernel with TMA-staged planes (FP32,
 * equal densities, N <= 4, nx a multiple of 4), 0 the generic tile kernel. Setting the environment variable
 * LBM_NPHASE_KERNEL=generic before lbm_nphase_create selects the generic
 * kernels everywhere. All compute the same step. */
int lbm_nphase_uses_pipelined_kernel(const lbm_nphase_t *h);

/* Self-test of the timeout path (not part of the paper). Launches, on the
 * handle's stream, one warp that waits with the library's bounded device
 * wait (about a second) on a barrier nothing signals; when the wait gives up
 * it sets the handle's device error word, exactly as a pipelined step kernel
 * whose copies never arrived would. The next lbm_nphase_moments or
 * lbm_nphase_diagnostics then returns LBM_ETIMEOUT and marks the handle, and
 * lbm_nphase_step returns LBM_ESTATE until lbm_nphase_init. Asynchronous;
 * faults nothing and leaves the context usable. */
lbm_status lbm_nphase_selftest_wait_timeout(lbm_nphase_t *h);

/* The last CUDA error code seen by the handle (0 if none). */
int lbm_nphase_cuda_error(const lbm_nphase_t *h);

/* Release the handle (not the workspace). NULL is accepted. */
lbm_status lbm_nphase_destroy(lbm_nphase_t *h);

/* Static description of a status code. */
const char *lbm_nphase_strerror(lbm_status s);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NPHASE_H */
