// Internal interface between the C-ABI host code and the per-precision CUDA
// kernel translation units. Not part of the public API.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (types only; no driver link)
#include <cuda_runtime.h>
#include <stddef.h>

#include "lbm_nphase.h"

namespace lbm {

constexpr int BX = 32;  // tile width (one warp along x)
constexpr int BY = 8;   // tile height
constexpr int NT = BX * BY;

enum Mode { MODE_STEP = 0, MODE_MOMENTS = 1, MODE_DIAG = 2 };

// Model constants in FP64; each precision unit converts them to its type.
// Index conventions: i, j over the N-1 order parameters; k over N phases.
struct Consts {
  int N, NP;
  double lam[4][4];    // lambda_ij (Eq. N14)
  double bulk;         // beta^2 / eta^2
  double a[4];         // a_i (Eq. N30)
  double tau_inv[4];   // 1 / tau_i
  double src[4];       // 1 - 1/(2 tau_i) (Eq. N26)
  double tg_inv;       // 1 / tau_g
  double ffac;         // 1 - 1/(2 tau_g) (Eq. 24)
  double jfac;         // 1 / (tau_g - 1/2) (Eq. N20_1)
  double grav[3];      // G = rho * grav
  double off[4], mul[4];  // varphi_j = off_j + mul_j phi_j (Eq. N12)
  double c0[5];        // gamma~_k / Gamma (Eq. N18)
  double Q[5][4];      // gamma~_k delta_kj - gamma~_k gamma~_j / Gamma
  double rho_base;     // N / Gamma (Eq. N29)
  double K[4];         // 1 - N gamma~_i / Gamma
  double kap[4];       // K_i mul_i: grad rho = sum kap_i grad phi_i
  double kmob[4];      // kap_i m_i: J~ = -sum kmob_i grad C_i
  double rho_t[5];     // rho~_k (initialisation)
  double sh, sg;       // 16-bit storage scales of h_k / w_k and g_k / w_k
};

// TMA descriptors of one state buffer for the pipelined step kernel.
struct TmaMaps {
  CUtensorMap hm, h0, pp, gm, up;
  // FP32 pipelined kernel: the halo column and row that wrap around a
  // periodic grid (boxes of 16 bytes x the box height, and one row x the
  // box width, of the h, d_0 and phi(t-1) arrays)
  CUtensorMap hmx, h0x, ppx, hmy, h0y, ppy;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType,
                                  cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

// Device state of one grid. Buffers [0] and [1] alternate every step.
struct Grid {
  int nx, ny, nz;   // nz = 1 for D2Q9
  int lattice;      // 0 D2Q9, 1 D3Q15
  size_t V;
  void *h0[2];      // rest slots: h^i_0 (FP64) or h^i_0 - phi_i(t-1): [N-1][V]
  void *hm[2];      // moving populations h^i_k, k = 1..8: [N-1][8][V]
  void *gm[2];      // NS populations g_k, k = 1..8: [8][V]
  void *phi_prev[2];  // phi_i(t-1): [N-1][V]
  void *u_prev[2];  // u(t-1): [D][V] (16-bit forms: [D + 1][V], p(t-1) last),
                    // ping-pong like phi_prev
  double *red;      // per-block partial sums of the diagnostics
  double *red_out;  // N + 2 reduced diagnostics
  int *err;         // device error word (1: a bounded wait gave up)
  double *scratch;  // FP64 staging of host inputs and outputs ([N + D][V]);
                    // initialisation keeps phi_i there ([N-1][V])
  int grad_scheme;  // 0: central (Eq. N31a), 1: mixed (Eq. N40)
  bool use_tma;     // pipelined kernel usable for this grid
  bool march3;      // D3Q15 step by the z-marching kernel
  bool tma3;        // ... with its planes staged by TMA (tma[] holds 4-D maps)
  TmaMaps tma[2];   // its descriptors, input buffer 0 or 1
};

struct Outputs {
  double *phi, *c, *u, *p, *rho;
};

// Launchers, one set per precision (lbm_fp64.cu, lbm_fp32.cu, lbm_mixed.cu).
// prec is an lbm_precision value; `cur` selects the input buffer.
cudaError_t launch_tile(int prec, const Consts &k, const Grid &g, int cur,
                        int mode, const Outputs &o, bool nonunif, bool wall,
                        cudaStream_t s);
cudaError_t launch_init(int prec, const Consts &k, const Grid &g, int cur,
                        const double *c, const double *u, double p0, bool wall,
                        cudaStream_t s);
cudaError_t launch_reduce(const Grid &g, int nparts, int nvals, cudaStream_t s);

#define LBM_DECLARE_PREC(SUFFIX)                                              \
  cudaError_t launch_tile_##SUFFIX(const Consts &, const Grid &, int, int,    \
                                   const Outputs &, bool, bool, cudaStream_t);\
  cudaError_t launch_init_##SUFFIX(const Consts &, const Grid &, int,         \
                                   const double *, const double *, double,    \
                                   bool, cudaStream_t);                       \
  bool encode_tma_##SUFFIX(const Consts &, Grid &, EncodeTiledFn);           \
  bool encode_tma3_##SUFFIX(const Consts &, Grid &, EncodeTiledFn);          \
  cudaError_t launch_tile3_##SUFFIX(const Consts &, const Grid &, int, int,   \
                                    const Outputs &, bool, bool, cudaStream_t);\
  cudaError_t launch_init3_##SUFFIX(const Consts &, const Grid &, int,        \
                                    const double *, const double *, double,   \
                                    bool, cudaStream_t);
LBM_DECLARE_PREC(f64)
LBM_DECLARE_PREC(f32)
LBM_DECLARE_PREC(bf16)
LBM_DECLARE_PREC(f16)
#undef LBM_DECLARE_PREC

inline int tiles_x(int nx) { return (nx + BX - 1) / BX; }
inline int tiles_y(int ny) { return (ny + BY - 1) / BY; }
// D3Q15 tiles: 32 x 4 x 2 nodes
inline int tiles3_x(int nx) { return (nx + 31) / 32; }
inline int tiles3_y(int ny) { return (ny + 3) / 4; }
inline int tiles3_z(int nz) { return (nz + 1) / 2; }
// CTAs of the generic step / moments / diagnostics kernel of a grid
inline size_t tiles_total(int lattice, int nx, int ny, int nz) {
  return lattice == 1 ? (size_t)tiles3_x(nx) * tiles3_y(ny) * tiles3_z(nz)
                      : (size_t)tiles_x(nx) * tiles_y(ny);
}

}  // namespace lbm

// One grid's handle (the opaque type of the C ABI).
struct lbm_nphase_t {
  lbm_nphase_params prm;
  lbm_nphase_model mdl;
  lbm::Consts k;
  lbm::Grid g;
  int prec;
  bool nonunif, wall;
  cudaStream_t stream;
  int device;
  double *stage;  // (N + 2) * V doubles: host <-> device staging
  int cur;        // buffer holding the state at the current time
  bool initialized, unstable;
  int64_t steps;
  int cuda_err;
  cudaStream_t cap;            // private stream for graph capture
  cudaGraphExec_t gexec[2];    // two steps starting at buffer 0 / 1
};

namespace lbm {
// lbm_nphase_init with the start state written into buffer `cur` (0 or 1),
// so that grids stepped together keep the same buffer parity.
lbm_status init_at(lbm_nphase_t *h, const double *c, const double *u,
                   double p0, int cur);
}  // namespace lbm
