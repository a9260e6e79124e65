// Fused time-step kernels of the N-phase phase-field lattice Boltzmann model
// (Yuan, Liang, Chai, Shi, arXiv:1904.12553) for sm_103a.
//
// Data layout (structure of arrays, x fastest, one plane per population):
//   h0[i][V]        rest population h^i_0 of order parameter i
//   hm[i][k-1][V]   moving populations h^i_k, k = 1..8
//   gm[k-1][V]      NS populations g_k, k = 1..8 (g_0 never influences u, p
//                   or phi: u has c_0 = 0 and Eq. N23 sums k >= 1)
//   phi_prev[2][i][V]   phi_i(t-1) (Eq. N27), ping-pong; u_prev[2][2][V] the same
//                   for u(t-1) (16-bit forms: [2][3][V], p(t-1) third)
// The stored populations are post-streaming values at their node (push
// scheme), so phi_i(x) = sum_k h^i_k(x) is local (Eq. N28).
//
// FP64 stores the rest population h^i_0 itself. The FP32 and 16-bit forms
// store d^i_0 = h^i_0 - phi_i(t-1) instead, a value of the size of the moving
// populations, and carry in it the exact rounding error of phi_i: the node's
// mass phi_prev + d_0 + sum_k h_k is then conserved by the collision up to
// the rounding of d_0 (~1e-11), where an O(1) FP32 rest slot would lose
// ~6e-8 per node and step, systematically in a near-steady state.
//
// One CTA owns a BX x BY tile. It sums the populations of the tile and of a
// halo ring of radius R into shared memory (phi), evaluates the stencils of
// Eq. N31 there, and for every own node computes C_i (Eqs. N17, N18),
// F = sum C_i grad phi_i + rho G, u (Eq. N22_1), p (Eq. N23), the NS
// collision (Eq. 24, Eq. 25, Eq. N20_1), the CH collisions (Eq. N24, Eq. N25,
// Eqs. N26-N27), and pushes the post-collision populations to the
// neighbours (periodic, or halfway bounce-back at y walls). With unequal
// pure-phase densities, J~ needs grad C_i, so the CTA also evaluates C on a
// ring of radius 1 and phi on a ring of radius 2 (R = 2).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "lbm_internal.h"

namespace lbm {

// D2Q9 (Section 3.1): k = 0 rest; 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1);
// 5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1).
__host__ __device__ constexpr int cx_of(int k) {
  return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int k) {
  return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int k) {
  return k == 0 ? 0 : (k <= 4 ? ((k + 1) % 4) + 1 : ((k - 5 + 2) % 4) + 5);
}
template <typename T>
__host__ __device__ constexpr T w_of(int k) {
  return k == 0 ? T(4) / T(9) : (k <= 4 ? T(1) / T(9) : T(1) / T(36));
}
static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 &&
                  opp_of(4) == 2 && opp_of(5) == 7 && opp_of(6) == 8 &&
                  opp_of(7) == 5 && opp_of(8) == 6,
              "opposite directions");

// Storage policy per precision. MIX: 16-bit moving populations in stored
// units s f_k / w_k. REF: stored relative to the advective part of their
// equilibrium (for g also its pressure part) at their source node (both
// 16-bit forms: without it BF16 misses the 1e-3 phi target on colliding drops
// by 13x and FP16 on a resting lens by up to 5x; without the pressure part
// BF16 drifts past it on small resting drops).
template <int P> struct Prec;
template <> struct Prec<LBM_FP64> {
  typedef double T;
  typedef double Sm;
  static constexpr bool MIX = false, REF = false;
};
template <> struct Prec<LBM_FP32> {
  typedef float T;
  typedef float Sm;
  static constexpr bool MIX = false, REF = false;
};
template <> struct Prec<LBM_MIX_BF16> {
  typedef float T;
  typedef __nv_bfloat16 Sm;
  static constexpr bool MIX = true, REF = true;
};
template <> struct Prec<LBM_MIX_FP16> {
  typedef float T;
  typedef __half Sm;
  static constexpr bool MIX = true, REF = true;
};

__device__ __forceinline__ float __fadd_rn_T(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double __fadd_rn_T(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float to_T(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_T(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_T(float v) { return v; }
__device__ __forceinline__ double to_T(double v) { return v; }
template <typename S> __device__ __forceinline__ S to_S(float v);
// FP32 -> BF16, round to nearest with ties to even, in integer arithmetic:
// add half an ulp of the target (0x7FFF) plus the lowest kept bit, then
// truncate the low 16 bits. Exact for every finite value (overflow rounds
// to infinity); on GB300 it ran the BF16 step 40% faster than the
// conversion instruction.
template <> __device__ __forceinline__ __nv_bfloat16 to_S(float v) {
  unsigned u = __float_as_uint(v);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return __ushort_as_bfloat16((unsigned short)(u >> 16));
}
template <> __device__ __forceinline__ __half to_S(float v) { return __float2half_rn(v); }
// Two values at once with the packed conversion (round to nearest even, the
// same bits as to_S): one instruction for two stores of the 16-bit forms.
__device__ __forceinline__ void to_S2(float a, float b, __nv_bfloat16 &ra, __nv_bfloat16 &rb) {
  const __nv_bfloat162 r = __floats2bfloat162_rn(a, b); ra = r.x; rb = r.y; }
__device__ __forceinline__ void to_S2(float a, float b, __half &ra, __half &rb) {
  const __half2 r = __floats2half2_rn(a, b); ra = r.x; rb = r.y; }
__device__ __forceinline__ void to_S2(float a, float b, float &ra, float &rb) { ra = a; rb = b; }
__device__ __forceinline__ void to_S2(double a, double b, double &ra, double &rb) { ra = a; rb = b; }
template <> __device__ __forceinline__ float to_S(float v) { return v; }
template <typename S> __device__ __forceinline__ S to_S(double v) { return v; }

// Kernel arguments: pointers of one step and the model constants in T.
template <int P> struct alignas(16) KArgs {  // 16: bulk-copy granule
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  int nx, ny;
  size_t V;
  const T *h0_in;
  const Sm *hm_in, *gm_in;
  T *h0_out;
  Sm *hm_out, *gm_out;
  const T *pp_in;  // phi_prev at t-1
  T *pp_out;       // phi_prev for the next step (phi at t)
  const T *u_in;   // u(t-1)
  T *u_out;        // u(t) for the next step
  double *o_phi, *o_c, *o_u, *o_p, *o_rho, *red;
  int *err;
  int mode;
  T lam[4][4], bulk, a[4], tau_inv[4], src[4], tg_inv, ffac, jfac, grav[2], grav_z;
  T off[4], mul[4], c0[5], Q[5][4], rho_base, K[4], kap[4], kmob[4];
  T sh_ld, sh_st, sg_ld, sg_st;  // 16-bit storage: value = S * w_k * ld
};

template <int P>
KArgs<P> make_args(const Consts &c, const Grid &g, int cur, int mode,
                   const Outputs &o) {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  KArgs<P> a;
  a.nx = g.nx;
  a.ny = g.ny;
  a.V = g.V;
  a.h0_in = (const T *)g.h0[cur];
  a.hm_in = (const Sm *)g.hm[cur];
  a.gm_in = (const Sm *)g.gm[cur];
  a.h0_out = (T *)g.h0[cur ^ 1];
  a.hm_out = (Sm *)g.hm[cur ^ 1];
  a.gm_out = (Sm *)g.gm[cur ^ 1];
  a.pp_in = (const T *)g.phi_prev[cur];
  a.pp_out = (T *)g.phi_prev[cur ^ 1];
  a.u_in = (const T *)g.u_prev[cur];
  a.u_out = (T *)g.u_prev[cur ^ 1];
  a.o_phi = o.phi;
  a.o_c = o.c;
  a.o_u = o.u;
  a.o_p = o.p;
  a.o_rho = o.rho;
  a.red = g.red;
  a.err = g.err;
  a.mode = mode;
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) a.lam[i][j] = (T)c.lam[i][j];
    a.a[i] = (T)c.a[i];
    a.tau_inv[i] = (T)c.tau_inv[i];
    a.src[i] = (T)c.src[i];
    a.off[i] = (T)c.off[i];
    a.mul[i] = (T)c.mul[i];
    a.K[i] = (T)c.K[i];
    a.kap[i] = (T)c.kap[i];
    a.kmob[i] = (T)c.kmob[i];
  }
  for (int k = 0; k < 5; ++k) {
    a.c0[k] = (T)c.c0[k];
    for (int j = 0; j < 4; ++j) a.Q[k][j] = (T)c.Q[k][j];
  }
  a.bulk = (T)c.bulk;
  a.tg_inv = (T)c.tg_inv;
  a.ffac = (T)c.ffac;
  a.jfac = (T)c.jfac;
  a.grav[0] = (T)c.grav[0];
  a.grav[1] = (T)c.grav[1];
  a.grav_z = (T)c.grav[2];
  a.rho_base = (T)c.rho_base;
  a.sh_ld = (T)(1.0 / c.sh);
  a.sh_st = (T)c.sh;
  a.sg_ld = (T)(1.0 / c.sg);
  a.sg_st = (T)c.sg;
  return a;
}

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Moving population k (1..8) of phase i, or NS population k, at node q as
// stored: the value itself (FP64, FP32) or, 16-bit forms, s f_k / w_k less
// the source-relative reference below (load_h_node, load_g_node add it).
template <int P>
__device__ __forceinline__ typename Prec<P>::T load_hm(const KArgs<P> &a, int i,
                                                       int k, size_t q) {
  return to_T(ldg(a.hm_in + ((size_t)(i * 8 + k - 1)) * a.V + q));
}
template <int P>
__device__ __forceinline__ typename Prec<P>::T load_gm(const KArgs<P> &a, int k,
                                                       size_t q) {
  return to_T(ldg(a.gm_in + ((size_t)(k - 1)) * a.V + q));
}

// 16-bit forms: every moving population is stored relative to part of its
// equilibrium (Eqs. 25, N25) evaluated at the node it was streamed from:
// slot k of node y holds
//     s h_k / w_k - 3 s (c_k . u) phi_i                               (h, phase i)
//     s g_k / w_k - s (3 p + rho~ (3 c_k.u + 4.5 (c_k.u)^2 - 1.5 |u|^2))  (g)
// (rho~ = the constant N/Gamma)
// with u = u(t), p = p(t), phi = phi(t) of the source node y - c_k (of y
// itself when y - c_k lies behind a wall: the slot was filled by bounce-back).
// The writer uses its own u(t), p(t), phi(t); the reader takes them as
// u(t-1), p(t-1), phi(t-1) of the source. The subtracted part is the bulk of
// a population (in a moving flow the advective part; at rest 3p of g), so
// the 16-bit value keeps its significant bits for the rest. Both sides
// compute it with the same rounded operations (no contraction), so a value
// decodes to exactly what its writer counted in the node's mass balance.
__device__ __forceinline__ float cdotu(int k, float ux, float uy) {
  const int cx = cx_of(k), cy = cy_of(k);
  const float a = cx > 0 ? ux : -ux, b = cy > 0 ? uy : -uy;
  return cx != 0 && cy != 0 ? __fadd_rn(a, b) : (cx != 0 ? a : b);
}
__device__ __forceinline__ double cdotu(int k, double ux, double uy) {
  return cx_of(k) * ux + cy_of(k) * uy;
}
// 3 s (c_k . u) f in stored units; s3 = 3 s.
__device__ __forceinline__ float adv_units(float cu, float f, float s3) {
  return __fmul_rn(__fmul_rn(cu, f), s3);
}
__device__ __forceinline__ double adv_units(double cu, double f, double s3) {
  return cu * f * s3;
}
// s rho~ (3 c_k.u + 4.5 (c_k.u)^2 - 1.5 |u|^2) in stored units; srho = s rho~.
__device__ __forceinline__ float g_ref(float cu, float ux, float uy, float srho) {
  const float uu = __fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy));
  const float in = __fadd_rn(__fadd_rn(__fmul_rn(3.0f, cu), __fmul_rn(4.5f, __fmul_rn(cu, cu))),
                             __fmul_rn(-1.5f, uu));
  return __fmul_rn(in, srho);
}
__device__ __forceinline__ double g_ref(double cu, double ux, double uy,
                                        double srho) {
  return (3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)) * srho;
}
// The same plus the pressure part 3 s p of the equilibrium; s3 = 3 s.
__device__ __forceinline__ float g_refp(float cu, float ux, float uy, float p,
                                        float srho, float s3) {
  return __fadd_rn(g_ref(cu, ux, uy, srho), __fmul_rn(p, s3));
}
__device__ __forceinline__ double g_refp(double cu, double ux, double uy,
                                         double p, double srho, double s3) {
  return g_ref(cu, ux, uy, srho) + p * s3;
}

// The node slot k of (x, y) was streamed from: (x, y) - c_k, periodic in x
// (and in y without walls); behind a wall, (x, y) itself.
template <bool WALL>
__device__ __forceinline__ size_t source_node(int x, int y, int k, int nx,
                                              int ny) {
  int sx = x - cx_of(k), sy = y - cy_of(k);
  if (WALL && (sy < 0 || sy >= ny)) {
    sx = x;
    sy = y;
  }
  sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
  sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
  return (size_t)sy * nx + sx;
}

// Moving populations of phase i (mov[0..7] = h_1..8) and the NS populations
// (g[1..8]) of node (x, y) at index q, in stored units, from global memory.
template <int P, bool WALL>
__device__ __forceinline__ void load_h_node(const KArgs<P> &a, int i, int x,
                                            int y, size_t q,
                                            typename Prec<P>::T *mov) {
  typedef typename Prec<P>::T T;
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    T v = load_hm<P>(a, i, k, q);
    if constexpr (Prec<P>::REF) {
      const size_t qs = source_node<WALL>(x, y, k, a.nx, a.ny);
      const T cu = cdotu(k, ldg(a.u_in + qs), ldg(a.u_in + a.V + qs));
      v = __fadd_rn(v, adv_units(cu, ldg(a.pp_in + (size_t)i * a.V + qs),
                                 T(3) * a.sh_st));
    }
    mov[k - 1] = v;
  }
}
template <int P, bool WALL>
__device__ __forceinline__ void load_g_node(const KArgs<P> &a, int x, int y,
                                            size_t q, typename Prec<P>::T *g) {
  typedef typename Prec<P>::T T;
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    T v = load_gm<P>(a, k, q);
    if constexpr (Prec<P>::REF) {
      const size_t qs = source_node<WALL>(x, y, k, a.nx, a.ny);
      const T sux = ldg(a.u_in + qs), suy = ldg(a.u_in + a.V + qs),
              spr = ldg(a.u_in + 2 * a.V + qs);
      v = __fadd_rn(v, g_refp(cdotu(k, sux, suy), sux, suy, spr, a.rho_base * a.sg_st,
                              T(3) * a.sg_st));
    }
    g[k] = v;
  }
}

// Order parameter of one node from its stored values. FP64: sum of the nine
// populations. Other forms: phi_prev + (d_0 + sum_{k>=1} h_k), with the exact
// rounding error of that last addition returned in err (TwoSum).
template <int P>
__device__ __forceinline__ typename Prec<P>::T node_phi(
    typename Prec<P>::T rest, const typename Prec<P>::T *mov,
    typename Prec<P>::T pp, typename Prec<P>::T &err,
    typename Prec<P>::T sh_ld) {
  typedef typename Prec<P>::T T;
  T small = rest;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if constexpr (Prec<P>::MIX)  // mov in stored units s h_k / w_k
      small = __fmaf_rn(w_of<T>(k + 1) * sh_ld, mov[k], small);
    else
      small = __fadd_rn_T(small, mov[k]);
  }
  if constexpr (P == LBM_FP64) {
    err = T(0);
    return small;
  } else {
    const T s = __fadd_rn(pp, small);
    const T bb = __fsub_rn(s, pp);
    err = __fadd_rn(__fsub_rn(pp, __fsub_rn(s, bb)), __fsub_rn(small, bb));
    return s;
  }
}

// Wrap an x coordinate periodically; y periodically or onto the wall rows
// (ghost rows repeat the adjacent fluid row).
__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}
template <bool WALL>
__device__ __forceinline__ int wrap_y(int v, int n) {
  if (WALL) return v < 0 ? 0 : (v >= n ? n - 1 : v);
  return wrap(v, n);
}

// Volume fractions (Eq. N18), density (Eq. N29) and h_i of Eq. N17 at one
// node from its order parameters. With equal pure-phase densities (EQ) the
// maps reduce exactly to c_k = phi_k + (1 - S)/N (k < N - 1),
// c_{N-1} = (1 - S)/N with S = sum_j phi_j, rho = rho~ and
// h_i = f_i - (1/N) sum_k f_k, f_k = c_k (1 - c_k)(1 - 2 c_k).
template <int P, int NP, bool EQ = false>
__device__ __forceinline__ void local_algebra(const KArgs<P> &a,
                                              const typename Prec<P>::T *ph,
                                              typename Prec<P>::T *c,
                                              typename Prec<P>::T &rho,
                                              typename Prec<P>::T *hf) {
  typedef typename Prec<P>::T T;
  if constexpr (EQ) {
    constexpr T invN = T(1) / T(NP + 1);
    T S = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) S += ph[j];
    const T base = (T(1) - S) * invN;
    T f[NP + 1], F = T(0);
#pragma unroll
    for (int k = 0; k <= NP; ++k) {
      const T ck = k < NP ? ph[k] + base : base;
      c[k] = ck;
      f[k] = ck * (T(1) - ck) * (T(1) - T(2) * ck);
      F += f[k];
    }
    rho = a.rho_base;
#pragma unroll
    for (int i = 0; i < NP; ++i) hf[i] = f[i] - F * invN;
  } else {
    T vp[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) vp[j] = a.off[j] + a.mul[j] * ph[j];
    rho = a.rho_base;
#pragma unroll
    for (int j = 0; j < NP; ++j) rho += a.K[j] * vp[j];
    T f[NP + 1];
#pragma unroll
    for (int k = 0; k <= NP; ++k) {
      T s = a.c0[k];
#pragma unroll
      for (int j = 0; j < NP; ++j) s += a.Q[k][j] * vp[j];
      c[k] = s;
      f[k] = s * (T(1) - s) * (T(1) - T(2) * s);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k <= NP; ++k) s += a.Q[k][i] * f[k];
      hf[i] = a.mul[i] * s;
    }
  }
}

// Isotropic central stencils of Eq. N31 on a shared-memory plane: the sums
// over the 8 neighbours folded pairwise.
template <typename T, int W>
__device__ __forceinline__ void stencil(const T *s, int ly, int lx, T &gx,
                                        T &gy, T &lap) {
  const T c = s[ly * W + lx];
  const T e = s[ly * W + lx + 1], w = s[ly * W + lx - 1];
  const T n = s[(ly + 1) * W + lx], so = s[(ly - 1) * W + lx];
  const T ne = s[(ly + 1) * W + lx + 1], nw = s[(ly + 1) * W + lx - 1];
  const T se = s[(ly - 1) * W + lx + 1], sw = s[(ly - 1) * W + lx - 1];
  gx = (e - w) * T(1.0 / 3.0) + ((ne + se) - (nw + sw)) * T(1.0 / 12.0);
  gy = (n - so) * T(1.0 / 3.0) + ((ne + nw) - (se + sw)) * T(1.0 / 12.0);
  lap = ((e + w) + (n + so) - T(4) * c) * T(2.0 / 3.0) +
        ((ne + nw) + (se + sw) - T(4) * c) * T(1.0 / 6.0);
}
template <typename T, int W>
__device__ __forceinline__ void gradient(const T *s, int ly, int lx, T &gx,
                                         T &gy) {
  const T e = s[ly * W + lx + 1], w = s[ly * W + lx - 1];
  const T n = s[(ly + 1) * W + lx], so = s[(ly - 1) * W + lx];
  const T ne = s[(ly + 1) * W + lx + 1], nw = s[(ly + 1) * W + lx - 1];
  const T se = s[(ly - 1) * W + lx + 1], sw = s[(ly - 1) * W + lx - 1];
  gx = (e - w) * T(1.0 / 3.0) + ((ne + se) - (nw + sw)) * T(1.0 / 12.0);
  gy = (n - so) * T(1.0 / 3.0) + ((ne + nw) - (se + sw)) * T(1.0 / 12.0);
}
template <typename T, int W>
__device__ __forceinline__ T laplacian(const T *s, int ly, int lx) {
  const T c = s[ly * W + lx];
  const T e = s[ly * W + lx + 1], w = s[ly * W + lx - 1];
  const T n = s[(ly + 1) * W + lx], so = s[(ly - 1) * W + lx];
  const T ne = s[(ly + 1) * W + lx + 1], nw = s[(ly + 1) * W + lx - 1];
  const T se = s[(ly - 1) * W + lx + 1], sw = s[(ly - 1) * W + lx - 1];
  return ((e + w) + (n + so) - T(4) * c) * T(2.0 / 3.0) +
         ((ne + nw) + (se + sw) - T(4) * c) * T(1.0 / 6.0);
}

// Isotropic mixed gradient of Eq. N40, read with -zeta(x + 2 c_i): the mean
// of the central and the second-order upwind directional differences.
template <typename T, int W>
__device__ __forceinline__ void gradient_mixed(const T *s, int ly, int lx,
                                               T &gx, T &gy) {
  const T c = s[ly * W + lx];
  T sx = T(0), sy = T(0);
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    const int dx = cx_of(k), dy = cy_of(k);
    const T d = -s[(ly + 2 * dy) * W + lx + 2 * dx] +
                T(5) * s[(ly + dy) * W + lx + dx] - T(3) * c -
                s[(ly - dy) * W + lx - dx];
    const T wd = w_of<T>(k) * d;
    if (dx != 0) sx += T(dx) * wd;
    if (dy != 0) sy += T(dy) * wd;
  }
  gx = sx * T(0.75);  // 1 / (4 c_s^2)
  gy = sy * T(0.75);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Per-node work shared by the kernels.
// ---------------------------------------------------------------------------

// Macroscopic quantities of one node at time t (steps a2-a6).
template <int P, int NP> struct NodeMac {
  typedef typename Prec<P>::T T;
  T ph[NP], gpx[NP], gpy[NP], Cv[NP], cc[NP + 1];
  T rho, grx, gry, Jx, Jy, Fx, Fy, ux, uy, uu, ugr, pr;
};

// phi and its stencils from the shared tile (centre ly, lx), C_i (from the
// shared C tile when densities differ), J~ and grad rho, F, u (Eq. N22_1)
// and p (Eq. N23). g[1..8] are the node's NS populations in stored units.
template <int P, int NP, bool NU, int SW, int CW, bool G40 = false>
__device__ __forceinline__ void node_macros(const KArgs<P> &a,
                                            const typename Prec<P>::T *sphi,
                                            int plane, const typename Prec<P>::T *sC,
                                            int cplane, int ly, int lx, int cly,
                                            int clx, const typename Prec<P>::T *g,
                                            NodeMac<P, NP> &m) {
  typedef typename Prec<P>::T T;
  {
    T lp[NP], hf[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      m.ph[i] = sphi[i * plane + ly * SW + lx];
      stencil<T, SW>(sphi + i * plane, ly, lx, m.gpx[i], m.gpy[i], lp[i]);
      if constexpr (G40)
        gradient_mixed<T, SW>(sphi + i * plane, ly, lx, m.gpx[i], m.gpy[i]);
    }
    local_algebra<P, NP, !NU>(a, m.ph, m.cc, m.rho, hf);
    if constexpr (NU) {
#pragma unroll
      for (int i = 0; i < NP; ++i) m.Cv[i] = sC[i * cplane + cly * CW + clx];
    } else {
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T Ci = a.bulk * hf[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) Ci -= a.lam[i][j] * lp[j];
        m.Cv[i] = Ci;
      }
    }
  }
  m.grx = T(0); m.gry = T(0); m.Jx = T(0); m.Jy = T(0);
  if constexpr (NU) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T cgx, cgy;
      if constexpr (G40)
        gradient_mixed<T, CW>(sC + i * cplane, cly, clx, cgx, cgy);
      else
        gradient<T, CW>(sC + i * cplane, cly, clx, cgx, cgy);
      m.Jx -= a.kmob[i] * cgx;
      m.Jy -= a.kmob[i] * cgy;
      m.grx += a.kap[i] * m.gpx[i];
      m.gry += a.kap[i] * m.gpy[i];
    }
  }
  m.Fx = m.rho * a.grav[0];
  m.Fy = m.rho * a.grav[1];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    m.Fx += m.Cv[i] * m.gpx[i];
    m.Fy += m.Cv[i] * m.gpy[i];
  }
  T mx = T(0), my = T(0), sg = T(0);
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    T gk = g[k];  // stored units -> g_k
    if constexpr (Prec<P>::MIX) gk *= w_of<T>(k) * a.sg_ld;
    mx += T(cx_of(k)) * gk;
    my += T(cy_of(k)) * gk;
    sg += gk;
  }
  const T rinv = T(1) / m.rho;
  m.ux = (mx + T(0.5) * m.Fx) * rinv;
  m.uy = (my + T(0.5) * m.Fy) * rinv;
  m.uu = m.ux * m.ux + m.uy * m.uy;
  m.ugr = m.ux * m.grx + m.uy * m.gry;
  // Eq. N23: c_s^2/(1-w_0) = 3/5; s_0(u) = -w_0 |u|^2 / (2 c_s^2)
  m.pr = T(0.6) * (sg + T(0.5) * m.ugr - m.rho * T(4.0 / 9.0) * T(1.5) * m.uu);
}

// Collisions and push streaming of one node (steps a7-a10). hreg[i][0] is
// h_0 (FP64) or d_0 (other forms), hreg[i][1..8] the moving populations and
// g[1..8] the NS populations (both in stored units), perr the rounding error
// of phi, pp phi_i(t-1), up u(t-1).
template <int P, int NP, bool NU, bool WALL>
__device__ __forceinline__ void collide_stream(
    const KArgs<P> &a, const NodeMac<P, NP> &m,
    const typename Prec<P>::T (&hreg)[NP][9], const typename Prec<P>::T *perr,
    const typename Prec<P>::T *g, const typename Prec<P>::T *pp,
    typename Prec<P>::T upx, typename Prec<P>::T upy, int gx, int gy) {
  typedef typename Prec<P>::T T;
  const int nx = a.nx, ny = a.ny;
  const size_t V = a.V;
  const size_t q = (size_t)gy * nx + gx;
  const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
  const int ym = gy == 0 ? ny - 1 : gy - 1, yp = gy == ny - 1 ? 0 : gy + 1;
  // Destination node and direction of population k after streaming.
  size_t dst[9];
  int dk[9];
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    const int cxi = cx_of(k), cyi = cy_of(k);
    int dx = cxi == 0 ? gx : (cxi > 0 ? xp : xm);
    int dy = cyi == 0 ? gy : (cyi > 0 ? yp : ym);
    dk[k] = k;
    if (WALL && ((cyi < 0 && gy == 0) || (cyi > 0 && gy == ny - 1))) {
      dy = gy;
      dx = gx;
      dk[k] = opp_of(k);
    }
    dst[k] = (size_t)dy * nx + dx;
  }
  constexpr bool MIX = Prec<P>::MIX;
  const T ux = m.ux, uy = m.uy, uu = m.uu, rho = m.rho;
  const T Fx = m.Fx, Fy = m.Fy, pr = m.pr;

  // NS collision (Eq. 24) with g^eq (Eq. 25) and G_k (Eq. N20_1), folded:
  //   g*_k = (1 - 1/tau_g) g_k + w_k t_k,
  //   t_k = A0 + C1 c.F + c.u (B1 + B2 c.u + D1 c.F [+ E1 c.grad(rho) + E2 c.J~]),
  // A0 = (3p - 3/2 rho |u|^2)/tau_g - (1 - 1/(2 tau_g))(3 u.F + 3/2 J~.u/(tau_g - 1/2)).
  // The u.grad(rho) term of G_k cancels against the trace part of its
  // (c c - c_s^2 I) contraction. 16-bit forms update s g_k / w_k directly.
  const T tg = a.tg_inv, ff = a.ffac;
  const T uF = ux * Fx + uy * Fy;
  const T Ju = (m.Jx * ux + m.Jy * uy) * a.jfac;
  const T A0 = tg * (T(3) * pr - T(1.5) * rho * uu) - ff * (T(3) * uF + T(1.5) * Ju);
  const T B1 = T(3) * tg * rho, B2 = T(4.5) * tg * rho;
  const T C1 = T(3) * ff, D1 = T(9) * ff;
  const T E1 = T(3) * ff, E2 = T(4.5) * ff * a.jfac;
  const T keep_g = T(1) - tg;
  // 16-bit forms: the writer's references, formed once per magnitude. Each
  // c_k.u (as cdotu rounds it) is +-um[j] with um = ux, uy, ux + uy, uy - ux,
  // and the rounded products 3 c.u, (c.u)^2 and (c.u) phi are odd or even in
  // it, so every reference below has the bits of g_refp / adv_units at cdotu.
  T um[4], g3u[4], g45[4];
  const T uut = MIX ? __fmul_rn(T(-1.5), __fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy))) : T(0);
  const T p3 = MIX ? __fmul_rn(pr, T(3) * a.sg_st) : T(0);
  if constexpr (MIX) {
    um[0] = ux;
    um[1] = uy;
    um[2] = cdotu(5, ux, uy);
    um[3] = cdotu(6, ux, uy);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      g3u[j] = __fmul_rn(T(3), um[j]);
      g45[j] = __fmul_rn(T(4.5), __fmul_rn(um[j], um[j]));
    }
  }
  // index of c_k.u's magnitude in um, and its sign (k = 1..8)
  auto mag = [](int k) { return (k == 1 || k == 3) ? 0 : ((k == 2 || k == 4) ? 1 : ((k == 5 || k == 7) ? 2 : 3)); };
  auto sgn = [](int k) { return (k == 1 || k == 2 || k == 5 || k == 6) ? T(1) : T(-1); };
  T gv[9];
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    const T cxk = T(cx_of(k)), cyk = T(cy_of(k));
    const T cu = cxk * ux + cyk * uy;
    const T cF = cxk * Fx + cyk * Fy;
    T inner = B1 + B2 * cu + D1 * cF;
    if constexpr (NU)
      inner += E1 * (cxk * m.grx + cyk * m.gry) + E2 * (cxk * m.Jx + cyk * m.Jy);
    const T t = A0 + C1 * cF + cu * inner;
    const int kk = dk[k];
    if constexpr (MIX) {  // relative to the equilibrium's parts at this node
      // direction kk: k, or opp(k) (the same magnitude, the other sign)
      const int j = mag(k);
      const T sk = kk == k ? sgn(k) : -sgn(k);
      const T sr = __fadd_rn(__fmul_rn(sk, g3u[j]), g45[j]);  // 3 c.u + 4.5 (c.u)^2
      const T ref = __fadd_rn(__fmul_rn(__fadd_rn(sr, uut), a.rho_base * a.sg_st), p3);
      gv[k] = keep_g * g[k] + a.sg_st * t - ref;
    } else
      a.gm_out[(size_t)(kk - 1) * V + dst[k]] = keep_g * g[k] + w_of<T>(k) * t;
  }
  if constexpr (MIX) {  // converted two at a time
#pragma unroll
    for (int k = 1; k < 9; k += 2) {
      typename Prec<P>::Sm s0, s1;
      to_S2(gv[k], gv[k + 1], s0, s1);
      a.gm_out[(size_t)(dk[k] - 1) * V + dst[k]] = s0;
      a.gm_out[(size_t)(dk[k + 1] - 1) * V + dst[k + 1]] = s1;
    }
  }

  // CH collisions (Eq. N24) with h^eq (Eq. N25) and R_k (Eqs. N26, N27),
  // folded: h*_k = (1 - 1/tau_i) h_k + w_k (alpha + c.beta), alpha =
  // a_i C_i / tau_i, beta = 3 (phi u / tau_i + (1 - 1/(2 tau_i)) d(phi u)).
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const T ph = m.ph[i];
    const T ti = a.tau_inv[i];
    const T aC = a.a[i] * m.Cv[i];
    const T dpx = ph * ux - pp[i] * upx, dpy = ph * uy - pp[i] * upy;
    T al = ti * aC;
    T bx = T(3) * (ti * ph * ux + a.src[i] * dpx);
    T by = T(3) * (ti * ph * uy + a.src[i] * dpy);
    if constexpr (MIX) {  // stored units s h_k / w_k
      al *= a.sh_st;
      bx *= a.sh_st;
      by *= a.sh_st;
    }
    const T keep = T(1) - ti;
    T moving_sum = T(0);
    if constexpr (MIX) {
      // relative to the advective part at this node (the slots' source),
      // converted two at a time; the mass balance uses each value as the
      // reader will decode it
      T hv[9], rf[9], um3[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) um3[j] = adv_units(um[j], ph, T(3) * a.sh_st);
#pragma unroll
      for (int k = 1; k < 9; ++k) {
        const T t = al + T(cx_of(k)) * bx + T(cy_of(k)) * by;
        rf[k] = __fmul_rn(dk[k] == k ? sgn(k) : -sgn(k), um3[mag(k)]);  // adv_units at cdotu(dk[k])
        hv[k] = keep * hreg[i][k] + t - rf[k];
      }
      typename Prec<P>::Sm sv[9];
#pragma unroll
      for (int k = 1; k < 9; k += 2) to_S2(hv[k], hv[k + 1], sv[k], sv[k + 1]);
#pragma unroll
      for (int k = 1; k < 9; ++k) {
        a.hm_out[((size_t)(i * 8 + dk[k] - 1)) * V + dst[k]] = sv[k];
        moving_sum = __fmaf_rn(w_of<T>(dk[k]) * a.sh_ld, __fadd_rn(to_T(sv[k]), rf[k]),
                               moving_sum);
      }
    } else {
#pragma unroll
      for (int k = 1; k < 9; ++k) {
        const T t = al + T(cx_of(k)) * bx + T(cy_of(k)) * by;
        const T hs = keep * hreg[i][k] + w_of<T>(k) * t;
        a.hm_out[((size_t)(i * 8 + dk[k] - 1)) * V + dst[k]] = hs;
        moving_sum = __fadd_rn_T(moving_sum, hs);
      }
    }
    T rest;
    if constexpr (P == LBM_FP64) {
      const T heq0 = ph + (w_of<T>(0) - T(1)) * aC;
      rest = keep * hreg[i][0] + ti * heq0;
    } else {
      // h*_0 = (phi + perr) - sum_{k>=1} h*_k (collision conserves sum_k h_k),
      // stored relative to phi: d*_0 = perr - sum_{k>=1} h*_k.
      rest = __fsub_rn(perr[i], moving_sum);
    }
    a.h0_out[(size_t)i * V + q] = rest;
    a.pp_out[(size_t)i * V + q] = ph;
  }
  a.u_out[q] = ux;
  a.u_out[V + q] = uy;
  if constexpr (Prec<P>::REF) a.u_out[2 * V + q] = pr;
}

// Position of ring entry r of a (BX + 2R) x (BY + 2R) tile: top R rows,
// bottom R rows, left R columns, right R columns.
template <int R>
__device__ __forceinline__ void ring_pos(int r, int &lx, int &ly) {
  constexpr int SW = BX + 2 * R;
  if (r < R * SW) {
    ly = r / SW; lx = r % SW;
  } else if (r < 2 * R * SW) {
    const int t = r - R * SW; ly = R + BY + t / SW; lx = t % SW;
  } else if (r < 2 * R * SW + R * BY) {
    const int t = r - 2 * R * SW; ly = R + t / R; lx = t % R;
  } else {
    const int t = r - 2 * R * SW - R * BY; ly = R + t / R; lx = R + BX + t % R;
  }
}

// phi_i at node (sx, sy) from global memory.
template <int P, int NP, bool WALL>
__device__ __forceinline__ void phi_global(const KArgs<P> &a, int sx, int sy,
                                           typename Prec<P>::T *out, int plane,
                                           int idx) {
  typedef typename Prec<P>::T T;
  const size_t q = (size_t)sy * a.nx + sx;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    T mov[8], err;
    load_h_node<P, WALL>(a, i, sx, sy, q, mov);
    const T pp = P == LBM_FP64 ? T(0) : ldg(a.pp_in + (size_t)i * a.V + q);
    out[i * plane + idx] =
        node_phi<P>(ldg(a.h0_in + (size_t)i * a.V + q), mov, pp, err, a.sh_ld);
  }
}

// ---------------------------------------------------------------------------
// The generic tile kernel (every precision and density case; MODE_STEP: one
// time step; MODE_MOMENTS: write the macroscopic fields; MODE_DIAG: per-CTA
// partial sums of the diagnostics).
// ---------------------------------------------------------------------------
template <int P, int NP, bool NU, bool WALL, bool G40>
__global__ void __launch_bounds__(NT) tile_kernel(const KArgs<P> a) {
  typedef typename Prec<P>::T T;
  constexpr int RG = G40 ? 2 : 1;          // reach of a gradient stencil
  constexpr int RC = NU ? RG : 0;          // C ring radius (for grad C)
  constexpr int R = RC + 1 > RG ? RC + 1 : RG;  // phi halo radius
  constexpr int SW = BX + 2 * R;           // shared tile width
  constexpr int SH = BY + 2 * R;           // shared tile height
  constexpr int CW = NU ? BX + 2 * RC : 1, CH = NU ? BY + 2 * RC : 1;
  __shared__ T sphi[NP][SH * SW];
  __shared__ T sC[NP][CH * CW];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int nx = a.nx, ny = a.ny;
  const size_t V = a.V;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = gx < nx && gy < ny;

  // 1. Own node: load all h^i_k, phi_i = sum_k h^i_k (Eq. N28). hreg[i][0]
  //    holds h_0 (FP64) or d_0 (other forms); perr the rounding error of phi.
  T hreg[NP][9], perr[NP];
  {
    const int sx = wrap(gx, nx), sy = wrap_y<WALL>(gy, ny);
    const size_t q = (size_t)sy * nx + sx;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      hreg[i][0] = ldg(a.h0_in + (size_t)i * V + q);
      load_h_node<P, WALL>(a, i, sx, sy, q, &hreg[i][1]);
      const T pp = P == LBM_FP64 ? T(0) : ldg(a.pp_in + (size_t)i * V + q);
      sphi[i][(ty + R) * SW + tx + R] =
          node_phi<P>(hreg[i][0], &hreg[i][1], pp, perr[i], a.sh_ld);
    }
  }
  // 2. Halo ring.
  constexpr int NRING = SW * SH - BX * BY;
  for (int r = tid; r < NRING; r += NT) {
    int lx, ly;
    ring_pos<R>(r, lx, ly);
    phi_global<P, NP, WALL>(a, wrap(x0 - R + lx, nx), wrap_y<WALL>(y0 - R + ly, ny),
                      &sphi[0][0], SH * SW, ly * SW + lx);
  }
  __syncthreads();

  // 3. Unequal densities: C_i on the tile and a ring of radius RC, then wall
  //    ghost rows of C repeat the adjacent fluid row.
  if constexpr (NU) {
    for (int r = tid; r < CW * CH; r += NT) {
      const int cy = r / CW, cxl = r % CW;
      T ph[NP], lp[NP], cc[NP + 1], rho, hf[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        ph[i] = sphi[i][(cy + R - RC) * SW + cxl + R - RC];
        lp[i] = laplacian<T, SW>(sphi[i], cy + R - RC, cxl + R - RC);
      }
      local_algebra<P, NP>(a, ph, cc, rho, hf);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T Ci = a.bulk * hf[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) Ci -= a.lam[i][j] * lp[j];
        sC[i][r] = Ci;
      }
    }
    __syncthreads();
    if constexpr (WALL) {
      for (int r = tid; r < CW * CH; r += NT) {
        const int cy = r / CW, cxl = r % CW;
        const int yg = y0 - RC + cy;
        if (yg < 0 || yg >= ny) {
          const int ys = yg < 0 ? 0 : ny - 1;
          const int cys = ys - y0 + RC;
#pragma unroll
          for (int i = 0; i < NP; ++i) sC[i][r] = sC[i][cys * CW + cxl];
        }
      }
      __syncthreads();
    }
  }

  // 4. Own node: stencils, C_i, forces, u, p.
  const size_t q = (size_t)(active ? gy : 0) * nx + (active ? gx : 0);
  T g[9];
  if (active) {
    load_g_node<P, WALL>(a, gx, gy, q, g);
  } else {
#pragma unroll
    for (int k = 1; k < 9; ++k) g[k] = T(0);
  }
  NodeMac<P, NP> m;
  node_macros<P, NP, NU, SW, CW, G40>(a, &sphi[0][0], SH * SW, &sC[0][0],
                                      CH * CW, ty + R, tx + R, ty + RC,
                                      tx + RC, g, m);

  if (a.mode == MODE_MOMENTS) {
    if (!active) return;
    if (a.o_phi)
#pragma unroll
      for (int i = 0; i < NP; ++i) a.o_phi[(size_t)i * V + q] = (double)m.ph[i];
    if (a.o_c)
#pragma unroll
      for (int k = 0; k <= NP; ++k) a.o_c[(size_t)k * V + q] = (double)m.cc[k];
    if (a.o_u) {
      a.o_u[q] = (double)m.ux;
      a.o_u[V + q] = (double)m.uy;
    }
    if (a.o_p) a.o_p[q] = (double)m.pr;
    if (a.o_rho) a.o_rho[q] = (double)m.rho;
    return;
  }
  if (a.mode == MODE_DIAG) {
    // mass_k, ke, umax: warp shuffle, then warps in fixed order.
    __shared__ double sred[NT / 32][NP + 3];
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k <= NP + 2; ++k) {
      double v;
      if (k <= NP) v = active ? (double)m.cc[k] : 0.0;
      else if (k == NP + 1) v = active ? 0.5 * (double)m.rho * (double)m.uu : 0.0;
      else v = active ? sqrt((double)m.uu) : 0.0;
      v = (k == NP + 2) ? warp_max(v) : warp_sum(v);
      if (lane == 0) sred[wid][k] = v;
    }
    __syncthreads();
    if (tid <= NP + 2) {
      double v = sred[0][tid];
      for (int w = 1; w < NT / 32; ++w)
        v = (tid == NP + 2) ? fmax(v, sred[w][tid]) : v + sred[w][tid];
      a.red[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (NP + 3) + tid] = v;
    }
    return;
  }
  if (!active) return;

  // 5-6. Collisions and streaming.
  T pp[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) pp[i] = ldg(a.pp_in + (size_t)i * V + q);
  collide_stream<P, NP, NU, WALL>(a, m, hreg, perr, g, pp, a.u_in[q],
                                  a.u_in[V + q], gx, gy);
}

// ---------------------------------------------------------------------------
// Pipelined step kernel for the FP32 and 16-bit forms with equal densities.
//
// Persistent CTAs walk the 32 x 8 tiles in raster order (tile b, b + grid,
// ...). A ring of S shared-memory stages holds the populations of the next
// tiles: one 3-D TMA box per array (all planes at once), the h and phi_prev
// planes with a halo of one row and HX columns (HX * element size = 16 B,
// the TMA alignment), completion counted on one mbarrier per stage. While a
// tile is computed, the loads of the following S - 1 tiles are in flight.
// Halo positions that wrap around the domain (periodic edges, wall ghost
// rows, ragged tails) are summed from global memory instead.
// ---------------------------------------------------------------------------
// Pipeline shape, chosen by timing the N=5 2048^2 step on GB300: 2 stages,
// u(t-1) staged with the tile. FP32: two phi tiles and one barrier per tile
// (the stage is refilled right after the tile's phi barrier, u(t-1) having
// been read before it; with the wrapped halos staged this took the step
// from 0.906 to 0.928 of the copy bandwidth), 185 KB, one CTA per SM.
// 16-bit forms (their populations decoded with phi(t-1) and u(t-1) of the
// source node: those two boxes carry two halo rows): one phi tile and two
// barriers per tile (the stage refilled after the second), 111 KB and 128
// registers, two CTAs per SM (a second phi tile would not leave room for two).
// Measured and rejected:
//  - FP32 (before the wrapped halos were staged): a third stage (227 KB,
//    ~28 KB of L1 left) -28%; one barrier per tile with one phi tile -23%;
//    one stage with two CTAs per SM -15%; 32 x 12 tiles (384
//    threads, 225 KB) -30%; a stage without halo columns (wrapped ring
//    columns from global memory, two CTAs per SM) -48%; g and u(t-1) loaded
//    from global memory before the wait instead of staged -19% (a third
//    stage on top, a further -6%); the ring's phi split over
//    (position, phase) pairs on all warps -1.5%; the stage refilled right
//    after the phi barrier (two barriers kept) -9%; 32 x 4 tiles with two
//    CTAs per SM (four stages in flight per SM) -27%; an L2 prefetch of the
//    tile one, two or four beyond the stages (cp.async.bulk.prefetch.tensor)
//    -35%, -37%, -48%. Instrumented, the kernel spends 13-19% of its time in
//    the stage wait; ncu counts it as long-scoreboard stalls (1.5 per
//    issued instruction).
//  - 16-bit with the source-relative encoding: one CTA per SM with one
//    barrier and a double-buffered phi tile -20% (3 stages -22%); the ring's
//    decode spread over all warps -6%. With plain scaled storage (an earlier
//    form: 2 stages, direct u(t-1), one barrier, two CTAs) the 16-bit step
//    ran 35% faster but missed the accuracy targets.
template <int P> struct TmaGeom {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  static constexpr int HXM = 16 / (int)sizeof(Sm);  // halo columns, moving planes
  static constexpr int HXR = 16 / (int)sizeof(T);   // halo columns, FP32 planes
  static constexpr int WM = BX + 2 * HXM;           // box widths
  static constexpr int WR = BX + 2 * HXR;
  static constexpr bool WIDE = sizeof(Sm) == 4;     // FP32 storage
  static constexpr int TBY = 8;                     // tile height
  static constexpr int NTH = BX * TBY;              // threads per CTA
  static constexpr int HB = TBY + 2;                // box height
  static constexpr int S = 2;                       // pipeline stages
  // 16-bit forms decode every population with phi(t-1) and u(t-1) of the
  // node it came from: the ring's sources lie two rows out, so these two
  // boxes carry two halo rows, and u(t-1) is staged with halo.
  static constexpr bool REF = Prec<P>::REF;
  static_assert(WIDE || REF, "16-bit storage is source-relative");
  static constexpr int RY = REF ? 2 : 1;            // halo rows, phi(t-1) and u(t-1)
  static constexpr int HBP = TBY + 2 * RY;          // their box height
  static constexpr int UW = REF ? WR : BX;          // u(t-1) box
  static constexpr int UH = REF ? HBP : TBY;
  static constexpr int UOX = REF ? HXR : 0, UOY = REF ? RY : 0;
  static constexpr int UPN = REF ? 3 : 2;           // u(t-1) planes (+ p(t-1))
  // FP32: the ring column and row that wrap around a periodic grid are
  // staged too (x: 16 bytes of columns at the far edge x box height; y: one
  // row x box width at the far edge), for tiles on the grid's edge.
  static constexpr bool WRAP = WIDE;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after ~2^22 polls (well over a second).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 16) __nanosleep(256);
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map,
                                            int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int P, int NP> struct TmaStage {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  typedef TmaGeom<P> G;
  static constexpr size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
  static constexpr size_t HM = al((size_t)8 * NP * G::HB * G::WM * sizeof(Sm));
  static constexpr size_t H0 = al((size_t)NP * G::HB * G::WR * sizeof(T));
  static constexpr size_t PP = al((size_t)NP * G::HBP * G::WR * sizeof(T));
  static constexpr size_t GM = al((size_t)8 * G::TBY * BX * sizeof(Sm));
  static constexpr size_t UP = al((size_t)G::UPN * G::UH * G::UW * sizeof(T));
  // wrapped halo column (x) and row (y) of the h, d_0, phi(t-1) arrays
  static constexpr size_t XHM = al((size_t)8 * NP * G::HB * G::HXM * sizeof(Sm));
  static constexpr size_t XH0 = al((size_t)NP * G::HB * G::HXR * sizeof(T));
  static constexpr size_t XPP = al((size_t)NP * G::HBP * G::HXR * sizeof(T));
  static constexpr size_t YHM = al((size_t)8 * NP * G::WM * sizeof(Sm));
  static constexpr size_t YH0 = al((size_t)NP * G::WR * sizeof(T));
  static constexpr size_t YPP = YH0;
  static constexpr size_t WRAPB = G::WRAP ? XHM + XH0 + XPP + YHM + YH0 + YPP : 0;
  static constexpr size_t BASE = HM + H0 + PP + GM + UP;  // offset of the wrap boxes
  static constexpr size_t BYTES = BASE + WRAPB;
  // bytes the TMA engine writes per stage (full boxes, including fill)
  static constexpr uint32_t TX =
      (uint32_t)((size_t)8 * NP * G::HB * G::WM * sizeof(Sm) +
                 (size_t)NP * G::HB * G::WR * sizeof(T) +
                 (size_t)NP * G::HBP * G::WR * sizeof(T) +
                 (size_t)8 * G::TBY * BX * sizeof(Sm) +
                 (size_t)G::UPN * G::UH * G::UW * sizeof(T));
  static constexpr uint32_t XTX =
      (uint32_t)(((size_t)8 * NP * G::HB * G::HXM) * sizeof(Sm) +
                 ((size_t)NP * G::HB * G::HXR + (size_t)NP * G::HBP * G::HXR) * sizeof(T));
  static constexpr uint32_t YTX =
      (uint32_t)((size_t)8 * NP * G::WM * sizeof(Sm) + (size_t)2 * NP * G::WR * sizeof(T));
  static constexpr size_t SPHI = al((size_t)NP * (G::TBY + 2) * (BX + 2) * sizeof(T));
  static constexpr int S = G::S;
  // FP32: two phi tiles (one barrier per tile, below); 16-bit forms: one
  static constexpr int NPHI = G::WIDE ? 2 : 1;
  static constexpr size_t SMEM = S * BYTES + NPHI * SPHI + 64;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

// Ring entry r of a (BX + 2) x (TBY + 2) tile: top row, bottom row, left
// column, right column.
template <int TBY>
__device__ __forceinline__ void ring_pos_1(int r, int &lx, int &ly) {
  constexpr int SW = BX + 2;
  if (r < SW) {
    ly = 0; lx = r;
  } else if (r < 2 * SW) {
    ly = TBY + 1; lx = r - SW;
  } else if (r < 2 * SW + TBY) {
    ly = 1 + (r - 2 * SW); lx = 0;
  } else {
    ly = 1 + (r - 2 * SW - TBY); lx = BX + 1;
  }
}

// WHOLE: the grid is whole tiles, more than one in each direction. Its
// edge tiles' boxes are then made periodic before use: the box column (x)
// and row (y, periodic grids) beyond the grid that the ring reads (and, in
// the 16-bit forms, the two that the sources read) are overwritten with the
// wrapped values from global memory, loaded before the stage's wait. Every
// tile then reads every position from its boxes at fixed offsets (a wall's
// ghost row is the adjacent row; a source behind a wall is the node
// itself): one branch-free path for all tiles. Other grids take a general
// path that reads wrapped positions from global memory.
template <int P, int NP, bool WALL, bool WHOLE>
__global__ void __launch_bounds__(TmaGeom<P>::NTH, TmaGeom<P>::WIDE ? 1 : 2)
    tile_kernel_tma(const KArgs<P> a, const __grid_constant__ TmaMaps maps,
                    int ntx, int ntiles) {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  typedef TmaGeom<P> G;
  typedef TmaStage<P, NP> St;
  constexpr int S = St::S;
  constexpr int TBY = G::TBY;
  constexpr int SW = BX + 2, SH = TBY + 2, PL = SW * SH;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = (uint64_t *)(smem + S * St::BYTES + St::NPHI * St::SPHI);
  // FP32: the stage is not read after the tile's phi barrier (u(t-1) is
  // loaded before it), so it is refilled right after that barrier, and with
  // two phi tiles (tile j uses tile j & 1) that is the tile's only barrier:
  // a thread at the next tile's barrier is done with this tile's phi tile.
  // The 16-bit forms (one phi tile, to keep two CTAs per SM) refill after a
  // second barrier at the end of the tile.
  constexpr bool ONEB = St::NPHI == 2;

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int nx = a.nx, ny = a.ny;
  const int nmine = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  // FP32 tiles on the edge of a periodic grid: which wrapped halo column
  // (1: x = -1, staged from x = nx - 4 .. nx - 1; 2: x = nx, from 0 .. 3)
  // and row (1: y = -1 from ny - 1; 2: y = ny from 0; none with walls,
  // whose ghost rows repeat a row of the box) are staged with the tile.
  auto halo_x = [&](int x0) {
    return !G::WRAP ? 0 : (x0 == 0 ? 1 : (x0 + BX == nx ? 2 : 0));
  };
  auto halo_y = [&](int y0) {
    return (!G::WRAP || WALL) ? 0 : (y0 == 0 ? 1 : (y0 + TBY == ny ? 2 : 0));
  };
  auto issue = [&](int j) {  // thread 0: TMA loads of my j-th tile
    const int t = blockIdx.x + j * gridDim.x;
    const int x0 = (t % ntx) * BX, y0 = (t / ntx) * TBY;
    unsigned char *st = smem + (j % S) * St::BYTES;
    uint64_t *b = bar + (j % S);
    const int wx = halo_x(x0), wy = halo_y(y0);
    mbar_expect_tx(b, St::TX + (wx ? St::XTX : 0u) + (wy ? St::YTX : 0u));
    tma_load_3d(st, &maps.hm, x0 - G::HXM, y0 - 1, 0, b);
    tma_load_3d(st + St::HM, &maps.h0, x0 - G::HXR, y0 - 1, 0, b);
    tma_load_3d(st + St::HM + St::H0, &maps.pp, x0 - G::HXR, y0 - G::RY, 0, b);
    tma_load_3d(st + St::HM + St::H0 + St::PP, &maps.gm, x0, y0, 0, b);
    tma_load_3d(st + St::HM + St::H0 + St::PP + St::GM, &maps.up, x0 - G::UOX,
                y0 - G::UOY, 0, b);
    if constexpr (G::WRAP) {
      unsigned char *w = st + St::BASE;
      if (wx) {
        const int xs = wx == 1 ? nx - G::HXR : 0;
        tma_load_3d(w, &maps.hmx, xs, y0 - 1, 0, b);
        tma_load_3d(w + St::XHM, &maps.h0x, xs, y0 - 1, 0, b);
        tma_load_3d(w + St::XHM + St::XH0, &maps.ppx, xs, y0 - 1, 0, b);
      }
      if (wy) {
        const int ys = wy == 1 ? ny - 1 : 0;
        w += St::XHM + St::XH0 + St::XPP;
        tma_load_3d(w, &maps.hmy, x0 - G::HXM, ys, 0, b);
        tma_load_3d(w + St::YHM, &maps.h0y, x0 - G::HXR, ys, 0, b);
        tma_load_3d(w + St::YHM + St::YH0, &maps.ppy, x0 - G::HXR, ys, 0, b);
      }
    }
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int j = 0; j < S && j < nmine; ++j) issue(j);
  }
  __syncthreads();

  int issued = nmine < S ? nmine : S;
  int failed_at = -1;
  for (int j = 0; j < nmine; ++j) {
    const int t = blockIdx.x + j * gridDim.x;
    const int x0 = (t % ntx) * BX, y0 = (t / ntx) * TBY;
    T *sphi = (T *)(smem + S * St::BYTES + (ONEB ? (j & 1) * St::SPHI : 0));
    unsigned char *stw = smem + (j % S) * St::BYTES;
    const unsigned char *st = stw;
    const Sm *shm = (const Sm *)st;
    const T *sh0 = (const T *)(st + St::HM);
    const T *spp = (const T *)(st + St::HM + St::H0);
    const Sm *sgm = (const Sm *)(st + St::HM + St::H0 + St::PP);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = WHOLE || (gx < nx && gy < ny);
    const T *sup = (const T *)(st + St::HM + St::H0 + St::PP + St::GM);

    // ---- the periodic patch of an edge tile (16-bit forms, WHOLE grids;
    // FP32 stages its wrapped halo by TMA instead, above) ----
    // Entries: x: hm and h0 one column, phi(t-1) and u(t-1) NC columns on
    // the wrapped side; y: hm, h0 one row, phi(t-1) and u(t-1) NC rows.
    // Entry e -> array (0 hm, 1 h0, 2 phi(t-1), 3 u(t-1)), plane and box
    // position.
    constexpr bool PATCH = G::REF && WHOLE;
    constexpr int NC = 2;                        // columns / rows of the sources
    constexpr int UPP = G::UPN;                  // u(t-1) planes patched
    constexpr int NXS = (9 * NP) * G::HB + NC * (NP * G::HBP + UPP * G::UH);
    constexpr int NYS = (9 * NP) * (BX + 2) + NC * (NP + UPP) * (BX + 2 * NC);
    constexpr int PM = PATCH ? (NXS + NYS + G::NTH - 1) / G::NTH : 1;
    const bool patch_x = PATCH && (x0 == 0 || x0 + BX == nx);
    const bool patch_y = PATCH && !WALL && (y0 == 0 || y0 + TBY == ny);
    const int nxs = patch_x ? NXS : 0, nys = patch_y ? NYS : 0;
    auto entry = [&](int e, int &arr, int &pl, int &bx, int &by) {
      const bool left = x0 == 0, bottom = y0 == 0;
      if (e < nxs) {
        int f = e;
        if (f < 8 * NP * G::HB) {
          arr = 0; pl = f / G::HB; by = f % G::HB; bx = left ? G::HXM - 1 : G::HXM + BX;
        } else if ((f -= 8 * NP * G::HB) < NP * G::HB) {
          arr = 1; pl = f / G::HB; by = f % G::HB; bx = left ? G::HXR - 1 : G::HXR + BX;
        } else {
          f -= NP * G::HB;
          const int two = f % NC;
          f /= NC;
          if (f < NP * G::HBP) {
            arr = 2; pl = f / G::HBP; by = f % G::HBP;
          } else {
            f -= NP * G::HBP;
            arr = 3; pl = f / G::UH; by = f % G::UH;
          }
          bx = left ? G::HXR - NC + two : G::HXR + BX + two;
        }
      } else {
        int f = e - nxs;
        if (f < (9 * NP) * (BX + 2)) {
          const int w = BX + 2;
          pl = f / w;
          arr = pl < 8 * NP ? 0 : 1;
          if (arr == 1) pl -= 8 * NP;
          by = bottom ? 0 : G::HB - 1;
          bx = (arr == 0 ? G::HXM : G::HXR) - 1 + f % w;
        } else {
          f -= (9 * NP) * (BX + 2);
          const int w = BX + 2 * NC;
          const int two = f % NC;
          f /= NC;
          pl = f / w;
          arr = pl < NP ? 2 : 3;
          if (arr == 3) pl -= NP;
          by = bottom ? two : G::HBP - NC + two;
          bx = G::HXR - NC + f % w;
        }
      }
    };
    // the patch's values, loaded before the wait (they do not depend on the
    // stage; a thread's loads are all in flight at once)
    uint32_t pv[PM];
    if (PATCH && (patch_x || patch_y)) {  // CTA-uniform
#pragma unroll
      for (int m = 0; m < PM; ++m) {
        const int e = tid + m * G::NTH;
        if (e < nxs + nys) {
          int arr, pl, bx, by;
          entry(e, arr, pl, bx, by);
          const int ox = arr == 0 ? G::HXM : (arr == 3 ? G::UOX : G::HXR);
          const int oy = arr < 2 ? 1 : G::RY;
          const size_t q = (size_t)pl * a.V +
                           (size_t)wrap(y0 - oy + by, ny) * nx + wrap(x0 - ox + bx, nx);
          const void *src = arr == 0 ? (const void *)(a.hm_in + q)
                            : arr == 1 ? (const void *)(a.h0_in + q)
                            : arr == 2 ? (const void *)(a.pp_in + q)
                                       : (const void *)(a.u_in + q);
          pv[m] = arr == 0 ? (uint32_t)__ldg((const unsigned short *)src)
                           : __ldg((const unsigned int *)src);
        }
      }
    }
    // A thread whose wait gave up still runs the phi sums below (on stale
    // shared data, harmlessly); the barrier after them makes the decision
    // to stop the same for the whole CTA.
    const bool ok = mbar_wait(bar + (j % S), (uint32_t)((j / S) & 1));
    if (PATCH && (patch_x || patch_y)) {  // the stage has landed: patch it
#pragma unroll
      for (int m = 0; m < PM; ++m) {
        const int e = tid + m * G::NTH;
        if (e < nxs + nys) {
          int arr, pl, bx, by;
          entry(e, arr, pl, bx, by);
          if (arr == 0) {
            ((unsigned short *)stw)[(pl * G::HB + by) * G::WM + bx] = (unsigned short)pv[m];
          } else if (arr == 1) {
            ((uint32_t *)(stw + St::HM))[(pl * G::HB + by) * G::WR + bx] = pv[m];
          } else if (arr == 2) {
            ((uint32_t *)(stw + St::HM + St::H0))[(pl * G::HBP + by) * G::WR + bx] = pv[m];
          } else {
            ((uint32_t *)(stw + St::HM + St::H0 + St::PP + St::GM))[(pl * G::UH + by) * G::UW + bx] =
                pv[m];
          }
        }
      }
      __syncthreads();
    }

    // 16-bit forms: u(t-1) and phi(t-1) of the node that slot k of node
    // (xn, yn) was streamed from; (cb, rb) is the node's position in the
    // u(t-1) and phi(t-1) boxes (of the node itself behind a wall).
    // WHOLE: always in the boxes. Otherwise tiles whose two-node
    // neighbourhood lies inside the grid find every source in the boxes at
    // a fixed offset, others read sources that wrap from global memory.
    const bool inner = PATCH || (x0 >= 2 && x0 + BX + 2 <= nx && y0 >= 2 && y0 + TBY + 2 <= ny);
    auto source = [&](int k, int xn, int yn, int cb, int rb, T &sux, T &suy,
                      T &spr, T *sph) {
      int r = rb - cy_of(k), c = cb - cx_of(k);
      bool box = true;
      if (!PATCH && !inner) {
        int sx = xn - cx_of(k), sy = yn - cy_of(k);
        if (WALL && (sy < 0 || sy >= ny)) {
          sx = xn; sy = yn; c = cb; r = rb;
        }
        box = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
      } else if (WALL) {
        const int sy = yn - cy_of(k);
        if (sy < 0 || sy >= ny) { c = cb; r = rb; }
      }
      if (box) {
        sux = sup[r * G::UW + c];
        suy = sup[(G::UH + r) * G::UW + c];
        spr = sup[(2 * G::UH + r) * G::UW + c];
#pragma unroll
        for (int i = 0; i < NP; ++i) sph[i] = spp[(i * G::HBP + r) * G::WR + c];
      } else {
        const size_t qs = source_node<WALL>(xn, yn, k, nx, ny);
        sux = ldg(a.u_in + qs);
        suy = ldg(a.u_in + a.V + qs);
        spr = ldg(a.u_in + 2 * a.V + qs);
#pragma unroll
        for (int i = 0; i < NP; ++i) sph[i] = ldg(a.pp_in + (size_t)i * a.V + qs);
      }
    };
    const T s3h = T(3) * a.sh_st, srg = a.rho_base * a.sg_st, s3g = T(3) * a.sg_st;

    // phi on the tile and its ring, from the staged boxes (the result goes
    // to sphi row `out_row`, by default the box row).
    auto box_phi = [&](int bxm, int bxr, int by, T *err, int out_row = -1) {
      T mv[NP][8];
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int k = 1; k < 9; ++k)
          mv[i][k - 1] = to_T(shm[((i * 8 + k - 1) * G::HB + by) * G::WM + bxm]);
      if constexpr (G::REF) {
        const int xn = x0 - G::HXR + bxr, yn = y0 - 1 + by;
#pragma unroll
        for (int k = 1; k < 9; ++k) {
          T sux, suy, spr, sph[NP];
          source(k, xn, yn, bxr, by - 1 + G::RY, sux, suy, spr, sph);
          const T cu = cdotu(k, sux, suy);
#pragma unroll
          for (int i = 0; i < NP; ++i)
            mv[i][k - 1] = __fadd_rn(mv[i][k - 1], adv_units(cu, sph[i], s3h));
        }
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T *mov = mv[i];
        const T rest = sh0[(i * G::HB + by) * G::WR + bxr];
        const T pp = spp[(i * G::HBP + by - 1 + G::RY) * G::WR + bxr];
        T e;
        sphi[i * PL + (out_row < 0 ? by : out_row) * SW + (bxr - G::HXR + 1)] =
            node_phi<P>(rest, mov, pp, e, a.sh_ld);
        if (err) err[i] = e;
      }
    };
    // own node (ly = ty + 1, lx = tx + 1; box column tx + HX, row ty + 1):
    // its populations go to registers once, for phi and for the collision.
    T perr[NP], hreg[NP][9], g[9], pp[NP];
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        hreg[i][0] = sh0[(i * G::HB + ty + 1) * G::WR + tx + G::HXR];
#pragma unroll
        for (int k = 1; k < 9; ++k)
          hreg[i][k] = to_T(shm[((i * 8 + k - 1) * G::HB + ty + 1) * G::WM + tx + G::HXM]);
        pp[i] = spp[(i * G::HBP + ty + G::RY) * G::WR + tx + G::HXR];
      }
#pragma unroll
      for (int k = 1; k < 9; ++k) g[k] = to_T(sgm[((k - 1) * TBY + ty) * BX + tx]);
      if constexpr (G::REF) {
#pragma unroll
        for (int k = 1; k < 9; ++k) {
          T sux, suy, spr, sph[NP];
          source(k, gx, gy, tx + G::HXR, ty + G::RY, sux, suy, spr, sph);
          const T cu = cdotu(k, sux, suy);
#pragma unroll
          for (int i = 0; i < NP; ++i)
            hreg[i][k] = __fadd_rn(hreg[i][k], adv_units(cu, sph[i], s3h));
          g[k] = __fadd_rn(g[k], g_refp(cu, sux, suy, spr, srg, s3g));
        }
      }
#pragma unroll
      for (int i = 0; i < NP; ++i)
        sphi[i * PL + (ty + 1) * SW + tx + 1] =
            node_phi<P>(hreg[i][0], &hreg[i][1], pp[i], perr[i], a.sh_ld);
    } else {
      phi_global<P, NP, WALL>(a, wrap(gx, nx), wrap_y<WALL>(gy, ny), sphi, PL,
                        (ty + 1) * SW + tx + 1);
    }
    // ring positions on warps 1..3 (threads 32 .. 32 + NRING - 1): warp 0
    // holds the thread that issues the stage refills
    constexpr int NRING = SW * SH - BX * TBY;
    static_assert(32 + NRING <= G::NTH, "one ring position per thread");
    if (tid >= 32 && tid < 32 + NRING) {
      int lx, ly;
      ring_pos_1<TBY>(tid - 32, lx, ly);
      const int rx = x0 - 1 + lx, ry = y0 - 1 + ly;
      const bool inx = rx >= 0 && rx < nx, iny = ry >= 0 && ry < ny;
      if (PATCH) {
        // a wall's ghost row is the adjacent row of the box
        const int by = WALL ? wrap_y<WALL>(ry, ny) - y0 + 1 : ly;
        box_phi(lx - 1 + G::HXM, lx - 1 + G::HXR, by, nullptr, ly);
      } else if (inx && iny) {
        box_phi(lx - 1 + G::HXM, lx - 1 + G::HXR, ly, nullptr);
      } else if constexpr (G::WRAP) {
        // staged wrapped column or row, a wall's ghost row from the box, or
        // (corners, ragged tails) global memory
        const int wx = halo_x(x0), wy = halo_y(y0);
        const unsigned char *w = st + St::BASE;
        auto wrap_phi = [&](const Sm *hmb, const T *h0b, const T *ppb, int pm, int pr,
                            int om, int orr) {
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            T mov[8], e;
#pragma unroll
            for (int k = 1; k < 9; ++k) mov[k - 1] = to_T(hmb[(i * 8 + k - 1) * pm + om]);
            sphi[i * PL + ly * SW + lx] =
                node_phi<P>(h0b[i * pr + orr], mov, ppb[i * pr + orr], e, a.sh_ld);
          }
        };
        if (iny && ((rx < 0 && wx == 1) || (rx >= nx && wx == 2))) {
          const int c = rx < 0 ? G::HXR - 1 : 0;
          wrap_phi((const Sm *)w, (const T *)(w + St::XHM), (const T *)(w + St::XHM + St::XH0),
                   G::HB * G::HXM, G::HB * G::HXR, ly * G::HXM + c, ly * G::HXR + c);
        } else if (inx && WALL) {
          box_phi(lx - 1 + G::HXM, lx - 1 + G::HXR, wrap_y<WALL>(ry, ny) - y0 + 1, nullptr,
                  ly);
        } else if (inx && ((ry < 0 && wy == 1) || (ry >= ny && wy == 2))) {
          w += St::XHM + St::XH0 + St::XPP;
          wrap_phi((const Sm *)w, (const T *)(w + St::YHM), (const T *)(w + St::YHM + St::YH0),
                   G::WM, G::WR, lx - 1 + G::HXM, lx - 1 + G::HXR);
        } else {
          phi_global<P, NP, WALL>(a, wrap(rx, nx), wrap_y<WALL>(ry, ny), sphi, PL,
                                  ly * SW + lx);
        }
      } else {
        phi_global<P, NP, WALL>(a, wrap(rx, nx), wrap_y<WALL>(ry, ny), sphi, PL,
                                ly * SW + lx);
      }
    }
    const T upx = sup[(ty + G::UOY) * G::UW + tx + G::UOX];
    const T upy = sup[(G::UH + ty + G::UOY) * G::UW + tx + G::UOX];
    // phi of the tile and its ring complete (and the decision to stop
    // CTA-wide).
    if (__syncthreads_or(!ok)) {
      failed_at = j;
      break;
    }
    if (ONEB && tid == 0 && issued < nmine) {  // the stage is free
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(issued);
      ++issued;
    }

    if (active) {
      NodeMac<P, NP> m;
      node_macros<P, NP, false, SW, 1>(a, sphi, PL, nullptr, 0, ty + 1, tx + 1,
                                       0, 0, g, m);
      collide_stream<P, NP, false, WALL>(a, m, hreg, perr, g, pp, upx, upy, gx, gy);
    }
    if (ONEB) continue;
    // Every thread is done with this tile's stage and phi tile: refill the
    // stage with the tile S ahead.
    __syncthreads();
    if (tid == 0 && issued < nmine) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(issued);
      ++issued;
    }
  }
  if (failed_at >= 0) {
    // Record the timeout, then let the copies still in flight (tiles
    // failed_at .. issued-1, one per stage) land, with the same bounded wait,
    // before the CTA's shared memory is released.
    if (tid == 0) {
      atomicExch(a.err, 1);
      for (int j = failed_at; j < issued; ++j)
        mbar_wait(bar + (j % S), (uint32_t)((j / S) & 1));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Initialisation: phi from c (inverse of Eqs. N2, N12), then h = h^eq and
// g = g^eq at the stencil C_i.
// ---------------------------------------------------------------------------
// phi_i (FP64) goes to phid[i][V] as well, for the stencils of the start;
// phid may be the array c came in (each node reads its own c first).
template <int P, int NP>
__global__ void init_phi_kernel(const KArgs<P> a, const double *c,
                                const double *__restrict__ u, double *phid,
                                double r0, double r1, double r2, double r3,
                                double r4) {
  typedef typename Prec<P>::T T;
  const double rt[5] = {r0, r1, r2, r3, r4};
  const double rN = rt[NP];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < a.V;
       q += (size_t)gridDim.x * blockDim.x) {
    const double cN = c[(size_t)NP * a.V + q];
    double ph[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const double ci = c[(size_t)i * a.V + q];
      ph[i] = (2.0 * (rt[i] * ci - rN * cN) - (rt[i] - rN)) / (rt[i] + rN);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      a.pp_out[(size_t)i * a.V + q] = (T)ph[i];
      phid[(size_t)i * a.V + q] = ph[i];
    }
    a.u_out[q] = u ? (T)u[q] : T(0);
    a.u_out[a.V + q] = u ? (T)u[a.V + q] : T(0);
  }
}

// Store an FP64 value in a storage type with one rounding (to nearest, ties
// to even). The 16-bit types go through FP32 rounded to odd (truncate, then
// set the last bit if anything was cut off), which keeps the second rounding
// exact: Boldo and Melquiond, "Emulation of FMA and correctly rounded sums:
// proved algorithms using rounding to odd" (IEEE Trans. Computers, 2008),
// for a target of at most 22 significant bits.
template <typename S> __device__ __forceinline__ S store_once(double v);
template <> __device__ __forceinline__ double store_once(double v) { return v; }
template <> __device__ __forceinline__ float store_once(double v) {
  return __double2float_rn(v);
}
__device__ __forceinline__ float float_round_odd(double v) {
  const float t = __double2float_rz(v);
  return (double)t == v ? t : __uint_as_float(__float_as_uint(t) | 1u);
}
template <> __device__ __forceinline__ __nv_bfloat16 store_once(double v) {
  return to_S<__nv_bfloat16>(float_round_odd(v));
}
template <> __device__ __forceinline__ __half store_once(double v) {
  return to_S<__half>(float_round_odd(v));
}

// Equilibrium start in FP64 for every storage form: phi (FP64, from
// init_phi_kernel) and its Laplacian, C_i (Eqs. N17, N18), h^eq (Eq. N25) and g^eq
// (Eq. 25) are computed in double with the constants `d`, and each stored
// value is rounded once into its form. The 16-bit references (and the FP32
// phi(t-1), u(t-1) they use) are those the step kernel decodes with.
template <int P, int NP, bool WALL>
__global__ void init_pop_kernel(const KArgs<P> a, const KArgs<LBM_FP64> d,
                                const double *__restrict__ phid,
                                const double *__restrict__ uin, double p0) {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  const int nx = a.nx, ny = a.ny;
  const size_t V = a.V;
  T *h0 = a.h0_out;
  Sm *hm = a.hm_out;
  Sm *gm = a.gm_out;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < V;
       q += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(q % nx), y = (int)(q / nx);
    double ph[NP], lp[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double s[9];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
          s[(dy + 1) * 3 + dx + 1] =
              phid[(size_t)i * V + (size_t)wrap_y<WALL>(y + dy, ny) * nx + wrap(x + dx, nx)];
      ph[i] = s[4];
      lp[i] = laplacian<double, 3>(s, 1, 1);
    }
    double cc[NP + 1], rho, hf[NP];
    local_algebra<LBM_FP64, NP>(d, ph, cc, rho, hf);
    const double ux = uin ? uin[q] : 0.0, uy = uin ? uin[V + q] : 0.0;
    const double uu = ux * ux + uy * uy;
    if constexpr (Prec<P>::REF) a.u_out[2 * V + q] = (T)p0;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
      const double cu = cx_of(k) * ux + cy_of(k) * uy;
      const double geq =
          w_of<double>(k) * (3.0 * p0 + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
      if constexpr (Prec<P>::MIX) {
        const size_t qs = source_node<WALL>(x, y, k, nx, ny);
        const T sux = a.u_out[qs], suy = a.u_out[V + qs];
        // every source starts at p0 (stored as its p(t-1) above)
        const T ref = Prec<P>::REF ? g_refp(cdotu(k, sux, suy), sux, suy, (T)p0,
                                            a.rho_base * a.sg_st, T(3) * a.sg_st)
                                   : T(0);
        gm[(size_t)(k - 1) * V + q] =
            store_once<Sm>(geq * (d.sg_st / w_of<double>(k)) - (double)ref);
      } else
        gm[(size_t)(k - 1) * V + q] = store_once<Sm>(geq);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double Ci = d.bulk * hf[i];
#pragma unroll
      for (int j = 0; j < NP; ++j) Ci -= d.lam[i][j] * lp[j];
      const double aC = d.a[i] * Ci;
      double moving = 0.0;  // sum of the moving populations as stored
#pragma unroll
      for (int k = 1; k < 9; ++k) {
        const double heq =
            w_of<double>(k) * (aC + 3.0 * ph[i] * (cx_of(k) * ux + cy_of(k) * uy));
        if constexpr (Prec<P>::MIX) {
          const size_t qs = source_node<WALL>(x, y, k, nx, ny);
          const T ref = Prec<P>::REF ? adv_units(cdotu(k, a.u_out[qs], a.u_out[V + qs]),
                                                 a.pp_out[(size_t)i * V + qs], T(3) * a.sh_st)
                                     : T(0);
          const Sm sv = store_once<Sm>(heq * (d.sh_st / w_of<double>(k)) - (double)ref);
          hm[((size_t)(i * 8 + k - 1)) * V + q] = sv;
          const T dec = Prec<P>::REF ? __fadd_rn(to_T(sv), ref) : to_T(sv);
          moving += (double)(w_of<T>(k) * a.sh_ld) * (double)dec;
        } else {
          const Sm hv = store_once<Sm>(heq);
          hm[((size_t)(i * 8 + k - 1)) * V + q] = hv;
          moving += (double)hv;
        }
      }
      // FP64: h_0 = h_0^eq. Other forms: d_0 = h_0 - phi(t-1) with phi(t-1)
      // the stored (rounded) phi, so that phi(t-1) + d_0 + sum_{k>=1} h_k is
      // phi up to the rounding of d_0.
      if constexpr (P == LBM_FP64)
        h0[(size_t)i * V + q] = ph[i] + (w_of<double>(0) - 1.0) * aC;
      else
        h0[(size_t)i * V + q] =
            store_once<T>((ph[i] - (double)a.pp_out[(size_t)i * V + q]) - moving);
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers for one precision.
// ---------------------------------------------------------------------------
template <int P, int NP, bool NU, bool WALL>
cudaError_t launch_tile_t(const Consts &c, const Grid &g, int cur, int mode,
                          const Outputs &o, cudaStream_t s) {
  const KArgs<P> a = make_args<P>(c, g, cur, mode, o);
  if constexpr (P != LBM_FP64 && !NU) {
    if (mode == MODE_STEP && g.use_tma && g.grad_scheme == 0) {
      typedef TmaStage<P, NP> St;
      constexpr int TBY = TmaGeom<P>::TBY;
      const bool whole = g.nx % BX == 0 && g.ny % TBY == 0 && g.nx > BX && g.ny > TBY;
      auto kern = whole ? tile_kernel_tma<P, NP, WALL, true> : tile_kernel_tma<P, NP, WALL, false>;
      static int max_ctas[2] = {0, 0};  // per instantiation: resident CTAs on the GPU
      int &mc = max_ctas[whole ? 1 : 0];
      if (mc == 0) {
        cudaError_t e = cudaFuncSetAttribute(
            kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)St::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TmaGeom<P>::NTH,
                                                          St::SMEM);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        mc = (per_sm > 0 ? per_sm : 1) * sms;
      }
      const int ntx = tiles_x(g.nx), ntiles = ntx * ((g.ny + TBY - 1) / TBY);
      const int grid = ntiles < mc ? ntiles : mc;
      kern<<<grid, dim3(BX, TBY), St::SMEM, s>>>(a, *(const TmaMaps *)&g.tma[cur], ntx, ntiles);
      return cudaGetLastError();
    }
  }
  dim3 grid(tiles_x(g.nx), tiles_y(g.ny)), block(BX, BY);
  if (g.grad_scheme == 1)
    tile_kernel<P, NP, NU, WALL, true><<<grid, block, 0, s>>>(a);
  else
    tile_kernel<P, NP, NU, WALL, false><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <int P, int NP>
cudaError_t launch_tile_np(const Consts &c, const Grid &g, int cur, int mode,
                           const Outputs &o, bool nonunif, bool wall,
                           cudaStream_t s) {
  if (nonunif)
    return wall ? launch_tile_t<P, NP, true, true>(c, g, cur, mode, o, s)
                : launch_tile_t<P, NP, true, false>(c, g, cur, mode, o, s);
  return wall ? launch_tile_t<P, NP, false, true>(c, g, cur, mode, o, s)
              : launch_tile_t<P, NP, false, false>(c, g, cur, mode, o, s);
}

template <int P>
cudaError_t launch_tile_p(const Consts &c, const Grid &g, int cur, int mode,
                          const Outputs &o, bool nonunif, bool wall,
                          cudaStream_t s) {
  switch (c.NP) {
    case 1: return launch_tile_np<P, 1>(c, g, cur, mode, o, nonunif, wall, s);
    case 2: return launch_tile_np<P, 2>(c, g, cur, mode, o, nonunif, wall, s);
    case 3: return launch_tile_np<P, 3>(c, g, cur, mode, o, nonunif, wall, s);
    case 4: return launch_tile_np<P, 4>(c, g, cur, mode, o, nonunif, wall, s);
  }
  return cudaErrorInvalidValue;
}

// Tensor maps of the pipelined kernel for both buffers; false if the grid
// does not meet TMA's alignment rules or an encode fails.
template <int P>
bool encode_tma_p(const Consts &c, Grid &g, EncodeTiledFn enc) {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  typedef TmaGeom<P> G;
  if constexpr (P == LBM_FP64) {
    return false;
  } else {
    if (!enc || g.nx % 8 != 0) return false;
    const int NP = c.NP;
    auto enc3 = [&](CUtensorMap *m, void *base, size_t es, int planes, int bw,
                    int bh, int bp) {
      const CUtensorMapDataType dt =
          es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
      const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny,
                                  (cuuint64_t)planes};
      const cuuint64_t strides[2] = {(cuuint64_t)g.nx * es,
                                     (cuuint64_t)g.nx * g.ny * es};
      const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bp};
      const cuuint32_t estr[3] = {1, 1, 1};
      return enc(m, dt, 3, base, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
      TmaMaps &m = *(TmaMaps *)&g.tma[b];
      bool ok = enc3(&m.hm, g.hm[b], sizeof(Sm), 8 * NP, G::WM, G::HB, 8 * NP) &&
                enc3(&m.h0, g.h0[b], sizeof(T), NP, G::WR, G::HB, NP) &&
                enc3(&m.pp, g.phi_prev[b], sizeof(T), NP, G::WR, G::HBP, NP) &&
                enc3(&m.gm, g.gm[b], sizeof(Sm), 8, BX, G::TBY, 8) &&
                enc3(&m.up, g.u_prev[b], sizeof(T), G::UPN, G::UW, G::UH, G::UPN);
      if (G::WRAP)
        ok = ok && enc3(&m.hmx, g.hm[b], sizeof(Sm), 8 * NP, G::HXM, G::HB, 8 * NP) &&
             enc3(&m.h0x, g.h0[b], sizeof(T), NP, G::HXR, G::HB, NP) &&
             enc3(&m.ppx, g.phi_prev[b], sizeof(T), NP, G::HXR, G::HBP, NP) &&
             enc3(&m.hmy, g.hm[b], sizeof(Sm), 8 * NP, G::WM, 1, 8 * NP) &&
             enc3(&m.h0y, g.h0[b], sizeof(T), NP, G::WR, 1, NP) &&
             enc3(&m.ppy, g.phi_prev[b], sizeof(T), NP, G::WR, 1, NP);
      if (!ok) return false;
    }
    return true;
  }
}

template <int P, int NP>
cudaError_t launch_init_np(const Consts &c, const Grid &g, int cur,
                           const double *cin, const double *uin, double p0,
                           bool wall, cudaStream_t s) {
  // The init kernels write into buffer `cur`: make_args puts the output
  // pointers at cur ^ 1, so pass cur ^ 1.
  const KArgs<P> a = make_args<P>(c, g, cur ^ 1, MODE_STEP, Outputs{});
  const int threads = 256;
  size_t blocks = (g.V + threads - 1) / threads;
  if (blocks > 65535u * 16u) blocks = 65535u * 16u;
  init_phi_kernel<P, NP><<<(unsigned)blocks, threads, 0, s>>>(
      a, cin, uin, g.scratch, c.rho_t[0], c.rho_t[1], c.rho_t[2], c.rho_t[3], c.rho_t[4]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const KArgs<LBM_FP64> d = make_args<LBM_FP64>(c, g, cur ^ 1, MODE_STEP, Outputs{});
  if (wall)
    init_pop_kernel<P, NP, true><<<(unsigned)blocks, threads, 0, s>>>(a, d, g.scratch, uin, p0);
  else
    init_pop_kernel<P, NP, false><<<(unsigned)blocks, threads, 0, s>>>(a, d, g.scratch, uin, p0);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_init_p(const Consts &c, const Grid &g, int cur,
                          const double *cin, const double *uin, double p0,
                          bool wall, cudaStream_t s) {
  switch (c.NP) {
    case 1: return launch_init_np<P, 1>(c, g, cur, cin, uin, p0, wall, s);
    case 2: return launch_init_np<P, 2>(c, g, cur, cin, uin, p0, wall, s);
    case 3: return launch_init_np<P, 3>(c, g, cur, cin, uin, p0, wall, s);
    case 4: return launch_init_np<P, 4>(c, g, cur, cin, uin, p0, wall, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm

#include "lbm_d3q15.cuh"

#define LBM_DEFINE_PREC(SUFFIX, P)                                             \
  namespace lbm {                                                              \
  cudaError_t launch_tile_##SUFFIX(const Consts &c, const Grid &g, int cur,    \
                                   int mode, const Outputs &o, bool nonunif,   \
                                   bool wall, cudaStream_t s) {                \
    return launch_tile_p<P>(c, g, cur, mode, o, nonunif, wall, s);             \
  }                                                                            \
  cudaError_t launch_init_##SUFFIX(const Consts &c, const Grid &g, int cur,    \
                                   const double *cin, const double *uin,       \
                                   double p0, bool wall, cudaStream_t s) {     \
    return launch_init_p<P>(c, g, cur, cin, uin, p0, wall, s);                 \
  }                                                                            \
  bool encode_tma_##SUFFIX(const Consts &c, Grid &g, EncodeTiledFn enc) {      \
    return encode_tma_p<P>(c, g, enc);                                         \
  }                                                                            \
  bool encode_tma3_##SUFFIX(const Consts &c, Grid &g, EncodeTiledFn enc) {     \
    return encode_tma3_p<P>(c, g, enc);                                        \
  }                                                                            \
  cudaError_t launch_tile3_##SUFFIX(const Consts &c, const Grid &g, int cur,   \
                                    int mode, const Outputs &o, bool nonunif,  \
                                    bool wall, cudaStream_t s) {               \
    return launch_tile3_p<P>(c, g, cur, mode, o, nonunif, wall, s);            \
  }                                                                            \
  cudaError_t launch_init3_##SUFFIX(const Consts &c, const Grid &g, int cur,   \
                                    const double *cin, const double *uin,      \
                                    double p0, bool wall, cudaStream_t s) {    \
    return launch_init3_p<P>(c, g, cur, cin, uin, p0, wall, s);                \
  }                                                                            \
  }
