// Three-dimensional variant on the D3Q15 lattice (Section 3.1): the same
// time step as the D2Q9 kernels with 15 velocities and the 14-neighbour
// stencils of Eq. N31. Grids are nx x ny x nz, node (x, y, z) at
// (z ny + y) nx + x, periodic in x and z, periodic or walled in y.
//
// Layout (per phase i): rest slot [i][V], moving populations [i][k-1][V]
// for k = 1..14, NS populations [k-1][V], phi(t-1) [i][V], u(t-1) [3][V].
// Included by lbm_kernels.cuh; instantiated per storage precision.
#pragma once

namespace lbm {

// D3Q15 (Section 3.1): 0 rest; 1..6 the faces (+x, +y, +z, -x, -y, -z);
// 7..14 the corners.
__host__ __device__ constexpr int c3x(int k) {
  return (k == 1 || k == 7 || k == 8 || k == 9 || k == 14) ? 1
         : (k == 4 || k == 10 || k == 11 || k == 12 || k == 13) ? -1 : 0;
}
__host__ __device__ constexpr int c3y(int k) {
  return (k == 2 || k == 7 || k == 8 || k == 10 || k == 13) ? 1
         : (k == 5 || k == 9 || k == 11 || k == 12 || k == 14) ? -1 : 0;
}
__host__ __device__ constexpr int c3z(int k) {
  return (k == 3 || k == 7 || k == 9 || k == 10 || k == 12) ? 1
         : (k == 6 || k == 8 || k == 11 || k == 13 || k == 14) ? -1 : 0;
}
template <typename T>
__host__ __device__ constexpr T w3_of(int k) {
  return k == 0 ? T(2) / T(9) : (k <= 6 ? T(1) / T(9) : T(1) / T(72));
}
__host__ __device__ constexpr int opp3(int k) {
  return k == 0 ? 0 : (k <= 6 ? (k <= 3 ? k + 3 : k - 3)
                              : (k == 7 ? 11 : k == 11 ? 7 : k == 8 ? 12 : k == 12 ? 8
                                 : k == 9 ? 13 : k == 13 ? 9 : k == 10 ? 14 : 10));
}
static_assert(c3x(opp3(8)) == -c3x(8) && c3y(opp3(8)) == -c3y(8) &&
                  c3z(opp3(8)) == -c3z(8) && c3x(opp3(10)) == -c3x(10) &&
                  c3y(opp3(13)) == -c3y(13) && c3z(opp3(9)) == -c3z(9),
              "D3Q15 opposites");

constexpr int BX3 = 32, BY3 = 4, BZ3 = 2, NT3 = BX3 * BY3 * BZ3;

template <int P> struct KArgs3 {
  KArgs<P> a;  // pointers, constants (u_in, u_out hold 3 planes)
  int nz;
};

// Stencils of Eq. N31 on a shared box (strides W, W * H): D3Q15 sums folded
// over the 7 pairs of opposite velocities.
template <typename T, int W, int H>
__device__ __forceinline__ void stencil3(const T *s, int lz, int ly, int lx,
                                         T *g, T &lap) {
  const int o = (lz * H + ly) * W + lx;
  const T c = s[o];
  T gx = T(0), gy = T(0), gz = T(0), l = T(0);
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    if (opp3(k) < k) continue;  // one of each pair
    const int d = (c3z(k) * H + c3y(k)) * W + c3x(k);
    const T p = s[o + d], m = s[o - d];
    const T wd = w3_of<T>(k) * (p - m);
    gx += T(c3x(k)) * wd;
    gy += T(c3y(k)) * wd;
    gz += T(c3z(k)) * wd;
    l += w3_of<T>(k) * (p + m - T(2) * c);
  }
  // pairs counted once: gradient 2 * sum / (2 c_s^2) = 3 sum; laplacian
  // 2 * sum / c_s^2 = 6 sum
  g[0] = T(3) * gx;
  g[1] = T(3) * gy;
  g[2] = T(3) * gz;
  lap = T(6) * l;
}

template <int P>
__device__ __forceinline__ typename Prec<P>::T load_hm3(const KArgs<P> &a, int i,
                                                        int k, size_t q) {
  return to_T(ldg(a.hm_in + ((size_t)(i * 14 + k - 1)) * a.V + q));
}

// 16-bit forms store every moving population relative to the advective (and
// for g the pressure) part of its equilibrium at the node it was streamed
// from, as in two dimensions (cdotu, adv_units, g_refp there): c_k . u with
// the same rounded operations on writer and reader (D3Q15 has face and corner
// velocities only).
__device__ __forceinline__ float cdotu3(int k, float ux, float uy, float uz) {
  const int cx = c3x(k), cy = c3y(k), cz = c3z(k);
  const float a = cx > 0 ? ux : -ux, b = cy > 0 ? uy : -uy, c = cz > 0 ? uz : -uz;
  if (cx != 0 && cy != 0 && cz != 0) return __fadd_rn(__fadd_rn(a, b), c);
  return cx != 0 ? a : (cy != 0 ? b : c);
}
__device__ __forceinline__ double cdotu3(int k, double ux, double uy, double uz) {
  return c3x(k) * ux + c3y(k) * uy + c3z(k) * uz;
}
__device__ __forceinline__ float g_ref3(float cu, float ux, float uy, float uz,
                                        float srho) {
  const float uu = __fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)),
                             __fmul_rn(uz, uz));
  const float in = __fadd_rn(__fadd_rn(__fmul_rn(3.0f, cu), __fmul_rn(4.5f, __fmul_rn(cu, cu))),
                             __fmul_rn(-1.5f, uu));
  return __fmul_rn(in, srho);
}
__device__ __forceinline__ double g_ref3(double cu, double ux, double uy,
                                         double uz, double srho) {
  return (3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy + uz * uz)) * srho;
}
// The same plus the pressure part 3 s p (s3 = 3 s); p(t-1) is the fourth
// plane of the u(t-1) buffers of the 16-bit forms.
template <typename T>
__device__ __forceinline__ T g_ref3p(T cu, T ux, T uy, T uz, T p, T srho, T s3) {
  return __fadd_rn(g_ref3(cu, ux, uy, uz, srho), __fmul_rn(p, s3));
}
// The node slot k of (x, y, z) was streamed from: (x, y, z) - c_k, periodic
// in x and z (and y without walls); behind a wall, (x, y, z) itself.
template <bool WALL>
__device__ __forceinline__ size_t source3(int x, int y, int z, int k, int nx,
                                          int ny, int nz) {
  int sx = x - c3x(k), sy = y - c3y(k), sz = z - c3z(k);
  if (WALL && (sy < 0 || sy >= ny)) {
    sx = x;
    sy = y;
    sz = z;
  }
  sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
  sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
  sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
  return ((size_t)sz * ny + sy) * nx + sx;
}
// The sources of one node's 14 moving slots, (x, y, z) - c_k, from wrapped
// x - 1..x + 1 and the row and plane offsets of y - 1..y + 1, z - 1..z + 1
// (computed once per node instead of once per slot); behind a wall in y the
// node itself. The same indices as source3.
template <bool WALL> struct Nb3 {
  size_t q, pz[3], ry[3];
  int xv[3];
  bool lo, hi;
  __device__ __forceinline__ Nb3(int x, int y, int z, size_t q_, int nx, int ny,
                                 int nz) {
    q = q_;
    xv[0] = x == 0 ? nx - 1 : x - 1;
    xv[1] = x;
    xv[2] = x + 1 >= nx ? x + 1 - nx : x + 1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      int yy = y + j - 1, zz = z + j - 1;
      if (WALL)
        yy = yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy);
      else
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
      zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
      ry[j] = (size_t)yy * nx;
      pz[j] = (size_t)zz * ny * nx;
    }
    lo = WALL && y == 0;
    hi = WALL && y == ny - 1;
  }
  __device__ __forceinline__ size_t src(int k) const {
    const int cx = c3x(k), cy = c3y(k), cz = c3z(k);
    if (WALL && ((cy > 0 && lo) || (cy < 0 && hi))) return q;
    return pz[1 - cz] + ry[1 - cy] + (size_t)xv[1 - cx];
  }
};

// phi_i of every phase at node (x, y, z) = q from the stored values (FP64:
// sum of the 15; other forms: phi(t-1) + (d_0 + sum_k h_k), TwoSum error
// dropped). 16-bit forms decode slot k with u(t-1), phi(t-1) of its source,
// looked up once for all phases. With OWN, the node's decoded h^i_1..14 and
// g_1..14 also go to own[slot * stride] (slot i * 14 + k - 1, then
// (NP - 1) * 14 + 13 + k for g), for the node's own step to read back.
template <int P, int NP, bool WALL, bool OWN = false>
__device__ __forceinline__ void node_phis3(const KArgs<P> &a, int nz, int x,
                                           int y, int z, size_t q,
                                           typename Prec<P>::T (&phi)[NP],
                                           typename Prec<P>::T *own = nullptr,
                                           int stride = 0) {
  typedef typename Prec<P>::T T;
  const size_t V = a.V;
  T small[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) small[i] = ldg(a.h0_in + (size_t)i * V + q);
  const Nb3<WALL> nb(x, y, z, q, a.nx, a.ny, nz);
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    T cu = T(0), ux = T(0), uy = T(0), uz = T(0);
    size_t qs = q;
    if constexpr (Prec<P>::REF) {
      qs = nb.src(k);
      ux = ldg(a.u_in + qs);
      uy = ldg(a.u_in + V + qs);
      uz = ldg(a.u_in + 2 * V + qs);
      cu = cdotu3(k, ux, uy, uz);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T x_ = load_hm3<P>(a, i, k, q);
      if constexpr (Prec<P>::REF)
        x_ = __fadd_rn(x_, adv_units(cu, ldg(a.pp_in + (size_t)i * V + qs), T(3) * a.sh_st));
      if constexpr (OWN) own[(i * 14 + k - 1) * stride] = x_;
      if constexpr (Prec<P>::MIX)
        small[i] = __fmaf_rn(w3_of<T>(k) * a.sh_ld, x_, small[i]);
      else
        small[i] = __fadd_rn_T(small[i], x_);
    }
    if constexpr (OWN) {
      T gk = to_T(ldg(a.gm_in + (size_t)(k - 1) * V + q));
      if constexpr (Prec<P>::REF)
        gk = __fadd_rn(gk, g_ref3p(cu, ux, uy, uz, ldg(a.u_in + 3 * V + qs),
                                   a.rho_base * a.sg_st, T(3) * a.sg_st));
      own[(NP * 14 + k - 1) * stride] = gk;
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if constexpr (P == LBM_FP64)
      phi[i] = small[i];
    else
      phi[i] = __fadd_rn(ldg(a.pp_in + (size_t)i * V + q), small[i]);
  }
}

template <bool WALL>
__device__ __forceinline__ size_t node3(int x, int y, int z, int nx, int ny,
                                        int nz) {
  return ((size_t)wrap(z, nz) * ny + wrap_y<WALL>(y, ny)) * nx + wrap(x, nx);
}

// The values a D3Q15 step reads at its own node: h^i_0 (FP64) or d^i_0 and
// h^i_1..14 (converted to T, stored units for the 16-bit forms), g_1..14 (the
// same), phi_i(t-1) and u(t-1).
template <int P, int NP> struct Own3 {
  typedef typename Prec<P>::T T;
  T h[NP][15], g[15], pp[NP], up[3];
};

template <int P, int NP, bool WALL>
__device__ __forceinline__ void load_own3(const KArgs<P> &a, int nz, int x,
                                          int y, int z, size_t q,
                                          Own3<P, NP> &o) {
  typedef typename Prec<P>::T T;
  const size_t V = a.V;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    o.h[i][0] = ldg(a.h0_in + (size_t)i * V + q);
#pragma unroll
    for (int k = 1; k < 15; ++k) o.h[i][k] = load_hm3<P>(a, i, k, q);
    o.pp[i] = ldg(a.pp_in + (size_t)i * V + q);
  }
#pragma unroll
  for (int k = 1; k < 15; ++k) o.g[k] = to_T(ldg(a.gm_in + (size_t)(k - 1) * V + q));
  if constexpr (Prec<P>::REF) {
    const Nb3<WALL> nb(x, y, z, q, a.nx, a.ny, nz);
#pragma unroll
    for (int k = 1; k < 15; ++k) {
      const size_t qs = nb.src(k);
      const T ux = ldg(a.u_in + qs), uy = ldg(a.u_in + V + qs),
              uz = ldg(a.u_in + 2 * V + qs);
      const T cu = cdotu3(k, ux, uy, uz);
#pragma unroll
      for (int i = 0; i < NP; ++i)
        o.h[i][k] = __fadd_rn(o.h[i][k], adv_units(cu, ldg(a.pp_in + (size_t)i * V + qs),
                                                   T(3) * a.sh_st));
      o.g[k] = __fadd_rn(o.g[k], g_ref3p(cu, ux, uy, uz, ldg(a.u_in + 3 * V + qs),
                                         a.rho_base * a.sg_st, T(3) * a.sg_st));
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) o.up[d] = a.u_in[(size_t)d * V + q];
}

// The same values, h and g decoded by node_phis3<..., OWN> into own[].
template <int P, int NP>
__device__ __forceinline__ void load_own3c(const KArgs<P> &a, size_t q,
                                           const typename Prec<P>::T *own,
                                           int stride, Own3<P, NP> &o) {
  const size_t V = a.V;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    o.h[i][0] = ldg(a.h0_in + (size_t)i * V + q);
#pragma unroll
    for (int k = 1; k < 15; ++k) o.h[i][k] = own[(i * 14 + k - 1) * stride];
    o.pp[i] = ldg(a.pp_in + (size_t)i * V + q);
  }
#pragma unroll
  for (int k = 1; k < 15; ++k) o.g[k] = own[(NP * 14 + k - 1) * stride];
#pragma unroll
  for (int d = 0; d < 3; ++d) o.up[d] = a.u_in[(size_t)d * V + q];
}

// phi_i from a node's values in registers, summed in the order of node_phis3.
template <int P>
__device__ __forceinline__ typename Prec<P>::T node_phi3r(
    const typename Prec<P>::T *h, typename Prec<P>::T pp,
    typename Prec<P>::T &err, typename Prec<P>::T sh_ld) {
  typedef typename Prec<P>::T T;
  T small = h[0];
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    if constexpr (Prec<P>::MIX)
      small = __fmaf_rn(w3_of<T>(k) * sh_ld, h[k], small);
    else
      small = __fadd_rn_T(small, h[k]);
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

// F = sum_i C_i grad phi_i + rho g, u (Eq. N22_1) and p (Eq. N23 on D3Q15)
// of one node from its stencil results and its NS populations g[1..14]
// (stored units).
template <int P, int NP>
__device__ __forceinline__ void macros3(
    const KArgs<P> &a, const typename Prec<P>::T (&gp)[NP][3],
    const typename Prec<P>::T *Cv, typename Prec<P>::T rho,
    const typename Prec<P>::T *gr, const typename Prec<P>::T (&g)[15],
    typename Prec<P>::T (&u)[3], typename Prec<P>::T (&F)[3],
    typename Prec<P>::T &uu, typename Prec<P>::T &pr) {
  typedef typename Prec<P>::T T;
  const T grav[3] = {a.grav[0], a.grav[1], a.grav_z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d] = rho * grav[d];
#pragma unroll
    for (int i = 0; i < NP; ++i) F[d] += Cv[i] * gp[i][d];
  }
  T mo[3] = {T(0), T(0), T(0)}, sg = T(0);
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    T gk = g[k];
    if constexpr (Prec<P>::MIX) gk *= w3_of<T>(k) * a.sg_ld;
    mo[0] += T(c3x(k)) * gk;
    mo[1] += T(c3y(k)) * gk;
    mo[2] += T(c3z(k)) * gk;
    sg += gk;
  }
  const T rinv = T(1) / rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = (mo[d] + T(0.5) * F[d]) * rinv;
  uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
  // Eq. N23 on D3Q15: c_s^2 / (1 - w_0) = 3/7, s_0 = -w_0 |u|^2 / (2 c_s^2)
  pr = T(3.0 / 7.0) * (sg + T(0.5) * ugr - rho * T(2.0 / 9.0) * T(1.5) * uu);
}

// Collisions of one D3Q15 node (Eqs. 24, N24 with Eqs. 25, N20_1, N25-N27),
// folded as in the D2Q9 kernels, and push streaming; phi(t) and u(t) become
// the next step's phi(t-1) and u(t-1).
template <int P, int NP, bool NU, bool WALL>
__device__ __forceinline__ void collide3(
    const KArgs<P> &a, int nz, const typename Prec<P>::T *ph,
    const typename Prec<P>::T *Cv, typename Prec<P>::T rho,
    const typename Prec<P>::T *gr, const typename Prec<P>::T *J,
    const Own3<P, NP> &o, const typename Prec<P>::T (&u)[3],
    const typename Prec<P>::T (&F)[3], typename Prec<P>::T uu,
    typename Prec<P>::T pr, size_t q, int gx, int gy, int gz) {
  typedef typename Prec<P>::T T;
  const int nx = a.nx, ny = a.ny;
  const size_t V = a.V;
  size_t dst[15];
  int dk[15];
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    const int yy = gy + c3y(k);
    if (WALL && (yy < 0 || yy >= ny)) {
      dst[k] = q;
      dk[k] = opp3(k);
    } else {
      dst[k] = node3<WALL>(gx + c3x(k), yy, gz + c3z(k), nx, ny, nz);
      dk[k] = k;
    }
  }
  constexpr bool MIX = Prec<P>::MIX;
  const T tg = a.tg_inv, ff = a.ffac;
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const T Ju = (J[0] * u[0] + J[1] * u[1] + J[2] * u[2]) * a.jfac;
  const T A0 = tg * (T(3) * pr - T(1.5) * rho * uu) - ff * (T(3) * uF + T(1.5) * Ju);
  const T B1 = T(3) * tg * rho, B2 = T(4.5) * tg * rho;
  const T C1 = T(3) * ff, D1 = T(9) * ff, E1 = T(3) * ff, E2 = T(4.5) * ff * a.jfac;
  const T keep_g = T(1) - tg;
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    const T cx = T(c3x(k)), cy = T(c3y(k)), cz = T(c3z(k));
    const T cu = cx * u[0] + cy * u[1] + cz * u[2];
    const T cF = cx * F[0] + cy * F[1] + cz * F[2];
    T inner = B1 + B2 * cu + D1 * cF;
    if constexpr (NU)
      inner += E1 * (cx * gr[0] + cy * gr[1] + cz * gr[2]) +
               E2 * (cx * J[0] + cy * J[1] + cz * J[2]);
    const T t = A0 + C1 * cF + cu * inner;
    if constexpr (MIX)
      a.gm_out[(size_t)(dk[k] - 1) * V + dst[k]] = to_S<typename Prec<P>::Sm>(
          keep_g * o.g[k] + a.sg_st * t -
          (Prec<P>::REF ? g_ref3p(cdotu3(dk[k], u[0], u[1], u[2]), u[0], u[1], u[2], pr,
                                  a.rho_base * a.sg_st, T(3) * a.sg_st)
                        : T(0)));
    else
      a.gm_out[(size_t)(dk[k] - 1) * V + dst[k]] = keep_g * o.g[k] + w3_of<T>(k) * t;
  }
  const T *up = o.up;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const T pp = o.pp[i];
    const T ti = a.tau_inv[i], aC = a.a[i] * Cv[i];
    T al = ti * aC, b[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      b[d] = T(3) * (ti * ph[i] * u[d] + a.src[i] * (ph[i] * u[d] - pp * up[d]));
    if constexpr (MIX) {
      al *= a.sh_st;
      for (int d = 0; d < 3; ++d) b[d] *= a.sh_st;
    }
    const T keep = T(1) - ti;
    T moving_sum = T(0), perr;
    // phi's rounding error of this node, from its values as loaded
    node_phi3r<P>(o.h[i], pp, perr, a.sh_ld);
#pragma unroll
    for (int k = 1; k < 15; ++k) {
      const T t = al + T(c3x(k)) * b[0] + T(c3y(k)) * b[1] + T(c3z(k)) * b[2];
      const T hk = o.h[i][k];
      const size_t oo = ((size_t)(i * 14 + dk[k] - 1)) * V + dst[k];
      if constexpr (MIX) {
        // relative to the advective part at this node, the slot's source
        const T ref = Prec<P>::REF
                          ? adv_units(cdotu3(dk[k], u[0], u[1], u[2]), ph[i], T(3) * a.sh_st)
                          : T(0);
        const auto sv = to_S<typename Prec<P>::Sm>(keep * hk + t - ref);
        a.hm_out[oo] = sv;
        moving_sum = __fmaf_rn(w3_of<T>(k) * a.sh_ld, __fadd_rn(to_T(sv), ref),
                               moving_sum);
      } else {
        const T hs = keep * hk + w3_of<T>(k) * t;
        a.hm_out[oo] = hs;
        moving_sum = __fadd_rn_T(moving_sum, hs);
      }
    }
    T rest;
    if constexpr (P == LBM_FP64) {
      rest = keep * o.h[i][0] + ti * (ph[i] + (w3_of<T>(0) - T(1)) * aC);
    } else {
      rest = __fsub_rn(perr, moving_sum);
    }
    a.h0_out[(size_t)i * V + q] = rest;
    a.pp_out[(size_t)i * V + q] = ph[i];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) a.u_out[(size_t)d * V + q] = u[d];
  if constexpr (Prec<P>::REF) a.u_out[3 * V + q] = pr;
}

template <int P, int NP, bool NU, bool WALL>
__global__ void __launch_bounds__(NT3, P == LBM_FP64 ? 1 : 2)
    tile3_kernel(const KArgs3<P> A) {
  typedef typename Prec<P>::T T;
  const KArgs<P> &a = A.a;
  constexpr int RC = NU ? 1 : 0;       // C ring radius
  constexpr int R = RC + 1;            // phi halo radius
  constexpr int W = BX3 + 2 * R, H = BY3 + 2 * R, D = BZ3 + 2 * R, PL = W * H * D;
  constexpr int CW = BX3 + 2 * RC, CH = BY3 + 2 * RC, CD = BZ3 + 2 * RC,
                CPL = CW * CH * CD;
  extern __shared__ __align__(16) unsigned char smem3[];
  T *sphi = (T *)smem3;
  T *sC = sphi + NP * PL;
  __shared__ double sred[NT3 / 32][8];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = (tz * BY3 + ty) * BX3 + tx;
  const int nx = a.nx, ny = a.ny, nz = A.nz;
  const size_t V = a.V;
  const int x0 = blockIdx.x * BX3, y0 = blockIdx.y * BY3, z0 = blockIdx.z * BZ3;
  const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
  const bool active = gx < nx && gy < ny && gz < nz;
  const size_t q = active ? (((size_t)gz * ny + gy) * nx + gx) : 0;

  // 1. phi on the box (tile + halo R), wrapped / ghost coordinates.
  for (int r = tid; r < PL; r += NT3) {
    const int lx = r % W, ly = (r / W) % H, lz = r / (W * H);
    const int hx = wrap(x0 - R + lx, nx), hy = wrap_y<WALL>(y0 - R + ly, ny),
              hz = wrap(z0 - R + lz, nz);
    const size_t q = ((size_t)hz * ny + hy) * nx + hx;
    T phv[NP];
    node_phis3<P, NP, WALL>(a, nz, hx, hy, hz, q, phv);
#pragma unroll
    for (int i = 0; i < NP; ++i) sphi[i * PL + r] = phv[i];
  }
  __syncthreads();
  // 2. Unequal densities: C on the tile and a ring of radius 1; wall ghost
  //    layers of C repeat the adjacent fluid layer.
  if constexpr (NU) {
    for (int r = tid; r < CPL; r += NT3) {
      const int cx = r % CW, cy = (r / CW) % CH, cz = r / (CW * CH);
      T ph[NP], lp[NP], cc[NP + 1], rho, hf[NP], gtmp[3];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        ph[i] = sphi[i * PL + ((cz + 1) * H + cy + 1) * W + cx + 1];
        stencil3<T, W, H>(sphi + i * PL, cz + 1, cy + 1, cx + 1, gtmp, lp[i]);
      }
      local_algebra<P, NP>(a, ph, cc, rho, hf);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T Ci = a.bulk * hf[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) Ci -= a.lam[i][j] * lp[j];
        sC[i * CPL + r] = Ci;
      }
    }
    __syncthreads();
    if constexpr (WALL) {
      for (int r = tid; r < CPL; r += NT3) {
        const int cx = r % CW, cy = (r / CW) % CH, cz = r / (CW * CH);
        const int yg = y0 - 1 + cy;
        if (yg < 0 || yg >= ny) {
          const int cys = (yg < 0 ? 0 : ny - 1) - y0 + 1;
#pragma unroll
          for (int i = 0; i < NP; ++i)
            sC[i * CPL + r] = sC[i * CPL + (cz * CH + cys) * CW + cx];
        }
      }
      __syncthreads();
    }
  }

  // 3. Own node: stencils, C, F, u, p.
  const int lz = tz + R, ly = ty + R, lx = tx + R;
  T ph[NP], gp[NP][3], Cv[NP], cc[NP + 1], rho;
  {
    T lp[NP], hf[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      ph[i] = sphi[i * PL + (lz * H + ly) * W + lx];
      stencil3<T, W, H>(sphi + i * PL, lz, ly, lx, gp[i], lp[i]);
    }
    local_algebra<P, NP, !NU>(a, ph, cc, rho, hf);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if constexpr (NU) {
        Cv[i] = sC[i * CPL + ((tz + 1) * CH + ty + 1) * CW + tx + 1];
      } else {
        T Ci = a.bulk * hf[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) Ci -= a.lam[i][j] * lp[j];
        Cv[i] = Ci;
      }
    }
  }
  T gr[3] = {T(0), T(0), T(0)}, J[3] = {T(0), T(0), T(0)};
  if constexpr (NU) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T cg[3], dummy;
      stencil3<T, CW, CH>(sC + i * CPL, tz + 1, ty + 1, tx + 1, cg, dummy);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        J[d] -= a.kmob[i] * cg[d];
        gr[d] += a.kap[i] * gp[i][d];
      }
    }
  }
  // own-node values (node 0 stands in for inactive threads)
  Own3<P, NP> own;
  load_own3<P, NP, WALL>(a, nz, active ? gx : 0, active ? gy : 0, active ? gz : 0,
                         q, own);
  T F[3], u[3], uu, pr;
  macros3<P, NP>(a, gp, Cv, rho, gr, own.g, u, F, uu, pr);
  if (a.mode == MODE_MOMENTS) {
    if (!active) return;
    if (a.o_phi)
      for (int i = 0; i < NP; ++i) a.o_phi[(size_t)i * V + q] = (double)ph[i];
    if (a.o_c)
      for (int k = 0; k <= NP; ++k) a.o_c[(size_t)k * V + q] = (double)cc[k];
    if (a.o_u)
      for (int d = 0; d < 3; ++d) a.o_u[(size_t)d * V + q] = (double)u[d];
    if (a.o_p) a.o_p[q] = (double)pr;
    if (a.o_rho) a.o_rho[q] = (double)rho;
    return;
  }
  if (a.mode == MODE_DIAG) {
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k <= NP + 2; ++k) {
      double v;
      if (k <= NP) v = active ? (double)cc[k] : 0.0;
      else if (k == NP + 1) v = active ? 0.5 * (double)rho * (double)uu : 0.0;
      else v = active ? sqrt((double)uu) : 0.0;
      v = (k == NP + 2) ? warp_max(v) : warp_sum(v);
      if (lane == 0) sred[wid][k] = v;
    }
    __syncthreads();
    if (tid <= NP + 2) {
      double v = sred[0][tid];
      for (int w = 1; w < NT3 / 32; ++w)
        v = (tid == NP + 2) ? fmax(v, sred[w][tid]) : v + sred[w][tid];
      const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.red[b * (NP + 3) + tid] = v;
    }
    return;
  }
  if (!active) return;

  collide3<P, NP, NU, WALL>(a, nz, ph, Cv, rho, gr, J, own, u, F, uu, pr, q,
                            gx, gy, gz);
}

// ---------------------------------------------------------------------------
// z-marching step kernel (equal densities, central scheme). A CTA owns a
// 32 x 8 column of the grid and walks a slab of z planes. phi of plane z + 1
// is summed on the column's tile and its xy ring into a rolling window of
// three planes (z - 1, z, z + 1) in shared memory, so a node's phi is summed
// once per slab (plus the 84 ring positions per 256 nodes of a plane)
// instead of on a 3-D halo box around every tile; the 14 stencil neighbours
// of a node of plane z then come from the window. The per-node step is the
// one of tile3_kernel (macros3, collide3).
// ---------------------------------------------------------------------------
constexpr int MX3 = 32, MY3 = 8, MT3 = MX3 * MY3;
// dynamic shared memory of march3_kernel: 14 (N - 1) + 14 decoded values
// per column, then the three-plane phi window (tile and xy ring)
template <int P, int NP> __host__ __device__ constexpr size_t march3_cache_bytes() {
  return (size_t)(NP * 14 + 14) * MT3 * sizeof(typename Prec<P>::T);
}
template <int P, int NP> __host__ __device__ constexpr size_t march3_smem() {
  return march3_cache_bytes<P, NP>() +
         (size_t)3 * NP * (MX3 + 2) * (MY3 + 2) * sizeof(typename Prec<P>::T);
}

// Eq. N31 on D3Q15 from three planes (z - 1, z, z + 1) of stride W, pairs of
// opposite velocities summed in the order of stencil3.
template <typename T, int W>
__device__ __forceinline__ void stencil3w(const T *pm, const T *p0, const T *pp,
                                          int ly, int lx, T *g, T &lap) {
  const int o = ly * W + lx;
  const T c = p0[o];
  T gx = T(0), gy = T(0), gz = T(0), l = T(0);
#pragma unroll
  for (int k = 1; k < 15; ++k) {
    if (opp3(k) < k) continue;
    const T *plus = c3z(k) > 0 ? pp : (c3z(k) < 0 ? pm : p0);
    const T *minus = c3z(k) > 0 ? pm : (c3z(k) < 0 ? pp : p0);
    const int d = c3y(k) * W + c3x(k);
    const T p = plus[o + d], m = minus[o - d];
    const T wd = w3_of<T>(k) * (p - m);
    gx += T(c3x(k)) * wd;
    gy += T(c3y(k)) * wd;
    gz += T(c3z(k)) * wd;
    l += w3_of<T>(k) * (p + m - T(2) * c);
  }
  g[0] = T(3) * gx;
  g[1] = T(3) * gy;
  g[2] = T(3) * gz;
  lap = T(6) * l;
}

// The step of one node of plane z from the phi window (planes z - 1, z, z + 1
// with the xy ring, stride SW) and the node's own values (equal densities).
template <int P, int NP, bool WALL, int SW, int PL>
__device__ __forceinline__ void march3_node(
    const KArgs<P> &a, int nz, const typename Prec<P>::T (*wm)[PL],
    const typename Prec<P>::T (*w0)[PL], const typename Prec<P>::T (*wp)[PL],
    int tx, int ty, const Own3<P, NP> &own, size_t q, int gx, int gy, int z) {
  typedef typename Prec<P>::T T;
  T ph[NP], gp[NP][3], Cv[NP], cc[NP + 1], rho;
  {
    T lp[NP], hf[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      ph[i] = w0[i][(ty + 1) * SW + tx + 1];
      stencil3w<T, SW>(wm[i], w0[i], wp[i], ty + 1, tx + 1, gp[i], lp[i]);
    }
    local_algebra<P, NP, true>(a, ph, cc, rho, hf);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T Ci = a.bulk * hf[i];
#pragma unroll
      for (int j = 0; j < NP; ++j) Ci -= a.lam[i][j] * lp[j];
      Cv[i] = Ci;
    }
  }
  const T gr[3] = {T(0), T(0), T(0)}, J[3] = {T(0), T(0), T(0)};
  T F[3], u[3], uu, pr;
  macros3<P, NP>(a, gp, Cv, rho, gr, own.g, u, F, uu, pr);
  collide3<P, NP, false, WALL>(a, nz, ph, Cv, rho, gr, J, own, u, F, uu, pr, q, gx, gy, z);
}

template <int P, int NP, bool WALL>
__global__ void __launch_bounds__(MT3, P == LBM_FP64 ? 1 : 2)
    march3_kernel(const KArgs3<P> A, int zlen) {
  typedef typename Prec<P>::T T;
  const KArgs<P> &a = A.a;
  constexpr int SW = MX3 + 2, SH = MY3 + 2, PL = SW * SH;
  // the own column's decoded h and g of the plane summed last, then the
  // window (march3_smem)
  extern __shared__ __align__(16) unsigned char smem_m3[];
  T *ocache = (T *)smem_m3;
  T(*win)[NP][PL] = (T(*)[NP][PL])(smem_m3 + march3_cache_bytes<P, NP>());
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * MX3 + tx;
  const int nx = a.nx, ny = a.ny, nz = A.nz;
  const int x0 = blockIdx.x * MX3, y0 = blockIdx.y * MY3;
  const int zs = blockIdx.z * zlen;
  const int ze = zs + zlen < nz ? zs + zlen : nz;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col = gx < nx && gy < ny;
  // window slot of plane z (z >= zs - 1)
  auto slot = [&](int z) { return (z - zs + 1) % 3; };
  // phi of plane z on the tile (wrapped where the tile overhangs the grid)
  // and its xy ring
  // (the own column's decoded values go to the cache, also on the two
  // planes outside the slab, where they are not used: a guard there cost
  // the 16-bit forms 40%)
  auto plane_phi = [&](int z) {
    T(*w)[PL] = win[slot(z)];
    const int zz = wrap(z, nz);
    {
      const int cx = wrap(gx, nx), cy = wrap_y<WALL>(gy, ny);
      const size_t q = ((size_t)zz * ny + cy) * nx + cx;
      T phv[NP];
      node_phis3<P, NP, WALL, true>(a, nz, cx, cy, zz, q, phv, ocache + tid, MT3);
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i][(ty + 1) * SW + tx + 1] = phv[i];
    }
    constexpr int NRING = PL - MT3;
    static_assert(NRING <= MT3, "one ring position per thread");
    if (tid < NRING) {
      int lx, ly;
      ring_pos_1<MY3>(tid, lx, ly);
      const int rx = wrap(x0 - 1 + lx, nx), ry = wrap_y<WALL>(y0 - 1 + ly, ny);
      const size_t q = ((size_t)zz * ny + ry) * nx + rx;
      T phv[NP];
      node_phis3<P, NP, WALL>(a, nz, rx, ry, zz, q, phv);
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i][ly * SW + lx] = phv[i];
    }
  };
  plane_phi(zs - 1);
  plane_phi(zs);
  for (int z = zs; z < ze; ++z) {
    // this plane's own-node values (decoded when phi of this plane was
    // summed) first, then phi of the next plane
    const size_t q = col ? ((size_t)z * ny + gy) * nx + gx : 0;
    Own3<P, NP> own;
    load_own3c<P, NP>(a, q, ocache + tid, MT3, own);
    plane_phi(z + 1);
    __syncthreads();
    if (col)
      march3_node<P, NP, WALL, SW, PL>(a, nz, win[slot(z - 1)], win[slot(z)],
                                       win[slot(z + 1)], tx, ty, own, q, gx, gy, z);
    __syncthreads();  // plane z - 1's slot is refilled next
  }
}

// ---------------------------------------------------------------------------
// The z-marching step with its planes staged by TMA (FP32, N <= 4, nx a
// multiple of 4): per plane one 4-D box per array, the column with one halo
// row and four halo columns (h^i_k, d^i_0, phi_i(t-1)) or the column alone
// (g_k, u(t-1)), into two stages; the boxes of plane z + 2 load while plane
// z + 1's phi is summed and plane z stepped. Ring positions that wrap around
// the grid (or lie on a wall's ghost row) and columns that overhang it read
// global memory; everything else comes from the stage, with the same
// arithmetic as march3_kernel. One CTA of 8 warps per SM.
// ---------------------------------------------------------------------------
template <int P, int NP> struct March3Stage {
  typedef typename Prec<P>::T T;
  static constexpr int HX = 16 / (int)sizeof(T);  // halo columns (16-byte TMA x)
  static constexpr int BW = MX3 + 2 * HX, BH = MY3 + 2;
  static constexpr size_t al(size_t b) { return (b + 127) & ~(size_t)127; }
  static constexpr size_t HM = al((size_t)NP * 14 * BH * BW * sizeof(T));
  static constexpr size_t H0 = al((size_t)NP * BH * BW * sizeof(T));
  static constexpr size_t PP = H0;
  static constexpr size_t GM = al((size_t)14 * MY3 * MX3 * sizeof(T));
  static constexpr size_t UP = al((size_t)3 * MY3 * MX3 * sizeof(T));
  static constexpr size_t BASE = HM + H0 + PP + GM + UP;  // offset of the wrap boxes
  static constexpr uint32_t TX =
      (uint32_t)(((size_t)NP * 16 * BH * BW + (size_t)17 * MY3 * MX3) * sizeof(T));
  static constexpr size_t WIN = (size_t)3 * NP * (MX3 + 2) * (MY3 + 2) * sizeof(T);
  // The ring column (x) and row (y) that wrap around a periodic grid are
  // staged too, for edge columns: 16 bytes of columns at the far x edge over
  // the box height, and one row at the far y edge over the box width, of
  // the h, d_0 and phi(t-1) arrays (16 NP planes). The row only where it
  // fits beside the rest (N <= 3).
  // (each box at a 128-byte boundary of shared memory, as TMA requires)
  static constexpr size_t XHM = al((size_t)14 * NP * BH * HX * sizeof(T));
  static constexpr size_t XH0 = al((size_t)NP * BH * HX * sizeof(T));
  static constexpr size_t XW = XHM + 2 * XH0;
  static constexpr size_t YHM = al((size_t)14 * NP * BW * sizeof(T));
  static constexpr size_t YH0 = al((size_t)NP * BW * sizeof(T));
  static constexpr size_t YW0 = YHM + 2 * YH0;
  static constexpr bool WRAP_Y = 2 * (BASE + XW + YW0) + WIN + 16 <= 232448;
  static constexpr size_t YW = WRAP_Y ? YW0 : 0;
  static constexpr uint32_t XTX = (uint32_t)((size_t)16 * NP * BH * HX * sizeof(T));
  static constexpr uint32_t YTX = (uint32_t)((size_t)16 * NP * BW * sizeof(T));
  static constexpr size_t BYTES = BASE + XW + YW;
  static constexpr size_t SMEM = 2 * BYTES + WIN + 16;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x,
                                            int y, int z, int w, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

template <int P, int NP, bool WALL>
__global__ void __launch_bounds__(MT3, 1)
    march3_tma_kernel(const KArgs3<P> A, const __grid_constant__ TmaMaps maps, int zlen) {
  typedef typename Prec<P>::T T;
  typedef March3Stage<P, NP> St;
  const KArgs<P> &a = A.a;
  constexpr int SW = MX3 + 2, SH = MY3 + 2, PL = SW * SH;
  constexpr int BW = St::BW, BH = St::BH, HX = St::HX;
  extern __shared__ __align__(128) unsigned char smem_t3[];
  T(*win)[NP][PL] = (T(*)[NP][PL])(smem_t3 + 2 * St::BYTES);
  uint64_t *bar = (uint64_t *)(smem_t3 + 2 * St::BYTES + St::WIN);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * MX3 + tx;
  const int nx = a.nx, ny = a.ny, nz = A.nz;
  const int x0 = blockIdx.x * MX3, y0 = blockIdx.y * MY3;
  const int zs = blockIdx.z * zlen;
  const int ze = zs + zlen < nz ? zs + zlen : nz;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool col = gx < nx && gy < ny;
  auto slot = [&](int z) { return (z - zs + 1) % 3; };
  // stage and barrier of plane p >= zs; the barrier's k-th completion
  // (parity k & 1) is the k-th plane loaded into that stage
  auto stage = [&](int p) { return smem_t3 + ((p - zs) & 1) * St::BYTES; };
  // which wrapped halo column (1: x = -1 from nx - 4 .. nx - 1; 2: x = nx
  // from 0 .. 3) and row (1: y = -1 from ny - 1; 2: y = ny from 0; none with
  // walls, whose ghost rows repeat a row of the box) this column stages
  const int wx = x0 == 0 ? 1 : (x0 + MX3 == nx ? 2 : 0);
  const int wy = (!St::WRAP_Y || WALL) ? 0 : (y0 == 0 ? 1 : (y0 + MY3 == ny ? 2 : 0));
  auto issue = [&](int p) {  // thread 0
    unsigned char *st = stage(p);
    uint64_t *b = bar + ((p - zs) & 1);
    const int pz = wrap(p, nz);
    mbar_expect_tx(b, St::TX + (wx ? St::XTX : 0u) + (wy ? St::YTX : 0u));
    tma_load_4d(st, &maps.hm, x0 - HX, y0 - 1, pz, 0, b);
    tma_load_4d(st + St::HM, &maps.h0, x0 - HX, y0 - 1, pz, 0, b);
    tma_load_4d(st + St::HM + St::H0, &maps.pp, x0 - HX, y0 - 1, pz, 0, b);
    tma_load_4d(st + St::HM + St::H0 + St::PP, &maps.gm, x0, y0, pz, 0, b);
    tma_load_4d(st + St::HM + St::H0 + St::PP + St::GM, &maps.up, x0, y0, pz, 0, b);
    unsigned char *w = st + St::BASE;
    if (wx) {  // planes h_1..14, d_0, phi(t-1) per phase: 14 NP, NP, NP
      const int xs = wx == 1 ? nx - HX : 0;
      tma_load_4d(w, &maps.hmx, xs, y0 - 1, pz, 0, b);
      tma_load_4d(w + St::XHM, &maps.h0x, xs, y0 - 1, pz, 0, b);
      tma_load_4d(w + St::XHM + St::XH0, &maps.ppx, xs, y0 - 1, pz, 0, b);
    }
    if (wy) {
      const int ys = wy == 1 ? ny - 1 : 0;
      w += St::XW;
      tma_load_4d(w, &maps.hmy, x0 - HX, ys, pz, 0, b);
      tma_load_4d(w + St::YHM, &maps.h0y, x0 - HX, ys, pz, 0, b);
      tma_load_4d(w + St::YHM + St::YH0, &maps.ppy, x0 - HX, ys, pz, 0, b);
    }
  };
  auto wait = [&](int p) {
    return mbar_wait(bar + ((p - zs) & 1), (uint32_t)(((p - zs) >> 1) & 1));
  };
  // phi from staged planes, summed as in node_phis3: planes `pst` apart in
  // the h (14 NP), d_0 (NP) and phi(t-1) (NP) arrays that start at hm, h0,
  // pp, the position at offset o in each plane
  auto sum_phis = [&](const T *hm, const T *h0, const T *pp, int pst, int o, T(&phv)[NP]) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T small = h0[i * pst + o];
#pragma unroll
      for (int k = 1; k < 15; ++k) small = __fadd_rn_T(small, hm[(i * 14 + k - 1) * pst + o]);
      phv[i] = __fadd_rn(pp[i * pst + o], small);
    }
  };
  // phi at box position (bx, by) of a stage
  auto box_phis = [&](const unsigned char *st, int bx, int by, T(&phv)[NP]) {
    sum_phis((const T *)st, (const T *)(st + St::HM), (const T *)(st + St::HM + St::H0),
             BH * BW, by * BW + bx, phv);
  };
  // phi of plane z on the tile and its xy ring, from global memory (plane
  // zs - 1) or from the stage (planes zs .. ze)
  auto plane_phi = [&](int z, bool staged) {
    T(*w)[PL] = win[slot(z)];
    const int zz = wrap(z, nz);
    {
      T phv[NP];
      if (staged && col) {
        box_phis(stage(z), tx + HX, ty + 1, phv);
      } else {
        const int cx = wrap(gx, nx), cy = wrap_y<WALL>(gy, ny);
        node_phis3<P, NP, WALL>(a, nz, cx, cy, zz, ((size_t)zz * ny + cy) * nx + cx, phv);
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i][(ty + 1) * SW + tx + 1] = phv[i];
    }
    // ring positions on warps 1..3 (threads 32 .. 32 + NRING - 1): warp 0
    // holds the thread that issues the plane copies
    constexpr int NRING = PL - MT3;
    static_assert(32 + NRING <= MT3, "one ring position per thread");
    if (tid >= 32 && tid < 32 + NRING) {
      int lx, ly;
      ring_pos_1<MY3>(tid - 32, lx, ly);
      const int X = x0 - 1 + lx, Y = y0 - 1 + ly;
      T phv[NP];
      const bool inx = X >= 0 && X < nx, iny = Y >= 0 && Y < ny;
      const unsigned char *wb = stage(z) + St::BASE;
      if (staged && inx && iny) {
        box_phis(stage(z), lx - 1 + HX, ly, phv);
      } else if (staged && iny && ((X < 0 && wx == 1) || (X >= nx && wx == 2))) {
        // the staged wrapped column
        sum_phis((const T *)wb, (const T *)(wb + St::XHM), (const T *)(wb + St::XHM + St::XH0),
                 BH * HX, ly * HX + (X < 0 ? HX - 1 : 0), phv);
      } else if (staged && inx && WALL) {  // a wall's ghost row: the adjacent row
        box_phis(stage(z), lx - 1 + HX, wrap_y<WALL>(Y, ny) - y0 + 1, phv);
      } else if (staged && inx && ((Y < 0 && wy == 1) || (Y >= ny && wy == 2))) {
        const unsigned char *yw = wb + St::XW;  // the staged wrapped row
        sum_phis((const T *)yw, (const T *)(yw + St::YHM), (const T *)(yw + St::YHM + St::YH0),
                 BW, lx - 1 + HX, phv);
      } else {
        const int rx = wrap(X, nx), ry = wrap_y<WALL>(Y, ny);
        node_phis3<P, NP, WALL>(a, nz, rx, ry, zz, ((size_t)zz * ny + ry) * nx + rx, phv);
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i][ly * SW + lx] = phv[i];
    }
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    issue(zs);
    if (zs + 1 <= ze) issue(zs + 1);
  }
  __syncthreads();
  plane_phi(zs - 1, false);
  bool ok = wait(zs);
  plane_phi(zs, true);
  int failed_at = -1;
  for (int z = zs; z < ze; ++z) {
    // own values of plane z from its stage, then the stage is free for
    // plane z + 2 once every thread has read it
    Own3<P, NP> own;
    if (col) {
      const unsigned char *st = stage(z);
      const T *hm = (const T *)st, *h0 = (const T *)(st + St::HM),
              *pp = (const T *)(st + St::HM + St::H0),
              *gm = (const T *)(st + St::HM + St::H0 + St::PP),
              *up = (const T *)(st + St::HM + St::H0 + St::PP + St::GM);
      const int o = (ty + 1) * BW + tx + HX;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        own.h[i][0] = h0[i * BH * BW + o];
#pragma unroll
        for (int k = 1; k < 15; ++k) own.h[i][k] = hm[(i * 14 + k - 1) * BH * BW + o];
        own.pp[i] = pp[i * BH * BW + o];
      }
#pragma unroll
      for (int k = 1; k < 15; ++k) own.g[k] = gm[((k - 1) * MY3 + ty) * MX3 + tx];
#pragma unroll
      for (int d = 0; d < 3; ++d) own.up[d] = up[(d * MY3 + ty) * MX3 + tx];
    }
    __syncthreads();
    if (tid == 0 && z + 2 <= ze) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(z + 2);
    }
    ok = wait(z + 1) && ok;
    plane_phi(z + 1, true);
    // phi of plane z + 1 complete, and the decision to stop CTA-wide
    if (__syncthreads_or(!ok)) {
      failed_at = z;
      break;
    }
    if (col)
      march3_node<P, NP, WALL, SW, PL>(a, nz, win[slot(z - 1)], win[slot(z)],
                                       win[slot(z + 1)], tx, ty, own,
                                       ((size_t)z * ny + gy) * nx + gx, gx, gy, z);
  }
  if (failed_at >= 0 || !ok) {
    // record the timeout and let the loads still in flight land (bounded)
    if (tid == 0) {
      atomicExch(a.err, 1);
      const int last = failed_at + 2 <= ze ? failed_at + 2 : ze;
      for (int p = (failed_at >= 0 ? failed_at + 1 : zs); p <= last; ++p) wait(p);
    }
    __syncthreads();
  }
}

// As init_phi_kernel: phi_i also to phid[i][V] in FP64 (phid may be c).
template <int P, int NP>
__global__ void init3_phi_kernel(const KArgs<P> a, const double *c,
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
    for (int i = 0; i < NP; ++i) {
      const double ci = c[(size_t)i * a.V + q];
      ph[i] = (2.0 * (rt[i] * ci - rN * cN) - (rt[i] - rN)) / (rt[i] + rN);
    }
    for (int i = 0; i < NP; ++i) {
      a.pp_out[(size_t)i * a.V + q] = (T)ph[i];
      phid[(size_t)i * a.V + q] = ph[i];
    }
    for (int d = 0; d < 3; ++d) a.u_out[(size_t)d * a.V + q] = u ? (T)u[(size_t)d * a.V + q] : T(0);
  }
}

// Equilibrium start in FP64 for every storage form (as init_pop_kernel in
// two dimensions): phi, its Laplacian, C_i, h^eq and g^eq in double with the
// constants `d`, each stored value rounded once into its form.
template <int P, int NP, bool WALL>
__global__ void init3_pop_kernel(const KArgs3<P> A, const KArgs<LBM_FP64> d,
                                 const double *__restrict__ phid,
                                 const double *__restrict__ uin, double p0) {
  typedef typename Prec<P>::T T;
  typedef typename Prec<P>::Sm Sm;
  const KArgs<P> &a = A.a;
  const int nx = a.nx, ny = a.ny, nz = A.nz;
  const size_t V = a.V;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < V;
       q += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(q % nx), y = (int)((q / nx) % ny), z = (int)(q / ((size_t)nx * ny));
    double ph[NP], lp[NP];
    for (int i = 0; i < NP; ++i) {
      double s[27];
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            s[((dz + 1) * 3 + dy + 1) * 3 + dx + 1] =
                phid[(size_t)i * V + node3<WALL>(x + dx, y + dy, z + dz, nx, ny, nz)];
      double gtmp[3];
      ph[i] = s[13];
      stencil3<double, 3, 3>(s, 1, 1, 1, gtmp, lp[i]);
    }
    double cc[NP + 1], rho, hf[NP];
    local_algebra<LBM_FP64, NP>(d, ph, cc, rho, hf);
    double u[3];
    for (int e = 0; e < 3; ++e) u[e] = uin ? uin[(size_t)e * V + q] : 0.0;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if constexpr (Prec<P>::REF) a.u_out[3 * V + q] = (T)p0;
    for (int k = 1; k < 15; ++k) {
      const double cu = c3x(k) * u[0] + c3y(k) * u[1] + c3z(k) * u[2];
      const double geq =
          w3_of<double>(k) * (3.0 * p0 + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
      if constexpr (Prec<P>::MIX) {
        const size_t qs = source3<WALL>(x, y, z, k, nx, ny, nz);
        const T sux = a.u_out[qs], suy = a.u_out[V + qs], suz = a.u_out[2 * V + qs];
        // every source starts at p0 (stored as its p(t-1) above)
        const T ref = Prec<P>::REF ? g_ref3p(cdotu3(k, sux, suy, suz), sux, suy, suz,
                                             (T)p0, a.rho_base * a.sg_st, T(3) * a.sg_st)
                                   : T(0);
        a.gm_out[(size_t)(k - 1) * V + q] =
            store_once<Sm>(geq * (d.sg_st / w3_of<double>(k)) - (double)ref);
      } else
        a.gm_out[(size_t)(k - 1) * V + q] = store_once<Sm>(geq);
    }
    for (int i = 0; i < NP; ++i) {
      double Ci = d.bulk * hf[i];
      for (int j = 0; j < NP; ++j) Ci -= d.lam[i][j] * lp[j];
      const double aC = d.a[i] * Ci;
      double moving = 0.0;  // sum of the moving populations as stored
      for (int k = 1; k < 15; ++k) {
        const double cu = c3x(k) * u[0] + c3y(k) * u[1] + c3z(k) * u[2];
        const double heq = w3_of<double>(k) * (aC + 3.0 * ph[i] * cu);
        if constexpr (Prec<P>::MIX) {
          const size_t qs = source3<WALL>(x, y, z, k, nx, ny, nz);
          const T ref =
              Prec<P>::REF
                  ? adv_units(cdotu3(k, a.u_out[qs], a.u_out[V + qs], a.u_out[2 * V + qs]),
                              a.pp_out[(size_t)i * V + qs], T(3) * a.sh_st)
                  : T(0);
          const Sm sv = store_once<Sm>(heq * (d.sh_st / w3_of<double>(k)) - (double)ref);
          a.hm_out[((size_t)(i * 14 + k - 1)) * V + q] = sv;
          moving += (double)(w3_of<T>(k) * a.sh_ld) * (double)__fadd_rn(to_T(sv), ref);
        } else {
          const Sm hv = store_once<Sm>(heq);
          a.hm_out[((size_t)(i * 14 + k - 1)) * V + q] = hv;
          moving += (double)hv;
        }
      }
      if constexpr (P == LBM_FP64)
        a.h0_out[(size_t)i * V + q] = ph[i] + (w3_of<double>(0) - 1.0) * aC;
      else
        a.h0_out[(size_t)i * V + q] =
            store_once<T>((ph[i] - (double)a.pp_out[(size_t)i * V + q]) - moving);
    }
  }
}

template <int P, int NP, bool NU, bool WALL>
cudaError_t launch_tile3_t(const Consts &c, const Grid &g, int cur, int mode,
                           const Outputs &o, cudaStream_t s) {
  typedef typename Prec<P>::T T;
  KArgs3<P> A;
  A.a = make_args<P>(c, g, cur, mode, o);
  A.nz = g.nz;
  if constexpr (!NU) {
    if (mode == MODE_STEP && g.march3) {
      // slabs of z planes: enough CTAs to fill the GPU (~1216), at least 8
      // planes per slab (each slab sums phi on two extra planes)
      const int txy = tiles_x(g.nx) * ((g.ny + MY3 - 1) / MY3);
      long long zl = ((long long)g.nz * txy + 1215) / 1216;
      if (zl < 8) zl = 8;
      if (zl > g.nz) zl = g.nz;
      const int zlen = (int)zl;
      dim3 grid(tiles_x(g.nx), (g.ny + MY3 - 1) / MY3, (g.nz + zlen - 1) / zlen);
      if constexpr (P == LBM_FP32 && NP <= 3) {
        if (g.tma3) {
          typedef March3Stage<P, NP> St;
          static bool tattr = false;
          if (!tattr) {
            cudaError_t e = cudaFuncSetAttribute(march3_tma_kernel<P, NP, WALL>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)St::SMEM);
            if (e != cudaSuccess) return e;
            tattr = true;
          }
          march3_tma_kernel<P, NP, WALL><<<grid, dim3(MX3, MY3), St::SMEM, s>>>(
              A, *(const TmaMaps *)&g.tma[cur], zlen);
          return cudaGetLastError();
        }
      }
      constexpr size_t msm = march3_smem<P, NP>();
      static bool mattr = false;
      if (!mattr) {
        cudaError_t e = cudaFuncSetAttribute(march3_kernel<P, NP, WALL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)msm);
        if (e != cudaSuccess) return e;
        mattr = true;
      }
      march3_kernel<P, NP, WALL><<<grid, dim3(MX3, MY3), msm, s>>>(A, zlen);
      return cudaGetLastError();
    }
  }
  constexpr int RC = NU ? 1 : 0, R = RC + 1;
  constexpr size_t smem = (size_t)NP * ((BX3 + 2 * R) * (BY3 + 2 * R) * (BZ3 + 2 * R) +
                                        (NU ? (BX3 + 2) * (BY3 + 2) * (BZ3 + 2) : 0)) *
                          sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tile3_kernel<P, NP, NU, WALL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(tiles3_x(g.nx), tiles3_y(g.ny), tiles3_z(g.nz)), block(BX3, BY3, BZ3);
  tile3_kernel<P, NP, NU, WALL><<<grid, block, smem, s>>>(A);
  return cudaGetLastError();
}

template <int P, int NP>
cudaError_t launch_tile3_np(const Consts &c, const Grid &g, int cur, int mode,
                            const Outputs &o, bool nonunif, bool wall,
                            cudaStream_t s) {
  if (nonunif)
    return wall ? launch_tile3_t<P, NP, true, true>(c, g, cur, mode, o, s)
                : launch_tile3_t<P, NP, true, false>(c, g, cur, mode, o, s);
  return wall ? launch_tile3_t<P, NP, false, true>(c, g, cur, mode, o, s)
              : launch_tile3_t<P, NP, false, false>(c, g, cur, mode, o, s);
}

// Tensor maps of the TMA z-marching kernel for both state buffers: each
// array as a 4-D tensor (x, y, z, plane); FP32 with 2 to 4 phases and nx a
// multiple of 4 (16-byte row pitch) only.
template <int P>
bool encode_tma3_p(const Consts &c, Grid &g, EncodeTiledFn enc) {
  if constexpr (P != LBM_FP32) {
    return false;
  } else {
    const int NP = c.NP;
    if (!enc || NP < 1 || NP > 3 || g.nx % 4 != 0) return false;
    typedef March3Stage<P, 1> S1;
    auto enc4 = [&](CUtensorMap *m, void *base, int planes, int bw, int bh) {
      const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                  (cuuint64_t)planes};
      const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4,
                                     (cuuint64_t)g.V * 4};
      const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 1, (cuuint32_t)planes};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
      TmaMaps &m = *(TmaMaps *)&g.tma[b];
      const bool ok = enc4(&m.hm, g.hm[b], 14 * NP, S1::BW, S1::BH) &&
                      enc4(&m.h0, g.h0[b], NP, S1::BW, S1::BH) &&
                      enc4(&m.pp, g.phi_prev[b], NP, S1::BW, S1::BH) &&
                      enc4(&m.gm, g.gm[b], 14, MX3, MY3) &&
                      enc4(&m.up, g.u_prev[b], 3, MX3, MY3) &&
                      // the wrapped halo column and row
                      enc4(&m.hmx, g.hm[b], 14 * NP, S1::HX, S1::BH) &&
                      enc4(&m.h0x, g.h0[b], NP, S1::HX, S1::BH) &&
                      enc4(&m.ppx, g.phi_prev[b], NP, S1::HX, S1::BH) &&
                      enc4(&m.hmy, g.hm[b], 14 * NP, S1::BW, 1) &&
                      enc4(&m.h0y, g.h0[b], NP, S1::BW, 1) &&
                      enc4(&m.ppy, g.phi_prev[b], NP, S1::BW, 1);
      if (!ok) return false;
    }
    return true;
  }
}

template <int P>
cudaError_t launch_tile3_p(const Consts &c, const Grid &g, int cur, int mode,
                           const Outputs &o, bool nonunif, bool wall,
                           cudaStream_t s) {
  switch (c.NP) {
    case 1: return launch_tile3_np<P, 1>(c, g, cur, mode, o, nonunif, wall, s);
    case 2: return launch_tile3_np<P, 2>(c, g, cur, mode, o, nonunif, wall, s);
    case 3: return launch_tile3_np<P, 3>(c, g, cur, mode, o, nonunif, wall, s);
    case 4: return launch_tile3_np<P, 4>(c, g, cur, mode, o, nonunif, wall, s);
  }
  return cudaErrorInvalidValue;
}

template <int P, int NP>
cudaError_t launch_init3_np(const Consts &c, const Grid &g, int cur,
                            const double *cin, const double *uin, double p0,
                            bool wall, cudaStream_t s) {
  KArgs3<P> A;
  A.a = make_args<P>(c, g, cur ^ 1, MODE_STEP, Outputs{});
  A.nz = g.nz;
  const int threads = 256;
  size_t blocks = (g.V + threads - 1) / threads;
  if (blocks > 65535u * 16u) blocks = 65535u * 16u;
  init3_phi_kernel<P, NP><<<(unsigned)blocks, threads, 0, s>>>(
      A.a, cin, uin, g.scratch, c.rho_t[0], c.rho_t[1], c.rho_t[2], c.rho_t[3], c.rho_t[4]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const KArgs<LBM_FP64> d = make_args<LBM_FP64>(c, g, cur ^ 1, MODE_STEP, Outputs{});
  if (wall)
    init3_pop_kernel<P, NP, true><<<(unsigned)blocks, threads, 0, s>>>(A, d, g.scratch, uin, p0);
  else
    init3_pop_kernel<P, NP, false><<<(unsigned)blocks, threads, 0, s>>>(A, d, g.scratch, uin, p0);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_init3_p(const Consts &c, const Grid &g, int cur,
                           const double *cin, const double *uin, double p0,
                           bool wall, cudaStream_t s) {
  switch (c.NP) {
    case 1: return launch_init3_np<P, 1>(c, g, cur, cin, uin, p0, wall, s);
    case 2: return launch_init3_np<P, 2>(c, g, cur, cin, uin, p0, wall, s);
    case 3: return launch_init3_np<P, 3>(c, g, cur, cin, uin, p0, wall, s);
    case 4: return launch_init3_np<P, 4>(c, g, cur, cin, uin, p0, wall, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
