// Batched ensemble: many independent grids (uneven sizes, N = 2..5, walls
// or periodic) advanced by one persistent launch per time step, replayed from
// a captured CUDA graph, with the tile height and the CTA-to-tile schedule
// chosen by measurement (lbm_nphase_batch_autotune).
//
// Each case is an ordinary single-grid handle carved from the batch
// workspace, so init, moments and diagnostics of a case are the single-grid
// entry points. The batch kernel walks a list of (case, tile) items; for each
// item it loads the case's kernel arguments into shared memory and runs the
// same per-node arithmetic as the single-grid kernels (node_macros,
// collide_stream), for FP32 storage and equal pure-phase densities.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "lbm_kernels.cuh"
#include "lbm_nphase.h"

namespace lbm {

// Per-case descriptor: kernel arguments for input buffer 0 and 1.
template <int P> struct BatchCase {
  KArgs<P> a[2];
  int np, wall, ntx, nty;
};

// One time step of one BX x TBY tile of one case (equal densities).
template <int P, int NP, bool WALL, int TBY>
__device__ __forceinline__ void tile_step_body(const KArgs<P> &a, int x0, int y0,
                                               typename Prec<P>::T *sphi) {
  typedef typename Prec<P>::T T;
  constexpr int SW = BX + 2, SH = TBY + 2, PL = SW * SH;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int nx = a.nx, ny = a.ny;
  const size_t V = a.V;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = gx < nx && gy < ny;
  T hreg[NP][9], perr[NP];
  {
    const int sx = wrap(gx, nx), sy = wrap_y<WALL>(gy, ny);
    const size_t q = (size_t)sy * nx + sx;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      hreg[i][0] = ldg(a.h0_in + (size_t)i * V + q);
#pragma unroll
      for (int k = 1; k < 9; ++k) hreg[i][k] = load_hm<P>(a, i, k, q);
      const T pp = ldg(a.pp_in + (size_t)i * V + q);
      sphi[i * PL + (ty + 1) * SW + tx + 1] =
          node_phi<P>(hreg[i][0], &hreg[i][1], pp, perr[i], a.sh_ld);
    }
  }
  constexpr int NRING = SW * SH - BX * TBY;
  for (int r = tid; r < NRING; r += BX * TBY) {
    int lx, ly;
    ring_pos_1<TBY>(r, lx, ly);
    phi_global<P, NP, WALL>(a, wrap(x0 - 1 + lx, nx), wrap_y<WALL>(y0 - 1 + ly, ny),
                      sphi, PL, ly * SW + lx);
  }
  __syncthreads();
  if (active) {
    const size_t q = (size_t)gy * nx + gx;
    T g[9], pp[NP];
#pragma unroll
    for (int k = 1; k < 9; ++k) g[k] = load_gm<P>(a, k, q);
#pragma unroll
    for (int i = 0; i < NP; ++i) pp[i] = ldg(a.pp_in + (size_t)i * V + q);
    NodeMac<P, NP> m;
    node_macros<P, NP, false, SW, 1>(a, sphi, PL, nullptr, 0, ty + 1, tx + 1, 0,
                                     0, g, m);
    collide_stream<P, NP, false, WALL>(a, m, hreg, perr, g, pp, a.u_in[q],
                                       a.u_in[V + q], gx, gy);
  }
  __syncthreads();  // sphi is reused by the next item
}

enum BatchSched { SCHED_STRIDE = 0, SCHED_LISTS = 1, SCHED_DYNAMIC = 2 };

template <int P, int TBY>
__global__ void __launch_bounds__(BX *TBY)
    batch_kernel(const BatchCase<P> *__restrict__ cases,
                 const int2 *__restrict__ items, int nitems,
                 const int *__restrict__ list_off, const int *__restrict__ list,
                 int sched, int chunk, int *counter, int cur) {
  typedef typename Prec<P>::T T;
  constexpr int SW = BX + 2, SH = TBY + 2;
  __shared__ KArgs<P> sa;
  __shared__ T sphi[4 * SW * SH];
  __shared__ int s_item, s_np, s_wall, s_ntx;
  const int tid = threadIdx.y * BX + threadIdx.x;
  int loaded = -1;
  int k = 0, cbase = 0, cleft = 0;  // dynamic: current chunk (thread 0)
  const int lbeg = sched == SCHED_LISTS ? list_off[blockIdx.x] : 0;
  const int lend = sched == SCHED_LISTS ? list_off[blockIdx.x + 1] : 0;
  for (;;) {
    int item;
    if (sched == SCHED_DYNAMIC) {
      if (tid == 0) {
        if (cleft == 0) {
          cbase = atomicAdd(counter, 1) * chunk;
          cleft = chunk;
        }
        s_item = cbase + chunk - cleft--;
      }
      __syncthreads();
      item = s_item;
      __syncthreads();
    } else if (sched == SCHED_LISTS) {
      item = lbeg + k < lend ? list[lbeg + k] : nitems;
    } else {
      item = blockIdx.x + k * gridDim.x;
    }
    ++k;
    if (item >= nitems) break;
    const int2 it = items[item];
    if (it.x != loaded) {
      // Case arguments into shared memory (word copy of a plain struct).
      const unsigned *src = (const unsigned *)&cases[it.x].a[cur];
      unsigned *dst = (unsigned *)&sa;
      for (int w = tid; w < (int)(sizeof(KArgs<P>) / 4); w += BX * TBY) dst[w] = src[w];
      if (tid == 0) {
        s_np = cases[it.x].np;
        s_wall = cases[it.x].wall;
        s_ntx = cases[it.x].ntx;
      }
      __syncthreads();
      loaded = it.x;
    }
    const int x0 = (it.y % s_ntx) * BX, y0 = (it.y / s_ntx) * TBY;
    switch (s_np * 2 + s_wall) {
      case 2: tile_step_body<P, 1, false, TBY>(sa, x0, y0, sphi); break;
      case 3: tile_step_body<P, 1, true, TBY>(sa, x0, y0, sphi); break;
      case 4: tile_step_body<P, 2, false, TBY>(sa, x0, y0, sphi); break;
      case 5: tile_step_body<P, 2, true, TBY>(sa, x0, y0, sphi); break;
      case 6: tile_step_body<P, 3, false, TBY>(sa, x0, y0, sphi); break;
      case 7: tile_step_body<P, 3, true, TBY>(sa, x0, y0, sphi); break;
      case 8: tile_step_body<P, 4, false, TBY>(sa, x0, y0, sphi); break;
      case 9: tile_step_body<P, 4, true, TBY>(sa, x0, y0, sphi); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Pipelined batch kernel (FP32 storage, 32 x 8 tiles): the tile body of
// tile_kernel_tma applied to (case, tile) items, with the boxes of the CTA's
// next item in flight while the current one is computed. Each stage holds one
// item's populations and a copy of its case's kernel arguments, all counted
// on the stage's mbarrier, so a change of case costs no extra barrier.
// Thread 0 issues the copies; it keeps the next item's descriptor (case,
// tile origin, N - 1 and walls: precomputed on the host) and the index of
// the one after it in flight one tile ahead, so that no global load or
// atomic sits between a finished tile and the next issue. Tensor maps live
// in global memory (written by the host before the launch) and are acquired
// through the tensormap proxy when the issuing thread meets a new case. A
// ring of S slots in shared memory tells the other threads what each stage
// holds (case -1: the CTA's items are done). Stages are sized for N - 1 = 4
// and laid out per item for its own N - 1.
// ---------------------------------------------------------------------------
typedef TmaGeom<LBM_FP32> BG;
typedef TmaStage<LBM_FP32, 4> BSt;
constexpr size_t kArgsBytes = sizeof(KArgs<LBM_FP32>);
static_assert(kArgsBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
constexpr size_t kStageStride = BSt::BYTES + ((kArgsBytes + 127) & ~(size_t)127);
constexpr size_t kBatchSmem = BSt::S * kStageStride + 2 * BSt::SPHI + 64;
static_assert(kBatchSmem <= 232448, "shared memory per CTA");

// Item descriptor of the pipelined kernel: case, tile origin, class 2 (N - 1)
// + walls; for a tile on the edge of a periodic case, which wrapped halo
// column (wx: 1 the column x = -1, staged from x = nx - 4 .. nx - 1; 2 the
// column x = nx, from 0 .. 3) and row (wy: 1 the row y = -1, from ny - 1; 2
// the row y = ny, from 0) are staged with it, and their first source column
// and row (xs, ys).
struct alignas(16) TmaItem {
  int c, x0, y0, cls, wx, wy, xs, ys;
};

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(m)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src,
                                          uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <int NP>
__device__ __forceinline__ void batch_issue_np(unsigned char *st, uint64_t *b,
                                               const TmaMaps *m,
                                               const KArgs<LBM_FP32> *args,
                                               const TmaItem &d) {
  typedef TmaStage<LBM_FP32, NP> St;
  const int x0 = d.x0, y0 = d.y0;
  mbar_expect_tx(b, St::TX + (uint32_t)kArgsBytes + (d.wx ? St::XTX : 0u) +
                        (d.wy ? St::YTX : 0u));
  tma_load_3d(st, &m->hm, x0 - BG::HXM, y0 - 1, 0, b);
  tma_load_3d(st + St::HM, &m->h0, x0 - BG::HXR, y0 - 1, 0, b);
  tma_load_3d(st + St::HM + St::H0, &m->pp, x0 - BG::HXR, y0 - 1, 0, b);
  tma_load_3d(st + St::HM + St::H0 + St::PP, &m->gm, x0, y0, 0, b);
  tma_load_3d(st + St::HM + St::H0 + St::PP + St::GM, &m->up, x0, y0, 0, b);
  // the wrapped halo column and row of an edge tile
  unsigned char *w = st + St::BASE;
  if (d.wx) {
    tma_load_3d(w, &m->hmx, d.xs, y0 - 1, 0, b);
    tma_load_3d(w + St::XHM, &m->h0x, d.xs, y0 - 1, 0, b);
    tma_load_3d(w + St::XHM + St::XH0, &m->ppx, d.xs, y0 - 1, 0, b);
  }
  if (d.wy) {
    w += St::XHM + St::XH0 + St::XPP;
    tma_load_3d(w, &m->hmy, x0 - BG::HXM, d.ys, 0, b);
    tma_load_3d(w + St::YHM, &m->h0y, x0 - BG::HXR, d.ys, 0, b);
    tma_load_3d(w + St::YHM + St::YH0, &m->ppy, x0 - BG::HXR, d.ys, 0, b);
  }
  bulk_load(st + BSt::BYTES, args, (uint32_t)kArgsBytes, b);
}

// One staged tile in two phases around one CTA barrier: (1) the own node's
// populations into registers and phi on the tile and its ring, (2)
// collisions and streaming. The register arrays are sized for N - 1 = 4 and
// shared by every (N - 1, walls) variant, so that the variants do not add up
// their live registers across the barrier.
struct TileRegs {
  float hreg[4][9], perr[4], pp[4], g[9], up[2];
};

template <int NP, bool WALL>
__device__ __forceinline__ void batch_tma_phi(const KArgs<LBM_FP32> &a,
                                              const unsigned char *st,
                                              float *sphi, int x0, int y0,
                                              int wx, int wy, TileRegs &r) {
  typedef float T;
  typedef typename Prec<LBM_FP32>::Sm Sm;
  typedef TmaStage<LBM_FP32, NP> St;
  constexpr int TBY = BG::TBY;
  constexpr int SW = BX + 2, SH = TBY + 2, PL = SW * SH;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int nx = a.nx, ny = a.ny;
  const Sm *shm = (const Sm *)st;
  const T *sh0 = (const T *)(st + St::HM);
  const T *spp = (const T *)(st + St::HM + St::H0);
  const Sm *sgm = (const Sm *)(st + St::HM + St::H0 + St::PP);
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < nx && gy < ny) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      r.hreg[i][0] = sh0[(i * BG::HB + ty + 1) * BG::WR + tx + BG::HXR];
#pragma unroll
      for (int k = 1; k < 9; ++k)
        r.hreg[i][k] = to_T(shm[((i * 8 + k - 1) * BG::HB + ty + 1) * BG::WM + tx + BG::HXM]);
      r.pp[i] = spp[(i * BG::HB + ty + 1) * BG::WR + tx + BG::HXR];
      sphi[i * PL + (ty + 1) * SW + tx + 1] = node_phi<LBM_FP32>(
          r.hreg[i][0], &r.hreg[i][1], r.pp[i], r.perr[i], a.sh_ld);
    }
#pragma unroll
    for (int k = 1; k < 9; ++k) r.g[k] = to_T(sgm[((k - 1) * TBY + ty) * BX + tx]);
    // u(t-1): the stage is not read after the tile's barrier
    const T *sup = (const T *)(st + St::HM + St::H0 + St::PP + St::GM);
    r.up[0] = sup[ty * BX + tx];
    r.up[1] = sup[(TBY + ty) * BX + tx];
  } else {
    phi_global<LBM_FP32, NP, WALL>(a, wrap(gx, nx), wrap_y<WALL>(gy, ny), sphi, PL,
                             (ty + 1) * SW + tx + 1);
  }
  // The ring's positions go to warps 1..3 (threads 32 .. 32 + NRING - 1):
  // warp 0 holds the thread that fetches the next item and issues its
  // copies, which then overlaps the ring sums instead of adding to them.
  constexpr int NRING = SW * SH - BX * TBY;
  static_assert(32 + NRING <= BX * TBY, "one ring position per thread");
  if (tid >= 32 && tid < 32 + NRING) {
    int lx, ly;
    ring_pos_1<TBY>(tid - 32, lx, ly);
    const int rx = x0 - 1 + lx, ry = y0 - 1 + ly;
    const bool inx = rx >= 0 && rx < nx, iny = ry >= 0 && ry < ny;
    // phi of one ring position from staged populations: hmb, h0b, ppb are
    // the moving, rest and phi(t-1) planes with plane strides pm, pr; om,
    // orr the position's offset in them
    auto staged_phi = [&](const Sm *hmb, const T *h0b, const T *ppb, int pm, int pr,
                          int om, int orr) {
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T mov[8], e;
#pragma unroll
        for (int k = 1; k < 9; ++k) mov[k - 1] = to_T(hmb[(i * 8 + k - 1) * pm + om]);
        sphi[i * PL + ly * SW + lx] =
            node_phi<LBM_FP32>(h0b[i * pr + orr], mov, ppb[i * pr + orr], e, a.sh_ld);
      }
    };
    const unsigned char *w = st + St::BASE;
    if (inx && (iny || WALL)) {
      // in the box; a wall's ghost row is the adjacent row of the box
      const int by = WALL ? wrap_y<WALL>(ry, ny) - y0 + 1 : ly;
      staged_phi(shm, sh0, spp, BG::HB * BG::WM, BG::HB * BG::WR,
                 by * BG::WM + lx - 1 + BG::HXM, by * BG::WR + lx - 1 + BG::HXR);
    } else if (iny && ((rx < 0 && wx == 1) || (rx >= nx && wx == 2))) {
      // the staged wrapped column
      const int c = rx < 0 ? BG::HXR - 1 : 0;
      staged_phi((const Sm *)w, (const T *)(w + St::XHM), (const T *)(w + St::XHM + St::XH0),
                 BG::HB * BG::HXM, BG::HB * BG::HXR, ly * BG::HXM + c, ly * BG::HXR + c);
    } else if (inx && ((ry < 0 && wy == 1) || (ry >= ny && wy == 2))) {
      // the staged wrapped row
      w += St::XHM + St::XH0 + St::XPP;
      staged_phi((const Sm *)w, (const T *)(w + St::YHM), (const T *)(w + St::YHM + St::YH0),
                 BG::WM, BG::WR, lx - 1 + BG::HXM, lx - 1 + BG::HXR);
    } else {
      // corners and ragged tails
      phi_global<LBM_FP32, NP, WALL>(a, wrap(rx, nx), wrap_y<WALL>(ry, ny), sphi, PL,
                               ly * SW + lx);
    }
  }
}

template <int NP, bool WALL>
__device__ __forceinline__ void batch_tma_collide(const KArgs<LBM_FP32> &a,
                                                  const float *sphi, int x0,
                                                  int y0, TileRegs &r) {
  constexpr int TBY = BG::TBY;
  constexpr int SW = BX + 2, PL = SW * (TBY + 2);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= a.nx || gy >= a.ny) return;
  float hreg[NP][9], perr[NP], pp[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    perr[i] = r.perr[i];
    pp[i] = r.pp[i];
#pragma unroll
    for (int k = 0; k < 9; ++k) hreg[i][k] = r.hreg[i][k];
  }
  NodeMac<LBM_FP32, NP> m;
  node_macros<LBM_FP32, NP, false, SW, 1>(a, sphi, PL, nullptr, 0, ty + 1,
                                          tx + 1, 0, 0, r.g, m);
  collide_stream<LBM_FP32, NP, false, WALL>(a, m, hreg, perr, r.g, pp, r.up[0],
                                            r.up[1], gx, gy);
}

__global__ void __launch_bounds__(BG::NTH, 1)
    batch_kernel_tma(const BatchCase<LBM_FP32> *__restrict__ cases,
                     const TmaMaps *__restrict__ maps, int ncases,
                     const TmaItem *__restrict__ items, int nitems,
                     const int *__restrict__ list_off,
                     const int *__restrict__ list, int sched, int chunk,
                     int *counter, int cur) {
  constexpr int S = BSt::S;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = (uint64_t *)(smem + S * kStageStride + 2 * BSt::SPHI);
  __shared__ TmaItem s_slot[S];
  const int tid = threadIdx.y * BX + threadIdx.x;

  // Schedule state (thread 0 only): the CTA's k-th item index, the
  // descriptor of the next item to issue and the index of the one after.
  int k = 0, issued = 0, fenced = -1, cbase = 0, cleft = 0;
  const int lbeg = sched == SCHED_LISTS ? list_off[blockIdx.x] : 0;
  const int lend = sched == SCHED_LISTS ? list_off[blockIdx.x + 1] : 0;
  auto next_index = [&]() -> int {
    int item;
    if (sched == SCHED_DYNAMIC) {
      if (cleft == 0) {
        cbase = atomicAdd(counter, 1) * chunk;
        cleft = chunk;
      }
      item = cbase + chunk - cleft--;
    }
    else if (sched == SCHED_LISTS) item = lbeg + k < lend ? list[lbeg + k] : nitems;
    else item = blockIdx.x + k * gridDim.x;
    ++k;
    return item;
  };
  const TmaItem none = {-1, 0, 0, 0, 0, 0, 0, 0};
  TmaItem d_next = none;
  int i_after = nitems;
  auto issue = [&](int j) {  // thread 0: the CTA's j-th item into stage j % S
    const int slot = j % S;
    const TmaItem d = d_next;
    if (d.c >= 0) {
      d_next = i_after < nitems ? items[i_after] : none;
      i_after = i_after < nitems ? next_index() : nitems;
    }
    s_slot[slot] = d;
    if (d.c < 0) return;
    const TmaMaps *m = maps + 2 * d.c + cur;
    if (d.c != fenced) {
      tensormap_acquire(&m->hm);
      tensormap_acquire(&m->h0);
      tensormap_acquire(&m->pp);
      tensormap_acquire(&m->gm);
      tensormap_acquire(&m->up);
      tensormap_acquire(&m->hmx);
      tensormap_acquire(&m->h0x);
      tensormap_acquire(&m->ppx);
      tensormap_acquire(&m->hmy);
      tensormap_acquire(&m->h0y);
      tensormap_acquire(&m->ppy);
      fenced = d.c;
    }
    unsigned char *st = smem + slot * kStageStride;
    const KArgs<LBM_FP32> *args = &cases[d.c].a[cur];
    switch (d.cls >> 1) {
      case 1: batch_issue_np<1>(st, bar + slot, m, args, d); break;
      case 2: batch_issue_np<2>(st, bar + slot, m, args, d); break;
      case 3: batch_issue_np<3>(st, bar + slot, m, args, d); break;
      default: batch_issue_np<4>(st, bar + slot, m, args, d); break;
    }
    ++issued;
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const int i0 = next_index();
    if (i0 < nitems) {
      d_next = items[i0];
      i_after = next_index();
    }
    for (int j = 0; j < S; ++j) issue(j);
  }
  __syncthreads();

  int failed_at = -1;
  for (int j = 0;; ++j) {
    const int slot = j % S;
    const TmaItem d = s_slot[slot];
    if (d.c < 0) break;
    const bool ok = mbar_wait(bar + slot, (uint32_t)((j / S) & 1));
    const unsigned char *st = smem + slot * kStageStride;
    // The case's arguments by value: read from the stage once per tile
    // (vector loads) and held in registers, not re-read at every use.
    const KArgs<LBM_FP32> sa = *(const KArgs<LBM_FP32> *)(st + BSt::BYTES);
    float *sphi = (float *)(smem + S * kStageStride + (j & 1) * BSt::SPHI);
    const int x0 = d.x0, y0 = d.y0;
    TileRegs r;
    switch (d.cls) {
      case 2: batch_tma_phi<1, false>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 3: batch_tma_phi<1, true>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 4: batch_tma_phi<2, false>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 5: batch_tma_phi<2, true>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 6: batch_tma_phi<3, false>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 7: batch_tma_phi<3, true>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 8: batch_tma_phi<4, false>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
      case 9: batch_tma_phi<4, true>(sa, st, sphi, x0, y0, d.wx, d.wy, r); break;
    }
    // A thread whose wait gave up ran the phi sums on stale shared data
    // (harmlessly); this barrier makes the decision to stop CTA-wide. Past
    // it no thread reads the stage (u(t-1) is in registers), so it is
    // refilled at once; the phi tile is double-buffered, so this is the
    // tile's only barrier (a thread at the next tile's barrier is done with
    // this tile's phi tile).
    if (__syncthreads_or(!ok)) {
      failed_at = j;
      break;
    }
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + S);
    }
    switch (d.cls) {
      case 2: batch_tma_collide<1, false>(sa, sphi, x0, y0, r); break;
      case 3: batch_tma_collide<1, true>(sa, sphi, x0, y0, r); break;
      case 4: batch_tma_collide<2, false>(sa, sphi, x0, y0, r); break;
      case 5: batch_tma_collide<2, true>(sa, sphi, x0, y0, r); break;
      case 6: batch_tma_collide<3, false>(sa, sphi, x0, y0, r); break;
      case 7: batch_tma_collide<3, true>(sa, sphi, x0, y0, r); break;
      case 8: batch_tma_collide<4, false>(sa, sphi, x0, y0, r); break;
      case 9: batch_tma_collide<4, true>(sa, sphi, x0, y0, r); break;
    }
  }
  if (failed_at >= 0) {
    // Every case's state is now suspect: flag all of them, then let the
    // copies still in flight (items failed_at .. issued-1) land, with the
    // same bounded wait, before the CTA's shared memory is released.
    if (tid == 0) {
      for (int c = 0; c < ncases; ++c) atomicExch(cases[c].a[0].err, 1);
      for (int j = failed_at; j < issued; ++j)
        mbar_wait(bar + (j % S), (uint32_t)((j / S) & 1));
    }
    __syncthreads();
  }
}

}  // namespace lbm

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
using lbm::BatchCase;
typedef BatchCase<LBM_FP32> Case32;

namespace {
constexpr int kTileHeights[2] = {4, 8};
constexpr int kMaxCtas = 4096;  // bound of the per-CTA schedule lists
size_t align256b(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

struct lbm_nphase_batch_t {
  int n;
  std::vector<lbm_nphase_t *> cases;
  cudaStream_t stream;     // caller's stream
  cudaStream_t cap;        // private stream for graph capture
  Case32 *d_cases;         // descriptors (device)
  lbm::TmaMaps *d_maps;    // tensor maps [case][input buffer] (device)
  bool tma_ok;             // every case has tensor maps (pipelined kernel)
  int2 *d_items;           // (case, tile) items (device)
  lbm::TmaItem *d_titems;  // the same items for the pipelined kernel
  int *d_list_off, *d_list, *d_counter;
  size_t items_cap, lists_cap;
  int nitems;
  lbm_nphase_batch_schedule sched;
  int max_ctas[2];         // resident CTAs per tile height (generic kernel)
  int max_ctas_tma;        // resident CTAs of the pipelined kernel
  cudaGraphExec_t exec[2]; // two steps starting at buffer 0 / 1
  int cur;
  int64_t steps;
  int cuda_err;
};

namespace {

lbm_status bfail(lbm_nphase_batch_t *b, cudaError_t e) {
  b->cuda_err = (int)e;
  return LBM_ECUDA;
}

size_t case_bytes(const lbm_nphase_params &p) {
  return align256b(lbm_nphase_workspace_bytes(&p));
}

size_t tiles_for(const lbm_nphase_params &p, int tby) {
  return (size_t)lbm::tiles_x(p.nx) * ((p.ny + tby - 1) / tby);
}

void destroy_graphs(lbm_nphase_batch_t *b) {
  for (int p = 0; p < 2; ++p)
    if (b->exec[p]) {
      cudaGraphExecDestroy(b->exec[p]);
      b->exec[p] = nullptr;
    }
}

cudaError_t launch_once(lbm_nphase_batch_t *b, cudaStream_t s, int cur) {
  const int ti = b->sched.tile_height == 4 ? 0 : 1;
  int grid = b->sched.ctas;
  if (b->sched.schedule == lbm::SCHED_DYNAMIC) {
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  if (b->sched.pipelined)
    lbm::batch_kernel_tma<<<grid, dim3(lbm::BX, lbm::BG::TBY), lbm::kBatchSmem, s>>>(
        b->d_cases, b->d_maps, b->n, b->d_titems, b->nitems, b->d_list_off,
        b->d_list, b->sched.schedule, b->sched.chunk, b->d_counter, cur);
  else if (ti == 0)
    lbm::batch_kernel<LBM_FP32, 4><<<grid, dim3(lbm::BX, 4), 0, s>>>(
        b->d_cases, b->d_items, b->nitems, b->d_list_off, b->d_list,
        b->sched.schedule, b->sched.chunk, b->d_counter, cur);
  else
    lbm::batch_kernel<LBM_FP32, 8><<<grid, dim3(lbm::BX, 8), 0, s>>>(
        b->d_cases, b->d_items, b->nitems, b->d_list_off, b->d_list,
        b->sched.schedule, b->sched.chunk, b->d_counter, cur);
  return cudaGetLastError();
}

// Work items and schedules for one tile height and CTA count.
lbm_status build_schedule(lbm_nphase_batch_t *b, lbm_nphase_batch_schedule s) {
  if (s.pipelined != 0 && s.pipelined != 1) return LBM_EINVAL;
  if (s.pipelined && !b->tma_ok) return LBM_EINVAL;
  if (s.pipelined) s.tile_height = lbm::BG::TBY;
  const int tby = s.tile_height;
  const int ti = tby == 4 ? 0 : 1;
  if (tby != 4 && tby != 8) return LBM_EINVAL;
  if (s.schedule < 0 || s.schedule > 2) return LBM_EINVAL;
  const int cap = s.pipelined ? b->max_ctas_tma : b->max_ctas[ti];
  if (s.chunk < 0) return LBM_EINVAL;
  if (s.chunk == 0) s.chunk = 1;
  if (s.ctas <= 0 || s.ctas > cap) s.ctas = cap;
  // Cases in order of decreasing work (cost of a tile ~ N), tiles of a case
  // consecutive (neighbouring tiles share halos in L2).
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int c) {
    const lbm_nphase_params &p = b->cases[c]->prm;
    return (double)tiles_for(p, tby) * p.N;
  };
  // Cases of one (N - 1, walls) class are kept together, so that the CTAs
  // running at one time mostly execute the same code.
  auto klass = [&](int c) {
    return b->cases[c]->k.NP * 2 + (b->cases[c]->wall ? 1 : 0);
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (klass(x) != klass(y)) return klass(x) > klass(y);
    return cost(x) > cost(y);
  });
  std::vector<int2> items;
  std::vector<double> icost;
  for (int c : order) {
    const size_t nt = tiles_for(b->cases[c]->prm, tby);
    for (size_t t = 0; t < nt; ++t) {
      items.push_back(make_int2(c, (int)t));
      icost.push_back(b->cases[c]->prm.N);
    }
  }
  if (items.size() > b->items_cap) return LBM_ENOMEM;
  // Per-CTA lists: the cost-ordered item sequence cut into contiguous runs of
  // equal total cost (tile cost ~ N), so that a CTA keeps one case's
  // arguments loaded and neighbouring tiles run on the same CTA.
  std::vector<int> off(s.ctas + 1, 0), list;
  {
    std::vector<std::vector<int>> bins(s.ctas);
    const double total = std::accumulate(icost.begin(), icost.end(), 0.0);
    const double share = total / s.ctas;
    int bin = 0;
    double acc = 0.0;
    for (size_t i = 0; i < items.size(); ++i) {
      if (acc >= share * (bin + 1) && bin + 1 < s.ctas) ++bin;
      bins[bin].push_back((int)i);
      acc += icost[i];
    }
    for (int k = 0; k < s.ctas; ++k) {
      off[k + 1] = off[k] + (int)bins[k].size();
      list.insert(list.end(), bins[k].begin(), bins[k].end());
    }
  }
  cudaError_t e;
  e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2),
                      cudaMemcpyHostToDevice, b->stream);
  std::vector<lbm::TmaItem> titems;
  if (s.pipelined) {
    titems.resize(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
      const lbm_nphase_t *h = b->cases[items[i].x];
      const int ntx = lbm::tiles_x(h->prm.nx), t = items[i].y;
      const int x0 = (t % ntx) * lbm::BX, y0 = (t / ntx) * tby;
      const int nx = h->prm.nx, ny = h->prm.ny;
      // wrapped halo column / row staged with an edge tile (periodic axes)
      const int wx = x0 == 0 ? 1 : (x0 + lbm::BX == nx ? 2 : 0);
      const int wy = h->wall ? 0 : (y0 == 0 ? 1 : (y0 + tby == ny ? 2 : 0));
      titems[i] = {items[i].x, x0, y0, h->k.NP * 2 + (h->wall ? 1 : 0), wx, wy,
                   wx == 1 ? nx - lbm::TmaGeom<LBM_FP32>::HXR : 0, wy == 1 ? ny - 1 : 0};
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_titems, titems.data(),
                          titems.size() * sizeof(lbm::TmaItem),
                          cudaMemcpyHostToDevice, b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_list_off, off.data(), off.size() * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_list, list.data(), list.size() * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  // descriptors: ntx/nty for this tile height
  std::vector<Case32> desc(b->n);
  for (int c = 0; c < b->n; ++c) {
    lbm_nphase_t *h = b->cases[c];
    const lbm::Outputs none = {nullptr, nullptr, nullptr, nullptr, nullptr};
    desc[c].a[0] = lbm::make_args<LBM_FP32>(h->k, h->g, 0, lbm::MODE_STEP, none);
    desc[c].a[1] = lbm::make_args<LBM_FP32>(h->k, h->g, 1, lbm::MODE_STEP, none);
    desc[c].np = h->k.NP;
    desc[c].wall = h->wall ? 1 : 0;
    desc[c].ntx = lbm::tiles_x(h->prm.nx);
    desc[c].nty = (h->prm.ny + tby - 1) / tby;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_cases, desc.data(), desc.size() * sizeof(Case32),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  b->nitems = (int)items.size();
  b->sched = s;
  // Two steps (buffer 0 -> 1 -> 0 and 1 -> 0 -> 1) captured as graphs.
  destroy_graphs(b);
  for (int p = 0; p < 2; ++p) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, e);
    cudaError_t e1 = launch_once(b, b->cap, p);
    cudaError_t e2 = launch_once(b, b->cap, p ^ 1);
    e = cudaStreamEndCapture(b->cap, &graph);
    if (e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[p], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, e);
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_nphase_batch_workspace_bytes(const lbm_nphase_params *params,
                                        int ncases) {
  if (!params || ncases <= 0) return 0;
  size_t total = 0, items = 0;
  for (int c = 0; c < ncases; ++c) {
    const lbm_nphase_params &p = params[c];
    if (p.precision != LBM_FP32) return 0;
    lbm_nphase_model m;
    if (lbm_nphase_derive(&p, &m) != LBM_OK || !m.uniform_density ||
        p.grad_scheme != 0 || p.lattice != 0)
      return 0;
    total += case_bytes(p);
    items += tiles_for(p, 4);
  }
  total += align256b(ncases * sizeof(Case32));
  total += align256b((size_t)ncases * 2 * sizeof(lbm::TmaMaps));
  total += align256b(items * sizeof(int2));
  total += align256b(items * sizeof(lbm::TmaItem));
  total += align256b((size_t)(kMaxCtas + 1) * sizeof(int));
  total += align256b(items * sizeof(int));
  total += align256b(sizeof(int));
  return total;
}

lbm_status lbm_nphase_batch_create(const lbm_nphase_params *params, int ncases,
                                   void *ws, size_t bytes, void *stream,
                                   lbm_nphase_batch_t **out) {
  if (!out || !params || ncases <= 0 || !ws || ((uintptr_t)ws & 255u))
    return LBM_EINVAL;
  *out = nullptr;
  const size_t need = lbm_nphase_batch_workspace_bytes(params, ncases);
  if (need == 0) return LBM_EINVAL;
  if (bytes < need) return LBM_ENOMEM;
  lbm_nphase_batch_t *b = new (std::nothrow) lbm_nphase_batch_t();
  if (!b) return LBM_ENOMEM;
  b->n = ncases;
  b->stream = (cudaStream_t)stream;
  char *base = (char *)ws;
  size_t off = 0, items = 0;
  lbm_status st = LBM_OK;
  for (int c = 0; c < ncases && st == LBM_OK; ++c) {
    lbm_nphase_t *h = nullptr;
    const size_t cb = case_bytes(params[c]);
    st = lbm_nphase_create(&params[c], base + off, cb, stream, &h);
    if (st == LBM_OK) b->cases.push_back(h);
    off += cb;
    items += tiles_for(params[c], 4);
  }
  if (st != LBM_OK) {
    lbm_nphase_batch_destroy(b);
    return st;
  }
  b->d_cases = (Case32 *)(base + off);
  off += align256b(ncases * sizeof(Case32));
  b->d_maps = (lbm::TmaMaps *)(base + off);
  off += align256b((size_t)ncases * 2 * sizeof(lbm::TmaMaps));
  b->d_items = (int2 *)(base + off);
  b->items_cap = items;
  off += align256b(items * sizeof(int2));
  b->d_titems = (lbm::TmaItem *)(base + off);
  off += align256b(items * sizeof(lbm::TmaItem));
  b->d_list_off = (int *)(base + off);
  off += align256b((size_t)(kMaxCtas + 1) * sizeof(int));
  b->d_list = (int *)(base + off);
  off += align256b(items * sizeof(int));
  b->d_counter = (int *)(base + off);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    lbm_nphase_batch_destroy(b);
    return LBM_ECUDA;
  }
  int dev = 0, sms = 0, per4 = 0, per8 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per4, lbm::batch_kernel<LBM_FP32, 4>, lbm::BX * 4, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per8, lbm::batch_kernel<LBM_FP32, 8>, lbm::BX * 8, 0);
  b->max_ctas[0] = std::min(std::max(per4, 1) * sms, kMaxCtas);
  b->max_ctas[1] = std::min(std::max(per8, 1) * sms, kMaxCtas);
  // Pipelined kernel: every case must have tensor maps (FP32 maps of both
  // buffers, copied next to the descriptors).
  b->tma_ok = true;
  for (lbm_nphase_t *h : b->cases) b->tma_ok = b->tma_ok && h->g.use_tma;
  b->max_ctas_tma = 0;
  if (b->tma_ok) {
    std::vector<lbm::TmaMaps> maps(2 * (size_t)ncases);
    for (int c = 0; c < ncases; ++c)
      for (int q = 0; q < 2; ++q) maps[2 * c + q] = b->cases[c]->g.tma[q];
    e = cudaMemcpyAsync(b->d_maps, maps.data(), maps.size() * sizeof(lbm::TmaMaps),
                        cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::batch_kernel_tma,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)lbm::kBatchSmem);
    int per = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per, lbm::batch_kernel_tma, lbm::BG::NTH, lbm::kBatchSmem);
    if (e != cudaSuccess) {
      b->cuda_err = (int)e;
      lbm_nphase_batch_destroy(b);
      return LBM_ECUDA;
    }
    b->max_ctas_tma = std::min(std::max(per, 1) * sms, kMaxCtas);
  }
  lbm_nphase_batch_schedule s0 = {8, lbm::SCHED_DYNAMIC, 0, 0, 1};
  st = build_schedule(b, s0);
  if (st != LBM_OK) {
    lbm_nphase_batch_destroy(b);
    return st;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_nphase_batch_init(lbm_nphase_batch_t *b, int c,
                                 const double *frac, const double *u,
                                 double p0) {
  if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
  return lbm::init_at(b->cases[c], frac, u, p0, b->cur);
}

lbm_status lbm_nphase_batch_step(lbm_nphase_batch_t *b, int64_t nsteps) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  for (lbm_nphase_t *h : b->cases)
    if (!h->initialized || h->unstable || h->cur != b->cur) return LBM_ESTATE;
  cudaError_t e = cudaSuccess;
  int64_t t = 0;
  for (; t + 2 <= nsteps && e == cudaSuccess; t += 2)
    e = cudaGraphLaunch(b->exec[b->cur], b->stream);
  if (e == cudaSuccess && t < nsteps) {
    e = launch_once(b, b->stream, b->cur);
    if (e == cudaSuccess) b->cur ^= 1;
  }
  if (e != cudaSuccess) return bfail(b, e);
  for (lbm_nphase_t *h : b->cases) {
    h->cur = b->cur;
    h->steps += nsteps;
  }
  b->steps += nsteps;
  return LBM_OK;
}

lbm_nphase_t *lbm_nphase_batch_case(lbm_nphase_batch_t *b, int c) {
  if (!b || c < 0 || c >= b->n) return nullptr;
  return b->cases[c];
}

lbm_status lbm_nphase_batch_moments(lbm_nphase_batch_t *b, int c, double *phi,
                                    double *cfrac, double *u, double *p,
                                    double *rho) {
  if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
  return lbm_nphase_moments(b->cases[c], phi, cfrac, u, p, rho);
}

lbm_status lbm_nphase_batch_diagnostics(lbm_nphase_batch_t *b, int c,
                                        double *mass, double *ke,
                                        double *umax) {
  if (!b || c < 0 || c >= b->n) return LBM_EINVAL;
  return lbm_nphase_diagnostics(b->cases[c], mass, ke, umax);
}

lbm_status lbm_nphase_batch_set_schedule(lbm_nphase_batch_t *b,
                                         const lbm_nphase_batch_schedule *s) {
  if (!b || !s) return LBM_EINVAL;
  return build_schedule(b, *s);
}

lbm_status lbm_nphase_batch_get_schedule(const lbm_nphase_batch_t *b,
                                         lbm_nphase_batch_schedule *s) {
  if (!b || !s) return LBM_EINVAL;
  *s = b->sched;
  return LBM_OK;
}

lbm_status lbm_nphase_batch_autotune(lbm_nphase_batch_t *b, int trial_steps,
                                     double *best_ms_per_step) {
  if (!b || trial_steps < 1) return LBM_EINVAL;
  for (lbm_nphase_t *h : b->cases)
    if (!h->initialized) return LBM_ESTATE;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return LBM_ECUDA;
  lbm_nphase_batch_schedule best = b->sched;
  float best_ms = 1e30f;
  lbm_status st = LBM_OK;
  // Candidates: the generic kernel at tile heights 4 and 8 and the
  // pipelined kernel (when every case has tensor maps), each with the
  // strided, list and dynamic schedules (chunks of 1, 4 and 16 items).
  std::vector<lbm_nphase_batch_schedule> cand;
  for (int v = 0; v < (b->tma_ok ? 3 : 2); ++v)
    for (int sc = 0; sc < 3; ++sc)
      for (int ch : {1, 4, 16}) {
        if (sc != lbm::SCHED_DYNAMIC && ch != 1) continue;
        cand.push_back({kTileHeights[v < 2 ? v : 1], sc, 0, v == 2 ? 1 : 0, ch});
      }
  for (size_t ci = 0; ci < cand.size() && st == LBM_OK; ++ci) {
    st = build_schedule(b, cand[ci]);
    if (st != LBM_OK) break;
    st = lbm_nphase_batch_step(b, 2);  // warm-up
    if (st != LBM_OK) break;
    cudaEventRecord(e0, b->stream);
    st = lbm_nphase_batch_step(b, 2 * trial_steps);
    cudaEventRecord(e1, b->stream);
    if (st != LBM_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = LBM_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)(2 * trial_steps);
    if (ms < best_ms) {
      best_ms = ms;
      best = b->sched;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  if (best_ms_per_step) *best_ms_per_step = best_ms;
  return build_schedule(b, best);
}

int lbm_nphase_batch_size(const lbm_nphase_batch_t *b) { return b ? b->n : 0; }

lbm_status lbm_nphase_batch_destroy(lbm_nphase_batch_t *b) {
  if (!b) return LBM_OK;
  destroy_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (lbm_nphase_t *h : b->cases) lbm_nphase_destroy(h);
  delete b;
  return LBM_OK;
}

}  // extern "C"
