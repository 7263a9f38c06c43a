// nrr_stencil.cu -- the relaxation hot path on sm_103a (arXiv 2501.14030,
// Sec. 2 relaxation system; Alg. 1 RHS -> BC -> RK substep, residual H and
// its L2 norm).
//
// One launch per RK4 stage evaluates the right-hand side at every evolved
// point -- the damped-wave RHS at interior points, the radiation condition on
// the outer ghost shell -- and applies the stage's RK4 update in the same
// pass.  Inner ghosts are never stored during a solve: the stencil reads the
// image point directly (phi periodicity, the xx0 < 0 and theta reflections),
// which is the inner boundary condition of Alg. 1 applied on read.
//
// Curvilinear grids: the reference metric, c^2 and the FD weights are folded
// into per-column weights (the metric is phi-independent), so the operator is
// 5*ng+1 fused multiply-adds on u plus the source term.
//
// Stage-kernel variants (chosen per grid by the autotuner): the column kernel
// (neighbours through the caches, 32-256 threads per block), register-staged
// tiles, a persistent grid-strided column kernel, 32 x 4 or (FP32) 32 x 8
// tiles fed by tensor (TMA) copies through an mbarrier ring, and multi-stage
// cooperative kernels (column items or tensor-copy tiles) that run whole
// chunks of RK4 steps with grid barriers; Cartesian grids have a column
// kernel and a tensor-copy kernel with separate ghost-shell blocks.  Each
// stage kernel may be launched with programmatic dependent launch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "nrr_internal.h"
#include "nrr_stencil.cuh"

namespace nrr {

namespace {

using namespace dev;


// Tiled curvilinear stage kernel (see stage_tile_block): grid (tiles in i0
// + 1 outer-shell column of blocks, tiles in i1, phi chunks of zc planes).
template <typename R, int NG, int KIND, int TY>
__global__ void __launch_bounds__(32 * TY)
    stage_tile_kernel(Geo g, StageArgs<R> a, int zc) {
  __shared__ R tile[2][TY + 2 * NG][32 + 2 * NG];
  pdl_trigger();
  stage_tile_block<R, NG, KIND, TY>(g, a, blockIdx.x, blockIdx.y, blockIdx.z, zc,
                                    tile);
}

// Column curvilinear stage kernel.  Thread = one (i0, i1) column of evolved
// points and ZC consecutive phi planes (grid y); all neighbours come from
// global memory (L1/L2).  Faster than the tiled kernel on small grids with
// few phi planes.
template <typename R, int NG, int KIND, int ZC>
__global__ void __launch_bounds__(256)
    stage_curvi_kernel(Geo g, StageArgs<R> a) {
  pdl_trigger();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (g.n0 + NG) * g.n1) return;
  stage_curvi_item<R, NG, KIND, ZC>(g, a, e, NG + blockIdx.y * ZC);
}

// SinhCylindrical column kernel: the interior columns as above (with the z
// direction read as stored), then the outer shell beyond the side and both
// ends; ZC phi planes per thread.
template <typename R, int NG, int KIND, int ZC>
__global__ void __launch_bounds__(256)
    stage_cyl_kernel(Geo g, StageArgs<R> a) {
  pdl_trigger();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.n0 * g.n1 + NG * g.n1 + 2 * NG * (g.n0 + NG)) return;
  stage_curvi_item<R, NG, KIND, ZC, false, true>(g, a, e, NG + blockIdx.y * ZC);
}

// Persistent column kernel: exactly (resident blocks x SMs) blocks stride
// over single (column, plane) items, so the remainder of the work is spread
// evenly over all SMs instead of forming a partial last wave.
template <typename R, int NG, int KIND>
__global__ void __launch_bounds__(128)
    stage_curvi_persistent_kernel(Geo g, StageArgs<R> a) {
  pdl_trigger();
  const int ncols = (g.n0 + NG) * g.n1;
  const int nitems = ncols * g.n2;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
       it += gridDim.x * blockDim.x)
    stage_curvi_item<R, NG, KIND, 1>(g, a, it % ncols, NG + it / ncols);
}

// Cartesian operator weights in the working precision, converted once per
// thread (a conversion from FP64 per use would run on the FP64 pipe).
template <typename R, int NG>
struct CartW {
  R c;
  R k[3][NG];
  __device__ __forceinline__ explicit CartW(const CartCoef &cc) : c(R(cc.cc)) {
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
      for (int j = 0; j < NG; j++) k[d][j] = R(cc.a[d][j]);
  }
};

template <typename R, int NG>
__device__ __forceinline__ R cart_operator(const Geo &g, const R *__restrict__ su,
                                           const CartW<R, NG> &w, int64_t p, R u0,
                                           R al, R bc2, int lin) {
  const int64_t st[3] = {1, g.s0, (int64_t)g.ncol};
  R lap = w.c * u0;
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int k = 1; k <= NG; k++)
      lap = fma(w.k[d][k - 1], ld(su + p + k * st[d]) + ld(su + p - k * st[d]), lap);
  return add_source(lap, u0, al, bc2, lin);
}

// Cartesian: uniform spacing, so the wave speed is one constant (1 on a lone
// grid; c^2 is in the folded weights, c multiplies the radiation term); every
// ghost is an outer ghost evolved by the radiation condition with
// d_r f = sum_i (x^i/r) D_i f (one-sided inward along directions in which the
// point lies outside, centred otherwise).  The per-launch constants
// (positions, 1 / (2 dxx)) are computed once on the host, and u and v share
// one 1/r: the FP64 division and square root are long instruction sequences
// on the FP64 pipe.
template <typename R>
struct CartShellC {
  R xmin[3];  // coordinate of padded index 0 + half a cell, per direction
  R dxx[3];   // spacing
  R inv2[3];  // 1 / (2 dxx)
};

template <typename R, int NG>
CartShellC<R> cart_shell_consts(const Geo &g) {
  CartShellC<R> sc;
  for (int d = 0; d < 3; d++) {
    sc.xmin[d] = (R)(g.xxmin[d] + (0.5 - NG) * g.dxx[d]);
    sc.dxx[d] = (R)g.dxx[d];
    sc.inv2[d] = (R)(0.5 / g.dxx[d]);
  }
  return sc;
}

// Radiation condition at ghost point (i0, i1, i2) for u and v together:
// k_f = -(d_r f + f / r) with d_r f = sum_d (x_d / r) D_d f, in the working
// precision.
template <typename R, int NG>
__device__ __forceinline__ void cart_shell_point(const Geo &g, const StageArgs<R> &a,
                                                 const CartShellC<R> &sc, int i0,
                                                 int i1, int i2, R &ku, R &kv) {
  const int ii[3] = {i0, i1, i2};
  const int nn[3] = {g.n0, g.n1, g.n2};
  const int64_t st[3] = {1, g.s0, (int64_t)g.ncol};
  const int64_t p = i0 + (int64_t)g.s0 * i1 + (int64_t)g.ncol * i2;
  R x[3], r2 = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    x[d] = fma(R(ii[d]), sc.dxx[d], sc.xmin[d]);
    r2 = fma(x[d], x[d], r2);
  }
  const R rinv = R(1) / sqrt(r2);
  const R u0 = ld(a.su + p), v0 = ld(a.sv + p);
  R dru = R(0), drv = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const R nx = mul_rn(x[d], rinv), inv2 = sc.inv2[d];
    R Du, Dv;
    if (ii[d] >= nn[d] + NG) {
      Du = mul_rn(fma(R(3), u0, fma(R(-4), ld(a.su + p - st[d]), ld(a.su + p - 2 * st[d]))), inv2);
      Dv = mul_rn(fma(R(3), v0, fma(R(-4), ld(a.sv + p - st[d]), ld(a.sv + p - 2 * st[d]))), inv2);
    } else if (ii[d] < NG) {
      Du = -mul_rn(fma(R(3), u0, fma(R(-4), ld(a.su + p + st[d]), ld(a.su + p + 2 * st[d]))), inv2);
      Dv = -mul_rn(fma(R(3), v0, fma(R(-4), ld(a.sv + p + st[d]), ld(a.sv + p + 2 * st[d]))), inv2);
    } else {
      Du = mul_rn(sub_rn(ld(a.su + p + st[d]), ld(a.su + p - st[d])), inv2);
      Dv = mul_rn(sub_rn(ld(a.sv + p + st[d]), ld(a.sv + p - st[d])), inv2);
    }
    dru = fma(nx, Du, dru);
    drv = fma(nx, Dv, drv);
  }
  const R c = R(a.cart.speed);
  ku = mul_rn(-c, fma(u0, rinv, dru));
  kv = mul_rn(-c, fma(v0, rinv, drv));
  if (linear_mode<R>(a.lin)) {
    ku += ld(a.fu + p);
    kv += ld(a.bc2 + p);
  }
}

template <typename R, int NG, int KIND>
__global__ void __launch_bounds__(256)
    stage_cart_kernel(Geo g, StageArgs<R> a, CartShellC<R> sc, int zc) {
  pdl_trigger();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ncol) return;
  pdl_wait();
  // Columns numbered interior first (i0 fastest), then the ring of ghost
  // columns around them: a warp then takes either the interior operator or
  // the radiation condition on a plane, not both one after the other.
  const int nint = g.n0 * g.n1;
  int i0, i1;
  if (e < nint) {
    i0 = NG + e % g.n0;
    i1 = NG + e / g.n0;
  } else {
    const int s = e - nint;
    if (s < 2 * NG * g.s0) {  // the NG ghost rows below and above
      const int r = s / g.s0;
      i0 = s - r * g.s0;
      i1 = r < NG ? r : g.n1 + r;
    } else {  // the NG ghost columns left and right of each interior row
      const int t = s - 2 * NG * g.s0, k = t % (2 * NG);
      i1 = NG + t / (2 * NG);
      i0 = k < NG ? k : g.n0 + k;
    }
  }
  const int col = i0 + g.s0 * i1;
  const int z0 = blockIdx.y * zc;
  const int z1 = min(z0 + zc, g.s2);
  const bool in01 = e < nint;
  const CartW<R, NG> w(a.cart);
  for (int i2 = z0; i2 < z1; i2++) {
    int64_t p = col + (int64_t)g.ncol * i2;
    R ku, kv;
    if (in01 && i2 >= NG && i2 < g.n2 + NG) {
      R u0 = ld(a.su + p), v0 = ld(a.sv + p);
      kv = cart_operator<R, NG>(g, a.su, w, p, u0, ld(a.alpha + p),
                                ld(a.bc2 + p), a.lin);
      ku = fma(-a.eta, u0, v0);
      if (linear_mode<R>(a.lin)) ku += ld(a.fu + p);
    } else {
      cart_shell_point<R, NG>(g, a, sc, i0, i1, i2, ku, kv);
    }
    stage_epilogue<R, KIND>(a, p, ku, kv);
  }
}

// ---------------------------------------------------------------------------
// Cartesian stage fed by tensor copies (variant 1; order 8, n0 % 32 == 0,
// n1 % 4 == 0, n2 and the plane chunk even).  Interior blocks: a 32 x 4
// column tile streams its chunk of planes, two per slot, through a 2-slot
// shared-memory ring (one 40 x 12 x 2 box of u with its halo, one 32 x 4 x 2
// box per operand array, completing on the slot's mbarrier; thread 0 refills
// a slot as soon as the block has read it).  Cartesian ghosts are all outer ghosts, stored and
// evolved, so the halo box needs no images; the i2 neighbours come from a
// register queue.  Extra blocks evolve the ghost shell with the radiation
// condition, one point per thread: first the two i2 slabs, then the ring of
// ghost columns on the interior planes.
// ---------------------------------------------------------------------------
using CartMaps = FieldSrc;  // su box (40, 12, 2), operand boxes (32, 4, 2)

constexpr int kCartTY = 4, kCartPZ = 2;
template <typename R>
__host__ __device__ constexpr int cart_slots() { return 2; }

__host__ __device__ __forceinline__ int64_t cart_shell_points(const Geo &g) {
  const int ng = g.ng;
  return 2 * (int64_t)ng * g.ncol +
         ((int64_t)g.ncol - (int64_t)g.n0 * g.n1) * g.n2;
}

// Grid constants of the shell points in the working precision, converted on
// the host (a conversion from FP64 per point would run on the FP64 pipe).
template <typename R, int NG, int KIND>
__global__ void __launch_bounds__(32 * kCartTY, sizeof(R) == 4 ? 6 : 1)
    stage_cart_tma_kernel(Geo g, StageArgs<R> a, const __grid_constant__ CartMaps maps,
                          CartShellC<R> sc, int zc) {
  constexpr int TY = kCartTY, PZ = kCartPZ, NS = cart_slots<R>();
  constexpr int TW = 32 + 2 * NG, TH = TY + 2 * NG;
  pdl_trigger();
  const int ntx = g.n0 / 32, nty = g.n1 / TY, nch = (g.n2 + zc - 1) / zc;
  const int nint = ntx * nty * nch;
  if ((int)blockIdx.x >= nint) {
    // ghost shell, one point per thread
    const int64_t w = (int64_t)(blockIdx.x - nint) * blockDim.x + threadIdx.x;
    if (w >= cart_shell_points(g)) return;
    int i0, i1, i2;
    const int64_t slab = 2 * (int64_t)NG * g.ncol;
    if (w < slab) {
      const int pl = (int)(w / g.ncol), rem = (int)(w - (int64_t)pl * g.ncol);
      i2 = pl < NG ? pl : g.n2 + pl;
      i1 = rem / g.s0;
      i0 = rem - i1 * g.s0;
    } else {
      const int64_t w2 = w - slab;
      const int nring = g.ncol - g.n0 * g.n1;
      const int rc = (int)(w2 % nring);
      i2 = NG + (int)(w2 / nring);
      const int band = NG * g.s0;  // the NG ghost rows below and above
      if (rc < 2 * band) {
        const int r = rc < band ? rc : rc - band;
        i1 = r / g.s0 + (rc < band ? 0 : g.n1 + NG);
        i0 = r - (r / g.s0) * g.s0;
      } else {
        const int r = rc - 2 * band;
        i1 = NG + r / (2 * NG);
        const int j = r - (r / (2 * NG)) * (2 * NG);
        i0 = j < NG ? j : g.n0 + j;
      }
    }
    pdl_wait();
    R ku, kv;
    cart_shell_point<R, NG>(g, a, sc, i0, i1, i2, ku, kv);
    stage_epilogue<R, KIND>(a, i0 + (int64_t)g.s0 * i1 + (int64_t)g.ncol * i2, ku, kv);
    return;
  }
  __shared__ __align__(128) TmaSlot<R, NG, TY, PZ> ring[NS];
  __shared__ __align__(8) uint64_t full[NS];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int tile_x = blockIdx.x % ntx, tile_y = (blockIdx.x / ntx) % nty,
            chunk = blockIdx.x / (ntx * nty);
  const int nc = g.ncol;
  const int z0 = NG + chunk * zc, z1 = min(z0 + zc, NG + g.n2);
  const int nslots = (z1 - z0) / PZ;
  const int i0 = NG + tile_x * 32 + tx, i1 = NG + tile_y * TY + ty;
  const int col = i0 + g.s0 * i1;
  const int j0b = tile_x * 32, j1b = tile_y * TY;
  const bool use_fu = linear_mode<R>(a.lin);
  constexpr bool use_b = KIND == STAGE_MID;
  constexpr bool use_acc = KIND == STAGE_MID || KIND == STAGE_LAST;
  const unsigned opmask = (1u << OP_SV) | (1u << OP_AL) | (1u << OP_BC) |
                          (use_fu ? 1u << OP_FU : 0u) |
                          (use_b ? (1u << OP_BU) | (1u << OP_BV) : 0u) |
                          (use_acc ? (1u << OP_AU) | (1u << OP_AV) : 0u);
  const uint32_t slot_bytes =
      (uint32_t)(PZ * (TW * TH + __popc(opmask) * TY * 32) * sizeof(R));
  // operator weights in the working precision
  const R wc = R(a.cart.cc);
  R wk[3][NG];
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int k = 0; k < NG; k++) wk[d][k] = R(a.cart.a[d][k]);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; k++) mbar_init_count(&full[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  pdl_wait();
  auto issue = [&](int pl, int sl) {
    mbar_arrive_expect(&full[sl], slot_bytes);
    fence_proxy_async_smem();
    tma_load_3d(&ring[sl].u[0][0][0], &maps.u, &full[sl], j0b, j1b, pl);
#pragma unroll
    for (int o = 0; o < 8; o++)
      if ((opmask >> o) & 1u)
        tma_load_3d(&ring[sl].op[o][0][0][0], &maps.op[o], &full[sl], NG + j0b,
                    NG + j1b, pl);
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < NS && k < nslots; k++) issue(z0 + PZ * k, k);
  // i2 queue of this column: planes i2 - NG .. i2 + NG of the slot's first
  // plane (ghost planes are stored: no wrap)
  R q[2 * NG + PZ];
#pragma unroll
  for (int k = 0; k < 2 * NG; k++) q[k + PZ] = ld(a.su + col + (int64_t)nc * (z0 - NG + k));
  R nq[PZ];
#pragma unroll
  for (int j = 0; j < PZ; j++) nq[j] = ld(a.su + col + (int64_t)nc * (z0 + NG + j));
  for (int base = 0, phase = 0; base < nslots; base += NS, phase ^= 1) {
#pragma unroll
    for (int sl = 0; sl < NS; sl++) {
      const int it = base + sl;
      if (it >= nslots) break;
      const int i2 = z0 + PZ * it;
      const bool ok = mbar_wait_parity(&full[sl], (uint32_t)phase);
      const TmaSlot<R, NG, TY, PZ> &S = ring[sl];
#pragma unroll
      for (int k = 0; k < 2 * NG; k++) q[k] = q[k + PZ];
#pragma unroll
      for (int j = 0; j < PZ; j++) q[2 * NG + j] = nq[j];
      if (__syncthreads_or(!ok)) {
        // a copy did not complete in time: record it, let the copies still
        // in flight (slots it .. it + NS - 1) land, bounded, and leave
        if (threadIdx.x == 0) {
          if (a.err) atomicExch(a.err, 1);
          for (int j = it; j < nslots && j < it + NS; j++)
            mbar_wait_parity(&full[j % NS], (uint32_t)((j / NS) & 1));
        }
        __syncthreads();
        return;
      }
      if (it + 1 < nslots) {
#pragma unroll
        for (int j = 0; j < PZ; j++)
          nq[j] = ld(a.su + col + (int64_t)nc * (i2 + PZ + NG + j));
      }
#pragma unroll
      for (int j = 0; j < PZ; j++) {
        const int64_t p = col + (int64_t)nc * (i2 + j);
        const R(&t)[TH][TW] = S.u[j];
        const R u0 = t[ty + NG][tx + NG];
        const R v0 = S.op[OP_SV][j][ty][tx];
        R a0 = wc * u0, a1 = R(0);
#pragma unroll
        for (int k = 1; k <= NG; k++) {
          a0 = fma(wk[0][k - 1], t[ty + NG][tx + NG + k] + t[ty + NG][tx + NG - k], a0);
          a1 = fma(wk[1][k - 1], t[ty + NG + k][tx + NG] + t[ty + NG - k][tx + NG], a1);
          a0 = fma(wk[2][k - 1], q[NG + j + k] + q[NG + j - k], a0);
        }
        const R kv = add_source(a0 + a1, u0, S.op[OP_AL][j][ty][tx],
                                S.op[OP_BC][j][ty][tx], a.lin);
        R ku = fma(-a.eta, u0, v0);
        if (use_fu) ku += S.op[OP_FU][j][ty][tx];
        if (KIND == STAGE_FIRST) {
          st(a.au + p, fma(a.wb, ku, u0));
          st(a.av + p, fma(a.wb, kv, v0));
          st(a.ou + p, fma(a.wa, ku, u0));
          st(a.ov + p, fma(a.wa, kv, v0));
        } else if (KIND == STAGE_MID) {
          st(a.au + p, fma(a.wb, ku, S.op[OP_AU][j][ty][tx]));
          st(a.av + p, fma(a.wb, kv, S.op[OP_AV][j][ty][tx]));
          st(a.ou + p, fma(a.wa, ku, S.op[OP_BU][j][ty][tx]));
          st(a.ov + p, fma(a.wa, kv, S.op[OP_BV][j][ty][tx]));
        } else if (KIND == STAGE_LAST) {
          st(a.ou + p, fma(a.wb, ku, S.op[OP_AU][j][ty][tx]));
          st(a.ov + p, fma(a.wb, kv, S.op[OP_AV][j][ty][tx]));
        } else {
          st(a.ou + p, ku);
          st(a.ov + p, kv);
        }
      }
      // refill this slot as soon as every thread is done with it: NS copies
      // in flight while the block waits for the next one
      if (it + NS < nslots) {
        __syncthreads();
        if (threadIdx.x == 0) issue(i2 + PZ * NS, sl);
      }
    }
  }
}

// Curvilinear stage fed by tensor copies (variant 3; order 8, n0 % 32 == 0,
// n1 % TY == 0): interior blocks run stage_tma_block on a 32 x TY column
// tile (TY = 4 or 8) and a chunk of phi planes with one 3-D tensor map per
// array (kernel parameter); the blocks after them evolve the outer shell,
// 32 TY / NG rows of i1 and the NG shell columns each.  Both tile heights
// keep 80 registers and 768 threads per SM in FP32.
template <typename R, int NG, int KIND, int TY>
__global__ void __launch_bounds__(32 * TY, sizeof(R) == 4 ? 24 / TY : 1)
    stage_curvi_tma_kernel(Geo g, StageArgs<R> a, const __grid_constant__ FieldSrc maps,
                           int zc) {
  constexpr int PZ = kCartPZ, NS = cart_slots<R>();
  pdl_trigger();
  const int ntx = g.n0 / 32, nty = g.n1 / TY, nch = chunks_z(g, zc);
  const int nint = ntx * nty * nch;
  if ((int)blockIdx.x >= nint) {
    constexpr int rows = 32 * TY / NG;
    const int nsb = (g.n1 + rows - 1) / rows;
    const int sidx = blockIdx.x - nint, chunk = sidx / nsb;
    const int row = threadIdx.x / NG, lane = threadIdx.x - row * NG;
    const int z0 = NG + chunk * zc;
    if (row < rows)
      stage_shell_rows<R, NG, KIND>(g, a, lane, NG + (sidx % nsb) * rows + row, z0,
                                    min(z0 + zc, NG + g.n2));
    return;
  }
  __shared__ __align__(128) TmaSlot<R, NG, TY, PZ, sizeof(R) == 4> ring[NS];
  __shared__ __align__(8) uint64_t full[NS];
  stage_tma_block<R, NG, KIND, TY, NS, PZ>(g, a, blockIdx.x % ntx,
                                            (blockIdx.x / ntx) % nty,
                                            blockIdx.x / (ntx * nty), zc, maps, ring,
                                            full, a.err);
}

// ---------------------------------------------------------------------------
// Multi-stage curvilinear kernel (variant 4): one cooperative launch runs
// `steps` RK4 steps -- every stage over all (column, plane) items of the
// evolved points, grid-strided -- with a grid barrier after each stage, so
// that small grids do not pay a launch and ramp per stage.  State written by
// an earlier stage is read through L2 (coherent loads); every barrier wait
// is bounded and records an expiry in the error flag.
// ---------------------------------------------------------------------------
template <typename R>
struct StageArgs4 {
  StageArgs<R> s[4];  // FIRST, MID, MID, LAST
};

template <typename R, int NG>
__global__ void __launch_bounds__(128)
    stage_curvi_multi_kernel(Geo g, StageArgs4<R> sa, int steps, unsigned *count) {
  pdl_trigger();
  const int ncols = (g.n0 + NG) * g.n1;
  const int nitems = ncols * g.n2;
  const int nthr = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned target = 0;
  for (int s = 0; s < steps; s++) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      for (int it = tid; it < nitems; it += nthr) {
        const int e = it % ncols, z = NG + it / ncols;
        if (k == 0)
          stage_curvi_item<R, NG, STAGE_FIRST, 1, true>(g, sa.s[0], e, z);
        else if (k == 3)
          stage_curvi_item<R, NG, STAGE_LAST, 1, true>(g, sa.s[3], e, z);
        else
          stage_curvi_item<R, NG, STAGE_MID, 1, true>(g, sa.s[k], e, z);
      }
      target += gridDim.x;
      grid_barrier(count, target, sa.s[0].err);
    }
  }
}

template <typename R, int NG>
cudaError_t launch_multi_ng(const Geo &g, const StageArgs4<R> &sa, int steps,
                            unsigned *count, int pdl, cudaStream_t st) {
  auto k = stage_curvi_multi_kernel<R, NG>;
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, 0);
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // as many items per thread as the resident grid needs, spread evenly
  const int64_t items = (int64_t)(g.n0 + NG) * g.n1 * g.n2;
  const int64_t ipt = (items + 128ll * per_sm * sms - 1) / (128ll * per_sm * sms);
  const int blocks = (int)((items + 128 * ipt - 1) / (128 * ipt));
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3(blocks);
  c.blockDim = dim3(128);
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // all blocks resident at once
  at[0].val.cooperative = 1;
  c.attrs = at;
  c.numAttrs = 1;
  (void)pdl;
  return cudaLaunchKernelEx(&c, k, g, sa, steps, count);
}

// Multi-stage tensor-copy kernel (variant 5; the grids of variant 3): the
// cooperative multi-stage launch of variant 4 over variant 3's work items --
// interior tiles staged through tensor copies, then shell blocks -- so that
// a block's stencil reads come from shared memory instead of a cache that
// each grid barrier leaves cold.  Tensor copies read global memory through
// the async proxy: every thread fences its stores of a stage before the
// barrier and the issuing thread fences again after it.  State read by
// plain loads (phi queue, image cells, shell) goes through L2.
struct FieldSrc4 {
  FieldSrc s[4];  // FIRST, MID, MID, LAST
};

template <typename R, int NG, int KIND>
__device__ __forceinline__ void multi_tma_stage(const Geo &g, const StageArgs<R> &a,
                                                const FieldSrc &maps, int zc,
                                                TmaSlot<R, NG, kCartTY, kCartPZ> *ring,
                                                uint64_t *full, bool &inited) {
  constexpr int TY = kCartTY, PZ = kCartPZ, NS = cart_slots<R>();
  constexpr int rows = 32 * TY / NG;
  const int ntx = g.n0 / 32, nty = g.n1 / TY, nch = chunks_z(g, zc);
  const int nint = ntx * nty * nch;
  const int nsb = (g.n1 + rows - 1) / rows;
  const int nitems = nint + nsb * nch;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // after an expired wait the remaining items are skipped (uniformly)
    if (__syncthreads_or(threadIdx.x == 0 && *(volatile int *)a.err != 0)) return;
    if (it < nint) {
      if (inited && threadIdx.x == 0)
        for (int k = 0; k < NS; k++) mbar_inval(&full[k]);
      inited = true;
      stage_tma_block<R, NG, KIND, TY, NS, PZ, FieldSrc, true>(
          g, a, it % ntx, (it / ntx) % nty, it / (ntx * nty), zc, maps, ring, full,
          a.err);
    } else {
      const int sidx = it - nint, chunk = sidx / nsb;
      const int row = threadIdx.x / NG, lane = threadIdx.x - row * NG;
      const int z0 = NG + chunk * zc;
      if (row < rows)
        stage_shell_rows<R, NG, KIND, true>(g, a, lane, NG + (sidx % nsb) * rows + row,
                                            z0, min(z0 + zc, NG + g.n2));
    }
  }
}

template <typename R, int NG>
__global__ void __launch_bounds__(32 * kCartTY, sizeof(R) == 4 ? 4 : 1)
    stage_curvi_multi_tma_kernel(Geo g, StageArgs4<R> sa,
                                 const __grid_constant__ FieldSrc4 maps, int zc,
                                 int steps, unsigned *count) {
  __shared__ __align__(128) TmaSlot<R, NG, kCartTY, kCartPZ> ring[cart_slots<R>()];
  __shared__ __align__(8) uint64_t full[cart_slots<R>()];
  pdl_trigger();
  bool inited = false;
  unsigned target = 0;
  for (int s = 0; s < steps; s++) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (k == 0)
        multi_tma_stage<R, NG, STAGE_FIRST>(g, sa.s[0], maps.s[0], zc, ring, full, inited);
      else if (k == 3)
        multi_tma_stage<R, NG, STAGE_LAST>(g, sa.s[3], maps.s[3], zc, ring, full, inited);
      else
        multi_tma_stage<R, NG, STAGE_MID>(g, sa.s[k], maps.s[k], zc, ring, full, inited);
      fence_proxy_async_all();
      target += gridDim.x;
      grid_barrier(count, target, sa.s[0].err);
      if (threadIdx.x == 0) fence_proxy_async_all();
    }
  }
}


// Residual H at interior points and the block partials of H^2 J, J over
// r < r_int (the volume-weighted L2 norm of Alg. 1's residual).
template <typename R, int NG, bool CYL = false>
__global__ void __launch_bounds__(128)
    residual_curvi_kernel(Geo g, const R *__restrict__ su,
                          const R *__restrict__ alpha, const R *__restrict__ bc2,
                          ColumnSet<R> col_set, const double *__restrict__ jac,
                          const double *__restrict__ rad, double r_int,
                          double *h_out, double *partials, int zc, int lin) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (e < g.n0 * g.n1) {
    const int col = (e % g.n0 + NG) + g.s0 * (e / g.n0 + NG);
    const double wt = rad[col] < r_int ? jac[col] : 0.0;
    const int z0 = NG + blockIdx.y * zc;
    residual_curvi_item<R, NG, CYL>(g, su, alpha, bc2, col_set, wt, e, z0,
                                    min(z0 + zc, NG + g.n2), lin, h_out, num, den);
  }
  block_sum2(num, den, partials + 2 * (blockIdx.x + gridDim.x * blockIdx.y));
}

template <typename R, int NG>
__global__ void __launch_bounds__(128)
    residual_cart_kernel(Geo g, const R *__restrict__ su,
                         const R *__restrict__ alpha, const R *__restrict__ bc2,
                         CartCoef cc, double r_int, double *h_out,
                         double *partials, int zc, int lin) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (e < g.n0 * g.n1) {
    const int i0 = e % g.n0 + NG, i1 = e / g.n0 + NG;
    const int z0 = NG + blockIdx.y * zc;
    const int z1 = min(z0 + zc, NG + g.n2);
    double x0 = g.xxmin[0] + (i0 - NG + 0.5) * g.dxx[0];
    double x1 = g.xxmin[1] + (i1 - NG + 0.5) * g.dxx[1];
    const CartW<R, NG> w(cc);
    for (int i2 = z0; i2 < z1; i2++) {
      int64_t p = i0 + (int64_t)g.s0 * (i1 + (int64_t)g.s1 * i2);
      R u0 = ld(su + p);
      // the operator carries the folded c^2 (exactly 1 on a lone grid)
      double H = (double)cart_operator<R, NG>(g, su, w, p, u0, ld(alpha + p),
                                              ld(bc2 + p), lin) /
                 (cc.speed * cc.speed);
      if (h_out) h_out[p] = H;
      double x2 = g.xxmin[2] + (i2 - NG + 0.5) * g.dxx[2];
      double wt = sqrt(x0 * x0 + x1 * x1 + x2 * x2) < r_int ? 1.0 : 0.0;
      num = fma(H * H, wt, num);
      den += wt;
    }
  }
  block_sum2(num, den, partials + 2 * (blockIdx.x + gridDim.x * blockIdx.y));
}

__global__ void norm_finalize_kernel(const double *partials, int nblocks,
                                     double *out) {
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    x += partials[2 * i];
    y += partials[2 * i + 1];
  }
  __shared__ double res[2];
  block_sum2(x, y, res);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = res[1] > 0.0 ? sqrt(res[0] / res[1]) : 0.0;
    out[1] = res[0];
    out[2] = res[1];
  }
}

template <typename R>
__global__ void fill_ghosts_kernel(Geo g, R *f) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.npts) return;
  int i0 = (int)(p % g.s0);
  int i1 = (int)((p / g.s0) % g.s1);
  int i2 = (int)(p / g.ncol);
  // (SinhCylindrical rows beyond the ends in z are evolved outer points)
  bool evolved = i0 >= g.ng &&
                 (g.coord == SINHCYLINDRICAL || (i1 >= g.ng && i1 < g.n1 + g.ng)) &&
                 i2 >= g.ng && i2 < g.n2 + g.ng;
  if (evolved) return;
  int j0 = i0, j1 = i1, j2 = i2;
  image_of(g, j0, j1, j2);
  dev::st(f + p, dev::ld(f + flat(g, j0, j1, j2)));
}

// Defect correction, set-up of one outer iteration at the FP64 state (u, v)
// whose FP64 right-hand side (with boundary conditions) is (ku, kv):
//   c^2 a = 7 alpha (c^2 beta) (1 + alpha u)^-8   (linearised source)
//   f_u = ku, f_v = kv                            (the defect, as forcing)
__global__ void dc_prepare_kernel(Geo g, const double *__restrict__ u,
                                  const double *__restrict__ alpha,
                                  const double *__restrict__ bc2,
                                  const double *__restrict__ ku,
                                  const double *__restrict__ kv, float *ac2,
                                  float *fu, float *fv) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.npts) return;
  double t = 1.0 / (1.0 + alpha[p] * u[p]);
  double t2 = t * t, t4 = t2 * t2;
  ac2[p] = (float)(7.0 * alpha[p] * bc2[p] * (t4 * t4));
  fu[p] = (float)ku[p];
  fv[p] = (float)kv[p];
}

// (u, v) += (d, w): the FP64 update with the FP32 increments.
__global__ void dc_update_kernel(double *u, double *v, const float *d,
                                 const float *w, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    u[i] += (double)d[i];
    v[i] += (double)w[i];
  }
}

__global__ void convert_d2f_kernel(const double *s, float *d, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}
__global__ void convert_f2d_kernel(const float *s, double *d, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (double)s[i];
}
__global__ void scale_kernel(double *f, double s, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] *= s;
}

constexpr int kTileY = 4;

// Launch with or without the programmatic-serialisation attribute (stage
// kernels only: each calls pdl_wait() before touching the state).
template <typename... P, typename... A>
void launch_stage_kernel(void (*k)(P...), dim3 grid, dim3 block, cudaStream_t st,
                         int pdl, A... args) {
  cudaLaunchConfig_t c = {};
  c.gridDim = grid;
  c.blockDim = block;
  c.dynamicSmemBytes = 0;
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = at;
  c.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&c, k, args...);
}

template <typename R, int NG, int KIND>
void launch_tile_kind(const Geo &g, const StageArgs<R> &a, int zc, int pdl,
                      cudaStream_t st) {
  dim3 grid(tiles_x(g) + 1, tiles_y<kTileY>(g), chunks_z(g, zc));
  launch_stage_kernel(stage_tile_kernel<R, NG, KIND, kTileY>, grid,
                      dim3(32 * kTileY), st, pdl, g, a, zc);
}

template <typename R, int NG, int KIND, int ZC>
void launch_column_zc(const Geo &g, const StageArgs<R> &a, int block, int pdl,
                      cudaStream_t st) {
  dim3 grid(((g.n0 + NG) * g.n1 + block - 1) / block, (g.n2 + ZC - 1) / ZC);
  launch_stage_kernel(stage_curvi_kernel<R, NG, KIND, ZC>, grid, dim3(block), st,
                      pdl, g, a);
}

template <typename R, int NG, int KIND, int ZC>
void launch_cyl_zc(const Geo &g, const StageArgs<R> &a, int block, int pdl,
                   cudaStream_t st) {
  const int ncols = g.n0 * g.n1 + NG * g.n1 + 2 * NG * (g.n0 + NG);
  dim3 grid((ncols + block - 1) / block, (g.n2 + ZC - 1) / ZC);
  launch_stage_kernel(stage_cyl_kernel<R, NG, KIND, ZC>, grid, dim3(block), st,
                      pdl, g, a);
}

template <typename R, int NG, int KIND>
void launch_cyl_kind(const Geo &g, const StageArgs<R> &a, int zc, int block,
                     int pdl, cudaStream_t st) {
  switch (zc) {
    case 1: launch_cyl_zc<R, NG, KIND, 1>(g, a, block, pdl, st); break;
    case 4: launch_cyl_zc<R, NG, KIND, 4>(g, a, block, pdl, st); break;
    default: launch_cyl_zc<R, NG, KIND, 2>(g, a, block, pdl, st); break;
  }
}

template <typename R, int NG, int KIND>
void launch_column_kind(const Geo &g, const StageArgs<R> &a, int zc, int block,
                        int pdl, cudaStream_t st) {
  switch (zc) {
    case 1: launch_column_zc<R, NG, KIND, 1>(g, a, block, pdl, st); break;
    case 4: launch_column_zc<R, NG, KIND, 4>(g, a, block, pdl, st); break;
    default: launch_column_zc<R, NG, KIND, 2>(g, a, block, pdl, st); break;
  }
}

// Blocks that fill every SM for one kernel (resident blocks per SM x SMs of
// the current device), looked up once per kernel instantiation.
template <typename K>
int filling_grid(K kernel) {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    cached = sms * (per_sm > 0 ? per_sm : 1);
  }
  return cached;
}

template <typename R, int NG, int KIND>
void launch_persistent_kind(const Geo &g, const StageArgs<R> &a, int pdl,
                            cudaStream_t st) {
  auto k = stage_curvi_persistent_kernel<R, NG, KIND>;
  const int items = (g.n0 + NG) * g.n1 * g.n2;
  const int blocks = min(filling_grid(k), (items + 127) / 128);
  launch_stage_kernel(k, dim3(blocks), dim3(128), st, pdl, g, a);
}

// Tensor maps of whole padded fields (3-D, i0 fastest) for the Cartesian
// tensor-copy stage, encoded once per (field, box) and reused.
using TensorMapEncodeFn = CUresult (*)(
    CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
    CUtensorMapFloatOOBfill);
struct FieldMapKey {
  const void *p;
  int esize, s0, s1, s2, b0, b1;
  bool operator<(const FieldMapKey &o) const {
    return std::tie(p, esize, s0, s1, s2, b0, b1) <
           std::tie(o.p, o.esize, o.s0, o.s1, o.s2, o.b0, o.b1);
  }
};
std::mutex g_fmap_mu;
std::map<FieldMapKey, CUtensorMap> g_fmaps;

bool field_map(CUtensorMap *out, const void *p, int esize, const Geo &g, int b0,
               int b1) {
  std::lock_guard<std::mutex> lock(g_fmap_mu);
  const FieldMapKey key{p, esize, g.s0, g.s1, g.s2, b0, b1};
  auto it = g_fmaps.find(key);
  if (it != g_fmaps.end()) {
    *out = it->second;
    return true;
  }
  auto enc = reinterpret_cast<TensorMapEncodeFn>(tensor_map_encoder());
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.s0, (cuuint64_t)g.s1, (cuuint64_t)g.s2};
  const cuuint64_t strides[2] = {(cuuint64_t)g.s0 * esize, (cuuint64_t)g.ncol * esize};
  const cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)kCartPZ};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  if (enc(&m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
          3, const_cast<void *>(p), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  g_fmaps[key] = m;
  *out = m;
  return true;
}

// Whether the Cartesian tensor-copy stage applies to this grid and launch.
bool cart_tma_ok(const Geo &g, int zc) {
  return g.ng == 4 && g.n0 % 32 == 0 && g.n1 % kCartTY == 0 && g.n2 % kCartPZ == 0 &&
         zc % kCartPZ == 0 && g.s0 % 4 == 0;
}

// Whether the curvilinear tensor-copy stage with tiles of ty rows applies
// to this grid and launch.
bool curvi_tma_ok(const Geo &g, int zc, int ty = kCartTY) {
  return g.ng == 4 && g.n0 % 32 == 0 && g.n1 % ty == 0 &&
         g.n2 % kCartPZ == 0 && zc % kCartPZ == 0 && g.s0 % 4 == 0;
}

// Maps of the arrays a stage kind reads: su with halo boxes, operands with
// tile boxes; false if the driver cannot encode them.
template <typename R, int NG, int KIND>
bool stage_field_maps(FieldSrc *m, const Geo &g, const StageArgs<R> &a, int b0u,
                      int b1u, int ty = kCartTY) {
  const int es = (int)sizeof(R);
  const R *ops[8] = {a.sv, a.alpha, a.bc2, a.fu, a.bu, a.bv, a.au, a.av};
  const bool use_fu = a.lin != 0 && sizeof(R) == 4;
  const bool use_b = KIND == STAGE_MID, use_acc = KIND == STAGE_MID || KIND == STAGE_LAST;
  const bool need[8] = {true, true, true, use_fu, use_b, use_b, use_acc, use_acc};
  if (!field_map(&m->u, a.su, es, g, b0u, b1u)) return false;
  if (!field_map(&m->ph, a.su, es, g, 32, ty)) return false;
  for (int o = 0; o < 8; o++) {
    if (need[o]) {
      if (!field_map(&m->op[o], ops[o], es, g, 32, ty)) return false;
    } else {
      m->op[o] = m->u;  // unused slot
    }
  }
  return true;
}

template <typename R, int NG, int KIND, int TY>
bool launch_curvi_tma_kind(const Geo &g, const StageArgs<R> &a, int zc, int pdl,
                           cudaStream_t st) {
  FieldSrc maps;
  if (!stage_field_maps<R, NG, KIND>(&maps, g, a, 32 + 2 * NG, TY + 2 * NG, TY))
    return false;
  constexpr int rows = 32 * TY / NG;
  const int nch = chunks_z(g, zc);
  const int nint = (g.n0 / 32) * (g.n1 / TY) * nch;
  const int nshell = ((g.n1 + rows - 1) / rows) * nch;
  launch_stage_kernel(stage_curvi_tma_kernel<R, NG, KIND, TY>, dim3(nint + nshell),
                      dim3(32 * TY), st, pdl, g, a, maps, zc);
  return true;
}

template <typename R, int NG, int KIND>
bool launch_cart_tma_kind(const Geo &g, const StageArgs<R> &a, int zc, int pdl,
                          cudaStream_t st) {
  CartMaps maps;
  if (!stage_field_maps<R, NG, KIND>(&maps, g, a, 32 + 2 * NG, kCartTY + 2 * NG))
    return false;
  const CartShellC<R> sc = cart_shell_consts<R, NG>(g);
  const int nint = (g.n0 / 32) * (g.n1 / kCartTY) * ((g.n2 + zc - 1) / zc);
  const int nshell = (int)((cart_shell_points(g) + 32 * kCartTY - 1) / (32 * kCartTY));
  launch_stage_kernel(stage_cart_tma_kernel<R, NG, KIND>, dim3(nint + nshell),
                      dim3(32 * kCartTY), st, pdl, g, a, maps, sc, zc);
  return true;
}

template <typename R, int NG>
bool launch_cart_tma(const Geo &g, int kind, const StageArgs<R> &a, int zc, int pdl,
                     cudaStream_t st) {
  if constexpr (NG != 4) {
    return false;
  } else {
    switch (kind) {
      case STAGE_FIRST: return launch_cart_tma_kind<R, NG, STAGE_FIRST>(g, a, zc, pdl, st);
      case STAGE_MID: return launch_cart_tma_kind<R, NG, STAGE_MID>(g, a, zc, pdl, st);
      case STAGE_LAST: return launch_cart_tma_kind<R, NG, STAGE_LAST>(g, a, zc, pdl, st);
      default: return launch_cart_tma_kind<R, NG, STAGE_RAW>(g, a, zc, pdl, st);
    }
  }
}

// One cooperative launch of the multi-stage tensor-copy kernel; false if
// the maps cannot be encoded (the caller falls back to variant 4's shape).
template <typename R, int NG>
bool launch_multi_tma(const Geo &g, const StageArgs4<R> &sa, int zc, int steps,
                      unsigned *count, cudaStream_t st, cudaError_t *err) {
  constexpr int b0 = 32 + 2 * NG, b1 = kCartTY + 2 * NG;
  FieldSrc4 maps;
  if (!stage_field_maps<R, NG, STAGE_FIRST>(&maps.s[0], g, sa.s[0], b0, b1) ||
      !stage_field_maps<R, NG, STAGE_MID>(&maps.s[1], g, sa.s[1], b0, b1) ||
      !stage_field_maps<R, NG, STAGE_MID>(&maps.s[2], g, sa.s[2], b0, b1) ||
      !stage_field_maps<R, NG, STAGE_LAST>(&maps.s[3], g, sa.s[3], b0, b1))
    return false;
  auto k = stage_curvi_multi_tma_kernel<R, NG>;
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * kCartTY, 0);
  }
  if (per_sm < 1) {
    *err = cudaErrorInvalidConfiguration;
    return true;
  }
  constexpr int rows = 32 * kCartTY / NG;
  const int nch = chunks_z(g, zc);
  const int items = (g.n0 / 32) * (g.n1 / kCartTY) * nch + ((g.n1 + rows - 1) / rows) * nch;
  // as many items per block as the resident grid needs, spread evenly
  const int ipb = (items + per_sm * sms - 1) / (per_sm * sms);
  const int blocks = (items + ipb - 1) / ipb;
  *err = cudaMemsetAsync(count, 0, sizeof(unsigned), st);
  if (*err != cudaSuccess) return true;
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3(blocks);
  c.blockDim = dim3(32 * kCartTY);
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  c.attrs = at;
  c.numAttrs = 1;
  *err = cudaLaunchKernelEx(&c, k, g, sa, maps, zc, steps, count);
  return true;
}

template <typename R, int NG>
void launch_curvi(const Geo &g, int kind, const StageArgs<R> &a,
                  const LaunchCfg &cfg, cudaStream_t st) {
  const int zc = cfg.zc, pdl = cfg.pdl;
  if (cfg.variant == 6) {
    // single stage launches of the two-stage shape: the column kernel
    LaunchCfg col = cfg;
    col.variant = 0;
    col.zc = 2;
    launch_curvi<R, NG>(g, kind, a, col, st);
    return;
  }
  if (cfg.variant == 4) {
    // single stage launches of the multi-stage shape: the column kernel
    LaunchCfg col = cfg;
    col.variant = 0;
    col.zc = 1;
    launch_curvi<R, NG>(g, kind, a, col, st);
    return;
  }
  if (cfg.variant == 5) {
    // single stage launches of the multi-stage tensor-copy shape: variant 3
    LaunchCfg tc = cfg;
    tc.variant = 3;
    launch_curvi<R, NG>(g, kind, a, tc, st);
    return;
  }
  if (cfg.variant == 3) {
    if constexpr (NG == 4) {
      // FP32: 256-thread blocks select tiles of 8 rows of i1, others 4 (an
      // FP64 ring of 8-row tiles would exceed 48 KB of static shared memory)
      if constexpr (sizeof(R) == 4) {
        if (cfg.block == 256 && curvi_tma_ok(g, zc, 8)) {
          bool ok = false;
          switch (kind) {
            case STAGE_FIRST: ok = launch_curvi_tma_kind<R, NG, STAGE_FIRST, 8>(g, a, zc, pdl, st); break;
            case STAGE_MID: ok = launch_curvi_tma_kind<R, NG, STAGE_MID, 8>(g, a, zc, pdl, st); break;
            case STAGE_LAST: ok = launch_curvi_tma_kind<R, NG, STAGE_LAST, 8>(g, a, zc, pdl, st); break;
            default: ok = launch_curvi_tma_kind<R, NG, STAGE_RAW, 8>(g, a, zc, pdl, st); break;
          }
          if (ok) return;
        }
      }
      if (curvi_tma_ok(g, zc)) {
        bool ok = false;
        switch (kind) {
          case STAGE_FIRST: ok = launch_curvi_tma_kind<R, NG, STAGE_FIRST, 4>(g, a, zc, pdl, st); break;
          case STAGE_MID: ok = launch_curvi_tma_kind<R, NG, STAGE_MID, 4>(g, a, zc, pdl, st); break;
          case STAGE_LAST: ok = launch_curvi_tma_kind<R, NG, STAGE_LAST, 4>(g, a, zc, pdl, st); break;
          default: ok = launch_curvi_tma_kind<R, NG, STAGE_RAW, 4>(g, a, zc, pdl, st); break;
        }
        if (ok) return;
      }
    }
    // not applicable here: the register-staged tiled kernel does the same work
    LaunchCfg tiled = cfg;
    tiled.variant = 1;
    launch_curvi<R, NG>(g, kind, a, tiled, st);
    return;
  }
  if (cfg.variant == 2) {
    switch (kind) {
      case STAGE_FIRST: launch_persistent_kind<R, NG, STAGE_FIRST>(g, a, pdl, st); break;
      case STAGE_MID: launch_persistent_kind<R, NG, STAGE_MID>(g, a, pdl, st); break;
      case STAGE_LAST: launch_persistent_kind<R, NG, STAGE_LAST>(g, a, pdl, st); break;
      default: launch_persistent_kind<R, NG, STAGE_RAW>(g, a, pdl, st); break;
    }
    return;
  }
  if (cfg.variant == 0) {
    switch (kind) {
      case STAGE_FIRST: launch_column_kind<R, NG, STAGE_FIRST>(g, a, zc, cfg.block, pdl, st); break;
      case STAGE_MID: launch_column_kind<R, NG, STAGE_MID>(g, a, zc, cfg.block, pdl, st); break;
      case STAGE_LAST: launch_column_kind<R, NG, STAGE_LAST>(g, a, zc, cfg.block, pdl, st); break;
      default: launch_column_kind<R, NG, STAGE_RAW>(g, a, zc, cfg.block, pdl, st); break;
    }
    return;
  }
  switch (kind) {
    case STAGE_FIRST: launch_tile_kind<R, NG, STAGE_FIRST>(g, a, zc, pdl, st); break;
    case STAGE_MID: launch_tile_kind<R, NG, STAGE_MID>(g, a, zc, pdl, st); break;
    case STAGE_LAST: launch_tile_kind<R, NG, STAGE_LAST>(g, a, zc, pdl, st); break;
    default: launch_tile_kind<R, NG, STAGE_RAW>(g, a, zc, pdl, st); break;
  }
}

template <typename R, int NG>
void launch_stage_ng(const Geo &g, int kind, const StageArgs<R> &a,
                     const LaunchCfg &cfg, cudaStream_t st) {
  if (g.coord == CARTESIAN) {
    if (cfg.variant == 1 && cart_tma_ok(g, cfg.zc) &&
        launch_cart_tma<R, NG>(g, kind, a, cfg.zc, cfg.pdl, st))
      return;
    dim3 grid((g.ncol + cfg.block - 1) / cfg.block, (g.s2 + cfg.zc - 1) / cfg.zc);
    dim3 blk(cfg.block);
    const CartShellC<R> sc = cart_shell_consts<R, NG>(g);
    switch (kind) {
      case STAGE_FIRST: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_FIRST>, grid, blk, st, cfg.pdl, g, a, sc, cfg.zc); break;
      case STAGE_MID: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_MID>, grid, blk, st, cfg.pdl, g, a, sc, cfg.zc); break;
      case STAGE_LAST: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_LAST>, grid, blk, st, cfg.pdl, g, a, sc, cfg.zc); break;
      default: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_RAW>, grid, blk, st, cfg.pdl, g, a, sc, cfg.zc); break;
    }
    return;
  }
  if (g.coord == SINHCYLINDRICAL) {
    // the column kernel only (the other stage-kernel variants treat the
    // second direction as theta)
    const int zc = (cfg.variant == 0 && (cfg.zc == 1 || cfg.zc == 2 || cfg.zc == 4))
                       ? cfg.zc : 1;
    switch (kind) {
      case STAGE_FIRST: launch_cyl_kind<R, NG, STAGE_FIRST>(g, a, zc, cfg.block, cfg.pdl, st); break;
      case STAGE_MID: launch_cyl_kind<R, NG, STAGE_MID>(g, a, zc, cfg.block, cfg.pdl, st); break;
      case STAGE_LAST: launch_cyl_kind<R, NG, STAGE_LAST>(g, a, zc, cfg.block, cfg.pdl, st); break;
      default: launch_cyl_kind<R, NG, STAGE_RAW>(g, a, zc, cfg.block, cfg.pdl, st); break;
    }
    return;
  }
  launch_curvi<R, NG>(g, kind, a, cfg, st);
}

template <typename R, int NG>
void launch_residual_ng(const Geo &g, const R *u, const R *alpha, const R *bc2,
                        ColumnSet<R> col, const CartCoef &cart,
                        const double *jac, const double *rad, double r_int,
                        double *h_out, double *partials, const LaunchCfg &cfg,
                        cudaStream_t st, int lin) {
  dim3 grid((g.n0 * g.n1 + cfg.block - 1) / cfg.block,
            (g.n2 + cfg.zc - 1) / cfg.zc);
  if (g.coord == CARTESIAN)
    residual_cart_kernel<R, NG><<<grid, cfg.block, 0, st>>>(
        g, u, alpha, bc2, cart, r_int, h_out, partials, cfg.zc, lin);
  else if (g.coord == SINHCYLINDRICAL)
    residual_curvi_kernel<R, NG, true><<<grid, cfg.block, 0, st>>>(
        g, u, alpha, bc2, col, jac, rad, r_int, h_out, partials, cfg.zc, lin);
  else
    residual_curvi_kernel<R, NG><<<grid, cfg.block, 0, st>>>(
        g, u, alpha, bc2, col, jac, rad, r_int, h_out, partials, cfg.zc, lin);
}

}  // namespace

template <typename R>
void launch_stage(const Geo &g, int kind, const StageArgs<R> &a,
                  const LaunchCfg &cfg, cudaStream_t st) {
  switch (g.ng) {
    case 2: launch_stage_ng<R, 2>(g, kind, a, cfg, st); break;
    case 4: launch_stage_ng<R, 4>(g, kind, a, cfg, st); break;
    case 5: launch_stage_ng<R, 5>(g, kind, a, cfg, st); break;
    default: break;
  }
}
template <typename R>
cudaError_t launch_stage_steps(const Geo &g, const StageArgs<R> (&sa)[4], int steps,
                               unsigned *count, const LaunchCfg &cfg,
                               cudaStream_t st) {
  StageArgs4<R> s4;
  for (int k = 0; k < 4; k++) s4.s[k] = sa[k];
  if (cfg.variant == 5 && g.ng == 4 && curvi_tma_ok(g, cfg.zc)) {
    cudaError_t e = cudaSuccess;
    if (launch_multi_tma<R, 4>(g, s4, cfg.zc, steps, count, st, &e)) return e;
  }
  switch (g.ng) {
    case 2: return launch_multi_ng<R, 2>(g, s4, steps, count, cfg.pdl, st);
    case 4: return launch_multi_ng<R, 4>(g, s4, steps, count, cfg.pdl, st);
    case 5: return launch_multi_ng<R, 5>(g, s4, steps, count, cfg.pdl, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_stage_steps<double>(const Geo &,
                                                const StageArgs<double> (&)[4], int,
                                                unsigned *, const LaunchCfg &,
                                                cudaStream_t);
template cudaError_t launch_stage_steps<float>(const Geo &,
                                               const StageArgs<float> (&)[4], int,
                                               unsigned *, const LaunchCfg &,
                                               cudaStream_t);

template void launch_stage<double>(const Geo &, int, const StageArgs<double> &,
                                   const LaunchCfg &, cudaStream_t);
template void launch_stage<float>(const Geo &, int, const StageArgs<float> &,
                                  const LaunchCfg &, cudaStream_t);

int residual_blocks(const Geo &g, const LaunchCfg &cfg) {
  return ((g.n0 * g.n1 + cfg.block - 1) / cfg.block) *
         ((g.n2 + cfg.zc - 1) / cfg.zc);
}

template <typename R>
void launch_residual(const Geo &g, const R *u, const R *alpha, const R *bc2,
                     ColumnSet<R> col, const CartCoef &cart, const double *jac,
                     const double *rad, double r_int, double *h_out,
                     double *partials, int *nblocks_out, const LaunchCfg &cfg,
                     cudaStream_t st, int lin) {
  switch (g.ng) {
    case 2: launch_residual_ng<R, 2>(g, u, alpha, bc2, col, cart, jac, rad, r_int, h_out, partials, cfg, st, lin); break;
    case 4: launch_residual_ng<R, 4>(g, u, alpha, bc2, col, cart, jac, rad, r_int, h_out, partials, cfg, st, lin); break;
    case 5: launch_residual_ng<R, 5>(g, u, alpha, bc2, col, cart, jac, rad, r_int, h_out, partials, cfg, st, lin); break;
    default: break;
  }
  if (nblocks_out) *nblocks_out = residual_blocks(g, cfg);
}
template void launch_residual<double>(const Geo &, const double *, const double *,
                                      const double *, ColumnSet<double>,
                                      const CartCoef &, const double *,
                                      const double *, double, double *,
                                      double *, int *, const LaunchCfg &,
                                      cudaStream_t, int);
template void launch_residual<float>(const Geo &, const float *, const float *,
                                     const float *, ColumnSet<float>,
                                     const CartCoef &, const double *,
                                     const double *, double, double *, double *,
                                     int *, const LaunchCfg &, cudaStream_t, int);

void launch_norm_finalize(const double *partials, int nblocks, double *out,
                          cudaStream_t st) {
  norm_finalize_kernel<<<1, 256, 0, st>>>(partials, nblocks, out);
}

template <typename R>
void launch_fill_ghosts(const Geo &g, R *f, cudaStream_t st) {
  if (g.coord == CARTESIAN) return;
  int64_t nb = (g.npts + 255) / 256;
  fill_ghosts_kernel<R><<<(unsigned)nb, 256, 0, st>>>(g, f);
}
template void launch_fill_ghosts<double>(const Geo &, double *, cudaStream_t);
template void launch_fill_ghosts<float>(const Geo &, float *, cudaStream_t);

void launch_convert(const double *src, float *dst, int64_t n, cudaStream_t st) {
  convert_d2f_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}
void launch_convert(const float *src, double *dst, int64_t n, cudaStream_t st) {
  convert_f2d_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}
void launch_dc_prepare(const Geo &g, const double *u, const double *alpha,
                       const double *bc2, const double *ku, const double *kv,
                       float *ac2, float *fu, float *fv, cudaStream_t st) {
  dc_prepare_kernel<<<(unsigned)((g.npts + 255) / 256), 256, 0, st>>>(
      g, u, alpha, bc2, ku, kv, ac2, fu, fv);
}
void launch_dc_update(double *u, double *v, const float *d, const float *w,
                      int64_t n, cudaStream_t st) {
  dc_update_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(u, v, d, w, n);
}

void launch_scale(double *f, double s, int64_t n, cudaStream_t st) {
  scale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, s, n);
}

}  // namespace nrr
