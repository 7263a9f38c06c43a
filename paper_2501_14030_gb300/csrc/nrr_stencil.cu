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
#include <cuda_runtime.h>

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

// Cartesian: uniform spacing, c = 1, every ghost is an outer ghost evolved by
// the radiation condition with d_r f = sum_i (x^i/r) D_i f (one-sided inward
// along directions in which the point lies outside, centred otherwise).
template <typename R, int NG>
__device__ __forceinline__ R cart_radiation(const Geo &g, const R *__restrict__ f,
                                            int i0, int i1, int i2, int64_t p) {
  const int ii[3] = {i0, i1, i2};
  const int nn[3] = {g.n0, g.n1, g.n2};
  const int64_t st[3] = {1, g.s0, (int64_t)g.ncol};
  R x[3], r2 = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    x[d] = R(g.xxmin[d] + (ii[d] - NG + 0.5) * g.dxx[d]);
    r2 = fma(x[d], x[d], r2);
  }
  R rinv = R(1) / sqrt(r2);
  R f0 = ld(f + p);
  R dr = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    R D;
    R inv2 = R(0.5 / g.dxx[d]);
    if (ii[d] >= nn[d] + NG)
      D = (R(3) * f0 - R(4) * ld(f + p - st[d]) + ld(f + p - 2 * st[d])) * inv2;
    else if (ii[d] < NG)
      D = -(R(3) * f0 - R(4) * ld(f + p + st[d]) + ld(f + p + 2 * st[d])) * inv2;
    else
      D = (ld(f + p + st[d]) - ld(f + p - st[d])) * inv2;
    dr = fma(x[d] * rinv, D, dr);
  }
  return -(dr + f0 * rinv);
}

template <typename R, int NG>
__device__ __forceinline__ R cart_operator(const Geo &g, const R *__restrict__ su,
                                           const CartCoef &cc, int64_t p, R u0,
                                           R al, R bc2, int lin) {
  const int64_t st[3] = {1, g.s0, (int64_t)g.ncol};
  R lap = R(cc.cc) * u0;
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int k = 1; k <= NG; k++)
      lap = fma(R(cc.a[d][k - 1]), ld(su + p + k * st[d]) + ld(su + p - k * st[d]),
                lap);
  return add_source(lap, u0, al, bc2, lin);
}

template <typename R, int NG, int KIND>
__global__ void __launch_bounds__(128)
    stage_cart_kernel(Geo g, StageArgs<R> a, int zc) {
  pdl_trigger();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ncol) return;
  pdl_wait();
  const int i0 = e % g.s0, i1 = e / g.s0;
  const int z0 = blockIdx.y * zc;
  const int z1 = min(z0 + zc, g.s2);
  const bool in01 = i0 >= NG && i0 < g.n0 + NG && i1 >= NG && i1 < g.n1 + NG;
  for (int i2 = z0; i2 < z1; i2++) {
    int64_t p = e + (int64_t)g.ncol * i2;
    R ku, kv;
    if (in01 && i2 >= NG && i2 < g.n2 + NG) {
      R u0 = ld(a.su + p), v0 = ld(a.sv + p);
      kv = cart_operator<R, NG>(g, a.su, a.cart, p, u0, ld(a.alpha + p),
                                ld(a.bc2 + p), a.lin);
      ku = fma(-a.eta, u0, v0);
      if (linear_mode<R>(a.lin)) ku += ld(a.fu + p);
    } else {
      ku = cart_radiation<R, NG>(g, a.su, i0, i1, i2, p);
      kv = cart_radiation<R, NG>(g, a.sv, i0, i1, i2, p);
      if (linear_mode<R>(a.lin)) {
        ku += ld(a.fu + p);
        kv += ld(a.bc2 + p);
      }
    }
    stage_epilogue<R, KIND>(a, p, ku, kv);
  }
}

// Residual H at interior points and the block partials of H^2 J, J over
// r < r_int (the volume-weighted L2 norm of Alg. 1's residual).
template <typename R, int NG>
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
    residual_curvi_item<R, NG>(g, su, alpha, bc2, col_set, wt, e, z0,
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
    for (int i2 = z0; i2 < z1; i2++) {
      int64_t p = i0 + (int64_t)g.s0 * (i1 + (int64_t)g.s1 * i2);
      R u0 = ld(su + p);
      double H = (double)cart_operator<R, NG>(g, su, cc, p, u0, ld(alpha + p),
                                              ld(bc2 + p), lin);
      if (h_out) h_out[p] = H;
      double x2 = g.xxmin[2] + (i2 - NG + 0.5) * g.dxx[2];
      double wt = sqrt(x0 * x0 + x1 * x1 + x2 * x2) < r_int ? 1.0 : 0.0;
      num += H * H * wt;
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
  bool evolved = i0 >= g.ng && i1 >= g.ng && i1 < g.n1 + g.ng && i2 >= g.ng &&
                 i2 < g.n2 + g.ng;
  if (evolved) return;
  int j0 = i0, j1 = i1, j2 = i2;
  image_of(g, j0, j1, j2);
  f[p] = f[flat(g, j0, j1, j2)];
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

template <typename R, int NG>
void launch_curvi(const Geo &g, int kind, const StageArgs<R> &a,
                  const LaunchCfg &cfg, cudaStream_t st) {
  const int zc = cfg.zc, pdl = cfg.pdl;
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
    dim3 grid((g.ncol + cfg.block - 1) / cfg.block, (g.s2 + cfg.zc - 1) / cfg.zc);
    dim3 blk(cfg.block);
    switch (kind) {
      case STAGE_FIRST: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_FIRST>, grid, blk, st, cfg.pdl, g, a, cfg.zc); break;
      case STAGE_MID: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_MID>, grid, blk, st, cfg.pdl, g, a, cfg.zc); break;
      case STAGE_LAST: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_LAST>, grid, blk, st, cfg.pdl, g, a, cfg.zc); break;
      default: launch_stage_kernel(stage_cart_kernel<R, NG, STAGE_RAW>, grid, blk, st, cfg.pdl, g, a, cfg.zc); break;
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
