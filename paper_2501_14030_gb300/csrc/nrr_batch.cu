// nrr_batch.cu -- many independent solves of uneven grid sizes relaxed
// together (arXiv 2501.14030, Sec. 5 "multiple, independent patches": N
// grids with no data sharing, there run on several streams).
//
// All solves share one arena per field; a device descriptor per solve holds
// its geometry, time step and field pointers.  Each RK4 stage is one launch
// over the work items of every active solve: a block map assigns each block
// to one solve and a run of its items, so a block never straddles two solves
// and the per-solve residual norms reduce deterministically.  The whole
// relaxation -- initial norm, then chunks of check_every steps with the norm
// and the per-solve stop test -- is one CUDA graph whose loop is a
// conditional WHILE node driven by an on-device control kernel (bounded by a
// chunk limit and a wall-clock limit read from the global timer).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/nrr.h"
#include "nrr_internal.h"
#include "nrr_stencil.cuh"

using namespace nrr;

namespace {

nrr_status bfail(nrr_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define BCUDA(call)                                                        \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      return bfail(NRR_ERR_CUDA, "%s: %s (%s:%d)", #call,                  \
                   cudaGetErrorString(e_), __FILE__, __LINE__);            \
  } while (0)
#define BTRY(expr)                \
  do {                            \
    nrr_status s_ = (expr);       \
    if (s_ != NRR_OK) return s_;  \
  } while (0)

// Everything a batched kernel needs about one solve.
struct SolveDev {
  Geo g;
  double dt, eta;
  // RK4 stage weights a_s dt and b_s dt, computed on the host per relax
  double wa[4], wb[4];
  float wa32[4], wb32[4], eta32;
  double *u, *v;                 // FP64 state
  double *ku, *kv;               // FP64 right-hand side (the defect)
  double *s64[2], *t64[2], *a64[2];  // FP64 stage buffers (FP64 mode)
  double *alpha, *bc2;
  ColumnSet<double> c64;
  float *d, *w;                  // FP32 increment state
  float *s32[2], *t32[2], *a32[2];
  float *ac2, *fu, *fv;          // linearised source and forcing
  ColumnSet<float> c32;
  double *jac, *rad;
  dev::ArenaSrc tf64, tf32;      // tensor maps of the FP64 / FP32 fields
};

// Control block of one relaxation, in device memory.
struct BatchCtl {
  int n;                 // solves
  int active_count;
  long long chunk;       // chunks done
  long long max_chunks;
  unsigned long long t0_ns, timeout_ns;
  int timed_out;
  double tol;
};

// --- RK4 stage arguments of one solve -------------------------------------
// Stage s of classical RK4: k_s at input state (y, s, t, s); accumulate
// b_s dt k_s; next input y + a_{s+1} dt k_s; the last stage writes y.
template <typename R>
__device__ __forceinline__ StageArgs<R> batch_stage_args(const SolveDev &sd,
                                                         int stage, int mode);

template <>
__device__ __forceinline__ StageArgs<double> batch_stage_args<double>(
    const SolveDev &sd, int stage, int mode) {
  StageArgs<double> a{};
  a.alpha = sd.alpha;
  a.bc2 = sd.bc2;
  a.col = sd.c64;
  a.eta = sd.eta;
  a.lin = 0;
  a.fu = nullptr;
  if (mode == 1) {  // the FP64 defect: one RHS evaluation at (u, v)
    a.su = sd.u;
    a.sv = sd.v;
    a.ou = sd.ku;
    a.ov = sd.kv;
    return a;
  }
  a.bu = sd.u;
  a.bv = sd.v;
  a.au = sd.a64[0];
  a.av = sd.a64[1];
  switch (stage) {
    case 0: a.su = sd.u; a.sv = sd.v; a.ou = sd.s64[0]; a.ov = sd.s64[1];
            a.wa = sd.wa[0]; a.wb = sd.wb[0]; break;
    case 1: a.su = sd.s64[0]; a.sv = sd.s64[1]; a.ou = sd.t64[0]; a.ov = sd.t64[1];
            a.wa = sd.wa[1]; a.wb = sd.wb[1]; break;
    case 2: a.su = sd.t64[0]; a.sv = sd.t64[1]; a.ou = sd.s64[0]; a.ov = sd.s64[1];
            a.wa = sd.wa[2]; a.wb = sd.wb[2]; break;
    default: a.su = sd.s64[0]; a.sv = sd.s64[1]; a.ou = sd.u; a.ov = sd.v;
             a.wa = sd.wa[3]; a.wb = sd.wb[3]; break;
  }
  return a;
}

template <>
__device__ __forceinline__ StageArgs<float> batch_stage_args<float>(
    const SolveDev &sd, int stage, int mode) {
  StageArgs<float> a{};
  a.alpha = sd.ac2;
  a.bc2 = sd.fv;
  a.fu = sd.fu;
  a.lin = 1;
  a.col = sd.c32;
  a.eta = sd.eta32;
  a.bu = sd.d;
  a.bv = sd.w;
  a.au = sd.a32[0];
  a.av = sd.a32[1];
  switch (stage) {
    case 0: a.su = sd.d; a.sv = sd.w; a.ou = sd.s32[0]; a.ov = sd.s32[1];
            a.wa = sd.wa32[0]; a.wb = sd.wb32[0]; break;
    case 1: a.su = sd.s32[0]; a.sv = sd.s32[1]; a.ou = sd.t32[0]; a.ov = sd.t32[1];
            a.wa = sd.wa32[1]; a.wb = sd.wb32[1]; break;
    case 2: a.su = sd.t32[0]; a.sv = sd.t32[1]; a.ou = sd.s32[0]; a.ov = sd.s32[1];
            a.wa = sd.wa32[2]; a.wb = sd.wb32[2]; break;
    default: a.su = sd.s32[0]; a.sv = sd.s32[1]; a.ou = sd.d; a.ov = sd.w;
             a.wa = sd.wa32[3]; a.wb = sd.wb32[3]; break;
  }
  (void)mode;
  return a;
}

// --- kernels ----------------------------------------------------------------
constexpr int kTileY = 4;
constexpr int kTmaPZ = 2;  // phi planes per ring slot (tensor-copy variant)
// ring slots per block: two (one slot pair in flight while one is computed);
// a deeper ring takes shared memory that L1 needs (measured slower)
template <typename R>
__host__ __device__ constexpr int tma_slots() { return 2; }
// i1 rows of the outer shell per shell block (NG columns each)
template <int NG>
__host__ __device__ constexpr int shell_rows() { return 32 * kTileY / NG; }

// Stage kernel over all solves: block b works on solve map[b].x, item
// map[b].y of it: first the interior tiles (i0 fastest, then i1, then phi
// chunks), then the outer-shell blocks (shell_rows() rows of i1 each, then
// phi chunks).  VAR 0: planes staged
// through registers (stage_tile_block); VAR 1: planes streamed by tensor
// copies through a ring of shared-memory slots (stage_tma_block; order 8,
// aligned grids), which records an expired copy wait in *err.
template <typename R, int NG, int KIND, int VAR>
__global__ void __launch_bounds__(32 * kTileY, VAR == 1 && sizeof(R) == 4 ? 6 : 1)
    batch_stage_kernel(const SolveDev *__restrict__ sds, const int2 *__restrict__ map,
                       const int *__restrict__ active, int stage, int mode, int zc,
                       int *err) {
  dev::pdl_trigger();
  const int2 bm = map[blockIdx.x];
  if (!active[bm.x]) return;
  const SolveDev &sd = sds[bm.x];
  const Geo g = sd.g;
  const StageArgs<R> a = batch_stage_args<R>(sd, stage, mode);
  const int nx = dev::tiles_x(g), ny = dev::tiles_y<kTileY>(g);
  const int nint = nx * ny * dev::chunks_z(g, zc);
  if (bm.y >= nint) {
    // outer shell: thread = (shell column, row) of shell_rows<NG>() rows
    constexpr int rows = shell_rows<NG>();
    const int nsb = (g.n1 + rows - 1) / rows;
    const int sidx = bm.y - nint, chunk = sidx / nsb;
    const int row = threadIdx.x / NG, lane = threadIdx.x - row * NG;
    const int z0 = NG + chunk * zc;
    if (row < rows)
      dev::stage_shell_rows<R, NG, KIND>(g, a, lane, NG + (sidx % nsb) * rows + row,
                                         z0, min(z0 + zc, NG + g.n2));
    return;
  }
  const int tile_x = bm.y % nx, tile_y = (bm.y / nx) % ny, chunk = bm.y / (nx * ny);
  if constexpr (VAR == 1) {
    __shared__ __align__(128) dev::TmaSlot<R, NG, kTileY, kTmaPZ, sizeof(R) == 4> ring[tma_slots<R>()];
    __shared__ __align__(8) uint64_t full[tma_slots<R>()];
    dev::stage_tma_block<R, NG, KIND, kTileY, tma_slots<R>(), kTmaPZ>(
        g, a, tile_x, tile_y, chunk, zc, sizeof(R) == 4 ? sd.tf32 : sd.tf64, ring,
        full, err);
  } else {
    __shared__ R tile[2][kTileY + 2 * NG][32 + 2 * NG];
    dev::stage_tile_block<R, NG, KIND, kTileY>(g, a, tile_x, tile_y, chunk, zc, tile);
  }
}

// Column variant of the stage kernel (as the single-grid column kernel):
// thread = one (i0, i1) column of evolved points (shell columns last) and ZC
// phi planes; block b covers 32 * kTileY columns of solve map[b].x, chunk
// map[b].y.  ZC is a template parameter and the register budget is capped
// (several blocks per SM), so that the FP64 pipe sees as many warps as in the
// single-grid kernel.
template <typename R, int NG, int KIND, int ZC>
__global__ void __launch_bounds__(32 * kTileY, ZC == 4 ? 4 : 6)
    batch_col_kernel(const SolveDev *__restrict__ sds, const int2 *__restrict__ map,
                     const int *__restrict__ active, int stage, int mode) {
  dev::pdl_trigger();
  const int2 bm = map[blockIdx.x];
  if (!active[bm.x]) return;
  const SolveDev &sd = sds[bm.x];
  const Geo g = sd.g;
  const StageArgs<R> a = batch_stage_args<R>(sd, stage, mode);
  const int ncols = (g.n0 + NG) * g.n1, ncb = (ncols + 32 * kTileY - 1) / (32 * kTileY);
  const int e = (bm.y % ncb) * 32 * kTileY + threadIdx.x;
  if (e >= ncols) return;
  dev::stage_curvi_item<R, NG, KIND, ZC>(g, a, e, NG + (bm.y / ncb) * ZC);
}

// FP64 residual partial sums over all solves (2 phi planes per item).
template <int NG>
__global__ void __launch_bounds__(128)
    batch_residual_kernel(const SolveDev *__restrict__ sds,
                          const int2 *__restrict__ map,
                          const int *__restrict__ active, double r_int,
                          double *partials) {
  const int2 bm = map[blockIdx.x];
  double num = 0.0, den = 0.0;
  if (active[bm.x]) {
    const SolveDev &sd = sds[bm.x];
    const Geo g = sd.g;
    const int ncols = g.n0 * g.n1;
    const int item = bm.y + threadIdx.x;
    if (item < ncols * ((g.n2 + 1) / 2)) {
      const int e = item % ncols;
      const int col = (e % g.n0 + NG) + g.s0 * (e / g.n0 + NG);
      const double wt = sd.rad[col] < r_int ? sd.jac[col] : 0.0;
      const int z0 = NG + (item / ncols) * 2;
      dev::residual_curvi_item<double, NG>(g, sd.u, sd.alpha, sd.bc2, sd.c64,
                                           wt, e, z0, min(z0 + 2, NG + g.n2),
                                           0, nullptr, num, den);
    }
  }
  dev::block_sum2(num, den, partials + 2 * blockIdx.x);
}

// Per-solve norm (one block per solve, fixed order) and the stop test.
__global__ void batch_finalize_kernel(const int2 *__restrict__ ranges,
                                      const double *__restrict__ partials,
                                      int *active, double *norms,
                                      long long *steps, BatchCtl *ctl,
                                      int check_every, int in_body) {
  const int s = blockIdx.x;
  double x = 0.0, y = 0.0;
  const int2 rg = ranges[s];
  if (active[s])
    for (int i = threadIdx.x; i < rg.y; i += blockDim.x) {
      x += partials[2 * (rg.x + i)];
      y += partials[2 * (rg.x + i) + 1];
    }
  __shared__ double res[2];
  dev::block_sum2(x, y, res);
  __syncthreads();
  if (threadIdx.x == 0 && active[s]) {
    double nrm = res[1] > 0.0 ? sqrt(res[0] / res[1]) : 0.0;
    norms[s] = nrm;
    // in the loop body the chunk counter still excludes the chunk just done
    steps[s] = (ctl->chunk + in_body) * (long long)check_every;
    if (!(nrm >= ctl->tol)) active[s] = 0;  // converged, or not finite
  }
}

// Counts active solves, advances the chunk counter and decides whether the
// WHILE body runs again.
__global__ void batch_control_kernel(const int *active, BatchCtl *ctl,
                                     cudaGraphConditionalHandle handle,
                                     int first) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int i = threadIdx.x; i < ctl->n; i += blockDim.x) c += active[i] != 0;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (first) {
      ctl->t0_ns = now;
      ctl->chunk = 0;
      ctl->timed_out = 0;
    } else {
      ctl->chunk += 1;
    }
    ctl->active_count = cnt;
    bool go = cnt > 0 && ctl->chunk < ctl->max_chunks;
    if (go && ctl->timeout_ns > 0 && now - ctl->t0_ns > ctl->timeout_ns) {
      ctl->timed_out = 1;
      go = false;
    }
    cudaGraphSetConditional(handle, go ? 1u : 0u);
  }
}

// Defect-correction set-up over all points of active solves (256 per block):
// linearised source, forcing from the FP64 RHS, increments from rest.
__global__ void batch_prepare_kernel(const SolveDev *__restrict__ sds,
                                     const int2 *__restrict__ map,
                                     const int *__restrict__ active) {
  const int2 bm = map[blockIdx.x];
  if (!active[bm.x]) return;
  const SolveDev &sd = sds[bm.x];
  const int64_t p = (int64_t)bm.y + threadIdx.x;
  if (p >= sd.g.npts) return;
  double t = 1.0 / (1.0 + sd.alpha[p] * sd.u[p]);
  double t2 = t * t, t4 = t2 * t2;
  sd.ac2[p] = (float)(7.0 * sd.alpha[p] * sd.bc2[p] * (t4 * t4));
  sd.fu[p] = (float)sd.ku[p];
  sd.fv[p] = (float)sd.kv[p];
  sd.d[p] = 0.f;
  sd.w[p] = 0.f;
}

__global__ void batch_update_kernel(const SolveDev *__restrict__ sds,
                                    const int2 *__restrict__ map,
                                    const int *__restrict__ active) {
  const int2 bm = map[blockIdx.x];
  if (!active[bm.x]) return;
  const SolveDev &sd = sds[bm.x];
  const int64_t p = (int64_t)bm.y + threadIdx.x;
  if (p >= sd.g.npts) return;
  sd.u[p] += (double)sd.d[p];
  sd.v[p] += (double)sd.w[p];
}

// dst[s][interior point] = (float) u of solve s (all solves of one size).
__global__ void batch_interior_kernel(const SolveDev *__restrict__ sds, int n,
                                      int64_t per, float *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * per) return;
  const int s = (int)(i / per);
  const int64_t q = i % per;
  const Geo g = sds[s].g;
  const int i0 = (int)(q % g.n0), i1 = (int)((q / g.n0) % g.n1),
            i2 = (int)(q / ((int64_t)g.n0 * g.n1));
  dst[i] = (float)sds[s].u[flat(g, i0 + g.ng, i1 + g.ng, i2 + g.ng)];
}

// v = eta u for every point of every solve (warm starts).
__global__ void batch_warm_v_kernel(const SolveDev *__restrict__ sds,
                                    const int2 *__restrict__ map) {
  const int2 bm = map[blockIdx.x];
  const SolveDev &sd = sds[bm.x];
  const int64_t p = (int64_t)bm.y + threadIdx.x;
  if (p >= sd.g.npts) return;
  sd.v[p] = sd.eta * sd.u[p];
}

__global__ void batch_zero_kernel(const SolveDev *__restrict__ sds,
                                  const int2 *__restrict__ map) {
  const int2 bm = map[blockIdx.x];
  const SolveDev &sd = sds[bm.x];
  const int64_t p = (int64_t)bm.y + threadIdx.x;
  if (p >= sd.g.npts) return;
  sd.u[p] = 0.0;
  sd.v[p] = 0.0;
}

}  // namespace

struct nrr_batch {
  int n = 0;
  int ng = 0;
  int with_fp64 = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t user_stream = nullptr;
  cudaEvent_t order_ev = nullptr;
  std::vector<Geo> geos;
  std::vector<SolveDev> host_sd;
  std::vector<void *> allocs;
  SolveDev *d_sd = nullptr;
  int *d_active = nullptr;
  double *d_norms = nullptr;
  long long *d_steps = nullptr;
  BatchCtl *d_ctl = nullptr;
  double *d_partials = nullptr;
  int2 *d_map_res = nullptr, *d_res_ranges = nullptr, *d_map_pts = nullptr;
  int nblk_res = 0, nblk_pts = 0;
  int2 *d_map_stage[5] = {};
  int nblk_stage[5] = {};
  int2 *d_map_col[3] = {};  // column variant, zc = 1, 2, 4
  int nblk_col[3] = {};
  int zc[2] = {1, 4};  // phi planes per block chunk: [0] FP64, [1] FP32
  // stage kernel: 0 register-staged tiles, 1 tensor-copy tiles, 2 columns
  // (FP32: 1 with zc 16 where the batch allows it, set at creation)
  int variant[2] = {2, 0};
  int tma_ok = 0;           // every solve meets the tensor-copy variant's shape
  int *d_err = nullptr;     // set by a stage kernel whose copy wait expired
  CUtensorMap *d_maps = nullptr;  // per solve: u / operand maps, FP32 then FP64
  int64_t total_points = 0, interior_points = 0;
  // relaxation graph and its key
  cudaGraphExec_t exec = nullptr;
  int g_mode = -1, g_every = 0, g_zc64 = 0, g_zc32 = 0, g_var64 = 0, g_var32 = 0;
  double g_r_int = 0.0;
};

namespace {

// Classical RK4 weights of one solve: stage offsets a = (1/2, 1/2, 1, 0) and
// update weights b = (1/6, 1/3, 1/3, 1/6), times dt.
void set_stage_weights(SolveDev &sd) {
  const double dt = sd.dt;
  const double wa[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double wb[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  for (int k = 0; k < 4; k++) {
    sd.wa[k] = wa[k];
    sd.wb[k] = wb[k];
    sd.wa32[k] = (float)wa[k];
    sd.wb32[k] = (float)wb[k];
  }
  sd.eta32 = (float)sd.eta;
}

template <typename T>
nrr_status balloc(nrr_batch *b, T **p, size_t count) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess)
    return bfail(NRR_ERR_OOM, "cudaMalloc of %zu bytes: %s", count * sizeof(T),
                 cudaGetErrorString(e));
  b->allocs.push_back(ptr);
  dbg_register(ptr, std::max<size_t>(count, 1) * sizeof(T));
  *p = static_cast<T *>(ptr);
  return NRR_OK;
}


// Block map over `per_solve(s)` items of every solve, `bs` items per block;
// ranges[s] = (first block of s, its block count).
template <typename F>
nrr_status build_map(nrr_batch *b, int bs, F per_solve, int2 **d_map, int *nblk,
                     int2 **d_ranges) {
  std::vector<int2> map, ranges;
  for (int s = 0; s < b->n; s++) {
    int64_t items = per_solve(b->geos[s]);
    int first = (int)map.size();
    for (int64_t i = 0; i < items; i += bs) map.push_back(make_int2(s, (int)i));
    ranges.push_back(make_int2(first, (int)map.size() - first));
  }
  BTRY(balloc(b, d_map, map.size()));
  BCUDA(cudaMemcpy(*d_map, map.data(), map.size() * sizeof(int2),
                   cudaMemcpyHostToDevice));
  *nblk = (int)map.size();
  if (d_ranges) {
    BTRY(balloc(b, d_ranges, ranges.size()));
    BCUDA(cudaMemcpy(*d_ranges, ranges.data(), ranges.size() * sizeof(int2),
                     cudaMemcpyHostToDevice));
  }
  return NRR_OK;
}

int zc_index(int zc) {  // planes per chunk 1, 2, 4, 8, 16 -> slots 0..4
  return zc <= 1 ? 0 : zc == 2 ? 1 : zc == 4 ? 2 : zc == 8 ? 3 : 4;
}

nrr_status stage_map(nrr_batch *b, int zc) {
  if (b->d_map_stage[zc_index(zc)]) return NRR_OK;
  const int ng = b->ng;
  return build_map(
      b, 1,
      [zc, ng](const Geo &g) {
        const int rows = ng == 2 ? shell_rows<2>() : ng == 5 ? shell_rows<5>()
                                                           : shell_rows<4>();
        return ((int64_t)dev::tiles_x(g) * dev::tiles_y<kTileY>(g) +
                (g.n1 + rows - 1) / rows) *
               dev::chunks_z(g, zc);
      },
      &b->d_map_stage[zc_index(zc)], &b->nblk_stage[zc_index(zc)], nullptr);
}

int col_index(int zc) { return zc <= 1 ? 0 : zc == 2 ? 1 : 2; }

nrr_status col_map(nrr_batch *b, int zc) {
  if (b->d_map_col[col_index(zc)]) return NRR_OK;
  const int ng = b->ng;
  return build_map(
      b, 1,
      [zc, ng](const Geo &g) {
        const int64_t ncols = (int64_t)(g.n0 + ng) * g.n1;
        return ((ncols + 32 * kTileY - 1) / (32 * kTileY)) * ((g.n2 + zc - 1) / zc);
      },
      &b->d_map_col[col_index(zc)], &b->nblk_col[col_index(zc)], nullptr);
}

// The launch map of the stage kernel for (variant, zc).
nrr_status stage_map_for(nrr_batch *b, int variant, int zc) {
  return variant == 2 ? col_map(b, zc) : stage_map(b, zc);
}

// Stage kernels go with programmatic dependent launch: a stage's blocks
// start while the previous kernel drains, and wait (griddepcontrol.wait, in
// the stage's device code) before they read anything a kernel of the solve
// writes.  What a stage reads before that -- its block map, the solves'
// descriptors and weights, and the active flags -- no kernel launched
// between two finalize kernels changes, and the kernels that precede a
// chunk's first stage are launched without the attribute, so the finalize
// kernel has completed.
template <typename... P, typename... A>
void launch_pdl(void (*k)(P...), unsigned blocks, cudaStream_t st, A... args) {
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3(blocks);
  c.blockDim = dim3(32 * kTileY);
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = at;
  c.numAttrs = 1;
  cudaLaunchKernelEx(&c, k, args...);
}

template <typename R, int NG, int KIND>
void launch_bstage_kind(nrr_batch *b, int zc, int stage, int mode,
                        cudaStream_t st) {
  if (b->variant[sizeof(R) == 4] == 2) {
    const int nb = b->nblk_col[col_index(zc)];
    const int2 *map = b->d_map_col[col_index(zc)];
    const SolveDev *sds = b->d_sd;
    const int *act = b->d_active;
    if (zc <= 1)
      launch_pdl(batch_col_kernel<R, NG, KIND, 1>, nb, st, sds, map, act, stage, mode);
    else if (zc == 2)
      launch_pdl(batch_col_kernel<R, NG, KIND, 2>, nb, st, sds, map, act, stage, mode);
    else
      launch_pdl(batch_col_kernel<R, NG, KIND, 4>, nb, st, sds, map, act, stage, mode);
    return;
  }
  const int2 *map = b->d_map_stage[zc_index(zc)];
  const int nb = b->nblk_stage[zc_index(zc)];
  const SolveDev *sds = b->d_sd;
  const int *act = b->d_active;
  if constexpr (NG == 4) {
    if (b->variant[sizeof(R) == 4] == 1) {
      launch_pdl(batch_stage_kernel<R, NG, KIND, 1>, nb, st, sds, map, act, stage, mode,
                 zc, b->d_err);
      return;
    }
  }
  launch_pdl(batch_stage_kernel<R, NG, KIND, 0>, nb, st, sds, map, act, stage, mode, zc,
             b->d_err);
}

template <typename R, int NG>
void launch_bstage_ng(nrr_batch *b, int zc, int stage, int mode,
                      cudaStream_t st) {
  if (mode == 1) {
    launch_bstage_kind<R, NG, STAGE_RAW>(b, zc, 0, mode, st);
    return;
  }
  switch (stage) {
    case 0: launch_bstage_kind<R, NG, STAGE_FIRST>(b, zc, 0, mode, st); break;
    case 3: launch_bstage_kind<R, NG, STAGE_LAST>(b, zc, 3, mode, st); break;
    default: launch_bstage_kind<R, NG, STAGE_MID>(b, zc, stage, mode, st); break;
  }
}

// One batched stage (mode 0) or the FP64 defect evaluation (mode 1).
template <typename R>
void launch_bstage(nrr_batch *b, int stage, int mode, cudaStream_t st) {
  const int zc = b->zc[sizeof(R) == 4];
  switch (b->ng) {
    case 2: launch_bstage_ng<R, 2>(b, zc, stage, mode, st); break;
    case 5: launch_bstage_ng<R, 5>(b, zc, stage, mode, st); break;
    default: launch_bstage_ng<R, 4>(b, zc, stage, mode, st); break;
  }
}

void launch_bresidual(nrr_batch *b, double r_int, cudaStream_t st) {
  switch (b->ng) {
    case 2: batch_residual_kernel<2><<<b->nblk_res, 128, 0, st>>>(b->d_sd, b->d_map_res, b->d_active, r_int, b->d_partials); break;
    case 5: batch_residual_kernel<5><<<b->nblk_res, 128, 0, st>>>(b->d_sd, b->d_map_res, b->d_active, r_int, b->d_partials); break;
    default: batch_residual_kernel<4><<<b->nblk_res, 128, 0, st>>>(b->d_sd, b->d_map_res, b->d_active, r_int, b->d_partials); break;
  }
}

// Body of one chunk: `every` RK4 steps (FP64) or one defect-correction outer
// iteration of `every` FP32 steps, then the FP64 norms and the stop test.
void launch_chunk(nrr_batch *b, int mode, int every, double r_int,
                  cudaGraphConditionalHandle h, cudaStream_t st) {
  if (mode == NRR_FP32_DC) {
    launch_bstage<double>(b, 0, 1, st);  // FP64 defect
    batch_prepare_kernel<<<b->nblk_pts, 256, 0, st>>>(b->d_sd, b->d_map_pts, b->d_active);
    for (int s = 0; s < every; s++)
      for (int k = 0; k < 4; k++) launch_bstage<float>(b, k, 0, st);
    batch_update_kernel<<<b->nblk_pts, 256, 0, st>>>(b->d_sd, b->d_map_pts, b->d_active);
  } else {
    for (int s = 0; s < every; s++)
      for (int k = 0; k < 4; k++) launch_bstage<double>(b, k, 0, st);
  }
  launch_bresidual(b, r_int, st);
  batch_finalize_kernel<<<b->n, 256, 0, st>>>(b->d_res_ranges, b->d_partials,
                                             b->d_active, b->d_norms,
                                             b->d_steps, b->d_ctl, every, 1);
  batch_control_kernel<<<1, 256, 0, st>>>(b->d_active, b->d_ctl, h, 0);
}

nrr_status build_relax_graph(nrr_batch *b, int mode, int every, double r_int) {
  if (b->exec && b->g_mode == mode && b->g_every == every &&
      b->g_r_int == r_int && b->g_zc64 == b->zc[0] && b->g_zc32 == b->zc[1] &&
      b->g_var64 == b->variant[0] && b->g_var32 == b->variant[1])
    return NRR_OK;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BTRY(stage_map_for(b, b->variant[0], b->zc[0]));
  BTRY(stage_map_for(b, b->variant[1], b->zc[1]));
  cudaGraph_t graph;
  BCUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  BCUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1,
                                         cudaGraphCondAssignDefault));
  // prologue: norms of the initial state and the first stop test
  BCUDA(cudaStreamBeginCaptureToGraph(b->stream, graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
  launch_bresidual(b, r_int, b->stream);
  batch_finalize_kernel<<<b->n, 256, 0, b->stream>>>(
      b->d_res_ranges, b->d_partials, b->d_active, b->d_norms, b->d_steps,
      b->d_ctl, every, 0);
  batch_control_kernel<<<1, 256, 0, b->stream>>>(b->d_active, b->d_ctl, handle, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return bfail(NRR_ERR_CUDA, "prologue capture: %s", cudaGetErrorString(e));
  }
  // the WHILE node after the prologue's sink nodes
  size_t nn = 0;
  BCUDA(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  BCUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
  std::vector<cudaGraphNode_t> sinks;
  for (auto nd : nodes) {
    size_t nout = 0;
    BCUDA(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout));
    if (nout == 0) sinks.push_back(nd);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  BCUDA(cudaGraphAddNode(&wnode, graph, sinks.data(), nullptr, sinks.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  BCUDA(cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
  launch_chunk(b, mode, every, r_int, handle, b->stream);
  e = cudaStreamEndCapture(b->stream, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return bfail(NRR_ERR_CUDA, "body capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return bfail(NRR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  b->g_mode = mode;
  b->g_every = every;
  b->g_r_int = r_int;
  b->g_zc64 = b->zc[0];
  b->g_zc32 = b->zc[1];
  b->g_var64 = b->variant[0];
  b->g_var32 = b->variant[1];
  return NRR_OK;
}

using TensorMapEncodeFn = CUresult (*)(
    CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
    CUtensorMapFloatOOBfill);

// 4-D tensor map (i0, i1, i2, field) over the fields of one solve: `base` is
// its field 0, consecutive fields `stride` elements apart; boxes of
// box0 x box1 x box2 points of one field.
bool encode_field_map(CUtensorMap *m, const void *base, const Geo &g,
                      int nfields, int64_t stride, int esize, int box0, int box1,
                      int box2) {
  auto enc = reinterpret_cast<TensorMapEncodeFn>(tensor_map_encoder());
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.s0, (cuuint64_t)g.s1, (cuuint64_t)g.s2,
                              (cuuint64_t)nfields};
  const cuuint64_t strides[3] = {(cuuint64_t)g.s0 * esize,
                                 (cuuint64_t)g.ncol * esize,
                                 (cuuint64_t)stride * esize};
  const cuuint32_t box[4] = {(cuuint32_t)box0, (cuuint32_t)box1, (cuuint32_t)box2, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
             4, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

nrr_status bbegin(nrr_batch *b) {
  BCUDA(cudaSetDevice(b->device));
  BCUDA(cudaEventRecord(b->order_ev, b->user_stream));
  BCUDA(cudaStreamWaitEvent(b->stream, b->order_ev, 0));
  return NRR_OK;
}

}  // namespace

extern "C" {

nrr_status nrr_batch_create(int n, const nrr_grid_desc *descs,
                            const int *npunct, const nrr_puncture *const *punct,
                            int flags, void *stream, nrr_batch **out) {
  if (!out) return bfail(NRR_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (n < 1 || !descs || !npunct || !punct)
    return bfail(NRR_ERR_INVALID_ARG, "need n >= 1 solves with descriptors and punctures");
  const int order = descs[0].fd_order;
  int64_t total = 0, nint = 0;
  size_t bytes = 0;
  for (int s = 0; s < n; s++) {
    const nrr_grid_desc &d = descs[s];
    {
      nrr_status st = check_grid_desc(&d);
      if (st != NRR_OK) return st;
    }
    if (d.coord != NRR_SINHSYMTP && d.coord != NRR_SPHERICAL &&
        d.coord != NRR_SINHSPHERICAL)
      return bfail(NRR_ERR_INVALID_ARG,
                   "solve %d: batches take SinhSymTP, Spherical or SinhSpherical grids", s);
    if (d.fd_order != order || (order != 4 && order != 8 && order != 10))
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: one FD order (4, 8 or 10) per batch", s);
    int ng = order / 2;
    if (d.n[0] < ng || d.n[1] < ng || d.n[2] < 2 || (d.n[2] & 1) ||
        d.n[0] > 4096 || d.n[1] > 4096 || d.n[2] > 4096)
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: bad grid size", s);
    if (d.coord == NRR_SINHSYMTP && !(d.amax > 0 && d.sinhwaa > 0 && d.bscale >= 0))
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: bad SinhSymTP parameters", s);
    if (d.coord == NRR_SPHERICAL && !(d.rmax > 0))
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: bad rmax", s);
    if (d.coord == NRR_SINHSPHERICAL && !(d.amax > 0 && d.sinhwaa > 0))
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: bad SinhSpherical parameters", s);
    if (npunct[s] < 1 || npunct[s] > 8 || !punct[s])
      return bfail(NRR_ERR_INVALID_ARG, "solve %d: need 1..8 punctures", s);
    for (int a = 0; a < npunct[s]; a++)
      if (!(punct[s][a].m > 0.0))
        return bfail(NRR_ERR_INVALID_ARG, "solve %d: puncture mass must be positive", s);
    Geo g = grid_geo(&d);
    total += g.npts;
    nint += (int64_t)g.n0 * g.n1 * g.n2;
    size_t per = (flags & 1) ? (12 * 8 + 11 * 4) : (6 * 8 + 11 * 4);
    bytes += (size_t)g.npts * per + (size_t)g.ncol * (12 * (5 * ng + 1 + 4) + 64);
  }
  if (total > ((int64_t)1 << 31))
    return bfail(NRR_ERR_INVALID_ARG, "batch exceeds 2^31 points");
  int dev = 0;
  BCUDA(cudaGetDevice(&dev));
  size_t free_b = 0, total_b = 0;
  BCUDA(cudaMemGetInfo(&free_b, &total_b));
  if (bytes + (size_t)(512u << 20) > free_b)
    return bfail(NRR_ERR_OOM, "batch needs %zu bytes, %zu free", bytes, free_b);

  nrr_batch *b = new (std::nothrow) nrr_batch();
  if (!b) return bfail(NRR_ERR_OOM, "host allocation failed");
  b->n = n;
  b->ng = order / 2;
  b->with_fp64 = flags & 1;
  b->device = dev;
  b->user_stream = static_cast<cudaStream_t>(stream);
  b->total_points = total;
  b->interior_points = nint;
  nrr_status st = [&]() -> nrr_status {
    BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BCUDA(cudaEventCreateWithFlags(&b->order_ev, cudaEventDisableTiming));
    BTRY(bbegin(b));
    const int ng = b->ng, nco = ncoef(ng);
    // arenas
    int64_t ctot = 0;
    for (int s = 0; s < n; s++) {
      b->geos.push_back(grid_geo(&descs[s]));
      ctot += b->geos[s].ncol;
    }
    const int n64 = b->with_fp64 ? 12 : 6;
    double *a64 = nullptr, *col64 = nullptr;
    float *a32 = nullptr, *col32 = nullptr;
    BTRY(balloc(b, &a64, (size_t)n64 * total));
    BTRY(balloc(b, &a32, (size_t)11 * total));
    BTRY(balloc(b, &col64, (size_t)(nco + 4 + 3 + 2 + 1 + 1 + 1 + 1) * ctot));
    BTRY(balloc(b, &col32, (size_t)(nco + 4) * ctot));
    BCUDA(cudaMemsetAsync(a64, 0, (size_t)n64 * total * 8, b->stream));
    BCUDA(cudaMemsetAsync(a32, 0, (size_t)11 * total * 4, b->stream));
    double *scal = nullptr;
    BTRY(balloc(b, &scal, (size_t)n));
    int *bad = nullptr;
    BTRY(balloc(b, &bad, 1));
    BCUDA(cudaMemsetAsync(bad, 0, sizeof(int), b->stream));
    int64_t off = 0;
    const int m = ng;
    double w1[7] = {0}, w2[7] = {0};
    for (int k = 0; k <= m; k++) {
      w1[k] = k == 0 ? 0.0 : fd_first(m, k);
      w2[k] = fd_second(m, k);
    }
    for (int s = 0; s < n; s++) {
      const Geo &g = b->geos[s];
      SolveDev sd{};
      sd.g = g;
      const int64_t np = g.npts;
      double *f64[12];
      for (int k = 0; k < n64; k++) f64[k] = a64 + (size_t)k * total + off;
      float *f32[11];
      for (int k = 0; k < 11; k++) f32[k] = a32 + (size_t)k * total + off;
      sd.u = f64[0]; sd.v = f64[1]; sd.ku = f64[2]; sd.kv = f64[3];
      sd.alpha = f64[4]; sd.bc2 = f64[5];
      if (b->with_fp64) {
        sd.s64[0] = f64[6]; sd.s64[1] = f64[7]; sd.t64[0] = f64[8];
        sd.t64[1] = f64[9]; sd.a64[0] = f64[10]; sd.a64[1] = f64[11];
      }
      sd.d = f32[0]; sd.w = f32[1];
      sd.s32[0] = f32[2]; sd.s32[1] = f32[3]; sd.t32[0] = f32[4];
      sd.t32[1] = f32[5]; sd.a32[0] = f32[6]; sd.a32[1] = f32[7];
      sd.ac2 = f32[8]; sd.fu = f32[9]; sd.fv = f32[10];
      b->host_sd.push_back(sd);
      off += np;
    }
    // Column arrays: one contiguous slab per solve in the [j][ncol] layout
    // of a single grid.
    {
      int64_t cur64 = 0, cur32 = 0;
      for (int s = 0; s < n; s++) {
        const Geo &g = b->geos[s];
        SolveDev &sd = b->host_sd[s];
        const int64_t nc = g.ncol;
        double *p = col64 + cur64;
        sd.c64.coef = p; p += (size_t)nco * nc;
        sd.c64.somm = p; p += 3 * nc;
        sd.c64.c2inv = p; p += nc;
        double *h = p; p += 3 * nc;
        double *gl = p; p += 2 * nc;
        sd.rad = p; p += nc;
        double *drdxx0 = p; p += nc;
        sd.jac = p; p += nc;
        double *dsmin = p; p += nc;
        cur64 = p - col64;
        float *q = col32 + cur32;
        sd.c32.coef = q; q += (size_t)nco * nc;
        sd.c32.somm = q; q += 3 * nc;
        sd.c32.c2inv = q; q += nc;
        cur32 = q - col32;
        launch_column_geometry(g, h, gl, sd.rad, drdxx0, sd.jac, dsmin, b->stream);
        launch_min_interior(g, dsmin, scal + s, b->stream);
        launch_column_coefs(g, h, gl, sd.rad, drdxx0, dsmin, scal + s, w1, w2,
                            sd.c64, sd.c32, b->stream);
        PunctureSet ps{};
        ps.n = npunct[s];
        for (int a = 0; a < npunct[s]; a++) {
          ps.p[a].m = punct[s][a].m;
          for (int k = 0; k < 3; k++) {
            ps.p[a].x[k] = punct[s][a].x[k];
            ps.p[a].P[k] = punct[s][a].P[k];
            ps.p[a].S[k] = punct[s][a].S[k];
          }
        }
        // FP32 copies of the source are not used by a batch: the FP32
        // forcing slots serve as their scratch.
        launch_source(g, ps, dsmin, scal + s, sd.alpha, sd.bc2, sd.fu, sd.fv,
                      bad, b->stream);
      }
      BCUDA(cudaGetLastError());
    }
    std::vector<double> dsg(n);
    int hbad = 0;
    BCUDA(cudaMemcpyAsync(dsg.data(), scal, n * sizeof(double),
                          cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    if (hbad) return bfail(NRR_ERR_INVALID_ARG, "a puncture lies on a grid point");
    for (int s = 0; s < n; s++) {
      if (!(dsg[s] > 0.0) || !std::isfinite(dsg[s]))
        return bfail(NRR_ERR_INVALID_ARG, "solve %d: degenerate spacing", s);
      b->host_sd[s].dt = 0.5 * dsg[s];  // CFL 0.5; nrr_batch_relax rescales
      b->host_sd[s].eta = 0.0;
    }
    BTRY(balloc(b, &b->d_sd, (size_t)n));
    BTRY(balloc(b, &b->d_active, (size_t)n));
    BTRY(balloc(b, &b->d_err, 1));
    BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
    // Tensor-copy stage variant: order 8, whole 32-wide tiles in i0 and 4-row
    // tiles in i1, and rows / field bases on 16-byte boundaries in both
    // precisions (s0 and every solve's offset multiples of 4 elements).
    b->tma_ok = ng == 4;
    for (int s = 0; s < n; s++) {
      const Geo &g = b->geos[s];
      if (g.n0 % 32 || g.n1 % kTileY || g.s0 % 4 || g.npts % 4) b->tma_ok = 0;
    }
    if (b->tma_ok) {
      std::vector<CUtensorMap> maps(4 * (size_t)n);
      BTRY(balloc(b, &b->d_maps, maps.size()));
      for (int s = 0; s < n && b->tma_ok; s++) {
        const Geo &g = b->geos[s];
        SolveDev &sd = b->host_sd[s];
        const int tw = 32 + 2 * ng, th = kTileY + 2 * ng;
        const int pz = kTmaPZ;
        bool ok = encode_field_map(&maps[4 * s + 0], sd.d, g, 11, total, 4, tw, th, pz) &&
                  encode_field_map(&maps[4 * s + 1], sd.d, g, 11, total, 4, 32, kTileY, pz) &&
                  encode_field_map(&maps[4 * s + 2], sd.u, g, n64, total, 8, tw, th, pz) &&
                  encode_field_map(&maps[4 * s + 3], sd.u, g, n64, total, 8, 32, kTileY, pz);
        if (!ok) {
          b->tma_ok = 0;
          break;
        }
        sd.tf32 = {b->d_maps + 4 * s + 0, b->d_maps + 4 * s + 1, sd.d, total};
        sd.tf64 = {b->d_maps + 4 * s + 2, b->d_maps + 4 * s + 3, sd.u, total};
      }
      if (b->tma_ok)
        BCUDA(cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                         cudaMemcpyHostToDevice));
    }
    // FP32 stages: the tensor-copy tiles over 16-plane chunks where every
    // solve allows them (the autotuner's choice on SinhSymTP batches of
    // 64x32x8 to 128x128x16; about half the time of the register-staged
    // tiles), else register-staged tiles over 4-plane chunks
    if (b->tma_ok) {
      b->variant[1] = 1;
      b->zc[1] = 16;
    }
    BTRY(balloc(b, &b->d_norms, (size_t)n));
    BTRY(balloc(b, &b->d_steps, (size_t)n));
    BTRY(balloc(b, &b->d_ctl, 1));
    BTRY(build_map(b, 128,
                   [ng](const Geo &g) { return (int64_t)g.n0 * g.n1 * ((g.n2 + 1) / 2); },
                   &b->d_map_res, &b->nblk_res, &b->d_res_ranges));
    BTRY(balloc(b, &b->d_partials, 2 * (size_t)b->nblk_res));
    BTRY(build_map(b, 256, [](const Geo &g) { return g.npts; }, &b->d_map_pts,
                   &b->nblk_pts, nullptr));
    // store the spacing for dt in the descriptor's dt slot (CFL applied later)
    for (int s = 0; s < n; s++) b->host_sd[s].dt = dsg[s];
    return NRR_OK;
  }();
  if (st != NRR_OK) {
    std::string msg = nrr_last_error();
    nrr_batch_destroy(b);
    set_last_error(msg.c_str());
    return st;
  }
  *out = b;
  return NRR_OK;
}

nrr_status nrr_batch_destroy(nrr_batch *b) {
  if (!b) return NRR_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (void *p : b->allocs) {
    dbg_unregister(p);
    cudaFree(p);
  }
  if (b->order_ev) cudaEventDestroy(b->order_ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return NRR_OK;
}

nrr_status nrr_batch_info(const nrr_batch *b, int64_t *total_points,
                          int64_t *interior_points) {
  if (!b) return bfail(NRR_ERR_INVALID_ARG, "null batch");
  if (total_points) *total_points = b->total_points;
  if (interior_points) *interior_points = b->interior_points;
  return NRR_OK;
}

nrr_status nrr_batch_relax(nrr_batch *b, const nrr_relax_opts *o,
                           nrr_relax_result *per_solve,
                           nrr_relax_result *total) {
  if (!b || !o) return bfail(NRR_ERR_INVALID_ARG, "null argument");
  if (o->mode != NRR_FP64 && o->mode != NRR_FP32_DC)
    return bfail(NRR_ERR_INVALID_ARG, "batches relax in NRR_FP64 or NRR_FP32_DC");
  if (o->mode == NRR_FP64 && !b->with_fp64)
    return bfail(NRR_ERR_INVALID_ARG, "batch created without FP64 stage buffers");
  if (!(o->tol > 0.0) || o->check_every < 1 || o->max_iters < 0 ||
      !(o->cfl > 0.0) || !(o->r_int > 0.0))
    return bfail(NRR_ERR_INVALID_ARG, "invalid relax options");
  if (o->initial != NRR_INIT_ZERO && o->initial != NRR_INIT_CURRENT &&
      o->initial != NRR_INIT_DEVICE)
    return bfail(NRR_ERR_INVALID_ARG,
                 "batches start from zero, the current state or set u (v = eta u)");
  auto t0 = std::chrono::steady_clock::now();
  BTRY(bbegin(b));
  const int every = (int)(o->mode == NRR_FP32_DC && o->inner_steps > 0
                              ? o->inner_steps : o->check_every);
  // per-solve dt and eta (stored spacing x CFL; eta dt = 2 pi CFL / n0)
  std::vector<SolveDev> sd = b->host_sd;
  for (int s = 0; s < b->n; s++) {
    sd[s].dt = o->cfl * b->host_sd[s].dt;
    sd[s].eta = o->eta > 0.0 ? o->eta : 2.0 * M_PI * o->cfl / (b->geos[s].n0 * sd[s].dt);
    set_stage_weights(sd[s]);
  }
  BCUDA(cudaMemcpyAsync(b->d_sd, sd.data(), sd.size() * sizeof(SolveDev),
                        cudaMemcpyHostToDevice, b->stream));
  if (o->initial == NRR_INIT_ZERO)
    batch_zero_kernel<<<b->nblk_pts, 256, 0, b->stream>>>(b->d_sd, b->d_map_pts);
  else if (o->initial == NRR_INIT_DEVICE)
    batch_warm_v_kernel<<<b->nblk_pts, 256, 0, b->stream>>>(b->d_sd, b->d_map_pts);
  std::vector<int> act(b->n, 1);
  BCUDA(cudaMemcpyAsync(b->d_active, act.data(), b->n * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream));
  BCUDA(cudaMemsetAsync(b->d_steps, 0, b->n * sizeof(long long), b->stream));
  BatchCtl ctl{};
  ctl.n = b->n;
  ctl.max_chunks = (o->max_iters + every - 1) / every;
  ctl.timeout_ns = o->timeout_ms > 0 ? (unsigned long long)o->timeout_ms * 1000000ull : 0;
  ctl.tol = o->tol;
  BCUDA(cudaMemcpyAsync(b->d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, b->stream));
  BTRY(build_relax_graph(b, o->mode, every, o->r_int));
  BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  BCUDA(cudaGraphLaunch(b->exec, b->stream));
  int herr = 0;
  BCUDA(cudaMemcpyAsync(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                        b->stream));
  std::vector<double> norms(b->n);
  std::vector<long long> steps(b->n);
  BCUDA(cudaMemcpyAsync(norms.data(), b->d_norms, b->n * sizeof(double),
                        cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaMemcpyAsync(steps.data(), b->d_steps, b->n * sizeof(long long),
                        cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaMemcpyAsync(act.data(), b->d_active, b->n * sizeof(int),
                        cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaMemcpyAsync(&ctl, b->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (herr)
    return bfail(NRR_ERR_TIMEOUT, "a stage kernel's shared-memory copy wait expired");
  int n_ok = 0, n_div = 0;
  int64_t max_steps = 0;
  double max_norm = 0.0;
  for (int s = 0; s < b->n; s++) {
    int status;
    if (!std::isfinite(norms[s])) {
      status = NRR_ERR_DIVERGED;
      n_div++;
    } else if (norms[s] < o->tol) {
      status = NRR_OK;
      n_ok++;
    } else {
      status = ctl.timed_out ? NRR_ERR_TIMEOUT : NRR_ERR_NOT_CONVERGED;
    }
    if (per_solve) {
      per_solve[s].iters = steps[s];
      per_solve[s].outer_iters = o->mode == NRR_FP32_DC ? steps[s] / every : 0;
      per_solve[s].final_norm = norms[s];
      per_solve[s].seconds = secs;
      per_solve[s].status = status;
    }
    max_steps = std::max<int64_t>(max_steps, steps[s]);
    if (std::isfinite(norms[s])) max_norm = std::max(max_norm, norms[s]);
  }
  nrr_status overall = n_ok == b->n ? NRR_OK
                       : n_div ? NRR_ERR_DIVERGED
                       : ctl.timed_out ? NRR_ERR_TIMEOUT
                                       : NRR_ERR_NOT_CONVERGED;
  if (total) {
    total->iters = max_steps;
    total->outer_iters = ctl.chunk;
    total->final_norm = max_norm;
    total->seconds = secs;
    total->status = overall;
  }
  if (overall != NRR_OK)
    return bfail(overall, "%d of %d solves converged", n_ok, b->n);
  return NRR_OK;
}

nrr_status nrr_batch_get_u(nrr_batch *b, int i, double *dst, int on_device) {
  if (!b || !dst) return bfail(NRR_ERR_INVALID_ARG, "null argument");
  if (i < 0 || i >= b->n) return bfail(NRR_ERR_INVALID_ARG, "solve %d out of range", i);
  BTRY(bbegin(b));
  const Geo &g = b->geos[i];
  launch_fill_ghosts<double>(g, b->host_sd[i].u, b->stream);
  BCUDA(cudaGetLastError());
  BCUDA(cudaMemcpyAsync(dst, b->host_sd[i].u, (size_t)g.npts * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  return NRR_OK;
}

nrr_status nrr_batch_set_u(nrr_batch *b, int i, const double *u, int on_device) {
  if (!b || !u) return bfail(NRR_ERR_INVALID_ARG, "null argument");
  if (i < 0 || i >= b->n) return bfail(NRR_ERR_INVALID_ARG, "solve %d out of range", i);
  BTRY(bbegin(b));
  BCUDA(cudaMemcpyAsync(b->host_sd[i].u, u, (size_t)b->geos[i].npts * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        b->stream));
  BCUDA(cudaStreamSynchronize(b->stream));
  return NRR_OK;
}

nrr_status nrr_batch_get_interior(nrr_batch *b, float *dst) {
  if (!b || !dst) return bfail(NRR_ERR_INVALID_ARG, "null argument");
  for (int s = 1; s < b->n; s++)
    if (b->geos[s].n0 != b->geos[0].n0 || b->geos[s].n1 != b->geos[0].n1 ||
        b->geos[s].n2 != b->geos[0].n2)
      return bfail(NRR_ERR_INVALID_ARG, "solves differ in size");
  BTRY(bbegin(b));
  const Geo &g = b->geos[0];
  const int64_t per = (int64_t)g.n0 * g.n1 * g.n2;
  BCUDA(cudaMemcpyAsync(b->d_sd, b->host_sd.data(), b->n * sizeof(SolveDev),
                        cudaMemcpyHostToDevice, b->stream));
  batch_interior_kernel<<<(unsigned)((b->n * per + 255) / 256), 256, 0, b->stream>>>(
      b->d_sd, b->n, per, dst);
  BCUDA(cudaGetLastError());
  BCUDA(cudaStreamSynchronize(b->stream));
  return NRR_OK;
}

nrr_status nrr_batch_set_launch(nrr_batch *b, int mode, int variant, int zc) {
  if (!b) return bfail(NRR_ERR_INVALID_ARG, "null batch");
  if (mode != NRR_FP64 && mode != NRR_FP32_DC)
    return bfail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32_DC");
  if (variant < 0 || variant > 2)
    return bfail(NRR_ERR_INVALID_ARG, "variant must be 0, 1 or 2");
  if (variant == 1 && !b->tma_ok)
    return bfail(NRR_ERR_INVALID_ARG,
                 "the tensor-copy variant needs order 8, n0 %% 32 == 0, n1 %% 4 == 0");
  if ((variant == 2 && zc != 1 && zc != 2 && zc != 4) ||
      (variant != 2 && zc != 2 && zc != 4 && zc != 8 && zc != 16))
    return bfail(NRR_ERR_INVALID_ARG,
                 "zc must be 1, 2 or 4 (columns) or 2, 4, 8 or 16 (tiles)");
  const int slot = mode == NRR_FP32_DC;
  b->variant[slot] = variant;
  b->zc[slot] = zc;
  return NRR_OK;
}

nrr_status nrr_batch_autotune(nrr_batch *b, int mode, int64_t trial_steps,
                              int *best_zc, double *best_ms_per_launch,
                              int *best_variant) {
  if (!b) return bfail(NRR_ERR_INVALID_ARG, "null batch");
  if (mode != NRR_FP64 && mode != NRR_FP32_DC)
    return bfail(NRR_ERR_INVALID_ARG, "mode must be NRR_FP64 or NRR_FP32_DC");
  if (mode == NRR_FP64 && !b->with_fp64)
    return bfail(NRR_ERR_INVALID_ARG, "batch created without FP64 stage buffers");
  if (trial_steps < 1) return bfail(NRR_ERR_INVALID_ARG, "trial_steps >= 1");
  BTRY(bbegin(b));
  // trials run on the current state: save and restore u, v of every solve
  // (FP32 trials only touch the FP32 increment buffers).
  std::vector<SolveDev> sd = b->host_sd;
  for (int s = 0; s < b->n; s++) {
    sd[s].dt = 0.5 * b->host_sd[s].dt;
    sd[s].eta = 2.0 * M_PI * 0.5 / (b->geos[s].n0 * sd[s].dt);
    set_stage_weights(sd[s]);
  }
  BCUDA(cudaMemcpyAsync(b->d_sd, sd.data(), sd.size() * sizeof(SolveDev),
                        cudaMemcpyHostToDevice, b->stream));
  std::vector<int> act(b->n, 1);
  BCUDA(cudaMemcpyAsync(b->d_active, act.data(), b->n * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream));
  const int slot = mode == NRR_FP32_DC;
  if (mode == NRR_FP64) {
    // keep u, v in the FP64 defect scratch of each solve
    for (int s = 0; s < b->n; s++) {
      size_t by = (size_t)b->geos[s].npts * sizeof(double);
      BCUDA(cudaMemcpyAsync(b->host_sd[s].ku, b->host_sd[s].u, by, cudaMemcpyDeviceToDevice, b->stream));
      BCUDA(cudaMemcpyAsync(b->host_sd[s].kv, b->host_sd[s].v, by, cudaMemcpyDeviceToDevice, b->stream));
    }
  }
  cudaEvent_t e0, e1;
  BCUDA(cudaEventCreate(&e0));
  BCUDA(cudaEventCreate(&e1));
  int best = b->zc[slot], best_var = b->variant[slot];
  double best_ms = 1e30;
  const int cands[9][2] = {{0, 2}, {0, 4}, {0, 8}, {0, 16}, {1, 4},
                           {1, 8}, {1, 16}, {2, 1}, {2, 2}};
  for (const auto &cv : cands) {
    const int var = cv[0], zc = cv[1];
    if (var == 1 && !b->tma_ok) continue;
    b->variant[slot] = var;
    b->zc[slot] = zc;
    BTRY(stage_map_for(b, var, zc));
    for (int rep = 0; rep < 2; rep++) {
      BCUDA(cudaEventRecord(e0, b->stream));
      for (int64_t t = 0; t < trial_steps; t++)
        for (int k = 0; k < 4; k++) {
          if (slot) launch_bstage<float>(b, k, 0, b->stream);
          else launch_bstage<double>(b, k, 0, b->stream);
        }
      BCUDA(cudaEventRecord(e1, b->stream));
      BCUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCUDA(cudaEventElapsedTime(&ms, e0, e1));
      double per = ms / (4.0 * (double)trial_steps);
      if (rep == 1 && per < best_ms) {
        best_ms = per;
        best = zc;
        best_var = var;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->zc[slot] = best;
  b->variant[slot] = best_var;
  int herr = 0;
  BCUDA(cudaMemcpy(&herr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr)
    return bfail(NRR_ERR_TIMEOUT, "a stage kernel's shared-memory copy wait expired");
  if (mode == NRR_FP64)
    for (int s = 0; s < b->n; s++) {
      size_t by = (size_t)b->geos[s].npts * sizeof(double);
      BCUDA(cudaMemcpyAsync(b->host_sd[s].u, b->host_sd[s].ku, by, cudaMemcpyDeviceToDevice, b->stream));
      BCUDA(cudaMemcpyAsync(b->host_sd[s].v, b->host_sd[s].kv, by, cudaMemcpyDeviceToDevice, b->stream));
    }
  BCUDA(cudaStreamSynchronize(b->stream));
  if (best_zc) *best_zc = best;
  if (best_ms_per_launch) *best_ms_per_launch = best_ms;
  if (best_variant) *best_variant = best_var;
  return NRR_OK;
}

}  // extern "C"
