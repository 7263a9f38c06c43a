// nrr_patch.cu -- two overlapping patches relaxed as one system (arXiv
// 2501.14030, Sec. 5: several patches of one solve on one GPU; Sec. 6:
// multipatch grids with interpolation between the patches).
//
// An outer patch (any coordinate family) and an inner Cartesian box.  The
// box's ghost points receive their values by tensor-product Lagrange
// interpolation of q points per direction in the outer patch's coordinates;
// the outer patch's interior points inside a smaller cube (the hole) receive
// theirs from the box in the same way.  Both patches share one time step and
// one wave-speed reference, the smaller of their smallest spacings, so that
// both run at the same Courant number (Sec. 2: wave speed proportional to the
// local spacing).  Each RK4 stage runs both patches' fused stage kernels and
// then one kernel per link that sets the receivers of the stage's output from
// the donor's output: RK4 combines stages linearly, so this is the coupling
// applied to the right-hand side at every stage.
//
// Links are built on the host (inverse coordinate maps, Lagrange weights,
// inner-ghost images) and kept in device memory; a donor point may never be
// a receiver of the other link, which the set-up checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <new>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/nrr.h"
#include "nrr_internal.h"
#include "nrr_stencil.cuh"

using namespace nrr;

namespace {

nrr_status pfail(nrr_status s, const char *fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define PCUDA(call)                                                         \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return pfail(NRR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Cartesian position of padded point (i0, i1, i2) of a grid.
void host_position(const Geo &g, int i0, int i1, int i2, double x[3]) {
  const double xx0 = g.xxmin[0] + (i0 - g.ng + 0.5) * g.dxx[0];
  const double xx1 = g.xxmin[1] + (i1 - g.ng + 0.5) * g.dxx[1];
  const double xx2 = g.xxmin[2] + (i2 - g.ng + 0.5) * g.dxx[2];
  const double s = [&] {
    if (g.coord == SINHSYMTP || g.coord == SINHSPHERICAL || g.coord == SINHCYLINDRICAL)
      return g.amax * std::sinh(xx0 / g.sinhwaa) / std::sinh(1.0 / g.sinhwaa);
    return xx0;
  }();
  switch (g.coord) {
    case CARTESIAN:
      x[0] = xx0, x[1] = xx1, x[2] = xx2;
      return;
    case SINHCYLINDRICAL:
      x[0] = s * std::cos(xx2), x[1] = s * std::sin(xx2);
      x[2] = g.zmax * std::sinh(xx1 / g.sinhwz) / std::sinh(1.0 / g.sinhwz);
      return;
    case SINHSYMTP:
      x[0] = s * std::sin(xx1) * std::cos(xx2), x[1] = s * std::sin(xx1) * std::sin(xx2);
      x[2] = std::sqrt(s * s + g.bscale * g.bscale) * std::cos(xx1);
      return;
    default:  // spherical-like: s = r
      x[0] = s * std::sin(xx1) * std::cos(xx2), x[1] = s * std::sin(xx1) * std::sin(xx2);
      x[2] = s * std::cos(xx1);
      return;
  }
}

// Coordinates xx of a Cartesian point in a grid's family, in the canonical
// range (xx0 >= 0, theta in [0, pi], phi in (-pi, pi]).
void host_coords(const Geo &g, const double x[3], double xx[3]) {
  const double rho2 = x[0] * x[0] + x[1] * x[1], rho = std::sqrt(rho2);
  if (g.coord == CARTESIAN) {
    xx[0] = x[0], xx[1] = x[1], xx[2] = x[2];
    return;
  }
  xx[2] = std::atan2(x[1], x[0]);
  const double z = x[2];
  if (g.coord == SINHCYLINDRICAL) {
    xx[0] = g.sinhwaa * std::asinh(rho * std::sinh(1.0 / g.sinhwaa) / g.amax);
    xx[1] = g.sinhwz * std::asinh(z * std::sinh(1.0 / g.sinhwz) / g.zmax);
    return;
  }
  if (g.coord == SINHSYMTP) {
    // rho = A sin(th), z = sqrt(A^2 + b^2) cos(th): A^2 is the positive root
    // of X^2 - (rho^2 + z^2 - b^2) X - rho^2 b^2 = 0 (written in a form that
    // does not cancel when the linear coefficient is negative)
    const double b2 = g.bscale * g.bscale, q = rho2 + z * z - b2;
    const double d = std::sqrt(q * q + 4.0 * rho2 * b2);
    const double A2 = q >= 0.0 ? 0.5 * (q + d) : (d > 0.0 ? 2.0 * rho2 * b2 / (d - q) : 0.0);
    const double A = std::sqrt(A2);
    xx[0] = g.sinhwaa * std::asinh(A * std::sinh(1.0 / g.sinhwaa) / g.amax);
    xx[1] = std::atan2(rho * std::sqrt(A2 + b2), z * A);
    return;
  }
  const double r = std::sqrt(rho2 + z * z);
  xx[0] = g.coord == SINHSPHERICAL
              ? g.sinhwaa * std::asinh(r * std::sinh(1.0 / g.sinhwaa) / g.amax)
              : r;
  xx[1] = std::atan2(rho, z);
}

// Lagrange weights of nodes base .. base+q-1 at position f (grid-index units).
void lagrange(int q, int base, double f, double *w) {
  for (int j = 0; j < q; j++) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < q; m++) {
      if (m == j) continue;
      num *= f - (double)(base + m);
      den *= (double)(j - m);
    }
    w[j] = num / den;
  }
}

struct HostLink {
  std::vector<int64_t> recv, donor;  // donor[r q^3 + k], k = a + q (b + q c)
  std::vector<double> w;             // w[r q^3 + k] = wxy[a + q b] wz[c]
  std::vector<double> wxy, wz;       // per receiver: q^2 and q factors
};

// Receivers (flat indices in `rg`) with their donor stencils in `dg`.
nrr_status build_link(const Geo &rg, const Geo &dg, const std::vector<int64_t> &recv,
                      int q, HostLink *out) {
  const int m = q * q * q;
  out->recv = recv;
  out->donor.resize(recv.size() * (size_t)m);
  out->w.resize(recv.size() * (size_t)m);
  out->wxy.resize(recv.size() * (size_t)q * q);
  out->wz.resize(recv.size() * (size_t)q);
  const int sd[3] = {dg.s0, dg.s1, dg.s2};
  for (size_t r = 0; r < recv.size(); r++) {
    const int64_t p = recv[r];
    const int i0 = (int)(p % rg.s0), i1 = (int)((p / rg.s0) % rg.s1),
              i2 = (int)(p / rg.ncol);
    double x[3], xx[3];
    host_position(rg, i0, i1, i2, x);
    host_coords(dg, x, xx);
    int base[3];
    double wd[3][6];
    for (int d = 0; d < 3; d++) {
      const double f = (xx[d] - dg.xxmin[d]) / dg.dxx[d] - 0.5 + dg.ng;
      base[d] = (int)std::floor(f) - (q / 2 - 1);
      if (base[d] < 0 || base[d] + q - 1 >= sd[d])
        return pfail(NRR_ERR_INVALID_ARG,
                     "receiver at (%.3g, %.3g, %.3g): its stencil leaves the donor patch",
                     x[0], x[1], x[2]);
      lagrange(q, base[d], f, wd[d]);
    }
    for (int b = 0; b < q; b++)
      for (int a = 0; a < q; a++) out->wxy[r * q * q + a + q * b] = wd[0][a] * wd[1][b];
    for (int c = 0; c < q; c++) out->wz[r * q + c] = wd[2][c];
    int k = 0;
    for (int c = 0; c < q; c++)
      for (int b = 0; b < q; b++)
        for (int a = 0; a < q; a++, k++) {
          int j0 = base[0] + a, j1 = base[1] + b, j2 = base[2] + c;
          if (dg.coord != CARTESIAN) image_of(dg, j0, j1, j2);
          out->donor[r * m + k] = flat(dg, j0, j1, j2);
          // the same product as the kernel forms: (wx wy) wz
          out->w[r * m + k] = out->wxy[r * q * q + a + q * b] * wd[2][c];
        }
  }
  return NRR_OK;
}

// One link on the device.
// Device form of a link, stencil-point-major ([j * n + r] for entry j of
// receiver r, so that the threads of a warp read consecutive entries), in
// the tensor-product structure of the stencil: the donor of stencil point
// (a, b, c) is column col[a + q b] (32-bit; patches of fewer than 2^31
// points) on plane planes[c] -- or planes[q + c], the plane at phi + pi, where
// bit a + q b of flip is set (columns whose image lies across the axis or
// the origin) -- and its weight is wxy[a + q b] wz[c].
struct DevLink {
  int64_t n = 0;
  int64_t ncol = 0;  // donor grid's points per plane
  int64_t *recv = nullptr;
  int32_t *col = nullptr;
  unsigned long long *flip = nullptr;
  int32_t *planes = nullptr;
  double *wxy = nullptr, *wz = nullptr;
};

// Receivers of the stage output (du, dv) from the donor's output (su, sv):
// one thread per receiver.  Each plane c of the stencil has its own
// accumulator (q independent FMA chains per field: the FP64 pipe needs them,
// since a small link gives few warps per SM), the q^2 products of a plane
// summed in order (b outer, then a), the planes' sums then added in order c
// = 0 .. q-1.
// T: the precision of the fields (FP64, or FP32 for the increments of the
// defect correction, whose weights are rounded to FP32 before the products).
template <int Q, typename T>
__global__ void __launch_bounds__(128)
    link_apply_kernel(int64_t n, int64_t ncol, const int64_t *__restrict__ recv,
                      const int32_t *__restrict__ col,
                      const unsigned long long *__restrict__ flip,
                      const int32_t *__restrict__ planes,
                      const double *__restrict__ wxy, const double *__restrict__ wz,
                      const T *su, const T *sv, T *du, T *dv) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int32_t cl[Q * Q];
  T wab[Q * Q];
#pragma unroll
  for (int ab = 0; ab < Q * Q; ab++) {
    cl[ab] = col[(int64_t)ab * n + r];
    wab[ab] = (T)wxy[(int64_t)ab * n + r];
  }
  const unsigned long long fm = flip[r];
  T a[Q], b[Q];
#pragma unroll
  for (int c = 0; c < Q; c++) {
    const T wc = (T)wz[(int64_t)c * n + r];
    const int64_t o0 = ncol * planes[(int64_t)c * n + r];
    const int64_t o1 = ncol * planes[(int64_t)(Q + c) * n + r];
    a[c] = T(0);
    b[c] = T(0);
#pragma unroll
    for (int ab = 0; ab < Q * Q; ab++) {
      const T w = wab[ab] * wc;
      const int64_t d = cl[ab] + (((fm >> ab) & 1ull) ? o1 : o0);
      a[c] = fma(w, su[d], a[c]);
      b[c] = fma(w, sv[d], b[c]);
    }
  }
  T sa = a[0], sb = b[0];
#pragma unroll
  for (int c = 1; c < Q; c++) {
    sa += a[c];
    sb += b[c];
  }
  du[recv[r]] = sa;
  dv[recv[r]] = sb;
}

// The same sums with the Q planes of a receiver on Q adjacent lanes (Q = 2
// or 4, so a receiver's lanes share a warp): Q times the threads and a Q
// times shorter chain per thread, for links too small to fill the GPU with
// one thread per receiver.  Each lane sums its plane in the same order, and
// the first lane adds the planes in order c = 0 .. Q-1: the results equal
// link_apply_kernel's bit for bit.
template <int Q, typename T>
__global__ void __launch_bounds__(128)
    link_apply_lanes_kernel(int64_t n, int64_t ncol, const int64_t *__restrict__ recv,
                            const int32_t *__restrict__ col,
                            const unsigned long long *__restrict__ flip,
                            const int32_t *__restrict__ planes,
                            const double *__restrict__ wxy,
                            const double *__restrict__ wz, const T *su, const T *sv,
                            T *du, T *dv) {
  static_assert(32 % Q == 0, "a receiver's lanes stay in one warp");
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = t / Q;
  const int c = (int)(t % Q);
  const bool live = r < n;
  T a = T(0), b = T(0);
  if (live) {
    const unsigned long long fm = flip[r];
    const T wc = (T)wz[(int64_t)c * n + r];
    const int64_t o0 = ncol * planes[(int64_t)c * n + r];
    const int64_t o1 = ncol * planes[(int64_t)(Q + c) * n + r];
#pragma unroll
    for (int ab = 0; ab < Q * Q; ab++) {
      const T w = (T)wxy[(int64_t)ab * n + r] * wc;
      const int64_t d = col[(int64_t)ab * n + r] + (((fm >> ab) & 1ull) ? o1 : o0);
      a = fma(w, su[d], a);
      b = fma(w, sv[d], b);
    }
  }
  // every lane of the warp takes part in the shuffles (the group of a
  // receiver past n computes nothing and stores nothing)
  const int lane = threadIdx.x & 31, base = lane - c;
  T sa = __shfl_sync(0xffffffffu, a, base), sb = __shfl_sync(0xffffffffu, b, base);
#pragma unroll
  for (int k = 1; k < Q; k++) {
    sa += __shfl_sync(0xffffffffu, a, base + k);
    sb += __shfl_sync(0xffffffffu, b, base + k);
  }
  if (live && c == 0) {
    du[recv[r]] = sa;
    dv[recv[r]] = sb;
  }
}

template <typename T>
void launch_link(const DevLink &l, int q, const T *su, const T *sv, T *du, T *dv,
                 cudaStream_t st) {
#define NRR_LINK(Q)                                                                     \
  link_apply_lanes_kernel<Q, T><<<(unsigned)((l.n * Q + 127) / 128), 128, 0, st>>>(    \
      l.n, l.ncol, l.recv, l.col, l.flip, l.planes, l.wxy, l.wz, su, sv, du, dv)
  switch (q) {
    case 2: NRR_LINK(2); break;
    case 6:
      link_apply_kernel<6, T><<<(unsigned)((l.n + 127) / 128), 128, 0, st>>>(
          l.n, l.ncol, l.recv, l.col, l.flip, l.planes, l.wxy, l.wz, su, sv, du, dv);
      break;
    default: NRR_LINK(4); break;
  }
#undef NRR_LINK
}

// The device form of host link `h` whose donor grid is `dg`: columns,
// flip bits and planes read off the donor list (and checked against it
// entry by entry), arrays transposed to stencil-point-major order.
bool compress_link(const HostLink &h, const Geo &dg, int q, std::vector<int32_t> &col,
                   std::vector<unsigned long long> &flip, std::vector<int32_t> &planes,
                   std::vector<double> &wxy, std::vector<double> &wz) {
  const int64_t n = (int64_t)h.recv.size(), nc = dg.ncol;
  const int q2 = q * q, m = q2 * q;
  col.assign((size_t)q2 * n, 0);
  flip.assign((size_t)n, 0ull);
  planes.assign((size_t)2 * q * n, 0);
  wxy.assign((size_t)q2 * n, 0.0);
  wz.assign((size_t)q * n, 0.0);
  for (int64_t r = 0; r < n; r++) {
    const int64_t *d = &h.donor[(size_t)r * m];
    // planes of column (0, 0) and their phi + pi partners; a flip bit says
    // that a column sits on the partner planes (its image lies across the
    // axis or the origin while column (0, 0)'s does not, or the reverse)
    int pl[2][6];
    for (int c = 0; c < q; c++) {
      const int z = (int)(d[q2 * c] / nc);
      const int zf = dg.coord == CARTESIAN ? z : wrap_phi(dg, z + dg.n2 / 2);
      pl[0][c] = z;
      pl[1][c] = zf;
    }
    unsigned long long fm = 0ull;
    for (int ab = 0; ab < q2; ab++) {
      const int64_t c0 = d[ab] % nc;
      const int z0 = (int)(d[ab] / nc);
      const int f = z0 == pl[0][0] ? 0 : (z0 == pl[1][0] ? 1 : -1);
      if (f < 0 || c0 > INT32_MAX) return false;
      col[(size_t)ab * n + r] = (int32_t)c0;
      if (f) fm |= 1ull << ab;
      for (int c = 0; c < q; c++)
        if (d[ab + q2 * c] != c0 + nc * pl[f][c]) return false;
      wxy[(size_t)ab * n + r] = h.wxy[(size_t)r * q2 + ab];
    }
    flip[(size_t)r] = fm;
    for (int c = 0; c < q; c++) {
      planes[(size_t)c * n + r] = pl[0][c];
      planes[(size_t)(q + c) * n + r] = pl[1][c];
      wz[(size_t)c * n + r] = h.wz[(size_t)r * q + c];
    }
  }
  return true;
}

// Partial sums (H^2 J, J) of one patch over its interior points that are
// not receivers and lie within r < r_int; J = h0 h1 h2 per column
// (curvilinear) or 1 (Cartesian).
__global__ void masked_norm_kernel(Geo g, const double *__restrict__ H,
                                   const unsigned char *__restrict__ mask,
                                   const double *__restrict__ jac,
                                   const double *__restrict__ rad, double r_int,
                                   double *partials) {
  const int64_t nint = (int64_t)g.n0 * g.n1 * g.n2;
  double num = 0.0, den = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nint;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(e % g.n0) + g.ng, i1 = (int)((e / g.n0) % g.n1) + g.ng,
              i2 = (int)(e / ((int64_t)g.n0 * g.n1)) + g.ng;
    const int64_t p = flat(g, i0, i1, i2);
    if (mask[p]) continue;
    double wt;
    if (g.coord == CARTESIAN) {
      const double x0 = g.xxmin[0] + (i0 - g.ng + 0.5) * g.dxx[0];
      const double x1 = g.xxmin[1] + (i1 - g.ng + 0.5) * g.dxx[1];
      const double x2 = g.xxmin[2] + (i2 - g.ng + 0.5) * g.dxx[2];
      wt = std::sqrt(x0 * x0 + x1 * x1 + x2 * x2) < r_int ? 1.0 : 0.0;
    } else {
      const int col = i0 + g.s0 * i1;
      wt = rad[col] < r_int ? jac[col] : 0.0;
    }
    const double h = H[p];
    num += h * h * wt;
    den += wt;
  }
  dev::block_sum2(num, den, partials + 2 * blockIdx.x);
}

constexpr int kNormBlocks = 512;  // per patch

}  // namespace

// One relaxation chunk (m RK4 steps of both patches with their links, then
// the residual norm) captured as a CUDA graph, with what it was captured for.
struct PatchChunkGraph {
  cudaGraphExec_t exec = nullptr;
  int mode = -1;
  int64_t m = 0;
  double dt = 0.0, eta = 0.0, r_int = 0.0;
  LaunchCfg cfg[2], cfg32[2];
};

struct nrr_patchset {
  nrr_grid *grid[2] = {nullptr, nullptr};  // outer, inner
  PatchChunkGraph chunk;
  // the inner patch's stage kernels run on `side`, concurrently with the
  // outer patch's on the outer grid's stream; fork / join order them
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  DevLink link[2];                          // receivers of grid[i]
  unsigned char *mask[2] = {nullptr, nullptr};
  double *partials = nullptr;               // 2 * kNormBlocks pairs
  double *norm = nullptr;                   // [3]
  double *host = nullptr;                   // pinned read-back
  int q = 4;
  double ds_ref = 0.0;
  int device = 0;
  std::vector<void *> allocs;
};

namespace {

template <typename T>
nrr_status palloc(nrr_patchset *ps, T **p, size_t count) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T) + 16);
  if (e != cudaSuccess)
    return pfail(NRR_ERR_OOM, "cudaMalloc of %zu bytes: %s", count * sizeof(T),
                 cudaGetErrorString(e));
  ps->allocs.push_back(ptr);
  dbg_register(ptr, count * sizeof(T) + 16);
  *p = static_cast<T *>(ptr);
  return NRR_OK;
}

// Every RK4 stage on both patches, then the links; `steps` steps on the
// outer grid's work stream.  The two patches' stage kernels of one stage
// are independent (each reads and writes only its own patch), so the inner
// patch's runs on a side stream that forks from the outer grid's stream
// before the stage and joins it before the links, which read both.  (Stage
// kernels launched this way go without programmatic dependent launch: the
// node before each is an event, not the previous stage.)
// R = double: the relaxation system; R = float: the defect correction's
// increment equation (the grids' FP32 increment fields, FP32 links).
template <typename R>
void launch_patch_steps(nrr_patchset *ps, double dt, double eta, int64_t steps) {
  static const int kinds[4] = {STAGE_FIRST, STAGE_MID, STAGE_MID, STAGE_LAST};
  GridView v[2] = {grid_view(ps->grid[0]), grid_view(ps->grid[1])};
  cudaStream_t st = v[0].stream;
  const cudaStream_t on[2] = {st, ps->side};
  constexpr bool f32 = sizeof(R) == 4;
  LaunchCfg cfg[2] = {f32 ? v[0].cfg32 : v[0].cfg64, f32 ? v[1].cfg32 : v[1].cfg64};
  cfg[0].pdl = cfg[1].pdl = 0;
  for (int64_t s = 0; s < steps; s++)
    for (int k = 0; k < 4; k++) {
      StageArgs<R> a[2];
      cudaEventRecord(ps->fork, st);
      cudaStreamWaitEvent(ps->side, ps->fork, 0);
      for (int i = 0; i < 2; i++) {
        if constexpr (f32)
          a[i] = rk4_stage_args<R>(v[i].dc32, v[i].c32, v[i].cart, v[i].err, k, dt, eta);
        else
          a[i] = rk4_stage_args<R>(v[i].f64, v[i].c64, v[i].cart, v[i].err, k, dt, eta);
        launch_stage<R>(v[i].geo, kinds[k], a[i], cfg[i], on[i]);
      }
      cudaEventRecord(ps->join, ps->side);
      cudaStreamWaitEvent(st, ps->join, 0);
      for (int i = 0; i < 2; i++) {
        const DevLink &l = ps->link[i];
        if (l.n == 0) continue;
        const int j = 1 - i;  // donor
        launch_link(l, ps->q, a[j].ou, a[j].ov, a[i].ou, a[i].ov, st);
      }
    }
}

// The two-patch residual norm of the current state into ps->norm[0].
void launch_patch_norm(nrr_patchset *ps, double r_int) {
  GridView v[2] = {grid_view(ps->grid[0]), grid_view(ps->grid[1])};
  cudaStream_t st = v[0].stream;
  for (int i = 0; i < 2; i++) {
    int nb = 0;
    launch_residual<double>(v[i].geo, v[i].f64.y[0], v[i].f64.alpha, v[i].f64.bc2,
                            v[i].c64, v[i].cart, v[i].jac, v[i].rad, r_int,
                            v[i].scratch, v[i].partials, &nb, v[i].res_cfg, st);
    masked_norm_kernel<<<kNormBlocks, 128, 0, st>>>(
        v[i].geo, v[i].scratch, ps->mask[i], v[i].jac, v[i].rad, r_int,
        ps->partials + 2 * kNormBlocks * i);
  }
  launch_norm_finalize(ps->partials, 2 * kNormBlocks, ps->norm, st);
}

nrr_status read_norm(nrr_patchset *ps, double *out) {
  cudaStream_t st = grid_view(ps->grid[0]).stream;
  PCUDA(cudaGetLastError());
  PCUDA(cudaMemcpyAsync(ps->host, ps->norm, sizeof(double), cudaMemcpyDeviceToHost, st));
  PCUDA(cudaStreamSynchronize(st));
  *out = ps->host[0];
  return NRR_OK;
}

bool same_cfg(const LaunchCfg &a, const LaunchCfg &b) {
  return a.block == b.block && a.zc == b.zc && a.variant == b.variant && a.pdl == b.pdl;
}

// One chunk on the outer grid's stream: NRR_FP64, m RK4 steps of both patches
// with their links; NRR_FP32_DC, one defect-correction outer iteration -- the
// FP64 defect and FP32 coefficients of each patch, m FP32 steps of both
// patches' increments with FP32 links, the FP64 update of each patch, and
// then the FP64 links on the updated state: the FP32 links interpolate the
// increments only to FP32 rounding, and receivers left that far from the
// FP64 interpolation of their donors would pose a slightly different
// discrete problem.  Then the coupled norm.
void launch_chunk(nrr_patchset *ps, int mode, int64_t m, double dt, double eta,
                  double r_int) {
  cudaStream_t st = grid_view(ps->grid[0]).stream;
  if (mode == NRR_FP32_DC) {
    for (int i = 0; i < 2; i++) dc_outer_prep(ps->grid[i], eta, st);
    launch_patch_steps<float>(ps, dt, eta, m);
    GridView v[2] = {grid_view(ps->grid[0]), grid_view(ps->grid[1])};
    for (int i = 0; i < 2; i++) dc_outer_update(ps->grid[i], st);
    for (int i = 0; i < 2; i++) {
      const DevLink &l = ps->link[i];
      if (l.n == 0) continue;
      const int j = 1 - i;  // donor
      launch_link<double>(l, ps->q, v[j].f64.y[0], v[j].f64.y[1], v[i].f64.y[0],
                          v[i].f64.y[1], st);
    }
  } else {
    launch_patch_steps<double>(ps, dt, eta, m);
  }
  launch_patch_norm(ps, r_int);
}

// The graph of one chunk for (mode, m, dt, eta, r_int) and the grids' current
// launch shapes: the cached one, or a new capture of the launches
// launch_chunk issues.  One graph launch then replaces them all.
nrr_status chunk_graph(nrr_patchset *ps, int mode, int64_t m, double dt, double eta,
                       double r_int, cudaGraphExec_t *out) {
  const GridView v0 = grid_view(ps->grid[0]), v1 = grid_view(ps->grid[1]);
  PatchChunkGraph &c = ps->chunk;
  if (c.exec && c.mode == mode && c.m == m && c.dt == dt && c.eta == eta &&
      c.r_int == r_int && same_cfg(c.cfg[0], v0.cfg64) && same_cfg(c.cfg[1], v1.cfg64) &&
      same_cfg(c.cfg32[0], v0.cfg32) && same_cfg(c.cfg32[1], v1.cfg32)) {
    *out = c.exec;
    return NRR_OK;
  }
  if (c.exec) {
    cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
  }
  cudaStream_t st = v0.stream;
  cudaGraph_t graph = nullptr;
  PCUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  launch_chunk(ps, mode, m, dt, eta, r_int);
  PCUDA(cudaStreamEndCapture(st, &graph));
  const cudaError_t e = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c.exec = nullptr;
    return pfail(NRR_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  c.mode = mode;
  c.m = m;
  c.dt = dt;
  c.eta = eta;
  c.r_int = r_int;
  c.cfg[0] = v0.cfg64;
  c.cfg[1] = v1.cfg64;
  c.cfg32[0] = v0.cfg32;
  c.cfg32[1] = v1.cfg32;
  *out = c.exec;
  return NRR_OK;
}

// Both grids' streams drained, so the outer grid's stream may take over
// both patches' state.
nrr_status begin(nrr_patchset *ps) {
  PCUDA(cudaSetDevice(ps->device));
  PCUDA(cudaStreamSynchronize(grid_view(ps->grid[1]).stream));
  PCUDA(cudaStreamSynchronize(grid_view(ps->grid[0]).stream));
  return NRR_OK;
}

}  // namespace

extern "C" {

nrr_status nrr_patchset_create(nrr_grid *outer, nrr_grid *inner, double hole, int q,
                               nrr_patchset **out) {
  if (!out) return pfail(NRR_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (!outer || !inner || outer == inner)
    return pfail(NRR_ERR_INVALID_ARG, "two distinct grids are needed");
  if (q != 2 && q != 4 && q != 6) return pfail(NRR_ERR_INVALID_ARG, "q must be 2, 4 or 6");
  if (!(hole > 0.0)) return pfail(NRR_ERR_INVALID_ARG, "hole must be positive");
  GridView vo = grid_view(outer), vi = grid_view(inner);
  if (vi.geo.coord != CARTESIAN)
    return pfail(NRR_ERR_INVALID_ARG, "the inner patch must be Cartesian");
  if (!vo.have_source || !vi.have_source)
    return pfail(NRR_ERR_STATE, "punctures must be set on both patches");
  if (q / 2 > vo.geo.ng || q / 2 > vi.geo.ng)
    return pfail(NRR_ERR_INVALID_ARG, "q/2 exceeds a patch's ghost width");
  if (vo.geo.npts >= (int64_t)1 << 31 || vi.geo.npts >= (int64_t)1 << 31)
    return pfail(NRR_ERR_INVALID_ARG, "patches must have fewer than 2^31 points");
  // the inner box's receivers: all its ghost points
  std::vector<int64_t> recv_in, recv_out;
  const Geo &gi = vi.geo, &go = vo.geo;
  for (int i2 = 0; i2 < gi.s2; i2++)
    for (int i1 = 0; i1 < gi.s1; i1++)
      for (int i0 = 0; i0 < gi.s0; i0++) {
        const bool in = i0 >= gi.ng && i0 < gi.ng + gi.n0 && i1 >= gi.ng &&
                        i1 < gi.ng + gi.n1 && i2 >= gi.ng && i2 < gi.ng + gi.n2;
        if (!in) recv_in.push_back(flat(gi, i0, i1, i2));
      }
  // the outer patch's hole: interior points with max(|x|, |y|, |z|) < hole
  for (int i2 = go.ng; i2 < go.ng + go.n2; i2++)
    for (int i1 = go.ng; i1 < go.ng + go.n1; i1++)
      for (int i0 = go.ng; i0 < go.ng + go.n0; i0++) {
        double x[3];
        host_position(go, i0, i1, i2, x);
        if (std::fmax(std::fabs(x[0]), std::fmax(std::fabs(x[1]), std::fabs(x[2]))) < hole)
          recv_out.push_back(flat(go, i0, i1, i2));
      }
  HostLink hl[2];
  nrr_status s = build_link(go, gi, recv_out, q, &hl[0]);
  if (s != NRR_OK) return s;
  s = build_link(gi, go, recv_in, q, &hl[1]);
  if (s != NRR_OK) return s;
  // no donor point of one link may be a receiver of the other
  std::vector<unsigned char> mk[2] = {std::vector<unsigned char>((size_t)go.npts, 0),
                                      std::vector<unsigned char>((size_t)gi.npts, 0)};
  for (int i = 0; i < 2; i++)
    for (int64_t p : hl[i].recv) mk[i][(size_t)p] = 1;
  for (int i = 0; i < 2; i++)
    for (int64_t d : hl[i].donor)
      if (mk[1 - i][(size_t)d])
        return pfail(NRR_ERR_INVALID_ARG,
                     "a donor point of the %s patch's receivers is itself a receiver "
                     "(make the hole smaller)", i == 0 ? "outer" : "inner");
  nrr_patchset *ps = new (std::nothrow) nrr_patchset();
  if (!ps) return pfail(NRR_ERR_OOM, "host allocation failed");
  ps->grid[0] = outer;
  ps->grid[1] = inner;
  ps->q = q;
  nrr_status st = [&]() -> nrr_status {
    PCUDA(cudaGetDevice(&ps->device));
    // one wave-speed reference and so one time step for both patches
    ps->ds_ref = std::fmin(vo.dsmin, vi.dsmin);
    nrr_status e = nrr_set_speed_reference(outer, ps->ds_ref);
    if (e != NRR_OK) return e;
    e = nrr_set_speed_reference(inner, ps->ds_ref);
    if (e != NRR_OK) return e;
    for (int i = 0; i < 2; i++) {
      DevLink &l = ps->link[i];
      const Geo &dg = i == 0 ? gi : go;  // donor of link i
      l.n = (int64_t)hl[i].recv.size();
      l.ncol = dg.ncol;
      std::vector<int32_t> col, planes;
      std::vector<unsigned long long> flip;
      std::vector<double> wxy, wz;
      if (!compress_link(hl[i], dg, q, col, flip, planes, wxy, wz))
        return pfail(NRR_ERR_INVALID_ARG,
                     "a receiver's donor stencil does not have the tensor-product "
                     "form (columns x planes) the device link uses");
      e = palloc(ps, &l.recv, (size_t)l.n);
      if (e == NRR_OK) e = palloc(ps, &l.col, col.size());
      if (e == NRR_OK) e = palloc(ps, &l.flip, flip.size());
      if (e == NRR_OK) e = palloc(ps, &l.planes, planes.size());
      if (e == NRR_OK) e = palloc(ps, &l.wxy, wxy.size());
      if (e == NRR_OK) e = palloc(ps, &l.wz, wz.size());
      if (e == NRR_OK) e = palloc(ps, &ps->mask[i], mk[i].size());
      if (e != NRR_OK) return e;
      PCUDA(cudaMemcpy(l.recv, hl[i].recv.data(), l.n * sizeof(int64_t),
                       cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(l.col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(l.flip, flip.data(), flip.size() * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(l.planes, planes.data(), planes.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(l.wxy, wxy.data(), wxy.size() * sizeof(double), cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(l.wz, wz.data(), wz.size() * sizeof(double), cudaMemcpyHostToDevice));
      PCUDA(cudaMemcpy(ps->mask[i], mk[i].data(), mk[i].size(), cudaMemcpyHostToDevice));
    }
    e = palloc(ps, &ps->partials, 4 * (size_t)kNormBlocks);
    if (e == NRR_OK) e = palloc(ps, &ps->norm, 4);
    if (e != NRR_OK) return e;
    PCUDA(cudaMallocHost(&ps->host, 4 * sizeof(double)));
    PCUDA(cudaStreamCreateWithFlags(&ps->side, cudaStreamNonBlocking));
    PCUDA(cudaEventCreateWithFlags(&ps->fork, cudaEventDisableTiming));
    PCUDA(cudaEventCreateWithFlags(&ps->join, cudaEventDisableTiming));
    return NRR_OK;
  }();
  if (st != NRR_OK) {
    nrr_patchset_destroy(ps);
    return st;
  }
  *out = ps;
  return NRR_OK;
}

nrr_status nrr_patchset_destroy(nrr_patchset *ps) {
  if (!ps) return NRR_OK;
  cudaSetDevice(ps->device);
  for (void *p : ps->allocs) {
    dbg_unregister(p);
    cudaFree(p);
  }
  if (ps->host) cudaFreeHost(ps->host);
  if (ps->chunk.exec) cudaGraphExecDestroy(ps->chunk.exec);
  if (ps->fork) cudaEventDestroy(ps->fork);
  if (ps->join) cudaEventDestroy(ps->join);
  if (ps->side) cudaStreamDestroy(ps->side);
  delete ps;
  return NRR_OK;
}

nrr_status nrr_patchset_info(const nrr_patchset *ps, int64_t *outer_receivers,
                             int64_t *inner_receivers, double *ds_ref) {
  if (!ps) return pfail(NRR_ERR_INVALID_ARG, "null patch set");
  if (outer_receivers) *outer_receivers = ps->link[0].n;
  if (inner_receivers) *inner_receivers = ps->link[1].n;
  if (ds_ref) *ds_ref = ps->ds_ref;
  return NRR_OK;
}

nrr_status nrr_patchset_timestep(const nrr_patchset *ps, double cfl, double *dt,
                                 double *eta_default) {
  if (!ps || !(cfl > 0.0)) return pfail(NRR_ERR_INVALID_ARG, "null patch set or cfl <= 0");
  const double d = cfl * ps->ds_ref;
  if (dt) *dt = d;
  if (eta_default)
    *eta_default = 2.0 * M_PI * cfl / (grid_view(ps->grid[0]).geo.n0 * d);
  return NRR_OK;
}

nrr_status nrr_patchset_step(nrr_patchset *ps, double dt, double eta, int64_t steps) {
  if (!ps || !(dt > 0.0) || steps < 0)
    return pfail(NRR_ERR_INVALID_ARG, "null patch set, dt <= 0 or steps < 0");
  nrr_status s = begin(ps);
  if (s != NRR_OK) return s;
  launch_patch_steps<double>(ps, dt, eta, steps);
  cudaStream_t st = grid_view(ps->grid[0]).stream;
  PCUDA(cudaGetLastError());
  PCUDA(cudaStreamSynchronize(st));
  return NRR_OK;
}

nrr_status nrr_patchset_residual(nrr_patchset *ps, double r_int, double *norm_out) {
  if (!ps || !norm_out || !(r_int > 0.0))
    return pfail(NRR_ERR_INVALID_ARG, "null argument or r_int <= 0");
  nrr_status s = begin(ps);
  if (s != NRR_OK) return s;
  launch_patch_norm(ps, r_int);
  return read_norm(ps, norm_out);
}

nrr_status nrr_patchset_relax(nrr_patchset *ps, const nrr_relax_opts *o,
                              nrr_relax_result *r) {
  if (!ps || !o) return pfail(NRR_ERR_INVALID_ARG, "null argument");
  if (o->mode != NRR_FP64 && o->mode != NRR_FP32_DC)
    return pfail(NRR_ERR_INVALID_ARG, "patch sets relax in NRR_FP64 or NRR_FP32_DC");
  if (o->mode == NRR_FP32_DC && o->inner_steps < 0)
    return pfail(NRR_ERR_INVALID_ARG, "inner_steps < 0");
  if (!(o->tol > 0.0) || o->check_every < 1 || o->max_iters < 0 || !(o->cfl > 0.0) ||
      !(o->r_int > 0.0))
    return pfail(NRR_ERR_INVALID_ARG, "invalid relax options");
  if (o->initial != NRR_INIT_ZERO && o->initial != NRR_INIT_CURRENT)
    return pfail(NRR_ERR_INVALID_ARG, "patch sets start from zero or the current state");
  using clk = std::chrono::steady_clock;
  const auto t_start = clk::now();
  auto elapsed_ms = [&] {
    return std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
  };
  nrr_status s = begin(ps);
  if (s != NRR_OK) return s;
  cudaStream_t st = grid_view(ps->grid[0]).stream;
  if (o->initial == NRR_INIT_ZERO)
    for (int i = 0; i < 2; i++) {
      GridView v = grid_view(ps->grid[i]);
      for (int c = 0; c < 2; c++)
        PCUDA(cudaMemsetAsync(v.f64.y[c], 0, (size_t)v.geo.npts * sizeof(double), st));
    }
  double dt = 0.0, eta_def = 0.0;
  nrr_patchset_timestep(ps, o->cfl, &dt, &eta_def);
  const double eta = o->eta > 0.0 ? o->eta : eta_def;
  double nrm = 0.0;
  launch_patch_norm(ps, o->r_int);
  s = read_norm(ps, &nrm);
  if (s != NRR_OK) return s;
  int64_t it = 0, outer = 0;
  // steps per chunk: FP64, the norm check interval; defect correction, the
  // FP32 steps of one outer iteration
  const int64_t every =
      o->mode == NRR_FP32_DC && o->inner_steps > 0 ? o->inner_steps : o->check_every;
  nrr_status why = NRR_ERR_NOT_CONVERGED;
  for (;;) {
    if (!std::isfinite(nrm)) {
      why = NRR_ERR_DIVERGED;
      break;
    }
    if (nrm < o->tol) {
      why = NRR_OK;
      break;
    }
    if (it >= o->max_iters) break;
    if (o->mode == NRR_FP32_DC && o->max_outer > 0 && outer >= o->max_outer) break;
    if (o->timeout_ms > 0 && elapsed_ms() > (double)o->timeout_ms) {
      why = NRR_ERR_TIMEOUT;
      break;
    }
    const int64_t m = std::min<int64_t>(every, o->max_iters - it);
    if (m == every) {
      cudaGraphExec_t exec = nullptr;
      s = chunk_graph(ps, o->mode, m, dt, eta, o->r_int, &exec);
      if (s != NRR_OK) return s;
      PCUDA(cudaGraphLaunch(exec, st));
    } else {  // a last, shorter chunk: launched one kernel at a time
      launch_chunk(ps, o->mode, m, dt, eta, o->r_int);
    }
    s = read_norm(ps, &nrm);
    if (s != NRR_OK) return s;
    it += m;
    outer++;
  }
  if (r) {
    r->iters = it;
    r->outer_iters = o->mode == NRR_FP32_DC ? outer : 0;
    r->final_norm = nrm;
    r->seconds = elapsed_ms() * 1e-3;
    r->status = why;
  }
  if (why == NRR_ERR_NOT_CONVERGED)
    return pfail(why, "patch set not converged after %lld steps (norm %.3e)",
                 (long long)it, nrm);
  if (why == NRR_ERR_DIVERGED)
    return pfail(why, "patch set residual not finite after %lld steps", (long long)it);
  if (why == NRR_ERR_TIMEOUT)
    return pfail(why, "patch set timeout after %lld steps", (long long)it);
  return NRR_OK;
}

}  // extern "C"
