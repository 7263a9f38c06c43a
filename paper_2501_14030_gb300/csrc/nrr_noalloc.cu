// nrr_noalloc.cu -- a residual-norm entry point that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc: an application whose own memory
// manager has taken the whole device and grants no further allocations, an
// embedding whose policy forbids allocation calls after start-up (they can
// synchronise the device and fail under a fixed budget), or a plug-in that
// is handed only the buffers it must read and write.  For them,
// nrr_residual_noalloc evaluates the residual H of a caller-owned u and its
// L2 norm without a grid object: the geometry and the Bowen-York source are
// recomputed per point, and the only scratch -- the per-block partial sums of
// the norm -- lives in the file-scope array below, which every GPU that loads
// the library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/nrr.h"
#include "nrr_common.cuh"
#include "nrr_internal.h"

namespace {

// Partial sums (H^2 J, J) of one block each: 2 doubles per block.
constexpr int kMaxBlocks = 32768;  // 512 KiB of scratch per device
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks];

nrr_status fail(nrr_status s, const char *fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  nrr::set_last_error(buf);  // reported by nrr_last_error()
  return s;
}

// Device address of the scratch array, looked up once per device with that
// device current.  The host-side symbol is only a stand-in and must never be
// passed to a kernel.  The address belongs to the device's context: it is
// remembered together with that context, and looked up again when the
// current context differs (after cudaDeviceReset, for instance, the runtime
// creates a new primary context and reloads the module).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

cudaError_t scratch_for_device(int dev, double **out) {
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  // No context current yet on this thread (ctx null), a context other than
  // the remembered one, or no lookup so far: look the address up.  The
  // lookup itself makes the device's primary context current.
  if (!g_scratch_ptr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!get || get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    g_scratch_ptr[dev] = static_cast<double *>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct Punctures {
  int n;
  double m[8], x[8][3], P[8][3], S[8][3];
};
struct FdWeights {
  double w1[6], w2[6];  // k = 0..ng
};

// lap(u) + beta (1 + alpha u)^-7 at one interior point, everything
// recomputed from the coordinate map and the punctures: scale factors and
// the Laplacian's first-derivative terms of the orthogonal reference metric,
// centred FD of the grid's order, Bowen-York curvature.
template <int NG>
__device__ double residual_point(const nrr::Geo &g, const Punctures &pz,
                                 const FdWeights &fw, const double *u,
                                 int i0, int i1, int i2, double *weight,
                                 double r_int) {
  using namespace nrr;
  double xx[3];
  int ii[3] = {i0, i1, i2};
  for (int d = 0; d < 3; d++) xx[d] = g.xxmin[d] + (ii[d] - NG + 0.5) * g.dxx[d];
  double h[3], gl[3] = {0.0, 0.0, 0.0}, X[3], r, J;
  if (g.coord == CARTESIAN) {
    h[0] = h[1] = h[2] = 1.0;
    X[0] = xx[0];
    X[1] = xx[1];
    X[2] = xx[2];
    r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    J = 1.0;
  } else {
    double st, ct, sp, cp;
    sincos(xx[1], &st, &ct);
    sincos(xx[2], &sp, &cp);
    if (g.coord == SINHSYMTP) {
      double w = g.sinhwaa, b = g.bscale, sh1 = sinh(1.0 / w);
      double A = g.amax * sinh(xx[0] / w) / sh1;
      double Ap = g.amax * cosh(xx[0] / w) / (w * sh1);
      double App = A / (w * w);
      double Z2 = A * A + b * b, V2 = A * A + b * b * st * st;
      h[0] = Ap * sqrt(V2 / Z2);
      h[1] = sqrt(V2);
      h[2] = A * st;
      gl[0] = (Z2 + A * A - A * Z2 * App / (Ap * Ap)) / (Ap * A * V2);
      gl[1] = ct / (st * V2);
      X[0] = A * st * cp;
      X[1] = A * st * sp;
      X[2] = sqrt(Z2) * ct;
    } else {
      double rr = xx[0];
      h[0] = 1.0;
      h[1] = rr;
      h[2] = rr * st;
      gl[0] = 2.0 / rr;
      gl[1] = ct / (rr * rr * st);
      X[0] = rr * st * cp;
      X[1] = rr * st * sp;
      X[2] = rr * ct;
    }
    r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    J = fabs(h[0] * h[1] * h[2]);
  }
  *weight = r < r_int ? J : 0.0;

  const int64_t p = flat(g, i0, i1, i2);
  const double u0 = u[p];
  double lap = 0.0;
  for (int d = 0; d < 3; d++) {
    double d2 = fw.w2[0] * u0, d1 = 0.0;
    for (int k = 1; k <= NG; k++) {
      int jp[3] = {i0, i1, i2}, jm[3] = {i0, i1, i2};
      jp[d] += k;
      jm[d] -= k;
      if (g.coord != CARTESIAN) {
        image_of(g, jp[0], jp[1], jp[2]);
        image_of(g, jm[0], jm[1], jm[2]);
      }
      double up = u[flat(g, jp[0], jp[1], jp[2])];
      double um = u[flat(g, jm[0], jm[1], jm[2])];
      d2 += fw.w2[k] * (up + um);
      d1 += fw.w1[k] * (up - um);
    }
    double inv = 1.0 / g.dxx[d];
    lap += d2 * inv * inv / (h[d] * h[d]) + gl[d] * d1 * inv;
  }

  double A6[6] = {0, 0, 0, 0, 0, 0};
  double psi = 1.0;
  for (int a = 0; a < pz.n; a++) {
    double dx[3] = {X[0] - pz.x[a][0], X[1] - pz.x[a][1], X[2] - pz.x[a][2]};
    double ra = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
    double n[3] = {dx[0] / ra, dx[1] / ra, dx[2] / ra};
    const double *P = pz.P[a], *S = pz.S[a];
    double Pn = P[0] * n[0] + P[1] * n[1] + P[2] * n[2];
    double q[3] = {S[1] * n[2] - S[2] * n[1], S[2] * n[0] - S[0] * n[2],
                   S[0] * n[1] - S[1] * n[0]};
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ja[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
      int i = ia[c], j = ja[c];
      double delta = i == j ? 1.0 : 0.0;
      A6[c] += 1.5 / (ra * ra) * (P[i] * n[j] + P[j] * n[i] - (delta - n[i] * n[j]) * Pn) +
               3.0 / (ra * ra * ra) * (q[i] * n[j] + q[j] * n[i]);
    }
    psi += pz.m[a] / (2.0 * ra);
  }
  double aa = A6[0] * A6[0] + A6[1] * A6[1] + A6[2] * A6[2] +
              2.0 * (A6[3] * A6[3] + A6[4] * A6[4] + A6[5] * A6[5]);
  double alpha = 1.0 / psi;
  double beta = 0.125 * aa * pow(alpha, 7.0);
  return lap + beta * pow(1.0 + alpha * u0, -7.0);
}

template <int NG>
__global__ void __launch_bounds__(128)
    residual_noalloc_kernel(nrr::Geo g, Punctures pz, FdWeights fw,
                            const double *__restrict__ u, double r_int,
                            double *h_out, double *scratch, int zc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (e < g.n0 * g.n1) {
    const int i0 = e % g.n0 + NG, i1 = e / g.n0 + NG;
    const int z0 = NG + blockIdx.y * zc, z1 = min(z0 + zc, NG + g.n2);
    for (int i2 = z0; i2 < z1; i2++) {
      double w;
      double H = residual_point<NG>(g, pz, fw, u, i0, i1, i2, &w, r_int);
      if (h_out) h_out[nrr::flat(g, i0, i1, i2)] = H;
      num = fma(H * H, w, num);
      den += w;
    }
  }
  // Fixed-order block sum; every block writes its own two slots, so no slot
  // read by the finalize kernel keeps a value from an earlier call.
  __shared__ double sx[4], sy[4];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sx[threadIdx.x >> 5] = num;
    sy[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int blk = blockIdx.x + gridDim.x * blockIdx.y;
    scratch[2 * blk] = sx[0] + sx[1] + sx[2] + sx[3];
    scratch[2 * blk + 1] = sy[0] + sy[1] + sy[2] + sy[3];
  }
}

__global__ void noalloc_finalize_kernel(const double *scratch, int nblocks,
                                        double *norm_out) {
  __shared__ double sx[256], sy[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    x += scratch[2 * i];
    y += scratch[2 * i + 1];
  }
  sx[threadIdx.x] = x;
  sy[threadIdx.x] = y;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sx[threadIdx.x] += sx[threadIdx.x + s];
      sy[threadIdx.x] += sy[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) norm_out[0] = sy[0] > 0.0 ? sqrt(sx[0] / sy[0]) : 0.0;
}

}  // namespace

extern "C" nrr_status nrr_residual_noalloc(const nrr_grid_desc *d, int npunct,
                                           const nrr_puncture *p,
                                           const double *u, double r_int,
                                           double *norm_out, double *h_out,
                                           void *stream) {
  using namespace nrr;
  if (!d || !p || !u || !norm_out)
    return fail(NRR_ERR_INVALID_ARG, "null argument");
  {
    nrr_status s = check_grid_desc(d);  // the check every entry point shares
    if (s != NRR_OK) return s;
  }
  if (d->coord == NRR_SINHSPHERICAL || d->coord == NRR_SINHCYLINDRICAL)
    return fail(NRR_ERR_INVALID_ARG,
                "the allocation-free residual takes SinhSymTP, Spherical or Cartesian grids");
  if (npunct < 1 || npunct > 8)
    return fail(NRR_ERR_INVALID_ARG, "need 1..8 punctures (got %d)", npunct);
  if (!(r_int > 0.0)) return fail(NRR_ERR_INVALID_ARG, "r_int must be positive");
  const int ng = d->fd_order / 2;
  const Geo g = grid_geo(d);
  if (g.npts > ((int64_t)1 << 31))
    return fail(NRR_ERR_INVALID_ARG, "grid exceeds 2^31 points");

  // Launch shape: 128 columns per block in x; phi planes per thread chosen
  // so that the block count fits the static scratch.
  // (64-bit products: n0 and n1 may each be up to 65536.)
  const int64_t ncols = (int64_t)g.n0 * g.n1;
  const int64_t bx64 = (ncols + 127) / 128;
  if (bx64 > kMaxBlocks)
    return fail(NRR_ERR_INVALID_ARG,
                "n0*n1 = %lld needs %lld partial sums; the static scratch holds %d",
                (long long)ncols, (long long)bx64, kMaxBlocks);
  const int bx = (int)bx64;  // 1 <= bx <= kMaxBlocks
  int by_max = kMaxBlocks / bx;
  int zc = (g.n2 + by_max - 1) / by_max;
  if (zc < 1) zc = 1;
  int by = (g.n2 + zc - 1) / zc;
  int nblocks = bx * by;

  Punctures pz{};
  pz.n = npunct;
  for (int a = 0; a < npunct; a++) {
    if (!(p[a].m > 0.0)) return fail(NRR_ERR_INVALID_ARG, "puncture mass must be positive");
    pz.m[a] = p[a].m;
    for (int k = 0; k < 3; k++) {
      pz.x[a][k] = p[a].x[k];
      pz.P[a][k] = p[a].P[k];
      pz.S[a][k] = p[a].S[k];
    }
  }
  FdWeights fw{};
  for (int k = 0; k <= ng; k++) {
    fw.w1[k] = k == 0 ? 0.0 : fd_first(ng, k);
    fw.w2[k] = fd_second(ng, k);
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NRR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(NRR_ERR_CUDA, "device index %d", dev);
  double *scratch = nullptr;
  e = scratch_for_device(dev, &scratch);
  if (e != cudaSuccess)
    return fail(NRR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid(bx, by);
  switch (ng) {
    case 2: residual_noalloc_kernel<2><<<grid, 128, 0, st>>>(g, pz, fw, u, r_int, h_out, scratch, zc); break;
    case 4: residual_noalloc_kernel<4><<<grid, 128, 0, st>>>(g, pz, fw, u, r_int, h_out, scratch, zc); break;
    default: residual_noalloc_kernel<5><<<grid, 128, 0, st>>>(g, pz, fw, u, r_int, h_out, scratch, zc); break;
  }
  noalloc_finalize_kernel<<<1, 256, 0, st>>>(scratch, nblocks, norm_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NRR_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  return NRR_OK;
}
