// nrr_warm.cu -- warm starts from the surrogate: training targets out of a
// batch of coarse solves, and prolongation of a coarse-grid u onto a finer
// grid of the same coordinate family (trilinear in the coordinates xx).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/nrr.h"
#include "nrr_internal.h"

using namespace nrr;

namespace {

nrr_status wfail(nrr_status s, const char *fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}


// Coarse value at padded coarse indices (j0, j1, j2): inner ghosts through
// their images, points beyond the outer boundary clamped to the last
// interior xx0 plane.
__device__ double coarse_at(const Geo &c, const float *uc, int j0, int j1, int j2) {
  if (j0 >= c.n0 + c.ng) j0 = c.n0 + c.ng - 1;
  image_of(c, j0, j1, j2);
  // far ghosts of a much finer grid can reflect past the interior: clamp
  j0 = min(max(j0, c.ng), c.n0 + c.ng - 1);
  j1 = min(max(j1, c.ng), c.n1 + c.ng - 1);
  j2 = min(max(j2, c.ng), c.n2 + c.ng - 1);
  const int i0 = j0 - c.ng, i1 = j1 - c.ng, i2 = j2 - c.ng;
  return (double)uc[(int64_t)i0 + (int64_t)c.n0 * (i1 + (int64_t)c.n1 * i2)];
}

__global__ void prolong_kernel(Geo c, const float *__restrict__ uc, Geo f,
                               double *uf) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.npts) return;
  const int k0 = (int)(p % f.s0), k1 = (int)((p / f.s0) % f.s1),
            k2 = (int)(p / f.ncol);
  const int k[3] = {k0, k1, k2};
  int lo[3];
  double t[3];
  for (int d = 0; d < 3; d++) {
    const double xx = f.xxmin[d] + (k[d] - f.ng + 0.5) * f.dxx[d];
    const double fi = (xx - c.xxmin[d]) / c.dxx[d] - 0.5;  // interior-relative
    const double fl = floor(fi);
    lo[d] = (int)fl + c.ng;  // padded coarse index
    t[d] = fi - fl;
  }
  double acc = 0.0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++)
      for (int e = 0; e < 2; e++) {
        const double w = (a ? t[0] : 1.0 - t[0]) * (b ? t[1] : 1.0 - t[1]) *
                         (e ? t[2] : 1.0 - t[2]);
        acc += w * coarse_at(c, uc, lo[0] + a, lo[1] + b, lo[2] + e);
      }
  uf[p] = acc;
}

}  // namespace

extern "C" nrr_status nrr_prolong(const nrr_grid_desc *coarse, const float *uc,
                                  const nrr_grid_desc *fine, double *uf,
                                  void *stream) {
  if (!coarse || !fine || !uc || !uf) return wfail(NRR_ERR_INVALID_ARG, "null argument");
  if (coarse->coord != fine->coord || coarse->coord == NRR_CARTESIAN ||
      coarse->coord == NRR_SINHCYLINDRICAL)
    return wfail(NRR_ERR_INVALID_ARG,
                 "prolongation needs two SinhSymTP, Spherical or SinhSpherical grids");
  if (coarse->coord == NRR_SINHSYMTP &&
      (coarse->amax != fine->amax || coarse->bscale != fine->bscale ||
       coarse->sinhwaa != fine->sinhwaa))
    return wfail(NRR_ERR_INVALID_ARG, "SinhSymTP parameters differ");
  if (coarse->coord == NRR_SPHERICAL && coarse->rmax != fine->rmax)
    return wfail(NRR_ERR_INVALID_ARG, "rmax differs");
  if (coarse->coord == NRR_SINHSPHERICAL &&
      (coarse->amax != fine->amax || coarse->sinhwaa != fine->sinhwaa))
    return wfail(NRR_ERR_INVALID_ARG, "SinhSpherical parameters differ");
  for (const nrr_grid_desc *d : {coarse, fine}) {
    nrr_status s = check_grid_desc(d);
    if (s != NRR_OK) return s;
  }
  const Geo c = grid_geo(coarse), f = grid_geo(fine);
  if (f.npts > ((int64_t)1 << 31)) return wfail(NRR_ERR_INVALID_ARG, "fine grid too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prolong_kernel<<<(unsigned)((f.npts + 255) / 256), 256, 0, st>>>(c, uc, f, uf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wfail(NRR_ERR_CUDA, "prolong launch: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return wfail(NRR_ERR_CUDA, "prolong: %s", cudaGetErrorString(e));
  return NRR_OK;
}
