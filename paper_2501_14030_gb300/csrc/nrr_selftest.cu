// nrr_selftest.cu -- exercises the expiry path of the bounded waits that the
// stage kernels use (mbarrier phase waits for tensor copies, grid barriers of
// the multi-stage kernel): each wait here is on something that never
// happens, so it must give up, record the error and return, leaving the
// context usable.  No GPU fault is involved.
#include <cuda_runtime.h>

#include "../../include/nrr.h"
#include "nrr_async.cuh"
#include "nrr_internal.h"

using namespace nrr;

namespace {

// which = 0: an mbarrier phase that nothing completes (no arrival, no copy).
// which = 1: a grid barrier that expects one arrival more than the grid has.
__global__ void wait_expiry_kernel(int which, unsigned *count, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (which == 0) {
    if (threadIdx.x == 0) {
      dev::mbar_init_count(&bar, 1);
      dev::mbar_init_fence();
    }
    __syncthreads();
    const bool ok = dev::mbar_wait_parity(&bar, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  } else {
    dev::grid_barrier(count, gridDim.x + 1, err);
  }
}

}  // namespace

extern "C" nrr_status nrr_selftest_wait_expiry(int which, void *stream,
                                               int *expired) {
  if ((which != 0 && which != 1) || !expired) {
    set_last_error("nrr_selftest_wait_expiry: which must be 0 or 1, expired non-null");
    return NRR_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_OOM;
  }
  int h[2] = {0, 0};
  e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) {
    wait_expiry_kernel<<<which == 0 ? 1 : 2, 32, 0, st>>>(
        which, reinterpret_cast<unsigned *>(d + 1), d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_CUDA;
  }
  *expired = h[0];
  return NRR_OK;
}
