// nrr_selftest.cu -- exercises the expiry path of the bounded waits that the
// stage kernels use (mbarrier phase waits for tensor copies, grid barriers of
// the multi-stage kernel): each wait here is on something that never
// happens, so it must give up, record the error and return, leaving the
// context usable.  No GPU fault is involved.
//
// It also holds two measurement hooks: the stage kernels' reciprocal over a
// caller's array (tested against correctly rounded division), and peak
// probes (FP64/FP32 FMA throughput, L2 read bandwidth) for the rooflines.
#include <cuda_runtime.h>

#include "../../include/nrr.h"
#include "nrr_async.cuh"
#include "nrr_internal.h"
#include "nrr_stencil.cuh"

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

template <typename R>
__global__ void recip_kernel(const R *__restrict__ s, R *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = dev::recip(s[i]);
}

// FMA throughput: kChains independent accumulators per thread, so that the
// pipe, not the latency of one chain, sets the rate.  The values stay near 1
// (multiplier just below 1, small addend), so no denormal or overflow slows
// the pipe; the sum is stored only under a condition the compiler cannot
// decide, which keeps the work alive.
constexpr int kChains = 8;
template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, R mul, R add,
                                                       R *sink) {
  R a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = R(1) + R(threadIdx.x + j) * R(1e-6);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = fma(a[j], mul, add);
  }
  R t = R(0);
#pragma unroll
  for (int j = 0; j < kChains; j++) t += a[j];
  if (t == R(-1)) sink[blockIdx.x] = t;
}

// L2 read bandwidth: every thread reads 16-byte words of a buffer that fits
// in L2, grid-stride, `reps` times over.
__global__ void __launch_bounds__(512) l2_probe_kernel(const float4 *__restrict__ buf,
                                                      int64_t n, int reps,
                                                      float *sink) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == -1.f) sink[blockIdx.x] = acc;
}

}  // namespace

extern "C" nrr_status nrr_selftest_recip(const void *s, void *out, int64_t n,
                                         int fp32, void *stream) {
  if (!s || !out || n < 0 || (fp32 != 0 && fp32 != 1)) {
    set_last_error("nrr_selftest_recip: null pointer, n < 0 or fp32 not 0/1");
    return NRR_ERR_INVALID_ARG;
  }
  if (n == 0) return NRR_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (fp32)
    recip_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(s),
                                                static_cast<float *>(out), n);
  else
    recip_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(s),
                                                 static_cast<double *>(out), n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_CUDA;
  }
  return NRR_OK;
}

namespace {

// Best of `reps` event-timed runs of launch(), in milliseconds.
template <typename F>
cudaError_t best_ms(cudaStream_t st, int reps, F launch, float *best) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  *best = 1e30f;
  launch();  // warm-up (clocks, L2 contents)
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    e = cudaEventRecord(e0, st);
    launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < *best) *best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" nrr_status nrr_probe_peaks(int64_t l2_bytes, void *stream,
                                      double *fp64_tflops, double *fp32_tflops,
                                      double *l2_gbs) {
  if (l2_bytes == 0) l2_bytes = (int64_t)48 << 20;
  if (l2_bytes < (1 << 20) || l2_bytes > ((int64_t)1 << 32)) {
    set_last_error("nrr_probe_peaks: l2_bytes must be 0 or in [1 MiB, 4 GiB]");
    return NRR_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_CUDA;
  }
  const int64_t n4 = l2_bytes / 16;
  float4 *buf = nullptr;
  float *sink = nullptr;
  e = cudaMalloc(&buf, (size_t)n4 * 16);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_OOM;
  }
  e = cudaMalloc(&sink, 1 << 20);
  if (e != cudaSuccess) {
    cudaFree(buf);
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_OOM;
  }
  e = cudaMemsetAsync(buf, 0, (size_t)n4 * 16, st);
  // FMA probes: 8 blocks of 256 threads per SM (full occupancy), 8 chains of
  // `iters` FMAs per thread
  const int fblocks = sms * 8, iters = 8192;
  const double fma_flops = 2.0 * kChains * (double)iters * fblocks * 256;
  float ms64 = 0.f, ms32 = 0.f, msl2 = 0.f;
  if (e == cudaSuccess)
    e = best_ms(st, 5, [&] {
      fma_probe_kernel<double><<<fblocks, 256, 0, st>>>(iters, 0.9999999, 1e-7,
                                                        reinterpret_cast<double *>(sink));
    }, &ms64);
  if (e == cudaSuccess)
    e = best_ms(st, 5, [&] {
      fma_probe_kernel<float><<<fblocks, 256, 0, st>>>(iters * 16, 0.9999f, 1e-4f, sink);
    }, &ms32);
  const int reps = 20, lblocks = sms * 4;
  if (e == cudaSuccess)
    e = best_ms(st, 5, [&] {
      l2_probe_kernel<<<lblocks, 512, 0, st>>>(buf, n4, reps, sink);
    }, &msl2);
  cudaFree(buf);
  cudaFree(sink);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return NRR_ERR_CUDA;
  }
  if (fp64_tflops) *fp64_tflops = fma_flops / (ms64 * 1e-3) / 1e12;
  if (fp32_tflops) *fp32_tflops = 16.0 * fma_flops / (ms32 * 1e-3) / 1e12;
  if (l2_gbs) *l2_gbs = (double)reps * n4 * 16 / (msl2 * 1e-3) / 1e9;
  return NRR_OK;
}

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
