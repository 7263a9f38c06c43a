// nrr_async.cuh -- mbarriers and tensor (TMA) copies (global -> shared
// memory, completing on an mbarrier) for the stage kernels' plane pipeline.
//
// Every wait is bounded: a wait that expires returns false and the caller
// records an error and drains its copies in flight before the block exits.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace nrr {
namespace dev {

// try_wait polls before a wait gives up: about a second on sm_103a (a poll
// suspends ~4 us when the phase is incomplete); a healthy copy completes in
// microseconds.
constexpr long long kAsyncWaitLimit = 1ll << 18;

__device__ __forceinline__ uint32_t shared_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init_count(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(shared_addr(bar)),
               "r"(count)
               : "memory");
}

// Makes barrier initialisation visible to the async proxy (tensor copies).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also raises the barrier's expected transaction bytes.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   shared_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(shared_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity) {
  for (long long i = 0; i < kAsyncWaitLimit; i++)
    if (mbar_test_parity(bar, parity)) return true;
  return false;
}

// Ends an mbarrier object's life so that its word can be initialised again
// (a block that runs several tiles in one launch).
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(shared_addr(bar)) : "memory");
}

// Orders this thread's generic-proxy accesses of all state spaces against
// its async-proxy ones: global stores of one stage before the tensor copies
// that later read them in the same launch.
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy ones (a buffer read by the threads is refilled).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Tiled tensor copy of one box at coordinates (x, y, z) of a 3-D tensor map
// (a kernel parameter or in global memory) into shared memory, completing
// on `bar`.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map,
                                            uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(shared_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(shared_addr(bar)), "r"(x),
      "r"(y), "r"(z)
      : "memory");
}

// Tiled tensor copy of one box at coordinates (x, y, z, w) of a 4-D tensor
// map (in global memory, written before the launch) into shared memory,
// completing on `bar`.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map,
                                            uint64_t *bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(shared_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(shared_addr(bar)), "r"(x),
      "r"(y), "r"(z), "r"(w)
      : "memory");
}

constexpr long long kBarrierPolls = 1ll << 22;

// Arrive at barrier `target` (cumulative arrivals expected) and wait for
// every block; thread 0 of each block arrives after the block's writes.
__device__ __forceinline__ void grid_barrier(unsigned *count, unsigned target,
                                             int *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    // once any barrier has expired no later one waits, so a launch spends
    // at most one bounded wait before it drains
    const bool expired = err && *(volatile int *)err != 0;
    for (long long i = 0; !expired; i++) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (i > kBarrierPolls) {
        if (err) atomicExch(err, 1);
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
}

}  // namespace dev
}  // namespace nrr
