// nrr_gemm.cu -- BF16 tensor-core GEMM on sm_103a (tcgen05 + TMA + TMEM) for
// the surrogate network: D[M,N] (FP32) = sum_k A[m,k] B[n,k], both operands
// K-major BF16 in global memory.
//
// One CTA computes a 128 x BN tile (BN = 64, 128 or 256) over a range of K.
// Warp 0 (one lane) streams 128x64 and BNx64 operand tiles into a shared-
// memory ring (3 stages for BN <= 128, two CTAs per SM; 4 stages for
// BN = 256, one CTA per SM) with TMA (128-byte swizzle); warp 1 (one lane)
// issues tcgen05.mma (M=128, N=BN, K=16 per instruction) into an FP32
// accumulator in tensor memory and releases each stage with tcgen05.commit;
// then all four warps read the accumulator back with tcgen05.ld (warp w owns
// rows 32w..32w+31) and store it.  Split-K: blockIdx.z takes one of S equal
// ranges of K and writes its partial tile to slice z of a workspace, and a
// second kernel sums the S slices in a fixed order (deterministic).  Every
// mbarrier wait is bounded: on expiry the kernel records an error in a device
// flag, skips the remaining work, frees its tensor memory and returns; the
// flag is read back only when the caller asks (nrr_gemm_status).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/nrr.h"
#include "nrr_internal.h"

namespace nrr {

namespace {

constexpr int BM = 128, BK = 64;
// Pipeline depth: for BN <= 128 three 128 x 64 + BN x 64 stages leave room
// for two CTAs per SM (one CTA's epilogue overlaps another's main loop); the
// 48 KB stages of BN = 256 take four and one CTA per SM.  The freed stages
// hold the accumulator tile for the coalesced store.
template <int BN>
__host__ __device__ constexpr int gemm_stages() { return BN == 256 ? 4 : 3; }
template <int BN>
__host__ __device__ constexpr int gemm_smem() {
  return gemm_stages<BN>() * (BM * BK * 2 + BN * BK * 2) + 1024 + 256;
}
constexpr long long kWaitLimit = 1ll << 18;  // try_wait polls (about a second)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on one phase of an mbarrier; false (and *err set) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          int *err, int code) {
  for (long long i = 0; i < kWaitLimit; i++)
    if (mbar_try(bar, parity)) return true;
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map,
                                            uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 64 BF16 (128 B), 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major.
template <int N>
__device__ __forceinline__ uint32_t mma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

// D + z * split_stride receives the partial product over K range z of
// gridDim.z (the whole K when gridDim.z == 1).
template <int BN>
__global__ void __launch_bounds__(128, BN == 256 ? 1 : 2)
    gemm_bf16_tn_kernel(const __grid_constant__ CUtensorMap map_a,
                        const __grid_constant__ CUtensorMap map_b, float *D,
                        int M, int K, int ldd, int64_t split_stride, int *err) {
  constexpr int STAGES = gemm_stages<BN>();
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  static_assert((size_t)BM * (BN + 4) * 4 <= (size_t)STAGES * (A_BYTES + B_BYTES),
                "the epilogue's row staging must fit in the pipeline buffers");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *done = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *issued = reinterpret_cast<int *>(tmem_slot + 1);  // k-blocks loaded

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // K range of this split: k-blocks kb0 .. kb0 + nk - 1 (nk >= 1, the host
  // keeps gridDim.z <= K / BK)
  const int nk_all = K / BK;
  const int kb0 = (int)((int64_t)nk_all * blockIdx.z / gridDim.z);
  const int nk = (int)((int64_t)nk_all * (blockIdx.z + 1) / gridDim.z) - kb0;
  D += (int64_t)blockIdx.z * split_stride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_addr(tmem_slot)),
        "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; kb++) {
      const int s = kb % STAGES;
      if (kb >= STAGES &&
          !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, err, 1))
        break;
      mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, &map_a, &full[s], (kb0 + kb) * BK, m0);
      tma_load_2d(sB + s * B_BYTES, &map_b, &full[s], (kb0 + kb) * BK, n0);
      *issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = mma_idesc<BN>();
    bool ok = true;
    for (int kb = 0; kb < nk && ok; kb++) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1, err, 2)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = sw128_desc(smem_addr(sA + s * A_BYTES));
      const uint64_t db = sw128_desc(smem_addr(sB + s * B_BYTES));
#pragma unroll
      for (int k = 0; k < BK / 16; k++) {
        // +32 bytes along K per instruction (encoded >> 4)
        const uint64_t off = (uint64_t)(k * 2);
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                tmem),
            "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
          "[%0];" ::"r"(smem_addr(&empty[s]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
        "[%0];" ::"r"(smem_addr(done))
        : "memory");
  }
  __syncwarp();

  // Epilogue: accumulator rows 32*warp + lane, BN columns.  Each warp moves
  // its 32 rows from tensor memory into the (now idle) pipeline buffers, one
  // row per thread, then stores them row by row with the whole warp, so that
  // every global store is a contiguous run of the output row.  Row stride
  // BN + 4 floats keeps both shared-memory passes free of bank conflicts.
  const bool ready = mbar_wait(done, 0, err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // tcgen05.ld is warp-collective: decide per warp, not per thread
  if (__all_sync(0xffffffffu, ready && *((volatile int *)err) == 0)) {
    constexpr int LDS = BN + 4;
    float *stage = reinterpret_cast<float *>(smem) + (size_t)32 * warp * LDS;
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int c = 0; c < BN; c += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, "
          "%7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
            "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
            "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15])
          : "r"(taddr + (uint32_t)c));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float4 *srow = reinterpret_cast<float4 *>(stage + lane * LDS + c);
#pragma unroll
      for (int q = 0; q < 4; q++)
        srow[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                              __uint_as_float(r[4 * q + 2]),
                              __uint_as_float(r[4 * q + 3]));
    }
    __syncwarp();
    for (int rr = 0; rr < 32; rr++) {
      const int row = m0 + 32 * warp + rr;
      if (row >= M) break;
      const float4 *src = reinterpret_cast<const float4 *>(stage + rr * LDS);
      float4 *dst = reinterpret_cast<float4 *>(D + (int64_t)row * ldd + n0);
#pragma unroll
      for (int c4 = lane; c4 < BN / 4; c4 += 32) dst[c4] = src[c4];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // No copy may still be landing in this CTA's shared memory when it exits:
    // wait (bounded) for the last phase issued on every stage.
    const int n_iss = *issued;
    for (int kb = n_iss - STAGES < 0 ? 0 : n_iss - STAGES; kb < n_iss; kb++)
      mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, err, 4);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(BN));
}

// ---- persistent variant (many output tiles, no K split) -------------------
//
// One CTA per SM walks the output tiles t = blockIdx.x, + gridDim.x, ...
// (N-tiles fastest, so the CTAs of a wave share the rows of A and stream all
// of B through L2).  Roles: warp 0 lane 0 loads operand stages with TMA into
// a ring that runs across tiles; warp 1 lane 0 issues the MMAs of tile i into
// accumulator buffer i % 2 of tensor memory (2 x BN columns); warps 2-5 read
// the other buffer back (tcgen05.ld, warp w owns TMEM lanes 32 (w % 4) ..
// + 31), write 32 x 32 FP32 boxes into 128-byte-swizzled staging buffers and
// store them with TMA, so a tile's epilogue overlaps the next tile's main
// loop.  Barriers: full/empty per ring stage, acc_full (MMA commit) and
// acc_empty (four epilogue warps) per accumulator buffer.  Every wait is
// bounded; on expiry the kernel records an error, every role stops, copies
// in flight are allowed to land and tensor memory is freed.
constexpr int PST_STAGES = 4;
constexpr int PST_THREADS = 192;
template <int BN>
__host__ __device__ constexpr int pst_smem() {
  return PST_STAGES * (BM * BK * 2 + BN * BK * 2) + 4 * 2 * 4096 + 1024 + 256;
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src,
                                             int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_addr(src)), "r"(x), "r"(y)
      : "memory");
}

// Tensor copy into the same CTA-relative shared-memory offset of every CTA in
// `mask` of this cluster, completing bytes on the mbarrier at the same
// offset in each of them.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map,
                                               uint64_t *bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// CL = 1: one CTA per SM walks the output tiles.  CL = 2: clusters of two CTAs
// walk pairs of vertically adjacent tiles (rows m0 and m0 + 128, the same
// columns): each CTA loads its own A rows and half of the shared B tile,
// multicast into both CTAs' rings, so B is read from L2 once per pair; a
// ring stage is refilled when both CTAs' MMAs have released it (the MMA
// commit arrives on the empty barriers of both), and the cluster meets at
// a barrier after set-up (no copy before the peer's barriers exist) and
// before exit (no copy into a CTA that has left).  map_b's box is BN / CL
// rows.
template <int BN, int CL>
__global__ void __launch_bounds__(PST_THREADS, 1)
    gemm_bf16_tn_persistent_kernel(const __grid_constant__ CUtensorMap map_a,
                                   const __grid_constant__ CUtensorMap map_b,
                                   const __grid_constant__ CUtensorMap map_d, int M,
                                   int N, int K, int *err) {
  static_assert(CL == 1 || CL == 2, "clusters of one or two CTAs");
  constexpr int STAGES = PST_STAGES;
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_BYTES;
  uint8_t *sOut = sB + STAGES * B_BYTES;  // 4 warps x 2 buffers x 4 KB
  uint64_t *full = reinterpret_cast<uint64_t *>(sOut + 4 * 2 * 4096);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *mma_done = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
  int *issued = reinterpret_cast<int *>(tmem_slot + 1);  // k-blocks loaded
  int *abort_flag = issued + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = N / BN, nk = K / BK;
  // work units: tiles (CL = 1) or vertical tile pairs (CL = 2), walked by
  // CTAs (or clusters) in steps of their number
  const int rank = CL == 2 ? (int)cluster_rank() : 0;
  const int units = ntn * (M / BM / CL), unit0 = blockIdx.x / CL,
            ustep = gridDim.x / CL;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CL);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(mma_done, 1);
    *issued = 0;
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_addr(tmem_slot)),
        "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if constexpr (CL == 2) cluster_sync();  // the peer's barriers exist
  const uint32_t tmem = *tmem_slot;
  volatile int *vabort = abort_flag;
  // the output tile of work unit u for this CTA
  auto tile_m0 = [&](int u) { return ((u / ntn) * CL + rank) * BM; };
  auto tile_n0 = [&](int u) { return (u % ntn) * BN; };

  if (warp == 0 && lane == 0) {
    // TMA producer: k-block g (counted over all of this CTA's tiles) goes
    // to stage g % STAGES
    int g = 0;
    for (int u = unit0; u < units && !*vabort; u += ustep) {
      const int m0 = tile_m0(u), n0 = tile_n0(u);
      for (int kb = 0; kb < nk && !*vabort; kb++, g++) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, err, 11)) {
          *vabort = 1;
          break;
        }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sA + s * A_BYTES, &map_a, &full[s], kb * BK, m0);
        if constexpr (CL == 2)
          tma_load_2d_mc(sB + s * B_BYTES + rank * (B_BYTES / 2), &map_b, &full[s],
                         kb * BK, n0 + rank * (BN / 2), (uint16_t)0x3);
        else
          tma_load_2d(sB + s * B_BYTES, &map_b, &full[s], kb * BK, n0);
        *issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: tile i of this CTA into accumulator buffer i % 2
    const uint32_t idesc = mma_idesc<BN>();
    int g = 0, i = 0;
    bool ok = true;
    for (int u = unit0; u < units && ok; u += ustep, i++) {
      const int buf = i & 1;
      if (i >= 2 && !mbar_wait(&acc_empty[buf], ((i >> 1) - 1) & 1, err, 12)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dtm = tmem + (uint32_t)(buf * BN);
      for (int kb = 0; kb < nk; kb++, g++) {
        const int s = g % STAGES;
        if (*vabort || !mbar_wait(&full[s], (g / STAGES) & 1, err, 13)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t da = sw128_desc(smem_addr(sA + s * A_BYTES));
        const uint64_t db = sw128_desc(smem_addr(sB + s * B_BYTES));
#pragma unroll
        for (int k = 0; k < BK / 16; k++) {
          const uint64_t off = (uint64_t)(k * 2);
          const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
              "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc));
        }
        if constexpr (CL == 2)
          // release the stage in both CTAs: the peer refills its half of B
          // in this CTA's ring too
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster"
              ".multicast::cluster.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])),
              "h"((uint16_t)0x3)
              : "memory");
        else
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
              "[%0];" ::"r"(smem_addr(&empty[s]))
              : "memory");
      }
      if (!ok) break;
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
          "[%0];" ::"r"(smem_addr(&acc_full[buf]))
          : "memory");
    }
    if (!ok) *vabort = 1;
    // every MMA issued so far has completed once this barrier flips
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
        "[%0];" ::"r"(smem_addr(mma_done))
        : "memory");
  } else if (warp >= 2) {
    // Epilogue: TMEM lanes 32 q .. 32 q + 31 are output rows m0 + 32 q + lane
    const int q = warp & 3;
    uint8_t *stg0 = sOut + (warp - 2) * 2 * 4096;
    int nst = 0;  // boxes stored by this warp (staging buffer nst % 2)
    int i = 0;
    for (int u = unit0; u < units; u += ustep, i++) {
      const int buf = i & 1;
      const bool ready = mbar_wait(&acc_full[buf], (i >> 1) & 1, err, 14);
      if (!__all_sync(0xffffffffu, ready && !*vabort)) {
        if (lane == 0) *vabort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = tile_m0(u), n0 = tile_n0(u);
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN);
#pragma unroll 1
      for (int c = 0; c < BN; c += 32, nst++) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
            "%8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, "
            "%23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
              "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
              "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr + (uint32_t)c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // the staging buffer written two boxes ago must have been read out
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        uint8_t *stg = stg0 + (nst & 1) * 4096;
        // row `lane`, 16-byte chunk j at (j ^ (lane & 7)): the 128-byte
        // swizzle of the output tensor map
#pragma unroll
        for (int j = 0; j < 8; j++)
          *reinterpret_cast<uint4 *>(stg + lane * 128 + ((j ^ (lane & 7)) << 4)) =
              make_uint4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&map_d, stg, n0 + c, m0 + 32 * q);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      // this warp has read its lanes of buffer buf
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                      smem_addr(&acc_empty[buf]))
                                  : "memory");
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // no copy may still be landing in shared memory, and no MMA may still
    // be writing tensor memory, when the CTA frees them and exits
    const int n_iss = *issued;
    for (int g = n_iss - STAGES < 0 ? 0 : n_iss - STAGES; g < n_iss; g++)
      mbar_wait(&full[g % STAGES], (g / STAGES) & 1, err, 15);
    mbar_wait(mma_done, 0, err, 16);
  }
  __syncthreads();
  // no CTA leaves while its peer may still copy into it
  if constexpr (CL == 2) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * BN));
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t,
                              void *, const cuuint64_t *, const cuuint64_t *,
                              const cuuint32_t *, const cuuint32_t *,
                              CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  return reinterpret_cast<EncodeFn>(tensor_map_encoder());
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, looked up once; null if the driver
// does not provide it.
void *tensor_map_encoder() {
  static void *fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = p;
  });
  return fn;
}

namespace {

// Tensor map of a row-major [rows][cols] BF16 matrix read in tiles of
// box_rows x 64 with 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *base, int rows, int cols,
              int box_rows) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base),
             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a row-major [rows][ld] FP32 matrix (cols used) written in
// 32 x 32 boxes with 128-byte swizzle (the persistent kernel's output).
bool make_out_map(CUtensorMap *m, const void *base, int rows, int cols, int ld) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// kind 0: BF16 operand map (box rows x 64); kind 1: FP32 output map (box
// 32 x 32, row stride `box` elements)
struct MapKey {
  const void *p;
  int rows, cols, box, kind;
  bool operator<(const MapKey &o) const {
    return std::tie(p, rows, cols, box, kind) <
           std::tie(o.p, o.rows, o.cols, o.box, o.kind);
  }
};
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_maps;

bool cached_map(CUtensorMap *out, const void *base, int rows, int cols, int box,
                int kind = 0) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  MapKey k{base, rows, cols, box, kind};
  auto it = g_maps.find(k);
  if (it != g_maps.end()) {
    *out = it->second;
    return true;
  }
  CUtensorMap m;
  if (!(kind == 0 ? make_map(&m, base, rows, cols, box)
                  : make_out_map(&m, base, rows, cols, box)))
    return false;
  g_maps[k] = m;
  *out = m;
  return true;
}

int *g_err = nullptr;
std::once_flag g_err_once;

// Sum of the S split-K slices ws[z][m][n] (row stride N) into D[m][n] (row
// stride ldd), in the order z = 0 .. S-1; four columns per thread.
__global__ void splitk_reduce_kernel(const float4 *__restrict__ ws, float *D,
                                     int M, int N, int ldd, int S) {
  const int64_t n4 = N / 4, total = (int64_t)M * n4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 acc = ws[i];
    for (int z = 1; z < S; z++) {
      const float4 v = ws[(int64_t)z * total + i];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    const int64_t m = i / n4, c = i - m * n4;
    reinterpret_cast<float4 *>(D + m * ldd)[c] = acc;
  }
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    return 1;
  return sms;
}

template <int BN>
cudaError_t launch_gemm(const CUtensorMap &ma, const CUtensorMap &mb, float *D,
                        int M, int N, int K, int ldd, int splits,
                        int64_t split_stride, cudaStream_t st) {
  constexpr int smem = gemm_smem<BN>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tn_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(N / BN, M / BM, splits);
  gemm_bf16_tn_kernel<BN><<<grid, 128, smem, st>>>(ma, mb, D, M, K, ldd, split_stride,
                                                  g_err);
  return cudaGetLastError();
}

template <int BN, int CL>
cudaError_t launch_gemm_persistent(const CUtensorMap &ma, const CUtensorMap &mb,
                                   const CUtensorMap &md, int M, int N, int K,
                                   int ctas, cudaStream_t st) {
  constexpr int smem = pst_smem<BN>();
  auto kern = gemm_bf16_tn_persistent_kernel<BN, CL>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t c = {};
  c.gridDim = dim3(ctas);
  c.blockDim = dim3(PST_THREADS);
  c.dynamicSmemBytes = smem;
  c.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  c.attrs = at;
  c.numAttrs = CL > 1 ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&c, kern, ma, mb, md, M, N, K, g_err);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

int *gemm_error_flag() {
  std::call_once(g_err_once, [] {
    if (cudaMalloc(&g_err, sizeof(int)) == cudaSuccess) cudaMemset(g_err, 0, sizeof(int));
  });
  return g_err;
}

// Kernel, tile width and K splits for a shape, each where the caller passed
// 0 (persistent: -1), as measured on GB300 at the surrogate's shapes:
// - more 128 x 128 output tiles than SMs and no K split: the persistent
//   kernel (the epilogue of one tile overlaps the next tile's main loop),
//   256 wide when that divides N, else 128 (else 64);
// - few output tiles and a long K (K / 64 >= 32): 128 wide (64 if it does
//   not divide N) and K split into about one CTA per SM, at least eight
//   k-blocks per split, so that the partial-sum traffic and the second
//   kernel stay small against the main loop;
// - otherwise one CTA per tile, the widest tile (256, 128, 64) that divides
//   N and still gives at least half as many CTAs as SMs (else 64): wide
//   tiles read fewer operand bytes per flop, narrow ones put more SMs on a
//   small product.
void gemm_plan(int M, int N, int K, int *bn, int *splits, int *persistent) {
  const int sms = device_sms();
  const int nk = K / BK;
  auto tiles = [&](int w) { return (int64_t)(N / w) * (M / BM); };
  const int64_t tiles128 = N >= 128 ? tiles(128) : tiles(64);
  if (*persistent < 0)
    *persistent = (*splits <= 1 && tiles128 > sms) ? 1 : 0;
  if (*persistent) {
    *splits = 1;
    if (*bn == 0) *bn = N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : 64;
    return;
  }
  const bool split_k = *splits != 1 && 2 * tiles128 <= sms && nk >= 32;
  if (*bn == 0) {
    if (split_k) {
      *bn = N % 128 == 0 ? 128 : 64;
    } else {
      *bn = 64;
      for (int w : {256, 128}) {
        if (N % w == 0 && 2 * tiles(w) >= sms) {
          *bn = w;
          break;
        }
      }
    }
  }
  if (*splits != 0) return;
  int sp = 1;
  if (split_k) sp = std::max(1, std::min(nk / 8, (int)(sms / tiles(*bn))));
  *splits = sp;
}

size_t gemm_workspace_bytes(int M, int N, int splits) {
  return splits > 1 ? (size_t)splits * M * N * sizeof(float) : 0;
}

nrr_status gemm_bf16_tn(const void *A, const void *B, float *D, int M, int N,
                        int K, int ldd, cudaStream_t st, char *msg, int msglen,
                        int bn, int splits, float *ws, size_t ws_bytes,
                        int persistent) {
  if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || M % BM || K % BK ||
      (N % 64) || ldd < N || (ldd % 4) ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) ||
      (reinterpret_cast<uintptr_t>(D) & 15)) {
    snprintf(msg, msglen,
             "gemm: need M %% 128 == 0, N %% 64 == 0, K %% 64 == 0, ldd >= N, "
             "ldd %% 4 == 0 and 16-byte aligned operands (M=%d N=%d K=%d ldd=%d)",
             M, N, K, ldd);
    return NRR_ERR_INVALID_ARG;
  }
  if ((bn != 0 && bn != 64 && bn != 128 && bn != 256) || (bn != 0 && N % bn) ||
      splits < 0 || splits > K / BK || splits > 65535 || persistent < -1 ||
      persistent > 2 || (persistent >= 1 && splits > 1) ||
      (persistent == 2 && M % (2 * BM))) {
    snprintf(msg, msglen,
             "gemm: tile width must be 0 (chosen), 64, 128 or 256 and divide N; "
             "splits 0 (chosen) .. K/64; persistent -1 (chosen), 0, 1 or 2 (2: M "
             "%% 256 == 0), and not with splits > 1 (bn=%d splits=%d "
             "persistent=%d N=%d K=%d)",
             bn, splits, persistent, N, K);
    return NRR_ERR_INVALID_ARG;
  }
  if (!gemm_error_flag()) {
    snprintf(msg, msglen, "gemm: error flag allocation failed");
    return NRR_ERR_OOM;
  }
  gemm_plan(M, N, K, &bn, &splits, &persistent);
  // clusters of two CTAs share B: each loads half of the B box
  const int cl = persistent == 2 ? 2 : 1;
  CUtensorMap ma, mb;
  if (!cached_map(&ma, A, M, K, BM) || !cached_map(&mb, B, N, K, bn / cl)) {
    snprintf(msg, msglen, "gemm: tensor map encoding failed");
    return NRR_ERR_CUDA;
  }
  if (persistent) {
    CUtensorMap md;
    if (!cached_map(&md, D, M, N, ldd, 1)) {
      snprintf(msg, msglen, "gemm: output tensor map encoding failed");
      return NRR_ERR_CUDA;
    }
    const int units = (N / bn) * (M / BM / cl);
    const int ctas = cl * std::min(units, device_sms() / cl);
    cudaError_t e;
    if (cl == 2)
      e = bn == 256 ? launch_gemm_persistent<256, 2>(ma, mb, md, M, N, K, ctas, st)
          : bn == 128 ? launch_gemm_persistent<128, 2>(ma, mb, md, M, N, K, ctas, st)
                      : launch_gemm_persistent<64, 2>(ma, mb, md, M, N, K, ctas, st);
    else
      e = bn == 256 ? launch_gemm_persistent<256, 1>(ma, mb, md, M, N, K, ctas, st)
          : bn == 128 ? launch_gemm_persistent<128, 1>(ma, mb, md, M, N, K, ctas, st)
                      : launch_gemm_persistent<64, 1>(ma, mb, md, M, N, K, ctas, st);
    if (e != cudaSuccess) {
      snprintf(msg, msglen, "gemm launch: %s", cudaGetErrorString(e));
      return NRR_ERR_CUDA;
    }
    return NRR_OK;
  }
  const size_t need = gemm_workspace_bytes(M, N, splits);
  bool own = false;
  if (splits > 1 && (!ws || ws_bytes < need)) {
    // stream-ordered temporary for the partial products
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&ws), need, st);
    if (e != cudaSuccess) {
      snprintf(msg, msglen, "gemm: split-K workspace of %zu bytes: %s", need,
               cudaGetErrorString(e));
      return NRR_ERR_OOM;
    }
    own = true;
  }
  float *dst = splits > 1 ? ws : D;
  const int ld = splits > 1 ? N : ldd;
  const int64_t stride = (int64_t)M * N;
  cudaError_t e = bn == 256 ? launch_gemm<256>(ma, mb, dst, M, N, K, ld, splits, stride, st)
                  : bn == 128 ? launch_gemm<128>(ma, mb, dst, M, N, K, ld, splits, stride, st)
                              : launch_gemm<64>(ma, mb, dst, M, N, K, ld, splits, stride, st);
  if (e == cudaSuccess && splits > 1) {
    const int64_t n4 = (int64_t)M * (N / 4);
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 8 * device_sms());
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(ws),
                                                 D, M, N, ldd, splits);
    e = cudaGetLastError();
  }
  if (own) cudaFreeAsync(ws, st);
  if (e != cudaSuccess) {
    snprintf(msg, msglen, "gemm launch: %s", cudaGetErrorString(e));
    return NRR_ERR_CUDA;
  }
  return NRR_OK;
}

nrr_status gemm_check_error(cudaStream_t st, char *msg, int msglen) {
  int h = 0;
  int *f = gemm_error_flag();
  if (!f) return NRR_OK;
  if (cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    snprintf(msg, msglen, "gemm: status read-back failed");
    return NRR_ERR_CUDA;
  }
  if (h) {
    snprintf(msg, msglen, "gemm: a pipeline wait expired (code %d)", h);
    cudaMemsetAsync(f, 0, sizeof(int), st);
    return NRR_ERR_TIMEOUT;
  }
  return NRR_OK;
}

}  // namespace nrr

extern "C" {

nrr_status nrr_gemm_bf16_tn_async(const void *A, const void *B, float *D, int M,
                                  int N, int K, int bn, int splits, int persistent,
                                  void *stream) {
  char msg[256] = {0};
  nrr_status s = nrr::gemm_bf16_tn(A, B, D, M, N, K, N, static_cast<cudaStream_t>(stream),
                                   msg, sizeof msg, bn, splits, nullptr, 0, persistent);
  if (s != NRR_OK) nrr::set_last_error(msg);
  return s;
}

nrr_status nrr_gemm_status(void *stream) {
  char msg[256] = {0};
  nrr_status s = nrr::gemm_check_error(static_cast<cudaStream_t>(stream), msg, sizeof msg);
  if (s != NRR_OK) nrr::set_last_error(msg);
  return s;
}

nrr_status nrr_gemm_bf16_tn(const void *A, const void *B, float *D, int M, int N,
                            int K, void *stream) {
  nrr_status s = nrr_gemm_bf16_tn_async(A, B, D, M, N, K, 0, 0, -1, stream);
  return s != NRR_OK ? s : nrr_gemm_status(stream);
}

}  // extern "C"
