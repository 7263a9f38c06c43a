// nrr_debug.cuh -- address checks of the NRR_DEBUG build.
//
// compute-sanitizer is not available where this library runs, so the debug
// build (compiled with -DNRR_DEBUG=1 into libnrr_debug.so) checks the
// addresses itself: every load and store that the stencil, boundary and
// residual kernels make through the helpers in nrr_stencil.cuh (ldc, ld, lds,
// st) must fall inside one of the device allocations that the library has
// registered (grid, batch, patch-system and surrogate buffers).  An access
// outside all of them is skipped -- a load returns zero, a store is dropped --
// and its address is recorded; nrr_debug_check() reports the first such
// address and the count.  Nothing traps, so the context stays usable.
//
// Each translation unit that includes this header has its own device copy of
// the range table (no relocatable device code); the host registry in
// nrr_api.cu copies the table into every unit's copy whenever an allocation
// is registered or released.  In the release build (NRR_DEBUG 0) the
// registry calls are no-ops and the helpers compile to plain accesses.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#ifndef NRR_DEBUG
#define NRR_DEBUG 0
#endif

namespace nrr {

constexpr int kDbgRanges = 128;

struct DbgTable {
  unsigned long long lo[kDbgRanges], hi[kDbgRanges];  // [lo, hi) byte ranges
  int n;
  unsigned long long bad;    // first refused address (0: none)
  unsigned long long count;  // refused accesses
};

// Host registry (nrr_api.cu).  dbg_register / dbg_unregister synchronise the
// device before they change the table (debug build only); dbg_register also
// fills the new allocation with NaN (all bits set), so that reads of memory
// the library never wrote show up as NaN.
void dbg_register(const void *p, size_t bytes);
void dbg_unregister(const void *p);
using DbgSync = void (*)(const DbgTable &);
using DbgRead = void (*)(unsigned long long *bad, unsigned long long *count);
void dbg_add_unit(DbgSync sync, DbgRead read);

}  // namespace nrr

#if NRR_DEBUG
// this translation unit's copy of the table
static __device__ nrr::DbgTable g_nrr_dbg;

namespace {
void nrr_dbg_sync(const nrr::DbgTable &t) {
  // the ranges only: the refusal record stays until it is read
  cudaMemcpyToSymbol(g_nrr_dbg, &t, offsetof(nrr::DbgTable, bad));
}
void nrr_dbg_read(unsigned long long *bad, unsigned long long *count) {
  unsigned long long rec[2] = {0, 0};
  if (cudaMemcpyFromSymbol(rec, g_nrr_dbg, sizeof rec,
                           offsetof(nrr::DbgTable, bad)) != cudaSuccess)
    return;
  if (rec[0] && !*bad) *bad = rec[0];
  *count += rec[1];
  const unsigned long long zero[2] = {0, 0};
  cudaMemcpyToSymbol(g_nrr_dbg, zero, sizeof zero, offsetof(nrr::DbgTable, bad));
}
struct NrrDbgUnit {
  NrrDbgUnit() { nrr::dbg_add_unit(nrr_dbg_sync, nrr_dbg_read); }
};
NrrDbgUnit g_nrr_dbg_unit;
}  // namespace

namespace nrr {
namespace dev {
// true if [p, p + bytes) lies inside a registered allocation; otherwise the
// address is recorded and the caller skips the access (not inlined: one
// copy per translation unit instead of one per load)
static __device__ __noinline__ bool dbg_ok(const void *p, int bytes) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  const int n = g_nrr_dbg.n;
  for (int i = 0; i < n; i++)
    if (a >= g_nrr_dbg.lo[i] && a + (unsigned long long)bytes <= g_nrr_dbg.hi[i])
      return true;
  atomicCAS(&g_nrr_dbg.bad, 0ull, a ? a : 1ull);
  atomicAdd(&g_nrr_dbg.count, 1ull);
  return false;
}
}  // namespace dev
}  // namespace nrr
#endif
