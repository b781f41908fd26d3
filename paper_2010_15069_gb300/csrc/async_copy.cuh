// Asynchronous global -> shared copies (bulk copies and 2D TMA tiles) tracked
// by shared-memory mbarriers, with bounded waits.
//
// Every wait gives up after about 2^31 clock cycles (about a second at GB300
// clocks): the block then records an error bit and leaves its loop, so a lost
// transfer shows up as SPGPE_ETIMEOUT instead of a hung kernel.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace spgpe {

constexpr long long kWaitCycles = 1ll << 31;
constexpr int kErrTimeout = 2;  // bit in the context's error flags
constexpr int kErrBounds = 4;   // bit in the context's error flags (bounds-checked builds only)

// Index check of the bounds-checked build (compiled with -DSPGPE_BOUNDS, the
// stand-in for a memory checker): an index i outside [0, n) sets kErrBounds in
// the error flags and the caller skips the access.  In the release build it is
// the constant true, so the kernels are unchanged.
__device__ __forceinline__ bool in_bounds(int *flags, long i, long n) {
#ifdef SPGPE_BOUNDS
  if (i < 0 || i >= n) {
    atomicOr(flags, kErrBounds);
    return false;
  }
#else
  (void)flags;
  (void)i;
  (void)n;
#endif
  return true;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; false after the cycle budget.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy accesses (a refill of a buffer the block has just used).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Contiguous bytes global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 2D tile global -> shared through a tensor map; x is the inner coordinate
// (its byte offset must be a multiple of 16), y the outer one.
__device__ __forceinline__ void tma_g2s_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// 2D tile shared -> global through a tensor map (bulk-group completion):
// issue, then commit; bulk_wait_read0 waits until every committed store has
// finished reading shared memory (the buffer may then be overwritten).
__device__ __forceinline__ void tma_s2g_2d(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk store complete (its writes performed)
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace spgpe
