// Shared-memory staging by the Tensor Memory Accelerator: mbarrier set-up, bounded waits
// (%globaltimer), a 2-D tiled copy (SSAO depth tiles) and a 1-D bulk copy (the compose's light
// list).  Every wait is bounded: a caller whose wait runs out falls back to reading global memory
// and waits once more (bounded) before its block exits, so that a late copy cannot land in the
// shared memory of a later block.
#pragma once

#include <cuda.h>  // CUtensorMap

#include "epbr_internal.cuh"

namespace epbr {

constexpr unsigned long long kTmaWaitNs = 50ull * 1000 * 1000;  // a copy takes microseconds

// Limit of the first wait for a staged copy, passed to the launches that stage by TMA; changed only
// by epbr_ssao_set_tile_wait (a test of the fallback paths sets 0: give up at once).
unsigned long long tma_first_wait_ns();
unsigned long long set_tma_first_wait_ns(unsigned long long ns);  // returns the previous limit

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for phase `parity` of the mbarrier for at most `limit_ns`; false when it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// One thread: arms the block's mbarrier for `bytes` and starts the 2-D tile copy of `map` at
// element (x, y) into `dst` (the tensor map's box fixes the tile's shape).
__device__ __forceinline__ void tma_load_tile_2d(const CUtensorMap* map, void* dst, unsigned bar, int x, int y,
                                                 unsigned bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// One thread: arms the block's mbarrier for `bytes` and starts a 1-D bulk copy of `bytes` bytes
// from global `src` to shared `dst` (both 16-byte aligned, `bytes` a multiple of 16).
__device__ __forceinline__ void tma_load_bulk(void* dst, const void* src, unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

}  // namespace epbr
