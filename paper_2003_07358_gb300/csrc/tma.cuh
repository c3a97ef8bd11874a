// Tensor-memory-accelerator (TMA) tile loads with an mbarrier, for sm_103a.
//
// One elected thread arms the CTA's mbarrier with the expected byte count and issues
// cp.async.bulk.tensor copies; every thread then waits on the barrier's phase with a
// bounded spin.  A wait that runs out sets bit kDevTimeoutTMA of the library's device
// status word (read by the host at the next synchronising call) and returns false,
// so a stuck copy can never hang the GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fhs {

constexpr unsigned kDevTimeoutTMA = 1u;   // device status bit: a TMA wait gave up
constexpr long long kTmaSpinLimit = 1ll << 22;

// The including translation unit defines `__device__ unsigned int g_dev_status` and
// `__device__ long long g_wait_first`: the length of the first phase of the bounded
// waits (0: kTmaSpinLimit; negative: no polls, the wait gives up at once), changed only
// by the fault-injection hook fhs_set_wait_limit.

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count));
  // make the initialised barrier visible to the async (TMA) proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes));
}

// 4-D tiled load of box `map` at coordinates (c0 innermost .. c3) into shared dst.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of the barrier; false (and the status bit) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  const long long first = g_wait_first > 0 ? g_wait_first : (g_wait_first < 0 ? 0 : kTmaSpinLimit);
  for (long long it = 0; it < first; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  atomicOr(&g_dev_status, kDevTimeoutTMA);
  // give the copies in flight a second bounded chance to land before the CTA moves on
  for (long long it = 0; it < kTmaSpinLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) break;
  }
  return false;
}

}  // namespace fhs
