// Helpers shared by the tcgen05 kernels: shared-memory addresses, bounded
// mbarrier waits and shared-memory matrix descriptors.
#pragma once

#include <cstdint>

namespace dtr {

constexpr long long kTcBudget = 2000000000LL;  // clock cycles a wait may take (~1 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}

// wait for the phase with the given parity to complete, for at most `budget` cycles
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(addr, parity)) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// bounded wait that also gives up as soon as another role has given up (*abort)
__device__ __forceinline__ bool mbar_wait_ab(uint32_t addr, uint32_t parity, volatile int *abort) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(addr, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kTcBudget) {
      *abort = 1;
      return false;
    }
  }
}

// shared-memory matrix descriptor without swizzle: start address, leading byte offset
// (between adjacent core matrices along K) and stride byte offset (between adjacent core
// matrices along M or N), in bytes; without swizzle these roles hold for K-major and
// MN-major operands alike (a core matrix is 8 rows of 16 contiguous bytes)
__device__ __forceinline__ uint64_t desc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

}  // namespace dtr
