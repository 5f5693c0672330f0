// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11),
// written from its published definition, and the Z4 code of a dof derived
// from it: counter {i/128, run, 0, 0}, key {seed, 0}, code = bits
// 2*(i%32)..+1 of output word (i%128)/32.  Code q means z0 = i^q.
#pragma once

#include "dtr_internal.cuh"

namespace dtr {

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                              uint64_t k1, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// 2-bit Z4 code of dof i for run `run`.
__device__ __forceinline__ int z4_code(uint64_t seed, int64_t run, int64_t i) {
  uint64_t w[4];
  philox4x64_10((uint64_t)(i >> 7), (uint64_t)run, 0ull, 0ull, seed, 0ull, w);
  return (int)((w[(i >> 5) & 3] >> (2 * (i & 31))) & 3ull);
}

// i^code * sign
template <typename C> __device__ __forceinline__ C z4_value(int code, int sign) {
  C z;
  z.x = (code == 0) ? 1.0 : (code == 2 ? -1.0 : 0.0);
  z.y = (code == 1) ? 1.0 : (code == 3 ? -1.0 : 0.0);
  z.x *= sign;
  z.y *= sign;
  return z;
}

}  // namespace dtr
