// Probing-vector generation z = z0 .* z_h (Algorithm 1, lines 3-6).
//
// z0: Z4 noise (Section 1) drawn with Philox4x64-10 (Salmon, Moraes, Dror &
// Shaw, SC'11), written here from that definition: counter {i/128, run, 0, 0},
// key {seed, 0}; the four 64-bit output words hold the 2-bit codes of 128
// consecutive dofs.  z_h: Sylvester Hadamard column over the nested
// hierarchical-probing colouring (Section 5.2).  All arithmetic is integer,
// so the result is bit-identical to any other implementation of the same
// definition.
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

// Internal layout [site][12][b]; one thread per (site, column).
__global__ void noise_internal_kernel(double2 *out, Geom g, uint64_t seed, int64_t run, int ncolors, int dilute12,
                                      int64_t q0, int nrhs, int b) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)g.V * b) return;
  const int j = (int)(tid % b);
  const int s = (int)(tid / b);
  double2 *o = out + (int64_t)s * 12 * b + j;
  if (j >= nrhs) {
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c * b] = make_double2(0.0, 0.0);
    return;
  }
  int xc[4];
  site_coords(g, s, xc);
  const int colour = hp_colour(xc, ncolors);
  const int64_t q = q0 + j;
  const int64_t hcol = dilute12 ? q / 12 : q;
  const int keep = dilute12 ? (int)(q % 12) : -1;
  const int sign = (__popcll((unsigned long long)(colour & hcol)) & 1) ? -1 : 1;
  // the 12 dofs of this site span at most two Philox blocks
  const int64_t i0 = (int64_t)s * 12;
  uint64_t w0[4], w1[4];
  philox4x64_10((uint64_t)(i0 >> 7), (uint64_t)run, 0ull, 0ull, seed, 0ull, w0);
  const int64_t blk1 = (i0 + 11) >> 7;
  if (blk1 != (i0 >> 7)) philox4x64_10((uint64_t)blk1, (uint64_t)run, 0ull, 0ull, seed, 0ull, w1);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const int64_t i = i0 + c;
    const uint64_t *w = ((i >> 7) == (i0 >> 7)) ? w0 : w1;
    const int code = (int)((w[(i >> 5) & 3] >> (2 * (i & 31))) & 3ull);
    double2 z = z4_value<double2>(code, sign);
    if (keep >= 0 && c != keep) z = make_double2(0.0, 0.0);
    o[c * b] = z;
  }
}

// Canonical layout (column-major N x nrhs); one thread per (dof, column).
__global__ void noise_canon_kernel(double2 *out, Geom g, uint64_t seed, int64_t run, int ncolors, int dilute12,
                                   int64_t q0, int nrhs) {
  const int64_t N = (int64_t)g.V * 12;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= N * nrhs) return;
  const int64_t i = tid % N;
  const int col = (int)(tid / N);
  const int s = (int)(i / 12);
  int xc[4];
  site_coords(g, s, xc);
  const int colour = hp_colour(xc, ncolors);
  const int64_t q = q0 + col;
  const int64_t hcol = dilute12 ? q / 12 : q;
  const int sign = (__popcll((unsigned long long)(colour & hcol)) & 1) ? -1 : 1;
  double2 z = z4_value<double2>(z4_code(seed, run, i), sign);
  if (dilute12 && (i % 12) != (q % 12)) z = make_double2(0.0, 0.0);
  out[tid] = z;
}

void launch_noise(double2 *out, const Geom &g, uint64_t seed, int64_t z0_index, int ncolors, int dilute12,
                  int64_t q0, int nrhs, int b, cudaStream_t st) {
  const int64_t n = (int64_t)g.V * b;
  const int T = 256;
  noise_internal_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(out, g, seed, z0_index, ncolors, dilute12, q0,
                                                                    nrhs, b); count_launches(1);
}

void launch_noise_canon(double2 *out, const Geom &g, uint64_t seed, int64_t z0_index, int ncolors, int dilute12,
                        int64_t q0, int nrhs, cudaStream_t st) {
  const int64_t n = (int64_t)g.V * 12 * nrhs;
  const int T = 256;
  noise_canon_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(out, g, seed, z0_index, ncolors, dilute12, q0, nrhs); count_launches(1);
}

}  // namespace dtr
