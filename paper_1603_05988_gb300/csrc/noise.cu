// Probing-vector generation z = z0 .* z_h (Algorithm 1; Section 5.2).
//
// z0: Z4 noise (Section 1) drawn with Philox4x64-10 (Salmon, Moraes, Dror &
// Shaw, SC'11), written here from that definition: counter {i/128, run, 0, 0},
// key {seed, 0}; the four 64-bit output words hold the 2-bit codes of 128
// consecutive dofs.  z_h: Sylvester Hadamard column over the nested
// hierarchical-probing colouring (Section 5.2).  All arithmetic is integer,
// so the result is bit-identical to any other implementation of the same
// definition.
#include "philox.cuh"

namespace dtr {

// Internal layout [site][12][b]; one thread per (site, column).  Column k of
// the block is global column G = g0 + k of the run-major sequence
// (run = run0 + G / ncols, probing index q = qoff + G % ncols).
// With `codes` non-NULL every entry is also written as one byte in the same layout:
// bits 0-1 the power c of i (z = i^c), bit 2 set for a zero (dilution, padding).
__global__ void noise_internal_kernel(double2 *out, Geom g, uint64_t seed, int64_t run0, int ncolors, int dilute12,
                                      int64_t g0, int64_t ncols, int64_t qoff, int nrhs, int b,
                                      unsigned char *codes) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)g.V * b) return;
  const int j = (int)(tid % b);
  const int s = (int)(tid / b);
  double2 *o = out + (int64_t)s * 12 * b + j;
  unsigned char *oc = codes ? codes + (int64_t)s * 12 * b + j : nullptr;
  if (j >= nrhs) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      o[c * b] = make_double2(0.0, 0.0);
      if (oc) oc[c * b] = 4;
    }
    return;
  }
  int xc[4];
  site_coords(g, s, xc);
  const int colour = hp_colour(xc, ncolors);
  const int64_t G = g0 + j;
  const int64_t run = run0 + G / ncols;
  const int64_t q = qoff + G % ncols;
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
    const bool zero = keep >= 0 && c != keep;
    if (zero) z = make_double2(0.0, 0.0);
    o[c * b] = z;
    if (oc) oc[c * b] = (unsigned char)(zero ? 4 : ((code + (sign < 0 ? 2 : 0)) & 3));
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

void launch_noise(double2 *out, const Geom &g, uint64_t seed, int64_t run0, int ncolors, int dilute12, int64_t g0,
                  int64_t ncols, int nrhs, int b, cudaStream_t st, int64_t qoff, unsigned char *codes) {
  const int64_t n = (int64_t)g.V * b;
  const int T = 256;
  noise_internal_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(out, g, seed, run0, ncolors, dilute12, g0, ncols,
                                                                    qoff, nrhs, b, codes); count_launches(1);
}

void launch_noise_canon(double2 *out, const Geom &g, uint64_t seed, int64_t z0_index, int ncolors, int dilute12,
                        int64_t q0, int nrhs, cudaStream_t st) {
  const int64_t n = (int64_t)g.V * 12 * nrhs;
  const int T = 256;
  noise_canon_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(out, g, seed, z0_index, ncolors, dilute12, q0, nrhs); count_launches(1);
}

}  // namespace dtr
