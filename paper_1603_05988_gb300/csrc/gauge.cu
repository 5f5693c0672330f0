// Random SU(3) gauge field generated on the device (the synthetic stand-in for
// the gauge ensembles of Section 6, whose configurations are not available).
//
// Link U_mu(x) = exp(i eps H) with H a Gaussian Hermitian traceless 3 x 3
// matrix, drawn as a pure function of (seed, site, mu):
//   * Philox4x64-10 (Salmon et al., SC'11) with key {seed, 1} and counter
//     {site, mu, c, 0}, c = 0..4: 20 words -> uniforms
//     u = ((w >> 11) + 1/2) 2^-53 in (0, 1);
//   * Box-Muller on consecutive pairs (u_2p, u_2p+1): r = sqrt(-2 ln u_2p),
//     normals r cos(2 pi u_2p+1), r sin(2 pi u_2p+1) -> n_0 .. n_19, of
//     which n_0 .. n_17 are used;
//   * G_ab = n_2(3a+b) + i n_2(3a+b)+1, H = (G + G^H)/2 - (Tr/3) 1;
//   * U = exp(i eps H) by scaling and squaring of the Taylor series: with
//     X = i eps H / 2^s and ||X||_F <= 1/4, U = (sum_{j<=12} X^j / j!)^(2^s)
//     (truncation below 1e-16 of the FP64 rounding), exact to FP64 rounding
//     in unitarity and det = exp(i eps Tr H) = 1.
// The noise stream uses key {seed, 0}, so the two never share a counter.
#include <cmath>

#include "dtr_internal.cuh"
#include "philox.cuh"

namespace dtr {

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ M3 m3_mul(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int l = 0; l < 3; ++l) s = caxpy(a.e[3 * i + l], b.e[3 * l + j], s);
      c.e[3 * i + j] = s;
    }
  return c;
}

// U_mu(x) for every (x, mu): out[(x*4 + mu)*9 + 3a + b], FP64
__global__ void k_make_links(double2 *__restrict__ out, int64_t nlinks, double eps, uint64_t seed) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t site = (uint64_t)(l >> 2), mu = (uint64_t)(l & 3);
    double n[20];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      uint64_t w[4];
      philox4x64_10(site, mu, (uint64_t)c, 0ull, seed, 1ull, w);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const double u0 = ((double)(w[2 * p] >> 11) + 0.5) * 0x1.0p-53;
        const double u1 = ((double)(w[2 * p + 1] >> 11) + 0.5) * 0x1.0p-53;
        const double r = sqrt(-2.0 * log(u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        n[4 * c + 2 * p] = r * cs;
        n[4 * c + 2 * p + 1] = r * sn;
      }
    }
    // H = (G + G^H)/2 - Tr/3, then X = i eps H
    double2 G[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] = make_double2(n[2 * q], n[2 * q + 1]);
    M3 X;
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) tr += G[4 * a].x;
    tr /= 3.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // H_ab = (G_ab + conj(G_ba)) / 2
        double2 h = make_double2(0.5 * (G[3 * a + b].x + G[3 * b + a].x), 0.5 * (G[3 * a + b].y - G[3 * b + a].y));
        if (a == b) h = make_double2(h.x - tr, 0.0);
        X.e[3 * a + b] = make_double2(-eps * h.y, eps * h.x);  // i eps h
      }
    // scaling: ||X / 2^s||_F <= 1/4
    double fro = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) fro += X.e[q].x * X.e[q].x + X.e[q].y * X.e[q].y;
    fro = sqrt(fro);
    int s = 0;
    while (fro > 0.25 && s < 60) {
      fro *= 0.5;
      ++s;
    }
    const double sc = ldexp(1.0, -s);
#pragma unroll
    for (int q = 0; q < 9; ++q) X.e[q] = cscale(X.e[q], sc);
    // Taylor series to degree 12 in Horner form: T = 1 + X/1 (1 + X/2 (1 + ... (1 + X/12)))
    M3 T;
#pragma unroll
    for (int q = 0; q < 9; ++q) T.e[q] = make_double2((q % 4 == 0) ? 1.0 : 0.0, 0.0);
    for (int j = 12; j >= 1; --j) {
      M3 P = m3_mul(X, T);
      const double inv = 1.0 / (double)j;
#pragma unroll
      for (int q = 0; q < 9; ++q) T.e[q] = make_double2(((q % 4 == 0) ? 1.0 : 0.0) + P.e[q].x * inv, P.e[q].y * inv);
    }
    for (int k = 0; k < s; ++k) T = m3_mul(T, T);
    double2 *o = out + l * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = T.e[q];
  }
}

void launch_make_links(double2 *U64, int64_t V, double eps, uint64_t seed, cudaStream_t st) {
  const int64_t nl = V * 4;
  int64_t grid = (nl + 127) / 128;
  if (grid > 65535LL * 16) grid = 65535LL * 16;
  k_make_links<<<(unsigned)grid, 128, 0, st>>>(U64, nl, eps, seed);
  count_launches(1);
}

}  // namespace dtr
