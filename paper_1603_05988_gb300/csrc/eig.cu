// Setup eigensolver: the deflation space of Section 5.1 (the k smallest
// singular triplets of A, as eigenpairs of the Hermitian Q = g5 A with
// sigma = |lambda|), computed on the GPU and handed to the estimator as a
// dtr_defl without leaving the device.
//
// Method: Chebyshev-filtered subspace iteration (Zhou & Saad, "Chebyshev-
// filtered subspace iteration", 2007) on S = A^H A = Q^2, whose wanted
// eigenvalues sigma^2 are the smallest of a positive definite operator, i.e.
// exterior ones, so the Rayleigh-Ritz step is reliable without solves (a
// Rayleigh-Ritz step for the indefinite Q itself can produce spurious Ritz
// values near 0).  Per iteration, for a basis Y of p >= k columns:
//   1. Y <- p_d(S) Y with the degree-d Chebyshev polynomial of the interval
//      [a, b] (a = the largest Ritz value of S kept last time, b an upper
//      bound of the spectrum), scaled to 1 at the smallest Ritz value, column
//      chunks at a time in the solver's multi-RHS layout;
//   2. QY = Q Y from the stored (rounded) Y;
//   3. M = (QY)^H QY, H = Y^H QY (split-K Gram kernels, FP32 products of the
//      stored values accumulated in FP32 over short dof runs and in FP64
//      across them, FP64 for FP64 storage);
//   4. host: harmonic Rayleigh-Ritz for the target 0 (Morgan 1991):
//      H c = nu M c, nu = 1/theta, on an M-orthonormal basis from canonical
//      orthogonalisation of M (directions with tiny eigenvalues dropped); the
//      wanted theta near 0 are the exterior |nu|, so no spurious small Ritz
//      values; eigenvalue = the harmonic Ritz value 1/nu (|1/lambda| stays
//      below 1/sigma_min even for unconverged vectors), sorted by |nu|;
//   5. Y <- Y C in place (row blocks through a per-CTA buffer), columns
//      normalised by a norms pass (which also gives the Ritz values of S for
//      the next filter interval); dropped columns are refilled with random
//      vectors; QY is not rotated (the next filter recomputes it);
//   6. true residuals ||Q y_j - theta_j y_j|| / (|theta_j| ||y_j||) of the stored y_j,
//      j < k, from a fresh stencil (or relative to the bound on ||A|| instead).
// The basis lives in the deflation handle's own buffer, row-major [dof][p]
// in FP64, FP32 or BF16 (the layout every deflation kernel reads), and is
// compacted in place to [dof][k], ordered by |lambda|, at the end; QY and the
// chunk fields live in the caller's workspace.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "deflate.cuh"
#include "herm_eig.cuh"
#include "philox.cuh"

namespace dtr {

// ------------------------------------------------------------ element access
__device__ __forceinline__ float2 ld2f(const float2 &v) { return v; }
__device__ __forceinline__ float2 ld2f(const bfc2 &v) { return __bfloat1622float2(v); }
__device__ __forceinline__ double2 ld2d(const double2 &v) { return v; }
__device__ __forceinline__ double2 ld2d(const float2 &v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld2d(const bfc2 &v) {
  const float2 f = __bfloat1622float2(v);
  return make_double2(f.x, f.y);
}
template <typename T> __device__ __forceinline__ T st2(double re, double im);
template <> __device__ __forceinline__ double2 st2<double2>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 st2<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ bfc2 st2<bfc2>(double re, double im) {
  return __floats2bfloat162_rn((float)re, (float)im);
}

// accumulation type of the Gram and rotation kernels
template <typename T> struct EigAcc { typedef float2 type; typedef float real; };
template <> struct EigAcc<double2> { typedef double2 type; typedef double real; };
__device__ __forceinline__ float2 ldacc(const float2 &v, float2 *) { return v; }
__device__ __forceinline__ float2 ldacc(const bfc2 &v, float2 *) { return __bfloat1622float2(v); }
__device__ __forceinline__ double2 ldacc(const double2 &v, double2 *) { return v; }

// ------------------------------------------------------------ basis kernels
// Columns [c0, c1) of Y get independent complex Gaussian entries (variance 1):
// Philox4x64-10 key {seed, 2}, counter {dof, column, draw, 0}, Box-Muller.
template <typename T>
__global__ void k_eig_random(T *__restrict__ Y, int64_t N, int p, int c0, int c1, uint64_t seed, uint64_t draw) {
  const int w = c1 - c0;
  const int64_t n = N * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w;
    const int j = c0 + (int)(e - i * w);
    uint64_t r[4];
    philox4x64_10((uint64_t)i, (uint64_t)j, draw, 0ull, seed, 2ull, r);
    const double u0 = ((double)(r[0] >> 11) + 0.5) * 0x1.0p-53;
    const double u1 = ((double)(r[1] >> 11) + 0.5) * 0x1.0p-53;
    const double rad = sqrt(-log(u0));  // |z|^2 ~ Exp(1): E|z|^2 = 1
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    Y[i * p + j] = st2<T>(rad * cs, rad * sn);
  }
}

// internal [dof][b] (the solver's [site][12][b]) <- columns [c0, c0 + w) of Y
template <typename T, typename C>
__global__ void k_eig_gather(const T *__restrict__ Y, int64_t N, int p, int c0, int w, C *__restrict__ X, int b) {
  const int64_t n = N * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b;
    const int j = (int)(e - i * b);
    C v;
    if (j < w) {
      const double2 y = ld2d(Y[i * p + c0 + j]);
      v.x = y.x;
      v.y = y.y;
    } else {
      v.x = 0;
      v.y = 0;
    }
    X[e] = v;
  }
}

// columns [c0, c0 + w) of Y <- internal X (times g5 if g5 != 0), rounded to T
template <typename T, typename C>
__global__ void k_eig_scatter(const C *__restrict__ X, int64_t N, int b, int w, T *__restrict__ Y, int p, int c0,
                              int g5) {
  const int64_t n = N * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w;
    const int j = (int)(e - i * w);
    const C v = X[i * b + j];
    const double s = (g5 && (i % 12) >= 6) ? -1.0 : 1.0;
    Y[i * p + c0 + j] = st2<T>(s * (double)v.x, s * (double)v.y);
  }
}

// Chebyshev step on internal fields: Y0 <- alpha (SY1 - c Y1) + beta Y0
template <typename C, typename R>
__global__ void k_eig_cheb(const C *__restrict__ SY1, const C *__restrict__ Y1, C *__restrict__ Y0, int64_t n,
                           R alpha, R beta, R c) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const C s = SY1[e], y1 = Y1[e], y0 = Y0[e];
    C o;
    o.x = alpha * (s.x - c * y1.x) + beta * y0.x;
    o.y = alpha * (s.y - c * y1.y) + beta * y0.y;
    Y0[e] = o;
  }
}

// ------------------------------------------------------------------- Gram
// partial[(chunk * na + ia) * nb + jb] = sum over the chunk's dofs i of
// conj(A[i, a0 + ia]) B[i, b0 + jb]; 64 x 64 output tiles, 256 threads, each
// a 4 x 4 sub-tile (rows ty + 16 r, columns tx + 16 c); 16 dofs per shared-memory
// step; FP32 sums over runs of kFlush dofs, added into FP64 (FP64 throughout
// for FP64 storage).  blockIdx.x = tile (fast), blockIdx.y = dof chunk, so the
// CTAs in flight share a chunk's rows through L2.
constexpr int kGT = 64, kGK = 16, kFlush = 512;
template <typename T>
__global__ void __launch_bounds__(256)
    k_eig_gram(const T *__restrict__ A, int pa, int a0, int na, const T *__restrict__ B, int pb, int b0, int nb,
               int64_t N, int nchunks, double2 *__restrict__ partial) {
  typedef typename EigAcc<T>::type AC;
  typedef typename EigAcc<T>::real AR;
  __shared__ AC As[kGK][kGT], Bs[kGK][kGT];
  const int tilesb = (nb + kGT - 1) / kGT;
  const int ti = blockIdx.x / tilesb, tj = blockIdx.x % tilesb;
  const int chunk = blockIdx.y;
  const int64_t i0 = N * chunk / nchunks, i1 = N * (chunk + 1) / nchunks;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  AC acc[4][4];
  double2 tot[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[r][c].x = acc[r][c].y = 0;
      tot[r][c] = make_double2(0.0, 0.0);
    }
  int since = 0;
  for (int64_t k0 = i0; k0 < i1; k0 += kGK) {
    __syncthreads();
    for (int q = threadIdx.x; q < kGK * kGT; q += 256) {
      const int kk = q / kGT, cc = q % kGT;
      const int64_t i = k0 + kk;
      const int ca = ti * kGT + cc, cb = tj * kGT + cc;
      AC va, vb;
      va.x = va.y = 0;
      vb.x = vb.y = 0;
      if (i < i1) {
        if (ca < na) va = ldacc(A[i * pa + a0 + ca], (AC *)nullptr);
        if (cb < nb) vb = ldacc(B[i * pb + b0 + cb], (AC *)nullptr);
      }
      As[kk][cc] = va;
      Bs[kk][cc] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      AC a[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // conj(a) b
          acc[r][c].x = fma(a[r].x, bv[c].x, fma(a[r].y, bv[c].y, acc[r][c].x));
          acc[r][c].y = fma(a[r].x, bv[c].y, fma(-a[r].y, bv[c].x, acc[r][c].y));
        }
    }
    since += kGK;
    if (since >= kFlush || k0 + kGK >= i1) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          tot[r][c].x += (double)acc[r][c].x;
          tot[r][c].y += (double)acc[r][c].y;
          acc[r][c].x = acc[r][c].y = (AR)0;
        }
      since = 0;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int ia = ti * kGT + ty + 16 * r, jb = tj * kGT + tx + 16 * c;
      if (ia < na && jb < nb) partial[((int64_t)chunk * na + ia) * nb + jb] = tot[r][c];
    }
}

// out[e] = sum over chunks (in order) of partial[chunk][e]
__global__ void k_eig_gram_reduce(const double2 *__restrict__ partial, int64_t ne, int nchunks,
                                  double2 *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) s = cadd(s, partial[(int64_t)c * ne + e]);
    out[e] = s;
  }
}

// --------------------------------------------------------------- rotation
// Y[i, 0:r] <- Y[i, 0:p] Cm (Cm row-major p x r, complex), in place: each CTA
// takes row blocks of 64 dofs in turn, computes all r outputs tile by tile
// (64 x 64 tiles, 16-wide steps over p, 4 x 4 per thread) into its own slot
// of `tmp`, then copies the block back.  Columns r .. p-1 are left as they are.
template <typename T>
__global__ void __launch_bounds__(256)
    k_eig_rotate(T *__restrict__ Y, int64_t N, int p, int r, const typename EigAcc<T>::type *__restrict__ Cm,
                 T *__restrict__ tmp) {
  typedef typename EigAcc<T>::type AC;
  __shared__ AC As[kGK][kGT], Bs[kGK][kGT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T *slot = tmp + (int64_t)blockIdx.x * kGT * r;
  const int64_t nblk = (N + kGT - 1) / kGT;
  const int ctiles = (r + kGT - 1) / kGT;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t row0 = blk * kGT;
    for (int ct = 0; ct < ctiles; ++ct) {
      AC acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c].x = acc[a][c].y = 0;
      for (int j0 = 0; j0 < p; j0 += kGK) {
        __syncthreads();
        for (int q = threadIdx.x; q < kGK * kGT; q += 256) {
          const int kk = q % kGK, rr = q / kGK;  // Y rows: 16 consecutive columns of a row per group
          const int64_t i = row0 + rr;
          AC v;
          v.x = v.y = 0;
          if (i < N && j0 + kk < p) v = ldacc(Y[i * p + j0 + kk], (AC *)nullptr);
          As[kk][rr] = v;
          const int kk2 = q / kGT, cc = q % kGT;
          AC w;
          w.x = w.y = 0;
          if (j0 + kk2 < p && ct * kGT + cc < r) w = Cm[(int64_t)(j0 + kk2) * r + ct * kGT + cc];
          Bs[kk2][cc] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
          AC a[4], bv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = As[kk][ty + 16 * q];
#pragma unroll
          for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              acc[q][c].x = fma(a[q].x, bv[c].x, fma(-a[q].y, bv[c].y, acc[q][c].x));
              acc[q][c].y = fma(a[q].x, bv[c].y, fma(a[q].y, bv[c].x, acc[q][c].y));
            }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int rr = ty + 16 * q, m = ct * kGT + tx + 16 * c;
          if (m < r) slot[(int64_t)rr * r + m] = st2<T>((double)acc[q][c].x, (double)acc[q][c].y);
        }
    }
    __syncthreads();
    // every output of this row block is in the slot: copy it over Y's rows
    const int nrow = (N - row0) < kGT ? (int)(N - row0) : kGT;
    for (int q = threadIdx.x; q < nrow * r; q += 256) {
      const int rr = q / r, m = q - rr * r;
      Y[(row0 + rr) * p + m] = slot[q];
    }
    __syncthreads();
  }
}

// True residuals of stored columns: AX = A X for the internal chunk X (the stored
// columns c0 .. c0 + w widened exactly), part[(chunk * k + c0 + j) * 2 + {0, 1}] =
// sum over the chunk's dofs of |g5 AX - theta_j X|^2 and |X|^2 (FP64).  256 threads:
// 256 / b dof groups x b columns, the groups summed in shared memory in a fixed order.
template <typename C>
__global__ void __launch_bounds__(256)
    k_eig_resid_int(const C *__restrict__ AX, const C *__restrict__ X, int64_t N, int b, int w, int c0, int k,
                    const double *__restrict__ theta, int nchunks, double *__restrict__ part) {
  __shared__ double sr[256], sy[256];
  const int j = threadIdx.x % b, grp = threadIdx.x / b, ngrp = 256 / b;
  const int64_t i0 = N * blockIdx.x / nchunks, i1 = N * (blockIdx.x + 1) / nchunks;
  double r2 = 0.0, y2 = 0.0;
  if (j < w) {
    const double th = theta[c0 + j];
    for (int64_t i = i0 + grp; i < i1; i += ngrp) {
      const C a = AX[i * b + j], x = X[i * b + j];
      const double s = (i % 12) >= 6 ? -1.0 : 1.0;
      const double dx = s * (double)a.x - th * (double)x.x, dy = s * (double)a.y - th * (double)x.y;
      r2 += dx * dx + dy * dy;
      y2 += (double)x.x * x.x + (double)x.y * x.y;
    }
  }
  sr[threadIdx.x] = r2;
  sy[threadIdx.x] = y2;
  __syncthreads();
  if (grp == 0 && j < w) {
    double a = 0.0, c = 0.0;
    for (int g = 0; g < ngrp; ++g) {
      a += sr[g * b + j];
      c += sy[g * b + j];
    }
    part[((int64_t)blockIdx.x * k + c0 + j) * 2] = a;
    part[((int64_t)blockIdx.x * k + c0 + j) * 2 + 1] = c;
  }
}

// part[chunk * r + j] = sum over the chunk's dofs of |Y[i, j]|^2, j < r (FP64)
template <typename T>
__global__ void k_eig_colnorm(const T *__restrict__ Y, int64_t N, int p, int r, int nchunks, double *__restrict__ part) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= r) return;
  const int64_t i0 = N * blockIdx.x / nchunks, i1 = N * (blockIdx.x + 1) / nchunks;
  double acc = 0.0;
  for (int64_t i = i0; i < i1; ++i) {
    const double2 y = ld2d(Y[i * p + j]);
    acc += y.x * y.x + y.y * y.y;
  }
  part[(int64_t)blockIdx.x * r + j] = acc;
}

// Y[i, j] *= s[j] for j < r
template <typename T>
__global__ void k_eig_scale(T *__restrict__ Y, int64_t N, int p, int r, const double *__restrict__ sc) {
  const int64_t n = N * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int j = (int)(e - i * r);
    const double2 y = ld2d(Y[i * p + j]);
    Y[i * p + j] = st2<T>(y.x * sc[j], y.y * sc[j]);
  }
}

// ------------------------------------------------------------- compaction
// rows [r0, r1) of Y (stride p, columns perm[0..k)) -> bounce (stride k) -> rows of Y with stride k
template <typename T>
__global__ void k_eig_compact_out(const T *__restrict__ Y, int p, int k, int64_t r0, int64_t r1,
                                  const int *__restrict__ perm, T *__restrict__ bounce) {
  const int64_t n = (r1 - r0) * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    bounce[e] = Y[(r0 + i) * p + perm[e - i * k]];
  }
}
template <typename T>
__global__ void k_eig_compact_in(const T *__restrict__ bounce, int k, int64_t r0, int64_t r1, T *__restrict__ Y) {
  const int64_t n = (r1 - r0) * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    Y[r0 * k + e] = bounce[e];
}

// ------------------------------------------------------------------- host
static unsigned grid_for(int64_t n, int per = 256) {
  int64_t g = (n + per - 1) / per;
  const int64_t cap = (int64_t)device_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

static size_t elem_bytes(dtr_prec s) { return s == DTR_F64 ? 16 : (s == DTR_F32 ? 8 : 4); }
static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct EigLayout {
  int p, b, nk, rot_grid;
  size_t qy, fields, partial, mats, cmat, rtmp, resid, bounce, total;
};

static int eig_basis_size(const dtr_eig_params *P) {
  int p = P->p > 0 ? P->p : P->k + (P->k / 8 > 16 ? P->k / 8 : 16);
  return (p + 15) / 16 * 16;
}

static EigLayout eig_layout(const dtr_lattice_s &lat, const dtr_eig_params *P) {
  EigLayout L;
  L.p = eig_basis_size(P);
  L.b = P->chunk > 0 ? pad_rhs(P->chunk) : 32;
  const int64_t N = lat.N;
  const size_t es = elem_bytes(P->store);
  const size_t cs = P->store == DTR_F64 ? 16 : 8;  // chunk fields: FP64 or FP32 arithmetic
  const int tiles = ((L.p + kGT - 1) / kGT) * ((L.p + kGT - 1) / kGT);
  int64_t nk = (4LL * device_sms() + tiles - 1) / tiles;
  const int64_t maxk = N / 4096 > 0 ? N / 4096 : 1;
  if (nk > maxk) nk = maxk;
  if (nk < 1) nk = 1;
  L.nk = (int)nk;
  L.rot_grid = 2 * device_sms();
  L.qy = al256((size_t)N * L.p * es);
  L.fields = 4 * al256((size_t)N * L.b * cs);
  L.partial = al256((size_t)L.nk * L.p * L.p * sizeof(double2));
  L.mats = 3 * al256((size_t)L.p * L.p * sizeof(double2));
  L.cmat = al256((size_t)L.p * L.p * 16);
  L.rtmp = al256((size_t)L.rot_grid * kGT * L.p * es);
  L.resid = al256((size_t)4 * device_sms() * L.p * 2 * sizeof(double)) + al256((size_t)L.p * sizeof(double)) +
            al256((size_t)L.p * sizeof(double)) + al256((size_t)L.p * sizeof(int));
  L.bounce = 0;  // the compaction reuses the chunk fields
  L.total = 256 + L.qy + L.fields + L.partial + L.mats + L.cmat + L.rtmp + L.resid;
  return L;
}

size_t eig_workspace_bytes(const dtr_lattice_s &lat, const dtr_eig_params *P) { return eig_layout(lat, P).total; }

template <typename T>
static int eig_gram(const T *A, int a0, int na, const T *B, int b0, int nb, int p, int64_t N, int nk,
                    double2 *partial, double2 *out, cudaStream_t st) {
  const int tiles = ((na + kGT - 1) / kGT) * ((nb + kGT - 1) / kGT);
  k_eig_gram<T><<<dim3(tiles, nk), 256, 0, st>>>(A, p, a0, na, B, p, b0, nb, N, nk, partial);
  count_launches(1);
  k_eig_gram_reduce<<<grid_for((int64_t)na * nb), 256, 0, st>>>(partial, (int64_t)na * nb, nk, out);
  count_launches(1);
  DTR_LAUNCH_CHECK("eigensolver Gram");
  return DTR_OK;
}

// Chebyshev filter of columns [c0, c0 + w) of Y, then QY of the stored result.
template <typename T, typename R>
static int eig_filter_chunk(const dtr_gauge_s *g, double m0, T *Y, T *QY, int p, int c0, int w, int b, int deg,
                            double a, double bnd, double x0, void *fields, size_t fbytes, cudaStream_t st) {
  typedef typename cplx_t<R>::type C;
  const int64_t N = g->lat.N;
  const Geom geo = geom_of(g->lat);
  const C *U = (const C *)(sizeof(R) == 8 ? (const void *)g->U64 : (const void *)g->U32);
  C *F[4];
  for (int q = 0; q < 4; ++q) F[q] = (C *)((char *)fields + q * fbytes);
  C *Y0 = F[0], *Y1 = F[1], *SY = F[2], *Tm = F[3];
  const int64_t n = N * b;
  k_eig_gather<T, C><<<grid_for(n), 256, 0, st>>>(Y, N, p, c0, w, Y1, b);
  count_launches(1);
  const double e = 0.5 * (bnd - a), c = 0.5 * (bnd + a);
  const double tau = (x0 - c) / e;  // < -1: the scaling point lies below the damped interval
  double sig = 1.0 / tau;
  for (int j = 1; j <= deg; ++j) {
    // SY = A^H A Y1
    launch_dslash<R>(U, Y1, Tm, geo, b, m0, 0, st);
    launch_dslash<R>(U, Tm, SY, geo, b, m0, 1, st);
    double alpha, beta;
    if (j == 1) {
      alpha = sig / e;
      beta = 0.0;
    } else {
      const double sig2 = 1.0 / (2.0 * tau - sig);
      alpha = 2.0 * sig2 / e;
      beta = -sig * sig2;
      sig = sig2;
    }
    // Y0 <- alpha (SY - c Y1) + beta Y0, then (Y0, Y1) <- (Y1, Y0)
    if (j == 1) DTR_CUDA(cudaMemsetAsync(Y0, 0, (size_t)n * sizeof(C), st));
    k_eig_cheb<C, R><<<grid_for(n), 256, 0, st>>>(SY, Y1, Y0, n, (R)alpha, (R)beta, (R)c);
    count_launches(1);
    C *t = Y0;
    Y0 = Y1;
    Y1 = t;
  }
  k_eig_scatter<T, C><<<grid_for(N * w), 256, 0, st>>>(Y1, N, b, w, Y, p, c0, 0);
  count_launches(1);
  // QY = g5 A Y from the stored (rounded) columns
  k_eig_gather<T, C><<<grid_for(n), 256, 0, st>>>(Y, N, p, c0, w, Y1, b);
  count_launches(1);
  launch_dslash<R>(U, Y1, Tm, geo, b, m0, 0, st);
  k_eig_scatter<T, C><<<grid_for(N * w), 256, 0, st>>>(Tm, N, b, w, QY, p, c0, 1);
  count_launches(1);
  DTR_LAUNCH_CHECK("eigensolver filter");
  return DTR_OK;
}

// Host complex products for the p x p Rayleigh-Ritz algebra (row-major, threaded over output rows):
// C (m x n) = A (m x l) B (l x n), and C (m x n) = A^H B with A (l x m), B (l x n).
static void zgemm_nn(const std::vector<zc> &A, int m, int l, const std::vector<zc> &B, int n, std::vector<zc> &C) {
  C.assign((size_t)m * n, zc(0.0, 0.0));
  host_parallel_for(m, 64, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      zc *o = &C[(size_t)i * n];
      for (int q = 0; q < l; ++q) {
        const zc a = A[(size_t)i * l + q];
        if (a == zc(0.0, 0.0)) continue;
        const zc *b = &B[(size_t)q * n];
        for (int j = 0; j < n; ++j) o[j] += a * b[j];
      }
    }
  });
}
static void zgemm_hn(const std::vector<zc> &A, int l, int m, const std::vector<zc> &B, int n, std::vector<zc> &C) {
  C.assign((size_t)m * n, zc(0.0, 0.0));
  host_parallel_for(m, 64, [&](int64_t lo, int64_t hi) {
    for (int q = 0; q < l; ++q) {
      const zc *b = &B[(size_t)q * n];
      for (int64_t i = lo; i < hi; ++i) {
        const zc a = std::conj(A[(size_t)q * m + i]);
        zc *o = &C[(size_t)i * n];
        for (int j = 0; j < n; ++j) o[j] += a * b[j];
      }
    }
  });
}
static void hermitise(std::vector<zc> &X, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      const zc h = 0.5 * (X[(size_t)i * n + j] + std::conj(X[(size_t)j * n + i]));
      X[(size_t)i * n + j] = h;
      X[(size_t)j * n + i] = std::conj(h);
    }
}

// residual partials of the k leading stored columns, from a fresh stencil on each stored chunk
template <typename T, typename R>
static int eig_true_residuals(const dtr_gauge_s *g, double m0, const T *Y, int p, int k, int b, const double *thd,
                              void *fields, size_t fbytes, int nch, double *rpart, cudaStream_t st) {
  typedef typename cplx_t<R>::type C;
  const int64_t N = g->lat.N;
  const Geom geo = geom_of(g->lat);
  const C *U = (const C *)(sizeof(R) == 8 ? (const void *)g->U64 : (const void *)g->U32);
  C *X = (C *)fields, *AX = (C *)((char *)fields + fbytes);
  for (int c0 = 0; c0 < k; c0 += b) {
    const int w = (k - c0) < b ? (k - c0) : b;
    k_eig_gather<T, C><<<grid_for(N * b), 256, 0, st>>>(Y, N, p, c0, w, X, b);
    launch_dslash<R>(U, X, AX, geo, b, m0, 0, st);
    k_eig_resid_int<C><<<nch, 256, 0, st>>>(AX, X, N, b, w, c0, k, thd, nch, rpart);
    count_launches(2);
  }
  DTR_LAUNCH_CHECK("eigensolver residuals");
  return DTR_OK;
}

static void mat_from_dev(const std::vector<double2> &src, int n, std::vector<zc> &dst) {
  dst.resize((size_t)n * n);
  for (size_t q = 0; q < (size_t)n * n; ++q) dst[q] = zc(src[q].x, src[q].y);
}

template <typename T>
static int eig_solve_t(const dtr_gauge_s *gauge, double m0, const dtr_eig_params *P, void *work, size_t work_bytes,
                       dtr_defl_s *D, double *res_out, dtr_eig_stats *stats, cudaStream_t st) {
  typedef typename EigAcc<T>::type AC;
  const auto t_start = std::chrono::steady_clock::now();
  const EigLayout L = eig_layout(gauge->lat, P);
  if (work_bytes < L.total) return fail(DTR_ENOMEM, "eigensolver workspace too small");
  const int64_t N = gauge->lat.N;
  const int p = L.p, k = P->k, b = L.b;
  T *Y = (T *)D->V;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  T *QY = (T *)w;                   w += L.qy;
  void *fields = w;                 w += L.fields;
  double2 *partial = (double2 *)w;  w += L.partial;
  w += al256((size_t)p * p * sizeof(double2));  // (spare p x p slot)
  double2 *Md = (double2 *)w;       w += al256((size_t)p * p * sizeof(double2));
  double2 *Hd = (double2 *)w;       w += al256((size_t)p * p * sizeof(double2));
  AC *Cd = (AC *)w;                 w += L.cmat;
  T *rtmp = (T *)w;                 w += L.rtmp;
  double *rpart = (double *)w;      w += al256((size_t)4 * device_sms() * p * 2 * sizeof(double));
  double *thd = (double *)w;        w += al256((size_t)p * sizeof(double));
  double *scd = (double *)w;        w += al256((size_t)p * sizeof(double));
  int *permd = (int *)w;
  const size_t fbytes = L.fields / 4;
  const bool f64 = P->store == DTR_F64;
  const uint64_t seed = P->seed;
  // spectrum of S = A^H A lies in [0, (|4 + m0| + 4)^2]: the hopping term of direction mu is
  // P- T+ + P+ T- with the spin projectors P+- = (1 +- gamma_mu)/2 commuting with the link-shifts
  // T+-, so its square is P- + P+ = 1 and it has norm 1; four directions add at most 4
  const double bnd = std::pow(std::fabs(4.0 + m0) + 4.0, 2) * 1.001;
  double a = P->first_cut > 0.0 ? P->first_cut : 0.1 * bnd;
  double x0 = 0.0;
  k_eig_random<T><<<grid_for(N * p), 256, 0, st>>>(Y, N, p, 0, p, seed, 0);
  count_launches(1);
  std::vector<double2> hM((size_t)p * p), hH((size_t)p * p);
  std::vector<zc> M, H, Wg, Zs;
  std::vector<double> g, mu, theta(k, 0.0), res(k, INFINITY);
  int it = 0, nconv = 0, r = p;
  double maxres = INFINITY;
  const double drop = f64 ? 1e-12 : (P->store == DTR_F32 ? 1e-7 : 1e-4);
  double t_filter = 0.0, t_gram = 0.0, t_host = 0.0, t_rot = 0.0;
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto secs_since = [&](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(now() - t).count();
  };
  for (it = 1; it <= P->max_iter; ++it) {
    const int deg = (it == 1 && P->first_degree > 0) ? P->first_degree : P->degree;
    auto tp = now();
    for (int c0 = 0; c0 < p; c0 += b) {
      const int wc = (p - c0) < b ? (p - c0) : b;
      int rc = f64 ? eig_filter_chunk<T, double>(gauge, m0, Y, QY, p, c0, wc, b, deg, a, bnd, x0, fields, fbytes, st)
                   : eig_filter_chunk<T, float>(gauge, m0, Y, QY, p, c0, wc, b, deg, a, bnd, x0, fields, fbytes, st);
      if (rc) return rc;
    }
    DTR_CUDA(cudaStreamSynchronize(st));
    t_filter += secs_since(tp);
    tp = now();
    int rc = eig_gram<T>(QY, 0, p, QY, 0, p, p, N, L.nk, partial, Md, st);
    if (!rc) rc = eig_gram<T>(Y, 0, p, QY, 0, p, p, N, L.nk, partial, Hd, st);
    if (rc) return rc;
    DTR_CUDA(cudaMemcpyAsync(hM.data(), Md, sizeof(double2) * p * p, cudaMemcpyDeviceToHost, st));
    DTR_CUDA(cudaMemcpyAsync(hH.data(), Hd, sizeof(double2) * p * p, cudaMemcpyDeviceToHost, st));
    DTR_CUDA(cudaStreamSynchronize(st));
    t_gram += secs_since(tp);
    tp = now();
    mat_from_dev(hM, p, M);
    mat_from_dev(hH, p, H);
    hermitise(M, p);  // the Grams are Hermitian up to rounding
    hermitise(H, p);
    // Harmonic Rayleigh-Ritz for the target 0: (Q y - theta y) orthogonal to Q span(Y), i.e.
    // H c = nu M c with nu = 1 / theta.  M is positive definite, so this is a Hermitian-definite
    // pencil whose wanted values (theta near 0) are its exterior ones (|nu| largest): no spurious
    // Ritz values near 0, which a Rayleigh-Ritz step for the indefinite Q could produce (its wanted
    // eigenvalues are interior ones).  M-orthonormal basis by canonical orthogonalisation,
    // M = W g W^H with directions of tiny g dropped.
    if (herm_eig(p, M, g, Wg)) return fail(DTR_ENOTCONV, "eigensolver: Gram eigendecomposition did not converge");
    const double gmax = g[p - 1];
    std::vector<int> keep;
    for (int i = p - 1; i >= 0; --i)
      if (g[i] > drop * gmax) keep.push_back(i);
    r = (int)keep.size();
    if (r < k) return fail(DTR_ENOTCONV, "eigensolver: the filtered basis lost rank below k");
    std::vector<zc> Bm((size_t)p * r);  // B = W_keep g^-1/2
    for (int i = 0; i < p; ++i)
      for (int q = 0; q < r; ++q) Bm[(size_t)i * r + q] = Wg[(size_t)i * p + keep[q]] / std::sqrt(g[keep[q]]);
    std::vector<zc> HB, Hh, Cr, GC;
    zgemm_nn(H, p, p, Bm, r, HB);
    zgemm_hn(Bm, p, r, HB, r, Hh);
    hermitise(Hh, r);
    std::vector<double> nu;
    if (herm_eig(r, Hh, nu, Zs)) return fail(DTR_ENOTCONV, "eigensolver: Rayleigh-Ritz did not converge");
    std::vector<int> ord(r);
    for (int q = 0; q < r; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return std::fabs(nu[x]) > std::fabs(nu[y]); });
    std::vector<zc> Zo((size_t)r * r);
    for (int x = 0; x < r; ++x)
      for (int q = 0; q < r; ++q) Zo[(size_t)x * r + q] = Zs[(size_t)x * r + ord[q]];
    zgemm_nn(Bm, p, r, Zo, r, Cr);  // harmonic Ritz coefficients, ||Q y_q|| = 1
    std::vector<AC> hC((size_t)p * r);
    for (int i = 0; i < p; ++i)
      for (int q = 0; q < r; ++q) {
        hC[(size_t)i * r + q].x = Cr[(size_t)i * r + q].real();
        hC[(size_t)i * r + q].y = Cr[(size_t)i * r + q].imag();
      }
    t_host += secs_since(tp);
    tp = now();
    // Y <- Y C (QY is rebuilt after the next filter, so it is not rotated)
    DTR_CUDA(cudaMemcpyAsync(Cd, hC.data(), sizeof(AC) * (size_t)p * r, cudaMemcpyHostToDevice, st));
    k_eig_rotate<T><<<L.rot_grid, 256, 0, st>>>(Y, N, p, r, Cd, rtmp);
    count_launches(1);
    int nch = 4 * device_sms();
    if (nch > N) nch = (int)N;
    // ||y_q||^2 of the rotated columns; then mu_q = ||Q y_q||^2 / ||y_q||^2 = 1 / ||y_q||^2 (the Ritz
    // value of S) and the columns are scaled to unit length.  The eigenvalue kept for a pair is the
    // harmonic Ritz value theta_q = 1 / nu_q: the same as the Rayleigh quotient y^H Q y / y^H y =
    // nu_q / ||y_q||^2 once a pair has converged, but for a vector that is not yet an eigenvector
    // the Rayleigh quotient of the indefinite Q can lie near 0, while |nu_q| = |y^H Q y| / ||Q y||^2
    // <= 1 / ||Q y|| <= 1 / sigma_min keeps 1 / theta bounded in the deflation
    k_eig_colnorm<T><<<dim3(nch, (r + 127) / 128), 128, 0, st>>>(Y, N, p, r, nch, rpart);
    count_launches(1);
    DTR_LAUNCH_CHECK("eigensolver rotation");
    std::vector<double> hn((size_t)nch * r), y2(r, 0.0), thq(r), sc(r);
    DTR_CUDA(cudaMemcpyAsync(hn.data(), rpart, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, st));
    DTR_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < nch; ++c)
      for (int q = 0; q < r; ++q) y2[q] += hn[(size_t)c * r + q];
    mu.assign(r, 0.0);
    double mu_lo = INFINITY, mu_hi = 0.0;
    for (int q = 0; q < r; ++q) {
      mu[q] = 1.0 / y2[q];
      thq[q] = 1.0 / nu[ord[q]];
      sc[q] = 1.0 / std::sqrt(y2[q]);
      mu_lo = std::min(mu_lo, mu[q]);
      mu_hi = std::max(mu_hi, mu[q]);
    }
    for (int j = 0; j < k; ++j) theta[j] = thq[j];
    DTR_CUDA(cudaMemcpyAsync(scd, sc.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    DTR_CUDA(cudaMemcpyAsync(thd, theta.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    k_eig_scale<T><<<grid_for(N * r), 256, 0, st>>>(Y, N, p, r, scd);
    count_launches(1);
    if (r < p) {
      k_eig_random<T><<<grid_for(N * (p - r)), 256, 0, st>>>(Y, N, p, r, p, seed, (uint64_t)it);
      count_launches(1);
    }
    // true residuals of the k leading stored Ritz vectors (a fresh stencil on each stored chunk,
    // so the rounding of the stored QY does not enter)
    {
      const int rc2 = f64 ? eig_true_residuals<T, double>(gauge, m0, Y, p, k, b, thd, fields, fbytes, nch, rpart, st)
                          : eig_true_residuals<T, float>(gauge, m0, Y, p, k, b, thd, fields, fbytes, nch, rpart, st);
      if (rc2) return rc2;
    }
    std::vector<double> hr((size_t)nch * k * 2);
    DTR_CUDA(cudaMemcpyAsync(hr.data(), rpart, sizeof(double) * hr.size(), cudaMemcpyDeviceToHost, st));
    DTR_CUDA(cudaStreamSynchronize(st));
    t_rot += secs_since(tp);
    maxres = 0.0;
    nconv = 0;
    for (int j = 0; j < k; ++j) {
      double r2 = 0.0, y2 = 0.0;
      for (int c = 0; c < nch; ++c) {
        r2 += hr[((size_t)c * k + j) * 2];
        y2 += hr[((size_t)c * k + j) * 2 + 1];
      }
      res[j] = std::sqrt(r2 / y2) / (P->tol_ref ? std::sqrt(bnd / 1.001) : std::fabs(theta[j]));
      if (res[j] <= P->tol) ++nconv;
      if (res[j] > maxres) maxres = res[j];
    }
    // next filter: damp the S spectrum above the largest kept Ritz value, scale at the smallest
    a = mu_hi;
    x0 = 0.5 * mu_lo;
    if (a >= bnd * 0.999) a = 0.5 * bnd;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (nconv == k) break;
    if (P->time_limit_s > 0.0 && secs >= P->time_limit_s) break;
  }
  if (it > P->max_iter) it = P->max_iter;
  // order the k pairs by |lambda| (ties by lambda) and compact [dof][p] -> [dof][k] in that
  // column order, in place (row chunks through a bounce buffer)
  std::vector<int> perm(k);
  for (int j = 0; j < k; ++j) perm[j] = j;
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) {
    return std::fabs(theta[x]) < std::fabs(theta[y]) || (std::fabs(theta[x]) == std::fabs(theta[y]) && theta[x] < theta[y]);
  });
  {
    std::vector<double> t2(k), r2(k);
    for (int j = 0; j < k; ++j) {
      t2[j] = theta[perm[j]];
      r2[j] = res[perm[j]];
    }
    theta.swap(t2);
    res.swap(r2);
  }
  DTR_CUDA(cudaMemcpyAsync(permd, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
  {
    T *bounce = (T *)fields;
    int64_t rows = (int64_t)(L.fields / (elem_bytes(P->store) * (size_t)k));
    if (rows > N) rows = N;
    for (int64_t r0 = 0; r0 < N; r0 += rows) {
      const int64_t r1 = (r0 + rows) < N ? r0 + rows : N;
      k_eig_compact_out<T><<<grid_for((r1 - r0) * k), 256, 0, st>>>(Y, p, k, r0, r1, permd, bounce);
      k_eig_compact_in<T><<<grid_for((r1 - r0) * k), 256, 0, st>>>(bounce, k, r0, r1, Y);
      count_launches(2);
    }
    DTR_LAUNCH_CHECK("eigensolver compaction");
  }
  // normalise: the Ritz vectors are unit vectors up to the storage rounding; lambda = theta
  std::vector<double> il(k);
  for (int j = 0; j < k; ++j) il[j] = 1.0 / theta[j];
  DTR_CUDA(cudaMemcpyAsync(D->inv_lambda, il.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  if (res_out)
    for (int j = 0; j < k; ++j) res_out[j] = res[j];
  if (stats) {
    stats->iterations = it;
    stats->converged = nconv;
    stats->basis = p;
    stats->max_residual = maxres;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    stats->cut = a;
    stats->bound = bnd;
    stats->t_filter = t_filter;
    stats->t_gram = t_gram;
    stats->t_host = t_host;
    stats->t_rotate = t_rot;
  }
  return DTR_OK;
}

int eig_solve(const dtr_gauge_s *g, double m0, const dtr_eig_params *P, void *work, size_t work_bytes,
              dtr_defl_s *D, double *res_out, dtr_eig_stats *stats, cudaStream_t st) {
  if (P->store == DTR_F64) return eig_solve_t<double2>(g, m0, P, work, work_bytes, D, res_out, stats, st);
  if (P->store == DTR_F32) return eig_solve_t<float2>(g, m0, P, work, work_bytes, D, res_out, stats, st);
  return eig_solve_t<bfc2>(g, m0, P, work, work_bytes, D, res_out, stats, st);
}

int eig_basis_columns(const dtr_eig_params *P) { return eig_basis_size(P); }

}  // namespace dtr
