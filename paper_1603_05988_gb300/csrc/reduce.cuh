// Deterministic per-RHS cross-block reductions with a last-block finalize.
//
// Threads are laid out so that column j = threadIdx.x & (b-1) is fixed for a
// thread (blockDim and the grid stride are multiples of b).  Each block
// reduces its NV complex values per column in shared memory (a fixed tree),
// writes them to partial[block][q][j], and the last block to arrive (ticket
// from an atomic counter) sums the partials of all blocks in a fixed order and
// calls the finalize functor once per column.  The result is bit-identical
// from run to run.
#pragma once

#include "dtr_internal.cuh"

namespace dtr {

constexpr int kBlock = 256;     // threads per block of every reducing kernel
constexpr int kMaxGrid = 2048;  // upper bound on the grid of reducing kernels

// Returns true in the last block; tot[q*b + j] (shared) then holds the sums.
template <int NV>
__device__ __forceinline__ bool block_reduce(const double2 (&v)[NV], int b, double2 *__restrict__ partial,
                                             unsigned int *counter, double2 *tot) {
  __shared__ double2 sh[NV * kBlock];
  __shared__ int is_last;
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q * kBlock + t] = v[q];
  __syncthreads();
  for (int stride = kBlock / 2; stride >= b; stride >>= 1) {
    if (t < stride) {
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[q * kBlock + t] = cadd(sh[q * kBlock + t], sh[q * kBlock + t + stride]);
    }
    __syncthreads();
  }
  if (t < b) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partial[((int64_t)blockIdx.x * NV + q) * b + t] = sh[q * kBlock + t];
  }
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // last block: P = NV*b (q, j) pairs, S = kBlock / P slices of the block range
  const int P = NV * b;
  const int S = kBlock / P;
  const int p = t % P, sl = t / P;
  double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0, a3 = a0;
  if (sl < S) {
    const int q = p / b, j = p % b;
    const int G = (int)gridDim.x;
    int blk = sl;
    for (; blk + 3 * S < G; blk += 4 * S) {
      a0 = cadd(a0, __ldcg(&partial[((int64_t)blk * NV + q) * b + j]));
      a1 = cadd(a1, __ldcg(&partial[((int64_t)(blk + S) * NV + q) * b + j]));
      a2 = cadd(a2, __ldcg(&partial[((int64_t)(blk + 2 * S) * NV + q) * b + j]));
      a3 = cadd(a3, __ldcg(&partial[((int64_t)(blk + 3 * S) * NV + q) * b + j]));
    }
    for (; blk < G; blk += S) a0 = cadd(a0, __ldcg(&partial[((int64_t)blk * NV + q) * b + j]));
  }
  const double2 acc = cadd(cadd(a0, a1), cadd(a2, a3));
  __syncthreads();
  sh[t] = acc;
  __syncthreads();
  if (t < P) {
    double2 s = sh[t];
    for (int k = 1; k < S; ++k) s = cadd(s, sh[k * P + t]);
    tot[t] = s;
  }
  __syncthreads();
  if (t == 0) *counter = 0u;
  return true;
}

inline unsigned reduce_grid(int64_t items, int sms) {
  int64_t g = (items + kBlock - 1) / kBlock;
  int64_t cap = (int64_t)sms * 2;
  if (cap > kMaxGrid) cap = kMaxGrid;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

int device_sms();

}  // namespace dtr
