// Persistent (single cooperative launch) batched BiCGStab.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "solver.cuh"

namespace dtr {

// Grid barrier state.  The per-launch part (up to `error`) is zeroed before
// every persistent launch; `error` and `cycles` are zeroed once per solve, so
// a timeout in any cycle stays visible to the host.
struct GridSync {
  unsigned int count;       // arrivals so far (barrier n completes at n * gridDim.x)
  int iters;                // BiCGStab iterations the launch executed (written by block 0)
  unsigned long long nt0;   // ~(earliest block entry), device global timer (ns), via atomicMax
  unsigned long long t1;    // latest block exit (ns)
  int error;                // sticky: a barrier wait gave up
  unsigned int cycles;      // defect-correction cycles run by the graph-driven loop
  int sel;                  // mixed solver: the next residual is the double-float update (1) or FP64 (0)
  int last_upd;             // mixed solver: the last residual computed was the double-float update
  int fp64_cert;            // mixed solver: ||x|| / ||z|| too large for the double-float true residual
};
constexpr size_t kGridSyncLaunchBytes = offsetof(GridSync, error);

// S: storage type of the Krylov vectors r, rhat, p, v, s, t (the arithmetic is
// in R; the iterate x is stored in R).  S = complex R, or __half2 /
// __nv_bfloat162 for the half-storage inner solve (FP32 arithmetic).
template <typename R, typename S = typename cplx_t<R>::type> struct PArgs {
  const typename cplx_t<R>::type *U;
  typename cplx_t<R>::type *x;
  S *r, *rhat, *p, *v, *s, *t;
  const typename cplx_t<R>::type *z;  // right-hand sides (true-residual cycles only)
  Geom g;
  int b, logb;
  R diag;
  Scal *sc;
  double2 *partial;  // [grid][2][b]
  GridSync *gs;
  int max_iters;     // iteration cap of one cycle (safety; per-column maxiter is in Scal)
  int max_cycles;    // true-residual restart cycles (with_resid only)
  int grid;          // requested CTAs (0 = all co-resident)
};

// with_resid = 1: cycles of (true residual r = z - A x, restart decision,
// iterations) until every column meets tol in the true residual (FP64 path);
// with_resid = 0: iterations only, from the caller-initialised state.
template <typename R> int launch_persistent(const PArgs<R> &pa, int with_resid, cudaStream_t st);
// Inner iterations with the Krylov vectors stored in S (FP16 or BF16), FP32 arithmetic.
template <typename S> int launch_persistent_half(const PArgs<float, S> &pa, cudaStream_t st);

// Optional timing of persistent launches (for roofline accounting): every
// block stamps the device global timer at entry and exit, and a one-thread
// kernel after the launch folds (last exit - first entry) and the iterations
// into a device accumulator (works inside CUDA graphs, where events cannot be
// recorded in a conditional body).
struct PersistProfile {
  bool on;
  double ms;
  long long launches;
  double site_rhs_iters;  // sum over launches of iterations * V * b
};
PersistProfile &persist_profile();
// Called after the stream has been synchronised: folds the device accumulator in.
void persist_profile_flush(cudaStream_t st);
// Enqueue the accounting kernel for the launch that just used `gs` (profiling on).
int persist_account(const GridSync *gs, double site_rhs, cudaStream_t st);
// Kernels launched by device-driven graph loops (counted on the device).
unsigned long long device_launch_count();
// Pointer to the device counter of graph-launched kernels.
unsigned long long *device_launch_counter();

// Launch one block at a barrier that expects two (the peer never arrives);
// reports whether the bounded wait gave up and the barrier's error word.
int selftest_barrier(long long budget, int *timed_out, int *error_word, cudaStream_t st);

}  // namespace dtr
