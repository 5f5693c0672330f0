// Persistent (single cooperative launch) batched BiCGStab.
#pragma once

#include "solver.cuh"

namespace dtr {

// Grid barrier state, zeroed before every launch.
struct GridSync {
  unsigned int count;  // arrivals so far (barrier n completes at n * gridDim.x)
  unsigned int gen;    // unused (layout kept)
  int error;
  int iters;  // BiCGStab iterations the launch executed (written by block 0 at exit)
};

template <typename R> struct PArgs {
  const typename cplx_t<R>::type *U;
  typename cplx_t<R>::type *x, *r, *rhat, *p, *v, *s, *t;
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

// Optional event timing of persistent launches (for roofline accounting).
struct PersistProfile {
  bool on;
  double ms;
  long long launches;
  double site_rhs_iters;  // sum over launches of iterations * V * b
};
PersistProfile &persist_profile();
// Called after the stream has been synchronised: folds the recorded launches in.
void persist_profile_flush(cudaStream_t st);

// Launch one block at a barrier that expects two (the peer never arrives);
// reports whether the bounded wait gave up and the barrier's error word.
int selftest_barrier(long long budget, int *timed_out, int *error_word, cudaStream_t st);

}  // namespace dtr
