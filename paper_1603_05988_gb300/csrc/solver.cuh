// Solver state shared between the solver and the estimator driver.
#pragma once

#include "dtr_internal.cuh"

namespace dtr {

constexpr int kFlagNaN = 1;
constexpr int kFlagBreakdown = 2;
constexpr int kMaxRestarts = 32;  // true-residual restarts / defect-correction cycles per column
constexpr double kInnerTolFloorF16 = 2e-4;   // least inner reduction asked of FP16-stored inner vectors
constexpr double kInnerTolFloorBF16 = 1e-2;  // and of BF16-stored ones

// Per-column Krylov scalars, resident in device memory (b <= 64 columns).
struct Scal {
  double2 rho[64], alpha[64], omega[64], beta[64];
  double rnorm2[64], bnorm2[64], rtrue2[64], scale[64];
  int active[64], iters[64], restarts[64], conv[64], flags[64];
  int n_active;
  int maxiter;
  double tol2;
};

template <typename R> struct KrylovVecs {
  typename cplx_t<R>::type *x, *r, *rhat, *p, *v, *t;
};

// Scratch the solver needs beyond the solution and right-hand-side blocks.
size_t solver_scratch_bytes(int64_t V, int b, int solver, int gmres_m = 16);

// Solve A x = z on internal-layout FP64 blocks of width b.  x holds the
// initial guess on entry.  *scal receives the device pointer of the final
// per-column statistics (inside `work`).
// x_is_zero: the caller guarantees x == 0 on entry (skips one FP64 stencil).
// async: with the persistent engine (FP64, or the graph-driven mixed solver)
// return as soon as the work is queued, without synchronising `st`; the caller
// reads *solver_error_word(work) after synchronising (non-zero = a grid barrier
// timed out, DTR_ETIMEOUT).  Other solvers synchronise regardless.
int solve_internal(const dtr_gauge_s *gauge, double m0, double2 *x, const double2 *z, int b,
                   const dtr_solve_params *p, void *work, size_t work_bytes, cudaStream_t st, Scal **scal,
                   int x_is_zero = 0, int async = 0);
// True if solve_internal honours `async` for these parameters.
bool solve_can_run_async(const dtr_solve_params *p);
// Device address of the solver's sticky barrier error word inside `work`.
int *solver_error_word(void *work);

// Graph-driven mixed solve: process-wide counts of captured graphs and of
// graph launches.
int graph_counters(unsigned long long *captures, unsigned long long *launches);

}  // namespace dtr
