// Per-column scalar algebra of BiCGStab, run by one thread per column in the
// block that finalises a grid-wide reduction (shared by both solver engines).
#pragma once

#include "solver.cuh"

namespace dtr {

// All run in the finalising block, thread j < b, with the grid totals of column j.

__device__ __forceinline__ void count_active(Scal *sc, int b) {
  // called by thread 0 after a __syncthreads in the caller
  int n = 0;
  for (int j = 0; j < b; ++j) n += sc->active[j];
  sc->n_active = n;
}

// true residual r = z - A x: tot = (||r||^2, ||z||^2)
__device__ __forceinline__ void fin_resid(Scal *sc, int j, double2 t0, int restart) {
  const double r2 = t0.x, z2 = t0.y;
  sc->bnorm2[j] = z2;
  sc->rtrue2[j] = r2;
  const bool nan = !(r2 == r2) || !(z2 == z2) || isinf(r2);
  const bool conv = (z2 == 0.0) || (r2 <= sc->tol2 * z2);
  sc->conv[j] = conv ? 1 : 0;
  if (nan) sc->flags[j] |= kFlagNaN;
  if (!conv && !nan && sc->iters[j] < sc->maxiter && sc->restarts[j] < kMaxRestarts && restart) {
    sc->active[j] = 1;
    sc->restarts[j] += 1;
    sc->rho[j] = make_double2(r2, 0.0);
    sc->rnorm2[j] = r2;
    sc->scale[j] = 1.0 / sqrt(r2);
  } else {
    sc->active[j] = 0;
  }
}

__device__ __forceinline__ void fin_alpha(Scal *sc, int j, double2 sigma) {
  if (!sc->active[j]) {
    sc->alpha[j] = make_double2(0.0, 0.0);
    return;
  }
  if (sigma.x == 0.0 && sigma.y == 0.0) {
    sc->flags[j] |= kFlagBreakdown;
    sc->active[j] = 0;
    sc->alpha[j] = make_double2(0.0, 0.0);
    return;
  }
  sc->alpha[j] = cdiv(sc->rho[j], sigma);
}

__device__ __forceinline__ void fin_omega(Scal *sc, int j, double2 ts, double2 tt) {
  if (!sc->active[j] || tt.x == 0.0) {
    sc->omega[j] = make_double2(0.0, 0.0);
    return;
  }
  sc->omega[j] = make_double2(ts.x / tt.x, ts.y / tt.x);
}

__device__ __forceinline__ void fin_beta(Scal *sc, int j, double2 rr0, double2 rr) {
  if (!sc->active[j]) {
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  sc->iters[j] += 1;
  const double rn2 = rr.x;
  sc->rnorm2[j] = rn2;
  if (!(rn2 == rn2) || isinf(rn2)) {
    sc->flags[j] |= kFlagNaN;
    sc->active[j] = 0;
    return;
  }
  if (rn2 <= sc->tol2 * sc->bnorm2[j]) {  // converged on the recursive residual
    sc->active[j] = 0;
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  if (sc->iters[j] >= sc->maxiter) {
    sc->active[j] = 0;
    return;
  }
  const double2 om = sc->omega[j];
  const double2 rho = sc->rho[j];
  if ((om.x == 0.0 && om.y == 0.0) || (rho.x == 0.0 && rho.y == 0.0)) {
    sc->flags[j] |= kFlagBreakdown;
    sc->active[j] = 0;
    return;
  }
  sc->beta[j] = cmul(cdiv(rr0, rho), cdiv(sc->alpha[j], om));
  sc->rho[j] = rr0;
}

// Merged omega/beta step of the three-barrier iteration.  From the reductions
// of the t = A s phase -- ts = t^H s, tt = t^H t, rs = rhat^H s, rt = rhat^H t,
// ss = s^H s -- everything the rest of the iteration needs follows without a
// further grid reduction:
//   omega  = ts / tt
//   rho'   = rhat^H (s - omega t)      = rs - omega rt
//   |r'|^2 = |s - omega t|^2            = ss - |ts|^2 / tt
//   beta   = (rho' / rho) (alpha / omega)
// (|r'|^2 is the recursive residual used only for the convergence test; the
// FP64 true residual certifies the result.)
__device__ __forceinline__ void fin_omega_beta(Scal *sc, int j, double2 ts, double2 tt, double2 rs, double2 rt,
                                               double2 ss) {
  if (!sc->active[j]) {
    sc->omega[j] = make_double2(0.0, 0.0);
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  sc->iters[j] += 1;
  double2 om = make_double2(0.0, 0.0);
  double rn2 = ss.x;
  if (tt.x > 0.0) {
    const double inv_tt = 1.0 / tt.x;
    om = make_double2(ts.x * inv_tt, ts.y * inv_tt);
    rn2 = ss.x - (ts.x * ts.x + ts.y * ts.y) * inv_tt;
    if (rn2 < 0.0) rn2 = 0.0;
  }
  sc->omega[j] = om;
  sc->rnorm2[j] = rn2;
  if (!(rn2 == rn2) || isinf(rn2)) {
    sc->flags[j] |= kFlagNaN;
    sc->active[j] = 0;
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  if (rn2 <= sc->tol2 * sc->bnorm2[j] || sc->iters[j] >= sc->maxiter) {
    sc->active[j] = 0;                 // x and r still take this iteration's update
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  const double2 rho = sc->rho[j];
  if ((om.x == 0.0 && om.y == 0.0) || (rho.x == 0.0 && rho.y == 0.0)) {
    sc->flags[j] |= kFlagBreakdown;
    sc->active[j] = 0;
    sc->beta[j] = make_double2(0.0, 0.0);
    return;
  }
  const double2 rho_new = csub(rs, cmul(om, rt));
  sc->beta[j] = cdiv(cmul(rho_new, sc->alpha[j]), cmul(rho, om));  // (rho'/rho)(alpha/omega), one division
  sc->rho[j] = rho_new;
}

}  // namespace dtr
