// Batched BiCGStab for A y = z (the solve step of Algorithm 1), one column per probing
// vector, all columns of a block advanced together with per-column scalars
// kept on the device.  Two drivers:
//   * plain FP64 BiCGStab with true-residual restarts;
//   * mixed precision: FP64 defect correction (r = z - A y in FP64, y
//     accumulated in FP64) around FP32 BiCGStab inner solves.
// Every iteration is five kernels: fused dslash + dot (alpha), s = r - alpha v,
// fused dslash + two dots (omega), fused x/r update + two dots (beta and the
// convergence test), p update.  The scalar algebra of each step runs in the
// last block of the reducing kernel, so the host only polls a device-side
// active-column count every `check_every` iterations.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "dslash_core.cuh"
#include "reduce.cuh"
#include "solver.cuh"
#include "krylov_fin.cuh"
#include "net.cuh"
#include "persist.cuh"

namespace dtr {

int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ------------------------------------------------------------------ kernels
template <typename R> struct Vec { typedef typename cplx_t<R>::type C; };

template <typename C> __device__ __forceinline__ C scal_as(double2 v) { return mk<C>(v.x, v.y); }

// acc += conj(a) * b, in the field's own precision (FP64 work on GB300 costs
// 61 FP32 operations; the block and grid sums that follow are FP64)
__device__ __forceinline__ double2 dot_acc(double2 acc, double2 a, double2 b) {
  return make_double2(acc.x + a.x * b.x + a.y * b.y, acc.y + a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 dot_acc(float2 acc, float2 a, float2 b) {
  return make_float2(acc.x + a.x * b.x + a.y * b.y, acc.y + a.x * b.y - a.y * b.x);
}
template <typename C> __device__ __forceinline__ double2 to_d2(C a) { return make_double2((double)a.x, (double)a.y); }

// r = z - A x; optionally rhat = p = r.  tot = (||r||^2, ||z||^2).
template <typename R, int KRYLOV>
__global__ void __launch_bounds__(kBlock) k_resid(const typename cplx_t<R>::type *__restrict__ U,
                                                  const typename cplx_t<R>::type *__restrict__ x,
                                                  const typename cplx_t<R>::type *__restrict__ z,
                                                  typename cplx_t<R>::type *__restrict__ r,
                                                  typename cplx_t<R>::type *__restrict__ rhat,
                                                  typename cplx_t<R>::type *__restrict__ p, Geom g, int b, int logb,
                                                  R diag, Scal *sc, Reduce red, int restart,
                                                  const int *run_flag, int run_if, int *mark,
                                                  const int *run_if_set = nullptr) {
  typedef typename cplx_t<R>::type C;
  __shared__ double2 tot[64];
  if (run_flag && *(volatile const int *)run_flag != run_if) return;  // not selected (uniform over the grid)
  if (run_if_set && *(volatile const int *)run_if_set == 0) return;    // (second condition, likewise)
  double2 acc[1] = {make_double2(0.0, 0.0)};
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    C o[12], self[12];
    dslash_site<1, R>(U, x, g, b, s, j, diag, o, self);
    const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const C zz = z[base + c * b];
      const C rr = csub(zz, o[c]);
      r[base + c * b] = rr;
      if (KRYLOV) {
        rhat[base + c * b] = rr;
        p[base + c * b] = rr;
      }
      acc[0].x += (double)rr.x * rr.x + (double)rr.y * rr.y;
      acc[0].y += (double)zz.x * zz.x + (double)zz.y * zz.y;
    }
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_resid(sc, threadIdx.x, tot[threadIdx.x], restart);
    __syncthreads();
    if (threadIdx.x == 0) {
      count_active(sc, b);
      if (mark) *mark = 0;
    }
  }
}

// x == 0: r = z (no stencil); tot = (||z||^2, ||z||^2)
__global__ void __launch_bounds__(kBlock) k_resid_zero(const double2 *__restrict__ z, double2 *__restrict__ r,
                                                       int64_t n, int b, Scal *sc, Reduce red) {
  __shared__ double2 tot[64];
  double2 acc[1] = {make_double2(0.0, 0.0)};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 zz = z[e];
    r[e] = zz;
    const double q = zz.x * zz.x + zz.y * zz.y;
    acc[0].x += q;
    acc[0].y += q;
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_resid(sc, threadIdx.x, tot[threadIdx.x], 1);
    __syncthreads();
    if (threadIdx.x == 0) count_active(sc, b);
  }
}

// Residual after a defect-correction cycle without an FP64 stencil: the cycle added
// e / (hs * scale) to x (k_mixed_accum), so r -= A e / (hs * scale), with A e
// evaluated in double-float arithmetic (links split into FP32 hi + lo, e exact in
// FP32): relative error ~2^-46 of |A| |e|, so r stays the true residual of x to
// ~1e-14 kappa |z| over all cycles.  tot = (||r||^2, ||z||^2 as stored).  A true
// residual (k_resid_df) confirms convergence before the solve reports it.
// (Two blocks per SM: the register cap spills ~500 B per thread to L1, yet the solve runs ~2% faster
// than with one block of 255-register threads.)
__global__ void __launch_bounds__(kBlock, 2) k_resid_update(const cdf *__restrict__ Udf, const float2 *__restrict__ e,
                                                         double2 *__restrict__ r, Geom g, int b, int logb, dff diag,
                                                         double hs, Scal *sc, Reduce red, const int *run_flag,
                                                         int run_if, int *mark) {
  __shared__ double2 tot[64];
  if (run_flag && *(volatile const int *)run_flag != run_if) return;  // not selected (uniform over the grid)
  double2 acc[1] = {make_double2(0.0, 0.0)};
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  const double inv = sc->active[j] ? 1.0 / (sc->scale[j] * hs) : 0.0;
  const F32AsDf ld{e};
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    const int64_t base = (int64_t)s * 12 * b + j;
    if (inv != 0.0) {
      cdf o[12], self[12];
      dslash_site_ld<1, dff>(Udf, ld, g, b, s, j, diag, o, self);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        double2 rr = r[base + c * b];
        rr.x = fma(-inv, (double)o[c].x.hi + (double)o[c].x.lo, rr.x);
        rr.y = fma(-inv, (double)o[c].y.hi + (double)o[c].y.lo, rr.y);
        r[base + c * b] = rr;
        acc[0].x += rr.x * rr.x + rr.y * rr.y;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const double2 rr = r[base + c * b];
        acc[0].x += rr.x * rr.x + rr.y * rr.y;
      }
    }
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_resid(sc, threadIdx.x, make_double2(tot[threadIdx.x].x, sc->bnorm2[threadIdx.x]), 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      count_active(sc, b);
      if (mark) *mark = 1;
    }
  }
}

// x (FP64) as double-float hi + lo for the true residual below: hi = x rounded to FP32, lo = the
// remainder rounded to FP32 (hi + lo equals x to ~2^-48 relative)
// It also measures ||x|| per column: where ||x|| / ||z|| exceeds kDfCertRatio (||z|| from the
// previous residual) the double-float residual's error (~1e-13 ||x|| / ||z||) would no longer be
// negligible next to a 1e-10 tolerance, and *fp64_cert selects the FP64 residual instead.
constexpr double kDfCertRatio = 30.0;
__global__ void __launch_bounds__(kBlock) k_split_df(const double2 *__restrict__ x, float2 *__restrict__ hi,
                                                     float2 *__restrict__ lo, int64_t n, int b, const Scal *sc,
                                                     Reduce red, int *fp64_cert, const int *run_flag, int run_if) {
  __shared__ double2 tot[64];
  __shared__ int any;
  if (run_flag && *(volatile const int *)run_flag != run_if) return;  // not selected (uniform over the grid)
  double2 acc[1] = {make_double2(0.0, 0.0)};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
    hi[e] = make_float2(hx, hy);
    lo[e] = make_float2(__double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
    acc[0].x += v.x * v.x + v.y * v.y;  // the grid stride is a multiple of b: one column per thread
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (threadIdx.x < b) {
      const double z2 = sc->bnorm2[threadIdx.x];
      if (z2 > 0.0 && tot[threadIdx.x].x > kDfCertRatio * kDfCertRatio * z2) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *fp64_cert = any;
  }
}

// True residual r = z - A x of the mixed solvers, with A x in double-float arithmetic on the
// split x (links split into FP32 hi + lo): each component carries an error of about 2^-46 times
// the sum of the stencil terms' magnitudes (~9 |x|), i.e. ~1e-13 ||x|| / ||z|| relative to z,
// a hundredth of a 1e-10 tolerance while ||x|| / ||z|| stays below ~10, on the FP32 pipe instead
// of the FP64 one (about a third of k_resid's time on this part).  tot = (||r||^2, ||z||^2).
__global__ void __launch_bounds__(kBlock, 2) k_resid_df(const cdf *__restrict__ Udf, const float2 *__restrict__ xhi,
                                                     const float2 *__restrict__ xlo, const double2 *__restrict__ z,
                                                     double2 *__restrict__ r, Geom g, int b, int logb, dff diag,
                                                     Scal *sc, Reduce red, int restart, const int *run_flag,
                                                     int run_if, int *mark, const int *fp64_cert) {
  __shared__ double2 tot[64];
  if (run_flag && *(volatile const int *)run_flag != run_if) return;  // not selected (uniform over the grid)
  if (*(volatile const int *)fp64_cert) return;                        // the FP64 residual runs instead
  double2 acc[1] = {make_double2(0.0, 0.0)};
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  const DfPairLoad ld{xhi, xlo};
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    const int64_t base = (int64_t)s * 12 * b + j;
    cdf o[12], self[12];
    dslash_site_ld<1, dff>(Udf, ld, g, b, s, j, diag, o, self);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 zz = z[base + c * b];
      const double2 rr = make_double2(zz.x - ((double)o[c].x.hi + (double)o[c].x.lo),
                                      zz.y - ((double)o[c].y.hi + (double)o[c].y.lo));
      r[base + c * b] = rr;
      acc[0].x += rr.x * rr.x + rr.y * rr.y;
      acc[0].y += zz.x * zz.x + zz.y * zz.y;
    }
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_resid(sc, threadIdx.x, tot[threadIdx.x], restart);
    __syncthreads();
    if (threadIdx.x == 0) {
      count_active(sc, b);
      if (mark) *mark = 0;
    }
  }
}

// The mixed solvers' true residual: split x into (xhi, xlo) (two n-element FP32 scratch fields,
// idle between inner solves) and measure ||x||, then r = z - A x in double-float arithmetic, or in
// FP64 where ||x|| / ||z|| is large (three launches, two of which run; gated like k_resid).
static void launch_true_resid_df(const dtr_gauge_s *gauge, const double2 *x, const double2 *z, double2 *r64,
                                 float2 *xhi, float2 *xlo, const Geom &g, int b, int logb, double m0, Scal *sc,
                                 const Reduce &red, int restart, const int *run_flag, int run_if, int *mark,
                                 int *fp64_cert, unsigned gd, unsigned gv, cudaStream_t st) {
  const int64_t n = (int64_t)g.V * 12 * b;
  k_split_df<<<gv, kBlock, 0, st>>>(x, xhi, xlo, n, b, sc, red, fp64_cert, run_flag, run_if);
  const float dh = (float)(4.0 + m0);
  k_resid_df<<<gd, kBlock, 0, st>>>((const cdf *)gauge->Udf, xhi, xlo, z, r64, g, b, logb,
                                    dff(dh, (float)((4.0 + m0) - (double)dh)), sc, red, restart, run_flag, run_if,
                                    mark, fp64_cert);
  k_resid<double, 0><<<gd, kBlock, 0, st>>>(gauge->U64, x, z, r64, nullptr, nullptr, g, b, logb, 4.0 + m0, sc, red,
                                            restart, run_flag, run_if, mark, fp64_cert);
}

// Whether cycles may end with the double-float residual update (r -= A e, cheaper than a
// true residual of x): k_mixed_accum then takes it for cycles predicted to stay well above
// tol and the true residual (k_resid_df) for the cycle predicted to converge, which also
// certifies the result, so a solve of c cycles runs c - 1 updates and one true residual.
// On unless DTR_RESID_UPDATE=0 (every cycle ends with the true residual).
static bool resid_update_enabled(int /*store*/) {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("DTR_RESID_UPDATE");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v != 0;
}

static dff split_df(double v) {
  const float h = (float)v;
  return dff(h, (float)(v - (double)h));
}

__global__ void __launch_bounds__(kBlock) k_dslash_df(const cdf *__restrict__ Udf, const float2 *__restrict__ in,
                                                      double2 *__restrict__ out, Geom g, int b, int logb, dff diag) {
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  const F32AsDf ld{in};
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    const int64_t base = (int64_t)s * 12 * b + j;
    cdf o[12], self[12];
    dslash_site_ld<1, dff>(Udf, ld, g, b, s, j, diag, o, self);
#pragma unroll
    for (int c = 0; c < 12; ++c)
      out[base + c * b] = make_double2((double)o[c].x.hi + (double)o[c].x.lo, (double)o[c].y.hi + (double)o[c].y.lo);
  }
}

void launch_dslash_df(const void *Udf, const float2 *in, double2 *out, const Geom &g, int b, double m0,
                      cudaStream_t st) {
  const int64_t n = (int64_t)g.V * b;
  int logb = 0;
  while ((1 << logb) < b) ++logb;
  k_dslash_df<<<reduce_grid(n, device_sms()), kBlock, 0, st>>>((const cdf *)Udf, in, out, g, b, logb,
                                                               split_df(4.0 + m0));
  count_launches(1);
}

// v = A p; sigma = rhat^H v -> alpha
template <typename R>
__global__ void __launch_bounds__(kBlock) k_dslash_alpha(const typename cplx_t<R>::type *__restrict__ U,
                                                         const typename cplx_t<R>::type *__restrict__ p,
                                                         const typename cplx_t<R>::type *__restrict__ rhat,
                                                         typename cplx_t<R>::type *__restrict__ v, Geom g, int b,
                                                         int logb, R diag, Scal *sc, Reduce red) {
  typedef typename cplx_t<R>::type C;
  __shared__ double2 tot[64];
  C a0 = mk<C>(0.0, 0.0);
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    C o[12], self[12];
    dslash_site<1, R>(U, p, g, b, s, j, diag, o, self);
    const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      v[base + c * b] = o[c];
      a0 = dot_acc(a0, rhat[base + c * b], o[c]);
    }
  }
  double2 acc[1] = {to_d2(a0)};
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_alpha(sc, threadIdx.x, tot[threadIdx.x]);
  }
}

// s = r - alpha v (in place in r)
template <typename R>
__global__ void __launch_bounds__(kBlock) k_supdate(typename cplx_t<R>::type *__restrict__ r,
                                                    const typename cplx_t<R>::type *__restrict__ v, int64_t n, int b,
                                                    const Scal *__restrict__ sc) {
  typedef typename cplx_t<R>::type C;
  const int j = threadIdx.x & (b - 1);
  const C a = scal_as<C>(sc->alpha[j]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    r[e] = caxpy(cneg(a), v[e], r[e]);
  }
}

// t = A s; (t^H s, t^H t) -> omega
template <typename R>
__global__ void __launch_bounds__(kBlock) k_dslash_omega(const typename cplx_t<R>::type *__restrict__ U,
                                                         const typename cplx_t<R>::type *__restrict__ sv,
                                                         typename cplx_t<R>::type *__restrict__ t, Geom g, int b,
                                                         int logb, R diag, Scal *sc, Reduce red) {
  typedef typename cplx_t<R>::type C;
  __shared__ double2 tot[128];
  C a0 = mk<C>(0.0, 0.0);
  R tt = 0;
  const int64_t n = (int64_t)g.V << logb;
  const int j = threadIdx.x & (b - 1);
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(it >> logb);
    C o[12], self[12];
    dslash_site<1, R>(U, sv, g, b, s, j, diag, o, self);
    const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      t[base + c * b] = o[c];
      a0 = dot_acc(a0, o[c], self[c]);
      tt += o[c].x * o[c].x + o[c].y * o[c].y;
    }
  }
  double2 acc[2] = {to_d2(a0), make_double2((double)tt, 0.0)};
  if (block_reduce<2>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_omega(sc, threadIdx.x, tot[threadIdx.x], tot[b + threadIdx.x]);
  }
}

// x += alpha p + omega s; r = s - omega t; (rhat^H r, r^H r) -> beta, convergence
template <typename R>
__global__ void __launch_bounds__(kBlock) k_xr_update(typename cplx_t<R>::type *__restrict__ x,
                                                      typename cplx_t<R>::type *__restrict__ r,
                                                      const typename cplx_t<R>::type *__restrict__ p,
                                                      const typename cplx_t<R>::type *__restrict__ t,
                                                      const typename cplx_t<R>::type *__restrict__ rhat, int64_t n,
                                                      int b, Scal *sc, Reduce red) {
  typedef typename cplx_t<R>::type C;
  __shared__ double2 tot[128];
  C a0 = mk<C>(0.0, 0.0);
  R rr = 0;
  const int j = threadIdx.x & (b - 1);
  const C a = scal_as<C>(sc->alpha[j]);
  const C w = scal_as<C>(sc->omega[j]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const C s = r[e];
    x[e] = caxpy(w, s, caxpy(a, p[e], x[e]));
    const C rn = caxpy(cneg(w), t[e], s);
    r[e] = rn;
    a0 = dot_acc(a0, rhat[e], rn);
    rr += rn.x * rn.x + rn.y * rn.y;
  }
  double2 acc[2] = {to_d2(a0), make_double2((double)rr, 0.0)};
  if (block_reduce<2>(acc, b, red.partial, red.counter, tot)) {
    if (threadIdx.x < b) fin_beta(sc, threadIdx.x, tot[threadIdx.x], tot[b + threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) count_active(sc, b);
  }
}

// p = r + beta (p - omega v) for active columns
template <typename R>
__global__ void __launch_bounds__(kBlock) k_pupdate(typename cplx_t<R>::type *__restrict__ p,
                                                    const typename cplx_t<R>::type *__restrict__ r,
                                                    const typename cplx_t<R>::type *__restrict__ v, int64_t n, int b,
                                                    const Scal *__restrict__ sc) {
  typedef typename cplx_t<R>::type C;
  const int j = threadIdx.x & (b - 1);
  if (!sc->active[j]) return;
  const C be = scal_as<C>(sc->beta[j]);
  const C w = scal_as<C>(sc->omega[j]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    p[e] = caxpy(be, caxpy(cneg(w), v[e], p[e]), r[e]);
  }
}

// mixed: r32 = hs * scale * r64 (scale = 1 / ||r64|| per column; hs = 1 for FP32
// storage, sqrt(12 V) for half storage, so that the entries are O(1) and stay in
// FP16's normal range), rhat = p = r32, e = 0 (inner columns = outer active).
// S: storage of the inner Krylov vectors; the inner iterate e is FP32.
template <typename S>
__global__ void __launch_bounds__(kBlock) k_mixed_init(const double2 *__restrict__ r64, S *__restrict__ r,
                                                       S *__restrict__ rhat, S *__restrict__ p,
                                                       float2 *__restrict__ e, int64_t n, int b,
                                                       const Scal *__restrict__ outer, double hs) {
  const int j = threadIdx.x & (b - 1);
  const double sc = outer->active[j] ? outer->scale[j] * hs : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = r64[i];
    const float2 f = make_float2((float)(v.x * sc), (float)(v.y * sc));
    CStore<S>::st(r, i, f);
    CStore<S>::st(rhat, i, f);
    CStore<S>::st(p, i, f);
    e[i] = make_float2(0.f, 0.f);
  }
}

__global__ void k_mixed_scal_init(const Scal *__restrict__ outer, Scal *inner, int b, double inner_tol2,
                                  int inner_maxiter, double hs2) {
  const int j = threadIdx.x;
  if (j < b) {
    const int act = outer->active[j];
    inner->active[j] = act;
    inner->rho[j] = make_double2(hs2, 0.0);  // rhat^H r0 = ||r32||^2 (rhat = r0 = r32)
    inner->bnorm2[j] = hs2;  // ||r32||^2 of a unit column scaled by hs
    inner->rnorm2[j] = hs2;
    inner->iters[j] = 0;
    inner->flags[j] = 0;
    inner->alpha[j] = inner->omega[j] = inner->beta[j] = make_double2(0.0, 0.0);
  }
  if (j == 0) {
    int n = 0;
    for (int q = 0; q < b; ++q) n += outer->active[q];
    inner->n_active = n;
    inner->tol2 = inner_tol2;
    inner->maxiter = inner_maxiter;
  }
}

// x64 += e / (hs * scale) for outer-active columns; fold inner iteration counts.
// With gs: choose the residual that ends this cycle (gs->sel): the double-float
// update if allowed and some active column is predicted (its last residual times the
// inner solve's achieved reduction) to stay more than 10x above tol, else the FP64
// residual, which then also certifies convergence.
__global__ void __launch_bounds__(kBlock) k_mixed_accum(double2 *__restrict__ x, const float2 *__restrict__ e,
                                                        int64_t n, int b, Scal *outer, const Scal *__restrict__ inner,
                                                        double hs, GridSync *gs, int allow_update) {
  if (gs && blockIdx.x == 0) {  // one column per thread of block 0
    const int q = threadIdx.x;
    int far = 0;
    if (q < b && outer->active[q]) {
      const double red2 = inner->bnorm2[q] > 0.0 ? inner->rnorm2[q] / inner->bnorm2[q] : 1.0;
      far = outer->rtrue2[q] * red2 > 100.0 * outer->tol2 * outer->bnorm2[q];
    }
    far = __syncthreads_or(far);
    if (q == 0) gs->sel = (allow_update && far) ? 1 : 0;
  }
  const int j = threadIdx.x & (b - 1);
  const int act = outer->active[j];
  const double inv = act ? 1.0 / (outer->scale[j] * hs) : 0.0;
  if (act) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const float2 v = e[i];
      double2 xv = x[i];
      xv.x = fma((double)v.x, inv, xv.x);
      xv.y = fma((double)v.y, inv, xv.y);
      x[i] = xv;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < b) {
    outer->iters[threadIdx.x] += inner->iters[threadIdx.x];
    outer->flags[threadIdx.x] |= inner->flags[threadIdx.x] & ~kFlagBreakdown;
  }
}

__global__ void k_scal_init(Scal *sc, int b, double tol2, int maxiter) {
  const int j = threadIdx.x;
  if (j < 64) {
    sc->active[j] = 0;
    sc->iters[j] = 0;
    sc->restarts[j] = 0;
    sc->conv[j] = 0;
    sc->flags[j] = 0;
    sc->rho[j] = sc->alpha[j] = sc->omega[j] = sc->beta[j] = make_double2(0.0, 0.0);
    sc->rnorm2[j] = sc->bnorm2[j] = sc->rtrue2[j] = 0.0;
    sc->scale[j] = 1.0;
  }
  if (j == 0) {
    sc->n_active = 0;
    sc->tol2 = tol2;
    sc->maxiter = maxiter;
  }
}

// ------------------------------------------------------------------ drivers
static int ilog2i(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

static int *pinned_flag() {
  static thread_local int *p = nullptr;
  if (!p) {
    if (cudaMallocHost((void **)&p, sizeof(int) * 4) != cudaSuccess) p = nullptr;
  }
  return p;
}

static int read_n_active(const Scal *sc, cudaStream_t st, int *out) {
  int *h = pinned_flag();
  if (!h) return fail(DTR_ECUDA, "cudaMallocHost for the convergence flag failed");
  DTR_CUDA(cudaMemcpyAsync(h, &sc->n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  *out = *h;
  return DTR_OK;
}

template <typename R>
static void launch_iteration(const typename cplx_t<R>::type *U, KrylovVecs<R> &K, const Geom &g, int b, double m0,
                             Scal *sc, Reduce red, cudaStream_t st) {
  const int sms = device_sms();
  const int logb = ilog2i(b);
  const int64_t sites_items = (int64_t)g.V * b;
  const int64_t n = sites_items * 12;
  const unsigned gd = reduce_grid(sites_items, sms);
  const unsigned gv = reduce_grid(n, sms);
  const R diag = (R)(4.0 + m0);
  k_dslash_alpha<R><<<gd, kBlock, 0, st>>>(U, K.p, K.rhat, K.v, g, b, logb, diag, sc, red); count_launches(1);
  k_supdate<R><<<gv, kBlock, 0, st>>>(K.r, K.v, n, b, sc); count_launches(1);
  k_dslash_omega<R><<<gd, kBlock, 0, st>>>(U, K.r, K.t, g, b, logb, diag, sc, red); count_launches(1);
  k_xr_update<R><<<gv, kBlock, 0, st>>>(K.x, K.r, K.p, K.t, K.rhat, n, b, sc, red); count_launches(1);
  k_pupdate<R><<<gv, kBlock, 0, st>>>(K.p, K.r, K.v, n, b, sc); count_launches(1);
}

template <typename R>
static int iterate(const typename cplx_t<R>::type *U, KrylovVecs<R> &K, const Geom &g, int b, double m0, Scal *sc,
                   Reduce red, int check_every, int max_total, cudaStream_t st) {
  int done = 0;
  while (done < max_total) {
    for (int c = 0; c < check_every; ++c) launch_iteration<R>(U, K, g, b, m0, sc, red, st);
    DTR_LAUNCH_CHECK("bicgstab iteration launch");
    done += check_every;
    int n_active = 0;
    int rc = read_n_active(sc, st, &n_active);
    if (rc) return rc;
    if (n_active == 0) break;
  }
  return DTR_OK;
}

static bool mixed_bicgstab(int solver) {
  return solver == DTR_SOLVER_MIXED_F32 || solver == DTR_SOLVER_MIXED_F16 || solver == DTR_SOLVER_MIXED_BF16;
}
// storage of the inner Krylov vectors: 0 FP32, 1 FP16, 2 BF16
static int inner_store(int solver) {
  return solver == DTR_SOLVER_MIXED_F16 ? 1 : solver == DTR_SOLVER_MIXED_BF16 ? 2 : 0;
}
// Relative residual reduction asked of one inner solve.  A recursion whose vectors are
// rounded to 11 (FP16) or 8 (BF16) significant bits stops paying beyond ~2e-4 or ~1e-2
// of reduction (measured: deeper requests cost more iterations than the defect-correction
// cycles they save; at 32^3x64 2e-4 is the loosest FP16 request that still reaches 1e-10
// in three cycles), so smaller requests are raised to that floor (the FP64 outer loop
// reaches the outer tolerance either way).
static double inner_tol_for(const dtr_solve_params *p) {
  double t = p->inner_tol > 0 ? p->inner_tol : 1e-5;
  const int store = inner_store(p->solver);
  const double floor = store == 1 ? kInnerTolFloorF16 : store == 2 ? kInnerTolFloorBF16 : 0.0;
  return t < floor ? floor : t;
}

size_t solver_scratch_bytes(int64_t V, int b, int solver, int gmres_m) {
  const size_t vec64 = ((size_t)V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  const size_t vec32 = ((size_t)V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  const size_t red = 256 + (size_t)kMaxGrid * 5 * 64 * sizeof(double2);
  const size_t scal = 2 * ((sizeof(Scal) + 255) / 256) * 256;
  const size_t fixed = 256 + red + scal + 256 + 256;
  if (mixed_bicgstab(solver)) return fixed + vec64 + 7 * vec32;  // half storage uses half of each slot
  if (solver == DTR_SOLVER_FGMRES_NET) return fixed + vec64 + 7 * vec32 + fgmres_scratch_bytes(V, b, gmres_m) + 256;
  return fixed + 6 * vec64;
}

static char *align256(char *p) { return (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255); }

static int read_gs_error(const GridSync *gs, cudaStream_t st) {
  int *h = pinned_flag();
  if (!h) return fail(DTR_ECUDA, "cudaMallocHost for the convergence flag failed");
  DTR_CUDA(cudaMemcpyAsync(h + 1, &gs->error, sizeof(int), cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  if (persist_profile().on) persist_profile_flush(st);
  if (h[1]) return fail(DTR_ETIMEOUT, "persistent solver barrier timed out");
  return DTR_OK;
}

// ------------------------------------------------ graph-driven mixed solve
// The whole defect-correction loop of the mixed solver as ONE CUDA graph: the
// first true residual, then a conditional WHILE node whose body is one cycle
// (FP32 inner init, persistent inner BiCGStab, FP64 accumulate, double-float
// update or true residual) and ends with k_loop_cond, which sets the loop condition from the
// number of columns still active.  No host round trip between cycles.

__global__ void k_loop_cond(cudaGraphConditionalHandle h, const Scal *__restrict__ outer, GridSync *gs,
                            unsigned int max_cycles, int first, unsigned long long *dev_launches,
                            unsigned int body_kernels) {
  if (threadIdx.x == 0) {
    if (first == 1) {
      gs->cycles = 0;
    } else if (first == 2) {
      // entry of the FP64-residual loop after the verification: cycles keep counting
    } else {
      gs->cycles += 1;
      if (dev_launches) atomicAdd(dev_launches, (unsigned long long)body_kernels);
    }
    const unsigned int go = (outer->n_active > 0 && gs->error == 0 && gs->cycles < max_cycles) ? 1u : 0u;
    cudaGraphSetConditional(h, go);
  }
}

namespace {

struct MixedState {
  const dtr_gauge_s *gauge;
  Geom g;
  int b, logb;
  double m0;
  double2 *x;
  const double2 *z;
  double2 *r64;
  KrylovVecs<float> K;
  float2 *sv;
  Scal *outer, *inner;
  Reduce red;
  GridSync *gs;
  unsigned gd, gv;
  double itol;
  int maxiter, grid;
  int store;  // inner Krylov vectors: 0 FP32, 1 FP16, 2 BF16
  double hs;  // inner right-hand-side scale (see k_mixed_init)
  int upd;    // cycles end with the double-float residual update (then one true-residual verification)
};

// inner iterations of one defect-correction cycle on the caller-initialised state
template <typename S>
static int launch_inner(const dtr_gauge_s *gauge, const KrylovVecs<float> &K, float2 *sv, const Geom &g, int b,
                        int logb, double m0, Scal *inner, const Reduce &red, GridSync *gs, int maxiter, int grid,
                        cudaStream_t st) {
  PArgs<float, S> pa;
  pa.U = gauge->U32;
  pa.x = K.x;
  pa.r = (S *)K.r; pa.rhat = (S *)K.rhat; pa.p = (S *)K.p; pa.v = (S *)K.v; pa.s = (S *)sv; pa.t = (S *)K.t;
  pa.z = nullptr;
  pa.g = g; pa.b = b; pa.logb = logb; pa.diag = (float)(4.0 + m0);
  pa.sc = inner; pa.partial = red.partial; pa.gs = gs;
  pa.max_iters = maxiter + 1;
  pa.max_cycles = 1;
  pa.grid = grid;
  if constexpr (std::is_same<S, float2>::value) return launch_persistent<float>(pa, 0, st);
  else return launch_persistent_half<S>(pa, st);
}

template <typename S>
static void launch_mixed_init(const double2 *r64, const KrylovVecs<float> &K, int64_t n, int b, const Scal *outer,
                              double hs, unsigned gv, cudaStream_t st) {
  k_mixed_init<S><<<gv, kBlock, 0, st>>>(r64, (S *)K.r, (S *)K.rhat, (S *)K.p, K.x, n, b, outer, hs);
}

static void mixed_init(int store, const double2 *r64, const KrylovVecs<float> &K, int64_t n, int b,
                       const Scal *outer, double hs, unsigned gv, cudaStream_t st) {
  if (store == 1) launch_mixed_init<__half2>(r64, K, n, b, outer, hs, gv, st);
  else if (store == 2) launch_mixed_init<__nv_bfloat162>(r64, K, n, b, outer, hs, gv, st);
  else launch_mixed_init<float2>(r64, K, n, b, outer, hs, gv, st);
  count_launches(1);
}

static int inner_solve(int store, const dtr_gauge_s *gauge, const KrylovVecs<float> &K, float2 *sv, const Geom &g,
                       int b, int logb, double m0, Scal *inner, const Reduce &red, GridSync *gs, int maxiter,
                       int grid, cudaStream_t st) {
  if (store == 1) return launch_inner<__half2>(gauge, K, sv, g, b, logb, m0, inner, red, gs, maxiter, grid, st);
  if (store == 2)
    return launch_inner<__nv_bfloat162>(gauge, K, sv, g, b, logb, m0, inner, red, gs, maxiter, grid, st);
  return launch_inner<float2>(gauge, K, sv, g, b, logb, m0, inner, red, gs, maxiter, grid, st);
}

// One defect-correction cycle after a residual: returns the kernels it launched.
int enqueue_inner(const MixedState &S, cudaStream_t st, int *kernels) {
  const int64_t n = (int64_t)S.g.V * 12 * S.b;
  mixed_init(S.store, S.r64, S.K, n, S.b, S.outer, S.hs, S.gv, st);
  k_mixed_scal_init<<<1, 64, 0, st>>>(S.outer, S.inner, S.b, S.itol * S.itol, S.maxiter, S.hs * S.hs);
  count_launches(1);
  DTR_LAUNCH_CHECK("inner init");
  DTR_CUDA(cudaMemsetAsync(S.gs, 0, kGridSyncLaunchBytes, st));
  int rc = inner_solve(S.store, S.gauge, S.K, S.sv, S.g, S.b, S.logb, S.m0, S.inner, S.red, S.gs, S.maxiter, S.grid,
                       st);
  if (rc) return rc;
  *kernels = 3 + (persist_profile().on ? 1 : 0);
  return DTR_OK;
}

struct GraphKey {
  int device;
  const void *U64, *U32;
  int L[4];
  double m0;
  const void *x, *z, *work;
  int b, x_is_zero, maxiter, grid, prof, store, upd, pad2;
  double tol, itol;
};

struct GraphEntry {
  GraphKey key;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  unsigned long long last_use;
};

std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
unsigned long long g_graph_tick = 0;
unsigned long long g_graph_captures = 0, g_graph_launches = 0;
constexpr size_t kMaxGraphs = 8;

struct CaptureStreams {
  cudaStream_t a = nullptr, b = nullptr;
};
thread_local CaptureStreams t_cap;

int capture_streams(cudaStream_t *a, cudaStream_t *b) {
  if (!t_cap.a) DTR_CUDA(cudaStreamCreateWithFlags(&t_cap.a, cudaStreamNonBlocking));
  if (!t_cap.b) DTR_CUDA(cudaStreamCreateWithFlags(&t_cap.b, cudaStreamNonBlocking));
  *a = t_cap.a;
  *b = t_cap.b;
  return DTR_OK;
}

// Record the graph; on any failure the capture is ended and nothing is kept.
int capture_mixed_graph(const MixedState &S, int x_is_zero, double tol2, int maxiter, cudaGraph_t *out) {
  cudaStream_t cs, cs2;
  int rc = capture_streams(&cs, &cs2);
  if (rc) return rc;
  cudaGraph_t graph = nullptr;
  DTR_CUDA(cudaGraphCreate(&graph, 0));
  capture_begin();
  int open = 0;  // captures in progress: 1 = cs, 2 = cs and cs2
  auto bail = [&](int code) {
    cudaGraph_t tmp = nullptr;
    if (open >= 2) cudaStreamEndCapture(cs2, &tmp);
    if (open >= 1) cudaStreamEndCapture(cs, &tmp);
    cudaGetLastError();
    cudaGraphDestroy(graph);
    capture_end();
    return code;
  };
#define CAP_CHECK(call)                                                        \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, "graph capture: " #call)); \
  } while (0)
  cudaGraphConditionalHandle h;
  CAP_CHECK(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
  CAP_CHECK(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  open = 1;
  const int64_t n = (int64_t)S.g.V * 12 * S.b;
  k_scal_init<<<1, 64, 0, cs>>>(S.outer, S.b, tol2, maxiter);
  if (x_is_zero)
    k_resid_zero<<<S.gv, kBlock, 0, cs>>>(S.z, S.r64, n, S.b, S.outer, S.red);
  else
    launch_true_resid_df(S.gauge, S.x, S.z, S.r64, S.K.v, S.K.t, S.g, S.b, S.logb, S.m0, S.outer, S.red, 1, nullptr,
                         0, &S.gs->last_upd, &S.gs->fp64_cert, S.gd, S.gv, cs);
  unsigned long long *devcnt = device_launch_counter();
  k_loop_cond<<<1, 32, 0, cs>>>(h, S.outer, S.gs, (unsigned)kMaxRestarts + 1, 1, devcnt, 0);
  CAP_CHECK(cudaGetLastError());
  cudaStreamCaptureStatus stc;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  CAP_CHECK(cudaStreamGetCaptureInfo(cs, &stc, nullptr, &capg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CAP_CHECK(cudaGraphAddNode(&cnode, capg, deps, nullptr, nd, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CAP_CHECK(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CAP_CHECK(cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  open = 2;
  int kin = 0;
  rc = enqueue_inner(S, cs2, &kin);
  if (rc) return bail(rc);
  k_mixed_accum<<<S.gv, kBlock, 0, cs2>>>(S.x, S.K.x, n, S.b, S.outer, S.inner, S.hs, S.gs, S.upd);
  if (S.upd)  // one of the two runs, as k_mixed_accum chose
    k_resid_update<<<S.gd, kBlock, 0, cs2>>>((const cdf *)S.gauge->Udf, S.K.x, S.r64, S.g, S.b, S.logb,
                                             split_df(4.0 + S.m0), S.hs, S.outer, S.red, &S.gs->sel, 1,
                                             &S.gs->last_upd);
  launch_true_resid_df(S.gauge, S.x, S.z, S.r64, S.K.v, S.K.t, S.g, S.b, S.logb, S.m0, S.outer, S.red, 1,
                       S.upd ? &S.gs->sel : nullptr, 0, &S.gs->last_upd, &S.gs->fp64_cert, S.gd, S.gv, cs2);
  k_loop_cond<<<1, 32, 0, cs2>>>(h, S.outer, S.gs, (unsigned)kMaxRestarts + 1, 0, devcnt,
                                 (unsigned)(kin + (S.upd ? 6 : 5)));
  CAP_CHECK(cudaGetLastError());
  cudaGraph_t tmp = nullptr;
  CAP_CHECK(cudaStreamEndCapture(cs2, &tmp));
  open = 1;
  if (S.upd) {
    // verification (when the loop ended on a double-float update): the true residual
    // of x decides; columns it finds short of tol continue in a second loop whose
    // cycles end with the true residual
    launch_true_resid_df(S.gauge, S.x, S.z, S.r64, S.K.v, S.K.t, S.g, S.b, S.logb, S.m0, S.outer, S.red, 1,
                         &S.gs->last_upd, 1, &S.gs->last_upd, &S.gs->fp64_cert, S.gd, S.gv, cs);
    cudaGraphConditionalHandle h2;
    CAP_CHECK(cudaGraphConditionalHandleCreate(&h2, graph, 0, 0));
    k_loop_cond<<<1, 32, 0, cs>>>(h2, S.outer, S.gs, (unsigned)kMaxRestarts + 1, 2, devcnt, 0);
    CAP_CHECK(cudaGetLastError());
    CAP_CHECK(cudaStreamGetCaptureInfo(cs, &stc, nullptr, &capg, &deps, nullptr, &nd));
    cudaGraphNodeParams cp2 = {cudaGraphNodeTypeConditional};
    cp2.conditional.handle = h2;
    cp2.conditional.type = cudaGraphCondTypeWhile;
    cp2.conditional.size = 1;
    cudaGraphNode_t cnode2;
    CAP_CHECK(cudaGraphAddNode(&cnode2, capg, deps, nullptr, nd, &cp2));
    cudaGraph_t body2 = cp2.conditional.phGraph_out[0];
    CAP_CHECK(cudaStreamUpdateCaptureDependencies(cs, &cnode2, nullptr, 1, cudaStreamSetCaptureDependencies));
    CAP_CHECK(cudaStreamBeginCaptureToGraph(cs2, body2, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    open = 2;
    rc = enqueue_inner(S, cs2, &kin);
    if (rc) return bail(rc);
    k_mixed_accum<<<S.gv, kBlock, 0, cs2>>>(S.x, S.K.x, n, S.b, S.outer, S.inner, S.hs, nullptr, 0);
    launch_true_resid_df(S.gauge, S.x, S.z, S.r64, S.K.v, S.K.t, S.g, S.b, S.logb, S.m0, S.outer, S.red, 1, nullptr,
                         0, &S.gs->last_upd, &S.gs->fp64_cert, S.gd, S.gv, cs2);
    k_loop_cond<<<1, 32, 0, cs2>>>(h2, S.outer, S.gs, (unsigned)kMaxRestarts + 1, 0, devcnt, (unsigned)(kin + 5));
    CAP_CHECK(cudaGetLastError());
    CAP_CHECK(cudaStreamEndCapture(cs2, &tmp));
    open = 1;
  }
  CAP_CHECK(cudaStreamEndCapture(cs, &tmp));
  open = 0;
#undef CAP_CHECK
  capture_end();
  *out = graph;
  return DTR_OK;
}

}  // namespace

int graph_counters(unsigned long long *captures, unsigned long long *launches) {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  *captures = g_graph_captures;
  *launches = g_graph_launches;
  return DTR_OK;
}

void graphs_release() {
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (auto &e : g_graphs) {
    cudaGraphExecDestroy(e.exec);
    cudaGraphDestroy(e.graph);
  }
  g_graphs.clear();
}

static int solve_mixed_graph(const MixedState &S, int x_is_zero, double tol2, int maxiter, const void *work,
                             cudaStream_t st) {
  GraphKey key;
  memset(&key, 0, sizeof(key));
  DTR_CUDA(cudaGetDevice(&key.device));
  key.U64 = S.gauge->U64;
  key.U32 = S.gauge->U32;
  for (int i = 0; i < 4; ++i) key.L[i] = S.g.L[i];
  key.m0 = S.m0;
  key.x = S.x;
  key.z = S.z;
  key.work = work;
  key.b = S.b;
  key.x_is_zero = x_is_zero;
  key.maxiter = maxiter;
  key.grid = S.grid;
  key.prof = persist_profile().on ? 1 : 0;
  key.tol = tol2;
  key.itol = S.itol;
  key.store = S.store;
  key.upd = S.upd;
  std::lock_guard<std::mutex> lock(g_graph_mu);
  GraphEntry *hit = nullptr;
  for (auto &e : g_graphs)
    if (!memcmp(&e.key, &key, sizeof(key))) hit = &e;
  if (!hit) {
    if (g_graphs.size() >= kMaxGraphs) {
      size_t lru = 0;
      for (size_t i = 1; i < g_graphs.size(); ++i)
        if (g_graphs[i].last_use < g_graphs[lru].last_use) lru = i;
      cudaGraphExecDestroy(g_graphs[lru].exec);
      cudaGraphDestroy(g_graphs[lru].graph);
      g_graphs.erase(g_graphs.begin() + lru);
    }
    GraphEntry e;
    e.key = key;
    int rc = capture_mixed_graph(S, x_is_zero, tol2, maxiter, &e.graph);
    if (rc) return rc;
    cudaError_t ce = cudaGraphInstantiate(&e.exec, e.graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(e.graph);
      return cuda_fail(ce, "graph instantiate");
    }
    ++g_graph_captures;
    g_graphs.push_back(e);
    hit = &g_graphs.back();
  }
  hit->last_use = ++g_graph_tick;
  DTR_CUDA(cudaGraphLaunch(hit->exec, st));
  // k_scal_init, first residual (one kernel for x = 0, else split + two residual kernels),
  // k_loop_cond (+ verification: split + two residual kernels, and its k_loop_cond); the
  // loop bodies count themselves on the device
  count_launches(3 + (x_is_zero ? 0 : 2) + (S.upd ? 4 : 0));
  ++g_graph_launches;
  return DTR_OK;
}

bool solve_can_run_async(const dtr_solve_params *p) {
  if (p->engine != 0) return false;
  return p->solver == DTR_SOLVER_BICGSTAB_F64 || (mixed_bicgstab(p->solver) && !p->no_graph);
}

int *solver_error_word(void *work) {
  char *w = align256((char *)work);
  w = align256(w + 256);
  w = align256(w + (size_t)kMaxGrid * 5 * 64 * sizeof(double2));
  w = align256(w + sizeof(Scal));
  w = align256(w + sizeof(Scal));
  return &((GridSync *)w)->error;
}

// x (internal FP64, initial guess in / solution out), z (internal FP64)
int solve_internal(const dtr_gauge_s *gauge, double m0, double2 *x, const double2 *z, int b,
                   const dtr_solve_params *p, void *work, size_t work_bytes, cudaStream_t st, Scal **scal_out,
                   int x_is_zero, int async) {
  const Geom g = geom_of(gauge->lat);
  const int64_t n = (int64_t)g.V * 12 * b;
  if (work_bytes < solver_scratch_bytes(g.V, b, p->solver, p->gmres_m))
    return fail(DTR_ENOMEM, "solver workspace too small");
  char *w = align256((char *)work);
  Reduce red;
  red.counter = (unsigned int *)w;
  w = align256(w + 256);
  red.partial = (double2 *)w;
  w = align256(w + (size_t)kMaxGrid * 5 * 64 * sizeof(double2));
  Scal *outer = (Scal *)w;
  w = align256(w + sizeof(Scal));
  Scal *inner = (Scal *)w;
  w = align256(w + sizeof(Scal));
  GridSync *gs = (GridSync *)w;
  w = align256(w + sizeof(GridSync));
  DTR_CUDA(cudaMemsetAsync(red.counter, 0, 256, st));
  DTR_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), st));  // error word read at exit even without a launch
  const int sms = device_sms();
  const int logb = ilog2i(b);
  const unsigned gd = reduce_grid((int64_t)g.V * b, sms);
  const unsigned gv = reduce_grid(n, sms);
  const int check = p->check_every > 0 ? p->check_every : 8;
  const bool persistent = p->engine == 0;
  const int store = inner_store(p->solver);
  const double hs = store ? std::sqrt(12.0 * (double)g.V) : 1.0;
  const double itol = inner_tol_for(p);
  if (store && !persistent) return fail(DTR_EINVAL, "half-storage inner solves need the persistent engine");
  if (mixed_bicgstab(p->solver) && persistent && !p->no_graph) {
    MixedState S;
    S.gauge = gauge; S.g = g; S.b = b; S.logb = logb; S.m0 = m0; S.x = x; S.z = z;
    S.r64 = (double2 *)w; w = align256(w + n * sizeof(double2));
    S.K.x = (float2 *)w;    w = align256(w + n * sizeof(float2));
    S.K.r = (float2 *)w;    w = align256(w + n * sizeof(float2));
    S.K.rhat = (float2 *)w; w = align256(w + n * sizeof(float2));
    S.K.p = (float2 *)w;    w = align256(w + n * sizeof(float2));
    S.K.v = (float2 *)w;    w = align256(w + n * sizeof(float2));
    S.K.t = (float2 *)w;    w = align256(w + n * sizeof(float2));
    S.sv = (float2 *)w;     w = align256(w + n * sizeof(float2));
    S.outer = outer; S.inner = inner; S.red = red; S.gs = gs; S.gd = gd; S.gv = gv;
    S.itol = itol;
    S.maxiter = p->maxiter;
    S.grid = p->grid;
    S.store = store;
    S.hs = hs;
    S.upd = resid_update_enabled(store) ? 1 : 0;
    *scal_out = outer;
    int rc = solve_mixed_graph(S, x_is_zero, p->tol * p->tol, p->maxiter, work, st);
    if (rc) return rc;
    return async ? DTR_OK : read_gs_error(gs, st);
  }
  k_scal_init<<<1, 64, 0, st>>>(outer, b, p->tol * p->tol, p->maxiter); count_launches(1);
  DTR_LAUNCH_CHECK("scalar init");
  *scal_out = outer;

  if (p->solver == DTR_SOLVER_BICGSTAB_F64) {
    KrylovVecs<double> K;
    K.x = x;
    K.r = (double2 *)w;    w = align256(w + n * sizeof(double2));
    K.rhat = (double2 *)w; w = align256(w + n * sizeof(double2));
    K.p = (double2 *)w;    w = align256(w + n * sizeof(double2));
    K.v = (double2 *)w;    w = align256(w + n * sizeof(double2));
    K.t = (double2 *)w;    w = align256(w + n * sizeof(double2));
    double2 *sv = (double2 *)w; w = align256(w + n * sizeof(double2));
    if (persistent) {
      DTR_CUDA(cudaMemsetAsync(gs, 0, kGridSyncLaunchBytes, st));
      PArgs<double> pa;
      pa.U = gauge->U64;
      pa.x = x; pa.r = K.r; pa.rhat = K.rhat; pa.p = K.p; pa.v = K.v; pa.s = sv; pa.t = K.t; pa.z = z;
      pa.g = g; pa.b = b; pa.logb = logb; pa.diag = 4.0 + m0;
      pa.sc = outer; pa.partial = red.partial; pa.gs = gs;
      pa.max_iters = p->maxiter + 1;
      pa.max_cycles = kMaxRestarts + 2;
      pa.grid = p->grid;
      int rc = launch_persistent<double>(pa, 1, st);
      if (rc) return rc;
      return async ? DTR_OK : read_gs_error(gs, st);
    }
    for (int cycle = 0; cycle <= kMaxRestarts; ++cycle) {
      k_resid<double, 1><<<gd, kBlock, 0, st>>>(gauge->U64, x, z, K.r, K.rhat, K.p, g, b, logb, 4.0 + m0, outer, red,
                                                 cycle < kMaxRestarts, nullptr, 0, nullptr); count_launches(1);
      DTR_LAUNCH_CHECK("residual");
      int n_active = 0;
      int rc = read_n_active(outer, st, &n_active);
      if (rc) return rc;
      if (n_active == 0) break;
      rc = iterate<double>(gauge->U64, K, g, b, m0, outer, red, check, p->maxiter + check, st);
      if (rc) return rc;
    }
    return DTR_OK;
  }
  if (mixed_bicgstab(p->solver) || p->solver == DTR_SOLVER_FGMRES_NET) {
    double2 *r64 = (double2 *)w; w = align256(w + n * sizeof(double2));
    KrylovVecs<float> K;
    K.x = (float2 *)w;    w = align256(w + n * sizeof(float2));
    K.r = (float2 *)w;    w = align256(w + n * sizeof(float2));
    K.rhat = (float2 *)w; w = align256(w + n * sizeof(float2));
    K.p = (float2 *)w;    w = align256(w + n * sizeof(float2));
    K.v = (float2 *)w;    w = align256(w + n * sizeof(float2));
    K.t = (float2 *)w;    w = align256(w + n * sizeof(float2));
    float2 *sv = (float2 *)w; w = align256(w + n * sizeof(float2));
    void *fg_work = w;
    const size_t fg_bytes = p->solver == DTR_SOLVER_FGMRES_NET ? fgmres_scratch_bytes(g.V, b, p->gmres_m) : 0;
    bool fgmres = p->solver == DTR_SOLVER_FGMRES_NET;
    std::vector<double> prev_rel(64, -1.0);
    // phase 1: each cycle ends with the residual k_mixed_accum chose (the double-float
    // update or the true residual; the other kernel exits at entry); when no column is
    // left active, a true residual verifies unless the last one already was one;
    // phase 2: any further cycles end with the true residual (the same kernel
    // sequence as the graph-driven loop)
    bool upd_phase = resid_update_enabled(store);
    for (int cycle = 0; cycle <= kMaxRestarts; ++cycle) {
      const int restart = cycle < kMaxRestarts;
      if (cycle == 0 && x_is_zero) {
        k_resid_zero<<<gv, kBlock, 0, st>>>(z, r64, n, b, outer, red);
        count_launches(1);
      } else if (cycle > 0 && upd_phase) {
        k_resid_update<<<gd, kBlock, 0, st>>>((const cdf *)gauge->Udf, K.x, r64, g, b, logb, split_df(4.0 + m0), hs,
                                              outer, red, &gs->sel, 1, &gs->last_upd);
        launch_true_resid_df(gauge, x, z, r64, K.v, K.t, g, b, logb, m0, outer, red, restart, &gs->sel, 0,
                             &gs->last_upd, &gs->fp64_cert, gd, gv, st);
        count_launches(4);
      } else {
        launch_true_resid_df(gauge, x, z, r64, K.v, K.t, g, b, logb, m0, outer, red, restart, nullptr, 0,
                             &gs->last_upd, &gs->fp64_cert, gd, gv, st);
        count_launches(3);
      }
      DTR_LAUNCH_CHECK("outer residual");
      int n_active = 0;
      int rc = read_n_active(outer, st, &n_active);
      if (rc) return rc;
      if (n_active == 0 && cycle > 0 && upd_phase) {  // verify if the last residual was the update
        launch_true_resid_df(gauge, x, z, r64, K.v, K.t, g, b, logb, m0, outer, red, restart, &gs->last_upd, 1,
                             &gs->last_upd, &gs->fp64_cert, gd, gv, st);
        count_launches(3);
        DTR_LAUNCH_CHECK("verification residual");
        upd_phase = false;
        rc = read_n_active(outer, st, &n_active);
        if (rc) return rc;
      }
      if (n_active == 0) break;
      mixed_init(store, r64, K, n, b, outer, hs, gv, st);
      k_mixed_scal_init<<<1, 64, 0, st>>>(outer, inner, b, itol * itol, p->maxiter, hs * hs); count_launches(1);
      DTR_LAUNCH_CHECK("inner init");
      if (fgmres) {
        // fall back to the BiCGStab inner solve if the last FGMRES cycle cut the true residual < 10x
        Scal h;
        DTR_CUDA(cudaMemcpyAsync(&h, outer, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        DTR_CUDA(cudaStreamSynchronize(st));
        bool stagnated = false;
        for (int j = 0; j < b; ++j) {
          if (!h.active[j]) continue;
          const double rel = h.bnorm2[j] > 0 ? std::sqrt(h.rtrue2[j] / h.bnorm2[j]) : 0.0;
          if (prev_rel[j] > 0 && rel > 0.1 * prev_rel[j]) stagnated = true;
          prev_rel[j] = rel;
        }
        if (stagnated) fgmres = false;
      }
      if (fgmres) {
        Scal h;
        DTR_CUDA(cudaMemcpyAsync(&h, outer, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        DTR_CUDA(cudaStreamSynchronize(st));
        std::vector<int> act(b), its(b, 0);
        for (int j = 0; j < b; ++j) act[j] = h.active[j];
        rc = fgmres_solve(gauge, m0, (const dtr_net_s *)p->net, K.r, K.x, b, act.data(), p->gmres_m, itol, p->maxiter,
                          fg_work, fg_bytes, its.data(), st);
        if (rc) return rc;
        DTR_CUDA(cudaMemcpyAsync(inner->iters, its.data(), sizeof(int) * b, cudaMemcpyHostToDevice, st));
      } else if (persistent) {
        DTR_CUDA(cudaMemsetAsync(gs, 0, kGridSyncLaunchBytes, st));
        rc = inner_solve(store, gauge, K, sv, g, b, logb, m0, inner, red, gs, p->maxiter, p->grid, st);
        if (rc) return rc;
      } else {
        rc = iterate<float>(gauge->U32, K, g, b, m0, inner, red, check, p->maxiter + check, st);
        if (rc) return rc;
      }
      k_mixed_accum<<<gv, kBlock, 0, st>>>(x, K.x, n, b, outer, inner, hs, upd_phase ? gs : nullptr, upd_phase ? 1 : 0);
      count_launches(1);
      DTR_LAUNCH_CHECK("defect accumulate");
    }
    if (persistent) return read_gs_error(gs, st);
    return DTR_OK;
  }
  return fail(DTR_EINVAL, "unknown solver");
}

}  // namespace dtr
