// Double-float ("df") arithmetic on the FP32 pipe: a value is hi + lo with two
// FP32 numbers, carried through exact products (Dekker/Veltkamp via FMA: the
// rounding error of a*b is fma(a, b, -a*b)) and exact sums (Knuth's TwoSum).
// About 2^-46 relative accuracy per operation, at roughly ten FP32
// instructions per operation: on GB300, where an FP64 instruction costs about
// sixty FP32 ones, this is the cheaper way to get near-FP64 accuracy for a
// stencil whose inputs are FP32 (the inner solver's iterate) and whose links
// are split once into hi + lo.
//
// The lo parts are not renormalised after every operation: each one holds a
// sum of rounding errors (and of the small cross terms), so it stays a few
// ulps of hi across the ~10^2 operations of one stencil evaluation.
// Explicitly rounded intrinsics keep the compiler from fusing or reordering
// the error-free transformations.
#pragma once

#include "dtr_internal.cuh"

namespace dtr {

struct dff {
  float hi, lo;
  __host__ __device__ dff() : hi(0.f), lo(0.f) {}
  __host__ __device__ dff(float h) : hi(h), lo(0.f) {}
  __host__ __device__ dff(float h, float l) : hi(h), lo(l) {}
};

// exact: s + e = a + b
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dff operator+(dff a, dff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dff(s, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}
__device__ __forceinline__ dff operator-(dff a) { return dff(-a.hi, -a.lo); }
__device__ __forceinline__ dff operator-(dff a, dff b) { return a + (-b); }
__device__ __forceinline__ dff operator*(dff a, dff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);  // exact rounding error of a.hi * b.hi
  return dff(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}

struct __align__(16) cdf {
  dff x, y;  // memory: Re hi, Re lo, Im hi, Im lo
};
template <> struct cplx_t<dff> { typedef cdf type; };

template <> __host__ __device__ __forceinline__ cdf mk<cdf>(double re, double im) {
  // only ever called with exact FP32 constants (zero); no FP64 work at run time
  cdf c;
  c.x = dff((float)re);
  c.y = dff((float)im);
  return c;
}
__device__ __forceinline__ cdf mkc2(dff re, dff im) {
  cdf c;
  c.x = re;
  c.y = im;
  return c;
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return mkc2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return mkc2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cdf cneg(cdf a) { return mkc2(-a.x, -a.y); }
__device__ __forceinline__ cdf cmuli(cdf a) { return mkc2(-a.y, a.x); }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) { return mkc2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__device__ __forceinline__ cdf cjmul(cdf a, cdf b) { return mkc2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
// a + s*b
__device__ __forceinline__ cdf caxpy(cdf s, cdf b, cdf a) { return cadd(a, cmul(s, b)); }

// FP32 field value as a df complex (exact)
struct F32AsDf {
  const float2 *__restrict__ f;
  __device__ __forceinline__ cdf operator()(int64_t idx) const {
    const float2 v = f[idx];
    return mkc2(dff(v.x), dff(v.y));
  }
};

}  // namespace dtr
