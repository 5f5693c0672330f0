// Double-float ("df") arithmetic on the FP32 pipe: a value is hi + lo with two
// FP32 numbers, carried through exact products (Dekker/Veltkamp via FMA: the
// rounding error of a*b is fma(a, b, -a*b)) and exact sums (Knuth's TwoSum).
// About 2^-46 relative accuracy per operation, at roughly ten FP32
// instructions per operation (five for complex operations, whose real and
// imaginary parts run in the two lanes of packed FP32x2 instructions): on
// GB300, where an FP64 instruction costs about sixty FP32 ones, this is the
// cheaper way to get near-FP64 accuracy for a stencil whose inputs are FP32
// (the inner solver's iterate) and whose links are split once into hi + lo.
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
// Complex operations with the real and imaginary parts in the two lanes of packed FP32x2
// instructions: every lane performs exactly the scalar operations above (same operands, same
// order, round to nearest), so the results are bit-identical to the scalar forms, in about half
// the instructions.
struct dff2 {
  float2 hi, lo;  // lane 0: real part, lane 1: imaginary part
};
__device__ __forceinline__ float2 f2neg(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ dff2 to2(cdf a) { return dff2{make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo)}; }
__device__ __forceinline__ cdf from2(dff2 a) { return mkc2(dff(a.hi.x, a.lo.x), dff(a.hi.y, a.lo.y)); }
// lane-wise df sum (TwoSum on hi, then lo)
__device__ __forceinline__ dff2 add2(dff2 a, dff2 b) {
  const float2 s = __fadd2_rn(a.hi, b.hi);
  const float2 bb = __fadd2_rn(s, f2neg(a.hi));
  const float2 e = __fadd2_rn(__fadd2_rn(a.hi, f2neg(__fadd2_rn(s, f2neg(bb)))), __fadd2_rn(b.hi, f2neg(bb)));
  return dff2{s, __fadd2_rn(__fadd2_rn(a.lo, b.lo), e)};
}
// the scalar df a times each lane of b
__device__ __forceinline__ dff2 mul_b(dff a, dff2 b) {
  const float2 ah = make_float2(a.hi, a.hi), al = make_float2(a.lo, a.lo);
  const float2 p = __fmul2_rn(ah, b.hi);
  const float2 e = __ffma2_rn(ah, b.hi, f2neg(p));
  return dff2{p, __ffma2_rn(ah, b.lo, __ffma2_rn(al, b.hi, e))};
}
__device__ __forceinline__ dff2 swap2(dff2 a) {
  return dff2{make_float2(a.hi.y, a.hi.x), make_float2(a.lo.y, a.lo.x)};
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return from2(add2(to2(a), to2(b))); }
__device__ __forceinline__ cdf cneg(cdf a) { return mkc2(-a.x, -a.y); }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cadd(a, cneg(b)); }
__device__ __forceinline__ cdf cmuli(cdf a) { return mkc2(-a.y, a.x); }
// (a.x b.x - a.y b.y, a.x b.y + a.y b.x)
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  const dff2 bb = to2(b);
  const dff2 p = mul_b(a.x, bb), q = mul_b(a.y, swap2(bb));
  return from2(add2(p, dff2{make_float2(-q.hi.x, q.hi.y), make_float2(-q.lo.x, q.lo.y)}));
}
// conj(a) * b = (a.x b.x + a.y b.y, a.x b.y - a.y b.x)
__device__ __forceinline__ cdf cjmul(cdf a, cdf b) {
  const dff2 bb = to2(b);
  const dff2 p = mul_b(a.x, bb), q = mul_b(a.y, swap2(bb));
  return from2(add2(p, dff2{make_float2(q.hi.x, -q.hi.y), make_float2(q.lo.x, -q.lo.y)}));
}
// a + s*b
__device__ __forceinline__ cdf caxpy(cdf s, cdf b, cdf a) { return cadd(a, cmul(s, b)); }

// FP64 field value held as double-float hi + lo arrays (written by k_split_df)
struct DfPairLoad {
  const float2 *__restrict__ hi;
  const float2 *__restrict__ lo;
  __device__ __forceinline__ cdf operator()(int64_t idx) const {
    const float2 h = hi[idx], l = lo[idx];
    return mkc2(dff(h.x, l.x), dff(h.y, l.y));
  }
};

// FP32 field value as a df complex (exact)
struct F32AsDf {
  const float2 *__restrict__ f;
  __device__ __forceinline__ cdf operator()(int64_t idx) const {
    const float2 v = f[idx];
    return mkc2(dff(v.x), dff(v.y));
  }
};

}  // namespace dtr
