// Per-(site, right-hand side) Wilson-Dirac stencil on the RHS-inner layout.
//
//   (A psi)(x) = (4 + m0) psi(x)
//     - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^H psi(x-mu) ]
//
// Chiral basis: g_mu = [[0, B_mu], [B_mu^H, 0]] in 2x2 spin blocks with
// B_x = -i s_1, B_y = -i s_2, B_z = -i s_3, B_t = 1 (s_k Pauli), all unitary.
// Writing psi = (u; l) (upper / lower spin pair) one has
//   (1 - g) psi = (h; -B^H h),  h  = u - B l
//   (1 + g) psi = (h'; B^H h'), h' = u + B l
// so each hop needs one 2-spin "half spinor", two SU(3) x colour-vector
// products and a spin reconstruction; B and B^H only permute components and
// multiply by +-1 or +-i.  Summing the eight hops:
//   out_u = (4+m0) u - 1/2 sum_mu (w_f + w_b)
//   out_l = (4+m0) l + 1/2 sum_mu B_mu^H (w_f - w_b)
// with w_f = U_mu(x) h_f, w_b = U_mu(x-mu)^H h'_b.
// A^H = g5 A g5 (g5 = diag(1,1,-1,-1)) is the same stencil with the sign of
// every lower-spin term flipped on input and output (sgn = -1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dtr_internal.cuh"

namespace dtr {

// Field loaders: value of the input field at internal index (site*12 + c)*b + j.
template <typename C> struct PlainLoad {
  const C *__restrict__ f;
  __device__ __forceinline__ C operator()(int64_t idx) const { return f[idx]; }
};
// s = r - a v evaluated on the fly (a is this thread's column scalar)
template <typename C> struct AxpyLoad {
  const C *__restrict__ r;
  const C *__restrict__ v;
  C a;
  __device__ __forceinline__ C operator()(int64_t idx) const { return caxpy(cneg(a), v[idx], r[idx]); }
};

// Complex values stored as S, computed as float2/double2: loads widen, stores round to nearest.
template <typename S> struct CStore {
  __device__ __forceinline__ static S ld(const S *p, int64_t i) { return p[i]; }
  __device__ __forceinline__ static void st(S *p, int64_t i, S v) { p[i] = v; }
};
template <> struct CStore<__half2> {
  __device__ __forceinline__ static float2 ld(const __half2 *p, int64_t i) { return __half22float2(p[i]); }
  __device__ __forceinline__ static void st(__half2 *p, int64_t i, float2 v) { p[i] = __float22half2_rn(v); }
};
template <> struct CStore<__nv_bfloat162> {
  __device__ __forceinline__ static float2 ld(const __nv_bfloat162 *p, int64_t i) {
    return __bfloat1622float2(p[i]);
  }
  __device__ __forceinline__ static void st(__nv_bfloat162 *p, int64_t i, float2 v) {
    p[i] = __float22bfloat162_rn(v);
  }
};
template <typename S, typename C> struct PlainLoadS {
  const S *__restrict__ f;
  __device__ __forceinline__ C operator()(int64_t idx) const { return CStore<S>::ld(f, idx); }
};
template <typename S, typename C> struct AxpyLoadS {
  const S *__restrict__ r;
  const S *__restrict__ v;
  C a;
  __device__ __forceinline__ C operator()(int64_t idx) const {
    return caxpy(cneg(a), CStore<S>::ld(v, idx), CStore<S>::ld(r, idx));
  }
};

// B_mu applied to a 2-spin vector l (component-wise over colour)
template <int MU, typename C> __device__ __forceinline__ C applyB(const C &l0, const C &l1, int row) {
  if (MU == 0) return row == 0 ? cneg(cmuli(l1)) : cneg(cmuli(l0));  // (-i l1, -i l0)
  if (MU == 1) return row == 0 ? cneg(l1) : l0;                       // (-l1, l0)
  if (MU == 2) return row == 0 ? cneg(cmuli(l0)) : cmuli(l1);         // (-i l0, i l1)
  return row == 0 ? l0 : l1;                                           // (l0, l1)
}
// B_mu^H applied to a 2-spin vector w
template <int MU, typename C> __device__ __forceinline__ C applyBH(const C &w0, const C &w1, int row) {
  if (MU == 0) return row == 0 ? cmuli(w1) : cmuli(w0);               // (i w1, i w0)
  if (MU == 1) return row == 0 ? w1 : cneg(w0);                       // (w1, -w0)
  if (MU == 2) return row == 0 ? cmuli(w0) : cneg(cmuli(w1));         // (i w0, -i w1)
  return row == 0 ? w0 : w1;                                           // (w0, w1)
}

// One direction mu: accumulate S_u += w_f + w_b, S_l += B^H (w_f - w_b).
template <int MU, int SGN, typename R, class LD>
__device__ __forceinline__ void hop_dir(const typename cplx_t<R>::type *__restrict__ U, const LD &in, const Geom &g,
                                        const int xc[4], int s, int b, int j, typename cplx_t<R>::type Su[2][3],
                                        typename cplx_t<R>::type Sl[2][3]) {
  typedef typename cplx_t<R>::type C;
  int xf[4] = {xc[0], xc[1], xc[2], xc[3]};
  int xb[4] = {xc[0], xc[1], xc[2], xc[3]};
  xf[MU] = (xc[MU] + 1 == g.L[MU]) ? 0 : xc[MU] + 1;
  xb[MU] = (xc[MU] == 0) ? g.L[MU] - 1 : xc[MU] - 1;
  const int sf = site_of(g, xf);
  const int sb = site_of(g, xb);

  C wf[2][3], wb[2][3];
  {  // forward: h = u - sgn B l from psi(x+mu); w_f = U_mu(x) h
    const int64_t p = (int64_t)sf * 12 * b + j;
    C u[2][3], l[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[0][a] = in(p + (0 * 3 + a) * b);
      u[1][a] = in(p + (1 * 3 + a) * b);
      l[0][a] = in(p + (2 * 3 + a) * b);
      l[1][a] = in(p + (3 * 3 + a) * b);
    }
    C h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        C bl = applyB<MU>(l[0][a], l[1][a], r);
        h[r][a] = SGN > 0 ? csub(u[r][a], bl) : cadd(u[r][a], bl);
      }
    }
    const C *Ul = U + ((int64_t)s * 4 + MU) * 9;
    C m[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) m[a][c] = Ul[a * 3 + c];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        C acc = cmul(m[a][0], h[r][0]);
        acc = caxpy(m[a][1], h[r][1], acc);
        acc = caxpy(m[a][2], h[r][2], acc);
        wf[r][a] = acc;
      }
  }
  {  // backward: h' = u + sgn B l from psi(x-mu); w_b = U_mu(x-mu)^H h'
    const int64_t p = (int64_t)sb * 12 * b + j;
    C u[2][3], l[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[0][a] = in(p + (0 * 3 + a) * b);
      u[1][a] = in(p + (1 * 3 + a) * b);
      l[0][a] = in(p + (2 * 3 + a) * b);
      l[1][a] = in(p + (3 * 3 + a) * b);
    }
    C h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        C bl = applyB<MU>(l[0][a], l[1][a], r);
        h[r][a] = SGN > 0 ? cadd(u[r][a], bl) : csub(u[r][a], bl);
      }
    }
    const C *Ul = U + ((int64_t)sb * 4 + MU) * 9;
    C m[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) m[a][c] = Ul[a * 3 + c];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // (U^H h)_a = sum_c conj(U[c][a]) h_c
        C acc = cjmul(m[0][a], h[r][0]);
        acc = cadd(acc, cjmul(m[1][a], h[r][1]));
        acc = cadd(acc, cjmul(m[2][a], h[r][2]));
        wb[r][a] = acc;
      }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const C d0 = csub(wf[0][a], wb[0][a]);
    const C d1 = csub(wf[1][a], wb[1][a]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      Su[r][a] = cadd(Su[r][a], cadd(wf[r][a], wb[r][a]));
      Sl[r][a] = cadd(Sl[r][a], applyBH<MU>(d0, d1, r));
    }
  }
}

template <typename C, typename R> __device__ __forceinline__ C mk_r(R re, R im) {
  C c;
  c.x = re;
  c.y = im;
  return c;
}

// out[c] (c = 3*spin + colour) = (A psi)(s) for right-hand side j; self = psi(s).
template <int SGN, typename R, class LD>
__device__ __forceinline__ void dslash_site_ld(const typename cplx_t<R>::type *__restrict__ U, const LD &in,
                                               const Geom &g, int b, int s, int j, R diag,
                                               typename cplx_t<R>::type out[12], typename cplx_t<R>::type self[12]) {
  typedef typename cplx_t<R>::type C;
  int xc[4];
  site_coords(g, s, xc);
  C Su[2][3], Sl[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Su[r][a] = mk<C>(0.0, 0.0);
      Sl[r][a] = mk<C>(0.0, 0.0);
    }
  hop_dir<0, SGN, R>(U, in, g, xc, s, b, j, Su, Sl);
  hop_dir<1, SGN, R>(U, in, g, xc, s, b, j, Su, Sl);
  hop_dir<2, SGN, R>(U, in, g, xc, s, b, j, Su, Sl);
  hop_dir<3, SGN, R>(U, in, g, xc, s, b, j, Su, Sl);
  const int64_t p = (int64_t)s * 12 * b + j;
#pragma unroll
  for (int c = 0; c < 12; ++c) self[c] = in(p + c * b);
  const R half = (R)0.5;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const C su = Su[r][a], sl = Sl[r][a];
      const C pu = self[r * 3 + a], pl = self[(r + 2) * 3 + a];
      out[r * 3 + a] = mk_r<C, R>(diag * pu.x - half * su.x, diag * pu.y - half * su.y);
      out[(r + 2) * 3 + a] = SGN > 0 ? mk_r<C, R>(diag * pl.x + half * sl.x, diag * pl.y + half * sl.y)
                                     : mk_r<C, R>(diag * pl.x - half * sl.x, diag * pl.y - half * sl.y);
    }
}

template <int SGN, typename R>
__device__ __forceinline__ void dslash_site(const typename cplx_t<R>::type *__restrict__ U,
                                            const typename cplx_t<R>::type *__restrict__ in, const Geom &g, int b,
                                            int s, int j, R diag, typename cplx_t<R>::type out[12],
                                            typename cplx_t<R>::type self[12]) {
  PlainLoad<typename cplx_t<R>::type> ld{in};
  dslash_site_ld<SGN, R>(U, ld, g, b, s, j, diag, out, self);
}

}  // namespace dtr
