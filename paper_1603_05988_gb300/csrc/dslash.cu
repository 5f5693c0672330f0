// Plain dslash (A or A^H) on internal fields, and the canonical <-> internal
// layout conversions used at the C-ABI boundary.
#include "dslash_core.cuh"

namespace dtr {

template <typename R, int SGN>
__global__ void __launch_bounds__(256) dslash_kernel(const typename cplx_t<R>::type *__restrict__ U,
                                                     const typename cplx_t<R>::type *__restrict__ in,
                                                     typename cplx_t<R>::type *__restrict__ out, Geom g, int b,
                                                     int logb, R diag) {
  typedef typename cplx_t<R>::type C;
  const int64_t n = (int64_t)g.V << logb;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(it & (b - 1));
    const int s = (int)(it >> logb);
    C o[12], self[12];
    dslash_site<SGN, R>(U, in, g, b, s, j, diag, o, self);
    C *q = out + (int64_t)s * 12 * b + j;
#pragma unroll
    for (int c = 0; c < 12; ++c) q[c * b] = o[c];
  }
}

static int ilog2(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

template <typename R>
void launch_dslash(const typename cplx_t<R>::type *U, const typename cplx_t<R>::type *in,
                   typename cplx_t<R>::type *out, const Geom &g, int b, double m0, int dagger, cudaStream_t st) {
  const int64_t n = (int64_t)g.V * b;
  const int T = 256;
  const unsigned grid = (unsigned)((n + T - 1) / T);
  if (dagger)
    dslash_kernel<R, -1><<<grid, T, 0, st>>>(U, in, out, g, b, ilog2(b), (R)(4.0 + m0));
  else
    dslash_kernel<R, 1><<<grid, T, 0, st>>>(U, in, out, g, b, ilog2(b), (R)(4.0 + m0));
  count_launches(1);
}

template void launch_dslash<double>(const double2 *, const double2 *, double2 *, const Geom &, int, double, int,
                                    cudaStream_t);
template void launch_dslash<float>(const float2 *, const float2 *, float2 *, const Geom &, int, double, int,
                                   cudaStream_t);

// ------------------------------------------------------------------ layouts
template <typename R>
__global__ void pack_kernel(const double2 *__restrict__ canon, typename cplx_t<R>::type *__restrict__ internal,
                            int64_t V, int nrhs, int b) {
  typedef typename cplx_t<R>::type C;
  const int64_t n = V * 12 * b;
  const int64_t N = V * 12;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    const int64_t i = e / b;  // dof index = site*12 + c
    double2 v = j < nrhs ? canon[(int64_t)j * N + i] : make_double2(0.0, 0.0);
    internal[e] = mk<C>(v.x, v.y);
  }
}

template <typename R>
__global__ void unpack_kernel(const typename cplx_t<R>::type *__restrict__ internal, double2 *__restrict__ canon,
                              int64_t V, int nrhs, int b) {
  const int64_t N = V * 12;
  const int64_t n = N * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % N;
    const int j = (int)(e / N);
    const typename cplx_t<R>::type v = internal[i * b + j];
    canon[e] = make_double2((double)v.x, (double)v.y);
  }
}

static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 65535LL * 16) g = 65535LL * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename R>
void launch_pack(const double2 *canon, typename cplx_t<R>::type *internal, int64_t V, int nrhs, int b,
                 cudaStream_t st) {
  pack_kernel<R><<<grid_for(V * 12 * b), 256, 0, st>>>(canon, internal, V, nrhs, b); count_launches(1);
}
template <typename R>
void launch_unpack(const typename cplx_t<R>::type *internal, double2 *canon, int64_t V, int nrhs, int b,
                   cudaStream_t st) {
  unpack_kernel<R><<<grid_for(V * 12 * nrhs), 256, 0, st>>>(internal, canon, V, nrhs, b); count_launches(1);
}

template void launch_pack<double>(const double2 *, double2 *, int64_t, int, int, cudaStream_t);
template void launch_pack<float>(const double2 *, float2 *, int64_t, int, int, cudaStream_t);
template void launch_unpack<double>(const double2 *, double2 *, int64_t, int, int, cudaStream_t);
template void launch_unpack<float>(const float2 *, double2 *, int64_t, int, int, cudaStream_t);

}  // namespace dtr
