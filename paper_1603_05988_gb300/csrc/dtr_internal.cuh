// Internal declarations shared by the libdtr translation units.
//
// Internal field layout ("RHS-inner"): a block of b right-hand sides is stored
// as [site][12][b] complex values, dof-component c = 3*spin + colour.  A warp
// then covers 32/b sites x b right-hand sides and every load of one component
// is a contiguous run of b complex numbers, while the 32/b lanes of a site
// share (broadcast) its gauge links.  b is the block width padded up to a
// power of two <= 64 (padding columns are zero and never iterate).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dtr.h"

namespace dtr {

// ------------------------------------------------------------ error plumbing
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
// process-wide count of kernels launched by the library
void count_launches(int n);
void capture_begin();
void capture_end();

#define DTR_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::dtr::cuda_fail(e_, #call); \
  } while (0)

#define DTR_LAUNCH_CHECK(what)                           \
  do {                                                   \
    cudaError_t e_ = cudaGetLastError();                 \
    if (e_ != cudaSuccess) return ::dtr::cuda_fail(e_, what); \
  } while (0)

// ------------------------------------------------------------------ complex
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
  C c; c.x = re; c.y = im; return c;
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cjmul(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double inv = 1.0 / (b.x * b.x + b.y * b.y);  // one division (FP64 divides are slow on this part)
  return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a + s*b with complex s
__host__ __device__ __forceinline__ double2 caxpy(double2 s, double2 b, double2 a) {
  return make_double2(fma(s.x, b.x, fma(-s.y, b.y, a.x)), fma(s.x, b.y, fma(s.y, b.x, a.y)));
}
__host__ __device__ __forceinline__ float2 caxpy(float2 s, float2 b, float2 a) {
  return make_float2(fmaf(s.x, b.x, fmaf(-s.y, b.y, a.x)), fmaf(s.x, b.y, fmaf(s.y, b.x, a.y)));
}
__host__ __device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
// multiply by i
__host__ __device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
__host__ __device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];
  int V;
  unsigned mg[3];  // division by L[0..2] as (umulhi(n, mg) + n) >> sh, exact for n < 2^31
  int sh[3];       // (a runtime integer division costs ~20 instructions, this three)
};

__device__ __forceinline__ int div_by(int n, unsigned m, int sh) {
  return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> sh);
}

__device__ __forceinline__ void site_coords(const Geom &g, int s, int c[4]) {
  const int r0 = div_by(s, g.mg[0], g.sh[0]);
  c[0] = s - r0 * g.L[0];
  const int r1 = div_by(r0, g.mg[1], g.sh[1]);
  c[1] = r0 - r1 * g.L[1];
  const int r2 = div_by(r1, g.mg[2], g.sh[2]);
  c[2] = r1 - r2 * g.L[2];
  c[3] = r2;
}
__device__ __forceinline__ int site_of(const Geom &g, const int c[4]) {
  return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// Hierarchical-probing colour of a site; ncolors in {1, 2, 16, 32, 256, ...}.
__host__ __device__ __forceinline__ int hp_colour(const int c[4], int ncolors) {
  if (ncolors <= 1) return 0;
  int col = (c[0] + c[1] + c[2] + c[3]) & 1;
  int n = 2;
  int level = 0;
  while (n < ncolors) {
    col += n * (((c[1] >> level) & 1) + 2 * ((c[2] >> level) & 1) + 4 * ((c[3] >> level) & 1));
    n *= 8;
    if (n >= ncolors) break;
    col += n * (((c[0] >> (level + 1)) + (c[1] >> (level + 1)) + (c[2] >> (level + 1)) + (c[3] >> (level + 1))) & 1);
    n *= 2;
    ++level;
  }
  return col;
}

// ------------------------------------------------------------------ handles
}  // namespace dtr

struct dtr_lattice_s {
  int dims[4];
  int64_t V;
  int64_t N;
};

struct dtr_gauge_s {
  dtr_lattice_s lat;
  double2 *U64;   // [site][mu][3][3], FP64
  float2 *U32;    // same layout, FP32
  void *Ubf16;    // BF16 links of the half-precision stencil, AoSoA over sites: three stored rows
                  // (36 complex per site) or two (24), see half_link_rows()
  void *Uf16;     // same, FP16
  void *Udf;      // [site][mu][3][3] FP64 links split into FP32 hi + lo (16 B per complex: Re hi, Re lo,
                  // Im hi, Im lo) for the double-float residual update of the mixed solvers
};

struct dtr_defl_s {
  dtr_lattice_s lat;
  int k;
  dtr_prec prec;
  void *V;            // row-major [dof][k] complex, FP64 (double2) or FP32 (float2)
  double *inv_lambda; // device, k
  double td[2];
  double tdg[16][2];  // T_D of Gamma_n (Gamma-insertion traces), valid where tdg_ok bit n is set
  unsigned tdg_ok;
  double2 *Ginv;      // device k x k (row-major) inverse of G = V^H g5 A V once the Galerkin correction is on
};

namespace dtr {

// Multiplier and shift for exact unsigned division by d >= 1 of any n < 2^31 (division
// by an invariant integer with an add step): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1.
inline void div_magic(int d, unsigned *m, int *l) {
  int k = 0;
  while ((1LL << k) < d) ++k;
  *l = k;
  *m = (unsigned)((((1ULL << 32) * (unsigned long long)((1LL << k) - d)) / (unsigned long long)d) + 1ULL);
}

inline Geom geom_of(const dtr_lattice_s &l) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = l.dims[i];
  for (int i = 0; i < 3; ++i) div_magic(g.L[i], &g.mg[i], &g.sh[i]);
  g.V = (int)l.V;
  return g;
}

// Padded block width: next power of two >= n, n <= 64.
inline int pad_rhs(int n) {
  int b = 1;
  while (b < n) b <<= 1;
  return b;
}

// Cross-block deterministic reduction scratch.
struct Reduce {
  double2 *partial;     // [max_blocks][slots][b]
  unsigned int *counter;
};

// ---------------------------------------------------------------- kernels
// pack canonical (column-major N x nrhs, c128) -> internal [site][12][b] of R
template <typename R>
void launch_pack(const double2 *canon, typename cplx_t<R>::type *internal, int64_t V, int nrhs, int b,
                 cudaStream_t st);
// unpack internal -> canonical
template <typename R>
void launch_unpack(const typename cplx_t<R>::type *internal, double2 *canon, int64_t V, int nrhs, int b,
                   cudaStream_t st);

// out = A in (dagger: A^H) on internal fields of width b
template <typename R>
void launch_dslash(const typename cplx_t<R>::type *U, const typename cplx_t<R>::type *in,
                   typename cplx_t<R>::type *out, const Geom &g, int b, double m0, int dagger, cudaStream_t st);
// out = A in on the internal layout, in FP32, arithmetic in double-float on the split links Udf
void launch_dslash_df(const void *Udf, const float2 *in, double2 *out, const Geom &g, int b, double m0,
                      cudaStream_t st);

// half-precision-storage stencil (dslash_half.cu)
size_t half_links_bytes(int64_t V);
int half_link_rows();
size_t half_field_bytes(int64_t V, int b);
void launch_pack_links_half(const double2 *U64, void *out, int64_t V, int bf16, cudaStream_t st);
// random SU(3) links U = exp(i eps H) generated on the device from (seed, site, mu) (gauge.cu)
void launch_make_links(double2 *U64, int64_t V, double eps, uint64_t seed, cudaStream_t st);
void launch_dslash_half_canon(const void *Uh, const double2 *in, double2 *out, void *work, const Geom &g, int nrhs,
                              int b, double m0, int bf16, cudaStream_t st);
void launch_dslash_half_raw(const void *Uh, void *work, const Geom &g, int b, double m0, int bf16, int reps,
                            cudaStream_t st);

// noise into internal FP64 layout of width b: block column k is global column
// g0 + k of the run-major sequence (ncols probing columns per run, runs from
// run0), probing column qoff + (g0 + k) % ncols of its run; columns nrhs..b-1
// are zero padding.  codes (or NULL): the same entries as one byte each, same
// layout: bits 0-1 the power c of i (z = i^c), bit 2 set for a zero.
void launch_noise(double2 *out, const Geom &g, uint64_t seed, int64_t run0, int ncolors, int dilute12, int64_t g0,
                  int64_t ncols, int nrhs, int b, cudaStream_t st, int64_t qoff = 0, unsigned char *codes = nullptr);
// noise into canonical layout
void launch_noise_canon(double2 *out, const Geom &g, uint64_t seed, int64_t z0_index, int ncolors,
                        int dilute12, int64_t q0, int nrhs, cudaStream_t st);

}  // namespace dtr
