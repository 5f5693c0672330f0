// Half-precision-storage Wilson dslash for lattices far larger than L2, where
// the stencil is bound by HBM bandwidth.
//
// Storage: spinors as BF16 or FP16 complex pairs, 48 bytes (three 16-byte
// words) per item (site, right-hand side), item = site * b + rhs.  Layout is
// AoSoA over items: word w of 32 consecutive items is one contiguous 512-byte
// run, so every warp-wide 16-byte load touches four consecutive 128-byte lines
// instead of the twelve a plain [item][12] record layout would (that layout
// made the kernel L1-wavefront bound).  Links, AoSoA over sites: all three
// rows (36 complex = nine 16-byte words per site; link mu is read from the
// three words holding slots 9mu..9mu+8), or in "2-row" form the first two rows
// (24 complex = six words), with the third rebuilt in registers as
// conj(row0 x row1), exact for SU(3) (see half_link_rows).  Arithmetic is FP32.
//
// Algorithmic traffic per site and right-hand side: 48 B in + 48 B out, plus
// 4 links x 36 B = 144 B per site shared by the b right-hand sides (96 B with
// two stored rows).  The
// eight neighbour reads of each spinor are served by L1/L2 (a t-slab of the
// lattice is a few MB), so DRAM traffic stays close to the algorithmic bytes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>

#include "dtr_internal.cuh"

namespace dtr {

template <typename H> struct HalfOps;
template <> struct HalfOps<__nv_bfloat162> {
  static __device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ __nv_bfloat162 from_f2(float2 v) { return __float22bfloat162_rn(v); }
};
template <> struct HalfOps<__half2> {
  static __device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }
  static __device__ __forceinline__ __half2 from_f2(float2 v) { return __float22half2_rn(v); }
};

// uint4 word index of word w (0..2) of spinor item `it`, and of link word w (0..5) of a site
// (word indices stay below 2^31 for every lattice the ABI accepts: V <= 2^26, b <= 64 is 2^32 items only for
//  the FP64 path; half fields are used with V * b * 3 < 2^31)
__host__ __device__ __forceinline__ int64_t spw(int64_t it, int w) { return (((it >> 5) * 3 + w) << 5) + (it & 31); }
__host__ __device__ __forceinline__ int spw32(int it, int w) { return (((it >> 5) * 3 + w) << 5) + (it & 31); }
__host__ __device__ __forceinline__ int64_t lkw(int64_t site, int w) { return (((site >> 5) * 6 + w) << 5) + (site & 31); }
__host__ __device__ __forceinline__ int lkw32(int site, int w) { return (((site >> 5) * 6 + w) << 5) + (site & 31); }
// links with all three rows stored: 36 complex (nine 16-byte words) per site
__host__ __device__ __forceinline__ int64_t lkw3(int64_t site, int w) { return (((site >> 5) * 9 + w) << 5) + (site & 31); }
__host__ __device__ __forceinline__ int lkw3_32(int site, int w) { return (((site >> 5) * 9 + w) << 5) + (site & 31); }

// 12 complex values of item `it` = 3 x 16-byte words
template <typename H> __device__ __forceinline__ void load12(const H *__restrict__ base, int it, float2 out[12]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(base);
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    const uint4 u = __ldg(q + spw32(it, w));
    const unsigned int words[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      H h;
      *reinterpret_cast<unsigned int *>(&h) = words[k];
      out[w * 4 + k] = HalfOps<H>::to_f2(h);
    }
  }
}
template <typename H> __device__ __forceinline__ void store12(H *__restrict__ base, int it, const float2 v[12]) {
  uint4 *q = reinterpret_cast<uint4 *>(base);
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    unsigned int words[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const H h = HalfOps<H>::from_f2(v[w * 4 + k]);
      words[k] = *reinterpret_cast<const unsigned int *>(&h);
    }
    q[spw32(it, w)] = make_uint4(words[0], words[1], words[2], words[3]);
  }
}

// link mu of a site stored with all three rows (complex slots 9mu..9mu+8 of the site's 36)
template <int MU, typename H>
__device__ __forceinline__ void load_link3(const H *__restrict__ U, int site, float2 m[3][3]) {
  constexpr int w0 = (9 * MU) / 4, off = (9 * MU) % 4;
  const uint4 *q = reinterpret_cast<const uint4 *>(U);
  const uint4 u0 = __ldg(q + lkw3_32(site, w0)), u1 = __ldg(q + lkw3_32(site, w0 + 1)),
              u2 = __ldg(q + lkw3_32(site, w0 + 2));
  const unsigned int words[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    H h;
    *reinterpret_cast<unsigned int *>(&h) = words[off + k];
    m[k / 3][k % 3] = HalfOps<H>::to_f2(h);
  }
}

// link mu of a site (two stored rows = complex slots 6mu..6mu+5 of the site's
// 24) -> full 3x3 in FP32
template <int MU, typename H>
__device__ __forceinline__ void load_link(const H *__restrict__ U, int site, float2 m[3][3]) {
  constexpr int w0 = (6 * MU) / 4, off = (6 * MU) % 4;
  const uint4 *q = reinterpret_cast<const uint4 *>(U);
  const uint4 u0 = __ldg(q + lkw32(site, w0)), u1 = __ldg(q + lkw32(site, w0 + 1));
  const unsigned int words[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
  float2 e[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    H h;
    *reinterpret_cast<unsigned int *>(&h) = words[off + k];
    e[k] = HalfOps<H>::to_f2(h);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    m[0][c] = e[c];
    m[1][c] = e[3 + c];
  }
  // row2 = conj(row0 x row1)
  m[2][0] = make_float2(m[0][1].x * m[1][2].x - m[0][1].y * m[1][2].y - (m[0][2].x * m[1][1].x - m[0][2].y * m[1][1].y),
                        -(m[0][1].x * m[1][2].y + m[0][1].y * m[1][2].x - (m[0][2].x * m[1][1].y + m[0][2].y * m[1][1].x)));
  m[2][1] = make_float2(m[0][2].x * m[1][0].x - m[0][2].y * m[1][0].y - (m[0][0].x * m[1][2].x - m[0][0].y * m[1][2].y),
                        -(m[0][2].x * m[1][0].y + m[0][2].y * m[1][0].x - (m[0][0].x * m[1][2].y + m[0][0].y * m[1][2].x)));
  m[2][2] = make_float2(m[0][0].x * m[1][1].x - m[0][0].y * m[1][1].y - (m[0][1].x * m[1][0].x - m[0][1].y * m[1][0].y),
                        -(m[0][0].x * m[1][1].y + m[0][0].y * m[1][1].x - (m[0][1].x * m[1][0].y + m[0][1].y * m[1][0].x)));
}

template <int MU> __device__ __forceinline__ float2 hB(const float2 &l0, const float2 &l1, int row) {
  if (MU == 0) return row == 0 ? make_float2(l1.y, -l1.x) : make_float2(l0.y, -l0.x);   // -i l
  if (MU == 1) return row == 0 ? make_float2(-l1.x, -l1.y) : l0;
  if (MU == 2) return row == 0 ? make_float2(l0.y, -l0.x) : make_float2(-l1.y, l1.x);
  return row == 0 ? l0 : l1;
}
template <int MU> __device__ __forceinline__ float2 hBH(const float2 &w0, const float2 &w1, int row) {
  if (MU == 0) return row == 0 ? make_float2(-w1.y, w1.x) : make_float2(-w0.y, w0.x);   // i w
  if (MU == 1) return row == 0 ? w1 : make_float2(-w0.x, -w0.y);
  if (MU == 2) return row == 0 ? make_float2(-w0.y, w0.x) : make_float2(w1.y, -w1.x);
  return row == 0 ? w0 : w1;
}

template <int MU, typename H, int ROWS>
__device__ __forceinline__ void half_hop(const H *__restrict__ U, const H *__restrict__ in, const Geom &g,
                                         const int xc[4], const int str[4], int s, int b, int j, float2 Su[2][3],
                                         float2 Sl[2][3]) {
  // neighbours by stride arithmetic (periodic wrap), int32 throughout
  const int last = g.L[MU] - 1;
  const int sf = s + (xc[MU] == last ? -last * str[MU] : str[MU]);
  const int sb = s + (xc[MU] == 0 ? last * str[MU] : -str[MU]);
  float2 wf[2][3], wb[2][3];
  {
    float2 v[12];
    load12<H>(in, sf * b + j, v);
    float2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float2 bl = hB<MU>(v[6 + a], v[9 + a], r);
        h[r][a] = make_float2(v[r * 3 + a].x - bl.x, v[r * 3 + a].y - bl.y);
      }
    float2 m[3][3];
    if (ROWS == 3) load_link3<MU, H>(U, s, m);
    else load_link<MU, H>(U, s, m);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          acc.x = fmaf(m[a][c].x, h[r][c].x, fmaf(-m[a][c].y, h[r][c].y, acc.x));
          acc.y = fmaf(m[a][c].x, h[r][c].y, fmaf(m[a][c].y, h[r][c].x, acc.y));
        }
        wf[r][a] = acc;
      }
  }
  {
    float2 v[12];
    load12<H>(in, sb * b + j, v);
    float2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float2 bl = hB<MU>(v[6 + a], v[9 + a], r);
        h[r][a] = make_float2(v[r * 3 + a].x + bl.x, v[r * 3 + a].y + bl.y);
      }
    float2 m[3][3];
    if (ROWS == 3) load_link3<MU, H>(U, sb, m);
    else load_link<MU, H>(U, sb, m);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // conj(U[c][a]) h_c
          acc.x = fmaf(m[c][a].x, h[r][c].x, fmaf(m[c][a].y, h[r][c].y, acc.x));
          acc.y = fmaf(m[c][a].x, h[r][c].y, fmaf(-m[c][a].y, h[r][c].x, acc.y));
        }
        wb[r][a] = acc;
      }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 d0 = make_float2(wf[0][a].x - wb[0][a].x, wf[0][a].y - wb[0][a].y);
    const float2 d1 = make_float2(wf[1][a].x - wb[1][a].x, wf[1][a].y - wb[1][a].y);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      Su[r][a].x += wf[r][a].x + wb[r][a].x;
      Su[r][a].y += wf[r][a].y + wb[r][a].y;
      const float2 bh = hBH<MU>(d0, d1, r);
      Sl[r][a].x += bh.x;
      Sl[r][a].y += bh.y;
    }
  }
}

// out = A in on half-precision AoSoA fields; thread per item (site, rhs), rhs fastest.
template <typename H, int MINB, int ROWS>
__global__ void __launch_bounds__(256, MINB) k_dslash_half(const H *__restrict__ U, const H *__restrict__ in,
                                                           H *__restrict__ out, Geom g, int b, float diag) {
  const int n = g.V * b;
  const int lb = (b & (b - 1)) == 0 ? __ffs(b) - 1 : -1;  // log2 b for a power-of-two width
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    const int j = lb >= 0 ? it & (b - 1) : it % b;
    const int s = lb >= 0 ? it >> lb : it / b;
    int xc[4];
    site_coords(g, s, xc);
    const int str[4] = {1, g.L[0], g.L[0] * g.L[1], g.L[0] * g.L[1] * g.L[2]};
    float2 Su[2][3], Sl[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) Su[r][a] = Sl[r][a] = make_float2(0.f, 0.f);
    half_hop<0, H, ROWS>(U, in, g, xc, str, s, b, j, Su, Sl);
    half_hop<1, H, ROWS>(U, in, g, xc, str, s, b, j, Su, Sl);
    half_hop<2, H, ROWS>(U, in, g, xc, str, s, b, j, Su, Sl);
    half_hop<3, H, ROWS>(U, in, g, xc, str, s, b, j, Su, Sl);
    float2 self[12], o[12];
    load12<H>(in, it, self);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 pu = self[r * 3 + a], pl = self[(r + 2) * 3 + a];
        o[r * 3 + a] = make_float2(diag * pu.x - 0.5f * Su[r][a].x, diag * pu.y - 0.5f * Su[r][a].y);
        o[(r + 2) * 3 + a] = make_float2(diag * pl.x + 0.5f * Sl[r][a].x, diag * pl.y + 0.5f * Sl[r][a].y);
      }
    store12<H>(out, it, o);
  }
}

// complex c of item `it` in an AoSoA half field (units of one complex = 4 bytes)
__host__ __device__ __forceinline__ int64_t spc(int64_t it, int c) { return spw(it, c >> 2) * 4 + (c & 3); }

// canonical complex128 (column-major N x nrhs) -> AoSoA half field of width b; padding columns zero
template <typename H>
__global__ void k_pack_half(const double2 *__restrict__ canon, H *__restrict__ out, int64_t V, int nrhs, int b) {
  const int64_t n = V * b * 12;
  const int64_t N = V * 12;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % 12);
    const int64_t it = e / 12;
    const int j = (int)(it % b);
    const int64_t s = it / b;
    const double2 v = j < nrhs ? canon[(int64_t)j * N + s * 12 + c] : make_double2(0.0, 0.0);
    out[spc(it, c)] = HalfOps<H>::from_f2(make_float2((float)v.x, (float)v.y));
  }
}

template <typename H>
__global__ void k_unpack_half(const H *__restrict__ in, double2 *__restrict__ canon, int64_t V, int nrhs, int b) {
  const int64_t N = V * 12;
  const int64_t n = N * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % N;
    const int j = (int)(e / N);
    const float2 f = HalfOps<H>::to_f2(in[spc((i / 12) * b + j, (int)(i % 12))]);
    canon[e] = make_double2((double)f.x, (double)f.y);
  }
}

// FP64 links [site][mu][3][3] -> two rows, half precision: the 24 complex
// slots of a site (slot 6mu + k = row k/3, column k%3 of link mu), AoSoA over sites
// all three rows: slot 9mu + k = row k/3, column k%3 of link mu
template <typename H> __global__ void k_pack_links_half3(const double2 *__restrict__ U, H *__restrict__ out, int64_t V) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < V * 36; e += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(e % 36);
    const int64_t site = e / 36;
    const int mu = slot / 9, k = slot % 9;
    const double2 v = U[(site * 4 + mu) * 9 + k];
    out[lkw3(site, slot >> 2) * 4 + (slot & 3)] = HalfOps<H>::from_f2(make_float2((float)v.x, (float)v.y));
  }
}

template <typename H> __global__ void k_pack_links_half(const double2 *__restrict__ U, H *__restrict__ out, int64_t V) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < V * 24; e += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(e % 24);
    const int64_t site = e / 24;
    const int mu = slot / 6, k = slot % 6;
    const double2 v = U[(site * 4 + mu) * 9 + k];
    out[lkw(site, slot >> 2) * 4 + (slot & 3)] = HalfOps<H>::from_f2(make_float2((float)v.x, (float)v.y));
  }
}

// CTAs per SM the half stencil is compiled for: 2 (no register spills) or 3
// (more warps in flight, some spills); DTR_HALF_OCCUPANCY=3 selects the latter.
static int half_occupancy() {
  static int occ = 0;
  if (!occ) {
    const char *e = getenv("DTR_HALF_OCCUPANCY");
    occ = (e && e[0] == '3') ? 3 : 2;
  }
  return occ;
}

// Links of the half-precision stencil: all three rows stored (default), 144 B per
// site, so a site and right-hand side moves exactly the algorithmic 240 B; or two
// rows with the third rebuilt in registers as conj(row0 x row1) (96 B of links,
// about 36 more FP32 instructions per hop).  DTR_HALF_LINKS=2 selects the
// latter; read once per process, before the first gauge field is packed.
int half_link_rows() {
  static int v = 0;
  if (!v) {
    const char *e = getenv("DTR_HALF_LINKS");
    v = (e && e[0] == '2') ? 2 : 3;
  }
  return v;
}

template <typename H>
static void launch_half_kernel(const H *U, const H *in, H *out, const Geom &g, int b, float diag, unsigned grid,
                               cudaStream_t st) {
  if (half_link_rows() == 3)
    k_dslash_half<H, 2, 3><<<grid, 256, 0, st>>>(U, in, out, g, b, diag);
  else if (half_occupancy() == 3)
    k_dslash_half<H, 3, 2><<<grid, 256, 0, st>>>(U, in, out, g, b, diag);
  else
    k_dslash_half<H, 2, 2><<<grid, 256, 0, st>>>(U, in, out, g, b, diag);
}

static unsigned g1(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 65535LL * 16) g = 65535LL * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// sizes rounded up to whole groups of 32 items / sites
size_t half_links_bytes(int64_t V) {
  return (size_t)((V + 31) / 32) * 32 * (half_link_rows() == 3 ? 36 : 24) * sizeof(__half2);
}
size_t half_field_bytes(int64_t V, int b) { return (size_t)((V * b + 31) / 32) * 32 * 12 * sizeof(__half2); }

void launch_pack_links_half(const double2 *U64, void *out, int64_t V, int bf16, cudaStream_t st) {
  if (half_link_rows() == 3) {
    if (bf16)
      k_pack_links_half3<__nv_bfloat162><<<g1(V * 36), 256, 0, st>>>(U64, (__nv_bfloat162 *)out, V);
    else
      k_pack_links_half3<__half2><<<g1(V * 36), 256, 0, st>>>(U64, (__half2 *)out, V);
  } else if (bf16) {
    k_pack_links_half<__nv_bfloat162><<<g1(V * 24), 256, 0, st>>>(U64, (__nv_bfloat162 *)out, V);
  } else {
    k_pack_links_half<__half2><<<g1(V * 24), 256, 0, st>>>(U64, (__half2 *)out, V);
  }
  count_launches(1);
}

void launch_dslash_half_canon(const void *Uh, const double2 *in, double2 *out, void *work, const Geom &g, int nrhs,
                              int b, double m0, int bf16, cudaStream_t st) {
  const int64_t V = g.V;
  char *w = (char *)work;
  const size_t fb = (half_field_bytes(V, b) + 255) / 256 * 256;
  if (bf16) {
    __nv_bfloat162 *a = (__nv_bfloat162 *)w, *o = (__nv_bfloat162 *)(w + fb);
    k_pack_half<__nv_bfloat162><<<g1(V * b * 12), 256, 0, st>>>(in, a, V, nrhs, b);
    launch_half_kernel<__nv_bfloat162>((const __nv_bfloat162 *)Uh, a, o, g, b, (float)(4.0 + m0), g1(V * b), st);
    k_unpack_half<__nv_bfloat162><<<g1(V * 12 * nrhs), 256, 0, st>>>(o, out, V, nrhs, b);
  } else {
    __half2 *a = (__half2 *)w, *o = (__half2 *)(w + fb);
    k_pack_half<__half2><<<g1(V * b * 12), 256, 0, st>>>(in, a, V, nrhs, b);
    launch_half_kernel<__half2>((const __half2 *)Uh, a, o, g, b, (float)(4.0 + m0), g1(V * b), st);
    k_unpack_half<__half2><<<g1(V * 12 * nrhs), 256, 0, st>>>(o, out, V, nrhs, b);
  }
  count_launches(3);
}

// back-to-back launches of the stencil alone on half fields in `work` (timing)
void launch_dslash_half_raw(const void *Uh, void *work, const Geom &g, int b, double m0, int bf16, int reps,
                            cudaStream_t st) {
  const int64_t V = g.V;
  char *w = (char *)work;
  const size_t fb = (half_field_bytes(V, b) + 255) / 256 * 256;
  for (int r = 0; r < reps; ++r) {
    if (bf16)
      launch_half_kernel<__nv_bfloat162>((const __nv_bfloat162 *)Uh, (const __nv_bfloat162 *)w,
                                         (__nv_bfloat162 *)(w + fb), g, b, (float)(4.0 + m0), g1(V * b), st);
    else
      launch_half_kernel<__half2>((const __half2 *)Uh, (const __half2 *)w, (__half2 *)(w + fb), g, b,
                                  (float)(4.0 + m0), g1(V * b), st);
    count_launches(1);
  }
}

}  // namespace dtr
