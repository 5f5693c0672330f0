// Deflation projection specialised to hierarchical-probing blocks (Section 5.2,
// Algorithm 1's deflation term with z = z0 .* z_h).
//
// All columns of an HP block share one z0 and differ only by the Hadamard
// sign H[c, j] of each site colour c (and, with dilution, by the dof type a
// they keep).  Hence
//     V^H z_(j,a)         = sum_c H[c, j] W_a[c]
//     V^H g5 z_(j,a)      = sum_c H[c, j] g5(a) W_a[c]
//     W_a[c][m]           = sum_{sites x of colour c} conj(V[12x + a][m]) z0(12x + a)
// and without dilution a column sums all twelve a.  W needs one pass over V
// per z0 with FP64 ADDITIONS only (z0 is 1, i, -1 or -i, so conj(v) z0 is a
// swap and sign change of v), instead of a complex multiply-add per column:
// 2 N k additions per run rather than 8 N k b flops per block.  On GB300, where
// FP64 runs at 1/61 of the FP32 rate, this is the difference between the
// projection costing as much as the solves and costing almost nothing.
//
// With V stored in FP32 or BF16 the additions of one 64-site tile run in FP32
// with compensation: every term is an exactly widened stored value with its
// sign flipped or its parts swapped, and each addition is an error-free
// transformation (Knuth's TwoSum: s + t = fl(s + t) + e exactly), the error
// words summed apart, so the tile's sum is carried as a pair (s, c) accurate
// to about 64 * 2^-48 relative; each tile's pair is added into FP64
// accumulators in a fixed order.  The pass stays on the FP32 pipe (seven FP32
// additions per term instead of one FP64 addition, 64x cheaper on GB300; the
// real and imaginary parts go through one packed FP32x2 TwoSum, and a thread's
// four elements share one probing code per site); FP64 V keeps plain FP64
// additions.  W of a run is computed once and reused by every block of that
// run (reuse_w).
#include <cstring>
#include <type_traits>

#include "deflate.cuh"
#include "philox.cuh"

namespace dtr {

constexpr int kHPMaxThreads = 512;
constexpr int kHPTile = 64;  // sites per shared-memory code tile
constexpr int kHPEpt = 4;    // row elements (dof type a, vector m) per thread and block row chunk

// Every site's deflation rows are one contiguous run of 12 k values
// (V[12x + a][m], row-major), so a block streams whole site runs: thread t
// keeps the kHPEpt consecutive elements e = e0 + kHPEpt t + j of the run (one
// 16-byte load for BF16 values, two for FP32; 12 k is a multiple of 4, so they
// never pass the end of the run), each with a fixed dof type a = e / k, and
// accumulates conj(V) z0 over the block's sites of one colour (four sites in
// flight).  blockIdx.y picks the chunk e0 of the run when 12 k > T kHPEpt.
// partial[(split*nc + c) * 12k + e].
// Tile accumulator: FP32 TwoSum pairs for FP32 / BF16 V, plain FP64 for FP64 V.
struct HPAccF {
  float2 s, c;  // running sum and the sum of the rounding errors
  __device__ __forceinline__ void zero() { s = c = make_float2(0.f, 0.f); }
  __device__ __forceinline__ static void two_sum(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
  }
  // both parts at once with packed FP32x2 additions (each lane rounds as __fadd_rn does)
  __device__ __forceinline__ static float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
  __device__ __forceinline__ void add(float re, float im) {
    const float2 x = make_float2(re, im);
    const float2 t = __fadd2_rn(s, x);
    const float2 bp = __fadd2_rn(t, neg2(s));
    const float2 e = __fadd2_rn(__fadd2_rn(s, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(x, neg2(bp)));
    s = t;
    c = __fadd2_rn(c, e);
  }
  __device__ __forceinline__ void flush(double2 &acc) const {
    acc.x += (double)s.x + (double)c.x;
    acc.y += (double)s.y + (double)c.y;
  }
};
struct HPAccD {
  double2 s;
  __device__ __forceinline__ void zero() { s = make_double2(0.0, 0.0); }
  __device__ __forceinline__ void add(double re, double im) {
    s.x += re;
    s.y += im;
  }
  __device__ __forceinline__ void flush(double2 &acc) const {
    acc.x += s.x;
    acc.y += s.y;
  }
};
template <typename VC> struct HPAcc { typedef HPAccF type; };
template <> struct HPAcc<double2> { typedef HPAccD type; };
__device__ __forceinline__ float2 hp_widen(const float2 &v) { return v; }
__device__ __forceinline__ float2 hp_widen(const bfc2 &v) { return __bfloat1622float2(v); }
__device__ __forceinline__ double2 hp_widen(const double2 &v) { return v; }

// four consecutive stored values (16-byte aligned: 12 k and the element offset are multiples of 4)
struct Four16 { uint4 w[1]; };
struct Four32 { uint4 w[2]; };
struct Four64 { uint4 w[4]; };
template <typename VC> struct FourOf;
template <> struct FourOf<bfc2> { typedef Four16 type; };
template <> struct FourOf<float2> { typedef Four32 type; };
template <> struct FourOf<double2> { typedef Four64 type; };
template <typename VC> __device__ __forceinline__ typename FourOf<VC>::type hp_load4(const VC *p) {
  typename FourOf<VC>::type f;
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
  for (int u = 0; u < (int)(sizeof(f) / 16); ++u) f.w[u] = __ldcs(q + u);
  return f;
}
template <typename VC> __device__ __forceinline__ VC hp_elem(const typename FourOf<VC>::type &f, int j) {
  VC v;
  memcpy(&v, reinterpret_cast<const char *>(f.w) + j * sizeof(VC), sizeof(VC));
  return v;
}

template <typename VC>
__global__ void __launch_bounds__(kHPMaxThreads, 2)
    k_hp_partial(const VC *__restrict__ Vd, const int *__restrict__ sites, int per_colour, int nc, int nsplit, int k,
                 uint64_t seed, int64_t run, CodeXform xf, double2 *__restrict__ partial) {
  typedef typename HPAcc<VC>::type AC;
  __shared__ unsigned char codes[kHPTile * 12];
  __shared__ int tile_sites[kHPTile];
  const int c = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  const int L = 12 * k;
  const int T = blockDim.x;
  const int e0 = blockIdx.y * T * kHPEpt + kHPEpt * threadIdx.x;  // this thread's first element
  const int s0 = (int)(((int64_t)per_colour * split) / nsplit);
  const int s1 = (int)(((int64_t)per_colour * (split + 1)) / nsplit);
  const int *list = sites + (int64_t)c * per_colour;
  int aj[kHPEpt];
  double2 acc[kHPEpt];
#pragma unroll
  for (int j = 0; j < kHPEpt; ++j) {
    const int e = e0 + j;
    aj[j] = e < L ? e / k : -1;
    acc[j] = make_double2(0.0, 0.0);
  }
  const bool live = e0 < L;  // all kHPEpt elements lie in the run when the first does
  const bool uni = live && aj[0] == aj[kHPEpt - 1];
  for (int t0 = s0; t0 < s1; t0 += kHPTile) {
    const int nt = (s1 - t0) < kHPTile ? (s1 - t0) : kHPTile;
    __syncthreads();
    for (int tt = threadIdx.x; tt < nt; tt += T) {
      // the 12 codes of one site: one Philox block of 128 dofs, or two if the site straddles
      const int x = list[t0 + tt];
      tile_sites[tt] = x;
      const int64_t i0 = (int64_t)x * 12;
      uint64_t w[4];
      int64_t blk = i0 >> 7;
      philox4x64_10((uint64_t)blk, (uint64_t)run, 0ull, 0ull, seed, 0ull, w);
      int raw[12];
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        const int64_t i = i0 + a;
        if ((i >> 7) != blk) {
          blk = i >> 7;
          philox4x64_10((uint64_t)blk, (uint64_t)run, 0ull, 0ull, seed, 0ull, w);
        }
        raw[a] = (int)((w[(i >> 5) & 3] >> (2 * (i & 31))) & 3ull);
      }
#pragma unroll
      for (int a = 0; a < 12; ++a) codes[tt * 12 + a] = (unsigned char)((raw[xf.src[a]] + xf.add[a]) & 3);
    }
    __syncthreads();
    AC tacc[kHPEpt];  // this tile's sums
#pragma unroll
    for (int j = 0; j < kHPEpt; ++j) tacc[j].zero();
    auto add = [&](int j, const VC vr, int code) {
      const auto vv = hp_widen(vr);
      // conj(v) * i^code: 0 -> (vx, -vy), 1 -> (vy, vx), 2 -> (-vx, vy), 3 -> (-vy, -vx)
      auto re = (code & 1) ? vv.y : vv.x;
      auto im = (code & 1) ? vv.x : -vv.y;
      if (code & 2) {
        re = -re;
        im = -im;
      }
      tacc[j].add(re, im);
    };
    constexpr int SF = 4;  // sites in flight
    typedef typename FourOf<VC>::type F4;
    // the kHPEpt elements of a thread share one dof type unless they straddle a multiple of k
    // (never when k is a multiple of 4): then one code per site serves all of them
    auto site = [&](const F4 &f, const unsigned char *cs) {
      if (!std::is_same<VC, double2>::value && uni) {  // (FP64 V keeps one path: its registers are full)
        const int c0 = cs[aj[0]];
#pragma unroll
        for (int j = 0; j < kHPEpt; ++j) add(j, hp_elem<VC>(f, j), c0);
      } else {
#pragma unroll
        for (int j = 0; j < kHPEpt; ++j) add(j, hp_elem<VC>(f, j), cs[aj[j]]);
      }
    };
    int u = 0;
    if (live) {
      for (; u + SF - 1 < nt; u += SF) {
        F4 f[SF];
#pragma unroll
        for (int q = 0; q < SF; ++q) f[q] = hp_load4<VC>(Vd + (int64_t)tile_sites[u + q] * L + e0);
#pragma unroll
        for (int q = 0; q < SF; ++q) site(f[q], codes + (u + q) * 12);
      }
      for (; u < nt; ++u) site(hp_load4<VC>(Vd + (int64_t)tile_sites[u] * L + e0), codes + u * 12);
    }
#pragma unroll
    for (int j = 0; j < kHPEpt; ++j) tacc[j].flush(acc[j]);
  }
  double2 *out = partial + ((int64_t)split * nc + c) * L;
#pragma unroll
  for (int j = 0; j < kHPEpt; ++j)
    if (aj[j] >= 0) out[e0 + j] = acc[j];
}

// Sum over splits (fixed order) and over the dof types of a group.  With
// dilution W[(c*12 + a)*k + m] keeps every dof type; without it
// W[(c*2 + h)*k + m] holds the upper (h = 0, a < 6) and lower (h = 1) spin
// halves, the only combinations the columns need.  Loads of one split are
// independent (unrolled over the group's dof types).
__global__ void k_hp_reduce(const double2 *__restrict__ partial, int nc, int nsplit, int k, int dilute12,
                            double2 *__restrict__ W) {
  const int64_t n12 = (int64_t)nc * 12 * k;
  const int groups = dilute12 ? 12 : 2;
  const int per = dilute12 ? 1 : 6;
  const int64_t n = (int64_t)nc * groups * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % k);
    const int cg = (int)(e / k);
    const int c = cg / groups, h = cg % groups;
    const double2 *base = partial + ((int64_t)c * 12 + h * per) * k + m;
    double2 s = make_double2(0.0, 0.0);
    if (per == 6) {
      for (int sp = 0; sp < nsplit; ++sp) {
        const double2 *q = base + (int64_t)sp * n12;
        double2 v[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) v[a] = q[(int64_t)a * k];
#pragma unroll
        for (int a = 0; a < 6; ++a) s = cadd(s, v[a]);
      }
    } else {
      int sp = 0;
      for (; sp + 3 < nsplit; sp += 4) {
        const double2 v0 = base[(int64_t)sp * n12], v1 = base[(int64_t)(sp + 1) * n12];
        const double2 v2 = base[(int64_t)(sp + 2) * n12], v3 = base[(int64_t)(sp + 3) * n12];
        s = cadd(s, v0);
        s = cadd(s, v1);
        s = cadd(s, v2);
        s = cadd(s, v3);
      }
      for (; sp < nsplit; ++sp) s = cadd(s, base[(int64_t)sp * n12]);
    }
    W[e] = s;
  }
}

// C (column-major k x 2b) for block columns col < nrhs (probing index q0 + col):
// C[col] = sum_c H[c, j] sum_{a in set} W_a[c],  C[b + col] = same with g5(a)
__global__ void k_hp_finish(const double2 *__restrict__ W, int nc, int k, int b, int nrhs, int64_t q0, int dilute12,
                            CodeXform xf, double2 *__restrict__ C) {
  const int64_t n = (int64_t)k * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % k);
    const int col = (int)(e / k);
    double2 cz = make_double2(0.0, 0.0), cg = make_double2(0.0, 0.0);
    if (col < nrhs) {
      const int64_t q = q0 + col;
      const int64_t j = dilute12 ? q / 12 : q;
      const int asel = dilute12 ? (int)xf.dst[q % 12] : -1;  // the column's dof type after the code transform
      constexpr int U = 8;  // colours in flight
      for (int c0 = 0; c0 < nc; c0 += U) {
        double2 up[U], lo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + u;
          up[u] = lo[u] = make_double2(0.0, 0.0);
          if (c < nc) {
            if (asel >= 0) {
              const double2 w = W[((int64_t)c * 12 + asel) * k + m];
              if (asel < 6) up[u] = w; else lo[u] = w;
            } else {
              up[u] = W[((int64_t)c * 2 + 0) * k + m];
              lo[u] = W[((int64_t)c * 2 + 1) * k + m];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + u;
          if (c < nc) {
            const double h = (__popcll((unsigned long long)(c & j)) & 1) ? -1.0 : 1.0;
            cz = cadd(cz, cscale(cadd(up[u], lo[u]), h));
            cg = cadd(cg, cscale(csub(up[u], lo[u]), h));
          }
        }
      }
    }
    C[(int64_t)col * k + m] = cz;
    C[(int64_t)(b + col) * k + m] = cg;
  }
}

// threads of a partial block: the row chunk 12k / kHPEpt, in whole warps, at most kHPMaxThreads
static int hp_threads(int k) {
  int t = (12 * k + kHPEpt - 1) / kHPEpt;
  t = (t + 31) / 32 * 32;
  return t < kHPMaxThreads ? t : kHPMaxThreads;
}
static int hp_rowchunks(int k) {
  const int per = hp_threads(k) * kHPEpt;
  return (12 * k + per - 1) / per;
}

static int hp_split(int nc, int per_colour, int k, int sms) {
  // about two blocks per SM (at least 16 sites per block, so the split
  // partials stay small next to the V stream)
  const int ny = hp_rowchunks(k);
  int ns = (2 * sms + nc * ny - 1) / (nc * ny);
  const int max_by_sites = per_colour / 16 > 0 ? per_colour / 16 : 1;
  if (ns > max_by_sites) ns = max_by_sites;
  if (ns < 1) ns = 1;
  return ns;
}

size_t defl_hp_scratch_bytes(int64_t V, int k, int b, int ncolors, int sms) {
  const int per = (int)(V / ncolors);
  const int ns = hp_split(ncolors, per, k, sms);
  const size_t part = (size_t)ns * ncolors * 12 * k * sizeof(double2);
  const size_t W = (size_t)ncolors * 12 * k * sizeof(double2);
  const size_t C = (size_t)k * 2 * b * sizeof(double2);
  return ((part + 255) / 256 + (W + 255) / 256 + (C + 255) / 256 + 2) * 256;
}

int defl_project_hp(const dtr_defl_s *D, const int *sites_by_colour, int ncolors, uint64_t seed, int64_t run,
                    int64_t q0, int nrhs, int dilute12, int b, double2 *d_dev, double2 *terms_dev, void *work,
                    size_t work_bytes, int sms, cudaStream_t st, const CodeXform *xf, double2 **C_out,
                    bool reuse_w) {
  const CodeXform x = xf ? *xf : code_xform_identity();
  const int64_t V = D->lat.V;
  const int k = D->k;
  if (work_bytes < defl_hp_scratch_bytes(V, k, b, ncolors, sms)) return fail(DTR_ENOMEM, "HP deflation scratch too small");
  const int per = (int)(V / ncolors);
  const int ns = hp_split(ncolors, per, k, sms);
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double2 *partial = (double2 *)w;
  w += (((size_t)ns * ncolors * 12 * k * sizeof(double2) + 255) / 256) * 256;
  double2 *W = (double2 *)w;
  w += (((size_t)ncolors * 12 * k * sizeof(double2) + 255) / 256) * 256;
  double2 *C = (double2 *)w;
  dim3 grid(ncolors * ns, hp_rowchunks(k));
  const int nthr = hp_threads(k);
  if (reuse_w) {
    // W of this run is already in the workspace
  } else if (D->prec == DTR_F64)
    k_hp_partial<double2><<<grid, nthr, 0, st>>>((const double2 *)D->V, sites_by_colour, per, ncolors, ns, k,
                                                  seed, run, x, partial);
  else if (D->prec == DTR_F32)
    k_hp_partial<float2><<<grid, nthr, 0, st>>>((const float2 *)D->V, sites_by_colour, per, ncolors, ns, k, seed,
                                                 run, x, partial);
  else
    k_hp_partial<bfc2><<<grid, nthr, 0, st>>>((const bfc2 *)D->V, sites_by_colour, per, ncolors, ns, k, seed, run,
                                               x, partial);
  if (!reuse_w) {
    count_launches(1);
    const int64_t nw = (int64_t)ncolors * 12 * k;
    k_hp_reduce<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(partial, ncolors, ns, k, dilute12, W);
    count_launches(1);
  }
  const int64_t nk = (int64_t)k * b;
  k_hp_finish<<<(unsigned)((nk + 127) / 128), 128, 0, st>>>(W, ncolors, k, b, nrhs, q0, dilute12, x, C);
  count_launches(1);
  if (d_dev) launch_defl_d(D, C, b, d_dev, terms_dev, st);
  DTR_LAUNCH_CHECK("HP deflation projection");
  if (C_out) *C_out = C;
  return DTR_OK;
}

}  // namespace dtr
