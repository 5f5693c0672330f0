// Deflation projection specialised to hierarchical-probing blocks (Section 5.2,
// Algorithm 1 line 8 with z = z0 .* z_h).
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
#include "deflate.cuh"
#include "philox.cuh"

namespace dtr {

constexpr int kHPThreads = 128;
constexpr int kHPTile = 64;  // sites per shared-memory code tile

// partial[((split*nc + c)*12 + a)*k + m]
template <typename VC>
__global__ void __launch_bounds__(kHPThreads)
    k_hp_partial(const VC *__restrict__ Vd, const int *__restrict__ sites, int per_colour, int nc, int nsplit, int k,
                 uint64_t seed, int64_t run, double2 *__restrict__ partial) {
  __shared__ unsigned char codes[kHPTile * 12];
  __shared__ int tile_sites[kHPTile];
  const int c = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  const int m = blockIdx.y * kHPThreads + threadIdx.x;
  const int s0 = (int)(((int64_t)per_colour * split) / nsplit);
  const int s1 = (int)(((int64_t)per_colour * (split + 1)) / nsplit);
  const int *list = sites + (int64_t)c * per_colour;
  double2 acc[12];
#pragma unroll
  for (int a = 0; a < 12; ++a) acc[a] = make_double2(0.0, 0.0);
  for (int t0 = s0; t0 < s1; t0 += kHPTile) {
    const int nt = (s1 - t0) < kHPTile ? (s1 - t0) : kHPTile;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt; idx += blockDim.x) tile_sites[idx] = list[t0 + idx];
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * 12; idx += blockDim.x)
      codes[idx] = (unsigned char)z4_code(seed, run, (int64_t)tile_sites[idx / 12] * 12 + (idx % 12));
    __syncthreads();
    if (m < k) {
      for (int u = 0; u < nt; ++u) {
        const int64_t i0 = (int64_t)tile_sites[u] * 12;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
          const VC vv = Vd[(i0 + a) * k + m];
          const int code = codes[u * 12 + a];
          const double vx = vv.x, vy = vv.y;
          // conj(v) * i^code: 0 -> (vx, -vy), 1 -> (vy, vx), 2 -> (-vx, vy), 3 -> (-vy, -vx)
          double re = (code & 1) ? vy : vx;
          double im = (code & 1) ? vx : -vy;
          if (code & 2) {
            re = -re;
            im = -im;
          }
          acc[a].x += re;
          acc[a].y += im;
        }
      }
    }
  }
  if (m < k) {
#pragma unroll
    for (int a = 0; a < 12; ++a) partial[(((int64_t)split * nc + c) * 12 + a) * k + m] = acc[a];
  }
}

// Sum over splits (fixed order).  With dilution W[(c*12 + a)*k + m] keeps every
// dof type; without it W[(c*2 + h)*k + m] holds the upper (h = 0, a < 6) and
// lower (h = 1) spin halves, the only combinations the columns need.
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
    double2 s = make_double2(0.0, 0.0);
    for (int sp = 0; sp < nsplit; ++sp)
      for (int a = h * per; a < (h + 1) * per; ++a) s = cadd(s, partial[(int64_t)sp * n12 + ((int64_t)c * 12 + a) * k + m]);
    W[e] = s;
  }
}

// C (column-major k x 2b) for block columns col < nrhs (probing index q0 + col):
// C[col] = sum_c H[c, j] sum_{a in set} W_a[c],  C[b + col] = same with g5(a)
__global__ void k_hp_finish(const double2 *__restrict__ W, int nc, int k, int b, int nrhs, int64_t q0, int dilute12,
                            double2 *__restrict__ C) {
  const int64_t n = (int64_t)k * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % k);
    const int col = (int)(e / k);
    double2 cz = make_double2(0.0, 0.0), cg = make_double2(0.0, 0.0);
    if (col < nrhs) {
      const int64_t q = q0 + col;
      const int64_t j = dilute12 ? q / 12 : q;
      const int asel = dilute12 ? (int)(q % 12) : -1;
      for (int c = 0; c < nc; ++c) {
        const double h = (__popcll((unsigned long long)(c & j)) & 1) ? -1.0 : 1.0;
        double2 up = make_double2(0.0, 0.0), lo = make_double2(0.0, 0.0);
        if (asel >= 0) {
          const double2 w = W[((int64_t)c * 12 + asel) * k + m];
          if (asel < 6) up = w; else lo = w;
        } else {
          up = W[((int64_t)c * 2 + 0) * k + m];
          lo = W[((int64_t)c * 2 + 1) * k + m];
        }
        cz = cadd(cz, cscale(cadd(up, lo), h));
        cg = cadd(cg, cscale(csub(up, lo), h));
      }
    }
    C[(int64_t)col * k + m] = cz;
    C[(int64_t)(b + col) * k + m] = cg;
  }
}

static int hp_split(int nc, int per_colour, int k, int sms) {
  // about two blocks per SM; more splits make the split reduction latency-bound
  const int mt = (k + kHPThreads - 1) / kHPThreads;
  int ns = (2 * sms + nc * mt - 1) / (nc * mt);
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
                    size_t work_bytes, int sms, cudaStream_t st) {
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
  dim3 grid(ncolors * ns, (k + kHPThreads - 1) / kHPThreads);
  if (D->prec == DTR_F64)
    k_hp_partial<double2><<<grid, kHPThreads, 0, st>>>((const double2 *)D->V, sites_by_colour, per, ncolors, ns, k,
                                                        seed, run, partial);
  else
    k_hp_partial<float2><<<grid, kHPThreads, 0, st>>>((const float2 *)D->V, sites_by_colour, per, ncolors, ns, k, seed,
                                                       run, partial);
  count_launches(1);
  const int64_t nw = (int64_t)ncolors * 12 * k;
  k_hp_reduce<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(partial, ncolors, ns, k, dilute12, W);
  count_launches(1);
  const int64_t nk = (int64_t)k * b;
  k_hp_finish<<<(unsigned)((nk + 127) / 128), 128, 0, st>>>(W, ncolors, k, b, nrhs, q0, dilute12, C);
  count_launches(1);
  launch_defl_d(C, D->inv_lambda, k, b, d_dev, terms_dev, st);
  DTR_LAUNCH_CHECK("HP deflation projection");
  return DTR_OK;
}

}  // namespace dtr
