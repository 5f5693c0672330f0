// Deflation projection (Section 5.2; Algorithm 1: the deflated part T_D and the deflation term).
//
// With V the right singular vectors stored as eigenvectors of Q = g5 A
// (signed eigenvalues lambda), the paper's quadrature z^H V L^-1 V^H (A^H z),
// L = Sigma^2, equals z^H V diag(1/lambda) V^H g5 z because V^H A^H =
// diag(lambda) V^H g5.  The tall-skinny contraction C = V^H [Z, g5 Z] is
// computed as two accumulators per (m, j): the upper-spin part P and the
// lower-spin part Q of V^H Z, so that V^H Z = P + Q and V^H g5 Z = P - Q.
//
// Layouts: V row-major [dof][k] (FP64 or FP32); Z internal [site][12][b] FP64.
// Partial sums per site chunk go to scratch and are reduced over chunks in a
// fixed order, so results are bit-reproducible.
#include "dtr_internal.cuh"
#include "deflate.cuh"

namespace dtr {

constexpr int kDeflBlock = 256;
constexpr int kMPT = 4;  // vectors m per thread per tile

template <typename VC>
__global__ void __launch_bounds__(kDeflBlock)
    k_defl_partial(const VC *__restrict__ Vd, const double2 *__restrict__ Z, int k, int b, int logb, int nsites,
                   int nchunks, double2 *__restrict__ partial) {
  const int G = kDeflBlock >> logb;  // m-groups per block
  const int tile = G * kMPT;
  const int chunk = blockIdx.x % nchunks;
  const int mt = blockIdx.x / nchunks;
  const int j = threadIdx.x & (b - 1);
  const int grp = threadIdx.x >> logb;
  const int s0 = (int)(((int64_t)nsites * chunk) / nchunks);
  const int s1 = (int)(((int64_t)nsites * (chunk + 1)) / nchunks);
  int m[kMPT];
  bool ok[kMPT];
#pragma unroll
  for (int q = 0; q < kMPT; ++q) {
    m[q] = mt * tile + grp + q * G;
    ok[q] = m[q] < k;
  }
  double2 P[kMPT], Q[kMPT];
#pragma unroll
  for (int q = 0; q < kMPT; ++q) P[q] = Q[q] = make_double2(0.0, 0.0);
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const int64_t i = (int64_t)s * 12 + c;
      const double2 z = Z[i * b + j];
#pragma unroll
      for (int q = 0; q < kMPT; ++q) {
        if (!ok[q]) continue;
        const double2 vv = vload(Vd[i * k + m[q]]);
        const double vx = vv.x, vy = vv.y;
        // conj(v) * z
        const double re = vx * z.x + vy * z.y, im = vx * z.y - vy * z.x;
        if (c < 6) {
          P[q].x += re;
          P[q].y += im;
        } else {
          Q[q].x += re;
          Q[q].y += im;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kMPT; ++q) {
    if (!ok[q]) continue;
    const int64_t base = (((int64_t)chunk * k + m[q]) * 2) * b + j;
    partial[base] = P[q];
    partial[base + b] = Q[q];
  }
}

// C (column-major k x 2b): C[m + k*j] = P + Q, C[m + k*(b+j)] = P - Q
__global__ void k_defl_reduce(const double2 *__restrict__ partial, int k, int b, int nchunks, double2 *__restrict__ C) {
  const int64_t n = (int64_t)k * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    const int m = (int)(e / b);
    double2 P = make_double2(0.0, 0.0), Q = make_double2(0.0, 0.0);
    for (int ch = 0; ch < nchunks; ++ch) {
      const int64_t base = (((int64_t)ch * k + m) * 2) * b + j;
      P = cadd(P, partial[base]);
      Q = cadd(Q, partial[base + b]);
    }
    C[(int64_t)j * k + m] = cadd(P, Q);
    C[(int64_t)(b + j) * k + m] = csub(P, Q);
  }
}

// d_j = sum_m conj(C[m, j]) C[m, b+j] / lambda_m ; optional per-m terms.
// One block per column; fixed-order block tree, so the result is reproducible.
__global__ void k_defl_d(const double2 *__restrict__ C, const double2 *__restrict__ Cr,
                         const double *__restrict__ inv_lambda, int k, int b, double2 *__restrict__ d,
                         double2 *__restrict__ terms) {
  __shared__ double2 sh[128];
  const int j = blockIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    const double2 a = C[(int64_t)j * k + m], g = Cr[(int64_t)(b + j) * k + m];
    const double2 t = cscale(cjmul(a, g), inv_lambda[m]);
    if (terms) terms[(int64_t)j * k + m] = t;
    acc = cadd(acc, t);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int stride = 64; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + stride]);
    __syncthreads();
  }
  if (threadIdx.x == 0) d[j] = sh[0];
}

// Galerkin form: y = G^-1 g_j (Cr[:, b + j]) per column, d_j = c_j^H y (fixed-order tree)
__global__ void k_defl_d_gram(const double2 *__restrict__ C, const double2 *__restrict__ Cr,
                              const double2 *__restrict__ Ginv, int k, int b, double2 *__restrict__ d,
                              double2 *__restrict__ terms) {
  __shared__ double2 sh[128];
  const int j = blockIdx.x;
  const double2 *g = Cr + (int64_t)(b + j) * k;
  double2 acc = make_double2(0.0, 0.0);
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    double2 y = make_double2(0.0, 0.0);
    for (int n = 0; n < k; ++n) y = caxpy(Ginv[(int64_t)m * k + n], g[n], y);
    const double2 t = cjmul(C[(int64_t)j * k + m], y);
    if (terms) terms[(int64_t)j * k + m] = t;
    acc = cadd(acc, t);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int stride = 64; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + stride]);
    __syncthreads();
  }
  if (threadIdx.x == 0) d[j] = sh[0];
}

// expansion weights W[j][m] = (Lambda^-1 g_j)_m or (G^-1 g_j)_m, g_j = C[:, b + j]
__global__ void k_defl_weights(const double2 *__restrict__ C, const double *__restrict__ inv_lambda,
                               const double2 *__restrict__ Ginv, int k, int b, double2 *__restrict__ W) {
  const int64_t n = (int64_t)k * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % k), j = (int)(e / k);
    const double2 *g = C + (int64_t)(b + j) * k;
    double2 y = make_double2(0.0, 0.0);
    if (Ginv) {
      for (int q = 0; q < k; ++q) y = caxpy(Ginv[(int64_t)m * k + q], g[q], y);
    } else {
      y = cscale(g[m], inv_lambda[m]);
    }
    W[e] = y;
  }
}

void launch_defl_d(const dtr_defl_s *D, const double2 *C, int b, double2 *d, double2 *terms, cudaStream_t st) {
  if (D->Ginv)
    k_defl_d_gram<<<b, 128, 0, st>>>(C, C, D->Ginv, D->k, b, d, terms);
  else
    k_defl_d<<<b, 128, 0, st>>>(C, C, D->inv_lambda, D->k, b, d, terms);
  count_launches(1);
}

void launch_defl_d2(const dtr_defl_s *D, const double2 *Cl, const double2 *Cr, int b, double2 *d, cudaStream_t st) {
  if (D->Ginv)
    k_defl_d_gram<<<b, 128, 0, st>>>(Cl, Cr, D->Ginv, D->k, b, d, nullptr);
  else
    k_defl_d<<<b, 128, 0, st>>>(Cl, Cr, D->inv_lambda, D->k, b, d, nullptr);
  count_launches(1);
}

// GZ[(x, t, c), j] = i^-phase[s] Z[(x, s, c), j] with perm[s] = t
__global__ void k_gamma_h(GammaMono g, const double2 *__restrict__ Z, double2 *__restrict__ GZ, int64_t n, int b) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    const int64_t xa = e / b;
    const int a = (int)(xa % 12);
    const int64_t x = xa / 12;
    const int s = a / 3, c = a % 3;
    const double2 v = Z[(x * 12 + s * 3 + c) * b + j];
    const int q = (4 - g.phase[s]) & 3;
    double2 w = v;
    if (q == 1) w = make_double2(-v.y, v.x);
    if (q == 2) w = make_double2(-v.x, -v.y);
    if (q == 3) w = make_double2(v.y, -v.x);
    GZ[(x * 12 + g.perm[s] * 3 + c) * b + j] = w;
  }
}

void launch_gamma_h(const GammaMono &g, const double2 *Z, double2 *GZ, int64_t V, int b, cudaStream_t st) {
  const int64_t n = V * 12 * b;
  unsigned grid = (unsigned)((n + 255) / 256);
  if (grid > 65535u * 8) grid = 65535u * 8;
  k_gamma_h<<<grid, 256, 0, st>>>(g, Z, GZ, n, b);
  count_launches(1);
}

// per (chunk of sites, Gamma, m): sum over the chunk's sites and dofs of
// conj(v[x, s, c]) g5(s) i^phase[s] v[x, perm[s], c]   (FP64)
template <typename VC>
__global__ void k_defl_tdg_partial(const VC *__restrict__ Vd, int k, int64_t nsite, int nchunks, GammaSet gs,
                                   double2 *__restrict__ part) {
  const int chunk = blockIdx.x;
  const int64_t x0 = (nsite * chunk) / nchunks, x1 = (nsite * (chunk + 1)) / nchunks;
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    double2 acc[16];
    for (int q = 0; q < gs.n; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t x = x0; x < x1; ++x) {
      double2 v[12];
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        v[a] = vload(Vd[(x * 12 + a) * k + m]);
      }
      for (int q = 0; q < gs.n; ++q) {
        const GammaMono g = gs.g[q];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const double sgn = sp < 2 ? 1.0 : -1.0;
          const int ph = g.phase[sp];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double2 w = v[g.perm[sp] * 3 + c];  // i^ph w
            if (ph == 1) w = make_double2(-w.y, w.x);
            if (ph == 2) w = make_double2(-w.x, -w.y);
            if (ph == 3) w = make_double2(w.y, -w.x);
            const double2 u = v[sp * 3 + c];
            acc[q].x += sgn * (u.x * w.x + u.y * w.y);
            acc[q].y += sgn * (u.x * w.y - u.y * w.x);
          }
        }
      }
    }
    for (int q = 0; q < gs.n; ++q) part[((int64_t)chunk * 16 + q) * k + m] = acc[q];
  }
}

__global__ void k_defl_tdg_reduce(const double2 *__restrict__ part, const double *__restrict__ inv_lambda, int k,
                                  int nchunks, int ng, double2 *__restrict__ td) {
  // one thread per Gamma, fixed order: deterministic
  const int q = threadIdx.x;
  if (blockIdx.x != 0 || q >= ng) return;
  double2 t = make_double2(0.0, 0.0);
  for (int m = 0; m < k; ++m) {
    double2 s = make_double2(0.0, 0.0);
    for (int ch = 0; ch < nchunks; ++ch) s = cadd(s, part[((int64_t)ch * 16 + q) * k + m]);
    t = cadd(t, cscale(s, inv_lambda[m]));
  }
  td[q] = t;
}

// x0 (internal [site][12][b]) = V diag(1/lambda) C[:, b:2b]
template <typename VC>
__global__ void k_defl_expand(const VC *__restrict__ Vd, const double2 *__restrict__ W, int k, int b, int64_t N,
                              double2 *__restrict__ x) {
  const int64_t n = N * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    const int64_t i = e / b;
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < k; ++m) {
      const double2 vv = vload(Vd[i * k + m]);
      acc = caxpy(vv, W[(int64_t)j * k + m], acc);
    }
    x[e] = acc;
  }
}

// T_D partials: part[chunk][m] = sum over the chunk's sites x and dof types a
// of g5(a) |V[12x + a][m]|^2.  Thread m of block (chunk, m-tile) walks the
// chunk's sites; a site's twelve rows are independent loads (12 in flight per
// thread), consecutive threads read consecutive m (coalesced).
constexpr int kTdThreads = 256;
template <typename VC>
__global__ void __launch_bounds__(kTdThreads)
    k_defl_td_partial(const VC *__restrict__ Vd, int k, int64_t nsite, int nchunks, double *__restrict__ part) {
  const int chunk = blockIdx.x;
  const int m = blockIdx.y * kTdThreads + threadIdx.x;
  if (m >= k) return;
  const int64_t x0 = (nsite * chunk) / nchunks, x1 = (nsite * (chunk + 1)) / nchunks;
  double acc = 0.0;
  for (int64_t x = x0; x < x1; ++x) {
    const VC *row = Vd + x * 12 * k + m;
    VC v[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) v[a] = __ldcs(row + (int64_t)a * k);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const double2 vv = vload(v[a]);
      const double a2 = vv.x * vv.x + vv.y * vv.y;
      acc += a < 6 ? a2 : -a2;
    }
  }
  part[(int64_t)chunk * k + m] = acc;
}

// T_D = sum_m (sum_chunk part[chunk][m]) / lambda_m: thread t sums m = t, t + T, ...
// (chunks in order), then a fixed shared-memory tree over the threads.
// Deterministic for a given (k, nchunks).
__global__ void __launch_bounds__(kTdThreads)
    k_defl_td_reduce(const double *__restrict__ part, const double *__restrict__ inv_lambda, int k, int nchunks,
                     double *__restrict__ td) {
  __shared__ double sh[kTdThreads];
  double t = 0.0;
  for (int m = threadIdx.x; m < k; m += kTdThreads) {
    double s = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) s += part[(int64_t)ch * k + m];
    t += s * inv_lambda[m];
  }
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int w = kTdThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *td = sh[0];
}

static int log2i(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

static int defl_chunks(int64_t V, int k, int b, int sms) {
  const int G = kDeflBlock / b;
  const int tiles = (k + G * kMPT - 1) / (G * kMPT);
  int64_t want = (2LL * sms + tiles - 1) / tiles;
  if (want > V) want = V;
  if (want < 1) want = 1;
  return (int)want;
}

size_t defl_scratch_bytes(int64_t V, int k, int b, int sms) {
  const int nch = defl_chunks(V, k, b, sms);
  size_t part = (size_t)nch * k * 2 * b * sizeof(double2);
  const size_t tc = defl_tc_scratch_bytes(V, k, b, sms);  // the tensor-core partials share this region
  if (tc > part) part = tc;
  const size_t C = (size_t)k * 2 * b * sizeof(double2);
  const size_t W = (size_t)k * b * sizeof(double2);
  const size_t d = 64 * sizeof(double2);
  return ((part + 255) / 256 + (C + 255) / 256 + (W + 255) / 256 + (d + 255) / 256 + 5) * 256;
}

// layout of the scratch: [status word, 256 B][partials][C][x0 weights]
int *defl_error_word(void *work) { return (int *)(((uintptr_t)work + 255) & ~(uintptr_t)255); }

int defl_project_internal(const dtr_defl_s *D, const double2 *Z, int b, double2 *d_dev, double2 *terms_dev,
                          double2 *x0_internal, double2 **C_out, void *work, size_t work_bytes, int sms,
                          cudaStream_t st, int z4, const unsigned char *Zc) {
  const int64_t V = D->lat.V;
  const int k = D->k;
  if (work_bytes < defl_scratch_bytes(V, k, b, sms)) return fail(DTR_ENOMEM, "deflation workspace too small");
  const int nch = defl_chunks(V, k, b, sms);
  const int G = kDeflBlock / b;
  const int tiles = (k + G * kMPT - 1) / (G * kMPT);
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  int *err = (int *)w;
  w += 256;
  double2 *partial = (double2 *)w;
  size_t partbytes = (size_t)nch * k * 2 * b * sizeof(double2);
  const size_t tcbytes = defl_tc_scratch_bytes(V, k, b, sms);
  if (tcbytes > partbytes) partbytes = tcbytes;
  w += ((partbytes + 255) / 256) * 256;
  double2 *C = (double2 *)w;
  w += (((size_t)k * 2 * b * sizeof(double2) + 255) / 256) * 256;
  double2 *Wx = (double2 *)w;
  w += (((size_t)k * b * sizeof(double2) + 255) / 256) * 256;
  const int logb = log2i(b);
  const int64_t nkb = (int64_t)k * b;
  if (z4 && defl_tc_enabled(D, b)) {
    DTR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    int rc = defl_contract_tc(D, Z, b, C, partial, partbytes, err, sms, st, Zc);
    if (rc) return rc;
  } else {
  if (D->prec == DTR_F64)
    k_defl_partial<double2><<<nch * tiles, kDeflBlock, 0, st>>>((const double2 *)D->V, Z, k, b, logb, (int)V, nch,
                                                                partial);
  else if (D->prec == DTR_F32)
    k_defl_partial<float2><<<nch * tiles, kDeflBlock, 0, st>>>((const float2 *)D->V, Z, k, b, logb, (int)V, nch,
                                                               partial);
  else
    k_defl_partial<bfc2><<<nch * tiles, kDeflBlock, 0, st>>>((const bfc2 *)D->V, Z, k, b, logb, (int)V, nch,
                                                             partial);
  count_launches(1);
  k_defl_reduce<<<(unsigned)((nkb + 255) / 256), 256, 0, st>>>(partial, k, b, nch, C); count_launches(1);
  }
  if (d_dev) launch_defl_d(D, C, b, d_dev, terms_dev, st);
  if (x0_internal) {
    k_defl_weights<<<(unsigned)((nkb + 255) / 256), 256, 0, st>>>(C, D->inv_lambda, D->Ginv, k, b, Wx);
    count_launches(1);
    const int64_t n = V * 12 * b;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (grid > 65535u * 8) grid = 65535u * 8;
    if (D->prec == DTR_F64)
      k_defl_expand<double2><<<grid, 256, 0, st>>>((const double2 *)D->V, Wx, k, b, V * 12, x0_internal);
    else if (D->prec == DTR_F32)
      k_defl_expand<float2><<<grid, 256, 0, st>>>((const float2 *)D->V, Wx, k, b, V * 12, x0_internal);
    else
      k_defl_expand<bfc2><<<grid, 256, 0, st>>>((const bfc2 *)D->V, Wx, k, b, V * 12, x0_internal);
    count_launches(1);
  }
  DTR_LAUNCH_CHECK("deflation projection");
  if (C_out) *C_out = C;
  return DTR_OK;
}

int defl_trace_TD(dtr_defl_s *D, cudaStream_t st) {
  const int64_t nsite = D->lat.V;
  const int k = D->k;
  const int mt = (k + kTdThreads - 1) / kTdThreads;
  int64_t nch64 = (8LL * device_sms() + mt - 1) / mt;  // about eight blocks per SM
  if (nch64 > nsite) nch64 = nsite;
  const int nch = (int)nch64;
  double *part = nullptr, *td = nullptr;
  DTR_CUDA(cudaMalloc((void **)&part, (size_t)nch * k * sizeof(double) + 256));
  td = (double *)((char *)part + (((size_t)nch * k * sizeof(double) + 127) / 128) * 128);
  const dim3 grid(nch, mt);
  if (D->prec == DTR_F64)
    k_defl_td_partial<double2><<<grid, kTdThreads, 0, st>>>((const double2 *)D->V, k, nsite, nch, part);
  else if (D->prec == DTR_F32)
    k_defl_td_partial<float2><<<grid, kTdThreads, 0, st>>>((const float2 *)D->V, k, nsite, nch, part);
  else
    k_defl_td_partial<bfc2><<<grid, kTdThreads, 0, st>>>((const bfc2 *)D->V, k, nsite, nch, part);
  count_launches(1);
  k_defl_td_reduce<<<1, kTdThreads, 0, st>>>(part, D->inv_lambda, k, nch, td); count_launches(1);
  cudaError_t e = cudaGetLastError();
  double h = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, td, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "T_D reduction");
  D->td[0] = h;
  D->td[1] = 0.0;
  return DTR_OK;
}

int defl_trace_TD_gamma(dtr_defl_s *D, unsigned want, cudaStream_t st) {
  GammaSet gs;
  gs.n = 0;
  int ids[16];
  for (int n = 0; n < 16; ++n)
    if (((want >> n) & 1u) && !((D->tdg_ok >> n) & 1u)) {
      if (!gamma_monomial(n, &gs.g[gs.n])) return fail(DTR_EINVAL, "Gamma table is not monomial");
      ids[gs.n++] = n;
    }
  if (gs.n == 0) return DTR_OK;
  if (D->Ginv) {
    double2 h[16];
    int rc = defl_tdg_gram(D, gs, h, st);
    if (rc) return rc;
    for (int q = 0; q < gs.n; ++q) {
      D->tdg[ids[q]][0] = h[q].x;
      D->tdg[ids[q]][1] = h[q].y;
      D->tdg_ok |= 1u << ids[q];
    }
    return DTR_OK;
  }
  const int64_t nsite = D->lat.V;
  const int k = D->k;
  int nch = 4 * device_sms();
  if (nch > nsite) nch = (int)nsite;
  double2 *part = nullptr, *td = nullptr;
  const size_t pbytes = (((size_t)nch * 16 * k * sizeof(double2) + 255) / 256) * 256;
  DTR_CUDA(cudaMalloc((void **)&part, pbytes + 16 * sizeof(double2)));
  td = (double2 *)((char *)part + pbytes);
  if (D->prec == DTR_F64)
    k_defl_tdg_partial<double2><<<nch, 128, 0, st>>>((const double2 *)D->V, k, nsite, nch, gs, part);
  else if (D->prec == DTR_F32)
    k_defl_tdg_partial<float2><<<nch, 128, 0, st>>>((const float2 *)D->V, k, nsite, nch, gs, part);
  else
    k_defl_tdg_partial<bfc2><<<nch, 128, 0, st>>>((const bfc2 *)D->V, k, nsite, nch, gs, part);
  count_launches(1);
  k_defl_tdg_reduce<<<1, 32, 0, st>>>(part, D->inv_lambda, k, nch, gs.n, td);
  count_launches(1);
  double2 h[16];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, td, sizeof(double2) * gs.n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "T_D of Gamma");
  for (int q = 0; q < gs.n; ++q) {
    D->tdg[ids[q]][0] = h[q].x;
    D->tdg[ids[q]][1] = h[q].y;
    D->tdg_ok |= 1u << ids[q];
  }
  return DTR_OK;
}

}  // namespace dtr
