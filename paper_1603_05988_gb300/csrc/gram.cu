// Galerkin (Gram) correction of the deflation space, in FP64.
//
// The deflated estimator (Algorithm 1) needs an approximation D of A^-1 on the
// deflation space.  With exact orthonormal eigenvectors V of Q = g5 A and
// their eigenvalues, D = V Lambda^-1 V^H g5 (Section 5.2 in the g5 form).  A
// stored V that is inexact (a loose eigensolver) or no longer orthonormal
// (rounded to FP32 or BF16) is better used through the Galerkin form
//     G = V^H g5 A V  (k x k),   D = V G^-1 V^H g5,   T_D = Tr(G^-1 V^H g5 V),
// which reduces to the Lambda form for exact eigenpairs and satisfies
// D A v = v for every v in span(V) whatever the basis.  G and V^H g5 V are
// k x k contractions over all N dofs, accumulated in FP64 from the stored V
// (widened exactly) and from A V computed by the FP64 stencil, 64 columns at a
// time; G is inverted on the host (Gauss-Jordan, partial pivoting, FP64).
#include <cmath>
#include <complex>
#include <vector>

#include "deflate.cuh"

namespace dtr {

// (T r)(s, c) = sign[s] i^phase[s] r(perm[s], c): a monomial spin transform
struct SpinXform {
  signed char perm[4], phase[4], sign[4];
};

static SpinXform xform_g5() {
  SpinXform t;
  for (int s = 0; s < 4; ++s) {
    t.perm[s] = (signed char)s;
    t.phase[s] = 0;
    t.sign[s] = s < 2 ? 1 : -1;
  }
  return t;
}

static SpinXform xform_g5_gamma(const GammaMono &g) {
  SpinXform t;
  for (int s = 0; s < 4; ++s) {
    t.perm[s] = g.perm[s];
    t.phase[s] = g.phase[s];
    t.sign[s] = s < 2 ? 1 : -1;  // g5 acts after Gamma: row s keeps g5(s)
  }
  return t;
}

// M[m][n] partial over a chunk of sites: sum conj(L[i][m]) (T R)[i][n]
// L, R row-major [dof][ld]; 16 x 16 tile of (m, n) per block, blockIdx.z = chunk
template <typename LC, typename RC>
__global__ void __launch_bounds__(256) k_gram_partial(const LC *__restrict__ L, int ldl, int kl,
                                                      const RC *__restrict__ R, int ldr, int kr, int64_t nsite,
                                                      int nchunks, SpinXform T, double2 *__restrict__ part) {
  __shared__ double2 Ls[12][16], Rs[12][16];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 16;
  const int chunk = blockIdx.z;
  const int64_t x0 = (nsite * chunk) / nchunks, x1 = (nsite * (chunk + 1)) / nchunks;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t x = x0; x < x1; ++x) {
    for (int e = threadIdx.x; e < 384; e += 256) {
      if (e < 192) {
        const int a = e >> 4, mm = m0 + (e & 15);
        Ls[a][e & 15] = mm < kl ? vload(L[(x * 12 + a) * ldl + mm]) : make_double2(0.0, 0.0);
      } else {
        const int e2 = e - 192;
        const int a = e2 >> 4, nn = n0 + (e2 & 15);
        const int s = a / 3, c = a % 3;
        double2 v = nn < kr ? vload(R[(x * 12 + T.perm[s] * 3 + c) * ldr + nn]) : make_double2(0.0, 0.0);
        const int ph = T.phase[s];
        if (ph == 1) v = make_double2(-v.y, v.x);
        if (ph == 2) v = make_double2(-v.x, -v.y);
        if (ph == 3) v = make_double2(v.y, -v.x);
        Rs[a][e2 & 15] = cscale(v, (double)T.sign[s]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const double2 l = Ls[a][tx], r = Rs[a][ty];
      acc.x += l.x * r.x + l.y * r.y;
      acc.y += l.x * r.y - l.y * r.x;
    }
    __syncthreads();
  }
  const int m = m0 + tx, n = n0 + ty;
  if (m < kl && n < kr) part[((int64_t)chunk * kl + m) * kr + n] = acc;
}

__global__ void k_gram_reduce(const double2 *__restrict__ part, int kl, int kr, int nchunks, double2 *__restrict__ M) {
  const int64_t n = (int64_t)kl * kr;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int ch = 0; ch < nchunks; ++ch) s = cadd(s, part[(int64_t)ch * n + e]);
    M[e] = s;
  }
}

// columns n0 .. n0+nb-1 of V (row-major [dof][k]) into the RHS-inner layout [site][12][b], FP64
template <typename VC>
__global__ void k_pack_vcols(const VC *__restrict__ V, int k, int n0, int nb, int b, int64_t ndof,
                             double2 *__restrict__ out) {
  const int64_t n = ndof * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    const int64_t i = e / b;
    out[e] = j < nb ? vload(V[i * k + n0 + j]) : make_double2(0.0, 0.0);
  }
}

namespace {

int grid_chunks(int kl, int kr, int64_t nsite) {
  const int tiles = ((kl + 15) / 16) * ((kr + 15) / 16);
  int ch = (4 * device_sms() + tiles - 1) / tiles;
  if (ch > nsite) ch = (int)nsite;
  if (ch < 1) ch = 1;
  return ch;
}

// M (host, kl x kr row-major) = L^H T R over all sites
template <typename LC, typename RC>
int gram_product(const LC *L, int ldl, int kl, const RC *R, int ldr, int kr, int64_t nsite, SpinXform T,
                 double2 *work, std::vector<std::complex<double>> &M, cudaStream_t st) {
  const int ch = grid_chunks(kl, kr, nsite);
  double2 *part = work;
  double2 *out = work + (size_t)ch * kl * kr;
  dim3 grid((kl + 15) / 16, (kr + 15) / 16, ch);
  k_gram_partial<LC, RC><<<grid, 256, 0, st>>>(L, ldl, kl, R, ldr, kr, nsite, ch, T, part);
  count_launches(1);
  const int64_t n = (int64_t)kl * kr;
  k_gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, kl, kr, ch, out);
  count_launches(1);
  M.resize((size_t)n);
  DTR_CUDA(cudaGetLastError());
  DTR_CUDA(cudaMemcpyAsync(M.data(), out, sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  return DTR_OK;
}

template <typename RC>
int gram_product_v(const dtr_defl_s *D, const RC *R, int ldr, int kr, SpinXform T, double2 *work,
                   std::vector<std::complex<double>> &M, cudaStream_t st) {
  const int k = D->k;
  const int64_t nsite = D->lat.V;
  if (D->prec == DTR_F64) return gram_product((const double2 *)D->V, k, k, R, ldr, kr, nsite, T, work, M, st);
  if (D->prec == DTR_F32) return gram_product((const float2 *)D->V, k, k, R, ldr, kr, nsite, T, work, M, st);
  return gram_product((const bfc2 *)D->V, k, k, R, ldr, kr, nsite, T, work, M, st);
}

size_t gram_work_elems(int k, int64_t nsite) {
  const int kb = k < 64 ? k : 64;
  const size_t a = (size_t)grid_chunks(k, k, nsite) * k * k;
  const size_t b = (size_t)grid_chunks(k, kb, nsite) * k * kb;
  return (a > b ? a : b) + (size_t)k * k;
}

// Gauss-Jordan inverse with partial pivoting (FP64 complex); false if singular
bool invert(std::vector<std::complex<double>> &A, int k) {
  std::vector<std::complex<double>> I((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) I[(size_t)i * k + i] = 1.0;
  for (int c = 0; c < k; ++c) {
    int p = c;
    for (int r = c + 1; r < k; ++r)
      if (std::abs(A[(size_t)r * k + c]) > std::abs(A[(size_t)p * k + c])) p = r;
    if (std::abs(A[(size_t)p * k + c]) == 0.0) return false;
    if (p != c)
      for (int j = 0; j < k; ++j) {
        std::swap(A[(size_t)p * k + j], A[(size_t)c * k + j]);
        std::swap(I[(size_t)p * k + j], I[(size_t)c * k + j]);
      }
    const std::complex<double> inv = 1.0 / A[(size_t)c * k + c];
    for (int j = 0; j < k; ++j) {
      A[(size_t)c * k + j] *= inv;
      I[(size_t)c * k + j] *= inv;
    }
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      const std::complex<double> f = A[(size_t)r * k + c];
      if (f == 0.0) continue;
      for (int j = 0; j < k; ++j) {
        A[(size_t)r * k + j] -= f * A[(size_t)c * k + j];
        I[(size_t)r * k + j] -= f * I[(size_t)c * k + j];
      }
    }
  }
  A.swap(I);
  return true;
}

std::complex<double> trace_product(const std::vector<std::complex<double>> &Gi,
                                   const std::vector<std::complex<double>> &M, int k) {
  std::complex<double> t = 0.0;
  for (int m = 0; m < k; ++m)
    for (int n = 0; n < k; ++n) t += Gi[(size_t)m * k + n] * M[(size_t)n * k + m];
  return t;
}

}  // namespace

int defl_gram(dtr_defl_s *D, const dtr_gauge_s *g, double m0, cudaStream_t st) {
  const int k = D->k;
  const int64_t nsite = D->lat.V, ndof = D->lat.N;
  if (g->lat.V != nsite) return fail(DTR_EINVAL, "gauge field of another lattice");
  const Geom geo = geom_of(D->lat);
  const int nbmax = k < 64 ? k : 64;
  const int b = pad_rhs(nbmax);
  const size_t welems = gram_work_elems(k, nsite);
  double2 *buf = nullptr;
  const size_t vbytes = (size_t)ndof * b * sizeof(double2);
  DTR_CUDA(cudaMalloc((void **)&buf, 2 * vbytes + welems * sizeof(double2) + 512));
  double2 *a = buf, *o = (double2 *)((char *)buf + vbytes);
  double2 *work = (double2 *)((char *)buf + 2 * vbytes);
  std::vector<std::complex<double>> G((size_t)k * k), M5, chunk;
  int rc = DTR_OK;
  for (int n0 = 0; n0 < k && rc == DTR_OK; n0 += 64) {
    const int nb = (k - n0) < 64 ? (k - n0) : 64;
    unsigned grid = (unsigned)((ndof * b + 255) / 256);
    if (grid > 65535u * 8) grid = 65535u * 8;
    if (D->prec == DTR_F64)
      k_pack_vcols<double2><<<grid, 256, 0, st>>>((const double2 *)D->V, k, n0, nb, b, ndof, a);
    else if (D->prec == DTR_F32)
      k_pack_vcols<float2><<<grid, 256, 0, st>>>((const float2 *)D->V, k, n0, nb, b, ndof, a);
    else
      k_pack_vcols<bfc2><<<grid, 256, 0, st>>>((const bfc2 *)D->V, k, n0, nb, b, ndof, a);
    count_launches(1);
    launch_dslash<double>(g->U64, a, o, geo, b, m0, 0, st);
    rc = gram_product_v(D, (const double2 *)o, b, nb, xform_g5(), work, chunk, st);  // (k x nb)
    if (rc) break;
    for (int m = 0; m < k; ++m)
      for (int j = 0; j < nb; ++j) G[(size_t)m * k + n0 + j] = chunk[(size_t)m * nb + j];
  }
  if (rc == DTR_OK) {
    if (D->prec == DTR_F64)
      rc = gram_product((const double2 *)D->V, k, k, (const double2 *)D->V, k, k, nsite, xform_g5(), work, M5, st);
    else if (D->prec == DTR_F32)
      rc = gram_product((const float2 *)D->V, k, k, (const float2 *)D->V, k, k, nsite, xform_g5(), work, M5, st);
    else
      rc = gram_product((const bfc2 *)D->V, k, k, (const bfc2 *)D->V, k, k, nsite, xform_g5(), work, M5, st);
  }
  cudaFree(buf);
  if (rc) return rc;
  std::vector<std::complex<double>> Gi = G;
  if (!invert(Gi, k)) return fail(DTR_EINVAL, "Gram matrix V^H g5 A V is singular");
  const std::complex<double> td = trace_product(Gi, M5, k);
  if (!D->Ginv) DTR_CUDA(cudaMalloc((void **)&D->Ginv, sizeof(double2) * k * k));
  DTR_CUDA(cudaMemcpy(D->Ginv, Gi.data(), sizeof(double2) * k * k, cudaMemcpyHostToDevice));
  D->td[0] = td.real();
  D->td[1] = td.imag();
  D->tdg_ok = 0u;  // T_D of every Gamma is recomputed in the Galerkin form
  return DTR_OK;
}

// T_D^G = Tr(G^-1 V^H g5 Gamma V) for the Gammas in `gs` (Galerkin form)
int defl_tdg_gram(const dtr_defl_s *D, const GammaSet &gs, double2 *out, cudaStream_t st) {
  const int k = D->k;
  const int64_t nsite = D->lat.V;
  std::vector<std::complex<double>> Gi((size_t)k * k), M;
  DTR_CUDA(cudaMemcpy(Gi.data(), D->Ginv, sizeof(double2) * k * k, cudaMemcpyDeviceToHost));
  double2 *work = nullptr;
  DTR_CUDA(cudaMalloc((void **)&work, gram_work_elems(k, nsite) * sizeof(double2)));
  int rc = DTR_OK;
  for (int q = 0; q < gs.n && rc == DTR_OK; ++q) {
    const SpinXform T = xform_g5_gamma(gs.g[q]);
    if (D->prec == DTR_F64)
      rc = gram_product((const double2 *)D->V, k, k, (const double2 *)D->V, k, k, nsite, T, work, M, st);
    else if (D->prec == DTR_F32)
      rc = gram_product((const float2 *)D->V, k, k, (const float2 *)D->V, k, k, nsite, T, work, M, st);
    else
      rc = gram_product((const bfc2 *)D->V, k, k, (const bfc2 *)D->V, k, k, nsite, T, work, M, st);
    if (rc == DTR_OK) {
      const std::complex<double> t = trace_product(Gi, M, k);
      out[q] = make_double2(t.real(), t.imag());
    }
  }
  cudaFree(work);
  return rc;
}

}  // namespace dtr
