// Flexible GMRES(m) inner solver for the mixed-precision defect correction,
// with the learned network as right preconditioner (identity if none).
//
// All columns of a block share the Arnoldi loop; each keeps its own
// Hessenberg matrix and Givens rotations (FP64, host).  Per Arnoldi step:
//   z_k = M(v_k);  w = A z_k;  two passes of classical Gram-Schmidt against
//   v_1..v_k (batched multi-dot kernels, fixed-order reductions);
//   h_{k+1,k} = |w|, v_{k+1} = w / h_{k+1,k}.
// Flexible GMRES keeps the z_k and updates x += sum_k y_k z_k at the end of a
// cycle (Saad 1993), so M may change from step to step or be nonlinear.
#include <cmath>
#include <vector>

#include "dslash_core.cuh"
#include "net.cuh"
#include "reduce.cuh"
#include "solver.cuh"

namespace dtr {

constexpr int kDotThreads = 256;

// part[blk][i][j] = sum over this block's elements of conj(Vb[i][e]) w[e]   (i = blockIdx.y)
__global__ void __launch_bounds__(kDotThreads) k_multidot(const float2 *__restrict__ basis, int64_t vstride,
                                                          const float2 *__restrict__ w, int64_t n, int b,
                                                          double2 *__restrict__ part) {
  __shared__ double2 sh[kDotThreads];
  const int i = blockIdx.y;
  const float2 *v = basis + (int64_t)i * vstride;
  float ax = 0.f, ay = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = v[e], c = w[e];
    ax += a.x * c.x + a.y * c.y;
    ay += a.x * c.y - a.y * c.x;
  }
  sh[threadIdx.x] = make_double2(ax, ay);
  __syncthreads();
  for (int st = kDotThreads / 2; st >= b; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + st]);
    __syncthreads();
  }
  if ((int)threadIdx.x < b) part[((int64_t)blockIdx.x * gridDim.y + i) * b + threadIdx.x] = sh[threadIdx.x];
}

__global__ void k_multidot_reduce(const double2 *__restrict__ part, int nblocks, int k, int b, double2 *__restrict__ h) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * b) return;
  double2 s = make_double2(0.0, 0.0);
  for (int blk = 0; blk < nblocks; ++blk) s = cadd(s, part[(int64_t)blk * k * b + e]);
  h[e] = s;
}

// w -= sum_i h[i][j] v_i
__global__ void k_gs_update(const float2 *__restrict__ basis, int64_t vstride, float2 *__restrict__ w, int64_t n, int b,
                            int k, const double2 *__restrict__ h) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e & (b - 1));
    float2 acc = w[e];
    for (int i = 0; i < k; ++i) {
      const double2 hh = h[(int64_t)i * b + j];
      acc = caxpy(make_float2((float)-hh.x, (float)-hh.y), basis[(int64_t)i * vstride + e], acc);
    }
    w[e] = acc;
  }
}

// dst = src * s[j] (per column scale)
__global__ void k_scale_cols(const float2 *__restrict__ src, float2 *__restrict__ dst, int64_t n, int b,
                             const double *__restrict__ s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float sc = (float)s[e & (b - 1)];
    const float2 v = src[e];
    dst[e] = make_float2(v.x * sc, v.y * sc);
  }
}

// x += sum_k y[k][j] z_k
__global__ void k_combine(const float2 *__restrict__ Z, int64_t vstride, float2 *__restrict__ x, int64_t n, int b, int k,
                          const double2 *__restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e & (b - 1));
    float2 acc = x[e];
    for (int i = 0; i < k; ++i) {
      const double2 yy = y[(int64_t)i * b + j];
      acc = caxpy(make_float2((float)yy.x, (float)yy.y), Z[(int64_t)i * vstride + e], acc);
    }
    x[e] = acc;
  }
}

// r = rhs - A x (FP32)
__global__ void __launch_bounds__(256) k_resid32(const float2 *__restrict__ U, const float2 *__restrict__ x,
                                                 const float2 *__restrict__ rhs, float2 *__restrict__ r, Geom g, int b,
                                                 int logb, float diag) {
  const int64_t n = (int64_t)g.V << logb;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(it & (b - 1));
    const int s = (int)(it >> logb);
    float2 o[12], self[12];
    dslash_site<1, float>(U, x, g, b, s, j, diag, o, self);
    const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
    for (int c = 0; c < 12; ++c) r[base + c * b] = csub(rhs[base + c * b], o[c]);
  }
}

size_t fgmres_scratch_bytes(int64_t V, int b, int m) {
  const size_t vec = ((size_t)V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  const size_t part = (size_t)kMaxGrid * 32 * 64 * sizeof(double2);
  // basis (m+1) + Z (m) + w + r + 2 network scratch, dot partials, small
  return (2 * (size_t)m + 5) * vec + part + 128 * 1024 + 4096;
}

static int ilg(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

// Solve A e = rhs (FP32 fields of width b, e zero on entry) to |r| <= tol |rhs| per
// column, restarted FGMRES(m), at most max_iters Arnoldi steps.  active (host, b)
// masks columns; iters_out (host, b) receives the Arnoldi steps each column used.
int fgmres_solve(const dtr_gauge_s *gauge, double m0, const dtr_net_s *net, const float2 *rhs, float2 *x, int b,
                 const int *active, int m, double tol, int max_iters, void *work, size_t work_bytes, int *iters_out,
                 cudaStream_t st) {
  if (m < 1 || m > 32) return fail(DTR_EINVAL, "gmres_m must be in [1, 32]");
  const Geom g = geom_of(gauge->lat);
  const int64_t n = (int64_t)g.V * 12 * b;
  if (work_bytes < fgmres_scratch_bytes(g.V, b, m)) return fail(DTR_ENOMEM, "FGMRES workspace too small");
  const size_t vec = ((size_t)n * sizeof(float2) + 255) / 256 * 256;
  const int64_t vstride = (int64_t)(vec / sizeof(float2));
  char *w8 = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  float2 *Vb = (float2 *)w8;                 w8 += (m + 1) * vec;
  float2 *Zb = (float2 *)w8;                 w8 += m * vec;
  float2 *wv = (float2 *)w8;                 w8 += vec;
  float2 *r = (float2 *)w8;                  w8 += vec;
  float2 *t0 = (float2 *)w8;                 w8 += vec;
  float2 *t1 = (float2 *)w8;                 w8 += vec;
  double2 *part = (double2 *)w8;             w8 += (size_t)kMaxGrid * 32 * 64 * sizeof(double2);
  double2 *hdev = (double2 *)w8;             w8 += 32 * 64 * sizeof(double2);
  double *sdev = (double *)w8;               w8 += 64 * sizeof(double);
  double2 *ydev = (double2 *)w8;
  const int sms = device_sms();
  const unsigned gv = reduce_grid(n, sms);
  const unsigned gd = reduce_grid((int64_t)g.V * b, sms);
  const int logb = ilg(b);
  const float diag = (float)(4.0 + m0);

  // host Hessenberg per column: H[j][row][col], Givens cs/sn, rhs g
  std::vector<std::vector<double2>> H(b, std::vector<double2>((m + 1) * m));
  std::vector<std::vector<double2>> gvec(b, std::vector<double2>(m + 1));
  std::vector<std::vector<double>> cs(b, std::vector<double>(m));
  std::vector<std::vector<double2>> sn(b, std::vector<double2>(m));
  std::vector<double2> hh((size_t)(m + 1) * 64);
  std::vector<double> beta(b), sc(64, 0.0), rnorm0(b, 1.0);
  std::vector<int> done(b, 0), kused(b, 0);
  for (int j = 0; j < b; ++j) {
    done[j] = active[j] ? 0 : 1;
    iters_out[j] = 0;
  }
  auto norms = [&](const float2 *v, std::vector<double> &out) -> int {
    k_multidot<<<dim3(gv, 1), kDotThreads, 0, st>>>(v, 0, v, n, b, part);
    k_multidot_reduce<<<1, 64, 0, st>>>(part, gv, 1, b, hdev);
    count_launches(2);
    DTR_CUDA(cudaMemcpyAsync(hh.data(), hdev, sizeof(double2) * b, cudaMemcpyDeviceToHost, st));
    DTR_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < b; ++j) out[j] = std::sqrt(hh[j].x > 0 ? hh[j].x : 0.0);
    return DTR_OK;
  };
  int total = 0;
  bool first = true;
  while (total < max_iters) {
    // r = rhs - A x (x = 0 on the first cycle)
    if (first) {
      DTR_CUDA(cudaMemcpyAsync(r, rhs, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    } else {
      k_resid32<<<gd, 256, 0, st>>>(gauge->U32, x, rhs, r, g, b, logb, diag);
      count_launches(1);
    }
    int rc = norms(r, beta);
    if (rc) return rc;
    if (first) {
      for (int j = 0; j < b; ++j) rnorm0[j] = beta[j] > 0 ? beta[j] : 1.0;
      first = false;
    }
    bool all = true;
    for (int j = 0; j < b; ++j) {
      if (!active[j] || beta[j] <= tol * rnorm0[j]) done[j] = 1;
      if (!done[j]) all = false;
    }
    if (all) break;
    for (int j = 0; j < b; ++j) {
      sc[j] = (!done[j] && beta[j] > 0) ? 1.0 / beta[j] : 0.0;
      std::fill(gvec[j].begin(), gvec[j].end(), make_double2(0.0, 0.0));
      gvec[j][0] = make_double2(done[j] ? 0.0 : beta[j], 0.0);
      kused[j] = 0;
    }
    DTR_CUDA(cudaMemcpyAsync(sdev, sc.data(), sizeof(double) * b, cudaMemcpyHostToDevice, st));
    k_scale_cols<<<gv, 256, 0, st>>>(r, Vb, n, b, sdev);
    count_launches(1);
    int k = 0;
    for (; k < m && total < max_iters; ++k, ++total) {
      float2 *vk = Vb + (int64_t)k * vstride;
      float2 *zk = Zb + (int64_t)k * vstride;
      if (net)
        net_apply(net, vk, zk, b, t0, t1, st);
      else
        DTR_CUDA(cudaMemcpyAsync(zk, vk, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
      launch_dslash<float>(gauge->U32, zk, wv, g, b, m0, 0, st);  // w = A z_k
      for (int pass = 0; pass < 2; ++pass) {
        k_multidot<<<dim3(gv, k + 1), kDotThreads, 0, st>>>(Vb, vstride, wv, n, b, part);
        k_multidot_reduce<<<(unsigned)(((k + 1) * b + 63) / 64), 64, 0, st>>>(part, gv, k + 1, b, hdev);
        k_gs_update<<<gv, 256, 0, st>>>(Vb, vstride, wv, n, b, k + 1, hdev);
        count_launches(3);
        DTR_CUDA(cudaMemcpyAsync(hh.data(), hdev, sizeof(double2) * (k + 1) * b, cudaMemcpyDeviceToHost, st));
        DTR_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < b; ++j)
          for (int i = 0; i <= k; ++i) {
            double2 &Hij = H[j][i * m + k];
            if (pass == 0) Hij = hh[(size_t)i * b + j];
            else Hij = cadd(Hij, hh[(size_t)i * b + j]);
          }
      }
      std::vector<double> wn(b);
      int rc2 = norms(wv, wn);
      if (rc2) return rc2;
      for (int j = 0; j < b; ++j) {
        H[j][(k + 1) * m + k] = make_double2(wn[j], 0.0);
        sc[j] = (!done[j] && wn[j] > 1e-300) ? 1.0 / wn[j] : 0.0;
      }
      DTR_CUDA(cudaMemcpyAsync(sdev, sc.data(), sizeof(double) * b, cudaMemcpyHostToDevice, st));
      k_scale_cols<<<gv, 256, 0, st>>>(wv, Vb + (int64_t)(k + 1) * vstride, n, b, sdev);
      count_launches(1);
      // Givens rotations per column (complex), residual estimate |g_{k+1}|
      bool all2 = true;
      for (int j = 0; j < b; ++j) {
        if (done[j]) continue;
        std::vector<double2> &Hj = H[j];
        for (int i = 0; i < k; ++i) {  // apply previous rotations to column k
          const double2 a = Hj[i * m + k], c2 = Hj[(i + 1) * m + k];
          const double c = cs[j][i];
          const double2 s = sn[j][i];
          // [a'; c2'] = [c, s; -conj(s), c] [a; c2]
          const double2 a1 = make_double2(c * a.x + s.x * c2.x - s.y * c2.y, c * a.y + s.x * c2.y + s.y * c2.x);
          const double2 c3 = make_double2(-(s.x * a.x + s.y * a.y) + c * c2.x, -(s.x * a.y - s.y * a.x) + c * c2.y);
          Hj[i * m + k] = a1;
          Hj[(i + 1) * m + k] = c3;
        }
        const double2 a = Hj[k * m + k];
        const double hb = Hj[(k + 1) * m + k].x;
        const double na = std::sqrt(a.x * a.x + a.y * a.y);
        const double den = std::sqrt(na * na + hb * hb);
        double c = 1.0;
        double2 s = make_double2(0.0, 0.0);
        if (den > 0) {
          if (na > 0) {
            c = na / den;
            // s = (a / |a|) * hb / den  -> rotates [a; hb] to [den * a/|a|; 0]
            s = make_double2(a.x / na * hb / den, a.y / na * hb / den);
            Hj[k * m + k] = make_double2(a.x / na * den, a.y / na * den);
          } else {
            c = 0.0;
            s = make_double2(1.0, 0.0);
            Hj[k * m + k] = make_double2(hb, 0.0);
          }
        }
        Hj[(k + 1) * m + k] = make_double2(0.0, 0.0);
        cs[j][k] = c;
        sn[j][k] = s;
        const double2 gk = gvec[j][k];
        gvec[j][k] = make_double2(c * gk.x, c * gk.y);
        gvec[j][k + 1] = make_double2(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
        kused[j] = k + 1;
        iters_out[j] += 1;
        const double res = std::sqrt(gvec[j][k + 1].x * gvec[j][k + 1].x + gvec[j][k + 1].y * gvec[j][k + 1].y);
        if (res <= tol * rnorm0[j] || hb <= 1e-300) done[j] = 2;  // converged within this cycle
        else all2 = false;
      }
      if (all2) {
        ++k;
        ++total;
        break;
      }
    }
    // y = R^-1 g per column (back substitution), x += Z y
    std::vector<double2> yh((size_t)m * b, make_double2(0.0, 0.0));
    for (int j = 0; j < b; ++j) {
      const int kk = kused[j];
      for (int i = kk - 1; i >= 0; --i) {
        double2 acc = gvec[j][i];
        for (int l = i + 1; l < kk; ++l) acc = csub(acc, cmul(H[j][i * m + l], yh[(size_t)l * b + j]));
        yh[(size_t)i * b + j] = cdiv(acc, H[j][i * m + i]);
      }
      if (done[j] == 2) done[j] = 1;
    }
    DTR_CUDA(cudaMemcpyAsync(ydev, yh.data(), sizeof(double2) * m * b, cudaMemcpyHostToDevice, st));
    k_combine<<<gv, 256, 0, st>>>(Zb, vstride, x, n, b, k, ydev);
    count_launches(1);
    DTR_LAUNCH_CHECK("fgmres cycle");
    if (net && net->tc) {
      const int rc3 = net_check_err(net, st);
      if (rc3) return rc3;
    }
  }
  return DTR_OK;
}

}  // namespace dtr
