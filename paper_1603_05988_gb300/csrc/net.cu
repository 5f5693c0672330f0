// Learned preconditioner: a 4-layer 4D convolutional network M ~ A^-1.
//
// Fields are the solver's complex fields read as 24 real channels per site
// (channel 2c + p is the real (p = 0) or imaginary (p = 1) part of dof c =
// 3*spin + colour), in the RHS-inner layout [site][12][b] of float2.  Layer l
// applies a 3^4 periodic stencil with weights W_l[o][co][ci] (o = offset index
// ((dt*3 + dz)*3 + dy)*3 + dx, displacement d - 1 per direction), no bias:
//   h_1 = W_0 * x,  h_{l+1} = W_l * phi(h_l),  y = W_3 * phi(h_3)
// phi is the identity or a leaky ReLU with slope 1/4; both are positively
// homogeneous, so M(a v) = a M(v) for a > 0 and the network needs no input
// normalisation inside a Krylov method.  Weights are stored in BF16 (the
// master copy and the Adam moments in FP32); arithmetic accumulates in FP32.
//
// Kernels: forward convolution (optionally applying phi to its input on the
// fly), backward-data convolution (flipped stencil, transposed channels, times
// phi'(h) of the layer below), backward-weights correlation (per-offset,
// per-chunk partial sums reduced in a fixed order), loss and its gradient, Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dtr_internal.cuh"
#include "net.cuh"

namespace dtr {

constexpr int kOffs = 81;
constexpr int kCh = 24;
constexpr int kOffChunk = 9;                   // offsets staged in shared memory at a time
constexpr int kConvThreads = 128;

__device__ __forceinline__ float act_f(float u, int act) { return (act && u < 0.f) ? 0.25f * u : u; }
__device__ __forceinline__ float act_d(float u, int act) { return (act && u < 0.f) ? 0.25f : 1.f; }

// site reached from s by displacement (dx, dy, dz, dt) in {-1, 0, 1}^4, periodic
__device__ __forceinline__ int disp_site(const Geom &g, const int xc[4], int o, int sign) {
  int c[4];
  int r = o;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int d = (r % 3) - 1;
    r /= 3;
    int v = xc[mu] + sign * d;
    if (v < 0) v += g.L[mu];
    if (v >= g.L[mu]) v -= g.L[mu];
    c[mu] = v;
  }
  return site_of(g, c);
}

// out(s, co, j) = sum_o sum_ci Wt[o][ci][co] * f(in(s + sign*d(o), ci, j))
//   forward:       sign = +1, Wt = W transposed to [o][ci][co], f = phi or identity
//   backward data: sign = -1, Wt = W as [o][co][ci] read as [o][ci'][co'] (transpose), then
//                  times phi'(hmul) of the layer below if given
// (the kernel always reads weights as [o][k][m] with k = summed channel, m = output channel)
__global__ void __launch_bounds__(kConvThreads)
    k_conv(const float2 *__restrict__ in, float2 *__restrict__ out, const float *__restrict__ Wkm, Geom g, int b,
           int logb, int sign, int act_in, const float2 *__restrict__ hmul, int act_mul) {
  __shared__ float w[kOffChunk][kCh][kCh];
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.V << logb;
  const bool live = it < n;
  const int j = it & (b - 1);
  const int s = it >> logb;
  int xc[4] = {0, 0, 0, 0};
  if (live) site_coords(g, s, xc);
  float acc[kCh];
#pragma unroll
  for (int m = 0; m < kCh; ++m) acc[m] = 0.f;
  for (int o0 = 0; o0 < kOffs; o0 += kOffChunk) {
    __syncthreads();
    for (int e = threadIdx.x; e < kOffChunk * kCh * kCh; e += blockDim.x) {
      const int oo = e / (kCh * kCh);
      (&w[0][0][0])[e] = (o0 + oo < kOffs) ? Wkm[(int64_t)o0 * kCh * kCh + e] : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    for (int oo = 0; oo < kOffChunk && o0 + oo < kOffs; ++oo) {
      const int nb = disp_site(g, xc, o0 + oo, sign);
      const float2 *p = in + ((int64_t)nb * 12) * b + j;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const float2 v = p[(int64_t)c * b];
        const float x0 = act_f(v.x, act_in), x1 = act_f(v.y, act_in);
        const float *w0 = &w[oo][2 * c][0];
        const float *w1 = &w[oo][2 * c + 1][0];
#pragma unroll
        for (int m = 0; m < kCh; ++m) acc[m] = fmaf(w0[m], x0, fmaf(w1[m], x1, acc[m]));
      }
    }
  }
  if (!live) return;
  float2 *q = out + ((int64_t)s * 12) * b + j;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    float2 r = make_float2(acc[2 * c], acc[2 * c + 1]);
    if (hmul) {
      const float2 h = hmul[((int64_t)s * 12 + c) * b + j];
      r.x *= act_d(h.x, act_mul);
      r.y *= act_d(h.y, act_mul);
    }
    q[(int64_t)c * b] = r;
  }
}

// dW[o][co][ci] partial over a chunk of items: sum g(s, co, j) * phi(a(s + d(o), ci, j))
__global__ void __launch_bounds__(288)
    k_conv_wgrad(const float2 *__restrict__ a, const float2 *__restrict__ gout, Geom g, int b, int logb, int act_in,
                 int nchunks, float *__restrict__ part) {
  __shared__ float ga[64][kCh];
  __shared__ float xa[64][kCh];
  const int o = blockIdx.x;
  const int chunk = blockIdx.y;
  const int n = g.V << logb;
  const int i0 = (int)(((int64_t)n * chunk) / nchunks), i1 = (int)(((int64_t)n * (chunk + 1)) / nchunks);
  const int t = threadIdx.x;                    // 288 threads: (co, ci pair) = (t / 12, 2 * (t % 12))
  const int co = t / 12, ci = 2 * (t % 12);
  float acc0 = 0.f, acc1 = 0.f;
  for (int base = i0; base < i1; base += 64) {
    const int cnt = (i1 - base) < 64 ? (i1 - base) : 64;
    __syncthreads();
    for (int e = t; e < cnt * 12; e += blockDim.x) {
      const int u = e / 12, c = e % 12;
      const int it = base + u;
      const int j = it & (b - 1), s = it >> logb;
      int xc[4];
      site_coords(g, s, xc);
      const int nb = disp_site(g, xc, o, +1);
      const float2 gv = gout[((int64_t)s * 12 + c) * b + j];
      const float2 av = a[((int64_t)nb * 12 + c) * b + j];
      ga[u][2 * c] = gv.x;
      ga[u][2 * c + 1] = gv.y;
      xa[u][2 * c] = act_f(av.x, act_in);
      xa[u][2 * c + 1] = act_f(av.y, act_in);
    }
    __syncthreads();
    for (int u = 0; u < cnt; ++u) {
      const float gg = ga[u][co];
      acc0 = fmaf(gg, xa[u][ci], acc0);
      acc1 = fmaf(gg, xa[u][ci + 1], acc1);
    }
  }
  float *pp = part + ((int64_t)chunk * kOffs + o) * kCh * kCh;
  pp[co * kCh + ci] = acc0;
  pp[co * kCh + ci + 1] = acc1;
}

__global__ void k_wgrad_reduce(const float *__restrict__ part, int nchunks, float *__restrict__ dW) {
  const int n = kOffs * kCh * kCh;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double sacc = 0.0;
    for (int c = 0; c < nchunks; ++c) sacc += part[(int64_t)c * n + e];
    dW[e] = (float)sacc;
  }
}

// per-column loss: L_j = |y_j - e_j|^2 / |e_j|^2 (fixed-order block partials), grad = 2 (y - e) / |e|^2
__global__ void k_loss_partial(const float2 *__restrict__ y, const float2 *__restrict__ e, int64_t n, int b,
                               double *__restrict__ part) {
  __shared__ double sd[256], se[256];
  double d2 = 0.0, e2 = 0.0;
  const int j = threadIdx.x & (b - 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = y[i], t = e[i];
    const double dx = (double)a.x - t.x, dy = (double)a.y - t.y;
    d2 += dx * dx + dy * dy;
    e2 += (double)t.x * t.x + (double)t.y * t.y;
  }
  sd[threadIdx.x] = d2;
  se[threadIdx.x] = e2;
  __syncthreads();
  for (int st = 128; st >= b; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sd[threadIdx.x] += sd[threadIdx.x + st];
      se[threadIdx.x] += se[threadIdx.x + st];
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < b) {
    part[((int64_t)blockIdx.x * 2 + 0) * b + j] = sd[threadIdx.x];
    part[((int64_t)blockIdx.x * 2 + 1) * b + j] = se[threadIdx.x];
  }
}

__global__ void k_loss_finish(const double *__restrict__ part, int nblocks, int b, int nrhs, double *__restrict__ col) {
  const int j = threadIdx.x;
  if (j >= b) return;
  double d2 = 0.0, e2 = 0.0;
  for (int k = 0; k < nblocks; ++k) {
    d2 += part[((int64_t)k * 2 + 0) * b + j];
    e2 += part[((int64_t)k * 2 + 1) * b + j];
  }
  col[2 * j] = j < nrhs && e2 > 0 ? d2 / e2 : 0.0;   // loss of column j
  col[2 * j + 1] = e2 > 0 ? e2 : 1.0;               // |e_j|^2
}

__global__ void k_loss_grad(const float2 *__restrict__ y, const float2 *__restrict__ e, int64_t n, int b, int nrhs,
                            const double *__restrict__ col, float2 *__restrict__ gy) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & (b - 1));
    const float sc = j < nrhs ? (float)(2.0 / col[2 * j + 1]) : 0.f;
    const float2 a = y[i], t = e[i];
    gy[i] = make_float2(sc * (a.x - t.x), sc * (a.y - t.y));
  }
}

// Adam on FP32 master weights; also refreshes the BF16 copy and the transposed FP32 copies
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ gr,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// W master [l][o][co][ci] -> BF16-rounded FP32 copies in both orders:
//   fwd [l][o][ci][co] (summed index ci first) and bwd [l][o][co][ci] (summed index co first)
__global__ void k_refresh(const float *__restrict__ w, float *__restrict__ wf, float *__restrict__ wb, int L) {
  const int per = kOffs * kCh * kCh;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * per; e += gridDim.x * blockDim.x) {
    const int l = e / per, r = e % per;
    const int o = r / (kCh * kCh), co = (r / kCh) % kCh, ci = r % kCh;
    const float q = __bfloat162float(__float2bfloat16_rn(w[e]));
    wf[(int64_t)l * per + (o * kCh + ci) * kCh + co] = q;
    wb[e] = q;
  }
}

// ------------------------------------------------------------------ host side
static unsigned gs1(int64_t n, int T = 256) {
  int64_t g = (n + T - 1) / T;
  if (g > 65535LL * 8) g = 65535LL * 8;
  return (unsigned)(g < 1 ? 1 : g);
}
static int lg(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

constexpr int kWChunks = 64;

size_t net_workspace_bytes(const dtr_net_s *net, int b) {
  const size_t vec = ((size_t)net->lat.V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  size_t wpart = (size_t)kWChunks * kOffs * kCh * kCh * sizeof(float);
  if (net_wgrad_tc_scratch_bytes() > wpart) wpart = net_wgrad_tc_scratch_bytes();
  // x, h1..h3, y, target, g_a, g_b, (grad scratch) + loss partials
  const size_t lparts = (2 * 2048 * 64 + 256) * sizeof(double);  // loss partials [block][2][b] + per-column sums
  return 10 * vec + wpart + lparts + 4096;
}

void net_refresh(dtr_net_s *net, cudaStream_t st) {
  k_refresh<<<gs1((int64_t)net->L * kOffs * kCh * kCh), 256, 0, st>>>(net->w, net->wf, net->wb, net->L);
  count_launches(1);
  net_refresh_tc(net, st);
}

int net_check_err(const dtr_net_s *net, cudaStream_t st) {
  int e = 0;
  DTR_CUDA(cudaMemcpyAsync(&e, net->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  if (e) {
    DTR_CUDA(cudaMemsetAsync(net->err, 0, sizeof(int), st));
    return fail(DTR_ETIMEOUT, "tensor-core convolution: a bounded wait ran out");
  }
  return DTR_OK;
}

// planar BF16 field of width b: 3 chunks x 16 bytes per site and column (half a float2 field)
static size_t planar_bytes(int64_t V, int b) { return ((size_t)V * 3 * b * 16 + 255) / 256 * 256; }

// y = M x on float2 internal fields of width b (x, y distinct); scratch: 2 vectors
void net_apply(const dtr_net_s *net, const float2 *x, float2 *y, int b, float2 *t0, float2 *t1, cudaStream_t st) {
  if (net->tc) {  // two planar BF16 fields fit in t0
    uint4 *pl[2] = {(uint4 *)t0, (uint4 *)((char *)t0 + planar_bytes(net->lat.V, b))};
    net_to_planar(x, pl[0], net->lat.V, b, st);
    for (int l = 0; l < net->L; ++l) {
      const bool last = l == net->L - 1;
      net_conv_tc(net, l, false, pl[l & 1], last ? nullptr : pl[(l + 1) & 1], last ? y : nullptr, nullptr, net->act,
                  b, st);
    }
    return;
  }
  const Geom g = geom_of(net->lat);
  const int n = (int)(net->lat.V * b);
  const int per = kOffs * kCh * kCh;
  const float2 *src = x;
  float2 *bufs[2] = {t0, t1};
  for (int l = 0; l < net->L; ++l) {
    float2 *dst = (l == net->L - 1) ? y : bufs[l & 1];
    k_conv<<<(n + kConvThreads - 1) / kConvThreads, kConvThreads, 0, st>>>(
        src, dst, net->wf + (int64_t)l * per, g, b, lg(b), +1, l > 0 ? net->act : 0, nullptr, 0);
    count_launches(1);
    src = dst;
  }
}

// Forward keeping pre-activations, loss, backward, optional Adam step.
// fields (float2, width b): x input, e target; returns per-column loss in col (host, 2*b doubles)
int net_train(dtr_net_s *net, const dtr_gauge_s *gauge, double m0, const float2 *x, const float2 *e, int b, int nrhs,
              double lr, int do_step, float *grad_host, double *loss_out, void *work, size_t work_bytes,
              cudaStream_t st) {
  if (work_bytes < net_workspace_bytes(net, b)) return fail(DTR_ENOMEM, "network workspace too small");
  const Geom g = geom_of(net->lat);
  const int n = (int)(net->lat.V * b);
  const int64_t nel = (int64_t)net->lat.V * 12 * b;
  const int per = kOffs * kCh * kCh;
  const int L = net->L;
  const size_t vec = ((size_t)net->lat.V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  float2 *h[5];  // h[0] = x (not stored), h[1..L-1] pre-activations, h[L] = y
  for (int l = 1; l <= L; ++l) {
    h[l] = (float2 *)w;
    w += vec;
  }
  float2 *ga = (float2 *)w; w += vec;
  float2 *gb = (float2 *)w; w += vec;
  float *wpart = (float *)w;
  w += std::max((size_t)kWChunks * per * sizeof(float), net_wgrad_tc_scratch_bytes());
  double *lpart = (double *)w;
  double *lcol = lpart + 2 * 2048 * 64;
  h[0] = const_cast<float2 *>(x);
  // tensor-core path: planar BF16 inputs of the layers a[0..L-1] (a[l] = phi(h[l]), a[0] = x) in h[1], h[2];
  // planar gradients in h[3]; the FP32 output y in h[L]
  const size_t pb = planar_bytes(net->lat.V, b);
  uint4 *pa[4] = {(uint4 *)h[1], (uint4 *)((char *)h[1] + pb), (uint4 *)h[2], (uint4 *)((char *)h[2] + pb)};
  uint4 *pg[2] = {(uint4 *)h[3], (uint4 *)((char *)h[3] + pb)};
  if (net->tc) {
    net_to_planar(x, pa[0], net->lat.V, b, st);
    for (int l = 0; l < L; ++l)
      net_conv_tc(net, l, false, pa[l], l < L - 1 ? pa[l + 1] : nullptr, l == L - 1 ? h[L] : nullptr, nullptr,
                  net->act, b, st);
  }
  // forward
  for (int l = 0; l < (net->tc ? 0 : L); ++l) {
    k_conv<<<(n + kConvThreads - 1) / kConvThreads, kConvThreads, 0, st>>>(h[l], h[l + 1], net->wf + (int64_t)l * per,
                                                                         g, b, lg(b), +1, l > 0 ? net->act : 0,
                                                                         nullptr, 0);
    count_launches(1);
  }
  // loss and dL/dy
  const unsigned lg_blocks = gs1(nel) > 1024 ? 1024 : gs1(nel);
  if (gauge) {
    // residual-weighted loss |A y - x|^2 / |x|^2 (= |A (y - e)|^2 / |A e|^2 since A e = x):
    // the quantity that controls A M as a right preconditioner; dL/dy = A^H [2 (A y - x) / |x|^2]
    launch_dslash<float>(gauge->U32, h[L], gb, g, b, m0, 0, st);
    k_loss_partial<<<lg_blocks, 256, 0, st>>>(gb, x, nel, b, lpart);
    k_loss_finish<<<1, 64, 0, st>>>(lpart, lg_blocks, b, nrhs, lcol);
    k_loss_grad<<<gs1(nel), 256, 0, st>>>(gb, x, nel, b, nrhs, lcol, gb);
    launch_dslash<float>(gauge->U32, gb, ga, g, b, m0, 1, st);
    count_launches(3);
  } else {
    k_loss_partial<<<lg_blocks, 256, 0, st>>>(h[L], e, nel, b, lpart);
    k_loss_finish<<<1, 64, 0, st>>>(lpart, lg_blocks, b, nrhs, lcol);
    k_loss_grad<<<gs1(nel), 256, 0, st>>>(h[L], e, nel, b, nrhs, lcol, ga);
    count_launches(3);
  }
  // backward
  if (net->tc) {
    net_to_planar(ga, pg[0], net->lat.V, b, st);
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
      net_wgrad_tc(net, pa[l], pg[cur], b, wpart, net->grad + (int64_t)l * per, st);
      if (l > 0) {
        net_conv_tc(net, l, true, pg[cur], pg[cur ^ 1], nullptr, pa[l], 0, b, st);
        cur ^= 1;
      }
    }
  }
  float2 *gcur = ga, *gnext = gb;
  for (int l = L - 1; l >= (net->tc ? L : 0); --l) {
    // weight gradient of layer l: input phi(h[l]) (identity for l = 0), output grad gcur
    k_conv_wgrad<<<dim3(kOffs, kWChunks), 288, 0, st>>>(h[l], gcur, g, b, lg(b), l > 0 ? net->act : 0, kWChunks,
                                                        wpart);
    k_wgrad_reduce<<<gs1(per), 256, 0, st>>>(wpart, kWChunks, net->grad + (int64_t)l * per);
    count_launches(2);
    if (l > 0) {  // data gradient: W_l^T (flipped) applied to gcur, times phi'(h[l])
      k_conv<<<(n + kConvThreads - 1) / kConvThreads, kConvThreads, 0, st>>>(
          gcur, gnext, net->wb + (int64_t)l * per, g, b, lg(b), -1, 0, h[l], net->act);
      count_launches(1);
      float2 *tmp = gcur;
      gcur = gnext;
      gnext = tmp;
    }
  }
  if (do_step) {
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    k_adam<<<gs1((int64_t)L * per), 256, 0, st>>>(net->w, net->m, net->v, net->grad, L * per, (float)lr, b1, b2, 1e-8f,
                                                   c1, c2);
    count_launches(1);
    net_refresh(net, st);
  }
  DTR_LAUNCH_CHECK("network training step");
  std::vector<double> col(2 * b);
  DTR_CUDA(cudaMemcpyAsync(col.data(), lcol, sizeof(double) * 2 * b, cudaMemcpyDeviceToHost, st));
  if (grad_host) DTR_CUDA(cudaMemcpyAsync(grad_host, net->grad, sizeof(float) * L * per, cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  double tot = 0.0;
  for (int j = 0; j < nrhs; ++j) tot += col[2 * j];
  *loss_out = tot;
  return net->tc ? net_check_err(net, st) : DTR_OK;
}

}  // namespace dtr
