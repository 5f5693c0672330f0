// W_d distance diagnostic (Section 6.2): how much of a matrix's off-diagonal
// weight sits at each lattice distance.  For sampled dofs i_q and the columns
// B e_(i_q) (device, canonical layout), W_d = mean over q of
//     sum over dofs j != i_q of sites at periodic Manhattan distance d from i_q's site
//     of |B_(j, i_q)|^2, divided by m_d (the number of sites at distance d),
// optionally restricted to sites of the same hierarchical-probing colour as
// i_q (the mask (H H^H) of normalised probing vectors).  For B = A^-1 or
// A^-1 - V Lambda^-1 V^H g5 the column and row of a dof have the same moduli
// (g5-Hermiticity), so columns stand for the rows the definition names.
#include <vector>

#include "dtr_internal.cuh"

namespace dtr {

// one block per (column q, distance d): fixed-order tree reduction, deterministic
__global__ void k_wd(const double2 *__restrict__ cols, int64_t N, const int64_t *__restrict__ dofs, Geom g, int maxd,
                     int ncolors, double *__restrict__ out) {
  __shared__ double sh[256];
  const int q = blockIdx.x / (maxd + 1), d = blockIdx.x % (maxd + 1);
  const int64_t i = dofs[q];
  int xi[4];
  site_coords(g, (int)(i / 12), xi);
  const int ci = ncolors > 1 ? hp_colour(xi, ncolors) : 0;
  const double2 *col = cols + (int64_t)q * N;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    if (j == i) continue;
    int xj[4];
    site_coords(g, (int)(j / 12), xj);
    int dist = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int t = xi[mu] > xj[mu] ? xi[mu] - xj[mu] : xj[mu] - xi[mu];
      dist += t < g.L[mu] - t ? t : g.L[mu] - t;
    }
    if (dist != d) continue;
    if (ncolors > 1 && hp_colour(xj, ncolors) != ci) continue;
    const double2 v = col[j];
    acc += v.x * v.x + v.y * v.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// number of sites at each periodic Manhattan distance 0..maxd from a site
static std::vector<double> distance_counts(const int L[4], int maxd) {
  std::vector<double> cnt(maxd + 1, 0.0);
  cnt[0] = 1.0;
  for (int mu = 0; mu < 4; ++mu) {
    std::vector<double> per(L[mu] / 2 + 1, 0.0);  // sites at distance t along one axis
    for (int x = 0; x < L[mu]; ++x) per[x < L[mu] - x ? x : L[mu] - x] += 1.0;
    std::vector<double> nxt(maxd + 1, 0.0);
    for (int a = 0; a <= maxd; ++a)
      for (int t = 0; t < (int)per.size() && a + t <= maxd; ++t) nxt[a + t] += cnt[a] * per[t];
    cnt.swap(nxt);
  }
  return cnt;
}

int wd_diagnostic(const dtr_lattice_s *lat, const double2 *cols, const int64_t *dofs_host, int ns, int maxd,
                  int ncolors, double *W, cudaStream_t st) {
  const Geom g = geom_of(*lat);
  const int64_t N = lat->N;
  for (int q = 0; q < ns; ++q)
    if (dofs_host[q] < 0 || dofs_host[q] >= N) return fail(DTR_EINVAL, "sampled dof out of range");
  int64_t *dofs = nullptr;
  double *out = nullptr;
  const size_t nout = (size_t)ns * (maxd + 1);
  DTR_CUDA(cudaMalloc((void **)&dofs, sizeof(int64_t) * ns + sizeof(double) * nout + 256));
  out = (double *)((char *)dofs + ((sizeof(int64_t) * ns + 255) / 256) * 256);
  std::vector<double> h(nout);
  cudaError_t e = cudaMemcpyAsync(dofs, dofs_host, sizeof(int64_t) * ns, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_wd<<<(unsigned)nout, 256, 0, st>>>(cols, N, dofs, g, maxd, ncolors, out);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dofs);
  if (e != cudaSuccess) return cuda_fail(e, "W_d diagnostic");
  const std::vector<double> m = distance_counts(g.L, maxd);
  for (int d = 0; d <= maxd; ++d) {
    double s = 0.0;
    for (int q = 0; q < ns; ++q) s += h[(size_t)q * (maxd + 1) + d] / m[d];
    W[d] = m[d] > 0 ? s / ns : 0.0;
  }
  return DTR_OK;
}

}  // namespace dtr
