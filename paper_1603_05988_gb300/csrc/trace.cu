// Algorithm 1 (deflatedHP, Section 5.2) for R independent z0 runs.
//
// For every run r and every block of probing columns the device generates
// z = z0_r .* z_h (lines 3-6), projects it on the deflation space (line 8,
// second term), solves A y = z (line 7) and reduces t = z^H y - d in FP64
// (line 8).  Trace_r = T_D + mean_j t_j (line 9).  The host keeps the
// per-sample record (also the per-m deflation terms, so a run can be replayed
// for any smaller k, Section 6.3) and forms the run statistics: the mean over
// runs, the variance over runs and its delete-1 jackknife error (Section 6.2).
#include <cmath>
#include <cstring>
#include <vector>

#include "deflate.cuh"
#include "reduce.cuh"
#include "solver.cuh"

namespace dtr {

// out[j] = sum_i conj(Z_ij) Y_ij - d[j]   (FP64, deterministic)
__global__ void __launch_bounds__(kBlock) k_zdot(const double2 *__restrict__ Z, const double2 *__restrict__ Y,
                                                 int64_t n, int b, const double2 *__restrict__ d,
                                                 double2 *__restrict__ out, Reduce red) {
  __shared__ double2 tot[64];
  double2 acc[1] = {make_double2(0.0, 0.0)};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 z = Z[e], y = Y[e];
    acc[0].x += z.x * y.x + z.y * y.y;
    acc[0].y += z.x * y.y - z.y * y.x;
  }
  if (block_reduce<1>(acc, b, red.partial, red.counter, tot)) {
    const int j = threadIdx.x;
    if (j < b) out[j] = d ? csub(tot[j], d[j]) : tot[j];
  }
}

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct TraceLayout {
  int b;
  size_t vec, zdot_red, solver, defl, hp, sites, small, total;
};

static TraceLayout trace_layout(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  TraceLayout L;
  L.b = pad_rhs(p->block);
  const int64_t V = g->lat.V;
  L.vec = al((size_t)V * 12 * L.b * sizeof(double2));
  L.zdot_red = al(256 + (size_t)kMaxGrid * 64 * sizeof(double2));
  L.solver = al(solver_scratch_bytes(V, L.b, p->solve.solver, p->solve.gmres_m));
  L.defl = D ? al(defl_scratch_bytes(V, D->k, L.b, device_sms())) : 0;
  const bool hp = D && p->ncolors > 1;
  L.hp = hp ? al(defl_hp_scratch_bytes(V, D->k, L.b, p->ncolors, device_sms())) : 0;
  L.sites = hp ? al((size_t)V * sizeof(int)) : 0;
  const int k = D ? D->k : 0;
  L.small = al(3 * 64 * sizeof(double2) + (size_t)k * 64 * sizeof(double2));
  L.total = 256 + 2 * L.vec + L.zdot_red + L.solver + L.defl + L.hp + L.sites + L.small;
  return L;
}

size_t trace_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  return trace_layout(g, D, p).total;
}

int trace_estimate(const dtr_gauge_s *gauge, double m0, const dtr_defl_s *D, const dtr_trace_params *p, void *work,
                   size_t work_bytes, dtr_trace_result *res, cudaStream_t st) {
  const TraceLayout L = trace_layout(gauge, D, p);
  if (work_bytes < L.total) return fail(DTR_ENOMEM, "trace workspace too small");
  const int b = L.b;
  const Geom g = geom_of(gauge->lat);
  const int64_t n = (int64_t)g.V * 12 * b;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double2 *Z = (double2 *)w;  w += L.vec;
  double2 *X = (double2 *)w;  w += L.vec;
  Reduce red;
  red.counter = (unsigned int *)w;
  red.partial = (double2 *)(w + 256);
  w += L.zdot_red;
  void *solver_work = w;      w += L.solver;
  void *defl_work = w;        w += L.defl;
  void *hp_work = w;          w += L.hp;
  int *sites_dev = (int *)w;  w += L.sites;
  double2 *d_dev = (double2 *)w;
  double2 *t_dev = d_dev + 64;
  double2 *terms_dev = d_dev + 192;
  DTR_CUDA(cudaMemsetAsync(red.counter, 0, 256, st));

  const int ncols = p->nvec * (p->dilute12 ? 12 : 1);
  const int R = p->n_z0;
  const int k = D ? D->k : 0;
  const double td = D ? D->td[0] : 0.0;
  const double td_im = D ? D->td[1] : 0.0;
  std::vector<double2> samples((size_t)R * p->nvec, make_double2(0.0, 0.0));
  std::vector<double2> tbuf(64), termbuf((size_t)k * 64);
  Scal sc_host;
  int64_t iters = 0, nsolves = 0;
  double maxres = 0.0;
  int all_conv = 1;
  int status = DTR_OK;
  const int sms = device_sms();
  if (res->replay) std::memset(res->replay, 0, sizeof(double) * 2 * (size_t)R * p->nvec * (k > 0 ? k : 1));

  // sites grouped by colour for the HP-structured projection (host counting sort)
  bool hp_ok = false;
  if (L.hp) {
    const int nc = p->ncolors;
    std::vector<int> count(nc, 0), col(g.V);
    for (int sidx = 0; sidx < g.V; ++sidx) {
      int xc[4];
      int r0 = sidx;
      xc[0] = r0 % g.L[0]; r0 /= g.L[0];
      xc[1] = r0 % g.L[1]; r0 /= g.L[1];
      xc[2] = r0 % g.L[2];
      xc[3] = r0 / g.L[2];
      col[sidx] = hp_colour(xc, nc);
      count[col[sidx]]++;
    }
    hp_ok = true;
    for (int c = 0; c < nc; ++c)
      if (count[c] != g.V / nc) hp_ok = false;
    if (hp_ok) {
      std::vector<int> list(g.V), pos(nc);
      for (int c = 0; c < nc; ++c) pos[c] = c * (g.V / nc);
      for (int sidx = 0; sidx < g.V; ++sidx) list[pos[col[sidx]]++] = sidx;
      DTR_CUDA(cudaMemcpyAsync(sites_dev, list.data(), sizeof(int) * g.V, cudaMemcpyHostToDevice, st));
      DTR_CUDA(cudaStreamSynchronize(st));
    }
  }

  // run-major sequence of (run, probing column) pairs, processed in blocks
  const int64_t total_cols = (int64_t)R * ncols;
  for (int64_t G0 = 0; G0 < total_cols; G0 += p->block) {
    {
      const int nb = (int)((total_cols - G0) < p->block ? (total_cols - G0) : p->block);
      const int64_t q0 = G0 % ncols;
      const bool one_run = q0 + nb <= ncols;
      launch_noise(Z, g, p->seed, p->z0_first, p->ncolors, p->dilute12, G0, ncols, nb, b, st);
      DTR_LAUNCH_CHECK("noise");
      if (D) {
        int rc;
        if (hp_ok && one_run && !p->use_x0)
          rc = defl_project_hp(D, sites_dev, p->ncolors, p->seed, p->z0_first + G0 / ncols, q0, nb, p->dilute12, b,
                               d_dev, res->replay ? terms_dev : nullptr, hp_work, L.hp, sms, st);
        else
          rc = defl_project_internal(D, Z, b, d_dev, res->replay ? terms_dev : nullptr, p->use_x0 ? X : nullptr,
                                     nullptr, defl_work, L.defl, sms, st);
        if (rc) return rc;
      }
      if (!D || !p->use_x0) DTR_CUDA(cudaMemsetAsync(X, 0, (size_t)n * sizeof(double2), st));
      Scal *sc = nullptr;
      int rc = solve_internal(gauge, m0, X, Z, b, &p->solve, solver_work, L.solver, st, &sc, !D || !p->use_x0);
      if (rc) return rc;
      k_zdot<<<reduce_grid(n, sms), kBlock, 0, st>>>(Z, X, n, b, D ? d_dev : nullptr, t_dev, red); count_launches(1);
      DTR_LAUNCH_CHECK("z^H y reduction");
      DTR_CUDA(cudaMemcpyAsync(tbuf.data(), t_dev, sizeof(double2) * b, cudaMemcpyDeviceToHost, st));
      DTR_CUDA(cudaMemcpyAsync(&sc_host, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
      if (D && res->replay)
        DTR_CUDA(cudaMemcpyAsync(termbuf.data(), terms_dev, sizeof(double2) * k * b, cudaMemcpyDeviceToHost, st));
      DTR_CUDA(cudaStreamSynchronize(st));
      for (int jj = 0; jj < nb; ++jj) {
        const int64_t Gc = G0 + jj;
        const int r = (int)(Gc / ncols);
        const int q = (int)(Gc % ncols);
        const int jv = p->dilute12 ? q / 12 : q;
        double2 &s = samples[(size_t)r * p->nvec + jv];
        s.x += tbuf[jj].x;
        s.y += tbuf[jj].y;
        iters += sc_host.iters[jj];
        const double rel = sc_host.bnorm2[jj] > 0 ? std::sqrt(sc_host.rtrue2[jj] / sc_host.bnorm2[jj]) : 0.0;
        if (rel > maxres || rel != rel) maxres = rel;
        if (!sc_host.conv[jj]) all_conv = 0;
        if (sc_host.flags[jj] & kFlagNaN) status = DTR_ENAN;
        if (res->replay && D) {
          double *rp = res->replay + 2 * (((size_t)r * p->nvec + jv) * k);
          for (int m = 0; m < k; ++m) {
            rp[2 * m] += termbuf[(size_t)jj * k + m].x;
            rp[2 * m + 1] += termbuf[(size_t)jj * k + m].y;
          }
        }
      }
      nsolves += nb;
    }
  }

  // run statistics (host, FP64)
  std::vector<double2> tr(R);
  double2 mean = make_double2(0.0, 0.0);
  for (int r = 0; r < R; ++r) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < p->nvec; ++j) s = cadd(s, samples[(size_t)r * p->nvec + j]);
    tr[r] = make_double2(td + s.x / p->nvec, td_im + s.y / p->nvec);
    mean = cadd(mean, tr[r]);
  }
  mean = cscale(mean, 1.0 / R);
  double var_runs = 0.0, jk = 0.0;
  if (R > 1) {
    for (int r = 0; r < R; ++r) {
      const double dx = tr[r].x - mean.x, dy = tr[r].y - mean.y;
      var_runs += dx * dx + dy * dy;
    }
    var_runs /= (R - 1);
    // delete-1 jackknife of the mean
    double2 tot = cscale(mean, (double)R);
    std::vector<double2> loo(R);
    double2 lm = make_double2(0.0, 0.0);
    for (int r = 0; r < R; ++r) {
      loo[r] = cscale(csub(tot, tr[r]), 1.0 / (R - 1));
      lm = cadd(lm, loo[r]);
    }
    lm = cscale(lm, 1.0 / R);
    for (int r = 0; r < R; ++r) {
      const double dx = loo[r].x - lm.x, dy = loo[r].y - lm.y;
      jk += dx * dx + dy * dy;
    }
    jk = std::sqrt(jk * (R - 1) / R);
  }
  double var_s = 0.0;
  const size_t ns = samples.size();
  if (ns > 1) {
    double2 sm = make_double2(0.0, 0.0);
    for (auto &s : samples) sm = cadd(sm, s);
    sm = cscale(sm, 1.0 / ns);
    for (auto &s : samples) {
      const double dx = s.x - sm.x, dy = s.y - sm.y;
      var_s += dx * dx + dy * dy;
    }
    var_s /= (ns - 1);
  }
  res->trace[0] = mean.x;
  res->trace[1] = mean.y;
  res->T_D[0] = td;
  res->T_D[1] = td_im;
  res->var_runs = var_runs;
  res->jk_err = jk;
  res->var_samples = var_s;
  res->n_solves = nsolves;
  res->iterations = iters;
  res->max_true_residual = maxres;
  res->all_converged = all_conv;
  if (res->samples)
    for (size_t i = 0; i < ns; ++i) {
      res->samples[2 * i] = samples[i].x;
      res->samples[2 * i + 1] = samples[i].y;
    }
  if (res->trace_runs)
    for (int r = 0; r < R; ++r) {
      res->trace_runs[2 * r] = tr[r].x;
      res->trace_runs[2 * r + 1] = tr[r].y;
    }
  if (status == DTR_OK && !all_conv) return fail(DTR_ENOTCONV, "some right-hand sides did not reach tol");
  if (status == DTR_ENAN) return fail(DTR_ENAN, "NaN or Inf in a residual norm");
  return DTR_OK;
}

}  // namespace dtr
