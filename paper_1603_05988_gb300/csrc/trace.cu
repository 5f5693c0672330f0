// Algorithm 1 (deflatedHP, Section 5.2) for R independent z0 runs.
//
// For every run r and every block of probing columns the device generates
// z = z0_r .* z_h, projects it on the deflation space (the deflation term d),
// solves A y = z and reduces the samples t = z^H y - d in FP64; the run's
// estimate is Trace_r = T_D + mean_j t_j.  The host keeps the
// per-sample record (also the per-m deflation terms, so a run can be replayed
// for any smaller k, Section 6.3) and forms the run statistics: the mean over
// runs, the variance over runs and its delete-1 jackknife error (Section 6.2).
#include <cmath>
#include <cstring>
#include <vector>

#include "deflate.cuh"
#include "gamma.cuh"
#include "reduce.cuh"
#include "solver.cuh"

namespace dtr {

// out[j] = sum_i conj(Z_ij) Y_ij - d[j]   (FP64, deterministic)
__global__ void __launch_bounds__(kBlock) k_zdot(const double2 *__restrict__ Z, const double2 *__restrict__ Y,
                                                 int64_t n, int b, const double2 *__restrict__ d,
                                                 double2 *__restrict__ out, double2 *__restrict__ ynorm,
                                                 Reduce red) {
  __shared__ double2 tot[2 * 64];
  double2 acc[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};  // z^H y ; (|y|^2, 0)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {  // four independent element pairs in flight
    double2 z[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      z[u] = __ldcs(Z + e + u * stride);
      y[u] = __ldcs(Y + e + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[0].x += z[u].x * y[u].x + z[u].y * y[u].y;
      acc[0].y += z[u].x * y[u].y - z[u].y * y[u].x;
      acc[1].x += y[u].x * y[u].x + y[u].y * y[u].y;
    }
  }
  for (; e < n; e += stride) {
    const double2 z = Z[e], y = Y[e];
    acc[0].x += z.x * y.x + z.y * y.y;
    acc[0].y += z.x * y.y - z.y * y.x;
    acc[1].x += y.x * y.x + y.y * y.y;
  }
  if (block_reduce<2>(acc, b, red.partial, red.counter, tot)) {
    const int j = threadIdx.x;
    if (j < b) {
      out[j] = d ? csub(tot[j], d[j]) : tot[j];
      ynorm[j] = tot[b + j];
    }
  }
}

// t^G_j = sum_x sum_(s,c) conj(z[x,s,c,j]) i^phase[s] y[x,perm[s],c,j] - dG_j for up to
// four Gammas per launch (one thread per site and column; FP64, deterministic)
template <int NG>
__global__ void __launch_bounds__(kBlock) k_zdot_gamma(const double2 *__restrict__ Z, const double2 *__restrict__ Y,
                                                       int64_t V, int b, int logb, GammaSet gs, int g0,
                                                       const double2 *__restrict__ dg, double2 *__restrict__ out,
                                                       Reduce red) {
  __shared__ double2 tot[NG * 64];
  double2 acc[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) acc[q] = make_double2(0.0, 0.0);
  const int64_t n = V << logb;
  const int j = threadIdx.x & (b - 1);
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (it >> logb) * 12 * b + j;
    double2 z[12], y[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      z[a] = __ldcs(Z + base + (int64_t)a * b);
      y[a] = __ldcs(Y + base + (int64_t)a * b);
    }
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      if (g0 + q >= gs.n) break;
      const GammaMono g = gs.g[g0 + q];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) {
        const int ph = g.phase[sp];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double2 w = y[g.perm[sp] * 3 + c];
          if (ph == 1) w = make_double2(-w.y, w.x);
          if (ph == 2) w = make_double2(-w.x, -w.y);
          if (ph == 3) w = make_double2(w.y, -w.x);
          const double2 u = z[sp * 3 + c];
          acc[q].x += u.x * w.x + u.y * w.y;
          acc[q].y += u.x * w.y - u.y * w.x;
        }
      }
    }
  }
  if (block_reduce<NG>(acc, b, red.partial, red.counter, tot)) {
    if ((int)threadIdx.x < b) {
      for (int q = 0; q < NG && g0 + q < gs.n; ++q) {
        const double2 t = tot[q * b + threadIdx.x];
        out[(g0 + q) * 64 + threadIdx.x] = dg ? csub(t, dg[(g0 + q) * 64 + threadIdx.x]) : t;
      }
    }
  }
}

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

static int ilog2(int b) {
  int l = 0;
  while ((1 << l) < b) ++l;
  return l;
}

// Run statistics of an (R x nvec) sample record (host, FP64, fixed order):
// Trace_r = T_D + mean_j t_j, their mean, variance over runs, delete-1
// jackknife error of the mean (Section 6.2), variance of the samples.
struct RunStats {
  double2 mean;
  std::vector<double2> tr;
  double var_runs, jk, var_s;
};

static RunStats run_stats(const double2 *samples, int R, int nvec, double td, double td_im) {
  RunStats o;
  o.tr.resize(R);
  o.mean = make_double2(0.0, 0.0);
  for (int r = 0; r < R; ++r) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < nvec; ++j) s = cadd(s, samples[(size_t)r * nvec + j]);
    o.tr[r] = make_double2(td + s.x / nvec, td_im + s.y / nvec);
    o.mean = cadd(o.mean, o.tr[r]);
  }
  o.mean = cscale(o.mean, 1.0 / R);
  o.var_runs = 0.0;
  o.jk = 0.0;
  if (R > 1) {
    for (int r = 0; r < R; ++r) {
      const double dx = o.tr[r].x - o.mean.x, dy = o.tr[r].y - o.mean.y;
      o.var_runs += dx * dx + dy * dy;
    }
    o.var_runs /= (R - 1);
    const double2 tot = cscale(o.mean, (double)R);
    std::vector<double2> loo(R);
    double2 lm = make_double2(0.0, 0.0);
    for (int r = 0; r < R; ++r) {
      loo[r] = cscale(csub(tot, o.tr[r]), 1.0 / (R - 1));
      lm = cadd(lm, loo[r]);
    }
    lm = cscale(lm, 1.0 / R);
    for (int r = 0; r < R; ++r) {
      const double dx = loo[r].x - lm.x, dy = loo[r].y - lm.y;
      o.jk += dx * dx + dy * dy;
    }
    o.jk = std::sqrt(o.jk * (R - 1) / R);
  }
  o.var_s = 0.0;
  const size_t ns = (size_t)R * nvec;
  if (ns > 1) {
    double2 sm = make_double2(0.0, 0.0);
    for (size_t i = 0; i < ns; ++i) sm = cadd(sm, samples[i]);
    sm = cscale(sm, 1.0 / ns);
    for (size_t i = 0; i < ns; ++i) {
      const double dx = samples[i].x - sm.x, dy = samples[i].y - sm.y;
      o.var_s += dx * dx + dy * dy;
    }
    o.var_s /= (ns - 1);
  }
  return o;
}

constexpr int kMaxLanes = 8;

struct TraceLayout {
  int b, lanes;
  size_t vec, zdot_red, solver, defl, hp, sites, small, gam, codes, lane, total;
};

// Lanes actually used: concurrency needs a solver that can run without
// synchronising the host.
static int trace_lanes(const dtr_trace_params *p) {
  int l = p->lanes < 1 ? 1 : p->lanes;
  if (l > kMaxLanes) l = kMaxLanes;
  if (l > 1 && !solve_can_run_async(&p->solve)) l = 1;
  return l;
}

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
  L.lanes = trace_lanes(p);
  // Gamma insertion: copy of the block's C (k x 2b), Gamma^H Z (generic projection), dG and tG (16 x 64)
  L.gam = p->n_gamma > 0 ? al((size_t)k * 2 * 64 * sizeof(double2)) + L.vec + 2 * al(16 * 64 * sizeof(double2)) : 0;
  // the block's entries as one-byte codes, read by the tensor-core contraction instead of the FP64 values
  L.codes = (D && defl_tc_enabled(D, L.b)) ? al((size_t)V * 12 * L.b) : 0;
  L.lane = 2 * L.vec + L.zdot_red + L.solver + L.defl + L.hp + L.small + L.gam + L.codes;
  L.total = 256 + L.sites + L.lanes * L.lane;
  return L;
}

size_t trace_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  return trace_layout(g, D, p).total;
}

// Per-lane device buffers, stream and pinned host staging.
struct Lane {
  cudaStream_t s = nullptr;
  double2 *Z = nullptr, *X = nullptr;
  Reduce red;
  void *solver_work = nullptr, *defl_work = nullptr, *hp_work = nullptr;
  double2 *d_dev = nullptr, *t_dev = nullptr, *yn_dev = nullptr, *terms_dev = nullptr;
  double2 *Cmain = nullptr, *GZ = nullptr, *dg = nullptr, *tg = nullptr;  // Gamma insertion
  unsigned char *Zc = nullptr;                  // Z as one-byte codes (tensor-core contraction)
  double2 *t_h = nullptr, *terms_h = nullptr, *tg_h = nullptr;  // pinned
  Scal *sc_h = nullptr;                         // pinned
  int *err_h = nullptr;                         // pinned
  size_t terms_cap = 0;
  int64_t G0 = 0;
  int nb = 0;
  int64_t hp_run = -1;   // z0 run whose per-colour sums W are in hp_work (-1: none)
};

// Library-owned streams and pinned staging of the extra lanes (per host thread).
struct LanePool {
  cudaStream_t s[kMaxLanes] = {};
  cudaEvent_t start = nullptr;
  double2 *t_h[kMaxLanes] = {}, *terms_h[kMaxLanes] = {}, *tg_h[kMaxLanes] = {};
  Scal *sc_h[kMaxLanes] = {};
  int *err_h[kMaxLanes] = {};
  size_t terms_cap[kMaxLanes] = {};
};
static thread_local LanePool t_pool;

static int lane_host_buffers(int l, int k) {
  LanePool &P = t_pool;
  if (!P.t_h[l]) DTR_CUDA(cudaMallocHost((void **)&P.t_h[l], 128 * sizeof(double2)));
  if (!P.tg_h[l]) DTR_CUDA(cudaMallocHost((void **)&P.tg_h[l], 16 * 64 * sizeof(double2)));
  if (!P.sc_h[l]) DTR_CUDA(cudaMallocHost((void **)&P.sc_h[l], sizeof(Scal)));
  if (!P.err_h[l]) DTR_CUDA(cudaMallocHost((void **)&P.err_h[l], 4 * sizeof(int)));
  const size_t need = (size_t)(k > 0 ? k : 1) * 64;
  if (P.terms_cap[l] < need) {
    if (P.terms_h[l]) cudaFreeHost(P.terms_h[l]);
    P.terms_h[l] = nullptr;
    P.terms_cap[l] = 0;
    DTR_CUDA(cudaMallocHost((void **)&P.terms_h[l], need * sizeof(double2)));
    P.terms_cap[l] = need;
  }
  return DTR_OK;
}

int trace_estimate(const dtr_gauge_s *gauge, double m0, const dtr_defl_s *D, const dtr_trace_params *p, void *work,
                   size_t work_bytes, dtr_trace_result *res, cudaStream_t st) {
  const TraceLayout L = trace_layout(gauge, D, p);
  if (work_bytes < L.total) return fail(DTR_ENOMEM, "trace workspace too small");
  const int b = L.b;
  const Geom g = geom_of(gauge->lat);
  const int64_t n = (int64_t)g.V * 12 * b;
  const int k = D ? D->k : 0;
  const int nlanes = L.lanes;
  const int sms = device_sms();
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  int *sites_dev = (int *)w;
  w += L.sites;
  Lane lanes[kMaxLanes];
  for (int l = 0; l < nlanes; ++l) {
    Lane &ln = lanes[l];
    char *q = w + (size_t)l * L.lane;
    ln.Z = (double2 *)q;  q += L.vec;
    ln.X = (double2 *)q;  q += L.vec;
    ln.red.counter = (unsigned int *)q;
    ln.red.partial = (double2 *)(q + 256);
    q += L.zdot_red;
    ln.solver_work = q;   q += L.solver;
    ln.defl_work = q;     q += L.defl;
    ln.hp_work = q;       q += L.hp;
    ln.d_dev = (double2 *)q;
    ln.t_dev = ln.d_dev + 64;
    ln.yn_dev = ln.d_dev + 128;
    ln.terms_dev = ln.d_dev + 192;
    q += L.small;
    if (L.gam) {
      ln.Cmain = (double2 *)q;  q += al((size_t)k * 2 * 64 * sizeof(double2));
      ln.GZ = (double2 *)q;     q += L.vec;
      ln.dg = (double2 *)q;     q += al(16 * 64 * sizeof(double2));
      ln.tg = (double2 *)q;     q += al(16 * 64 * sizeof(double2));
    }
    if (L.codes) ln.Zc = (unsigned char *)q;
    int rc = lane_host_buffers(l, k);
    if (rc) return rc;
    ln.t_h = t_pool.t_h[l];
    ln.tg_h = t_pool.tg_h[l];
    ln.terms_h = t_pool.terms_h[l];
    ln.sc_h = t_pool.sc_h[l];
    ln.err_h = t_pool.err_h[l];
    if (nlanes == 1) {
      ln.s = st;
    } else {
      if (!t_pool.s[l]) DTR_CUDA(cudaStreamCreateWithFlags(&t_pool.s[l], cudaStreamNonBlocking));
      ln.s = t_pool.s[l];
    }
  }
  // the solve of each lane runs on its share of the SMs unless the caller fixed the grid
  dtr_solve_params sp = p->solve;
  if (nlanes > 1 && sp.grid == 0) sp.grid = sms / nlanes > 0 ? sms / nlanes : 1;
  auto drain = [&]() {
    for (int l = 0; l < nlanes; ++l) cudaStreamSynchronize(lanes[l].s);
  };

  const int ncols = p->nvec * (p->dilute12 ? 12 : 1);
  const int64_t qoff = p->vec_first * (p->dilute12 ? 12 : 1);  // first probing column of each run
  const int R = p->n_z0;
  const double td = D ? D->td[0] : 0.0;
  const double td_im = D ? D->td[1] : 0.0;
  std::vector<double2> samples((size_t)R * p->nvec, make_double2(0.0, 0.0));
  int64_t iters = 0, nsolves = 0;
  double maxres = 0.0;
  int all_conv = 1;
  int status = DTR_OK;
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
    }
  }
  // Gamma insertion: monomial tables, and T_D^G cached in the deflation handle
  const int ng = p->n_gamma;
  GammaSet gset;
  gset.n = ng;
  unsigned gmask = 0;
  for (int q = 0; q < ng; ++q) {
    if (!gamma_monomial(p->gamma[q], &gset.g[q])) return fail(DTR_EINVAL, "Gamma table is not monomial");
    gmask |= 1u << p->gamma[q];
  }
  if (ng && D) {
    int rc = defl_trace_TD_gamma(const_cast<dtr_defl_s *>(D), gmask, st);
    if (rc) return rc;
  }
  std::vector<double2> gsamples((size_t)ng * R * p->nvec, make_double2(0.0, 0.0));
  std::vector<double> ynorm((size_t)R * p->nvec, 0.0);  // |A^-1 z|^2 per probing vector
  // the lanes start after everything queued on the caller's stream
  if (nlanes > 1) {
    if (!t_pool.start) DTR_CUDA(cudaEventCreateWithFlags(&t_pool.start, cudaEventDisableTiming));
    DTR_CUDA(cudaEventRecord(t_pool.start, st));
    for (int l = 0; l < nlanes; ++l) DTR_CUDA(cudaStreamWaitEvent(lanes[l].s, t_pool.start, 0));
  }
  for (int l = 0; l < nlanes; ++l) {
    DTR_CUDA(cudaMemsetAsync(lanes[l].red.counter, 0, 256, lanes[l].s));
    if (D) DTR_CUDA(cudaMemsetAsync(defl_error_word(lanes[l].defl_work), 0, sizeof(int), lanes[l].s));
  }

  // Enqueue the whole pipeline of one block of probing columns on its lane.
  auto enqueue_block = [&](Lane &ln, int64_t G0) -> int {
    const cudaStream_t s = ln.s;
    const int nb = (int)((R * (int64_t)ncols - G0) < p->block ? (R * (int64_t)ncols - G0) : p->block);
    ln.G0 = G0;
    ln.nb = nb;
    const int64_t q0 = G0 % ncols;
    const bool one_run = q0 + nb <= ncols;
    launch_noise(ln.Z, g, p->seed, p->z0_first, p->ncolors, p->dilute12, G0, ncols, nb, b, s, qoff, ln.Zc);
    DTR_LAUNCH_CHECK("noise");
    if (D) {
      int rc;
      const bool hp_block = hp_ok && one_run && !p->use_x0;
      double2 *Cm = nullptr;
      if (hp_block) {
        // the per-colour sums W of a z0 run serve every block of that run: they are
        // recomputed only when this lane moves to another run (or a Gamma pass
        // overwrote them)
        const int64_t run = p->z0_first + G0 / ncols;
        rc = defl_project_hp(D, sites_dev, p->ncolors, p->seed, run, qoff + q0, nb, p->dilute12, b, ln.d_dev,
                             res->replay ? ln.terms_dev : nullptr, ln.hp_work, L.hp, sms, s, nullptr, &Cm,
                             ln.hp_run == run);
        ln.hp_run = run;
      } else
        rc = defl_project_internal(D, ln.Z, b, ln.d_dev, res->replay ? ln.terms_dev : nullptr,
                                   p->use_x0 ? ln.X : nullptr, &Cm, ln.defl_work, L.defl, sms, s, 1, ln.Zc);
      if (rc) return rc;
      if (ng) {
        // d^G_j = (V^H Gamma^H z_j)^H Lambda^-1 (V^H g5 z_j): the g5 half of this block's C is kept
        DTR_CUDA(cudaMemcpyAsync(ln.Cmain, Cm, sizeof(double2) * (size_t)k * 2 * b, cudaMemcpyDeviceToDevice, s));
        for (int q = 0; q < ng; ++q) {
          double2 *Cg = nullptr;
          if (hp_block) {
            const CodeXform xf = code_xform_gamma_h(gset.g[q]);
            rc = defl_project_hp(D, sites_dev, p->ncolors, p->seed, p->z0_first + G0 / ncols, qoff + q0, nb,
                                 p->dilute12, b, nullptr, nullptr, ln.hp_work, L.hp, sms, s, &xf, &Cg);
            ln.hp_run = -1;
          } else {
            launch_gamma_h(gset.g[q], ln.Z, ln.GZ, g.V, b, s);
            rc = defl_project_internal(D, ln.GZ, b, ln.tg, nullptr, nullptr, &Cg, ln.defl_work, L.defl, sms, s, 1);
          }
          if (rc) return rc;
          launch_defl_d2(D, Cg, ln.Cmain, b, ln.dg + q * 64, s);
        }
      }
    }
    if (!D || !p->use_x0) DTR_CUDA(cudaMemsetAsync(ln.X, 0, (size_t)n * sizeof(double2), s));
    Scal *sc = nullptr;
    int rc = solve_internal(gauge, m0, ln.X, ln.Z, b, &sp, ln.solver_work, L.solver, s, &sc, !D || !p->use_x0,
                            nlanes > 1);
    if (rc) return rc;
    k_zdot<<<reduce_grid(n, sms), kBlock, 0, s>>>(ln.Z, ln.X, n, b, D ? ln.d_dev : nullptr, ln.t_dev, ln.yn_dev,
                                                  ln.red);
    count_launches(1);
    DTR_LAUNCH_CHECK("z^H y reduction");
    for (int q0g = 0; q0g < ng; q0g += 4) {
      k_zdot_gamma<4><<<reduce_grid((int64_t)g.V * b, sms), kBlock, 0, s>>>(
          ln.Z, ln.X, g.V, b, ilog2(b), gset, q0g, D ? ln.dg : nullptr, ln.tg, ln.red);
      count_launches(1);
    }
    if (ng) {
      DTR_LAUNCH_CHECK("z^H Gamma y reduction");
      DTR_CUDA(cudaMemcpyAsync(ln.tg_h, ln.tg, sizeof(double2) * 64 * ng, cudaMemcpyDeviceToHost, s));
    }
    DTR_CUDA(cudaMemcpyAsync(ln.t_h, ln.t_dev, sizeof(double2) * 128, cudaMemcpyDeviceToHost, s));  // t, |y|^2
    DTR_CUDA(cudaMemcpyAsync(ln.sc_h, sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
    if (D && res->replay)
      DTR_CUDA(cudaMemcpyAsync(ln.terms_h, ln.terms_dev, sizeof(double2) * k * b, cudaMemcpyDeviceToHost, s));
    if (nlanes > 1)
      DTR_CUDA(cudaMemcpyAsync(ln.err_h, solver_error_word(ln.solver_work), sizeof(int), cudaMemcpyDeviceToHost, s));
    if (D) DTR_CUDA(cudaMemcpyAsync(ln.err_h + 1, defl_error_word(ln.defl_work), sizeof(int), cudaMemcpyDeviceToHost, s));
    return DTR_OK;
  };
  // Fold one finished block into the host records (in block order: the
  // result does not depend on the lane count).
  auto fold_block = [&](const Lane &ln) {
    for (int jj = 0; jj < ln.nb; ++jj) {
      const int64_t Gc = ln.G0 + jj;
      const int r = (int)(Gc / ncols);
      const int q = (int)(Gc % ncols);
      const int jv = p->dilute12 ? q / 12 : q;
      double2 &sm = samples[(size_t)r * p->nvec + jv];
      sm.x += ln.t_h[jj].x;
      sm.y += ln.t_h[jj].y;
      ynorm[(size_t)r * p->nvec + jv] += ln.t_h[64 + jj].x;
      iters += ln.sc_h->iters[jj];
      const double rel = ln.sc_h->bnorm2[jj] > 0 ? std::sqrt(ln.sc_h->rtrue2[jj] / ln.sc_h->bnorm2[jj]) : 0.0;
      if (rel > maxres || rel != rel) maxres = rel;
      if (!ln.sc_h->conv[jj]) all_conv = 0;
      if (ln.sc_h->flags[jj] & kFlagNaN) status = DTR_ENAN;
      for (int q = 0; q < ng; ++q) {
        double2 &gs_ = gsamples[((size_t)q * R + r) * p->nvec + jv];
        gs_.x += ln.tg_h[q * 64 + jj].x;
        gs_.y += ln.tg_h[q * 64 + jj].y;
      }
      if (res->replay && D) {
        double *rp = res->replay + 2 * (((size_t)r * p->nvec + jv) * k);
        for (int m = 0; m < k; ++m) {
          rp[2 * m] += ln.terms_h[(size_t)jj * k + m].x;
          rp[2 * m + 1] += ln.terms_h[(size_t)jj * k + m].y;
        }
      }
    }
    nsolves += ln.nb;
  };

  // run-major sequence of (run, probing column) pairs, in blocks; a wave puts
  // one block on every lane
  const int64_t total_cols = (int64_t)R * ncols;
  for (int64_t G0 = 0; G0 < total_cols; G0 += (int64_t)nlanes * p->block) {
    int used = 0;
    for (int l = 0; l < nlanes && G0 + (int64_t)l * p->block < total_cols; ++l) {
      const int rc = enqueue_block(lanes[l], G0 + (int64_t)l * p->block);
      if (rc) {
        drain();
        return rc;
      }
      ++used;
    }
    for (int l = 0; l < used; ++l) DTR_CUDA(cudaStreamSynchronize(lanes[l].s));
    for (int l = 0; l < used; ++l) {
      if (nlanes > 1 && *lanes[l].err_h) return fail(DTR_ETIMEOUT, "persistent solver barrier timed out");
      if (D && lanes[l].err_h[1]) return fail(DTR_ETIMEOUT, "tensor-core deflation stage timed out");
      fold_block(lanes[l]);
    }
  }

  // run statistics (host, FP64)
  const RunStats st0 = run_stats(samples.data(), R, p->nvec, td, td_im);
  res->trace[0] = st0.mean.x;
  res->trace[1] = st0.mean.y;
  res->T_D[0] = td;
  res->T_D[1] = td_im;
  res->var_runs = st0.var_runs;
  res->jk_err = st0.jk;
  res->var_samples = st0.var_s;
  res->n_solves = nsolves;
  res->iterations = iters;
  res->max_true_residual = maxres;
  res->all_converged = all_conv;
  const size_t ns = samples.size();
  if (res->samples)
    for (size_t i = 0; i < ns; ++i) {
      res->samples[2 * i] = samples[i].x;
      res->samples[2 * i + 1] = samples[i].y;
    }
  if (res->trace_runs)
    for (int r = 0; r < R; ++r) {
      res->trace_runs[2 * r] = st0.tr[r].x;
      res->trace_runs[2 * r + 1] = st0.tr[r].y;
    }
  {  // E |A^-1 z|^2 = ||A^-1||_F^2 for noise with E z z^H = 1 (Z4, probing, dilution groups summed)
    const size_t nsmp = ynorm.size();
    double m = 0.0;
    for (double v : ynorm) m += v;
    m /= (double)nsmp;
    double v2 = 0.0;
    for (double v : ynorm) v2 += (v - m) * (v - m);
    res->frob2 = m;
    res->frob2_err = nsmp > 1 ? std::sqrt(v2 / (double)(nsmp - 1) / (double)nsmp) : 0.0;
  }
  for (int q = 0; q < ng; ++q) {
    const double gtd = D ? D->tdg[p->gamma[q]][0] : 0.0, gtd_im = D ? D->tdg[p->gamma[q]][1] : 0.0;
    const double2 *gsq = gsamples.data() + (size_t)q * R * p->nvec;
    const RunStats sg = run_stats(gsq, R, p->nvec, gtd, gtd_im);
    res->gamma_trace[2 * q] = sg.mean.x;
    res->gamma_trace[2 * q + 1] = sg.mean.y;
    res->gamma_T_D[2 * q] = gtd;
    res->gamma_T_D[2 * q + 1] = gtd_im;
    res->gamma_var_runs[q] = sg.var_runs;
    res->gamma_jk_err[q] = sg.jk;
    if (res->gamma_samples)
      for (size_t i = 0; i < (size_t)R * p->nvec; ++i) {
        res->gamma_samples[2 * ((size_t)q * R * p->nvec + i)] = gsq[i].x;
        res->gamma_samples[2 * ((size_t)q * R * p->nvec + i) + 1] = gsq[i].y;
      }
  }
  if (status == DTR_OK && !all_conv) return fail(DTR_ENOTCONV, "some right-hand sides did not reach tol");
  if (status == DTR_ENAN) return fail(DTR_ENAN, "NaN or Inf in a residual norm");
  return DTR_OK;
}

}  // namespace dtr
