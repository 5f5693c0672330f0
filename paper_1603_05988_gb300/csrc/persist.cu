// Persistent batched BiCGStab: the whole iteration loop of a block of
// right-hand sides in ONE cooperative launch (one CTA per SM, co-resident),
// with grid-wide barriers instead of kernel boundaries and no host polling.
//
// Per iteration, three phases separated by barriers:
//   P1  v = A p                      partial  rhat^H v                 -> alpha
//   P2  t = A s, s = r - alpha v     partials t^H s, t^H t, rhat^H s,
//       (s formed on the fly at       rhat^H t, s^H s                  -> omega, and
//        neighbours, stored at own    rho' = rhat^H s - omega rhat^H t, |r'|^2 =
//        site)                        s^H s - |t^H s|^2 / t^H t -> beta, convergence
//   P3  x += alpha p + omega s, r = s - omega t, p = r + beta (p - omega v)
// so the r-reduction of textbook BiCGStab folds into the omega reduction.
// Each reduction is finished by the LAST block to reach the barrier: it sums
// the per-block partials in a fixed order (deterministic), runs the scalar
// algebra once per column and only then releases the barrier, so every block
// reads the same scalars afterwards.
//
// Barriers are bounded: a block that waits longer than kSpinBudget clock
// cycles sets an error word and the whole grid leaves the kernel, so a fault
// in co-residency can never hang the GPU; the host turns the error word into
// DTR_ETIMEOUT.  Launch is cooperative (cudaLaunchCooperativeKernel refuses a
// grid that cannot be co-resident).
#include <mutex>
#include <vector>

#include "dslash_core.cuh"
#include "krylov_fin.cuh"
#include "persist.cuh"
#include "reduce.cuh"

namespace dtr {

constexpr long long kSpinBudget = 4000000000LL;  // ~2 s at 2 GHz

// Bounded grid barrier for `expected` blocks; `fin` runs in the last-arriving
// block (all its threads) before the barrier opens.  Returns false if the
// wait exceeded `budget` clock cycles or another block reported an error.
template <class F>
__device__ __forceinline__ bool gsync_n(GridSync *gs, unsigned int expected, long long budget, F &&fin) {
  __shared__ int s_last, s_err;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g0 = *(volatile unsigned int *)&gs->gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gs->count, 1u);
    s_last = (arrived == expected - 1);
    s_err = 0;
    if (!s_last) {
      const long long t0 = clock64();
      while (*(volatile unsigned int *)&gs->gen == g0) {
        if (*(volatile int *)&gs->error) {
          s_err = 1;
          break;
        }
        if (clock64() - t0 > budget) {
          atomicExch(&gs->error, 1);
          s_err = 1;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (s_last) {
    fin();
    __syncthreads();
    if (threadIdx.x == 0) {
      gs->count = 0u;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    }
    __syncthreads();
  }
  return !s_err;
}

template <class F> __device__ __forceinline__ bool gsync(GridSync *gs, F &&fin) {
  return gsync_n(gs, gridDim.x, kSpinBudget, fin);
}

// Self-test: one block waits at a barrier that expects two blocks, so the
// peer never arrives and the bounded wait must give up with the error word set.
__global__ void k_barrier_probe(GridSync *gs, long long budget, int *out) {
  const bool ok = gsync_n(gs, 2u, budget, [] {});
  if (threadIdx.x == 0) out[0] = ok ? 0 : 1;
}

int selftest_barrier(long long budget, int *timed_out, int *error_word, cudaStream_t st) {
  GridSync *gs = nullptr;
  int *out = nullptr;
  DTR_CUDA(cudaMalloc((void **)&gs, sizeof(GridSync) + 64));
  out = (int *)((char *)gs + sizeof(GridSync) + 32);
  cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GridSync) + 64, st);
  if (e == cudaSuccess) {
    k_barrier_probe<<<1, 64, 0, st>>>(gs, budget, out);
    count_launches(1);
    e = cudaGetLastError();
  }
  int h[2] = {0, 0};
  GridSync hs;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h[0], out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, gs, sizeof(GridSync), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(gs);
  if (e != cudaSuccess) return cuda_fail(e, "barrier self-test");
  *timed_out = h[0];
  *error_word = hs.error;
  return DTR_OK;
}

// Reduce NV values per column over the block (fixed tree) into partial[block][q][j].
template <int NV, int T>
__device__ __forceinline__ void block_partial(const double2 (&v)[NV], int b, double2 *__restrict__ partial,
                                              double2 *sh) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q * T + t] = v[q];
  __syncthreads();
  for (int stride = T / 2; stride >= b; stride >>= 1) {
    if (t < stride) {
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[q * T + t] = cadd(sh[q * T + t], sh[q * T + t + stride]);
    }
    __syncthreads();
  }
  if (t < b) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partial[((int64_t)blockIdx.x * NV + q) * b + t] = sh[q * T + t];
    __threadfence();
  }
}

// Last block: tot[q*b + j] = sum over all blocks of partial[blk][q][j], fixed order.
// (A warp-parallel variant with shuffle trees measured slower on GB300 at the
// 8^4 workload: 2.9 vs 2.3 ms per 16-RHS solve.)
template <int NV, int T>
__device__ __forceinline__ void grid_total(int b, const double2 *__restrict__ partial, double2 *sh, double2 *tot) {
  const int t = threadIdx.x;
  const int P = NV * b;
  const int G = gridDim.x;
  if (P > T) {
    for (int p = t; p < P; p += T) {
      const int q = p / b, j = p % b;
      double2 a0 = make_double2(0.0, 0.0);
      for (int blk = 0; blk < G; ++blk) a0 = cadd(a0, __ldcg(&partial[((int64_t)blk * NV + q) * b + j]));
      tot[p] = a0;
    }
    __syncthreads();
    return;
  }
  const int S = T / P;
  const int p = t % P, sl = t / P;
  double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0, a3 = a0;
  if (sl < S) {
    const int q = p / b, j = p % b;
    int blk = sl;
    for (; blk + 3 * S < G; blk += 4 * S) {
      a0 = cadd(a0, __ldcg(&partial[((int64_t)blk * NV + q) * b + j]));
      a1 = cadd(a1, __ldcg(&partial[((int64_t)(blk + S) * NV + q) * b + j]));
      a2 = cadd(a2, __ldcg(&partial[((int64_t)(blk + 2 * S) * NV + q) * b + j]));
      a3 = cadd(a3, __ldcg(&partial[((int64_t)(blk + 3 * S) * NV + q) * b + j]));
    }
    for (; blk < G; blk += S) a0 = cadd(a0, __ldcg(&partial[((int64_t)blk * NV + q) * b + j]));
  }
  const double2 acc = cadd(cadd(a0, a1), cadd(a2, a3));
  __syncthreads();
  sh[t] = acc;
  __syncthreads();
  if (t < P) {
    double2 s = sh[t];
    for (int k = 1; k < S; ++k) s = cadd(s, sh[k * P + t]);
    tot[t] = s;
  }
  __syncthreads();
}

template <typename C> __device__ __forceinline__ C ldcg_scal(const double2 *p) {
  const double2 v = __ldcg(p);
  return mk<C>(v.x, v.y);
}

template <typename R, int T, int WITH_RESID>
__global__ void __launch_bounds__(T, 1) k_bicgstab_persistent(PArgs<R> a) {
  typedef typename cplx_t<R>::type C;
  __shared__ double2 sh[5 * T];
  __shared__ double2 tot[5 * 64];
  const int b = a.b, logb = a.logb;
  const int j = threadIdx.x & (b - 1);
  const int64_t nsite = (int64_t)a.g.V << logb;
  const int64_t nel = nsite * 12;
  const int64_t stride = (int64_t)gridDim.x * T;
  const int64_t t0 = (int64_t)blockIdx.x * T + threadIdx.x;
  Scal *sc = a.sc;
  const int cycles = WITH_RESID ? a.max_cycles : 1;
  int done = 0;

  for (int cycle = 0; cycle < cycles; ++cycle) {
    if (WITH_RESID) {  // r = z - A x ; rhat = p = r ; (||r||^2, ||z||^2) -> restart decision
      double2 acc[1] = {make_double2(0.0, 0.0)};
      for (int64_t it = t0; it < nsite; it += stride) {
        const int s = (int)(it >> logb);
        C o[12], self[12];
        dslash_site<1, R>(a.U, a.x, a.g, b, s, j, a.diag, o, self);
        const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const C zz = a.z[base + c * b];
          const C rr = csub(zz, o[c]);
          a.r[base + c * b] = rr;
          a.rhat[base + c * b] = rr;
          a.p[base + c * b] = rr;
          acc[0].x += (double)rr.x * rr.x + (double)rr.y * rr.y;
          acc[0].y += (double)zz.x * zz.x + (double)zz.y * zz.y;
        }
      }
      block_partial<1, T>(acc, b, a.partial, sh);
      const bool ok = gsync(a.gs, [&] {
        grid_total<1, T>(b, a.partial, sh, tot);
        if (threadIdx.x < b) fin_resid(sc, threadIdx.x, tot[threadIdx.x], 1);
        const int na = __syncthreads_count(threadIdx.x < b && sc->active[threadIdx.x]);
        if (threadIdx.x == 0) sc->n_active = na;
      });
      if (!ok) return;
      if (__ldcg(&sc->n_active) == 0) break;
    }
    for (int iter = 0; iter < a.max_iters; ++iter) {
      ++done;
      if (blockIdx.x == 0 && threadIdx.x == 0) a.gs->iters = done;
      {  // P1: v = A p ; rhat^H v -> alpha   (per-thread sums in R, block/grid sums in FP64)
        R ax = 0, ay = 0;
        for (int64_t it = t0; it < nsite; it += stride) {
          const int s = (int)(it >> logb);
          C o[12], self[12];
          dslash_site<1, R>(a.U, a.p, a.g, b, s, j, a.diag, o, self);
          const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            a.v[base + c * b] = o[c];
            const C rh = a.rhat[base + c * b];
            ax += rh.x * o[c].x + rh.y * o[c].y;
            ay += rh.x * o[c].y - rh.y * o[c].x;
          }
        }
        double2 acc[1] = {make_double2((double)ax, (double)ay)};
        block_partial<1, T>(acc, b, a.partial, sh);
        const bool ok = gsync(a.gs, [&] {
          grid_total<1, T>(b, a.partial, sh, tot);
          if (threadIdx.x < b) fin_alpha(sc, threadIdx.x, tot[threadIdx.x]);
        });
        if (!ok) return;
      }
      {  // P2: t = A s with s = r - alpha v on the fly ; five dots -> omega, beta, convergence
        const C al = ldcg_scal<C>(&sc->alpha[j]);
        AxpyLoad<C> ld{a.r, a.v, al};
        R tsx = 0, tsy = 0, tt = 0, rsx = 0, rsy = 0, rtx = 0, rty = 0, ss = 0;
        for (int64_t it = t0; it < nsite; it += stride) {
          const int s = (int)(it >> logb);
          C o[12], self[12];
          dslash_site_ld<1, R>(a.U, ld, a.g, b, s, j, a.diag, o, self);
          const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            a.t[base + c * b] = o[c];
            a.s[base + c * b] = self[c];
            const C rh = a.rhat[base + c * b];
            tsx += o[c].x * self[c].x + o[c].y * self[c].y;
            tsy += o[c].x * self[c].y - o[c].y * self[c].x;
            tt += o[c].x * o[c].x + o[c].y * o[c].y;
            rsx += rh.x * self[c].x + rh.y * self[c].y;
            rsy += rh.x * self[c].y - rh.y * self[c].x;
            rtx += rh.x * o[c].x + rh.y * o[c].y;
            rty += rh.x * o[c].y - rh.y * o[c].x;
            ss += self[c].x * self[c].x + self[c].y * self[c].y;
          }
        }
        double2 acc[5] = {make_double2((double)tsx, (double)tsy), make_double2((double)tt, 0.0),
                          make_double2((double)rsx, (double)rsy), make_double2((double)rtx, (double)rty),
                          make_double2((double)ss, 0.0)};
        block_partial<5, T>(acc, b, a.partial, sh);
        const bool ok = gsync(a.gs, [&] {
          grid_total<5, T>(b, a.partial, sh, tot);
          if (threadIdx.x < b)
            fin_omega_beta(sc, threadIdx.x, tot[threadIdx.x], tot[b + threadIdx.x], tot[2 * b + threadIdx.x],
                           tot[3 * b + threadIdx.x], tot[4 * b + threadIdx.x]);
          const int na = __syncthreads_count(threadIdx.x < b && sc->active[threadIdx.x]);
          if (threadIdx.x == 0) sc->n_active = na;
        });
        if (!ok) return;
      }
      {  // P3: x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
        const C al = ldcg_scal<C>(&sc->alpha[j]);
        const C om = ldcg_scal<C>(&sc->omega[j]);
        const C be = ldcg_scal<C>(&sc->beta[j]);
        const bool act = __ldcg(&sc->active[j]) != 0;
        for (int64_t e = t0; e < nel; e += stride) {
          const C sv = a.s[e];
          const C pv = a.p[e];
          a.x[e] = caxpy(om, sv, caxpy(al, pv, a.x[e]));
          const C rn = caxpy(cneg(om), a.t[e], sv);
          a.r[e] = rn;
          if (act) a.p[e] = caxpy(be, caxpy(cneg(om), a.v[e], pv), rn);
        }
        const bool stop = __ldcg(&sc->n_active) == 0;
        if (stop && !WITH_RESID) break;  // kernel exit orders these writes for the host
        const bool ok = gsync(a.gs, [] {});  // p (and x for the residual phase) read at neighbours next
        if (!ok) return;
        if (stop) break;
      }
    }
  }
}

// ----------------------------------------------------------- launch profile
struct PendingLaunch {
  cudaEvent_t e0, e1;
  GridSync *gs;
  double site_rhs;
};
static PersistProfile g_prof = {false, 0.0, 0, 0.0};
static std::vector<PendingLaunch> g_pending;
static std::mutex g_prof_mu;

PersistProfile &persist_profile() { return g_prof; }

void persist_profile_flush(cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  for (auto &pl : g_pending) {
    float ms = 0.f;
    GridSync h;
    if (cudaEventElapsedTime(&ms, pl.e0, pl.e1) == cudaSuccess &&
        cudaMemcpy(&h, pl.gs, sizeof(GridSync), cudaMemcpyDeviceToHost) == cudaSuccess) {
      g_prof.ms += ms;
      g_prof.launches += 1;
      g_prof.site_rhs_iters += (double)h.iters * pl.site_rhs;
    }
    cudaEventDestroy(pl.e0);
    cudaEventDestroy(pl.e1);
  }
  g_pending.clear();
  (void)st;
}

template <typename R, int T, int W> static int launch_one(const PArgs<R> &pa, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab_persistent<R, T, W>, T, 0);
    if (e != cudaSuccess) return cuda_fail(e, "persistent solver occupancy");
    if (nb < 1) return fail(DTR_ECUDA, "persistent solver cannot be resident");
    max_grid = nb * device_sms();
    if (max_grid > kMaxGrid) max_grid = kMaxGrid;
  }
  const int grid = (pa.grid > 0 && pa.grid < max_grid) ? pa.grid : max_grid;
  PArgs<R> copy = pa;
  void *args[] = {&copy};
  PendingLaunch pl;
  const bool prof = g_prof.on;
  if (prof) {
    DTR_CUDA(cudaEventCreate(&pl.e0));
    DTR_CUDA(cudaEventCreate(&pl.e1));
    DTR_CUDA(cudaEventRecord(pl.e0, st));
  }
  DTR_CUDA(cudaLaunchCooperativeKernel((const void *)k_bicgstab_persistent<R, T, W>, dim3(grid), dim3(T), args, 0,
                                       st));
  count_launches(1);
  if (prof) {
    DTR_CUDA(cudaEventRecord(pl.e1, st));
    pl.gs = pa.gs;
    pl.site_rhs = (double)pa.g.V * pa.b;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_pending.push_back(pl);
  }
  return DTR_OK;
}

template <typename R> int launch_persistent(const PArgs<R> &pa, int with_resid, cudaStream_t st);

template <> int launch_persistent<double>(const PArgs<double> &pa, int with_resid, cudaStream_t st) {
  return with_resid ? launch_one<double, 256, 1>(pa, st) : launch_one<double, 256, 0>(pa, st);
}
template <> int launch_persistent<float>(const PArgs<float> &pa, int with_resid, cudaStream_t st) {
  return with_resid ? launch_one<float, 512, 1>(pa, st) : launch_one<float, 512, 0>(pa, st);
}

}  // namespace dtr
