// Persistent batched BiCGStab: the whole iteration loop of a block of
// right-hand sides in ONE cooperative launch (one CTA per SM, co-resident),
// with grid-wide barriers instead of kernel boundaries and no host polling.
//
// Per iteration, three phases separated by barriers:
//   P1  v = A p                      partial  rhat^H v                 -> alpha
//   P2  t = A s, s = r - alpha v     partials t^H s, t^H t, rhat^H s,
//       (s formed on the fly at       rhat^H t, s^H s                  -> omega, and
//        neighbours and at the own    rho' = rhat^H s - omega rhat^H t, |r'|^2 =
//        site, never stored)          s^H s - |t^H s|^2 / t^H t -> beta, convergence
//   P3  s = r - alpha v again, x += alpha p + omega s, r = s - omega t,
//       p = r + beta (p - omega v)   (recomputing s from r and v, which P3 reads
//       anyway, saves the write and read of a stored s: one vector pass in 16)
// so the r-reduction of textbook BiCGStab folds into the omega reduction.
//
// Reductions are all-reduce barriers: each block reduces its per-thread sums
// (warp shuffles, then a fixed order over warps) to one partial per value and
// column, arrives at a counting barrier, and once every block has arrived
// EVERY block sums all partials in the same fixed order and runs the scalar
// algebra on its own shared-memory copy of the per-column scalars.  All blocks
// therefore hold bit-identical scalars without a second (release) round trip;
// block 0 writes the scalars back to global memory when the kernel ends.
// Partials are double-buffered by barrier parity: a block can be at most one
// barrier ahead of the slowest block, so it never overwrites partials that
// another block is still reading.
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
#include <cstring>
#include <type_traits>

#include "persist.cuh"
#include "reduce.cuh"

namespace dtr {

constexpr long long kSpinBudget = 4000000000LL;  // ~2 s at 2 GHz
// Largest persistent grid: two buffers of 5 x 64 partials per block fit the
// solver's reduction scratch (kMaxGrid x 5 x 64 double2).
constexpr int kPersistMaxGrid = kMaxGrid / 2;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Counting grid barrier: arrive, then wait until `target` arrivals in total
// (the barrier's sequence number times the grid size).  Returns false if the
// wait exceeded `budget` clock cycles or another block reported an error.
// Ordering without full fences: thread 0 arrives with a release reduction and
// polls with acquire loads; the block barriers before and after extend that to
// the whole block (the writes of the block's threads happen before the
// release, and the acquire happens before their later reads).
__device__ __forceinline__ bool grid_arrive_wait(GridSync *gs, unsigned int target, long long budget) {
  __shared__ int s_err;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_err = 0;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gs->count) : "memory");
    const long long t0 = clock64();
    while (true) {
      unsigned int c;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&gs->count) : "memory");
      if (c >= target) break;
      if (*(volatile int *)&gs->error) {
        s_err = 1;
        break;
      }
      if (clock64() - t0 > budget) {
        atomicExch(&gs->error, 1);
        s_err = 1;
        break;
      }
    }
  }
  __syncthreads();
  return !s_err;
}

// Self-test: one block waits at a barrier that expects two arrivals, so the
// peer never arrives and the bounded wait must give up with the error word set.
__global__ void k_barrier_probe(GridSync *gs, long long budget, int *out) {
  const bool ok = grid_arrive_wait(gs, 2u, budget);
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

// Block sums of NV complex per-thread values (type A) of column
// j = threadIdx.x & (b-1): butterfly over the lanes of one column inside a
// warp, then a fixed-order sum over the warps holding that column; written to
// part[block * NV*b + q*b + j].
template <int NV, int T, typename A>
__device__ __forceinline__ void block_sums(A (&vx)[NV], A (&vy)[NV], int b, typename cplx_t<A>::type *part,
                                           A *shw) {
  typedef typename cplx_t<A>::type CA;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int off = 16; off >= b; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      vx[q] += __shfl_xor_sync(0xffffffffu, vx[q], off);
      vy[q] += __shfl_xor_sync(0xffffffffu, vy[q], off);
    }
  }
  const int bw = b < 32 ? b : 32;  // distinct columns per warp
  if (lane < bw) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      shw[((w * NV + q) * 2 + 0) * 32 + lane] = vx[q];
      shw[((w * NV + q) * 2 + 1) * 32 + lane] = vy[q];
    }
  }
  __syncthreads();
  const int P = NV * b;
  const int cw = b > 32 ? b / 32 : 1;  // warps per full set of columns
  for (int pp = threadIdx.x; pp < P; pp += T) {
    const int q = pp / b, j = pp % b;
    A sx = 0, sy = 0;
    for (int ww = j >> 5; ww < T / 32; ww += cw) {
      sx += shw[((ww * NV + q) * 2 + 0) * 32 + (j & 31)];
      sy += shw[((ww * NV + q) * 2 + 1) * 32 + (j & 31)];
    }
    CA v;
    v.x = sx;
    v.y = sy;
    part[(int64_t)blockIdx.x * P + pp] = v;
  }
  // (ordered for the other blocks by the barrier: __syncthreads, then thread
  // 0's fence before its arrival)
}

// Every block: tot[p] = sum over blocks of part[blk * P + p], fixed order
// (slices of contiguous blocks, 16 independent loads in flight per thread;
// the threads of a warp read consecutive p, so the loads coalesce).  The sums
// run in the partials' own precision: FP32 for the FP32 engine, whose inner
// solve is certified by the FP64 true residual of the outer loop (FP64
// arithmetic runs at 1/64 of the FP32 rate on this part, and every block
// repeats these sums).
template <int T, typename CA>
__device__ __forceinline__ void grid_sums(int P, const CA *__restrict__ part, CA *sh, double2 *tot) {
  typedef decltype(CA().x) A;
  const int t = threadIdx.x;
  const int G = gridDim.x;
  const int S = P <= T ? T / P : 1;
  const int ch = (G + S - 1) / S;
  for (int p0 = 0; p0 < P; p0 += T) {  // one pass unless P > T
    const int pp = p0 + (P <= T ? t % P : t);
    const int sl = P <= T ? t / P : 0;
    A ax = 0, ay = 0;
    if (sl < S && pp < P) {
      const int lo = sl * ch;
      const int hi = min(G, lo + ch);
      const CA *src = part + pp;
      for (int k0 = lo; k0 < hi; k0 += 16) {
        CA v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          if (k0 + u < hi) {
            v[u] = __ldcg(src + (int64_t)(k0 + u) * P);
          } else {
            v[u].x = 0;
            v[u].y = 0;
          }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          ax += v[u].x;
          ay += v[u].y;
        }
      }
    }
    if (P <= T) {
      sh[t].x = ax;
      sh[t].y = ay;
      __syncthreads();
      if (t < P) {
        A sx = sh[t].x, sy = sh[t].y;
        for (int k = 1; k < S; ++k) {
          sx += sh[k * P + t].x;
          sy += sh[k * P + t].y;
        }
        tot[t] = make_double2((double)sx, (double)sy);
      }
      __syncthreads();
    } else if (pp < P) {
      tot[pp] = make_double2((double)ax, (double)ay);
    }
  }
  __syncthreads();
}

template <typename C> __device__ __forceinline__ C mkc(const double2 v) { return mk<C>(v.x, v.y); }

// four complex values stored as S (4 bytes each) in one 16-byte word
template <typename S> __device__ __forceinline__ void unpack4(const uint4 w, float2 (&c)[4]) {
  S h[4];
  memcpy(h, &w, sizeof(w));
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = CStore<S>::ld(h, k);
}
template <typename S> __device__ __forceinline__ uint4 pack4(const float2 (&c)[4]) {
  S h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) CStore<S>::st(h, k, c[k]);
  uint4 w;
  memcpy(&w, h, sizeof(w));
  return w;
}

template <typename R, int T, int WITH_RESID, typename S = typename cplx_t<R>::type>
__global__ void __launch_bounds__(T, 1) k_bicgstab_persistent(PArgs<R, S> a) {
  typedef typename cplx_t<R>::type C;
  typedef CStore<S> SS;
  __shared__ typename cplx_t<R>::type sh[T];
  __shared__ double2 tot[5 * 64];
  __shared__ R shw[(T / 32) * 5 * 2 * 32];
  __shared__ Scal ss;  // this block's copy of the per-column scalars
  const int b = a.b, logb = a.logb;
  const int j = threadIdx.x & (b - 1);
  const int64_t nsite = (int64_t)a.g.V << logb;
  const int64_t nel = nsite * 12;
  const int64_t stride = (int64_t)gridDim.x * T;
  const int64_t t0 = (int64_t)blockIdx.x * T + threadIdx.x;
  const unsigned int G = gridDim.x;
  C *part[2] = {(C *)a.partial, (C *)a.partial + (int64_t)5 * 64 * G};
  unsigned int nbar = 0;  // barriers passed
  if (threadIdx.x == 0) atomicMax(&a.gs->nt0, ~global_ns());
  {
    const int *src = (const int *)a.sc;
    int *dst = (int *)&ss;
    for (int i = threadIdx.x; i < (int)(sizeof(Scal) / sizeof(int)); i += T) dst[i] = __ldcg(src + i);
  }
  __syncthreads();
  const int cycles = WITH_RESID ? a.max_cycles : 1;
  int done = 0;
  bool ok = true;

  for (int cycle = 0; ok && cycle < cycles; ++cycle) {
    if (WITH_RESID) {  // r = z - A x ; rhat = p = r ; (||r||^2, ||z||^2) -> restart decision
      R vx[1] = {0}, vy[1] = {0};
      for (int64_t it = t0; it < nsite; it += stride) {
        const int s = (int)(it >> logb);
        C o[12], self[12];
        dslash_site<1, R>(a.U, a.x, a.g, b, s, j, a.diag, o, self);
        const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const C zz = a.z[base + c * b];
          const C rr = csub(zz, o[c]);
          SS::st(a.r, base + c * b, rr);
          SS::st(a.rhat, base + c * b, rr);
          SS::st(a.p, base + c * b, rr);
          vx[0] += rr.x * rr.x + rr.y * rr.y;
          vy[0] += zz.x * zz.x + zz.y * zz.y;
        }
      }
      C *pb = part[nbar & 1];
      block_sums<1, T, R>(vx, vy, b, pb, shw);
      ok = grid_arrive_wait(a.gs, ++nbar * G, kSpinBudget);
      if (!ok) break;
      grid_sums<T>(b, pb, sh, tot);
      if (threadIdx.x < b) fin_resid(&ss, threadIdx.x, tot[threadIdx.x], 1);
      const int na = __syncthreads_count(threadIdx.x < b && ss.active[threadIdx.x]);
      if (threadIdx.x == 0) ss.n_active = na;
      if (na == 0) break;
    }
    for (int iter = 0; iter < a.max_iters; ++iter) {
      ++done;
      if (blockIdx.x == 0 && threadIdx.x == 0) a.gs->iters = done;
      {  // P1: v = A p ; rhat^H v -> alpha   (per-thread sums in R, block/grid sums in FP64)
        R vx[1] = {0}, vy[1] = {0};
        const PlainLoadS<S, C> ldp{a.p};
        for (int64_t it = t0; it < nsite; it += stride) {
          const int s = (int)(it >> logb);
          C o[12], self[12];
          dslash_site_ld<1, R>(a.U, ldp, a.g, b, s, j, a.diag, o, self);
          const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            SS::st(a.v, base + c * b, o[c]);
            const C rh = SS::ld(a.rhat, base + c * b);
            vx[0] += rh.x * o[c].x + rh.y * o[c].y;
            vy[0] += rh.x * o[c].y - rh.y * o[c].x;
          }
        }
        C *pb = part[nbar & 1];
        block_sums<1, T, R>(vx, vy, b, pb, shw);
        ok = grid_arrive_wait(a.gs, ++nbar * G, kSpinBudget);
        if (!ok) break;
        grid_sums<T>(b, pb, sh, tot);
        if (threadIdx.x < b) fin_alpha(&ss, threadIdx.x, tot[threadIdx.x]);
        __syncthreads();
      }
      int n_active = 0;
      {  // P2: t = A s with s = r - alpha v on the fly ; five dots -> omega, beta, convergence
        const C al = mkc<C>(ss.alpha[j]);
        AxpyLoadS<S, C> ld{a.r, a.v, al};
        R vx[5] = {0, 0, 0, 0, 0}, vy[5] = {0, 0, 0, 0, 0};
        for (int64_t it = t0; it < nsite; it += stride) {
          const int s = (int)(it >> logb);
          C o[12], self[12];
          dslash_site_ld<1, R>(a.U, ld, a.g, b, s, j, a.diag, o, self);
          const int64_t base = (int64_t)s * 12 * b + j;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            SS::st(a.t, base + c * b, o[c]);
            const C rh = SS::ld(a.rhat, base + c * b);
            vx[0] += o[c].x * self[c].x + o[c].y * self[c].y;  // t^H s
            vy[0] += o[c].x * self[c].y - o[c].y * self[c].x;
            vx[1] += o[c].x * o[c].x + o[c].y * o[c].y;        // t^H t
            vx[2] += rh.x * self[c].x + rh.y * self[c].y;      // rhat^H s
            vy[2] += rh.x * self[c].y - rh.y * self[c].x;
            vx[3] += rh.x * o[c].x + rh.y * o[c].y;            // rhat^H t
            vy[3] += rh.x * o[c].y - rh.y * o[c].x;
            vx[4] += self[c].x * self[c].x + self[c].y * self[c].y;  // s^H s
          }
        }
        C *pb = part[nbar & 1];
        block_sums<5, T, R>(vx, vy, b, pb, shw);
        ok = grid_arrive_wait(a.gs, ++nbar * G, kSpinBudget);
        if (!ok) break;
        grid_sums<T>(5 * b, pb, sh, tot);
        if (threadIdx.x < b)
          fin_omega_beta(&ss, threadIdx.x, tot[threadIdx.x], tot[b + threadIdx.x], tot[2 * b + threadIdx.x],
                         tot[3 * b + threadIdx.x], tot[4 * b + threadIdx.x]);
        n_active = __syncthreads_count(threadIdx.x < b && ss.active[threadIdx.x]);
        if (threadIdx.x == 0) ss.n_active = n_active;
      }
      {  // P3: s = r - alpha v ; x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
        // (v is needed wherever alpha != 0, also by a column that converged in this iteration)
        const C al = mkc<C>(ss.alpha[j]);
        const C om = mkc<C>(ss.omega[j]);
        const C be = mkc<C>(ss.beta[j]);
        const C mom = cneg(om), mal = cneg(al);
        const bool act = ss.active[j] != 0;
        const bool nv = act || ss.alpha[j].x != 0.0 || ss.alpha[j].y != 0.0;
        constexpr int U = 4;  // independent elements (or FP32 pairs) in flight per thread
        int64_t e = t0;
        if constexpr (sizeof(R) == 4 && std::is_same<S, float2>::value) {
          if (b >= 2) {  // FP32: two adjacent columns j, j+1 per 16-byte access
          const int j0 = (2 * threadIdx.x) & (b - 1);
          const C al1 = mkc<C>(ss.alpha[j0 + 1]), om1 = mkc<C>(ss.omega[j0 + 1]);
          const C be1 = mkc<C>(ss.beta[j0 + 1]), mom1 = cneg(om1);
          const C al0 = mkc<C>(ss.alpha[j0]), om0 = mkc<C>(ss.omega[j0]);
          const C be0 = mkc<C>(ss.beta[j0]), mom0 = cneg(om0);
          const bool act0 = ss.active[j0] != 0, act1 = ss.active[j0 + 1] != 0;
          const bool nv2 = act0 || act1 || ss.alpha[j0].x != 0.0 || ss.alpha[j0].y != 0.0 ||
                           ss.alpha[j0 + 1].x != 0.0 || ss.alpha[j0 + 1].y != 0.0;
          const C mal0 = cneg(al0), mal1 = cneg(al1);
          const int64_t n2 = nel >> 1;
          float4 *X = (float4 *)a.x, *Rr = (float4 *)a.r, *Pp = (float4 *)a.p;
          const float4 *Tt = (const float4 *)a.t, *Vv = (const float4 *)a.v;
          auto upd = [&](float4 rv, float4 pv, float4 xv, float4 tv, float4 vv, int64_t q) {
            const C s0 = caxpy(mal0, mk<C>(vv.x, vv.y), mk<C>(rv.x, rv.y));
            const C s1 = caxpy(mal1, mk<C>(vv.z, vv.w), mk<C>(rv.z, rv.w));
            const C p0 = mk<C>(pv.x, pv.y), p1 = mk<C>(pv.z, pv.w);
            const C x0 = caxpy(om0, s0, caxpy(al0, p0, mk<C>(xv.x, xv.y)));
            const C x1 = caxpy(om1, s1, caxpy(al1, p1, mk<C>(xv.z, xv.w)));
            X[q] = make_float4(x0.x, x0.y, x1.x, x1.y);
            const C r0 = caxpy(mom0, mk<C>(tv.x, tv.y), s0);
            const C r1 = caxpy(mom1, mk<C>(tv.z, tv.w), s1);
            Rr[q] = make_float4(r0.x, r0.y, r1.x, r1.y);
            if (act0 || act1) {
              const C q0 = act0 ? caxpy(be0, caxpy(mom0, mk<C>(vv.x, vv.y), p0), r0) : p0;
              const C q1 = act1 ? caxpy(be1, caxpy(mom1, mk<C>(vv.z, vv.w), p1), r1) : p1;
              Pp[q] = make_float4(q0.x, q0.y, q1.x, q1.y);
            }
          };
          int64_t f = t0;
          for (; f + (U - 1) * stride < n2; f += U * stride) {
            float4 rv[U], pv[U], xv[U], tv[U], vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int64_t q = f + u * stride;
              rv[u] = Rr[q];
              pv[u] = Pp[q];
              xv[u] = X[q];
              tv[u] = Tt[q];
              vv[u] = nv2 ? Vv[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) upd(rv[u], pv[u], xv[u], tv[u], vv[u], f + u * stride);
          }
          for (; f < n2; f += stride)
            upd(Rr[f], Pp[f], X[f], Tt[f], nv2 ? Vv[f] : make_float4(0.f, 0.f, 0.f, 0.f), f);
          e = nel;  // done
          }
        }
        if constexpr (!std::is_same<S, C>::value) {
          if (b >= 4) {  // half storage: four adjacent columns per 16-byte access; x in FP32
            const int j0 = (4 * threadIdx.x) & (b - 1);
            C al4[4], om4[4], be4[4], mom4[4], mal4[4];
            bool act4[4], any = false, anyv = false;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              al4[w] = mkc<C>(ss.alpha[j0 + w]);
              om4[w] = mkc<C>(ss.omega[j0 + w]);
              be4[w] = mkc<C>(ss.beta[j0 + w]);
              mom4[w] = cneg(om4[w]);
              mal4[w] = cneg(al4[w]);
              act4[w] = ss.active[j0 + w] != 0;
              any = any || act4[w];
              anyv = anyv || act4[w] || ss.alpha[j0 + w].x != 0.0 || ss.alpha[j0 + w].y != 0.0;
            }
            const int64_t n4 = nel >> 2;
            float4 *X = (float4 *)a.x;
            uint4 *Rr = (uint4 *)a.r, *Pp = (uint4 *)a.p;
            const uint4 *Tt = (const uint4 *)a.t, *Vv = (const uint4 *)a.v;
            auto upd = [&](uint4 rw, uint4 pw, float4 xa, float4 xb, uint4 tw, uint4 vw, int64_t q) {
              C sv[4], pv[4], tv[4], vv[4], rn[4], pn[4];
              unpack4<S>(rw, sv);
              unpack4<S>(pw, pv);
              unpack4<S>(tw, tv);
              unpack4<S>(vw, vv);
              C xv[4] = {mk<C>(xa.x, xa.y), mk<C>(xa.z, xa.w), mk<C>(xb.x, xb.y), mk<C>(xb.z, xb.w)};
#pragma unroll
              for (int w = 0; w < 4; ++w) {
                sv[w] = caxpy(mal4[w], vv[w], sv[w]);  // s = r - alpha v
                xv[w] = caxpy(om4[w], sv[w], caxpy(al4[w], pv[w], xv[w]));
                rn[w] = caxpy(mom4[w], tv[w], sv[w]);
                pn[w] = act4[w] ? caxpy(be4[w], caxpy(mom4[w], vv[w], pv[w]), rn[w]) : pv[w];
              }
              X[2 * q] = make_float4(xv[0].x, xv[0].y, xv[1].x, xv[1].y);
              X[2 * q + 1] = make_float4(xv[2].x, xv[2].y, xv[3].x, xv[3].y);
              Rr[q] = pack4<S>(rn);
              if (any) Pp[q] = pack4<S>(pn);
            };
            const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
            int64_t f = t0;
            for (; f + stride < n4; f += 2 * stride) {
              uint4 rw[2], pw[2], tw[2], vw[2];
              float4 xa[2], xb[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int64_t q = f + u * stride;
                rw[u] = Rr[q];
                pw[u] = Pp[q];
                xa[u] = X[2 * q];
                xb[u] = X[2 * q + 1];
                tw[u] = Tt[q];
                vw[u] = anyv ? Vv[q] : zero4;
              }
#pragma unroll
              for (int u = 0; u < 2; ++u) upd(rw[u], pw[u], xa[u], xb[u], tw[u], vw[u], f + u * stride);
            }
            for (; f < n4; f += stride) upd(Rr[f], Pp[f], X[2 * f], X[2 * f + 1], Tt[f], anyv ? Vv[f] : zero4, f);
            e = nel;  // done
          }
        }
        for (; e + (U - 1) * stride < nel; e += U * stride) {
          C sv[U], pv[U], xv[U], tv[U], vv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t q = e + u * stride;
            sv[u] = SS::ld(a.r, q);
            pv[u] = SS::ld(a.p, q);
            xv[u] = a.x[q];
            tv[u] = SS::ld(a.t, q);
            vv[u] = nv ? SS::ld(a.v, q) : mk<C>(0.0, 0.0);
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t q = e + u * stride;
            sv[u] = caxpy(mal, vv[u], sv[u]);  // s = r - alpha v
            a.x[q] = caxpy(om, sv[u], caxpy(al, pv[u], xv[u]));
            const C rn = caxpy(mom, tv[u], sv[u]);
            SS::st(a.r, q, rn);
            if (act) SS::st(a.p, q, caxpy(be, caxpy(mom, vv[u], pv[u]), rn));
          }
        }
        for (; e < nel; e += stride) {
          const C vv = nv ? SS::ld(a.v, e) : mk<C>(0.0, 0.0);
          const C sv = caxpy(mal, vv, SS::ld(a.r, e));
          const C pv = SS::ld(a.p, e);
          a.x[e] = caxpy(om, sv, caxpy(al, pv, a.x[e]));
          const C rn = caxpy(mom, SS::ld(a.t, e), sv);
          SS::st(a.r, e, rn);
          if (act) SS::st(a.p, e, caxpy(be, caxpy(mom, vv, pv), rn));
        }
        const bool stop = n_active == 0;
        if (stop && !WITH_RESID) break;  // kernel exit orders these writes for the host
        ok = grid_arrive_wait(a.gs, ++nbar * G, kSpinBudget);  // p (and x) are read at neighbours next
        if (!ok || stop) break;
      }
    }
  }
  // block 0 publishes the per-column scalars (identical in every block)
  __syncthreads();
  if (blockIdx.x == 0) {
    const int *src = (const int *)&ss;
    int *dst = (int *)a.sc;
    for (int i = threadIdx.x; i < (int)(sizeof(Scal) / sizeof(int)); i += T) dst[i] = src[i];
  }
  if (threadIdx.x == 0) atomicMax(&a.gs->t1, global_ns());
}

// ----------------------------------------------------------- launch profile
struct DevProf {
  unsigned long long launches;
  unsigned long long ns;
  double site_rhs_iters;
};
__device__ DevProf g_devprof;
__device__ unsigned long long g_dev_launches;  // kernels launched inside device-driven graph loops

__global__ void k_persist_account(const GridSync *__restrict__ gs, double site_rhs) {
  if (threadIdx.x == 0) {
    const unsigned long long t0 = ~gs->nt0, t1 = gs->t1;
    atomicAdd(&g_devprof.launches, 1ull);
    atomicAdd(&g_devprof.ns, t1 > t0 ? t1 - t0 : 0ull);
    atomicAdd(&g_devprof.site_rhs_iters, (double)gs->iters * site_rhs);
  }
}

static PersistProfile g_prof = {false, 0.0, 0, 0.0};
static std::mutex g_prof_mu;

PersistProfile &persist_profile() { return g_prof; }

void persist_profile_flush(cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  DevProf h, z = {0, 0, 0.0};
  if (cudaMemcpyFromSymbol(&h, g_devprof, sizeof(DevProf)) != cudaSuccess) return;
  if (cudaMemcpyToSymbol(g_devprof, &z, sizeof(DevProf)) != cudaSuccess) return;
  g_prof.ms += (double)h.ns * 1e-6;
  g_prof.launches += (long long)h.launches;
  g_prof.site_rhs_iters += h.site_rhs_iters;
  (void)st;
}

int persist_account(const GridSync *gs, double site_rhs, cudaStream_t st) {
  k_persist_account<<<1, 32, 0, st>>>(gs, site_rhs);
  count_launches(1);
  DTR_CUDA(cudaGetLastError());
  return DTR_OK;
}

unsigned long long device_launch_count() {
  unsigned long long h = 0;
  if (cudaMemcpyFromSymbol(&h, g_dev_launches, sizeof(h)) != cudaSuccess) return 0;
  return h;
}

unsigned long long *device_launch_counter() {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_dev_launches) != cudaSuccess) return nullptr;
  return (unsigned long long *)p;
}

template <typename R, int T, int W, typename S>
static int launch_one(const PArgs<R, S> &pa, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab_persistent<R, T, W, S>, T, 0);
    if (e != cudaSuccess) return cuda_fail(e, "persistent solver occupancy");
    if (nb < 1) return fail(DTR_ECUDA, "persistent solver cannot be resident");
    max_grid = nb * device_sms();
    if (max_grid > kPersistMaxGrid) max_grid = kPersistMaxGrid;
  }
  const int grid = (pa.grid > 0 && pa.grid < max_grid) ? pa.grid : max_grid;
  PArgs<R, S> copy = pa;
  void *args[] = {&copy};
  DTR_CUDA(cudaLaunchCooperativeKernel((const void *)k_bicgstab_persistent<R, T, W, S>, dim3(grid), dim3(T), args,
                                       0, st));
  count_launches(1);
  if (g_prof.on) return persist_account(pa.gs, (double)pa.g.V * pa.b, st);
  return DTR_OK;
}

template <typename R> int launch_persistent(const PArgs<R> &pa, int with_resid, cudaStream_t st);

template <> int launch_persistent<double>(const PArgs<double> &pa, int with_resid, cudaStream_t st) {
  return with_resid ? launch_one<double, 256, 1, double2>(pa, st) : launch_one<double, 256, 0, double2>(pa, st);
}
template <> int launch_persistent<float>(const PArgs<float> &pa, int with_resid, cudaStream_t st) {
  return with_resid ? launch_one<float, 512, 1, float2>(pa, st) : launch_one<float, 512, 0, float2>(pa, st);
}
template <typename S> int launch_persistent_half(const PArgs<float, S> &pa, cudaStream_t st) {
  return launch_one<float, 512, 0, S>(pa, st);
}
template int launch_persistent_half<__half2>(const PArgs<float, __half2> &, cudaStream_t);
template int launch_persistent_half<__nv_bfloat162>(const PArgs<float, __nv_bfloat162> &, cudaStream_t);

}  // namespace dtr
