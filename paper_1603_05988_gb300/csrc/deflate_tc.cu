// Deflation contraction on the 5th-generation tensor cores (tcgen05), for a
// deflation space stored in BF16 and Z4-valued probing blocks.
//
// C = V^H [Z, g5 Z] (Section 5.2; Algorithm 1, line 8) is a tall-skinny
// complex contraction over all N dofs.  With V in BF16 and Z in {0, +-1, +-i}
// (exact in BF16) it is a real BF16 GEMM with FP32 accumulation:
//     D[m, n] = sum_K A[m, K] B[n, K],   K = (dof i, re/im c),
//     A[m, (i, c)] = (Re, Im) V[i][m]   -- V's stored BF16 pairs, as they lie
//     B[4j + q, (i, c)]: q = 0 -> (Re z, Im z), q = 1 -> (Im z, -Re z),
//                        q = 2, 3 -> the same times g5(i),  z = Z[i][j]
// so that V^H z_j = D[m, 4j] + i D[m, 4j + 1] and V^H g5 z_j = D[m, 4j + 2] +
// i D[m, 4j + 3].  Each CTA takes one 128-row tile of m and one chunk of dofs
// (split K): its threads stage A and B in shared memory (two stages of 64 dofs,
// eight MMAs of K = 16 each), one thread issues tcgen05.mma with the FP32
// accumulator in tensor memory (TMEM), tcgen05.commit signals an mbarrier when
// a stage's MMAs have read their operands, and the epilogue reads TMEM with
// tcgen05.ld into FP64 partials.  The partials of all chunks are summed in FP64
// in a fixed order (deterministic).
//
// Shared-memory operands are K-major without swizzle: 8 rows x 16 bytes core
// matrices stored contiguously (128 B), the two core matrices of a K = 16 step
// 128 B apart, consecutive 8-row groups 256 B apart.
//
// Every wait is bounded: a stage whose MMAs do not complete within the budget
// sets an error word (the host returns DTR_ETIMEOUT), waits once more, frees
// the TMEM it holds and leaves.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdlib>

#include "deflate.cuh"

namespace dtr {

constexpr int kTcThreads = 256;
constexpr int kTcStageDofs = 64;   // dofs per pipeline stage (8 K-steps of 8 dofs = 16 BF16 values)
constexpr int kTcM = 128;          // rows of m per CTA (MMA M)
constexpr int kTcABytes = kTcM * kTcStageDofs * 2 * 2;  // 128 rows x 128 BF16 = 32 KB per stage
constexpr long long kTcBudget = 2000000000LL;           // ~1 s at 2 GHz

struct TcArgs {
  const bfc2 *V;       // row-major [dof][k]
  const double2 *Z;    // internal [site][12][b] (dof-major, b columns)
  int k, b, logb, N;   // N = MMA N = max(16, 4b); logb = log2 b when b is a power of two, else -1
  int vec4;            // rows of V 16-byte aligned (k % 4 == 0): four m per load
  int64_t ndof;
  int64_t chunk_dofs;  // multiple of kTcStageDofs
  int nchunks, kpad;
  double *part;        // [chunk][kpad][N]
  int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start >> 4, leading (K) byte offset >> 4,
// stride (M/N) byte offset >> 4, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// thread 0 waits, every thread gets its verdict (the whole block takes the same path)
__device__ __forceinline__ bool block_wait(uint32_t addr, uint32_t parity) {
  int okv = 1;
  if (threadIdx.x == 0) okv = mbar_wait(addr, parity, kTcBudget) ? 1 : 0;
  return __syncthreads_and(okv) != 0;
}

// byte offset of operand element (row, kk) within one stage, kk in [0, 128) BF16 of the stage
__device__ __forceinline__ uint32_t op_off(int row, int kk, int rows) {
  const int ks = kk >> 4, kl = kk & 15;
  return (uint32_t)(ks * rows * 32 + (row >> 3) * 256 + (kl >> 3) * 128 + (row & 7) * 16 + (kl & 7) * 2);
}

__device__ __forceinline__ uint32_t pick4(const uint4 &v, int g) {
  return (g & 2) ? ((g & 1) ? v.w : v.z) : ((g & 1) ? v.y : v.x);
}

__device__ __forceinline__ uint32_t bf2_bits(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(kTcThreads, 2) k_defl_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int N = a.N;
  const uint32_t bbytes = (uint32_t)N * kTcStageDofs * 2 * 2;
  const uint32_t stage_bytes = kTcABytes + bbytes;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, chunk = blockIdx.y;
  const int m0 = mt * kTcM;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  const int64_t c0 = (int64_t)chunk * a.chunk_dofs;
  int64_t c1 = c0 + a.chunk_dofs;
  if (c1 > a.ndof) c1 = a.ndof;
  const int nst = c1 > c0 ? (int)((c1 - c0 + kTcStageDofs - 1) / kTcStageDofs) : 0;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  bool ok = true;
  if (4 * a.b < N) {  // rows 4b .. N-1 of B (b < 4) are padding: zero once in both buffers
    for (int idx = tid; idx < 2 * kTcStageDofs * (N - 4 * a.b); idx += kTcThreads) {
      const int per = kTcStageDofs * (N - 4 * a.b);
      const int bf = idx / per, r = idx - bf * per;
      const int dl = r / (N - 4 * a.b), n = 4 * a.b + r % (N - 4 * a.b);
      *reinterpret_cast<uint32_t *>(smem + bf * stage_bytes + kTcABytes + op_off(n, 2 * dl, N)) = 0u;
    }
  }

  for (int s = 0; s < nst && ok; ++s) {
    const int buf = s & 1;
    if (s >= 2) {  // the MMAs of stage s - 2 have read this buffer
      ok = block_wait(smem_u32(&mbar[buf]), (uint32_t)(((s - 2) >> 1) & 1));
      if (!ok) {
        if (tid == 0) atomicExch(a.err, 1);
        break;
      }
    }
    unsigned char *A = smem + buf * stage_bytes;
    unsigned char *B = A + kTcABytes;
    const int64_t d0 = c0 + (int64_t)s * kTcStageDofs;
    // A: unit (dof quad dq, m quad) -> four 16-byte loads (4 m of one dof each), a 4 x 4
    // transpose in registers and four 16-byte stores (4 dofs of one m each: one row of a
    // core matrix).  Lane l stores row 4l + ((f + l/2) mod 4) in its f-th store, so each
    // quarter-warp writes eight distinct rows of a core matrix: no bank conflicts.
    {
      uint4 va[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int dq = warp + 8 * h;
        const int mm = m0 + 4 * lane;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = (int)(d0 + 4 * dq + e);
          va[h][e] = make_uint4(0u, 0u, 0u, 0u);
          if (i < c1) {
            const bfc2 *src = a.V + (int64_t)i * a.k + mm;
            if (a.vec4 && mm + 3 < a.k) {
              va[h][e] = __ldcs(reinterpret_cast<const uint4 *>(src));
            } else {
              uint32_t w4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
              for (int f = 0; f < 4; ++f)
                if (mm + f < a.k) w4[f] = *reinterpret_cast<const uint32_t *>(src + f);
              va[h][e] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int dq = warp + 8 * h;
        unsigned char *Aq = A + (dq >> 1) * (kTcM * 32) + (dq & 1) * 128;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int g = (f + (lane >> 1)) & 3;
          const int m = 4 * lane + g;
          const uint4 w = make_uint4(pick4(va[h][0], g), pick4(va[h][1], g), pick4(va[h][2], g), pick4(va[h][3], g));
          *reinterpret_cast<uint4 *>(Aq + (m >> 3) * 256 + (m & 7) * 16) = w;
        }
      }
    }
    // B: unit (dof quad dq, column j) -> four FP64 probing values, then the four operand
    // rows 4j + q, each one 16-byte store (same rotation of q by j/2 as for A)
    {
      const int r12 = (int)(d0 % 12);
      for (int idx = tid; idx < 16 * a.b; idx += kTcThreads) {
        const int dq = a.logb >= 0 ? idx >> a.logb : idx / a.b, j = idx - dq * a.b;
        double2 zv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = (int)(d0 + 4 * dq + e);
          zv[e] = make_double2(0.0, 0.0);
          if (i < c1) zv[e] = __ldcs(a.Z + (int64_t)i * a.b + j);
        }
        unsigned char *Bq = B + (dq >> 1) * (N * 32) + (dq & 1) * 128;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int q = (f + (j >> 1)) & 3;
          const int n = 4 * j + q;
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float zr = (float)zv[e].x, zi = (float)zv[e].y;
            const float sg = ((q & 2) && (r12 + 4 * dq + e) % 12 >= 6) ? -1.f : 1.f;
            w[e] = (q & 1) ? bf2_bits(sg * zi, -sg * zr) : bf2_bits(sg * zr, sg * zi);
          }
          *reinterpret_cast<uint4 *>(Bq + (n >> 3) * 256 + (n & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(A), sb = smem_u32(B);
#pragma unroll
      for (int ks = 0; ks < kTcStageDofs / 8; ++ks) {
        const uint64_t adesc = mma_desc(sa + (uint32_t)ks * kTcM * 32);
        const uint64_t bdesc = mma_desc(sb + (uint32_t)ks * N * 32);
        const uint32_t acc = (s > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[buf]))
                   : "memory");
    }
  }
  if (ok && nst > 0) {  // all MMAs done (they complete in order)
    const int L = nst - 1;
    ok = block_wait(smem_u32(&mbar[L & 1]), (uint32_t)((L >> 1) & 1));
    if (!ok && tid == 0) atomicExch(a.err, 1);
  }
  if (!ok && nst > 0) {  // let anything still in flight drain before the TMEM is freed
    const int L = nst - 1;
    block_wait(smem_u32(&mbar[L & 1]), (uint32_t)((L >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows m) and half of the N columns
  const int quad = warp & 3, half = warp >> 2;
  const int m = quad * 32 + lane;
  const int halfN = N >> 1;
  double *out = a.part + ((int64_t)chunk * a.kpad + m0 + m) * N;
  for (int col = half * halfN; col < (half + 1) * halfN; col += 8) {
    uint32_t r[8];
    if (ok && nst > 0) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col)
          : "memory");
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = 0u;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) out[col + u] = (double)__uint_as_float(r[u]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// C[col * k + m] from the chunk partials, fixed order over chunks
__global__ void k_defl_tc_reduce(const double *__restrict__ part, int nchunks, int k, int kpad, int b, int N,
                                 double2 *__restrict__ C) {
  const int64_t n = (int64_t)k * 2 * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % k);
    const int col = (int)(e / k);
    const int j = col % b, g5 = col >= b;
    const int nre = 4 * j + (g5 ? 2 : 0);
    double re = 0.0, im = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) {
      const double *p = part + ((int64_t)ch * kpad + m) * N;
      re += p[nre];
      im += p[nre + 1];
    }
    C[e] = make_double2(re, im);
  }
}

static void tc_shape(int64_t ndof, int k, int b, int sms, int *N, int *mtiles, int *nchunks, int64_t *chunk_dofs) {
  *N = 4 * b < 16 ? 16 : 4 * b;
  *mtiles = (k + kTcM - 1) / kTcM;
  const int per_sm = *N <= 64 ? 2 : 1;  // CTAs that fit an SM's shared memory
  int nc = (per_sm * sms + *mtiles - 1) / *mtiles;
  if (nc < 1) nc = 1;
  int64_t cd = (ndof + nc - 1) / nc;
  cd = (cd + kTcStageDofs - 1) / kTcStageDofs * kTcStageDofs;
  *chunk_dofs = cd;
  *nchunks = (int)((ndof + cd - 1) / cd);
}

static std::atomic<unsigned long long> g_tc_calls{0};
unsigned long long defl_tc_calls() { return g_tc_calls.load(std::memory_order_relaxed); }

bool defl_tc_enabled(const dtr_defl_s *D, int b) {
  static int env = -1;
  if (env < 0) {
    const char *e = getenv("DTR_DEFL_TC");
    env = (e && e[0] == '0') ? 0 : 1;
  }
  // dof indices are 32-bit inside the kernel
  return env && D->prec == DTR_BF16 && b >= 1 && b <= 64 && D->lat.N < ((int64_t)1 << 31) - 2 * kTcStageDofs;
}

size_t defl_tc_scratch_bytes(int64_t V, int k, int b, int sms) {
  int N, mt, nc;
  int64_t cd;
  tc_shape(V * 12, k, b, sms, &N, &mt, &nc, &cd);
  return ((size_t)nc * mt * kTcM * N * sizeof(double) + 255) / 256 * 256 + 256;
}

int defl_contract_tc(const dtr_defl_s *D, const double2 *Z, int b, double2 *C, void *scratch, size_t scratch_bytes,
                     int *err_dev, int sms, cudaStream_t st) {
  const int k = D->k;
  const int64_t ndof = D->lat.N;
  int N, mt, nc;
  int64_t cd;
  tc_shape(ndof, k, b, sms, &N, &mt, &nc, &cd);
  if (scratch_bytes < defl_tc_scratch_bytes(D->lat.V, k, b, sms)) return fail(DTR_ENOMEM, "tensor-core scratch too small");
  TcArgs a;
  a.V = (const bfc2 *)D->V;
  a.Z = Z;
  a.k = k;
  a.b = b;
  a.logb = 0;
  while ((1 << a.logb) < b) ++a.logb;
  if ((1 << a.logb) != b) a.logb = -1;
  a.N = N;
  a.vec4 = (k % 4) == 0;
  a.ndof = ndof;
  a.chunk_dofs = cd;
  a.nchunks = nc;
  a.kpad = mt * kTcM;
  a.part = (double *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  a.err = err_dev;
  const size_t smem = 2 * ((size_t)kTcABytes + (size_t)N * kTcStageDofs * 4) + 64;
  DTR_CUDA(cudaFuncSetAttribute(k_defl_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_defl_tc<<<dim3(mt, nc), kTcThreads, smem, st>>>(a);
  count_launches(1);
  g_tc_calls.fetch_add(1, std::memory_order_relaxed);
  const int64_t n = (int64_t)k * 2 * b;
  k_defl_tc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.part, nc, k, a.kpad, b, N, C);
  count_launches(1);
  DTR_LAUNCH_CHECK("tensor-core deflation contraction");
  return DTR_OK;
}

}  // namespace dtr
