// Deflation contraction on the 5th-generation tensor cores (tcgen05), for a
// deflation space stored in BF16 and Z4-valued probing blocks.
//
// C = V^H [Z, g5 Z] (Section 5.2; Algorithm 1's deflation term) is a tall-skinny
// complex contraction over all N dofs.  With V in BF16 and Z in {0, +-1, +-i}
// (exact in BF16) it is a real BF16 GEMM with FP32 accumulation over K = dof:
//     D[r, n] = sum_i A[r, i] B[n, i]
//     A[2m + c, i] = c-th part (Re, Im) of V[i][m]   -- V's stored row, as it lies
//     B[4j + q, i] = Re z, Im z, g5 Re z, g5 Im z  (q = 0..3),  z = Z[i][j]
// so that V^H z_j = (D[2m, 4j] + D[2m+1, 4j+1]) + i (D[2m, 4j+1] - D[2m+1, 4j])
// and the same with columns 4j+2, 4j+3 for g5 z_j.  The block comes either as
// its FP64 values or, when the noise generator wrote them, as one-byte codes
// (z = i^c or 0), so that the kernel reads V plus one byte per entry of Z.
//
// A is MN-major in memory (r contiguous in a row of V), so the tensor memory
// accelerator (TMA) moves it untouched: per stage of 64 dofs, four 64 x 64 boxes
// with the 128-byte swizzle, which is the canonical MN-major SWIZZLE_128B operand
// layout.  B is built in the K-major layout without swizzle from the FP64 probing
// values, with integer operations on their high words (exact for values BF16
// holds; FP64 instructions are scarce on this GPU).  Each CTA takes 256 rows r
// (128 complex m: two M = 128 MMAs per K step, two accumulators in tensor
// memory) and one chunk of dofs (split K), one CTA per SM, with warp roles: a
// lane of warp 0 streams A through a 5-6 stage ring, a lane of warp 1 issues the
// MMAs, warps 2-9 build B into two buffers from probing values loaded two
// stages ahead; full/empty mbarriers
// order them (tcgen05.commit arrives on a stage's empty barrier once its MMAs
// have read their operands).  The epilogue
// reads tensor memory with tcgen05.ld into FP32 partials, which a warp per
// output combines into C and sums over chunks in FP64 in a fixed order
// (deterministic).
//
// Every wait is bounded: a role whose wait exceeds the budget sets a shared
// abort flag that ends the other roles' waits and an error word (the host
// returns DTR_ETIMEOUT); the CTA then waits once more for what it has in
// flight, frees its tensor memory and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <atomic>
#include <cstdlib>
#include <mutex>

#include "deflate.cuh"
#include "tc.cuh"

namespace dtr {

constexpr int kTcThreads = 320;  // warp 0: TMA, warp 1: MMA, warps 2-9: B
constexpr int kTcStageDofs = 64;  // dofs per pipeline stage (four K steps of 16)
constexpr int kTcRows = 256;      // rows r = 2m + c per CTA (two MMAs of M = 128)
constexpr int kTcBox = 64;        // TMA box: 64 BF16 (128 bytes, the swizzle span) x 64 dofs
constexpr int kTcABytes = kTcRows * kTcStageDofs * 2;  // 32 KB per stage
constexpr size_t kTcMaxSmem = 232448;                  // opt-in shared memory per block

struct TcArgs {
  const double2 *Z;    // internal [site][12][b] (dof-major, b columns)
  const unsigned char *Zc;  // or NULL: the same block as one byte per entry (bits 0-1: z = i^c, bit 2: zero),
                            // 16x fewer bytes than the FP64 values
  int k, b, logb, N;   // N = MMA N = 4b rounded up to 16; logb = log2 b when b is a power of two, else -1
  int ndof;            // dof indices fit 32 bits (checked on the host)
  int chunk_dofs;      // multiple of kTcStageDofs
  int kpad;            // rows r of the partials: 256 x row tiles
  float *part;         // [chunk][kpad][N], the FP32 accumulators of each chunk
  int *err;
};

// K-major operand without swizzle: core matrices of 8 rows x 16 bytes, the two core
// matrices of a K step 128 bytes apart (leading), 8-row groups 256 bytes apart (stride)
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr) { return desc_noswz(saddr, 128u, 256u); }

// MN-major operand with the 128-byte swizzle: atoms of 64 BF16 (MN) x 8 rows (K) of
// 1 KB; the next 64 MN elements one TMA box (8 KB) further (leading), the next 8 K
// rows 1 KB further (stride)
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(8192u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// BF16 bits of an FP64 value that BF16 holds exactly (zero, or a normal number with at
// most 8 significant bits, such as the Z4 entries 0, +-1), from the high word of the
// FP64 value alone: sign, exponent rebiased from 1023 to 127, top 7 fraction bits.
// Integer operations only: FP64 instructions are scarce on this GPU.
__device__ __forceinline__ uint32_t bf16_of_exact_f64(uint32_t hi) {
  const uint32_t sign = (hi >> 16) & 0x8000u, mag = hi & 0x7FFFFFFFu;
  const uint32_t bits = sign | ((((mag >> 20) - 1023u + 127u) & 0xFFu) << 7) | ((mag >> 13) & 0x7Fu);
  return mag == 0u ? sign : bits;
}

constexpr int kTcBuilders = kTcThreads - 64;  // warps 2 .. 9 build B

// Warp roles: lane 0 of warp 0 issues the TMA copies of A into an S-stage ring, lane 0
// of warp 1 issues the MMAs, warps 2-9 build B (two buffers) from the probing values
// they load into registers two stages ahead; full/empty mbarriers order the three, so
// no block-wide barrier sits inside the stage loop.  Warps 0-7 run the epilogue.
// UNITS = (dof octet, column) pairs of B per builder thread = ceil(8 b / 256).  NB = B buffers (two:
// four buffers for narrow blocks measured no faster, k = 256 and 1000 at b = 16).
template <int S, int UNITS, int NB>
__global__ void __launch_bounds__(kTcThreads, 1) k_defl_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // the 128-byte swizzle repeats every 1 KB: operand buffers start on a 1 KB boundary
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int N = a.N;
  const uint32_t bbytes = (uint32_t)N * kTcStageDofs * 2;
  unsigned char *Abuf = smem;
  unsigned char *Bbuf = smem + S * kTcABytes;
  uint64_t *afull = reinterpret_cast<uint64_t *>(Bbuf + NB * bbytes);  // A of a stage has landed
  uint64_t *aempty = afull + S;                                        // MMAs have read an A buffer
  uint64_t *bfull = aempty + S;                                        // B of a stage is built
  uint64_t *bempty = bfull + NB;                                       // MMAs have read a B buffer
  uint64_t *accf = bempty + NB;                                        // every MMA has completed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
  int *consumed = reinterpret_cast<int *>(tslot + 2);  // A stages the MMA lane saw land
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rt = blockIdx.x, chunk = blockIdx.y;
  uint32_t ncols = 32;
  while ((int)ncols < 2 * N) ncols <<= 1;

  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < S; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&afull[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&aempty[q])) : "memory");
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bfull[q])), "r"(kTcBuilders) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bempty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(accf)) : "memory");
    *abort = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (4 * a.b < N) {  // rows 4b .. N-1 of B are padding: zero once in every buffer
    const int pad = N - 4 * a.b;
    for (int idx = tid; idx < NB * 8 * pad; idx += kTcThreads) {
      const int bf = idx / (8 * pad), r = idx - bf * 8 * pad;
      const int o = r / pad, n = 4 * a.b + r % pad;
      *reinterpret_cast<uint4 *>(Bbuf + bf * bbytes + (o >> 1) * (N * 32) + (o & 1) * 128 + (n >> 3) * 256 +
                                 (n & 7) * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
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

  const int cbeg = chunk * a.chunk_dofs;
  const int c1 = cbeg + a.chunk_dofs < a.ndof ? cbeg + a.chunk_dofs : a.ndof;
  const int nst = c1 > cbeg ? (c1 - cbeg + kTcStageDofs - 1) / kTcStageDofs : 0;
  const int x0 = rt * kTcRows;  // first BF16 of the rows in a row of V
  int tma_issued = 0;           // producer lane: stages whose copies were issued
  int mma_issued = 0;           // MMA lane: stages whose MMAs were issued

  if (warp == 0) {
    if (lane == 0) {
      // boxes wholly past row 2k are not fetched (their accumulator rows are never read)
      const int nbox = (2 * a.k - x0 + kTcBox - 1) / kTcBox < kTcRows / kTcBox
                           ? (2 * a.k - x0 + kTcBox - 1) / kTcBox
                           : kTcRows / kTcBox;
      for (int st = 0; st < nst; ++st) {
        const int q = st % S;
        if (st >= S && !mbar_wait_ab(smem_u32(&aempty[q]), (uint32_t)((st / S - 1) & 1), abort)) break;
        const uint32_t fb = smem_u32(&afull[q]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                     "r"(nbox * kTcBox * kTcStageDofs * 2)
                     : "memory");
        const uint32_t dst = smem_u32(Abuf + q * kTcABytes);
        const int y = cbeg + st * kTcStageDofs;
        for (int bx = 0; bx < nbox; ++bx)
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
              "%3}], [%4];" ::"r"(dst + bx * (kTcBox * kTcStageDofs * 2)),
              "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x0 + bx * kTcBox), "r"(y), "r"(fb)
              : "memory");
        tma_issued = st + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      for (int s = 0; s < nst; ++s) {
        if (!mbar_wait_ab(smem_u32(&afull[s % S]), (uint32_t)((s / S) & 1), abort)) break;
        *consumed = s + 1;
        if (!mbar_wait_ab(smem_u32(&bfull[s % NB]), (uint32_t)((s / NB) & 1), abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(Abuf + (s % S) * kTcABytes), sb = smem_u32(Bbuf + (s % NB) * bbytes);
#pragma unroll
        for (int ks = 0; ks < kTcStageDofs / 16; ++ks) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint64_t adesc =
                desc_mn_sw128(sa + (uint32_t)h * (2 * kTcBox * kTcStageDofs * 2) + (uint32_t)ks * 2048u);
            const uint64_t bdesc = desc_kmajor(sb + (uint32_t)ks * N * 32);
            const uint32_t acc = (s > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(h * N)),
                "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&aempty[s % S]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bempty[s % NB]))
                     : "memory");
        mma_issued = s + 1;
      }
      // one more commit: accf completes once every MMA issued above has completed
      if (mma_issued > 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accf))
                     : "memory");
    }
  } else {
    // builders: unit (dof octet o, column j) -> rows 4j + q of B, one 16-byte store each
    // (8 dofs of one row: a row of a core matrix); rotating q by j/2 keeps a quarter-warp
    // on eight distinct rows of a core matrix (no bank conflicts)
    const int tb = tid - 64;
    // two register sets of probing values (high words of Re z and Im z, all the BF16
    // operand needs): the loads for stage s + 2 are issued right after stage s is built
    uint2 za[UNITS][8], zb[UNITS][8];
    auto load_Z = [&](int st, uint2 (&zv)[UNITS][8]) {
      const int d0 = cbeg + st * kTcStageDofs;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int idx = tb + u * kTcBuilders;
        const int o = a.logb >= 0 ? idx >> a.logb : idx / a.b, j = idx - o * a.b;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const int i = d0 + 8 * o + g;
          zv[u][g] = make_uint2(0u, a.Zc ? 4u : 0u);
          if (st < nst && idx < 8 * a.b && i < c1) {
            if (a.Zc) {
              zv[u][g] = make_uint2(0u, (uint32_t)__ldcs(a.Zc + (int64_t)i * a.b + j));
            } else {
              const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(a.Z + (int64_t)i * a.b + j));
              zv[u][g] = make_uint2(w.y, w.w);
            }
          }
        }
      }
    };
    // build B of stage s from zv, then reuse zv for the loads of stage s + 2
    auto step = [&](int s, uint2 (&zv)[UNITS][8]) -> bool {
      if (s >= NB && !mbar_wait_ab(smem_u32(&bempty[s % NB]), (uint32_t)(((s / NB) - 1) & 1), abort)) return false;
      const int d0 = cbeg + s * kTcStageDofs;
      const int r12 = d0 % 12;
      unsigned char *B = Bbuf + (s % NB) * bbytes;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int idx = tb + u * kTcBuilders;
        if (idx >= 8 * a.b) continue;
        const int o = a.logb >= 0 ? idx >> a.logb : idx / a.b, j = idx - o * a.b;
        unsigned char *Bq = B + (o >> 1) * (N * 32) + (o & 1) * 128;
        uint32_t re[8], im[8], g5[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          if (a.Zc) {  // code c: z = i^c (bit 0: imaginary, bit 1: negative), bit 2: zero
            const uint32_t c = zv[u][g].y;
            const uint32_t v = ((c & 4u) ? 0u : 0x3F80u) | ((c & 2u) ? 0x8000u : 0u);
            re[g] = (c & 1u) ? 0u : v;
            im[g] = (c & 1u) ? v : 0u;
          } else {
            re[g] = bf16_of_exact_f64(zv[u][g].x);
            im[g] = bf16_of_exact_f64(zv[u][g].y);
          }
          g5[g] = (r12 + 8 * o + g) % 12 >= 6 ? 0x8000u : 0u;  // g5 = -1 on spins 2, 3
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int q = (f + (j >> 1)) & 3;
          const int n = 4 * j + q;
          uint32_t x[8];
#pragma unroll
          for (int g = 0; g < 8; ++g) x[g] = ((q & 1) ? im[g] : re[g]) ^ ((q & 2) ? g5[g] : 0u);
          *reinterpret_cast<uint4 *>(Bq + (n >> 3) * 256 + (n & 7) * 16) =
              make_uint4(x[0] | (x[1] << 16), x[2] | (x[3] << 16), x[4] | (x[5] << 16), x[6] | (x[7] << 16));
        }
      }
      load_Z(s + 2, zv);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull[s % NB])) : "memory");
      return true;
    };
    load_Z(0, za);
    load_Z(1, zb);
    for (int s = 0; s < nst; s += 2) {
      if (!step(s, za)) break;
      if (s + 1 < nst && !step(s + 1, zb)) break;
    }
  }
  __syncthreads();
  // drain: every issued copy lands and every issued MMA completes before the shared
  // and tensor memory are given back; any shortfall is an error
  int vote = 1;
  if (tid == 0) {
    for (int st = *consumed; st < tma_issued; ++st)
      if (!mbar_wait(smem_u32(&afull[st % S]), (uint32_t)((st / S) & 1), kTcBudget)) vote = 0;
  }
  if (tid == 32) {
    if (mma_issued > 0 && !mbar_wait(smem_u32(accf), 0u, kTcBudget)) vote = 0;
    if (mma_issued != nst) vote = 0;
  }
  if (tid == 0 && *abort) vote = 0;
  const bool ok = __syncthreads_and(vote) != 0;
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warps 0-3 read the accumulator of rows 0-127 (columns 0 .. N-1), warps 4-7
  // that of rows 128-255 (columns N .. 2N-1); warp w reads TMEM lanes 32 (w % 4) .. + 31
  const int quad = warp & 3, h = warp >> 2;
  const int r = h * 128 + quad * 32 + lane;
  float *out = a.part + ((int64_t)chunk * a.kpad + x0 + r) * N;
  for (int col = 0; col < (warp < 8 ? N : 0); col += 8) {
    uint32_t v[8];
    if (ok && nst > 0) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(h * N + col))
          : "memory");
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0u;
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2)
      *reinterpret_cast<float2 *>(out + col + u) = make_float2(__uint_as_float(v[u]), __uint_as_float(v[u + 1]));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// C[col * k + m] from the chunk partials (rows r = 2m + c):
// V^H z = (D[2m, re] + D[2m+1, im]) + i (D[2m, im] - D[2m+1, re]), summed in FP64 over
// the chunks by one warp per output: lane l takes chunks l, l + 32, ... in order, then a
// fixed butterfly combines the lanes (the same order on every call: deterministic)
__global__ void k_defl_tc_reduce(const float *__restrict__ part, int nchunks, int k, int kpad, int b, int N,
                                 double2 *__restrict__ C) {
  const int64_t n = (int64_t)k * 2 * b;
  const int lane = threadIdx.x & 31;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int m = (int)(e % k);
    const int col = (int)(e / k);
    const int j = col % b, g5 = col >= b;
    const int nre = 4 * j + (g5 ? 2 : 0);
    double re = 0.0, im = 0.0;
    for (int ch = lane; ch < nchunks; ch += 32) {
      const float2 pr = *reinterpret_cast<const float2 *>(part + ((int64_t)ch * kpad + 2 * m) * N + nre);
      const float2 pi = *reinterpret_cast<const float2 *>(part + ((int64_t)ch * kpad + 2 * m + 1) * N + nre);
      re += (double)pr.x + (double)pi.y;
      im += (double)pr.y - (double)pi.x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) C[e] = make_double2(re, im);
  }
}

static void tc_shape(int64_t ndof, int k, int b, int sms, int *N, int *rtiles, int *nchunks, int *chunk_dofs) {
  *N = (4 * b + 15) / 16 * 16;  // MMA N for M = 128: a multiple of 16 in [16, 256]
  *rtiles = (2 * k + kTcRows - 1) / kTcRows;
  int nc = (sms + *rtiles - 1) / *rtiles;  // one CTA per SM
  if (nc < 1) nc = 1;
  int64_t cd = (ndof + nc - 1) / nc;
  cd = (cd + kTcStageDofs - 1) / kTcStageDofs * kTcStageDofs;
  *chunk_dofs = (int)cd;
  *nchunks = (int)((ndof + cd - 1) / cd);
}

// B buffers for an MMA width N, and the stages of A that fit beside them, the barriers and the
// 1 KB alignment slack
static int tc_bbufs(int /*N*/) { return 2; }
static int tc_stages(int N, size_t *smem) {
  const size_t fixed = (size_t)tc_bbufs(N) * N * kTcStageDofs * 2 + 1024 + 256;
  int S = (int)((kTcMaxSmem - fixed) / kTcABytes);
  if (S > 6) S = 6;
  *smem = (size_t)S * kTcABytes + fixed;
  return S;
}

static std::atomic<unsigned long long> g_tc_calls{0};
unsigned long long defl_tc_calls() { return g_tc_calls.load(std::memory_order_relaxed); }

bool defl_tc_enabled(const dtr_defl_s *D, int b) {
  static int env = -1;
  if (env < 0) {
    const char *e = getenv("DTR_DEFL_TC");
    env = (e && e[0] == '0') ? 0 : 1;
  }
  // rows of V are TMA-addressable when their byte length 4k is a multiple of 16;
  // dof indices are 32-bit inside the kernel
  return env && D->prec == DTR_BF16 && b >= 1 && b <= 64 && D->k % 4 == 0 &&
         D->lat.N < ((int64_t)1 << 31) - 2 * kTcStageDofs;
}

size_t defl_tc_scratch_bytes(int64_t V, int k, int b, int sms) {
  int N, rt, nc, cd;
  tc_shape(V * 12, k, b, sms, &N, &rt, &nc, &cd);
  return ((size_t)nc * rt * kTcRows * N * sizeof(float) + 255) / 256 * 256 + 256;
}

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

int defl_contract_tc(const dtr_defl_s *D, const double2 *Z, int b, double2 *C, void *scratch, size_t scratch_bytes,
                     int *err_dev, int sms, cudaStream_t st, const unsigned char *Zc) {
  const int k = D->k;
  const int64_t ndof = D->lat.N;
  int N, rt, nc, cd;
  tc_shape(ndof, k, b, sms, &N, &rt, &nc, &cd);
  if (scratch_bytes < defl_tc_scratch_bytes(D->lat.V, k, b, sms)) return fail(DTR_ENOMEM, "tensor-core scratch too small");
  if (k % 4 != 0 || ((uintptr_t)D->V & 15u)) return fail(DTR_EINVAL, "deflation rows not TMA-addressable");
  PFN_cuTensorMapEncodeTiled_v12000 encode = tmap_encoder();
  if (!encode) return fail(DTR_ECUDA, "cuTensorMapEncodeTiled unavailable");
  // V as a 2D BF16 tensor: 2k values per row (contiguous), ndof rows 4k bytes apart
  alignas(64) CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)2 * k, (cuuint64_t)ndof};
  const cuuint64_t gstride[1] = {(cuuint64_t)k * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTcBox, (cuuint32_t)kTcStageDofs};
  const cuuint32_t estride[2] = {1, 1};
  if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, D->V, gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return fail(DTR_ECUDA, "cuTensorMapEncodeTiled failed");
  TcArgs a;
  a.Z = Z;
  a.Zc = Zc;
  a.k = k;
  a.b = b;
  a.logb = 0;
  while ((1 << a.logb) < b) ++a.logb;
  if ((1 << a.logb) != b) a.logb = -1;
  a.N = N;
  a.ndof = (int)ndof;
  a.chunk_dofs = cd;
  a.kpad = rt * kTcRows;
  a.part = (float *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  a.err = err_dev;
  size_t smem;
  const int S = tc_stages(N, &smem);
  const int units = (8 * b + kTcBuilders - 1) / kTcBuilders;
  const dim3 grid(rt, nc);
  const int nbb = tc_bbufs(N);
#define DTR_TC_LAUNCH(SS, UU, NN)                                                                                  \
  if (S == SS && units == UU && nbb == NN) {                                                                       \
    DTR_CUDA(cudaFuncSetAttribute(k_defl_tc<SS, UU, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_defl_tc<SS, UU, NN><<<grid, kTcThreads, smem, st>>>(tmap, a);                                                \
  } else
  DTR_TC_LAUNCH(6, 1, 2) DTR_TC_LAUNCH(5, 2, 2) {
    return fail(DTR_EINVAL, "tensor-core contraction: no pipeline for this block width");
  }
#undef DTR_TC_LAUNCH
  count_launches(1);
  g_tc_calls.fetch_add(1, std::memory_order_relaxed);
  const int64_t n = (int64_t)k * 2 * b;  // one warp per output
  k_defl_tc_reduce<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(a.part, nc, k, a.kpad, b, N, C);
  count_launches(1);
  DTR_LAUNCH_CHECK("tensor-core deflation contraction");
  return DTR_OK;
}

}  // namespace dtr
