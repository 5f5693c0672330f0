// Learned preconditioner on the tensor cores: the 3^4 convolution as an implicit
// GEMM on tcgen05 (BF16 operands, FP32 accumulation in tensor memory).
//
// Activations between layers are BF16 in a planar layout: for column j, three
// planes of 8-channel chunks, plane c holding channels 8c .. 8c+7 of every site as
// 16 bytes ([j][c][site] of uint4, sites in lexicographic order, x fastest).
//
// A CTA owns an output tile of 8 (x) x 16 (y) sites of one z, one column j, and
// walks along t through a segment of kCvSeg tiles.  For each t it keeps the halo
// slab (x 10, y 18, z 3 sites around the tile, one t) of every chunk in a ring of
// four slab slots in shared memory, so a tile loads one new slab, not three.  In
// a slab the sites of one chunk are 16-byte rows with x fastest, so for any
// displacement (dx, dy, dz) the 128 tile sites shifted by it form a K-major
// operand without swizzle: 8 consecutive x rows are a core matrix, the next y row
// is 160 bytes further (stride), the next chunk one plane further (leading).
// Every offset o of the stencil is therefore a K-major A operand (M = 128 sites,
// N = 32 output channels, K = 16 input channels per MMA) whose descriptor just
// starts at the shifted address: no im2col copy.  The 3 x-displacements x 3
// chunks of a (dt, dz, dy) group are 9 K slices; a leading offset of 16 bytes
// makes the second K slice of an MMA the same plane shifted by one site in x, so
// the slices pair into five MMAs per group (135 per tile instead of 162 with one
// offset per pair of MMAs); the planes are stored in the order (chunk 2, chunk 0,
// chunk 1) and the odd slice is paired with a zero block of weights.  The
// weights of all 81 offsets (B, K-major: 8 output-channel rows x 16 bytes per
// core matrix, 24 real rows of 32) stay in shared memory for the whole launch.
//
// Warp roles: warps 0-3 read the accumulators (tcgen05.ld, thread = TMEM lane =
// tile site) and write the output, lane 0 of warp 4 copies the weights (bulk
// copy) and issues the MMAs, warps 5-9 load the halo slabs.  Two accumulator
// buffers let the epilogue of tile t overlap the MMAs of tile t + 1; mbarriers
// order the roles, and every wait is bounded (a wait that runs out sets a shared
// abort flag and an error word; the host reports DTR_ETIMEOUT).
//
// The same kernel runs the backward-data convolution (offsets reflected, weights
// transposed) and multiplies by phi'(h) of the layer below in its epilogue.  The
// weight gradient (k_wgrad_tc) is a second tcgen05 GEMM, over the tile's sites.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "dtr_internal.cuh"
#include "net.cuh"
#include "tc.cuh"

namespace dtr {

constexpr int kCvX = 8, kCvY = 16;                       // output tile (M = 128 sites)
constexpr int kCvHX = kCvX + 2, kCvHY = kCvY + 2;        // halo extents in x, y (z: 3)
constexpr int kCvPlane = 3 * kCvHY * kCvHX * 16;         // 8640 B: one chunk of a slab
constexpr int kCvSlab = 3 * kCvPlane;                    // 25920 B
constexpr int kCvSlots = 4;                              // slab ring
constexpr int kCvSlabItems = 3 * 3 * kCvHY * kCvHX;      // 16-byte rows per slab (1620)
constexpr int kCvWBlk = 32 * 16;                         // B block: 32 output rows x 8 summed channels
constexpr int kCvWGrp = 9 * kCvWBlk;                     // B bytes per (dt, dz, dy) group of 3 offsets
constexpr int kCvWBytes = 27 * kCvWGrp + 512;            // + a zero block
constexpr int kCvSeg = 8;                                // tiles per work item (along t)
constexpr int kCvThreads = 320;
constexpr int kCvLoaders = 160;                          // warps 5-9
constexpr int kCvLoadIters = (kCvSlabItems + kCvLoaders - 1) / kCvLoaders;
constexpr size_t kCvSmem = (size_t)kCvSlots * kCvSlab + kCvWBytes + 256 + 128;

struct ConvTcArgs {
  const uint4 *in;      // planar BF16 input field
  const uint4 *wtc;     // B operand of all offsets (kCvWBytes)
  uint4 *out_planar;    // planar BF16 output (phi applied if act_out), or NULL
  float2 *out_f2;       // FP32 output in the [site][12][b] layout, or NULL
  const uint4 *mask;    // backward: planar phi(h) of the layer below (phi' from its sign), or NULL
  Geom g;
  int b;                // columns
  int act_out;          // apply the leaky ReLU to the planar output
  int act_mask;         // multiply by phi'(mask)
  int nxb, nyb, nseg;   // tiles in x and y, segments along t
  int items;
  int *err;
};

__device__ __forceinline__ int wrapc(int v, int L) {
  v %= L;
  return v < 0 ? v + L : v;
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t bf_pack(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

struct CvItem {
  int x0, y0, z, j, t0, ts;
};

__device__ __forceinline__ CvItem cv_item(const ConvTcArgs &a, int i) {
  CvItem it;
  const int seg = i % a.nseg;
  int r = i / a.nseg;
  it.x0 = (r % a.nxb) * kCvX;
  r /= a.nxb;
  it.y0 = (r % a.nyb) * kCvY;
  r /= a.nyb;
  it.z = r % a.g.L[2];
  it.j = r / a.g.L[2];
  it.t0 = seg * kCvSeg;
  it.ts = a.g.L[3] - it.t0 < kCvSeg ? a.g.L[3] - it.t0 : kCvSeg;
  return it;
}

__global__ void __launch_bounds__(kCvThreads, 1) k_conv_tc(ConvTcArgs a) {
  extern __shared__ unsigned char cv_smem_raw[];
  unsigned char *smem = cv_smem_raw + ((128u - (smem_u32(cv_smem_raw) & 127u)) & 127u);
  unsigned char *slots = smem;
  unsigned char *W = smem + kCvSlots * kCvSlab;
  uint64_t *full = reinterpret_cast<uint64_t *>(W + kCvWBytes);  // a slab has landed (kCvLoaders arrivals)
  uint64_t *empty = full + kCvSlots;                              // MMAs are done with a slab
  uint64_t *accfull = empty + kCvSlots;                           // a tile's MMAs have completed
  uint64_t *accempty = accfull + 2;                               // the epilogue has read a buffer (128)
  uint64_t *wfull = accempty + 2;                                 // weights have landed
  uint64_t *done = wfull + 1;                                     // every MMA has completed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int q = 0; q < kCvSlots; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[q])), "r"(kCvLoaders) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])) : "memory");
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accfull[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&accempty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(wfull)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const Geom &g = a.g;
  int mma_tiles = 0;      // MMA lane: tiles whose MMAs were issued
  bool w_issued = false;  // MMA lane: the weight copy was issued

  if (warp == 4) {
    if (lane == 0) {
      const uint32_t wf = smem_u32(wfull);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wf), "r"(kCvWBytes) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(W)),
          "l"(a.wtc), "r"(kCvWBytes), "r"(wf)
          : "memory");
      w_issued = true;
      // D = FP32, A = B = BF16, both K-major; N = 32, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      const uint32_t sW = smem_u32(W), sZero = sW + 27 * kCvWGrp, sSlots = smem_u32(slots);
      bool ok = mbar_wait_ab(wf, 0u, abort);
      int waited = 0;  // slabs (counted over the CTA's items) whose arrival was awaited
      int nb = 0;      // first slab of the current item
      for (int i = blockIdx.x; ok && i < a.items; i += gridDim.x) {
        const CvItem it = cv_item(a, i);
        for (int k = 0; k < it.ts; ++k) {
          for (; waited < nb + k + 3; ++waited)
            if (!mbar_wait_ab(smem_u32(&full[waited % kCvSlots]), (uint32_t)((waited / kCvSlots) & 1), abort)) {
              ok = false;
              break;
            }
          if (!ok) break;
          const int buf = mma_tiles & 1;
          if (mma_tiles >= 2 &&
              !mbar_wait_ab(smem_u32(&accempty[buf]), (uint32_t)(((mma_tiles >> 1) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(buf * 32);
          // Per (dt, dz, dy) group the 3 x-displacements x 3 chunks are 9 K slices of 8 channels, done
          // in five MMAs: with the leading offset at 16 B the second K slice is the first one's plane
          // shifted by one site in x, so slices (chunk, dx 0) and (chunk, dx 1) pair up for each chunk;
          // (chunk 0, dx 2) pairs with (chunk 1, dx 2) one plane further, and (chunk 2, dx 2) with a
          // zero block of weights.  Descriptors are constant steps from per-tile bases, added to the
          // start-address field (address >> 4 in the low 14 bits: shared addresses stay below 256 KB,
          // so no carry leaves it).
          uint64_t ap[3], aq[3];
#pragma unroll
          for (int dt = 0; dt < 3; ++dt) {
            const uint32_t sa = sSlots + (uint32_t)(((nb + k + dt) % kCvSlots) * kCvSlab);
            ap[dt] = desc_noswz(sa, 16u, kCvHX * 16);
            aq[dt] = desc_noswz(sa, kCvPlane, kCvHX * 16);
          }
          const uint64_t bp = desc_noswz(sW, 512u, 128u);
          const uint64_t bz = desc_noswz(sW + 4096u, sZero - (sW + 4096u), 128u);
          constexpr uint64_t PL = kCvPlane >> 4, GW = kCvWGrp >> 4;
#pragma unroll
          for (int gi = 0; gi < 27; ++gi) {
            const int dy = gi % 3, dz = (gi / 3) % 3, dt = gi / 9;
            const uint64_t ro = (uint64_t)((dz * kCvHY + dy) * kCvHX);  // the group's (dz, dy) row, dx = 0
            const uint64_t wg = (uint64_t)gi * GW;
            const uint64_t adesc[5] = {ap[dt] + ro, ap[dt] + ro + PL, ap[dt] + ro + 2 * PL, aq[dt] + ro + 2 + PL,
                                       aq[dt] + ro + 2};
            const uint64_t bdesc[5] = {bp + wg, bp + wg + 64, bp + wg + 128, bp + wg + 192, bz + wg - (wg << 16)};
#pragma unroll
            for (int q = 0; q < 5; ++q)
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(adesc[q]), "l"(bdesc[q]), "r"(idesc), "r"((gi > 0 || q > 0) ? 1u : 0u)
                  : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&accfull[buf]))
                       : "memory");
          // slab nb + k has served its last tile; after the segment's last tile so have the two above it
          const int rel = k == it.ts - 1 ? 3 : 1;
          for (int q = 0; q < rel; ++q)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[(nb + k + q) % kCvSlots]))
                         : "memory");
          ++mma_tiles;
        }
        nb += it.ts + 2;
      }
      if (mma_tiles > 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
  } else if (warp >= 5) {
    // halo loaders: slab n of the CTA's sequence goes to slot n % 4 once the MMAs are done
    // with slab n - 4
    const int lt = tid - 5 * 32;
    int n = 0;
    bool ok = true;
    // this thread's rows of a slab: shared-memory offset (fixed) and, per item, the input
    // index of the row's site at t = 0 (the slab of t adds t x the 3D volume)
    int soff[kCvLoadIters], gofs[kCvLoadIters];
#pragma unroll
    for (int q = 0; q < kCvLoadIters; ++q) {
      const int idx = lt + q * kCvLoaders;
      const int c = idx / (kCvSlabItems / 3), rem = idx - c * (kCvSlabItems / 3);
      soff[q] = idx < kCvSlabItems ? (c == 2 ? 0 : c + 1) * kCvPlane + rem * 16 : -1;  // planes (chunk 2, 0, 1)
    }
    const int vol3 = g.L[0] * g.L[1] * g.L[2];
    for (int i = blockIdx.x; ok && i < a.items; i += gridDim.x) {
      const CvItem it = cv_item(a, i);
#pragma unroll
      for (int q = 0; q < kCvLoadIters; ++q) {
        const int idx = lt + q * kCvLoaders;
        const int c = idx / (kCvSlabItems / 3), rem = idx - c * (kCvSlabItems / 3);
        const int iz = rem / (kCvHY * kCvHX), rem2 = rem - iz * (kCvHY * kCvHX);
        const int iy = rem2 / kCvHX, ix = rem2 - iy * kCvHX;
        const int xs = wrapc(it.x0 - 1 + ix, g.L[0]), ys = wrapc(it.y0 - 1 + iy, g.L[1]);
        const int zs = wrapc(it.z - 1 + iz, g.L[2]);
        gofs[q] = (it.j * 3 + c) * g.V + xs + g.L[0] * (ys + g.L[1] * zs);
      }
      for (int u = 0; u < it.ts + 2; ++u, ++n) {
        const int slot = n % kCvSlots;
        if (n >= kCvSlots &&
            !mbar_wait_ab(smem_u32(&empty[slot]), (uint32_t)(((n / kCvSlots) - 1) & 1), abort)) {
          ok = false;
          break;
        }
        const int tofs = wrapc(it.t0 - 1 + u, g.L[3]) * vol3;
        unsigned char *base = slots + slot * kCvSlab;
        uint4 v[kCvLoadIters];
#pragma unroll
        for (int q = 0; q < kCvLoadIters; ++q)
          if (soff[q] >= 0) v[q] = __ldg(a.in + (int64_t)gofs[q] + tofs);
#pragma unroll
        for (int q = 0; q < kCvLoadIters; ++q)
          if (soff[q] >= 0) *reinterpret_cast<uint4 *>(base + soff[q]) = v[q];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[slot])) : "memory");
      }
    }
  } else {
    // epilogue: thread = TMEM lane = tile row m = 8 * (y - y0) + (x - x0)
    const int m = warp * 32 + lane;
    const int gy = m >> 3, gx = m & 7;
    int tiles = 0;
    bool ok = true;
    for (int i = blockIdx.x; ok && i < a.items; i += gridDim.x) {
      const CvItem it = cv_item(a, i);
      for (int k = 0; k < it.ts; ++k, ++tiles) {
        const int buf = tiles & 1;
        if (!mbar_wait_ab(smem_u32(&accfull[buf]), (uint32_t)((tiles >> 1) & 1), abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[24];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta)
            : "memory");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
            : "r"(ta + 16u)
            : "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[buf])) : "memory");
        const int xs = it.x0 + gx, ys = it.y0 + gy;
        if (xs >= g.L[0] || ys >= g.L[1]) continue;
        const int site = xs + g.L[0] * (ys + g.L[1] * (it.z + g.L[2] * (it.t0 + k)));
        float h[24];
#pragma unroll
        for (int c = 0; c < 24; ++c) h[c] = __uint_as_float(r[c]);
        if (a.mask && a.act_mask) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const uint4 mk = __ldg(a.mask + ((int64_t)(it.j * 3 + c)) * g.V + site);
            const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (bf_lo(mw[q]) < 0.f) h[8 * c + 2 * q] *= 0.25f;
              if (bf_hi(mw[q]) < 0.f) h[8 * c + 2 * q + 1] *= 0.25f;
            }
          }
        }
        if (a.out_f2) {
          float2 *q = a.out_f2 + (int64_t)site * 12 * a.b + it.j;
#pragma unroll
          for (int d2 = 0; d2 < 12; ++d2) q[(int64_t)d2 * a.b] = make_float2(h[2 * d2], h[2 * d2 + 1]);
        }
        if (a.out_planar) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float x = h[8 * c + q];
              u[q] = (a.act_out && x < 0.f) ? 0.25f * x : x;
            }
            a.out_planar[((int64_t)(it.j * 3 + c)) * g.V + site] =
                make_uint4(bf_pack(u[0], u[1]), bf_pack(u[2], u[3]), bf_pack(u[4], u[5]), bf_pack(u[6], u[7]));
          }
        }
      }
    }
  }
  __syncthreads();
  // drain: the weight copy and every issued MMA complete before shared and tensor
  // memory are given back; any shortfall is an error
  int vote = 1;
  if (tid == 4 * 32) {
    if (w_issued && !mbar_wait(smem_u32(wfull), 0u, kTcBudget)) vote = 0;
    if (mma_tiles > 0 && !mbar_wait(smem_u32(done), 0u, kTcBudget)) vote = 0;
  }
  if (tid == 0 && *abort) vote = 0;
  const bool ok = __syncthreads_and(vote) != 0;
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------- weight gradient
// dW[o][co][ci] = sum over columns j and sites s of g(s, co) a(s + d(o), ci) as a GEMM over K = the
// 128 sites of a tile: D[(dt, ci), co] per spatial displacement (dx, dy, dz).  Both operands are
// MN-major (a 16-byte row holds 8 channels of one site, the 8 sites of an x row are consecutive
// rows): A = the halo slabs of t-1, t, t+1, whose 9 chunk planes are consecutive in shared memory
// (planes 0..8 = (dt, position), 16 B x 8 rows per core matrix; without swizzle the leading offset
// steps along K, here to the next y row 160 B further, and the stride offset along M, here to the
// next chunk plane), M = 128 rows of which 72 are real; B = the tile's
// gradient g (N = 32 columns of which 24 are real).  The slab ring has six positions, the first two
// mirrored behind the last four, so the three slabs of a tile are always contiguous.  27
// displacements x 32 columns exceed the 512 columns of tensor memory: CTAs of class 0 take
// displacements 0-13, class 1 the rest, each accumulating over all of its tiles; a fixed-order
// reduction over the CTAs of a class gives dW.
constexpr int kWgSlotsPhys = 6;
constexpr int kWgGPlane = kCvY * kCvX * 16;              // 2048 B: one chunk of the tile's gradient
constexpr int kWgGBytes = 3 * kWgGPlane;                 // 6 KB per gradient tile
constexpr int kWgDisp0 = 14;                             // displacements of class 0 (class 1: 13)
// A reads up to 15 planes past the first slab of a triple that starts at position 3
constexpr size_t kWgSpan = (size_t)3 * kCvSlab + 16 * kCvPlane;
constexpr size_t kWgSmem = kWgSpan + 1024 + 256 + 128;   // >= 6 slots + 2 gradient tiles (checked below)
static_assert((size_t)kWgSlotsPhys * kCvSlab + 2 * kWgGBytes + 2048 <= kWgSpan + 1024,
              "gradient tiles lie inside the span the A operand may read");

struct WgradTcArgs {
  const uint4 *a;   // planar BF16 layer input
  const uint4 *gp;  // planar BF16 gradient of the layer output
  Geom g;
  int b, nxb, nyb, nseg, items;
  float *part;      // [cta][14 displacements][128 rows][32 columns]
  int *err;
};

__device__ __forceinline__ CvItem wg_item(const WgradTcArgs &a, int i) {
  CvItem it;
  const int seg = i % a.nseg;
  int r = i / a.nseg;
  it.x0 = (r % a.nxb) * kCvX;
  r /= a.nxb;
  it.y0 = (r % a.nyb) * kCvY;
  r /= a.nyb;
  it.z = r % a.g.L[2];
  it.j = r / a.g.L[2];
  it.t0 = seg * kCvSeg;
  it.ts = a.g.L[3] - it.t0 < kCvSeg ? a.g.L[3] - it.t0 : kCvSeg;
  return it;
}

__global__ void __launch_bounds__(kCvThreads, 1) k_wgrad_tc(WgradTcArgs a) {
  extern __shared__ unsigned char wg_smem_raw[];
  unsigned char *smem = wg_smem_raw + ((128u - (smem_u32(wg_smem_raw) & 127u)) & 127u);
  unsigned char *slots = smem;
  unsigned char *G = smem + kWgSlotsPhys * kCvSlab;             // two gradient tiles
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kWgSpan + 1024);
  uint64_t *empty = full + kCvSlots;
  uint64_t *gfull = empty + kCvSlots;
  uint64_t *gempty = gfull + 2;
  uint64_t *done = gempty + 2;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cls = blockIdx.x & 1, ncta = (gridDim.x + 1 - cls) >> 1, cta = blockIdx.x >> 1;
  const int d0 = cls ? kWgDisp0 : 0, nd = cls ? 27 - kWgDisp0 : kWgDisp0;

  if (tid == 0) {
    for (int q = 0; q < kCvSlots; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[q])), "r"(kCvLoaders) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])) : "memory");
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&gfull[q])), "r"(kCvLoaders) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&gempty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the unused rows and columns of the operands read whatever lies in the span: make it finite
  for (int e = tid; e < (int)(kWgSpan / 16); e += kCvThreads)
    reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const Geom &g = a.g;
  int mma_tiles = 0;

  if (warp == 4) {
    if (lane == 0) {
      // D = FP32, A = B = BF16, both MN-major; N = 32, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t sSlots = smem_u32(slots), sG = smem_u32(G);
      bool ok = true;
      int waited = 0, nb = 0;
      for (int i = cta; ok && i < a.items; i += ncta) {
        const CvItem it = wg_item(a, i);
        for (int k = 0; k < it.ts; ++k) {
          for (; waited < nb + k + 3; ++waited)
            if (!mbar_wait_ab(smem_u32(&full[waited % kCvSlots]), (uint32_t)((waited / kCvSlots) & 1), abort)) {
              ok = false;
              break;
            }
          const int gb = mma_tiles & 1;
          if (!ok || !mbar_wait_ab(smem_u32(&gfull[gb]), (uint32_t)((mma_tiles >> 1) & 1), abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // the triple of slabs starts at ring position (nb + k) % 4 and is contiguous (mirrors)
          const uint32_t tri = sSlots + (uint32_t)(((nb + k) % kCvSlots) * kCvSlab);
          const uint32_t gt = sG + (uint32_t)(gb * kWgGBytes);
          // descriptors at displacement 0 and K step 0; the others differ by constant address steps
          // added to the start-address field (shared addresses stay below 256 KB: no carry)
          const uint64_t a00 = desc_noswz(tri, kCvHX * 16, kCvPlane);
          const uint64_t b00 = desc_noswz(gt, kCvX * 16, kWgGPlane);
          for (int dd = 0; dd < nd; ++dd) {
            const int dsp = d0 + dd;
            const int dx = dsp % 3, dy = (dsp / 3) % 3, dz = dsp / 9;
            const uint64_t a0 = a00 + (uint64_t)((dz * kCvHY + dy) * kCvHX + dx);
#pragma unroll
            for (int ks = 0; ks < kCvY / 2; ++ks) {
              const uint64_t ad = a0 + (uint64_t)(ks * 2 * kCvHX);  // two y rows of 160 B per K step
              const uint64_t bd = b00 + (uint64_t)(ks * 2 * kCvX);  // two rows of 8 sites x 16 B
              const uint32_t acc = (mma_tiles > 0 || ks > 0) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(dd * 32)),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&gempty[gb]))
                       : "memory");
          const int rel = k == it.ts - 1 ? 3 : 1;
          for (int q = 0; q < rel; ++q)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[(nb + k + q) % kCvSlots]))
                         : "memory");
          ++mma_tiles;
        }
        nb += it.ts + 2;
      }
      if (mma_tiles > 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
  } else if (warp >= 5) {
    // loaders: per item the slabs t0-1 and t0, then per tile k the slab t0+k+1 and the gradient tile
    const int lt = tid - 5 * 32;
    int n = 0, tiles = 0;
    bool ok = true;
    // this thread's rows of a slab: shared-memory offset (fixed) and, per item, the input index
    // of the row's site at t = 0 (as in k_conv_tc)
    int soff[kCvLoadIters], gofs[kCvLoadIters];
#pragma unroll
    for (int q = 0; q < kCvLoadIters; ++q) {
      const int idx = lt + q * kCvLoaders;
      const int c = idx / (kCvSlabItems / 3), rem = idx - c * (kCvSlabItems / 3);
      soff[q] = idx < kCvSlabItems ? (c == 2 ? 0 : c + 1) * kCvPlane + rem * 16 : -1;
    }
    const int vol3 = g.L[0] * g.L[1] * g.L[2];
    auto item_rows = [&](const CvItem &it) {
#pragma unroll
      for (int q = 0; q < kCvLoadIters; ++q) {
        const int idx = lt + q * kCvLoaders;
        const int c = idx / (kCvSlabItems / 3), rem = idx - c * (kCvSlabItems / 3);
        const int iz = rem / (kCvHY * kCvHX), rem2 = rem - iz * (kCvHY * kCvHX);
        const int iy = rem2 / kCvHX, ix = rem2 - iy * kCvHX;
        const int xs = wrapc(it.x0 - 1 + ix, g.L[0]), ys = wrapc(it.y0 - 1 + iy, g.L[1]);
        const int zs = wrapc(it.z - 1 + iz, g.L[2]);
        gofs[q] = (it.j * 3 + c) * g.V + xs + g.L[0] * (ys + g.L[1] * zs);
      }
    };
    auto load_slab = [&](const CvItem &it, int u) -> bool {
      const int slot = n % kCvSlots;
      if (n >= kCvSlots && !mbar_wait_ab(smem_u32(&empty[slot]), (uint32_t)(((n / kCvSlots) - 1) & 1), abort))
        return false;
      const int tofs = wrapc(it.t0 - 1 + u, g.L[3]) * vol3;
      uint4 v[kCvLoadIters];
#pragma unroll
      for (int q = 0; q < kCvLoadIters; ++q)
        if (soff[q] >= 0) v[q] = __ldg(a.a + (int64_t)gofs[q] + tofs);
#pragma unroll
      for (int q = 0; q < kCvLoadIters; ++q) {
        if (soff[q] >= 0) {
          *reinterpret_cast<uint4 *>(slots + slot * kCvSlab + soff[q]) = v[q];
          if (slot < 2) *reinterpret_cast<uint4 *>(slots + (slot + kCvSlots) * kCvSlab + soff[q]) = v[q];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[slot])) : "memory");
      ++n;
      return true;
    };
    auto load_g = [&](const CvItem &it, int k) -> bool {
      const int gb = tiles & 1;
      if (tiles >= 2 && !mbar_wait_ab(smem_u32(&gempty[gb]), (uint32_t)(((tiles >> 1) - 1) & 1), abort))
        return false;
      const int tt = it.t0 + k;
      for (int idx = lt; idx < 3 * kCvX * kCvY; idx += kCvLoaders) {
        const int c = idx / (kCvX * kCvY), rem = idx - c * (kCvX * kCvY);
        const int gy = rem / kCvX, gx = rem - gy * kCvX;
        const int xs = it.x0 + gx, ys = it.y0 + gy;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);  // sites outside the lattice contribute nothing
        if (xs < g.L[0] && ys < g.L[1])
          v = __ldg(a.gp + ((int64_t)(it.j * 3 + c)) * g.V + (xs + g.L[0] * (ys + g.L[1] * (it.z + g.L[2] * tt))));
        const int pos = c == 2 ? 0 : c + 1;  // the same plane order as the slabs: D columns follow it
        *reinterpret_cast<uint4 *>(G + gb * kWgGBytes + pos * kWgGPlane + rem * 16) = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&gfull[gb])) : "memory");
      ++tiles;
      return true;
    };
    for (int i = cta; ok && i < a.items; i += ncta) {
      const CvItem it = wg_item(a, i);
      item_rows(it);
      ok = load_slab(it, 0) && load_slab(it, 1);
      for (int k = 0; ok && k < it.ts; ++k) ok = load_slab(it, k + 2) && load_g(it, k);
    }
  }
  __syncthreads();
  int vote = 1;
  if (tid == 4 * 32 && mma_tiles > 0 && !mbar_wait(smem_u32(done), 0u, kTcBudget)) vote = 0;
  if (tid == 0 && *abort) vote = 0;
  const bool ok = __syncthreads_and(vote) != 0;
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warps 0-3, thread = TMEM lane = row m; a CTA without tiles writes zeros
  const bool any = __syncthreads_or(mma_tiles > 0) != 0;
  const bool have = ok && any;
  if (warp < 4) {
    const int m = warp * 32 + lane;
    float *out = a.part + ((int64_t)blockIdx.x * kWgDisp0 * 128 + m) * 32;
    for (int dd = 0; dd < nd; ++dd) {
      for (int col = 0; col < 32; col += 16) {
        uint32_t r[16];
        if (have) {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];\n"
              "tcgen05.wait::ld.sync.aligned;\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dd * 32 + col))
              : "memory");
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) r[q] = 0u;
        }
        float4 *o4 = reinterpret_cast<float4 *>(out + (int64_t)dd * 128 * 32 + col);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          o4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                              __uint_as_float(r[4 * q + 3]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// dW[o][co][ci] from the partials of the CTAs of both classes, summed in FP64 in CTA order
__global__ void k_wgrad_tc_reduce(const float *__restrict__ part, int nctas, float *__restrict__ dW) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 81 * 576; e += gridDim.x * blockDim.x) {
    const int o = e / 576, co = (e / 24) % 24, ci = e % 24;
    const int dx = o % 3, dy = (o / 3) % 3, dz = (o / 9) % 3, dt = o / 27;
    const int dsp = (dz * 3 + dy) * 3 + dx;
    const int cls = dsp >= kWgDisp0 ? 1 : 0, dd = dsp - (cls ? kWgDisp0 : 0);
    const int c = ci >> 3, pos = c == 2 ? 0 : c + 1;
    const int m = (dt * 3 + pos) * 8 + (ci & 7);
    const int pc = co >> 3, ppos = pc == 2 ? 0 : pc + 1;
    const int n = ppos * 8 + (co & 7);
    double s = 0.0;
    for (int q = cls; q < nctas; q += 2) s += part[(((int64_t)q * kWgDisp0 + dd) * 128 + m) * 32 + n];
    dW[e] = (float)s;
  }
}

// float2 field [site][12][b] -> planar BF16 [j][c][site] (8 channels per 16 bytes)
__global__ void k_to_planar(const float2 *__restrict__ x, uint4 *__restrict__ p, int V, int b) {
  const int64_t n = (int64_t)V * 3 * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e % V);
    const int64_t r = e / V;
    const int c = (int)(r % 3), j = (int)(r / 3);
    const float2 *q = x + ((int64_t)s * 12 + 4 * c) * b + j;
    const float2 v0 = q[0], v1 = q[b], v2 = q[2 * b], v3 = q[3 * b];
    p[e] = make_uint4(bf_pack(v0.x, v0.y), bf_pack(v1.x, v1.y), bf_pack(v2.x, v2.y), bf_pack(v3.x, v3.y));
  }
}

// master weights [L][o][co][ci] (FP32) -> B operands of the tensor-core convolution, per layer
// kCvWBytes: per (dt, dz, dy) group gi (offsets o = 3 gi + dx), nine blocks of [32 output rows][8 summed
// channels] in the order the MMAs pair them: (dx, chunk) = (0,2) (1,2) (0,0) (1,0) (0,1) (1,1) (2,0)
// (2,1) (2,2); forward: row = co, summed = ci of W[o][co][ci]; backward data: offset reflected
// (o -> 80 - o) and transposed, row = ci, summed = co; rows 24-31 and the trailing block are zero
__global__ void k_refresh_tc(const float *__restrict__ w, unsigned short *__restrict__ wf,
                             unsigned short *__restrict__ wb, int L) {
  const int per = kCvWBytes / 2;  // BF16 elements per layer
  const int bdx[9] = {0, 1, 0, 1, 0, 1, 2, 2, 2}, bch[9] = {2, 2, 0, 0, 1, 1, 0, 1, 2};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * per; e += gridDim.x * blockDim.x) {
    const int l = e / per, r = e % per;
    unsigned short vf = 0, vb = 0;
    if (r < 27 * (kCvWGrp / 2)) {
      const int gi = r / (kCvWGrp / 2), rr = r % (kCvWGrp / 2);
      const int blk = rr / (kCvWBlk / 2), n = (rr / 8) % 32, q = rr % 8;  // block, row, element
      if (n < 24) {
        const int o = 3 * gi + bdx[blk], k = 8 * bch[blk] + q;
        const float *wl = w + (int64_t)l * 81 * 576;
        const __nv_bfloat16 f = __float2bfloat16_rn(wl[(o * 24 + n) * 24 + k]);          // W[o][co=n][ci=k]
        const __nv_bfloat16 bk = __float2bfloat16_rn(wl[((80 - o) * 24 + k) * 24 + n]);  // W[80-o][co=k][ci=n]
        vf = *reinterpret_cast<const unsigned short *>(&f);
        vb = *reinterpret_cast<const unsigned short *>(&bk);
      }
    }
    wf[e] = vf;
    wb[e] = vb;
  }
}

// ------------------------------------------------------------------ host side
static unsigned gsz(int64_t n, int T = 256) {
  int64_t g = (n + T - 1) / T;
  if (g > 65535LL * 8) g = 65535LL * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

size_t net_tc_weight_bytes(int L) { return (size_t)L * kCvWBytes; }

void net_refresh_tc(dtr_net_s *net, cudaStream_t st) {
  k_refresh_tc<<<gsz((int64_t)net->L * kCvWBytes / 2), 256, 0, st>>>(
      net->w, reinterpret_cast<unsigned short *>(net->wtc_f), reinterpret_cast<unsigned short *>(net->wtc_b), net->L);
  count_launches(1);
}

void net_to_planar(const float2 *x, uint4 *p, int64_t V, int b, cudaStream_t st) {
  k_to_planar<<<gsz(V * 3 * b), 256, 0, st>>>(x, p, (int)V, b);
  count_launches(1);
}

void net_conv_tc(const dtr_net_s *net, int layer, bool backward, const uint4 *in, uint4 *out_planar, float2 *out_f2,
                 const uint4 *mask, int act_out, int b, cudaStream_t st) {
  const int sms = device_sms();
  // per call: the attribute belongs to the current device's context
  cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCvSmem);
  ConvTcArgs a;
  a.in = in;
  a.wtc = reinterpret_cast<const uint4 *>((backward ? net->wtc_b : net->wtc_f) + (size_t)layer * kCvWBytes);
  a.out_planar = out_planar;
  a.out_f2 = out_f2;
  a.mask = mask;
  a.g = geom_of(net->lat);
  a.b = b;
  a.act_out = act_out;
  a.act_mask = mask ? net->act : 0;
  a.nxb = (a.g.L[0] + kCvX - 1) / kCvX;
  a.nyb = (a.g.L[1] + kCvY - 1) / kCvY;
  a.nseg = (a.g.L[3] + kCvSeg - 1) / kCvSeg;
  a.items = a.nxb * a.nyb * a.g.L[2] * b * a.nseg;
  a.err = net->err;
  const int grid = a.items < sms ? a.items : sms;
  k_conv_tc<<<grid, kCvThreads, kCvSmem, st>>>(a);
  count_launches(1);
}

size_t net_wgrad_tc_scratch_bytes() { return (size_t)device_sms() * kWgDisp0 * 128 * 32 * sizeof(float); }

void net_wgrad_tc(const dtr_net_s *net, const uint4 *a, const uint4 *gp, int b, float *part, float *dW,
                  cudaStream_t st) {
  const int sms = device_sms();
  cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
  WgradTcArgs w;
  w.a = a;
  w.gp = gp;
  w.g = geom_of(net->lat);
  w.b = b;
  w.nxb = (w.g.L[0] + kCvX - 1) / kCvX;
  w.nyb = (w.g.L[1] + kCvY - 1) / kCvY;
  w.nseg = (w.g.L[3] + kCvSeg - 1) / kCvSeg;
  w.items = w.nxb * w.nyb * w.g.L[2] * b * w.nseg;
  w.part = part;
  w.err = net->err;
  const int grid = sms & ~1;  // an even number of CTAs: both classes alike
  k_wgrad_tc<<<grid, kCvThreads, kWgSmem, st>>>(w);
  k_wgrad_tc_reduce<<<gsz(81 * 576), 256, 0, st>>>(part, grid, dW);
  count_launches(2);
}


}  // namespace dtr
