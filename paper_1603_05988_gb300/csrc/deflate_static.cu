// Allocation-free deflation projection: dtr_deflate_project_static.
//
// Some callers cannot let a library allocate device memory or hand it a
// workspace: for example a host application whose device memory is entirely
// owned by its own pool allocator (so a cudaMalloc would fail or fragment the
// pool), or code that runs where allocation is forbidden by the host program's
// rules (fixed-memory production runs that reserve all device memory up
// front).  For them this entry point computes the same d_j (and optionally the
// coefficients C) as dtr_deflate_project, but keeps its scratch -- the
// per-chunk partial sums and C -- in a file-scope __device__ array of fixed
// size instead of a caller workspace, and calls no allocating routine.
//
// Limits: k <= DTR_STATIC_MAX_K (128) deflation vectors and
// nrhs <= DTR_STATIC_MAX_RHS (16) right-hand sides per call; the array is
// 64 chunks x 128 x 2 x 16 + 128 x 32 + 16 complex doubles (about 4.3 MB) and
// every GPU that loads the library holds it until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host that name
// is only a stand-in, not a device address.  The device address belongs to
// the copy of the module loaded in one CUDA context, and a new context (after
// cudaDeviceReset, or a primary context released and created again) may load
// it elsewhere.  So the address is looked up with cudaGetSymbolAddress on the
// first call made in each context (with that context's device current) and
// cached under the context's unique id (cuCtxGetId), never under the device
// ordinal alone.  That first call in a context should therefore come before
// any stream capture.  All calls share the one array, so calls whose work
// overlaps on the GPU (different streams, different host threads) race; every
// slot a call reads was written earlier in that same call, so nothing needs
// clearing between calls.
//
// Cost: the partial kernel runs 64 site chunks x ceil(k / (4 * 256 / b))
// blocks (at most 128 blocks), each walking V / 64 sites one after another,
// so it uses a fraction of the GPU and is far slower than
// dtr_deflate_project at large lattices (roughly the time to stream V once
// per block row of m values at a few hundred GB/s): it is meant for modest
// problems, within its k <= 128, nrhs <= 16 limits.
#include <cudaTypedefs.h>

#include <mutex>
#include <unordered_map>

#include "deflate.cuh"
#include "dtr_internal.cuh"

namespace dtr {

constexpr int kSChunks = 64;
constexpr int kSBlock = 256;
constexpr int kSMPT = 4;
constexpr size_t kSPartial = (size_t)kSChunks * DTR_STATIC_MAX_K * 2 * DTR_STATIC_MAX_RHS;
constexpr size_t kSC = (size_t)DTR_STATIC_MAX_K * 2 * DTR_STATIC_MAX_RHS;
constexpr size_t kSD = DTR_STATIC_MAX_RHS;

static __device__ __align__(256) double2 g_static_scratch[kSPartial + kSC + kSD];

// partial[((chunk*k + m)*2 + {0: upper spins, 1: lower spins})*b + j]
template <typename VC>
__global__ void __launch_bounds__(kSBlock)
    k_static_partial(const VC *__restrict__ Vd, const double2 *__restrict__ z, int64_t N, int k, int nrhs, int b,
                     int logb, int nsites, int nchunks, double2 *__restrict__ partial) {
  const int G = kSBlock >> logb;
  const int tile = G * kSMPT;
  const int chunk = blockIdx.x % nchunks;
  const int mt = blockIdx.x / nchunks;
  const int j = threadIdx.x & (b - 1);
  const int grp = threadIdx.x >> logb;
  const int s0 = (int)(((int64_t)nsites * chunk) / nchunks);
  const int s1 = (int)(((int64_t)nsites * (chunk + 1)) / nchunks);
  double2 P[kSMPT], Q[kSMPT];
#pragma unroll
  for (int q = 0; q < kSMPT; ++q) P[q] = Q[q] = make_double2(0.0, 0.0);
  for (int s = s0; s < s1; ++s) {
    for (int c = 0; c < 12; ++c) {
      const int64_t i = (int64_t)s * 12 + c;
      const double2 zz = j < nrhs ? z[(int64_t)j * N + i] : make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kSMPT; ++q) {
        const int m = mt * tile + grp + q * G;
        if (m >= k) continue;
        const double2 vv = vload(Vd[i * k + m]);
        const double vx = vv.x, vy = vv.y;
        const double re = vx * zz.x + vy * zz.y, im = vx * zz.y - vy * zz.x;
        if (c < 6) {
          P[q].x += re;
          P[q].y += im;
        } else {
          Q[q].x += re;
          Q[q].y += im;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kSMPT; ++q) {
    const int m = mt * tile + grp + q * G;
    if (m >= k) continue;
    const int64_t base = (((int64_t)chunk * k + m) * 2) * b + j;
    partial[base] = P[q];
    partial[base + b] = Q[q];
  }
}

// C column-major k x 2b; d_j = sum_m conj(C[m,j]) C[m,b+j] / lambda_m
__global__ void k_static_finish(const double2 *__restrict__ partial, const double *__restrict__ inv_lambda, int k,
                                int b, int nchunks, double2 *__restrict__ C, double2 *__restrict__ d) {
  const int j = threadIdx.x;
  if (j >= b) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int m = 0; m < k; ++m) {
    double2 P = make_double2(0.0, 0.0), Q = make_double2(0.0, 0.0);
    for (int ch = 0; ch < nchunks; ++ch) {
      const int64_t base = (((int64_t)ch * k + m) * 2) * b + j;
      P = cadd(P, partial[base]);
      Q = cadd(Q, partial[base + b]);
    }
    const double2 cz = cadd(P, Q), cg = csub(P, Q);
    C[(int64_t)j * k + m] = cz;
    C[(int64_t)(b + j) * k + m] = cg;
    acc = cadd(acc, cscale(cjmul(cz, cg), inv_lambda[m]));
  }
  d[j] = acc;
}

static std::mutex g_static_mu;
static std::unordered_map<unsigned long long, double2 *> g_static_ptr;  // context id -> array address

struct CtxEntryPoints {
  PFN_cuCtxGetCurrent_v4000 current = nullptr;
  PFN_cuCtxGetId_v12000 id = nullptr;
};

static const CtxEntryPoints &ctx_entry_points() {
  static CtxEntryPoints ep;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      ep.current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      ep.id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  });
  return ep;
}

// Device address of g_static_scratch in the current context, looked up once
// per context (keyed by the context's unique id, so a context created after a
// reset never reuses an address from the old one).
static int static_scratch(double2 **out) {
  const CtxEntryPoints &ep = ctx_entry_points();
  if (!ep.current || !ep.id) {  // no way to name the context: look the address up every call
    void *p = nullptr;
    DTR_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    *out = (double2 *)p;
    return DTR_OK;
  }
  CUcontext ctx = nullptr;
  if (ep.current(&ctx) != CUDA_SUCCESS || !ctx) {
    // no context bound to this thread yet: the runtime binds the current
    // device's primary context on its first call that needs one
    void *p = nullptr;
    DTR_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    if (ep.current(&ctx) != CUDA_SUCCESS || !ctx) return fail(DTR_ECUDA, "no current CUDA context");
  }
  unsigned long long id = 0;
  if (ep.id(ctx, &id) != CUDA_SUCCESS) return fail(DTR_ECUDA, "cuCtxGetId failed");
  std::lock_guard<std::mutex> lock(g_static_mu);
  auto it = g_static_ptr.find(id);
  if (it == g_static_ptr.end()) {
    void *p = nullptr;
    DTR_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    it = g_static_ptr.emplace(id, (double2 *)p).first;
  }
  *out = it->second;
  return DTR_OK;
}

}  // namespace dtr

using namespace dtr;

extern "C" int dtr_deflate_project_static(dtr_defl d, const double *z, int nrhs, double *d_out, double *coeff_out,
                                          void *stream) {
  if (d && d->Ginv) return dtr::fail(DTR_EINVAL, "the allocation-free projection supports the eigenvalue form only "
                                               "(not a Galerkin-corrected deflation space)");
  if (!d || !z || !d_out) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > DTR_STATIC_MAX_RHS)
    return fail(DTR_EINVAL, "dtr_deflate_project_static: nrhs must be in [1, DTR_STATIC_MAX_RHS = 16]");
  if (d->k > DTR_STATIC_MAX_K)
    return fail(DTR_EINVAL, "dtr_deflate_project_static: k above DTR_STATIC_MAX_K = 128");
  double2 *scratch = nullptr;
  int rc = static_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  int logb = 0;
  while ((1 << logb) < b) ++logb;
  const int k = d->k;
  const int64_t V = d->lat.V;
  const int nch = (int)(V < kSChunks ? V : kSChunks);
  const int tiles = (k + (kSBlock / b) * kSMPT - 1) / ((kSBlock / b) * kSMPT);
  double2 *partial = scratch;
  double2 *C = scratch + kSPartial;
  double2 *dd = C + kSC;
  if (d->prec == DTR_F64)
    k_static_partial<double2><<<nch * tiles, kSBlock, 0, st>>>((const double2 *)d->V, (const double2 *)z, d->lat.N, k,
                                                               nrhs, b, logb, (int)V, nch, partial);
  else if (d->prec == DTR_F32)
    k_static_partial<float2><<<nch * tiles, kSBlock, 0, st>>>((const float2 *)d->V, (const double2 *)z, d->lat.N, k,
                                                              nrhs, b, logb, (int)V, nch, partial);
  else
    k_static_partial<bfc2><<<nch * tiles, kSBlock, 0, st>>>((const bfc2 *)d->V, (const double2 *)z, d->lat.N, k,
                                                            nrhs, b, logb, (int)V, nch, partial);
  count_launches(1);
  k_static_finish<<<1, 32, 0, st>>>(partial, d->inv_lambda, k, b, nch, C, dd);
  count_launches(1);
  DTR_LAUNCH_CHECK("static deflation projection");
  DTR_CUDA(cudaMemcpyAsync(d_out, dd, sizeof(double2) * nrhs, cudaMemcpyDeviceToDevice, st));
  if (coeff_out) {
    const size_t colbytes = sizeof(double2) * k;
    DTR_CUDA(cudaMemcpyAsync(coeff_out, C, colbytes * nrhs, cudaMemcpyDeviceToDevice, st));
    DTR_CUDA(cudaMemcpyAsync((char *)coeff_out + colbytes * nrhs, C + (size_t)b * k, colbytes * nrhs,
                             cudaMemcpyDeviceToDevice, st));
  }
  return DTR_OK;
}
