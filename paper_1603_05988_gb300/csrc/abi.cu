// C-ABI entry points of libdtr (declared in include/dtr.h): argument checks,
// handle management, layout conversion at the boundary and dispatch to the
// kernels.  No exception or trap crosses the boundary; failures return a
// status code and leave a message for dtr_last_error().
#include <atomic>

#include <cuda_bf16.h>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "deflate.cuh"
#include "dtr_internal.cuh"
#include "net.cuh"
#include "persist.cuh"
#include "solver.cuh"

namespace dtr {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

static thread_local int t_capture_depth = 0;  // > 0 while this thread captures a CUDA graph

// Host-side count of kernel launches; launches recorded while capturing a
// graph are not executions and are counted when the graph runs instead.
void count_launches(int n) {
  if (!t_capture_depth) g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}
void capture_begin() { ++t_capture_depth; }
void capture_end() { --t_capture_depth; }

void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return DTR_ECUDA;
}

size_t trace_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p);
size_t eig_workspace_bytes(const dtr_lattice_s &lat, const dtr_eig_params *P);
int eig_solve(const dtr_gauge_s *g, double m0, const dtr_eig_params *P, void *work, size_t work_bytes,
              dtr_defl_s *D, double *res_out, dtr_eig_stats *stats, cudaStream_t st);
int eig_basis_columns(const dtr_eig_params *P);
size_t tune_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p);
int defl_gram(dtr_defl_s *D, const dtr_gauge_s *g, double m0, cudaStream_t st);
int wd_diagnostic(const dtr_lattice_s *lat, const double2 *cols, const int64_t *dofs_host, int ns, int maxd,
                  int ncolors, double *W, cudaStream_t st);
int trace_autotune(const dtr_gauge_s *g, double m0, const dtr_defl_s *D, const dtr_trace_params *p, int reps,
                   int force, void *work, size_t work_bytes, dtr_tune_result *out, cudaStream_t st);
int trace_estimate(const dtr_gauge_s *gauge, double m0, const dtr_defl_s *D, const dtr_trace_params *p, void *work,
                   size_t work_bytes, dtr_trace_result *res, cudaStream_t st);

// round to nearest even, componentwise
__global__ void k_to_bf16(const double2 *__restrict__ a, __nv_bfloat162 *__restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __floats2bfloat162_rn((float)a[i].x, (float)a[i].y);
}

// FP64 links as FP32 hi + lo pairs (hi = nearest FP32, lo = nearest FP32 to the remainder)
__global__ void k_split_links(const double2 *__restrict__ a, float4 *__restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    const float hx = (float)v.x, hy = (float)v.y;
    b[i] = make_float4(hx, (float)(v.x - (double)hx), hy, (float)(v.y - (double)hy));
  }
}

__global__ void k_to_f32(const double2 *__restrict__ a, float2 *__restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

static unsigned grid1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 65535LL * 8) g = 65535LL * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

static int valid_ncolors(int nc) {
  if (nc == 1 || nc == 2) return 1;
  int n = 2;
  while (n < nc) {
    n *= 8;
    if (n == nc) return 1;
    if (n > nc) return 0;
    n *= 2;
    if (n == nc) return 1;
  }
  return 0;
}

static int colour_period(int nc) {
  if (nc == 1) return 1;
  int n = 2, period = 2, level = 0;
  while (n < nc) {
    n *= 8;
    if ((1 << (level + 1)) > period) period = 1 << (level + 1);
    if (n >= nc) break;
    n *= 2;
    period = 1 << (level + 2);
    ++level;
  }
  return period;
}

static int check_colouring(const dtr_lattice_s &l, int ncolors) {
  if (!valid_ncolors(ncolors)) return fail(DTR_EINVAL, "ncolors must be 1, 2, 16, 32, 256, 512, ...");
  const int per = colour_period(ncolors);
  for (int i = 0; i < 4; ++i)
    if (l.dims[i] % per) return fail(DTR_EINVAL, "lattice extents must be multiples of the colouring period");
  return DTR_OK;
}

}  // namespace dtr

using namespace dtr;

extern "C" {

const char *dtr_last_error(void) { return g_err.c_str(); }
const char *dtr_version(void) { return "dtr 0.1 (sm_103a)"; }

int dtr_selftest_barrier(int64_t budget_cycles, int *timed_out, int *error_word, void *stream) {
  if (!timed_out || !error_word || budget_cycles < 1 || budget_cycles > (1LL << 31))
    return fail(DTR_EINVAL, "budget_cycles must be in [1, 2^31] and outputs non-null");
  return selftest_barrier((long long)budget_cycles, timed_out, error_word, (cudaStream_t)stream);
}

int dtr_profile_persistent(int enable, double *ms, int64_t *launches, double *site_rhs_iterations) {
  PersistProfile &p = persist_profile();
  if (p.on) {
    DTR_CUDA(cudaDeviceSynchronize());
    persist_profile_flush(nullptr);
  }
  if (ms) *ms = p.ms;
  if (launches) *launches = p.launches;
  if (site_rhs_iterations) *site_rhs_iterations = p.site_rhs_iters;
  if (enable >= 0) {
    p.on = enable != 0;
    p.ms = 0.0;
    p.launches = 0;
    p.site_rhs_iters = 0.0;
  }
  return DTR_OK;
}

int dtr_graph_stats(uint64_t *captures, uint64_t *launches) {
  if (!captures || !launches) return fail(DTR_EINVAL, "null argument");
  unsigned long long c = 0, l = 0;
  graph_counters(&c, &l);
  *captures = c;
  *launches = l;
  return DTR_OK;
}

uint64_t dtr_kernel_launches(void) {
  return (uint64_t)g_launches.load(std::memory_order_relaxed) + (uint64_t)device_launch_count();
}

int dtr_make_lattice(const int dims[4], dtr_lattice *out) {
  if (!dims || !out) return fail(DTR_EINVAL, "null argument");
  int64_t V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || (dims[i] & 1)) return fail(DTR_EINVAL, "lattice extents must be even and >= 2");
    V *= dims[i];
  }
  if (V > (1LL << 26)) return fail(DTR_EINVAL, "lattice volume above 2^26 sites");
  dtr_lattice_s *l = new (std::nothrow) dtr_lattice_s;
  if (!l) return fail(DTR_ENOMEM, "host allocation failed");
  for (int i = 0; i < 4; ++i) l->dims[i] = dims[i];
  l->V = V;
  l->N = 12 * V;
  *out = l;
  return DTR_OK;
}

void dtr_destroy_lattice(dtr_lattice lat) { delete lat; }

int dtr_lattice_info(dtr_lattice lat, int dims[4], int64_t *volume, int64_t *ndof) {
  if (!lat) return fail(DTR_EINVAL, "null lattice");
  if (dims)
    for (int i = 0; i < 4; ++i) dims[i] = lat->dims[i];
  if (volume) *volume = lat->V;
  if (ndof) *ndof = lat->N;
  return DTR_OK;
}

// Allocate a gauge handle and fill its FP64 links from host memory (links_host
// != NULL) or with the device generator (eps, seed), then derive the FP32,
// double-float split and half-precision copies the kernels read.
static int gauge_create(dtr_lattice lat, const double *links_host, double eps, uint64_t seed, dtr_gauge *out) {
  dtr_gauge_s *g = new (std::nothrow) dtr_gauge_s;
  if (!g) return fail(DTR_ENOMEM, "host allocation failed");
  g->lat = *lat;
  g->U64 = nullptr;
  g->U32 = nullptr;
  g->Ubf16 = nullptr;
  g->Uf16 = nullptr;
  g->Udf = nullptr;
  const int64_t n = lat->V * 4 * 9;
  cudaError_t e = cudaMalloc((void **)&g->U64, n * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void **)&g->U32, n * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&g->Udf, n * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&g->Ubf16, half_links_bytes(lat->V));
  if (e == cudaSuccess) e = cudaMalloc(&g->Uf16, half_links_bytes(lat->V));
  if (e == cudaSuccess) {
    if (links_host) {
      e = cudaMemcpy(g->U64, links_host, n * sizeof(double2), cudaMemcpyHostToDevice);
    } else {
      launch_make_links(g->U64, lat->V, eps, seed, 0);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    k_to_f32<<<grid1d(n), 256>>>(g->U64, g->U32, n); count_launches(1);
    k_split_links<<<grid1d(n), 256>>>(g->U64, (float4 *)g->Udf, n); count_launches(1);
    launch_pack_links_half(g->U64, g->Ubf16, lat->V, 1, 0);
    launch_pack_links_half(g->U64, g->Uf16, lat->V, 0, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(g->U64);
    cudaFree(g->U32);
    cudaFree(g->Ubf16);
    cudaFree(g->Uf16);
    cudaFree(g->Udf);
    delete g;
    return cuda_fail(e, links_host ? "gauge upload" : "gauge generation");
  }
  *out = g;
  return DTR_OK;
}

int dtr_gauge_from_host(dtr_lattice lat, const double *links_host, dtr_gauge *out) {
  if (!lat || !links_host || !out) return fail(DTR_EINVAL, "null argument");
  return gauge_create(lat, links_host, 0.0, 0, out);
}

int dtr_make_gauge(dtr_lattice lat, double eps, uint64_t seed, dtr_gauge *out) {
  if (!lat || !out) return fail(DTR_EINVAL, "null argument");
  if (!(eps >= 0.0) || !(eps <= 100.0)) return fail(DTR_EINVAL, "eps must be in [0, 100]");
  return gauge_create(lat, nullptr, eps, seed, out);
}

int dtr_gauge_to_host(dtr_gauge g, double *links_host) {
  if (!g || !links_host) return fail(DTR_EINVAL, "null argument");
  DTR_CUDA(cudaMemcpy(links_host, g->U64, g->lat.V * 4 * 9 * sizeof(double2), cudaMemcpyDeviceToHost));
  return DTR_OK;
}

void dtr_destroy_gauge(dtr_gauge g) {
  if (!g) return;
  cudaFree(g->U64);
  cudaFree(g->U32);
  cudaFree(g->Ubf16);
  cudaFree(g->Uf16);
  cudaFree(g->Udf);
  delete g;
}

size_t dtr_dslash_workspace_bytes(dtr_lattice lat, int nrhs) {
  if (!lat || nrhs < 1 || nrhs > 64) return 0;
  const int b = pad_rhs(nrhs);
  return 2 * (((size_t)lat->V * 12 * b * sizeof(double2) + 255) / 256 * 256) + 256;
}

int dtr_dslash(dtr_gauge g, double m0, const double *in, double *out, int nrhs, int dagger, dtr_prec prec,
               void *work, size_t work_bytes, void *stream) {
  if (!g || !in || !out || !work) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64) return fail(DTR_EINVAL, "nrhs must be in [1, 64]");
  if (prec != DTR_F64 && prec != DTR_F32 && prec != DTR_BF16 && prec != DTR_F16 && prec != DTR_DF32)
    return fail(DTR_EINVAL, "unknown dslash precision");
  if (prec == DTR_DF32 && dagger) return fail(DTR_EINVAL, "double-float dslash supports dagger = 0 only");
  if ((prec == DTR_BF16 || prec == DTR_F16) && dagger)
    return fail(DTR_EINVAL, "half-precision storage dslash supports dagger = 0 only");
  if ((prec == DTR_BF16 || prec == DTR_F16) && g->lat.V * nrhs * 3 >= (1LL << 31))
    return fail(DTR_EINVAL, "half-precision storage dslash: V * nrhs too large");
  if (work_bytes < dtr_dslash_workspace_bytes(&g->lat, nrhs)) return fail(DTR_ENOMEM, "dslash workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const Geom geo = geom_of(g->lat);
  const size_t vb = ((size_t)g->lat.V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  if (prec == DTR_BF16 || prec == DTR_F16) {
    const int bf = prec == DTR_BF16;
    launch_dslash_half_canon(bf ? g->Ubf16 : g->Uf16, (const double2 *)in, (double2 *)out, w, geo, nrhs, nrhs, m0,
                             bf, st);
  } else if (prec == DTR_DF32) {
    float2 *a = (float2 *)w;
    double2 *o = (double2 *)(w + vb);
    launch_pack<float>((const double2 *)in, a, g->lat.V, nrhs, b, st);
    launch_dslash_df(g->Udf, a, o, geo, b, m0, st);
    launch_unpack<double>(o, (double2 *)out, g->lat.V, nrhs, b, st);
  } else if (prec == DTR_F64) {
    double2 *a = (double2 *)w, *o = (double2 *)(w + vb);
    launch_pack<double>((const double2 *)in, a, g->lat.V, nrhs, b, st);
    launch_dslash<double>(g->U64, a, o, geo, b, m0, dagger, st);
    launch_unpack<double>(o, (double2 *)out, g->lat.V, nrhs, b, st);
  } else {
    float2 *a = (float2 *)w, *o = (float2 *)(w + vb);
    launch_pack<float>((const double2 *)in, a, g->lat.V, nrhs, b, st);
    launch_dslash<float>(g->U32, a, o, geo, b, m0, dagger, st);
    launch_unpack<float>(o, (double2 *)out, g->lat.V, nrhs, b, st);
  }
  DTR_LAUNCH_CHECK("dslash");
  return DTR_OK;
}

int dtr_half_link_rows(void) { return half_link_rows(); }

int dtr_time_dslash(dtr_gauge g, double m0, int nrhs, dtr_prec prec, int reps, void *work, size_t work_bytes,
                    double *avg_ms, void *stream) {
  if (!g || !work || !avg_ms) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64 || reps < 1) return fail(DTR_EINVAL, "nrhs must be in [1, 64] and reps >= 1");
  if (prec != DTR_F64 && prec != DTR_F32 && prec != DTR_BF16 && prec != DTR_F16)
    return fail(DTR_EINVAL, "unknown dslash precision");
  if (work_bytes < dtr_dslash_workspace_bytes(&g->lat, nrhs)) return fail(DTR_ENOMEM, "dslash workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const Geom geo = geom_of(g->lat);
  const size_t vb = ((size_t)g->lat.V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  DTR_CUDA(cudaMemsetAsync(w, 0, 2 * vb, st));
  if (prec == DTR_BF16 || prec == DTR_F16) {  // half fields use b = nrhs exactly (no padding)
    const int bf = prec == DTR_BF16;
    cudaEvent_t h0, h1;
    DTR_CUDA(cudaEventCreate(&h0));
    DTR_CUDA(cudaEventCreate(&h1));
    launch_dslash_half_raw(bf ? g->Ubf16 : g->Uf16, w, geo, nrhs, m0, bf, 1, st);  // warm
    DTR_CUDA(cudaEventRecord(h0, st));
    launch_dslash_half_raw(bf ? g->Ubf16 : g->Uf16, w, geo, nrhs, m0, bf, reps, st);
    DTR_CUDA(cudaEventRecord(h1, st));
    DTR_CUDA(cudaEventSynchronize(h1));
    float hms = 0.f;
    DTR_CUDA(cudaEventElapsedTime(&hms, h0, h1));
    cudaEventDestroy(h0);
    cudaEventDestroy(h1);
    DTR_LAUNCH_CHECK("half dslash timing");
    *avg_ms = (double)hms / reps;
    return DTR_OK;
  }
  cudaEvent_t e0, e1;
  DTR_CUDA(cudaEventCreate(&e0));
  DTR_CUDA(cudaEventCreate(&e1));
  DTR_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) {
    if (prec == DTR_F64)
      launch_dslash<double>(g->U64, (const double2 *)w, (double2 *)(w + vb), geo, b, m0, 0, st);
    else
      launch_dslash<float>(g->U32, (const float2 *)w, (float2 *)(w + vb), geo, b, m0, 0, st);
  }
  DTR_CUDA(cudaEventRecord(e1, st));
  DTR_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DTR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DTR_LAUNCH_CHECK("dslash timing");
  *avg_ms = (double)ms / reps;
  return DTR_OK;
}

int dtr_gen_noise(dtr_lattice lat, uint64_t seed, int64_t z0_index, int ncolors, int dilute12, int64_t q0, int nrhs,
                  double *out, void *stream) {
  if (!lat || !out) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || q0 < 0 || z0_index < 0) return fail(DTR_EINVAL, "bad column range");
  int rc = check_colouring(*lat, ncolors);
  if (rc) return rc;
  launch_noise_canon((double2 *)out, geom_of(*lat), seed, z0_index, ncolors, dilute12, q0, nrhs,
                     (cudaStream_t)stream);
  DTR_LAUNCH_CHECK("noise");
  return DTR_OK;
}

void dtr_solve_params_default(dtr_solve_params *p) {
  if (!p) return;
  p->tol = 1e-10;
  p->maxiter = 5000;
  p->solver = DTR_SOLVER_BICGSTAB_F64;
  p->check_every = 8;
  p->inner_tol = 1e-5;
  p->engine = 0;
  p->grid = 0;
  p->net = nullptr;
  p->gmres_m = 16;
  p->no_graph = 0;
}

static int check_solve_params(const dtr_solve_params *p) {
  if (!p) return fail(DTR_EINVAL, "null solve params");
  if (!(p->tol > 0.0) || p->maxiter < 1) return fail(DTR_EINVAL, "tol must be > 0 and maxiter >= 1");
  if (p->solver != DTR_SOLVER_BICGSTAB_F64 && p->solver != DTR_SOLVER_MIXED_F32 && p->solver != DTR_SOLVER_FGMRES_NET &&
      p->solver != DTR_SOLVER_MIXED_F16 && p->solver != DTR_SOLVER_MIXED_BF16)
    return fail(DTR_EINVAL, "unknown solver");
  if (p->solver == DTR_SOLVER_FGMRES_NET && (p->gmres_m < 1 || p->gmres_m > 32))
    return fail(DTR_EINVAL, "gmres_m must be in [1, 32]");
  if (p->engine != 0 && p->engine != 1) return fail(DTR_EINVAL, "engine must be 0 (persistent) or 1 (per-step)");
  if ((p->solver == DTR_SOLVER_MIXED_F16 || p->solver == DTR_SOLVER_MIXED_BF16) && p->engine != 0)
    return fail(DTR_EINVAL, "half-storage inner solves need the persistent engine");
  if (p->grid < 0) return fail(DTR_EINVAL, "grid must be >= 0");
  return DTR_OK;
}

size_t dtr_solve_workspace_bytes(dtr_lattice lat, int nrhs, const dtr_solve_params *p) {
  if (!lat || !p || nrhs < 1 || nrhs > 64) return 0;
  const int b = pad_rhs(nrhs);
  const size_t vb = ((size_t)lat->V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  return 256 + 2 * vb + solver_scratch_bytes(lat->V, b, p->solver, p->gmres_m);
}

int dtr_solve_batch(dtr_gauge g, double m0, const double *z, double *y, int nrhs, const dtr_solve_params *p,
                    void *work, size_t work_bytes, dtr_solve_stat *stats, void *stream) {
  if (!g || !z || !y || !work) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64) return fail(DTR_EINVAL, "nrhs must be in [1, 64]");
  int rc = check_solve_params(p);
  if (rc) return rc;
  const size_t need = dtr_solve_workspace_bytes(&g->lat, nrhs, p);
  if (work_bytes < need) return fail(DTR_ENOMEM, "solver workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const size_t vb = ((size_t)g->lat.V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double2 *X = (double2 *)w, *Z = (double2 *)(w + vb);
  launch_pack<double>((const double2 *)z, Z, g->lat.V, nrhs, b, st);
  launch_pack<double>((const double2 *)y, X, g->lat.V, nrhs, b, st);
  DTR_LAUNCH_CHECK("pack");
  Scal *sc = nullptr;
  rc = solve_internal(g, m0, X, Z, b, p, w + 2 * vb, work_bytes - (size_t)(w + 2 * vb - (char *)work), st, &sc);
  if (rc) return rc;
  launch_unpack<double>(X, (double2 *)y, g->lat.V, nrhs, b, st);
  DTR_LAUNCH_CHECK("unpack");
  Scal h;
  DTR_CUDA(cudaMemcpyAsync(&h, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
  DTR_CUDA(cudaStreamSynchronize(st));
  int all = 1, nan = 0;
  for (int j = 0; j < nrhs; ++j) {
    if (!h.conv[j]) all = 0;
    if (h.flags[j] & kFlagNaN) nan = 1;
    if (stats) {
      stats[j].iterations = h.iters[j];
      stats[j].restarts = h.restarts[j];
      stats[j].converged = h.conv[j];
      stats[j].pad_ = h.flags[j];
      stats[j].true_residual = h.bnorm2[j] > 0 ? std::sqrt(h.rtrue2[j] / h.bnorm2[j]) : 0.0;
    }
  }
  if (nan) return fail(DTR_ENAN, "NaN or Inf in a residual norm");
  if (!all) return fail(DTR_ENOTCONV, "some right-hand sides did not reach tol within maxiter");
  return DTR_OK;
}

int dtr_defl_create(dtr_lattice lat, int k, dtr_prec prec, const double *V_host, const double *lambda_host,
                    dtr_defl *out) {
  if (!lat || !V_host || !lambda_host || !out) return fail(DTR_EINVAL, "null argument");
  if (k < 1) return fail(DTR_EINVAL, "k must be >= 1");
  if (prec != DTR_F64 && prec != DTR_F32 && prec != DTR_BF16)
    return fail(DTR_EINVAL, "deflation storage must be DTR_F64, DTR_F32 or DTR_BF16");
  for (int m = 0; m < k; ++m)
    if (!(lambda_host[m] != 0.0) || !std::isfinite(lambda_host[m]))
      return fail(DTR_EINVAL, "lambda must be finite and non-zero");
  const int64_t N = lat->N;
  // canonical column-major N x k -> row-major [dof][k]
  std::vector<double2> rowmajor;
  try {
    rowmajor.resize((size_t)N * k);
  } catch (...) {
    return fail(DTR_ENOMEM, "host allocation failed");
  }
  const double2 *src = (const double2 *)V_host;
  for (int m = 0; m < k; ++m)
    for (int64_t i = 0; i < N; ++i) rowmajor[(size_t)i * k + m] = src[(size_t)m * N + i];
  dtr_defl_s *D = new (std::nothrow) dtr_defl_s;
  if (D) {
    D->tdg_ok = 0u;
    D->Ginv = nullptr;
  }
  if (!D) return fail(DTR_ENOMEM, "host allocation failed");
  D->lat = *lat;
  D->k = k;
  D->prec = prec;
  D->V = nullptr;
  D->inv_lambda = nullptr;
  std::vector<double> inv(k);
  for (int m = 0; m < k; ++m) inv[m] = 1.0 / lambda_host[m];
  cudaError_t e = cudaMalloc(&D->inv_lambda, k * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(D->inv_lambda, inv.data(), k * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (prec == DTR_F64) {
      e = cudaMalloc(&D->V, (size_t)N * k * sizeof(double2));
      if (e == cudaSuccess)
        e = cudaMemcpy(D->V, rowmajor.data(), (size_t)N * k * sizeof(double2), cudaMemcpyHostToDevice);
    } else {
      double2 *tmp = nullptr;
      e = cudaMalloc(&D->V, (size_t)N * k * (prec == DTR_F32 ? sizeof(float2) : sizeof(__nv_bfloat162)));
      if (e == cudaSuccess) e = cudaMalloc(&tmp, (size_t)N * k * sizeof(double2));
      if (e == cudaSuccess) e = cudaMemcpy(tmp, rowmajor.data(), (size_t)N * k * sizeof(double2), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        if (prec == DTR_F32)
          k_to_f32<<<grid1d((int64_t)N * k), 256>>>(tmp, (float2 *)D->V, (int64_t)N * k);
        else
          k_to_bf16<<<grid1d((int64_t)N * k), 256>>>(tmp, (__nv_bfloat162 *)D->V, (int64_t)N * k);
        count_launches(1);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      cudaFree(tmp);
    }
  }
  if (e != cudaSuccess) {
    cudaFree(D->V);
    cudaFree(D->inv_lambda);
    delete D;
    return cuda_fail(e, "deflation space upload");
  }
  int rc = defl_trace_TD(D, 0);
  if (rc) {
    cudaFree(D->V);
    cudaFree(D->inv_lambda);
    delete D;
    return rc;
  }
  *out = D;
  return DTR_OK;
}

int dtr_defl_trace(dtr_defl d, double td[2]) {
  if (!d || !td) return fail(DTR_EINVAL, "null argument");
  td[0] = d->td[0];
  td[1] = d->td[1];
  return DTR_OK;
}

void dtr_eig_params_default(dtr_eig_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->k = 32;
  p->degree = 48;
  p->max_iter = 100;
  p->chunk = 32;
  p->store = DTR_F64;
  p->tol = 1e-2;
}

size_t dtr_eig_workspace_bytes(dtr_lattice lat, const dtr_eig_params *p) {
  if (!lat || !p || p->k < 1) return 0;
  return eig_workspace_bytes(*lat, p);
}

int dtr_eig_deflation(dtr_gauge g, double m0, const dtr_eig_params *p, void *work, size_t work_bytes,
                      double *residuals, dtr_eig_stats *stats, dtr_defl *out, void *stream) {
  if (!g || !p || !work || !out) return fail(DTR_EINVAL, "null argument");
  if (p->store != DTR_F64 && p->store != DTR_F32 && p->store != DTR_BF16)
    return fail(DTR_EINVAL, "eigensolver storage must be DTR_F64, DTR_F32 or DTR_BF16");
  const int nb = eig_basis_columns(p);
  if (p->k < 1 || p->degree < 0 || p->first_degree < 0 || p->max_iter < 1 || !(p->tol > 0.0) ||
      p->chunk < 0 || p->chunk > 64 || (p->p > 0 && p->p < p->k) || (int64_t)nb * 4 > g->lat.N)
    return fail(DTR_EINVAL, "bad eigensolver parameters (k >= 1, p >= k, 4 p <= N, chunk <= 64, tol > 0)");
  const size_t es = p->store == DTR_F64 ? sizeof(double2) : (p->store == DTR_F32 ? sizeof(float2) : 4);
  dtr_defl_s *D = new (std::nothrow) dtr_defl_s;
  if (!D) return fail(DTR_ENOMEM, "host allocation failed");
  D->tdg_ok = 0u;
  D->Ginv = nullptr;
  D->lat = g->lat;
  D->k = p->k;
  D->prec = p->store;
  D->V = nullptr;
  D->inv_lambda = nullptr;
  // the basis of nb columns lives in the handle's buffer and is compacted to k columns at the end
  cudaError_t e = cudaMalloc(&D->V, (size_t)g->lat.N * nb * es);
  if (e == cudaSuccess) e = cudaMalloc(&D->inv_lambda, p->k * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(D->V);
    cudaFree(D->inv_lambda);
    delete D;
    return fail(DTR_ENOMEM, std::string("eigensolver basis allocation failed: ") + cudaGetErrorString(e));
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = eig_solve(g, m0, p, work, work_bytes, D, residuals, stats, st);
  if (rc == DTR_OK) rc = defl_trace_TD(D, st);
  if (rc != DTR_OK) {
    cudaFree(D->V);
    cudaFree(D->inv_lambda);
    delete D;
    return rc;
  }
  *out = D;
  return DTR_OK;
}

int dtr_defl_to_host(dtr_defl d, double *V_host, double *lambda_host) {
  if (!d) return fail(DTR_EINVAL, "null argument");
  const int k = d->k;
  const int64_t N = d->lat.N;
  if (lambda_host) {
    std::vector<double> il(k);
    DTR_CUDA(cudaMemcpy(il.data(), d->inv_lambda, k * sizeof(double), cudaMemcpyDeviceToHost));
    for (int m = 0; m < k; ++m) lambda_host[m] = 1.0 / il[m];
  }
  if (V_host) {
    const size_t es = d->prec == DTR_F64 ? sizeof(double2) : (d->prec == DTR_F32 ? sizeof(float2) : 4);
    std::vector<unsigned char> raw;
    try {
      raw.resize((size_t)N * k * es);
    } catch (...) {
      return fail(DTR_ENOMEM, "host allocation failed");
    }
    DTR_CUDA(cudaMemcpy(raw.data(), d->V, raw.size(), cudaMemcpyDeviceToHost));
    double2 *dst = (double2 *)V_host;
    for (int64_t i = 0; i < N; ++i)
      for (int m = 0; m < k; ++m) {
        const size_t q = (size_t)i * k + m;
        double re, im;
        if (d->prec == DTR_F64) {
          const double *v = (const double *)raw.data() + 2 * q;
          re = v[0];
          im = v[1];
        } else if (d->prec == DTR_F32) {
          const float *v = (const float *)raw.data() + 2 * q;
          re = v[0];
          im = v[1];
        } else {  // BF16 pair: the high 16 bits of an FP32 value each
          const uint16_t *v = (const uint16_t *)raw.data() + 2 * q;
          uint32_t ur = (uint32_t)v[0] << 16, ui = (uint32_t)v[1] << 16;
          float fr, fi;
          std::memcpy(&fr, &ur, 4);
          std::memcpy(&fi, &ui, 4);
          re = fr;
          im = fi;
        }
        dst[(size_t)m * N + i] = make_double2(re, im);
      }
  }
  return DTR_OK;
}

void dtr_destroy_defl(dtr_defl d) {
  if (!d) return;
  cudaFree(d->V);
  cudaFree(d->inv_lambda);
  cudaFree(d->Ginv);
  delete d;
}

int dtr_defl_gram(dtr_defl d, dtr_gauge g, double m0, void *stream) {
  if (!d || !g) return fail(DTR_EINVAL, "null argument");
  return defl_gram(d, g, m0, (cudaStream_t)stream);
}

size_t dtr_deflate_workspace_bytes(dtr_defl d, int nrhs) {
  if (!d || nrhs < 1 || nrhs > 64) return 0;
  const int b = pad_rhs(nrhs);
  const size_t vb = ((size_t)d->lat.V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  return 256 + 2 * vb + 256 * 3 + 64 * sizeof(double2) + defl_scratch_bytes(d->lat.V, d->k, b, device_sms());
}

int dtr_deflate_project(dtr_defl d, const double *z, int nrhs, double *d_out, double *coeff_out, double *x0_out,
                        void *work, size_t work_bytes, void *stream) {
  if (!d || !z || !d_out || !work) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64) return fail(DTR_EINVAL, "nrhs must be in [1, 64]");
  if (work_bytes < dtr_deflate_workspace_bytes(d, nrhs)) return fail(DTR_ENOMEM, "deflation workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const size_t vb = ((size_t)d->lat.V * 12 * b * sizeof(double2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double2 *Z = (double2 *)w;
  double2 *X0 = (double2 *)(w + vb);
  double2 *dd = (double2 *)(w + 2 * vb);
  char *scratch = w + 2 * vb + 256 + 64 * sizeof(double2);
  const size_t scratch_bytes = work_bytes - (size_t)(scratch - (char *)work);
  launch_pack<double>((const double2 *)z, Z, d->lat.V, nrhs, b, st);
  double2 *C = nullptr;
  int rc = defl_project_internal(d, Z, b, dd, nullptr, x0_out ? X0 : nullptr, &C, scratch, scratch_bytes,
                                 device_sms(), st);
  if (rc) return rc;
  DTR_CUDA(cudaMemcpyAsync(d_out, dd, sizeof(double2) * nrhs, cudaMemcpyDeviceToDevice, st));
  if (coeff_out) {
    const size_t colbytes = sizeof(double2) * d->k;
    DTR_CUDA(cudaMemcpyAsync(coeff_out, C, colbytes * nrhs, cudaMemcpyDeviceToDevice, st));
    DTR_CUDA(cudaMemcpyAsync((char *)coeff_out + colbytes * nrhs, C + (size_t)b * d->k, colbytes * nrhs,
                             cudaMemcpyDeviceToDevice, st));
  }
  if (x0_out) launch_unpack<double>(X0, (double2 *)x0_out, d->lat.V, nrhs, b, st);
  DTR_LAUNCH_CHECK("deflate project");
  return DTR_OK;
}

// ------------------------------------------------------------ network
int dtr_net_create(dtr_lattice lat, int act, const float *weights_host, double init_scale, double noise,
                   uint64_t seed, dtr_net *out) {
  if (!lat || !out) return fail(DTR_EINVAL, "null argument");
  if (act != 0 && act != 1) return fail(DTR_EINVAL, "act must be 0 (identity) or 1 (leaky ReLU)");
  const int L = DTR_NET_LAYERS;
  const size_t per = 81 * 24 * 24, nw = L * per;
  std::vector<float> w(nw, 0.f);
  if (weights_host) {
    std::memcpy(w.data(), weights_host, nw * sizeof(float));
  } else {
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto unif = [&]() {  // 64-bit LCG (Knuth MMIX constants), top 53 bits
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (size_t i = 0; i < nw; i += 2) {  // Box-Muller
      const double u1 = unif(), u2 = unif();
      const double r = std::sqrt(-2.0 * std::log(u1));
      w[i] = (float)(noise * r * std::cos(6.283185307179586 * u2));
      if (i + 1 < nw) w[i + 1] = (float)(noise * r * std::sin(6.283185307179586 * u2));
    }
    for (int l = 0; l < L; ++l)
      for (int c = 0; c < 24; ++c) w[l * per + 40 * 576 + c * 24 + c] += (float)(l == 0 ? init_scale : 1.0);
  }
  dtr_net_s *n = new (std::nothrow) dtr_net_s;
  if (!n) return fail(DTR_ENOMEM, "host allocation failed");
  n->lat = *lat;
  n->L = L;
  n->act = act;
  n->step = 0;
  n->tc = 1;
  n->w = n->m = n->v = n->grad = n->wf = n->wb = nullptr;
  n->wtc_f = n->wtc_b = nullptr;
  n->err = nullptr;
  float **bufs[6] = {&n->w, &n->m, &n->v, &n->grad, &n->wf, &n->wb};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc((void **)bufs[i], nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void **)&n->wtc_f, net_tc_weight_bytes(L));
  if (e == cudaSuccess) e = cudaMalloc((void **)&n->wtc_b, net_tc_weight_bytes(L));
  if (e == cudaSuccess) e = cudaMalloc((void **)&n->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(n->w, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, nw * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->grad, 0, nw * sizeof(float));
  if (e == cudaSuccess) {
    net_refresh(n, 0);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    for (int i = 0; i < 6; ++i) cudaFree(*bufs[i]);
    cudaFree(n->wtc_f);
    cudaFree(n->wtc_b);
    cudaFree(n->err);
    delete n;
    return cuda_fail(e, "network create");
  }
  *out = n;
  return DTR_OK;
}

void dtr_destroy_net(dtr_net n) {
  if (!n) return;
  cudaFree(n->w);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->grad);
  cudaFree(n->wf);
  cudaFree(n->wb);
  cudaFree(n->wtc_f);
  cudaFree(n->wtc_b);
  cudaFree(n->err);
  delete n;
}

int dtr_net_set_precision(dtr_net n, dtr_prec prec) {
  if (!n) return fail(DTR_EINVAL, "null argument");
  if (prec != DTR_BF16 && prec != DTR_F32) return fail(DTR_EINVAL, "network precision must be DTR_BF16 or DTR_F32");
  n->tc = prec == DTR_BF16;
  return DTR_OK;
}

int dtr_net_get_weights(dtr_net n, int bf16_rounded, float *host) {
  if (!n || !host) return fail(DTR_EINVAL, "null argument");
  DTR_CUDA(cudaMemcpy(host, bf16_rounded ? n->wb : n->w, sizeof(float) * DTR_NET_WEIGHTS, cudaMemcpyDeviceToHost));
  return DTR_OK;
}

size_t dtr_net_workspace_bytes(dtr_net n, int nrhs) {
  if (!n || nrhs < 1 || nrhs > 64) return 0;
  const int b = pad_rhs(nrhs);
  const size_t vec = ((size_t)n->lat.V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  return 256 + 2 * vec + net_workspace_bytes(n, b);
}

int dtr_net_apply(dtr_net n, const double *in, double *out, int nrhs, void *work, size_t work_bytes, void *stream) {
  if (!n || !in || !out || !work) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64) return fail(DTR_EINVAL, "nrhs must be in [1, 64]");
  if (work_bytes < dtr_net_workspace_bytes(n, nrhs)) return fail(DTR_ENOMEM, "network workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const size_t vec = ((size_t)n->lat.V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  float2 *x = (float2 *)w, *y = (float2 *)(w + vec), *t0 = (float2 *)(w + 2 * vec), *t1 = (float2 *)(w + 3 * vec);
  launch_pack<float>((const double2 *)in, x, n->lat.V, nrhs, b, st);
  net_apply(n, x, y, b, t0, t1, st);
  launch_unpack<float>(y, (double2 *)out, n->lat.V, nrhs, b, st);
  DTR_LAUNCH_CHECK("network apply");
  return n->tc ? net_check_err(n, st) : DTR_OK;
}

int dtr_net_train_step(dtr_net n, dtr_gauge g, double m0, const double *in, const double *target, int nrhs, double lr,
                       int do_step, double *loss, float *grad_host, void *work, size_t work_bytes, void *stream) {
  if (!n || !in || !target || !loss || !work) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64) return fail(DTR_EINVAL, "nrhs must be in [1, 64]");
  if (work_bytes < dtr_net_workspace_bytes(n, nrhs)) return fail(DTR_ENOMEM, "network workspace too small");
  if (g && g->lat.V != n->lat.V) return fail(DTR_EINVAL, "gauge field on another lattice");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const size_t vec = ((size_t)n->lat.V * 12 * b * sizeof(float2) + 255) / 256 * 256;
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  float2 *x = (float2 *)w, *e = (float2 *)(w + vec);
  launch_pack<float>((const double2 *)in, x, n->lat.V, nrhs, b, st);
  launch_pack<float>((const double2 *)target, e, n->lat.V, nrhs, b, st);
  DTR_LAUNCH_CHECK("pack training pair");
  return net_train(n, g, m0, x, e, b, nrhs, lr, do_step, grad_host, loss, w + 2 * vec, work_bytes - 2 * vec - 256, st);
}

static int check_trace_params(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  if (!p) return fail(DTR_EINVAL, "null trace params");
  int rc = check_solve_params(&p->solve);
  if (rc) return rc;
  if (p->block < 1 || p->block > 64) return fail(DTR_EINVAL, "block must be in [1, 64]");
  if (p->n_z0 < 1 || p->nvec < 1 || p->z0_first < 0) return fail(DTR_EINVAL, "n_z0 and nvec must be >= 1");
  rc = check_colouring(g->lat, p->ncolors);
  if (rc) return rc;
  if (p->ncolors > 1 && p->nvec > p->ncolors) return fail(DTR_EINVAL, "nvec must be <= ncolors");
  if (p->ncolors == 1 && p->nvec != 1) return fail(DTR_EINVAL, "plain Z4 noise (ncolors = 1) has nvec = 1");
  if (p->vec_first < 0 || (p->ncolors == 1 && p->vec_first != 0) ||
      (p->ncolors > 1 && p->vec_first + p->nvec > p->ncolors))
    return fail(DTR_EINVAL, "vec_first + nvec must be <= ncolors (vec_first = 0 for plain Z4 noise)");
  if (D && (D->lat.V != g->lat.V)) return fail(DTR_EINVAL, "deflation space built for another lattice");
  if (p->n_gamma < 0 || p->n_gamma > 16) return fail(DTR_EINVAL, "n_gamma must be in [0, 16]");
  for (int q = 0; q < p->n_gamma; ++q)
    if (p->gamma[q] < 0 || p->gamma[q] > 15) return fail(DTR_EINVAL, "Gamma indices must be in [0, 15]");
  return DTR_OK;
}

size_t dtr_trace_workspace_bytes(dtr_gauge g, dtr_defl d, const dtr_trace_params *p) {
  if (!g || !p || p->block < 1 || p->block > 64) return 0;
  return trace_workspace_bytes(g, d, p);
}

int dtr_trace_estimate(dtr_gauge g, double m0, dtr_defl d, const dtr_trace_params *p, void *work, size_t work_bytes,
                       dtr_trace_result *res, void *stream) {
  if (!g || !res || !work) return fail(DTR_EINVAL, "null argument");
  int rc = check_trace_params(g, d, p);
  if (rc) return rc;
  return trace_estimate(g, m0, d, p, work, work_bytes, res, (cudaStream_t)stream);
}

size_t dtr_time_deflate_workspace_bytes(dtr_defl d, int nrhs) {
  if (!d || nrhs < 1 || nrhs > 64) return 0;
  const int b = pad_rhs(nrhs);
  return (((size_t)d->lat.V * 12 * b * sizeof(double2) + 255) / 256) * 256 + 64 * sizeof(double2) + 256 +
         defl_scratch_bytes(d->lat.V, d->k, b, device_sms()) + 256 + (((size_t)d->lat.V * 12 * b + 255) / 256) * 256;
}

int dtr_time_deflate(dtr_defl d, int nrhs, int reps, void *work, size_t work_bytes, double *avg_ms, void *stream) {
  if (!d || !work || !avg_ms) return fail(DTR_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 64 || reps < 1) return fail(DTR_EINVAL, "nrhs must be in [1, 64] and reps >= 1");
  if (work_bytes < dtr_time_deflate_workspace_bytes(d, nrhs)) return fail(DTR_ENOMEM, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int b = pad_rhs(nrhs);
  const Geom geo = geom_of(d->lat);
  char *w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double2 *Z = (double2 *)w;
  w += (((size_t)d->lat.V * 12 * b * sizeof(double2) + 255) / 256) * 256;
  double2 *dd = (double2 *)w;
  w += 64 * sizeof(double2) + 256;
  const size_t sb = defl_scratch_bytes(d->lat.V, d->k, b, device_sms());
  unsigned char *Zc = (unsigned char *)(w + ((sb + 255) / 256) * 256);  // the block as one-byte codes
  launch_noise(Z, geo, 0x5EED, 0, 1, 0, 0, 1, nrhs, b, st, 0, Zc);  // one Z4 vector per column
  int rc = defl_project_internal(d, Z, b, dd, nullptr, nullptr, nullptr, w, sb, device_sms(), st, 1, Zc);  // warm
  if (rc) return rc;
  cudaEvent_t e0, e1;
  DTR_CUDA(cudaEventCreate(&e0));
  DTR_CUDA(cudaEventCreate(&e1));
  DTR_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < reps && rc == DTR_OK; ++r)
    rc = defl_project_internal(d, Z, b, dd, nullptr, nullptr, nullptr, w, sb, device_sms(), st, 1, Zc);
  DTR_CUDA(cudaEventRecord(e1, st));
  DTR_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DTR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int herr = 0;
  DTR_CUDA(cudaMemcpy(&herr, defl_error_word(w), sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return fail(DTR_ETIMEOUT, "tensor-core deflation stage timed out");
  *avg_ms = ms / reps;
  return DTR_OK;
}

uint64_t dtr_tensor_core_contractions(void) { return (uint64_t)defl_tc_calls(); }

int dtr_wd(dtr_lattice lat, const double *cols, const int64_t *dofs, int ns, int maxd, int ncolors, double *W,
           void *stream) {
  if (!lat || !cols || !dofs || !W) return fail(DTR_EINVAL, "null argument");
  if (ns < 1 || maxd < 0 || maxd > 4096) return fail(DTR_EINVAL, "need ns >= 1 and 0 <= maxd <= 4096");
  if (ncolors > 1) {
    int rc = check_colouring(*lat, ncolors);
    if (rc) return rc;
  }
  return wd_diagnostic(lat, (const double2 *)cols, dofs, ns, maxd, ncolors, W, (cudaStream_t)stream);
}

size_t dtr_trace_autotune_workspace_bytes(dtr_gauge g, dtr_defl d, const dtr_trace_params *p) {
  if (!g || !p || p->block > 64) return 0;
  return tune_workspace_bytes(g, d, p);
}

int dtr_trace_autotune(dtr_gauge g, double m0, dtr_defl d, const dtr_trace_params *p, int reps, int force,
                       void *work, size_t work_bytes, dtr_tune_result *out, void *stream) {
  if (!g || !p || !work || !out) return fail(DTR_EINVAL, "null argument");
  if (p->block > 64) return fail(DTR_EINVAL, "block must be <= 64 (or <= 0 to tune it)");
  dtr_trace_params q = *p;
  if (q.block <= 0) q.block = 16;  // for the parameter checks only
  int rc = check_trace_params(g, d, &q);
  if (rc) return rc;
  return trace_autotune(g, m0, d, p, reps, force, work, work_bytes, out, (cudaStream_t)stream);
}

}  // extern "C"
