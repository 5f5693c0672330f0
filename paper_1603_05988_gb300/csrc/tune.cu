// Autotuner of the estimator's launch shape.
//
// The estimator's throughput on one GPU depends on how much independent work
// is in flight: a block of b right-hand sides at a small lattice leaves the
// GPU latency-bound, so several blocks solved concurrently on their own
// streams and SM shares ("lanes") run faster than one.  The tuner times real
// trace waves (one block per lane, lanes z0 runs of the caller's problem) for
// every candidate (lane count; RHS block as well when the caller leaves it
// open), keeps the fastest in RHS solves per second, and caches the choice per
// problem shape (device, lattice, deflation size, solver, colouring, vectors
// per run, block) so later calls return at once.
#include <chrono>
#include <cstring>
#include <mutex>
#include <vector>

#include "deflate.cuh"
#include "dtr_internal.cuh"
#include "solver.cuh"

namespace dtr {

int trace_estimate(const dtr_gauge_s *gauge, double m0, const dtr_defl_s *D, const dtr_trace_params *p, void *work,
                   size_t work_bytes, dtr_trace_result *res, cudaStream_t st);
size_t trace_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p);

namespace {

struct TuneKey {
  int device;
  int L[4];
  int k, solver, engine, no_graph, ncolors, nvec, block, dilute12;
};

struct TuneEntry {
  TuneKey key;
  dtr_tune_result res;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

const int kLaneCands[] = {1, 2, 4, 8};
const int kBlockCands[] = {8, 16, 32, 64};

TuneKey make_key(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  TuneKey key;
  std::memset(&key, 0, sizeof(key));
  cudaGetDevice(&key.device);
  for (int i = 0; i < 4; ++i) key.L[i] = g->lat.dims[i];
  key.k = D ? D->k : 0;
  key.solver = p->solve.solver;
  key.engine = p->solve.engine;
  key.no_graph = p->solve.no_graph;
  key.ncolors = p->ncolors;
  key.nvec = p->nvec;
  key.block = p->block;
  key.dilute12 = p->dilute12;
  return key;
}

// A candidate's parameters: one wave = `lanes` blocks of `block` columns.  When a run
// has more columns than a wave, the wave takes the first lanes x block probing columns of one
// run (so timing a candidate costs one wave, not a whole run of hundreds of vectors).
dtr_trace_params candidate(const dtr_trace_params *p, int lanes, int block) {
  dtr_trace_params q = *p;
  q.lanes = lanes;
  q.block = block;
  const int per = p->dilute12 ? 12 : 1;
  const int ncols = p->nvec * per;
  const int64_t want = (int64_t)lanes * block;               // columns in one wave
  if (ncols > want) {
    q.n_z0 = 1;
    q.nvec = (int)((want + per - 1) / per);
    return q;
  }
  q.n_z0 = (int)((want + ncols - 1) / ncols);
  if (q.n_z0 < 1) q.n_z0 = 1;
  return q;
}

}  // namespace

size_t tune_workspace_bytes(const dtr_gauge_s *g, const dtr_defl_s *D, const dtr_trace_params *p) {
  size_t mx = 0;
  for (int lanes : kLaneCands) {
    if (p->block > 0) {
      const dtr_trace_params q = candidate(p, lanes, p->block);
      const size_t b = trace_workspace_bytes(g, D, &q);
      if (b > mx) mx = b;
    } else {
      for (int blk : kBlockCands) {
        const dtr_trace_params q = candidate(p, lanes, blk);
        const size_t b = trace_workspace_bytes(g, D, &q);
        if (b > mx) mx = b;
      }
    }
  }
  return mx;
}

int trace_autotune(const dtr_gauge_s *g, double m0, const dtr_defl_s *D, const dtr_trace_params *p, int reps,
                   int force, void *work, size_t work_bytes, dtr_tune_result *out, cudaStream_t st) {
  const TuneKey key = make_key(g, D, p);
  if (!force) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &e : g_tune)
      if (!std::memcmp(&e.key, &key, sizeof(key))) {
        *out = e.res;
        out->cached = 1;
        return DTR_OK;
      }
  }
  if (reps < 1) reps = 3;
  dtr_tune_result best;
  std::memset(&best, 0, sizeof(best));
  std::vector<int> blocks;
  if (p->block > 0)
    blocks.push_back(p->block);
  else
    blocks.assign(std::begin(kBlockCands), std::end(kBlockCands));
  const int64_t seed_base = 0x7475000;  // runs used only for timing, far from user runs
  int tried = 0;
  for (int blk : blocks) {
    for (int lanes : kLaneCands) {
      const dtr_trace_params q = candidate(p, lanes, blk);
      const size_t need = trace_workspace_bytes(g, D, &q);
      if (need > work_bytes) continue;
      dtr_trace_result r;
      std::memset(&r, 0, sizeof(r));
      dtr_trace_params qq = q;
      qq.z0_first = seed_base;
      int rc = trace_estimate(g, m0, D, &qq, work, work_bytes, &r, st);  // warm-up (graph capture)
      if (rc && rc != DTR_ENOTCONV) return rc;
      DTR_CUDA(cudaStreamSynchronize(st));
      const auto t0 = std::chrono::steady_clock::now();
      for (int i = 0; i < reps; ++i) {
        qq.z0_first = seed_base + 1 + (int64_t)i * q.n_z0;
        rc = trace_estimate(g, m0, D, &qq, work, work_bytes, &r, st);
        if (rc && rc != DTR_ENOTCONV) return rc;
      }
      DTR_CUDA(cudaStreamSynchronize(st));
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      const double cols = (double)q.n_z0 * q.nvec * (q.dilute12 ? 12 : 1) * reps;
      const double rate = sec > 0 ? cols / sec : 0.0;
      if (tried < 16) {
        best.table_lanes[tried] = lanes;
        best.table_block[tried] = blk;
        best.table_rhs_per_s[tried] = rate;
      }
      ++tried;
      if (rate > best.rhs_per_s) {
        best.rhs_per_s = rate;
        best.lanes = lanes;
        best.block = blk;
      }
    }
  }
  if (!tried) return fail(DTR_ENOMEM, "autotune workspace too small for any candidate");
  best.n_tried = tried < 16 ? tried : 16;
  best.cached = 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    bool found = false;
    for (auto &e : g_tune)
      if (!std::memcmp(&e.key, &key, sizeof(key))) {
        e.res = best;
        found = true;
      }
    if (!found) g_tune.push_back(TuneEntry{key, best});
  }
  *out = best;
  return DTR_OK;
}

}  // namespace dtr
