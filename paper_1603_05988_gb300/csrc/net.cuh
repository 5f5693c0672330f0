// Learned preconditioner network handle and entry points shared with the solver.
#pragma once

#include "dtr_internal.cuh"

struct dtr_net_s {
  dtr_lattice_s lat;
  int L;          // layers (4)
  int act;        // 0 identity, 1 leaky ReLU (slope 1/4)
  float *w;       // master FP32 [L][81][24 co][24 ci]
  float *m, *v;   // Adam moments
  float *grad;    // last gradient
  float *wf;      // BF16-rounded copy ordered [L][81][ci][co] (forward)
  float *wb;      // BF16-rounded copy ordered [L][81][co][ci] (backward data)
  long long step;
};

namespace dtr {

size_t net_workspace_bytes(const dtr_net_s *net, int b);
void net_refresh(dtr_net_s *net, cudaStream_t st);
void net_apply(const dtr_net_s *net, const float2 *x, float2 *y, int b, float2 *t0, float2 *t1, cudaStream_t st);
// gauge == nullptr: error loss sum_j |y_j - e_j|^2 / |e_j|^2; otherwise the
// residual-weighted loss sum_j |A y_j - x_j|^2 / |x_j|^2
int net_train(dtr_net_s *net, const dtr_gauge_s *gauge, double m0, const float2 *x, const float2 *e, int b, int nrhs,
              double lr, int do_step, float *grad_host, double *loss_out, void *work, size_t work_bytes,
              cudaStream_t st);

size_t fgmres_scratch_bytes(int64_t V, int b, int m);
int fgmres_solve(const dtr_gauge_s *gauge, double m0, const dtr_net_s *net, const float2 *rhs, float2 *x, int b,
                 const int *active, int m, double tol, int max_iters, void *work, size_t work_bytes, int *iters_out,
                 cudaStream_t st);

}  // namespace dtr
