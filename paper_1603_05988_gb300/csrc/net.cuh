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
  unsigned char *wtc_f, *wtc_b;  // B operands of the tensor-core convolution, per layer (forward, backward data)
  int *err;       // set by a tensor-core kernel whose bounded wait ran out
  int tc;         // 1: BF16 activations, convolutions on the tensor cores; 0: FP32 on the CUDA cores
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

int device_sms();

// tensor-core convolution (net_tc.cu)
size_t net_tc_weight_bytes(int L);
void net_refresh_tc(dtr_net_s *net, cudaStream_t st);
void net_to_planar(const float2 *x, uint4 *p, int64_t V, int b, cudaStream_t st);
void net_conv_tc(const dtr_net_s *net, int layer, bool backward, const uint4 *in, uint4 *out_planar, float2 *out_f2,
                 const uint4 *mask, int act_out, int b, cudaStream_t st);
size_t net_wgrad_tc_scratch_bytes();
// dW of one layer (81 x 24 x 24, [o][co][ci]) from the planar layer input a and output gradient gp
void net_wgrad_tc(const dtr_net_s *net, const uint4 *a, const uint4 *gp, int b, float *part, float *dW,
                  cudaStream_t st);
// DTR_ETIMEOUT (and clears the word) if a tensor-core kernel gave up a wait; synchronises st
int net_check_err(const dtr_net_s *net, cudaStream_t st);

size_t fgmres_scratch_bytes(int64_t V, int b, int m);
int fgmres_solve(const dtr_gauge_s *gauge, double m0, const dtr_net_s *net, const float2 *rhs, float2 *x, int b,
                 const int *active, int m, double tol, int max_iters, void *work, size_t work_bytes, int *iters_out,
                 cudaStream_t st);

}  // namespace dtr
