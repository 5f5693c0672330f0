// Deflation-space kernels shared by the C-ABI entry points and the estimator.
#pragma once

#include <cuda_bf16.h>

#include "dtr_internal.cuh"
#include "gamma.cuh"

namespace dtr {

// Storage types of the deflation space V (DTR_F64, DTR_F32, DTR_BF16), widened
// exactly to FP64 where the kernels accumulate.
typedef __nv_bfloat162 bfc2;
__device__ __forceinline__ double2 vload(const double2 &v) { return v; }
__device__ __forceinline__ double2 vload(const float2 &v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 vload(const bfc2 &v) {
  return make_double2(__bfloat162float(v.x), __bfloat162float(v.y));
}

// Scratch for one projection of a width-b block.
size_t defl_scratch_bytes(int64_t V, int k, int b, int sms);  // includes k x b expansion weights

// C = V^H [Z, g5 Z] (k x 2b, kept in scratch; *C_out points at it),
// d_dev[j] = sum_m conj(C[m,j]) C[m,b+j] / lambda_m, terms_dev (k x b, or
// NULL) the per-m terms, x0_internal (or NULL) = V diag(1/lambda) C[:, b:].
// z4: the caller guarantees Z's entries are 0, +-1 or +-i (probing noise); with
// a BF16-stored V the contraction then runs on the tensor cores (deflate_tc.cu),
// and a stalled tensor-core stage raises *defl_error_word(work).
// Zc (or NULL): Z's entries as one-byte codes (launch_noise), read by the tensor-core path
// instead of the FP64 values.
int defl_project_internal(const dtr_defl_s *D, const double2 *Z, int b, double2 *d_dev, double2 *terms_dev,
                          double2 *x0_internal, double2 **C_out, void *work, size_t work_bytes, int sms,
                          cudaStream_t st, int z4 = 0, const unsigned char *Zc = nullptr);
int *defl_error_word(void *work);
// tensor-core contraction C = V^H [Z, g5 Z] for BF16 V and Z4-valued Z (deflate_tc.cu)
bool defl_tc_enabled(const dtr_defl_s *D, int b);
size_t defl_tc_scratch_bytes(int64_t V, int k, int b, int sms);
int defl_contract_tc(const dtr_defl_s *D, const double2 *Z, int b, double2 *C, void *scratch, size_t scratch_bytes,
                     int *err_dev, int sms, cudaStream_t st, const unsigned char *Zc = nullptr);
unsigned long long defl_tc_calls();

// d_j (and per-m terms, or NULL) from C (column-major k x 2b): with the
// eigenvalue form sum_m conj(C[m, j]) C[m, b+j] / lambda_m, with the Galerkin
// correction (D->Ginv) c_j^H G^-1 g_j, per-m terms conj(c_jm) (G^-1 g_j)_m.
void launch_defl_d(const dtr_defl_s *D, const double2 *C, int b, double2 *d, double2 *terms, cudaStream_t st);
// d_j from Cl[:, j] and Cr[:, b + j] (Gamma insertion: Cl = V^H Gamma^H Z).
void launch_defl_d2(const dtr_defl_s *D, const double2 *Cl, const double2 *Cr, int b, double2 *d, cudaStream_t st);
// Galerkin correction: G = V^H g5 A V from the stored V and the gauge field, G^-1
// kept on the device, T_D = Tr(G^-1 V^H g5 V) (gram.cu).
int defl_gram(dtr_defl_s *D, const dtr_gauge_s *g, double m0, cudaStream_t st);
// T_D of the Gammas in gs in the Galerkin form, Tr(G^-1 V^H g5 Gamma V).
int defl_tdg_gram(const dtr_defl_s *D, const GammaSet &gs, double2 *out, cudaStream_t st);
// GZ = (Gamma^H (x) 1) Z on the internal layout [site][12][b].
void launch_gamma_h(const GammaMono &g, const double2 *Z, double2 *GZ, int64_t V, int b, cudaStream_t st);
// T_D of every Gamma_n in `want` (bit n) not yet cached in D: sum_m v_m^H g5 Gamma v_m / lambda_m.
int defl_trace_TD_gamma(dtr_defl_s *D, unsigned want, cudaStream_t st);

// Projection of an HP block (all columns share one z0 run; columns are
// probing indices q0 .. q0+nrhs-1) from per-colour sums of V^H z0.
// sites_by_colour: V site indices grouped by colour, V/ncolors per colour.
size_t defl_hp_scratch_bytes(int64_t V, int k, int b, int ncolors, int sms);
// xf (or NULL = identity) transforms the z0 codes of every site first, so the
// projection is that of Gamma^H z (Gamma-insertion); d_dev may then be NULL
// (no d_j); *C_out (or NULL) receives the address of C in `work`.
// reuse_w: W in `work` already holds this run's per-colour sums (same D, seed,
// run, dilution, identity transform): only the per-column finish runs.
int defl_project_hp(const dtr_defl_s *D, const int *sites_by_colour, int ncolors, uint64_t seed, int64_t run,
                    int64_t q0, int nrhs, int dilute12, int b, double2 *d_dev, double2 *terms_dev, void *work,
                    size_t work_bytes, int sms, cudaStream_t st, const CodeXform *xf = nullptr,
                    double2 **C_out = nullptr, bool reuse_w = false);

// T_D = sum_m v_m^H g5 v_m / lambda_m from the stored V (FP64 accumulation).
int defl_trace_TD(dtr_defl_s *D, cudaStream_t st);

int device_sms();

}  // namespace dtr
