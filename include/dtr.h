/*
 * dtr.h -- C ABI of libdtr: the deflated Hutchinson estimator of Tr(A^-1) for
 * the 4D Wilson-Dirac matrix A on one NVIDIA GB300 (sm_103a).
 *
 * Method: Gambhir, Stathopoulos & Orginos, "Deflation as a method of variance
 * reduction for estimating the trace of a matrix inverse" (arXiv:1603.05988),
 * Algorithm 1 (deflatedHP), Section 5.2.  Each entry point below names the
 * passage that defines the operation it performs.
 *
 * ---------------------------------------------------------------- conventions
 * Lattice      periodic, dims = {Lx, Ly, Lz, Lt}, every extent even;
 *              site = x + Lx*(y + Ly*(z + Lz*t)); V = Lx*Ly*Lz*Lt.
 * Spinor field complex128 stored as interleaved (re, im) doubles; N = 12 V
 *              degrees of freedom, dof i = 12*site + 3*spin + colour
 *              (4 spins x 3 colours per site, Section 1).  A block of nrhs
 *              fields is column-major N x nrhs: complex element (i, j) at
 *              complex offset j*N + i.
 * Links        complex128, U[site][mu][a][b] (row a, column b of the SU(3)
 *              matrix U_mu(site)), mu = 0..3 <-> x, y, z, t: 4*V*9 complex.
 * Operator     (A psi)(x) = (4 + m0) psi(x)
 *                  - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                               + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]
 *              with the chiral basis gamma_k = [[0, -i s_k], [i s_k, 0]]
 *              (k = x, y, z; s_k Pauli), gamma_t = [[0, 1], [1, 0]],
 *              gamma_5 = diag(1, 1, -1, -1).  A is gamma_5-Hermitian:
 *              A^H = gamma_5 A gamma_5.
 *
 * Ownership    Vectors passed to an entry point are caller-owned memory; the
 *              library never frees them.  Pointers documented as "device"
 *              must be device memory (or managed) of the current device;
 *              "host" pointers are ordinary host memory.  Handles
 *              (dtr_lattice, dtr_gauge, dtr_defl) are opaque, own their
 *              device memory and are released with the matching
 *              dtr_destroy_* call.  Workspace is caller-owned device memory
 *              of at least the size the matching *_workspace_bytes call
 *              returns; its contents are scratch between calls.
 * Streams      `stream` is a cudaStream_t passed as void* (NULL = legacy
 *              default stream).  Work is stream-ordered; calls that return
 *              host values synchronise that stream before returning.
 * Errors       every int-returning call returns DTR_OK (0) or one of the
 *              DTR_E* codes; dtr_last_error() returns a message for the most
 *              recent failure on the calling thread.  No call aborts, traps
 *              or throws across the ABI.
 * Threads      handles may be shared between threads only for read-only use
 *              (concurrent calls that use one workspace race).
 */
#ifndef DTR_H
#define DTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DTR_OK 0
#define DTR_EINVAL 1     /* bad argument (null pointer, size, unsupported combination) */
#define DTR_ENOMEM 2     /* device allocation by a handle failed, or workspace too small */
#define DTR_ECUDA 3      /* a CUDA runtime call failed; message has the CUDA error */
#define DTR_ENOTCONV 4   /* solver hit maxiter; results and per-RHS stats still written */
#define DTR_ENAN 5       /* NaN/Inf met in a residual norm; per-RHS stats still written */
#define DTR_ETIMEOUT 6   /* a grid barrier of the persistent solver timed out (no hang: the kernel exits) */

typedef struct dtr_lattice_s *dtr_lattice;
typedef struct dtr_gauge_s *dtr_gauge;
typedef struct dtr_defl_s *dtr_defl;
typedef struct dtr_net_s *dtr_net;

/* Storage precision of a field or of the deflation space. */
typedef enum {
  DTR_F64 = 0,
  DTR_F32 = 1,
  DTR_BF16 = 2,
  DTR_F16 = 3,
  DTR_DF32 = 4  /* dtr_dslash only: input rounded to FP32, arithmetic in double-float (pairs of FP32
                   numbers with exact products and sums, ~2^-46 relative per operation) on links split
                   into FP32 hi + lo: the stencil of the mixed solvers' outer-residual update */
} dtr_prec;

/* Krylov solver for A y = z (the solve step of Algorithm 1; the paper does not name one). */
typedef enum {
  DTR_SOLVER_BICGSTAB_F64 = 0,   /* plain FP64 BiCGStab */
  DTR_SOLVER_MIXED_F32 = 1,      /* FP32 BiCGStab inner solves inside FP64 defect correction */
  DTR_SOLVER_FGMRES_NET = 2,     /* FP32 flexible GMRES(m) inner solves, right-preconditioned by a
                                    dtr_net, inside FP64 defect correction; falls back to the BiCGStab
                                    inner solve if a cycle cuts the true residual less than 10x */
  DTR_SOLVER_MIXED_F16 = 3,      /* as DTR_SOLVER_MIXED_F32, with the inner Krylov vectors (r, r^, p, v,
                                    s, t) stored in FP16 and the inner right-hand side scaled to entries of
                                    RMS 1; FP32 arithmetic and FP32 inner iterate; the stencil reads its
                                    input in FP16.  Persistent engine only.  inner_tol below 2e-4 is
                                    raised to 2e-4 (deeper inner solves of an FP16-stored recursion cost
                                    more iterations than the cycles they save) */
  DTR_SOLVER_MIXED_BF16 = 4      /* the same with BF16 storage; inner_tol floor 1e-2 */
} dtr_solver;

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char *dtr_last_error(void);

/* Library version string. */
const char *dtr_version(void);

/* Launch accounting of the persistent solver kernel (roofline figures).
 * Writes the totals accumulated since the last reset -- summed CUDA-event
 * duration of the persistent launches (ms, events recorded on the launching
 * stream), number of launches, and the sum over launches of (iterations
 * executed x lattice sites x block width) -- to the non-NULL outputs (host),
 * then, if enable >= 0, resets the totals and switches accounting on
 * (enable = 1) or off (0).  enable = -1 only reads.  Accounting adds two
 * event records per launch. */
int dtr_profile_persistent(int enable, double *ms, int64_t *launches, double *site_rhs_iterations);

/* Number of CUDA kernels the library has launched in this process (all
 * threads, all devices), for launch accounting by callers. */
uint64_t dtr_kernel_launches(void);

/* CUDA-graph use of the mixed solver (no_graph = 0, persistent engine): graphs captured so far and
 * graph launches, process-wide.  A graph is captured once per distinct argument set (device,
 * gauge, lattice, m0, buffers, block, tolerances, limits) and reused; at most 8 are cached. */
int dtr_graph_stats(uint64_t *captures, uint64_t *launches);

/* Self-test of the bounded grid barrier the persistent solver uses (its
 * failure-detection path, exercised without faulting anything): one block
 * waits at a barrier that expects two blocks, so the wait must give up after
 * about budget_cycles SM clock cycles (1 .. 2^31).  *timed_out (host)
 * receives 1 if the wait gave up, *error_word the barrier's error flag after
 * the kernel.  Synchronises `stream`.  The solver itself uses a budget of
 * about two seconds and turns a timed-out barrier into DTR_ETIMEOUT. */
int dtr_selftest_barrier(int64_t budget_cycles, int *timed_out, int *error_word, void *stream);

/* ------------------------------------------------------------------ lattice */
/* Describe a periodic 4D lattice (Section 6: 4D lattice, 12 dof per site).
 * dims: host array of 4 positive even extents.  *out receives the handle.
 * DTR_EINVAL if any extent is odd or < 2, or V * 12 overflows int32 ranges
 * the kernels index with (V <= 2^26). */
int dtr_make_lattice(const int dims[4], dtr_lattice *out);
void dtr_destroy_lattice(dtr_lattice lat);
/* Query: dims (4 ints), volume V and N = 12 V (any output may be NULL). */
int dtr_lattice_info(dtr_lattice lat, int dims[4], int64_t *volume, int64_t *ndof);

/* -------------------------------------------------------------------- gauge */
/* Random SU(3) gauge field generated on the device: the coefficient field of
 * the Dirac matrix of Section 6 (whose gauge ensembles are not available, so a
 * seeded random field stands in).  Every link is a pure function of
 * (seed, site, mu): U_mu(x) = exp(i eps H) with H = (G + G^H)/2 - Tr/3, G a
 * 3 x 3 matrix of complex Gaussians (real and imaginary parts N(0, 1)) drawn by
 * Philox4x64-10 (Salmon et al., SC'11) with key {seed, 1} and counters
 * {site, mu, c, 0}, c = 0..4, through Box-Muller on 53-bit uniforms
 * u = ((w >> 11) + 1/2) 2^-53: normal 4c + 2p and 4c + 2p + 1 are
 * sqrt(-2 ln u_2p) (cos, sin)(2 pi u_2p+1) of output words 2p, 2p + 1 of
 * counter c, and G_ab = n_2(3a+b) + i n_2(3a+b)+1.  The exponential is exact to
 * FP64 rounding (unitary, det 1).  eps in [0, 100] (eps = 0: the free field).
 * Builds the same internal copies as dtr_gauge_from_host.  Synchronous.
 * DTR_EINVAL (bad argument), DTR_ECUDA (allocation or launch failed). */
int dtr_make_gauge(dtr_lattice lat, double eps, uint64_t seed, dtr_gauge *out);
/* Upload SU(3) links (host pointer, canonical layout above, 4*V*9 complex128)
 * and build the library's internal copies (FP64, FP32, double-float split and
 * half precision).  Synchronous. */
int dtr_gauge_from_host(dtr_lattice lat, const double *links_host, dtr_gauge *out);
/* Copy the FP64 links back to a host buffer in the canonical layout. */
int dtr_gauge_to_host(dtr_gauge g, double *links_host);
void dtr_destroy_gauge(dtr_gauge g);

/* ------------------------------------------------------------------- dslash */
/* out = A in (dagger = 0) or out = A^H in (dagger = 1), for nrhs fields.
 * Operator definition above (the matrix of Algorithm 1; A^H is the product
 * of Algorithm 1's deflated part and deflation term).  in, out: device, canonical N x nrhs
 * complex128, must not overlap.  prec selects the arithmetic: DTR_F64;
 * DTR_F32 (fields rounded to FP32, FP32 math, result widened to FP64);
 * DTR_BF16 / DTR_F16 (half-precision storage of the fields and of the links,
 * all three rows by default, or the first two rows with the third rebuilt as
 * the conjugated cross product of the first two when dtr_half_link_rows()
 * returns 2; FP32 math; dagger = 0 only).
 * work: device workspace of dtr_dslash_workspace_bytes(lat, nrhs) bytes. */
size_t dtr_dslash_workspace_bytes(dtr_lattice lat, int nrhs);
int dtr_dslash(dtr_gauge g, double m0, const double *in, double *out, int nrhs, int dagger,
               dtr_prec prec, void *work, size_t work_bytes, void *stream);

/* Rows per link stored for the half-precision stencils: 3 (default; 240 B per site and right-hand side
 * in all) or 2 (environment DTR_HALF_LINKS=2 before the first gauge field: 192 B, the third row rebuilt
 * in registers as conj(row0 x row1)). */
int dtr_half_link_rows(void);

/* Benchmark hook for the stencil of the operator above: launches the
 * library's internal dslash kernel (the one the solver's fused kernels share)
 * `reps` times back to back on internal-layout fields of width nrhs held in
 * `work` (zero-filled first), times the launches with CUDA events recorded on
 * `stream`, and writes the average duration of one launch in milliseconds to
 * *avg_ms (host).  work: dtr_dslash_workspace_bytes(lat, nrhs) bytes.
 * Synchronises `stream`. */
int dtr_time_dslash(dtr_gauge g, double m0, int nrhs, dtr_prec prec, int reps, void *work, size_t work_bytes,
                    double *avg_ms, void *stream);

/* -------------------------------------------------------------------- noise */
/* Probing vectors z = z0 .* z_h (Algorithm 1; Section 5.2).
 *   z0(i)  = i^q(i), q(i) in {0,1,2,3} the 2-bit code of dof i taken from
 *            Philox4x64-10 (Salmon et al., SC'11) with key {seed, 0} and
 *            counter {i / 128, z0_index, 0, 0}: output word (i % 128) / 32,
 *            bits 2*(i % 32) .. 2*(i % 32) + 1.
 *   z_h    = Sylvester Hadamard column j over the hierarchical-probing colour
 *            of the dof's site: H[c, j] = (-1)^popcount(c & j).  Colours:
 *            bit 0 = parity of x+y+z+t; then for l = 0, 1, ...: 3 bits
 *            ((y>>l)&1, (z>>l)&1, (t>>l)&1), then 1 bit parity of
 *            sum_mu (x_mu >> (l+1)).  ncolors in {1, 2, 16, 32, 256, 512, ...}
 *            (1 = plain Z4 noise); every extent must be a multiple of the
 *            colouring period (2, 2, 4, 4, 8, 8, ... for those counts).
 *   dilute12 != 0: column q = 12*j + a keeps only dofs with i % 12 == a.
 * Writes columns q0 .. q0+nrhs-1 to out (device, canonical N x nrhs
 * complex128).  Bit-exact: every entry is exactly 0, +-1 or +-i. */
int dtr_gen_noise(dtr_lattice lat, uint64_t seed, int64_t z0_index, int ncolors, int dilute12,
                  int64_t q0, int nrhs, double *out, void *stream);

/* ------------------------------------------------------------------- solver */
typedef struct {
  double tol;          /* stop when ||z - A y|| / ||z|| <= tol (true residual: FP64 for the FP64
                          solver; for the mixed solvers z - A y with A y in double-float arithmetic,
                          relative error ~1e-13 ||y|| / ||z||) */
  int maxiter;         /* cap on inner iterations per RHS (summed over restarts) */
  int solver;          /* dtr_solver */
  int check_every;     /* iterations between host convergence checks (>= 1) */
  double inner_tol;    /* mixed solver: relative residual reduction per inner solve */
  int engine;          /* 0: persistent cooperative kernel (one launch per solve / inner solve);
                          1: one kernel per BiCGStab step, host polls every check_every iterations */
  int grid;            /* persistent engine: CTAs to launch (0 = every SM; clamped to what can be
                          co-resident) */
  dtr_net net;         /* DTR_SOLVER_FGMRES_NET: preconditioner (NULL = unpreconditioned FGMRES) */
  int gmres_m;         /* DTR_SOLVER_FGMRES_NET: restart length, 1..32 */
  int no_graph;        /* DTR_SOLVER_MIXED_F32 with the persistent engine: 0 = run the whole
                          defect-correction loop as one CUDA graph (a device-driven WHILE node,
                          no host round trip between cycles; the graph is captured on first use
                          and cached per argument set), 1 = host-driven launches */
} dtr_solve_params;

typedef struct {
  int iterations;      /* inner Krylov iterations this RHS was active */
  int restarts;        /* true-residual restarts / defect-correction cycles */
  int converged;       /* 1 if the true residual met tol */
  int pad_;
  double true_residual;/* ||z - A y|| / ||z|| recomputed in FP64 at exit */
} dtr_solve_stat;

/* Fill *p with defaults: tol 1e-10, maxiter 5000, FP64 BiCGStab, check 8,
 * inner_tol 1e-5, persistent engine. */
void dtr_solve_params_default(dtr_solve_params *p);

/* Solve A y = z for nrhs right-hand sides at once (the solve step of Algorithm 1).
 * z: device, canonical N x nrhs; y: device, canonical N x nrhs, used as the
 * initial guess on entry (zero it for none), solution on exit.  stats: host
 * array of nrhs entries, or NULL.  Returns DTR_ENOTCONV if any RHS missed
 * tol within maxiter (y and stats still written). */
size_t dtr_solve_workspace_bytes(dtr_lattice lat, int nrhs, const dtr_solve_params *p);
int dtr_solve_batch(dtr_gauge g, double m0, const double *z, double *y, int nrhs,
                    const dtr_solve_params *p, void *work, size_t work_bytes,
                    dtr_solve_stat *stats, void *stream);

/* --------------------------------------------------------------- deflation */
/* Deflation space (Section 5.2): k right singular vectors of A given as
 * eigenvectors v_m of the Hermitian matrix Q = gamma_5 A, with signed
 * eigenvalues lambda_m (sigma_m = |lambda_m|).  Then U = A V Sigma^-1 is
 * never formed: U = gamma_5 V sign(Lambda), and
 *   T_D = Tr(Lambda_{A^HA}^-1 V^H A^H V) = sum_m v_m^H gamma_5 v_m / lambda_m
 *   z^H V Lambda_{A^HA}^-1 V^H A^H z  = z^H V diag(1/lambda) V^H gamma_5 z.
 * V: HOST, canonical N x k complex128 column-major; lambda: host, k doubles
 * (non-zero).  The library copies V to device memory in precision prec
 * (DTR_F64, DTR_F32, or DTR_BF16 rounded to nearest even: 4 bytes per
 * complex value) and computes T_D in FP64 from the stored copy; every
 * kernel widens the stored values exactly to FP64, so the estimator stays
 * unbiased for the rounded V. */
int dtr_defl_create(dtr_lattice lat, int k, dtr_prec prec, const double *V_host,
                    const double *lambda_host, dtr_defl *out);
/* T_D (Algorithm 1's deflated part) as (re, im) in td[2] (host). */
int dtr_defl_trace(dtr_defl d, double td[2]);
/* Galerkin (Gram) correction, computed in FP64 on the GPU: with G = V^H gamma_5 A V
 * (k x k, A from gauge g at mass m0, V the stored copy widened exactly),
 * the deflation operator becomes D = V G^-1 V^H gamma_5 in place of
 * V Lambda^-1 V^H gamma_5: the same for exact eigenpairs, exact on span(V)
 * (D A v = v) for any basis, which matters when V is inexact or rounded to
 * FP32/BF16.  From then on T_D = Tr(G^-1 V^H gamma_5 V), d_j = c_j^H G^-1 g_j
 * (c = V^H z, g = V^H gamma_5 z), x0 = V G^-1 g, and T_D of a Gamma is
 * Tr(G^-1 V^H gamma_5 Gamma V); the per-m replay terms become conj(c_m)(G^-1 g)_m,
 * whose prefixes are no longer the k' < k estimates.  Cost: k FP64 stencils
 * plus two k x k x N FP64 contractions; G^-1 by Gauss-Jordan on the host.
 * Synchronises `stream`.  DTR_EINVAL if G is singular. */
int dtr_defl_gram(dtr_defl d, dtr_gauge g, double m0, void *stream);
void dtr_destroy_defl(dtr_defl d);

/* ------------------------------------------------------ setup eigensolver */
/* The deflation space of Section 5.1 computed on the GPU: the k eigenpairs of
 * Q = gamma_5 A with smallest |lambda| (the k smallest singular triplets of A,
 * sigma = |lambda|, U = gamma_5 V sign(lambda)), returned as a dtr_defl in
 * storage precision `store` without leaving the device.  The paper computes it
 * once before the estimator to a loose 1e-2 residual with an external
 * eigensolver; the estimator stays unbiased for any space (Section 5.2).
 * Method: Chebyshev-filtered subspace iteration on S = A^H A = Q^2 with a basis
 * of p >= k columns (degree `degree` per iteration, interval [cut, bound],
 * bound = (|4 + m0| + 4)^2 >= ||A||^2), then a harmonic Rayleigh-Ritz step for
 * the target 0 (H c = nu M c with H = Y^H Q Y, M = (QY)^H QY, nu = 1/lambda: the
 * wanted lambda are the pencil's exterior values, so no spurious Ritz values
 * near 0), signed lambda = the harmonic Ritz values 1/nu (equal to the Rayleigh quotients for
 * converged pairs; for unconverged ones |1/lambda| <= 1/sigma_min stays bounded).  The basis is stored
 * row-major [dof][p] in the handle's own buffer and compacted to [dof][k],
 * ordered by |lambda|; the Gram products, rotations and residuals (a fresh
 * stencil on the stored vectors) run in the library's kernels, the p x p
 * eigenproblems on the host (FP64 Householder tridiagonalisation and
 * implicit QL).  Memory: the handle holds N p elements
 * (16, 8 or 4 bytes) until destroyed; the workspace holds QY (N p elements),
 * four chunk fields and p x p matrices (dtr_eig_workspace_bytes). */
typedef struct {
  int k;               /* wanted eigenpairs (deflation vectors), >= 1 */
  int p;               /* basis columns, >= k (0: k + max(16, k / 8), rounded up to a multiple of 16) */
  int degree;          /* Chebyshev degree of every iteration after the first */
  int first_degree;    /* degree of the first iteration, from random vectors (0: degree) */
  int max_iter;        /* iterations at most */
  int chunk;           /* basis columns filtered at once (1..64; 0: 32) */
  dtr_prec store;      /* storage of the basis and of the result: DTR_F64 (FP64 stencils), DTR_F32 or DTR_BF16
                          (FP32 stencils) */
  int tol_ref;         /* 0: residuals relative to |lambda_j|; 1: relative to the bound |4 + m0| + 4 on ||A||
                          (the scale of a tolerance stated relative to the matrix norm) */
  double tol;          /* stop when every ||Q v_j - lambda_j v_j|| <= tol ref_j ||v_j||, j < k */
  double first_cut;    /* the first filter damps S above this value (0: a tenth of the bound) */
  double time_limit_s; /* stop after the iteration that passes this wall time (0: no limit) */
  uint64_t seed;       /* random start: Philox4x64-10 key {seed, 2} */
} dtr_eig_params;

typedef struct {
  int iterations;      /* iterations run */
  int converged;       /* of the k pairs, how many met tol */
  int basis;           /* p used */
  int pad_;
  double max_residual; /* largest relative residual of the k pairs */
  double seconds;      /* wall time of the call */
  double cut;          /* last filter interval [cut, bound] */
  double bound;
  double t_filter;     /* wall seconds in the Chebyshev filter and QY, */
  double t_gram;       /* in the three Gram products, */
  double t_host;       /* in the host Rayleigh-Ritz algebra, */
  double t_rotate;     /* and in the rotations and residuals */
} dtr_eig_stats;

/* Defaults: k 32, p 0, degree 48, first_degree 0, max_iter 100, chunk 32, DTR_F64, tol 1e-2. */
void dtr_eig_params_default(dtr_eig_params *p);
size_t dtr_eig_workspace_bytes(dtr_lattice lat, const dtr_eig_params *p);
/* residuals: host k doubles (the relative residual of each pair) or NULL; stats: host or NULL.
 * *out receives a new handle (destroy with dtr_destroy_defl) whose lambda are the signed Ritz
 * values and whose T_D is computed from the stored V.  Synchronises `stream`.  DTR_EINVAL (bad
 * parameters), DTR_ENOMEM (basis allocation failed or workspace too small), DTR_ENOTCONV (a
 * small eigenproblem failed, or the filtered basis lost rank below k), DTR_ECUDA.  Running out of
 * iterations or time is not an error: stats and residuals say how far it got. */
int dtr_eig_deflation(dtr_gauge g, double m0, const dtr_eig_params *p, void *work, size_t work_bytes,
                      double *residuals, dtr_eig_stats *stats, dtr_defl *out, void *stream);
/* Copy a deflation space back: V_host (host, canonical N x k column-major complex128, the stored
 * values widened exactly) and lambda_host (host, k); either may be NULL.  Synchronous. */
int dtr_defl_to_host(dtr_defl d, double *V_host, double *lambda_host);

/* Deflation projection of a block of probing vectors (Algorithm 1's deflation term,
 * second term; Section 5.2):
 *   C = V^H [Z, gamma_5 Z]                       (k x 2 nrhs, FP64)
 *   d_j = sum_m conj(C[m, j]) C[m, nrhs + j] / lambda_m
 * z: device, canonical N x nrhs.  d_out: device, nrhs complex128.
 * coeff_out: device k x 2 nrhs complex128 column-major, or NULL.
 * x0_out: device canonical N x nrhs, or NULL: receives the deflated solution
 *   V diag(1/lambda) V^H gamma_5 z = A_D^-1 z.
 * work: device workspace of dtr_deflate_workspace_bytes(d, nrhs) bytes. */
size_t dtr_deflate_workspace_bytes(dtr_defl d, int nrhs);
int dtr_deflate_project(dtr_defl d, const double *z, int nrhs, double *d_out, double *coeff_out,
                        double *x0_out, void *work, size_t work_bytes, void *stream);

/* Allocation-free variant of dtr_deflate_project, for callers that cannot
 * allocate device memory or supply a workspace (for instance an application
 * whose device memory is wholly owned by its own pool allocator, or a
 * fixed-memory production run that reserves all device memory up front).
 * There is no counterpart in the paper: it computes the same d_out (and
 * optionally coeff_out, same layouts as dtr_deflate_project; no x0) with its
 * scratch held in a fixed file-scope device array of about 4.3 MB, present on
 * every GPU that loads the library until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 * Limits: nrhs <= DTR_STATIC_MAX_RHS and k <= DTR_STATIC_MAX_K, else
 * DTR_EINVAL.  The first call in each CUDA context (with that context's device
 * current) looks up the array's device address, which is then cached under the
 * context's unique id, so a context created after a reset never reuses a stale
 * address; make that first call before any stream capture.  All calls share
 * the array: calls whose GPU work overlaps (other streams or host threads)
 * race, so serialise them.  It supports the eigenvalue form only
 * (DTR_EINVAL after dtr_defl_gram).  Cost: its partial kernel runs at most
 * 128 blocks, each walking V / 64 sites in turn, so at large lattices it is
 * far slower than dtr_deflate_project (it is meant for modest problems). */
#define DTR_STATIC_MAX_K 128
#define DTR_STATIC_MAX_RHS 16
int dtr_deflate_project_static(dtr_defl d, const double *z, int nrhs, double *d_out, double *coeff_out,
                               void *stream);

/* --------------------------------------------------- learned preconditioner */
/* A 4-layer 4D convolutional network M ~ A^-1 (the learned preconditioner of
 * the FGMRES solver; no counterpart in the paper, which does not name its
 * solver).  A field's 12 complex dofs per site are 24 real channels
 * (channel 2c+p = real (p=0) / imaginary (p=1) part of dof c).  Layer l is a
 * periodic 3^4 stencil W_l[o][co][ci], o = ((dt*3+dz)*3+dy)*3+dx for the
 * displacement (dx-1, dy-1, dz-1, dt-1), no bias:
 *   y = W_3 * phi(W_2 * phi(W_1 * phi(W_0 * x)))
 * phi = identity (act = 0) or leaky ReLU with slope 1/4 (act = 1).  Weights
 * are used in BF16 (FP32 master copy and Adam moments on the device);
 * arithmetic accumulates in FP32.  Weight arrays (host) are 4*81*24*24 FP32
 * in [l][o][co][ci] order. */
#define DTR_NET_LAYERS 4
#define DTR_NET_WEIGHTS (4 * 81 * 24 * 24)
/* weights_host NULL: identity at the centre offset (first layer times
 * init_scale) plus N(0, noise^2) from `seed`. */
int dtr_net_create(dtr_lattice lat, int act, const float *weights_host, double init_scale, double noise,
                   uint64_t seed, dtr_net *out);
void dtr_destroy_net(dtr_net net);
/* Copy the weights to host: master FP32 (bf16_rounded = 0) or the BF16 values
 * the kernels use (1). */
int dtr_net_get_weights(dtr_net net, int bf16_rounded, float *weights_host);
/* Arithmetic of the network's kernels.  DTR_BF16 (the default): the layers'
 * inputs and the back-propagated gradients are stored in BF16 and every
 * convolution runs on the tensor cores (tcgen05, FP32 accumulation), the weight
 * gradient on the CUDA cores from the BF16 fields; DTR_F32: FP32 fields and
 * CUDA-core convolutions.  Returns DTR_EINVAL for any other value. */
int dtr_net_set_precision(dtr_net net, dtr_prec prec);
size_t dtr_net_workspace_bytes(dtr_net net, int nrhs);
/* out = M in for nrhs fields (device, canonical N x nrhs complex128). */
int dtr_net_apply(dtr_net net, const double *in, double *out, int nrhs, void *work, size_t work_bytes,
                  void *stream);
/* One training step on (residual, error) pairs (in_j, target_j) with
 * A target_j = in_j (device, canonical).  Loss (host *loss):
 *   g == NULL:  L = sum_j |M in_j - target_j|^2 / |target_j|^2
 *   g != NULL:  L = sum_j |A M in_j - in_j|^2 / |in_j|^2  (A from g and m0;
 *               the residual norm of A M, which governs right preconditioning)
 * gradient dL/dW with respect to the BF16 weights (copied to grad_host if
 * non-NULL), and, if do_step, one Adam step (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8). */
int dtr_net_train_step(dtr_net net, dtr_gauge g, double m0, const double *in, const double *target, int nrhs,
                       double lr, int do_step, double *loss, float *grad_host, void *work, size_t work_bytes,
                       void *stream);

/* ---------------------------------------------------------------- estimator */
typedef struct {
  uint64_t seed;       /* noise seed (Philox key) */
  int64_t z0_first;    /* first z0 run index */
  int n_z0;            /* R: independent runs of Algorithm 1, one z0 each */
  int ncolors;         /* hierarchical-probing colours (1 = plain Z4 noise) */
  int nvec;            /* s: probing vectors per run (<= ncolors, or 1 if ncolors = 1) */
  int dilute12;        /* 12-fold spin-colour dilution of each probing vector */
  int block;           /* right-hand sides solved per launch */
  int use_x0;          /* start each solve from the deflated solution A_D^-1 z */
  dtr_solve_params solve;
  int lanes;           /* blocks in flight at once (0 or 1 = one at a time): each lane has its own
                          stream and workspace slice, and a solve whose grid is 0 runs on
                          (SMs / lanes) CTAs, so independent blocks share the GPU.  Used by the
                          persistent engine with the graph-driven mixed solver or the FP64 solver;
                          otherwise one lane.  Results do not depend on the lane count. */
  int n_gamma;         /* Gamma-insertion traces Tr(Gamma_n A^-1) estimated alongside (0..16) */
  int gamma[16];       /* their Clifford indices n (0..15): Gamma_n = g1^n0 g2^n1 g3^n2 g4^n3 for the
                          bits n0..n3 of n (Gamma_0 = 1, Gamma_15 = g5), chiral basis.  The same noise,
                          solves and deflation space serve every Gamma (end of Section 5.2). */
  int64_t vec_first;   /* first probing vector of each run: the call uses Hadamard columns vec_first ..
                          vec_first + nvec - 1 (<= ncolors; 0 for plain Z4 noise), so a run of Algorithm 1
                          can be split over several calls whose samples add up; trace_runs then averages
                          this call's vectors only.  0 = from the first vector. */
} dtr_trace_params;

typedef struct {
  double trace[2];      /* mean over runs of Trace_r (Algorithm 1's estimate), (re, im) */
  double T_D[2];        /* deflated part (Algorithm 1) */
  double var_runs;      /* sample variance over runs of Trace_r (complex form) */
  double jk_err;        /* delete-1 jackknife standard error of trace (complex form) */
  double var_samples;   /* sample variance of the individual samples t_j */
  int64_t n_solves;     /* right-hand sides solved */
  int64_t iterations;   /* inner Krylov iterations summed over right-hand sides */
  double max_true_residual;
  int all_converged;
  int pad_;
  /* optional caller-owned HOST outputs (NULL to skip):
   *   samples     2 * n_z0 * nvec doubles: t_j = sum over dilution of
   *               z^H y - z^H V Lambda^-1 V^H A^H z, run-major
   *   trace_runs  2 * n_z0 doubles: Trace_r after nvec vectors
   *   replay      2 * n_z0 * nvec * k doubles: per-vector, per-m deflation
   *               terms conj(C[m,j]) C[m,b+j] / lambda_m, so the estimate
   *               can be replayed for any k' <= k (Section 6.3) */
  double *samples;
  double *trace_runs;
  double *replay;
  /* Gamma-insertion outputs (params n_gamma > 0), index q over params.gamma:
   *   gamma_trace[2q..]  mean over runs of T_D^G + mean_j t_j^G, t_j^G = z^H Gamma y - z^H Gamma D z
   *   gamma_T_D[2q..]    T_D^G = Tr(Gamma V Lambda^-1 V^H g5) = sum_m v_m^H g5 Gamma v_m / lambda_m
   *   gamma_var_runs[q], gamma_jk_err[q]  as var_runs, jk_err
   *   gamma_samples      optional caller-owned HOST 2 * n_gamma * n_z0 * nvec doubles (q-major) */
  double *gamma_samples;
  double gamma_trace[32];
  double gamma_T_D[32];
  double gamma_var_runs[16];
  double gamma_jk_err[16];
  /* ||A^-1||_F^2 estimated as the mean over probing vectors of |A^-1 z|^2 (unbiased: E z z^H = 1),
   * and its standard error: the total the variance model (Theorem 2) starts from */
  double frob2;
  double frob2_err;
} dtr_trace_result;

/* Algorithm 1 (deflatedHP) for R = n_z0 runs: for each run r and each block
 * of probing vectors: generate z = z0_r .* z_h, project onto the deflation
 * space, solve A y = z, reduce t_j = z^H y - d_j in FP64; Trace_r = T_D +
 * mean_j t_j.  defl may be NULL (no deflation, T_D = 0).  work: device
 * workspace of dtr_trace_workspace_bytes bytes (it grows with lanes).  Waits for
 * the work already queued on `stream`, and returns with all its own work done. */
size_t dtr_trace_workspace_bytes(dtr_gauge g, dtr_defl d, const dtr_trace_params *p);
int dtr_trace_estimate(dtr_gauge g, double m0, dtr_defl d, const dtr_trace_params *p,
                       void *work, size_t work_bytes, dtr_trace_result *res, void *stream);

/* Deflation contraction C = V^H [Z, gamma_5 Z] of the estimator's probing blocks (entries 0, +-1, +-i)
 * when V is stored in BF16 and k is a multiple of 4 (rows of V TMA-addressable): a BF16 GEMM on the
 * tensor cores (tcgen05, A moved by TMA, FP32 accumulation in tensor memory per chunk of dofs, FP64
 * across chunks in a fixed order).  dtr_trace_estimate uses it for every such block that is not a
 * hierarchical-probing block of one z0 run (those take the per-colour addition pass).
 * dtr_time_deflate times it: CUDA events on `stream`, average ms per contraction of an nrhs-column Z4
 * block (nrhs 1..64, reps >= 1), after one warm-up; for other storage precisions it times the CUDA-core
 * contraction.  work: device, at least dtr_time_deflate_workspace_bytes(d, nrhs) bytes, caller-owned.
 * Returns DTR_EINVAL (bad arguments), DTR_ENOMEM (workspace too small), DTR_ETIMEOUT (a tensor-core
 * stage wait gave up; the kernel returned without faulting) or DTR_ECUDA.  Synchronises `stream`.
 * dtr_tensor_core_contractions counts tensor-core contractions launched in this process. */
size_t dtr_time_deflate_workspace_bytes(dtr_defl d, int nrhs);
int dtr_time_deflate(dtr_defl d, int nrhs, int reps, void *work, size_t work_bytes, double *avg_ms, void *stream);
uint64_t dtr_tensor_core_contractions(void);

/* ----------------------------------------------------------- diagnostics */
/* W_d distance diagnostic (Section 6.2).  cols: device, canonical N x ns complex128 (column q =
 * B e_(dofs[q]) for the matrix B under study, e.g. A^-1 or its deflated remainder; by
 * g5-Hermiticity a column has the moduli of the row the definition names); dofs: host, the ns
 * sampled dof indices; ncolors > 1 keeps only sites of the sampled site's probing colour (the mask
 * of ncolors normalised hierarchical-probing vectors), 0 or 1 none.  W (host, maxd + 1) receives
 * W_d = mean over q of (sum of |B_jq|^2 over dofs j != dofs[q] at sites of periodic Manhattan
 * distance d) / (number of sites at distance d).  Synchronises `stream`. */
int dtr_wd(dtr_lattice lat, const double *cols, const int64_t *dofs, int ns, int maxd, int ncolors, double *W,
           void *stream);

/* ------------------------------------------------------------- autotuner */
typedef struct {
  int lanes;                  /* chosen blocks in flight (trace_params.lanes) */
  int block;                  /* chosen right-hand sides per block (trace_params.block) */
  double rhs_per_s;           /* its measured throughput */
  int n_tried;                /* candidates timed (table below, in the order tried) */
  int cached;                 /* 1 if returned from the cache without timing */
  int table_lanes[16];
  int table_block[16];
  double table_rhs_per_s[16];
} dtr_tune_result;

/* Pick the launch shape of dtr_trace_estimate for this problem by timing it:
 * every candidate lane count (1, 2, 4, 8), and every RHS block (8, 16, 32, 64)
 * if p->block <= 0 (else p->block only), runs one warm-up and `reps` timed
 * waves of real trace estimates (lanes blocks each, on z0 runs reserved for
 * tuning; a wave is the first lanes x block probing columns of a run when a run
 * has more) on `stream`; the fastest in RHS solves per second wins.  The choice
 * is cached per (device, lattice, k, solver, engine, graph use, ncolors, nvec,
 * block, dilution); force = 1 re-times.  work holds up to
 * dtr_trace_autotune_workspace_bytes bytes; candidates whose workspace does not
 * fit in work_bytes are skipped (DTR_ENOMEM if none fits).  The caller then
 * sets p->lanes and p->block from the result. */
size_t dtr_trace_autotune_workspace_bytes(dtr_gauge g, dtr_defl d, const dtr_trace_params *p);
int dtr_trace_autotune(dtr_gauge g, double m0, dtr_defl d, const dtr_trace_params *p, int reps, int force,
                       void *work, size_t work_bytes, dtr_tune_result *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTR_H */
