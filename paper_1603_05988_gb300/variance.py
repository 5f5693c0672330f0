"""Variance model of the deflated estimator (Theorem 2, Corollary) and the W_d
distance diagnostic (Section 6.2), driven by the library.

Theorem 2 gives, for a matrix B = A^-1 whose singular vectors behave like random
unitaries, the expected Z4 variance after deflating its k largest singular
values sigma_1 >= ... >= sigma_k (the inverses of A's k smallest):
    E Var(k) = (N - k)(1 - 1/N)(V_k + mu_k^2) = (1 - 1/N) (||A^-1||_F^2 - sum_{m<=k} sigma_m^2),
so the whole curve follows from the deflation space's eigenvalues and one
number, ||A^-1||_F^2, which every trace run estimates for free (the mean of
|A^-1 z|^2 over its probing vectors, `frob2` of dtr.trace_estimate).  The
Corollary makes it monotone in k; weighing it against the cost per vector
predicts the k that minimises variance x time.  (A is not Hermitian; the
Hermitian form of the theorem needs the singular values' mean, which a trace
run does not estimate.)
"""
import numpy as np


def sigma_from_lambda(lam):
    """Singular values of A^-1 from the signed eigenvalues of g5 A (|lambda| = sigma(A)), descending."""
    return np.sort(1.0 / np.abs(np.asarray(lam, dtype=float)))[::-1]


def expected_variance(frob2, sigma_top, N, ks=None):
    """E Var(k) of Theorem 2 (non-Hermitian) for k = 0 .. len(sigma_top) (or the given ks)."""
    s2 = np.concatenate([[0.0], np.cumsum(np.asarray(sigma_top, dtype=float) ** 2)])
    ks = np.arange(len(s2)) if ks is None else np.asarray(ks)
    return (1.0 - 1.0 / N) * (frob2 - s2[ks])


def predict_k(frob2, sigma_top, N, t_vector, t_per_k):
    """k minimising E Var(k) x (t_vector + k t_per_k): time per vector at k = 0 and the
    added time per vector and deflation vector.  Returns (k, curve)."""
    ev = expected_variance(frob2, sigma_top, N)
    cost = t_vector + np.arange(len(ev)) * t_per_k
    curve = ev * cost
    return int(np.argmin(curve)), curve


def wd_diagnostic(gauge, m0, dofs, maxd, defl=None, ncolors=0, tol=1e-12):
    """W_d of B = A^-1 (or, with a deflation space, A^-1 - V Lambda^-1 V^H g5) from
    the library's own solves: columns B e_i for the sampled dofs (at most 64)."""
    import torch
    from . import dtr
    lat = gauge.lat
    dofs = np.asarray(dofs, dtype=np.int64)
    if len(dofs) > 64:
        raise ValueError("at most 64 sampled dofs per call")
    E = torch.zeros((len(dofs), lat.N), dtype=torch.complex128, device="cuda")
    E[torch.arange(len(dofs)), torch.from_numpy(dofs).cuda()] = 1.0
    Y, st = dtr.solve_batch(gauge, m0, E, params=dtr.solve_params(tol=tol, solver="f64"))
    if defl is not None:
        _, _, x0 = dtr.deflate_project(defl, E, want_x0=True)
        Y = Y - x0
    return dtr.wd(lat, Y, dofs, maxd, ncolors)
