"""Setup: approximate k smallest singular triplets of A for the deflation space.

Section 5.1 computes the deflation space once, before the estimator runs, as
the lowest eigenpairs of A^H A (the paper used an external eigensolver with a
multigrid preconditioner and a loose 1e-2 residual tolerance, which is enough
because the estimator stays unbiased for any deflation space).  Here the
eigenpairs of the Hermitian Q = gamma5 A (Q^H Q = A^H A, sigma = |lambda|) are
found by subspace iteration on B = Q^-1 = A^-1 gamma5 with a Rayleigh-Ritz
step for B (whose wanted eigenvalues 1/lambda are the exterior ones; a
Rayleigh-Ritz step for the indefinite Q itself would produce spurious
interior Ritz values):

    W = B X = A^-1 gamma5 X          batched solves through the library
    M = X^H W,  M c = mu c           (p x p, FP64, host; X orthonormal)
    Ritz pairs (1/mu, X c), sorted by |mu| descending
    X <- orth(W C)                   power step on the Ritz vectors

The solves run in libdtr; the p x p eigenproblem, the tall-skinny products
and the re-orthonormalisation use torch/numpy, off the estimator's hot path.
"""
import numpy as np


def _orthonormalise_rows(X):
    """CholeskyQR2 on the rows of X (p x N): Gram on the GPU, p x p Cholesky on the host."""
    import torch
    for _ in range(2):
        G = (X.conj() @ X.T).cpu().numpy()           # G[a, b] = x_a^H x_b
        G = 0.5 * (G + G.conj().T)
        L = np.linalg.cholesky(G)                     # G = L L^H
        Linv = np.linalg.inv(L)
        X = (torch.from_numpy(np.ascontiguousarray(Linv.conj())).to(X.device) @ X).contiguous()
    return X


def _gamma5(X):
    p, N = X.shape
    Y = X.clone()
    Y.view(p, N // 12, 4, 3)[:, :, 2:, :] *= -1
    return Y


def smallest_gamma5_eigpairs(gauge, m0, k, p=None, iters=100, tol=1e-2, seed=0, solve_tol=1e-8,
                             solver="mixed_f32", chunk=64, check_every=5, verbose=False):
    """Return (V (N, k) complex128 numpy, lam (k,) signed, rel. residuals (k,), iterations)."""
    import torch

    from . import dtr
    N = gauge.lat.N
    p = p or int(np.ceil(1.5 * k)) + 8
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    X = (torch.randn((p, N), generator=gen, dtype=torch.float64)
         + 1j * torch.randn((p, N), generator=gen, dtype=torch.float64)).to("cuda")
    X = _orthonormalise_rows(X)                       # rows: orthonormal basis vectors
    params = dtr.solve_params(tol=solve_tol, solver=solver)
    res = np.full(k, np.inf)
    lam = None
    Xr = None
    it = 0
    for it in range(1, iters + 1):
        G5X = _gamma5(X)
        W = torch.empty_like(X)
        for c0 in range(0, p, chunk):
            c1 = min(p, c0 + chunk)
            y, _ = dtr.solve_batch(gauge, m0, G5X[c0:c1].contiguous(), params=params, allow_notconv=True)
            W[c0:c1] = y
        M = (X.conj() @ W.T).cpu().numpy()            # M[a, b] = x_a^H Q^-1 x_b
        M = 0.5 * (M + M.conj().T)
        mu, c = np.linalg.eigh(M)
        order = np.argsort(-np.abs(mu))
        mu, c = mu[order], c[:, order]
        lam = 1.0 / mu
        Ct = torch.from_numpy(np.ascontiguousarray(c)).to("cuda")
        Xr = (Ct.T @ X).contiguous()                  # Ritz vectors (orthonormal rows)
        if it % check_every == 0 or it == iters:
            QX = _gamma5(dtr.dslash_many(gauge, m0, Xr[:k].contiguous(), chunk=chunk))
            r = QX - torch.from_numpy(lam[:k]).to("cuda")[:, None] * Xr[:k]
            res = torch.linalg.norm(r, dim=1).cpu().numpy() / np.abs(lam[:k])
            if verbose:
                print("subspace it %d: max rel residual %.3e, |lambda| %.4f..%.4f"
                      % (it, res.max(), abs(lam[0]), abs(lam[k - 1])))
            if res.max() <= tol:
                break
        X = _orthonormalise_rows((Ct.T @ W).contiguous())
    V = Xr[:k].cpu().numpy().T.copy()
    return V, np.asarray(lam[:k]), res, it
