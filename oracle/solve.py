"""Reference linear solvers for A y = z (oracle; test infrastructure).

The solve step of Algorithm 1 (A y = z); the paper does not name the solver.
The oracle uses methods different from the CUDA library's BiCGStab:
  dense_solve   LU (numpy.linalg.solve), small N;
  cgnr          conjugate gradients on the normal equations A^H A y = A^H z,
                run to a true relative residual ||z - A y|| / ||z|| <= tol.
"""
import numpy as np


def dense_solve(Adense, Z):
    return np.linalg.solve(Adense, Z)


def cgnr(A, Z, tol=1e-13, maxiter=20000, AH=None):
    """CG on A^H A y = A^H z for every column of Z (A: scipy sparse matrix, or
    any operator supporting A @ X together with its adjoint AH).

    Columns iterate together (each with its own scalars); iteration stops when
    every column's true residual ||z - A y|| / ||z|| is below tol.
    Returns (Y, iterations, relative true residuals).
    """
    Z = np.asarray(Z, dtype=np.complex128)
    single = Z.ndim == 1
    if single:
        Z = Z[:, None]
    if AH is None:
        AH = A.conj().T.tocsr()
    Y = np.zeros_like(Z)
    R = Z.copy()                     # r = z - A y
    S = AH @ R                       # s = A^H r (normal-equation residual)
    P = S.copy()
    gamma = np.sum(np.abs(S) ** 2, axis=0)
    znorm = np.linalg.norm(Z, axis=0)
    znorm[znorm == 0] = 1.0
    it = 0
    for it in range(1, maxiter + 1):
        Q = A @ P
        qq = np.sum(np.abs(Q) ** 2, axis=0)
        alpha = np.where(qq > 0, gamma / np.where(qq > 0, qq, 1.0), 0.0)
        Y += P * alpha
        R -= Q * alpha
        S = AH @ R
        gnew = np.sum(np.abs(S) ** 2, axis=0)
        beta = np.where(gamma > 0, gnew / np.where(gamma > 0, gamma, 1.0), 0.0)
        P = S + P * beta
        gamma = gnew
        if np.all(np.linalg.norm(R, axis=0) / znorm <= tol * 0.5):
            break
    res = np.linalg.norm(Z - A @ Y, axis=0) / znorm
    if single:
        return Y[:, 0], it, res
    return Y, it, res
