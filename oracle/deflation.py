"""Deflation space and deflated quadratures (oracle; test infrastructure).

Section 5.1: the deflation space is the k smallest singular triplets of A,
found as eigenpairs (Lambda, V) of A^H A.  Section 5.2: with U = A V Sigma^-1
and Sigma = Lambda^(1/2),
    T_D = Tr(V Sigma^-1 U^H) = Tr(Lambda^-1 V^H A^H V)
and each Hutchinson quadrature subtracts z^H V Lambda^-1 V^H (A^H z), so U is
never stored (Algorithm 1: the deflated part T_D and the deflation term).  This module evaluates exactly
those literal expressions with an explicit A^H.

The triplets themselves (small lattices only) come from the dense Hermitian
eigendecomposition of Q = gamma5 A: since gamma5 A is Hermitian (A is
gamma5-Hermitian) and Q^H Q = A^H A, its eigenvectors are right singular
vectors of A with sigma = |lambda|.  Ordering: |lambda| ascending, ties by
lambda ascending.  The signed lambda are returned too, because the CUDA
library takes the deflation space in that form.
"""
import numpy as np

from . import wilson as _wilson


def smallest_triplets(Adense, k):
    """(V, lam, sigma): k eigenvectors of gamma5 A with smallest |lambda|.

    gamma5 is taken from oracle.gamma via the spinor-level apply, not a table.
    """
    N = Adense.shape[0]
    G5A = _wilson.gamma5_vec(Adense)       # gamma5 applied to every column
    Q = 0.5 * (G5A + G5A.conj().T)          # symmetrise away rounding
    lam, W = np.linalg.eigh(Q)
    order = np.lexsort((lam, np.abs(lam)))
    lam = lam[order][:k]
    V = W[:, order][:, :k]
    return V, lam, np.abs(lam)


def T_D(AH, V, sigma):
    """Algorithm 1's deflated part: T_D = Tr(Lambda^-1 V^H A^H V) with Lambda = Sigma^2."""
    Lam = sigma ** 2
    AHV = AH @ V
    return complex(np.sum(np.einsum("im,im->m", np.conj(V), AHV) / Lam))


def quadrature(AH, V, sigma, z):
    """Algorithm 1's deflation term: z^H V Lambda^-1 V^H (A^H z).

    z may be (N,) or (N, nrhs); returns one value per column.
    """
    Lam = sigma ** 2
    Z = z if z.ndim == 2 else z[:, None]
    c = V.conj().T @ (AH @ Z)               # V^H (A^H z)      k x nrhs
    w = V.conj().T @ Z                      # V^H z            k x nrhs
    out = np.sum(np.conj(w) * c / Lam[:, None], axis=0)
    return out if z.ndim == 2 else out[0]


def quadrature_gamma5(V, lam, z):
    """The same deflation term with the left singular vectors taken from the
    right ones through gamma5 (U = gamma5 V sign(lambda), valid because
    gamma5 A is Hermitian): z^H V diag(1/lambda) V^H gamma5 z.

    For eigenvectors of gamma5 A this equals `quadrature` (pinned by a test);
    for any other (V, lambda) it is still an unbiased deflation of the
    estimator, whose deflated trace is `T_D_gamma5`.
    """
    Z = z if z.ndim == 2 else z[:, None]
    c = V.conj().T @ _wilson.gamma5_vec(Z)      # V^H gamma5 z
    w = V.conj().T @ Z                          # V^H z
    out = np.sum(np.conj(w) * c / lam[:, None], axis=0)
    return out if z.ndim == 2 else out[0]


def T_D_gamma5(V, lam):
    """Tr(V diag(1/lambda) V^H gamma5) = sum_m v_m^H gamma5 v_m / lambda_m."""
    return complex(np.sum(np.einsum("im,im->m", np.conj(V), _wilson.gamma5_vec(V)) / lam))


def deflation_operator(AH, V, sigma):
    """Dense D = V Lambda^-1 V^H A^H (small N), the deflated part of A^-1."""
    AHd = AH.toarray() if hasattr(AH, "toarray") else np.asarray(AH)
    return (V / (sigma ** 2)[None, :]) @ (V.conj().T @ AHd)


def bf16_round(V):
    """Round complex128 values to bfloat16 (round to nearest even on the float32 bits), returned as complex128:
    the copy a library keeps when it stores V in BF16."""
    def r(x):
        f = np.ascontiguousarray(x, dtype=np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(V.real) + 1j * r(V.imag)


def galerkin(Adense, V):
    """Galerkin deflation with a basis V that need not be orthonormal or exact (Section 5.2's
    V Lambda^-1 V^H A^H with Lambda replaced by the k x k matrix it approximates):
        G = V^H g5 A V,   D = V G^-1 V^H g5,   T_D = Tr(G^-1 V^H g5 V).
    Returns (D, T_D, G).  For exact orthonormal eigenvectors of g5 A, G = Lambda (signed)."""
    G5V = _wilson.gamma5_vec(V)
    G = G5V.conj().T @ (Adense @ V)
    Gi = np.linalg.inv(G)
    D = V @ Gi @ G5V.conj().T
    TD = complex(np.trace(Gi @ (V.conj().T @ G5V)))
    return D, TD, G


def galerkin_terms(Adense, V, Z):
    """d_j = z_j^H D z_j of the Galerkin deflation for the columns of Z, and T_D."""
    D, TD, _ = galerkin(Adense, V)
    return np.einsum("ij,ij->j", np.conj(Z), D @ Z), TD
