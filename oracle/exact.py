"""Exact quantities the estimator targets (oracle; test infrastructure).

  trace_inverse_lu   Tr(A^-1) from a dense LU factorisation (small N).
  z4_variance        eq. (1.2), Section 1: Var = ||A^-1||_F^2 - sum_i |A^-1_ii|^2,
                     the off-diagonal Frobenius norm of A^-1.
  free_field_*       closed forms for U = 1 (all links identity).  In momentum
                     space A(p) = a_p + i sum_mu gamma_mu sin p_mu with
                     a_p = m0 + sum_mu (1 - cos p_mu), p_mu = 2 pi n_mu / L_mu,
                     so A(p)^-1 = (a_p - i sum gamma sin p)/(a_p^2 + sum sin^2 p)
                     (the gammas anticommute and square to 1).  Summing the
                     12 x 12 trace over momenta gives Tr(A^-1); every diagonal
                     entry equals Tr/N by translation invariance, and
                     ||A^-1||_F^2 = 12 sum_p 1/(a_p^2 + sum sin^2 p).  Section 6.1
                     uses the free-field spectrum to complete the singular
                     spectrum.
  theorem1_variance  Theorem 2.1, eqs. (2.2)-(2.3): Var(t(A_R)) from the SVD of
                     the (inverse) matrix and Delta = (U o conj V)^H (U o conj V).
  example_3x3        the 3x3 example after Theorem 2.1 (Section 2).
"""
import itertools

import numpy as np


def trace_inverse_lu(Adense):
    """Tr(A^-1) by LU: solve A X = I column block by column block."""
    Ainv = np.linalg.inv(Adense)
    return np.trace(Ainv), Ainv


def z4_variance(B):
    """eq. (1.2): ||B||_F^2 - sum_i |B_ii|^2 for the matrix whose trace is estimated."""
    return float(np.sum(np.abs(B) ** 2) - np.sum(np.abs(np.diag(B)) ** 2))


def z4_enumeration(B):
    """Mean and variance of z^H B z over ALL 4^n Z4 vectors (brute force, n <= 6)."""
    n = B.shape[0]
    vals = np.array([1, 1j, -1, -1j])
    samples = []
    for codes in itertools.product(range(4), repeat=n):
        z = vals[list(codes)]
        samples.append(np.vdot(z, B @ z))
    s = np.array(samples)
    mean = s.mean()
    var = np.mean(np.abs(s - mean) ** 2)
    return mean, var


def _momenta(dims):
    grids = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    return [g.ravel() for g in grids]


def free_field_trace(dims, m0):
    """Tr(A^-1) for U = 1 on a periodic lattice: 12 sum_p a_p/(a_p^2 + sum sin^2 p)."""
    p = _momenta(dims)
    a = m0 + sum(1.0 - np.cos(pm) for pm in p)
    s2 = sum(np.sin(pm) ** 2 for pm in p)
    return float(12.0 * np.sum(a / (a * a + s2)))


def free_field_frobenius2(dims, m0):
    """||A^-1||_F^2 for U = 1: 12 sum_p 1/(a_p^2 + sum sin^2 p)."""
    p = _momenta(dims)
    a = m0 + sum(1.0 - np.cos(pm) for pm in p)
    s2 = sum(np.sin(pm) ** 2 for pm in p)
    return float(12.0 * np.sum(1.0 / (a * a + s2)))


def free_field_z4_variance(dims, m0):
    """eq. (1.2) for U = 1: ||A^-1||_F^2 - N (Tr/N)^2 (all diagonal entries equal)."""
    N = 12 * int(np.prod(dims))
    tr = free_field_trace(dims, m0)
    return free_field_frobenius2(dims, m0) - tr * tr / N


def free_field_singular_values(dims, m0):
    """Singular values of A for U = 1: sqrt(a_p^2 + sum sin^2 p), each 12-fold."""
    p = _momenta(dims)
    a = m0 + sum(1.0 - np.cos(pm) for pm in p)
    s2 = sum(np.sin(pm) ** 2 for pm in p)
    return np.sort(np.repeat(np.sqrt(a * a + s2), 12))


def theorem1_variance(B, k):
    """Theorem 2.1: Var(t(B_R)) after deflating the k LARGEST singular triplets of B.

    B = U S V^H;  Delta_ml = sum_i conj(U_im) V_im U_il conj(V_il)  (eq. 2.2)
    Var(t(B_R)) = sum_{m>k} s_m^2 - sum_{m,l>k} s_m s_l Delta_ml      (eq. 2.3)
    """
    U, s, Vh = np.linalg.svd(B)
    V = Vh.conj().T
    W = U * np.conj(V)  # U o conj(V)
    Delta = W.conj().T @ W
    sr = s[k:]
    D = Delta[k:, k:]
    return float(np.real(np.sum(sr ** 2) - sr @ D @ sr))


def theorem1_difference(B, k):
    """eq. (2.4): Var(t(B)) - Var(t(B_R)) written with the k deflated triplets."""
    U, s, Vh = np.linalg.svd(B)
    V = Vh.conj().T
    W = U * np.conj(V)
    Delta = W.conj().T @ W
    N = len(s)
    out = 0.0
    for m in range(k):
        out += s[m] ** 2 * (1.0 - Delta[m, m])
        for l in range(m + 1, N):
            out -= s[m] * s[l] * (Delta[m, l] + Delta[l, m])
    return float(np.real(out))


def deflated_remainder(B, k):
    """B_R = U_2 S_2 V_2^H: B with its k largest singular triplets removed (eq. 2.1)."""
    U, s, Vh = np.linalg.svd(B)
    return (U[:, k:] * s[k:]) @ Vh[k:, :]


def example_3x3(d, s):
    """The Section 2 example: ratio Var(t(A)) / Var(t(A_R)) for parameters (d, s).

    U is the orthogonal factor of the QR factorisation of [[-1,d,d],[d,1,1],[d,1,-1]],
    A = U diag(1+2s, 1+s, 1) U^T and A_R drops the largest triplet.
    """
    M = np.array([[-1.0, d, d], [d, 1.0, 1.0], [d, 1.0, -1.0]])
    U, _ = np.linalg.qr(M)
    A = U @ np.diag([1 + 2 * s, 1 + s, 1.0]) @ U.T
    Ar = U[:, 1:] @ np.diag([1 + s, 1.0]) @ U[:, 1:].T
    return z4_variance(A) / z4_variance(Ar)
