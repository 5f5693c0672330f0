"""Traces Tr(Gamma A^-1) with the deflation space reused (oracle; test infrastructure).

The paper (end of Section 5.2) notes that the same splitting serves traces with
an inexpensive matrix Gamma inserted:
    Tr(Gamma A^-1) = Tr(Gamma V Lambda^-1 V^H A^H) + Tr(Gamma A^-1 - Gamma V Lambda^-1 V^H A^H),
computed like Algorithm 1 with a Gamma product at each step.  This module is
that estimator in the paper's literal form (explicit A^H, Lambda = Sigma^2):
    T_D^G = Tr(Lambda^-1 V^H A^H Gamma V),
    t_j   = z_j^H Gamma y_j - z_j^H Gamma V Lambda^-1 V^H A^H z_j,   y_j = A^-1 z_j.

Gamma ranges over the 16 elements of the Clifford basis (acting on spin,
identity on colour):  Gamma_n = g1^n0 g2^n1 g3^n2 g4^n3 for the bits n0..n3 of
n = 0..15 (ordered product; Gamma_0 = 1, Gamma_15 = g1 g2 g3 g4 = g5).
"""
import numpy as np

from . import gamma as _gamma


def clifford(n):
    """4x4 spin matrix Gamma_n = g1^(n&1) g2^(n>>1&1) g3^(n>>2&1) g4^(n>>3&1)."""
    g = _gamma.gammas()
    G = np.eye(4, dtype=np.complex128)
    for mu in range(4):
        if (n >> mu) & 1:
            G = G @ g[mu]
    return G


def apply(G, X):
    """(Gamma (x) 1_colour) on every site of X: (N,) or (N, ncol), index 12*site + 3*spin + colour."""
    Y = X if X.ndim == 2 else X[:, None]
    Vs = Y.shape[0] // 12
    T = Y.reshape(Vs, 4, 3, -1)
    out = np.einsum("st,xtcj->xscj", G, T).reshape(Y.shape)
    return out if X.ndim == 2 else out[:, 0]


def dense(G, N):
    """Gamma (x) 1_colour on N = 12 V dofs as a dense matrix (small N only)."""
    return apply(G, np.eye(N, dtype=np.complex128))


def T_D_gamma(AH, V, sigma, G):
    """Tr(Gamma V Lambda^-1 V^H A^H) = Tr(Lambda^-1 V^H A^H Gamma V), Lambda = Sigma^2."""
    Lam = sigma ** 2
    M = V.conj().T @ (AH @ apply(G, V))
    return complex(np.sum(np.diag(M) / Lam))


def deflated_hp_gamma(AH, solve, Z, G, V=None, sigma=None, group=1):
    """Algorithm 1 with Gamma inserted, over the columns of Z (already z0 .* z_h).

    Returns dict(T_D, t per sample (sum over the dilution group), trace
    running mean + T_D after each sample)."""
    ncol = Z.shape[1]
    assert ncol % group == 0
    s = ncol // group
    TD = T_D_gamma(AH, V, sigma, G) if V is not None else 0.0
    Y = solve(Z)
    GY = apply(G, Y)
    q = np.einsum("ij,ij->j", np.conj(Z), GY)
    if V is not None:
        Lam = sigma ** 2
        left = V.conj().T @ apply(G.conj().T, Z)          # V^H Gamma^H z
        right = V.conj().T @ (AH @ Z)                      # V^H A^H z
        q = q - np.einsum("mj,m,mj->j", np.conj(left), 1.0 / Lam, right)
    t = q.reshape(s, group).sum(axis=1)
    trace = np.cumsum(t) / np.arange(1, s + 1) + TD
    return {"T_D": TD, "t": t, "trace": trace}
