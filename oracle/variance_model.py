"""Variance model of the deflated estimator and the W_d distance diagnostic
(oracle; test infrastructure).

Theorem 2 (Section 4): with sigma_1 >= ... >= sigma_N the singular values of the
matrix B whose trace is estimated (here B = A^-1, so sigma_m = 1/sigma_m(A)),
deflating the k largest leaves N - k values with mean mu_k and variance V_k,
and for Z4 noise and singular vectors that behave like random unitaries
    non-Hermitian B:  E Var = (N - k)(1 - 1/N)(V_k + mu_k^2)
    Hermitian B:      E Var = (N - k)(V_k N/(N+1) + mu_k^2 k/(N+1)).
Corollary: the ratio to the undeflated value (k = 0) is <= 1 for non-Hermitian
B; for Hermitian B it is below 1 only under the stated condition.

W_d (Section 6.2): for a set S of sampled rows i (lattice dofs), the squared
entries |B_ij| over the sites j at lattice (periodic Manhattan) distance d,
averaged over the m_d such sites and over S.  Readings: a row's own site at
d = 0 counts its other dofs (the diagonal entry is excluded, as in eq. (1.2));
the probing mask (H H^H) uses normalised probing vectors, i.e. it keeps the
entries between sites of the same colour and zeroes the rest.
"""
import numpy as np

from . import noise as _noise


def tail_moments(sigma_desc, k):
    t = np.asarray(sigma_desc[k:], dtype=float)
    mu = t.mean()
    return mu, np.mean((t - mu) ** 2)


def expected_variance(sigma_desc, k, hermitian=False):
    """Theorem 2: E Var of the k-deflated Z4 estimator (sigma sorted descending)."""
    N = len(sigma_desc)
    mu, Vk = tail_moments(sigma_desc, k)
    if hermitian:
        return (N - k) * (Vk * N / (N + 1) + mu ** 2 * k / (N + 1))
    return (N - k) * (1.0 - 1.0 / N) * (Vk + mu ** 2)


def variance_ratio(sigma_desc, k, hermitian=False):
    """Corollary: E Var(k) / E Var(0)."""
    return expected_variance(sigma_desc, k, hermitian) / expected_variance(sigma_desc, 0, hermitian)


def haar_unitary(N, rng):
    """Haar-distributed unitary (QR of a complex Gaussian with the phases of R's diagonal removed)."""
    Z = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))


def z4_variance(B):
    """eq. (1.2): ||B - diag(diag(B))||_F^2."""
    return float(np.sum(np.abs(B) ** 2) - np.sum(np.abs(np.diag(B)) ** 2))


def site_distance(dims, s1, s2):
    """Periodic Manhattan distance between lattice sites (index x fastest)."""
    d = 0
    for L in dims:
        a, b = s1 % L, s2 % L
        s1 //= L
        s2 //= L
        t = abs(a - b)
        d += min(t, L - t)
    return d


def wd(B_rows, rows, dims, maxd, ncolors=0):
    """W_d for d = 0..maxd from the listed rows of B (B_rows[q] = row rows[q], length N = 12 V)."""
    V = int(np.prod(dims))
    col = _noise.hp_colour(dims, ncolors) if ncolors else np.zeros(V, dtype=np.int64)
    out = np.zeros(maxd + 1)
    counts = np.zeros(maxd + 1)
    # m_d: number of sites at distance d from a site (translation invariant)
    for s in range(V):
        d = site_distance(dims, 0, s)
        if d <= maxd:
            counts[d] += 1
    for q, i in enumerate(rows):
        si = i // 12
        acc = np.zeros(maxd + 1)
        for s in range(V):
            d = site_distance(dims, si, s)
            if d > maxd:
                continue
            if col[s] != col[si]:
                continue
            vals = np.abs(B_rows[q][12 * s:12 * s + 12]) ** 2
            if s == si:
                vals = vals.copy()
                vals[i % 12] = 0.0
            acc[d] += vals.sum()
        out += acc / counts
    return out / len(rows)

