"""Pins of the Gamma-insertion oracle (Tr(Gamma A^-1) with the deflation space
reused, end of Section 5.2) against what the mathematics fixes."""
import itertools

import numpy as np
import pytest

from oracle import deflation, estimator, exact, gamma, gamma_insertion as gi, noise, wilson
from paper_1603_05988_gb300 import synth


def test_clifford_basis():
    G = [gi.clifford(n) for n in range(16)]
    assert np.allclose(G[0], np.eye(4))
    assert np.allclose(G[15], gamma.gamma5())
    assert np.allclose(G[15], np.diag([1, 1, -1, -1]))
    for n in range(16):
        assert np.allclose(G[n] @ G[n].conj().T, np.eye(4))          # unitary
        assert np.count_nonzero(np.abs(G[n]) > 1e-12) == 4             # one entry per row
    gram = np.array([[np.trace(a.conj().T @ b) for b in G] for a in G])
    assert np.allclose(gram, 4 * np.eye(16))                            # a basis of 4x4 matrices


@pytest.fixture(scope="module")
def small():
    dims, m0 = (2, 2, 2, 4), -0.4
    U = synth.random_su3_links(dims, 0.5, 31)
    A = wilson.explicit(U, dims, m0)
    Ad = A.toarray()
    Ainv = np.linalg.inv(Ad)
    return dict(dims=dims, A=A, AH=wilson.explicit_dagger(U, dims, m0), Ad=Ad, Ainv=Ainv, N=Ad.shape[0])


@pytest.mark.parametrize("n", [0, 1, 6, 9, 15])
def test_full_deflation_gives_exact_trace(small, n):
    """k = N with exact triplets: D = A^-1, every t_j = 0, Trace = T_D^G = Tr(G A^-1)."""
    c = small
    G = gi.clifford(n)
    V, lam, sig = deflation.smallest_triplets(c["Ad"], c["N"])
    exact_tr = np.trace(gi.dense(G, c["N"]) @ c["Ainv"])
    Z = noise.noise_vectors(c["dims"], 3, 0, 1, False, 0, 3)
    out = gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, Z, G, V, sig)
    assert abs(out["T_D"] - exact_tr) <= 1e-10 * max(1.0, abs(exact_tr))
    assert np.abs(out["t"]).max() <= 1e-9 * abs(exact_tr if abs(exact_tr) > 1 else 1.0)


@pytest.mark.parametrize("n", [0, 3, 10, 15])
def test_complete_probing_with_dilution_is_exact(n):
    """Complete HP colouring of 4^4 (256 colours = every site) with 12-fold
    dilution: each column is supported on one dof, so any z0 gives Tr(G A^-1)."""
    dims, m0 = (4, 4, 4, 4), -0.4
    U = synth.random_su3_links(dims, 0.5, 1000)
    Ad = wilson.explicit(U, dims, m0).toarray()
    Ainv = np.linalg.inv(Ad)
    AH = wilson.explicit_dagger(U, dims, m0)
    G = gi.clifford(n)
    Z = noise.noise_vectors(dims, 5, 2, 256, True, 0, 256 * 12)
    out = gi.deflated_hp_gamma(AH, lambda Z: Ainv @ Z, Z, G, group=12)
    exact_tr = np.trace(gi.dense(G, Ad.shape[0]) @ Ainv)
    assert abs(out["trace"][-1] - exact_tr) <= 1e-11 * abs(np.trace(Ainv))


def test_z4_mean_and_variance_by_enumeration():
    """Every Z4 code on 6 of the 12 dofs of one site (the other 6 held at 1): the
    mean and variance of z^H (G B) z equal the closed forms that the argument
    behind eq. (1.2) gives for this partly fixed vector, for G = Gamma (x) 1."""
    rng = np.random.default_rng(4)
    N = 12                                   # one site: Gamma acts on its 4 spins x 3 colours
    B = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for n in (2, 7, 15):
        GB = gi.dense(gi.clifford(n), N) @ B
        vals = []
        units = np.array([1, 1j, -1, -1j])
        # 4^12 is too many; enumerate the first 6 dofs, the rest held at z = 1
        rest = np.ones(N - 6, dtype=np.complex128)
        for codes in itertools.product(range(4), repeat=6):
            z = np.concatenate([units[list(codes)], rest])
            vals.append(np.vdot(z, GB @ z))
        vals = np.array(vals)
        # exact values for z = (u, 1): mean = sum_{i<6} GB_ii + sum_{i,j>=6} GB_ij ; variance = sum over pairs
        # with at least one index < 6 and i != j of |GB_ij|^2
        M = GB
        mean = np.trace(M[:6, :6]) + M[6:, 6:].sum()
        var = (np.sum(np.abs(M[:6, :6]) ** 2) - np.sum(np.abs(np.diag(M[:6, :6])) ** 2)
               + np.sum(np.abs(M[:6, 6:].sum(axis=1)) ** 2) + np.sum(np.abs(M[6:, :6].sum(axis=0)) ** 2))
        assert abs(vals.mean() - mean) <= 1e-10 * abs(mean)
        assert abs(np.mean(np.abs(vals - vals.mean()) ** 2) - var) <= 1e-9 * var


def test_unbiased_for_any_deflation_space(small):
    """Tr(G D) + Tr(G (A^-1 - D)) = Tr(G A^-1) for arbitrary V, sigma: the expectation of the
    estimator (exact average over a complete set of unit vectors) is exact."""
    c = small
    N = c["N"]
    G = gi.clifford(5)
    V = synth.random_orthonormal(N, 7, 2)
    sig = np.linspace(0.5, 2.0, 7)
    out = gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, np.eye(N, dtype=np.complex128), G, V, sig)
    exact_tr = np.trace(gi.dense(G, N) @ c["Ainv"])
    assert abs(out["trace"][-1] - (out["T_D"] + out["t"].sum() / N)) <= 1e-12 * abs(exact_tr)   # running mean
    assert abs(out["T_D"] + out["t"].sum() - exact_tr) <= 1e-10 * abs(exact_tr)


def test_identity_gamma_is_the_plain_estimator(small):
    c = small
    V, lam, sig = deflation.smallest_triplets(c["Ad"], 9)
    Z = noise.noise_vectors(c["dims"], 8, 1, 1, False, 0, 6)
    a = gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, Z, gi.clifford(0), V, sig)
    b = estimator.deflated_hp(c["AH"], lambda Z: c["Ainv"] @ Z, Z, V, sig)
    assert np.allclose(a["t"], b["t"], rtol=1e-12, atol=1e-12)
    assert abs(a["T_D"] - b["T_D"]) <= 1e-12 * abs(b["T_D"])
