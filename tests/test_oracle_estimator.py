"""Pins of the oracle's estimator, deflation and variance formulas.

Each test checks the oracle against something other than itself: exhaustive
enumeration, the exact trace from LU, Theorem 2.1 evaluated from an SVD,
statistics of many samples, the paper's 3x3 example, or trace identities
that hold for ANY deflation space.
"""
import os

import numpy as np
import pytest

from oracle import deflation, estimator, exact, noise, solve, wilson
from paper_1603_05988_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


@pytest.mark.parametrize("n,seed", [(3, 0), (4, 1), (5, 2)])
def test_z4_variance_formula_by_enumeration(n, seed):
    """eq. (1.2) equals the exact variance over all 4^n Z4 vectors."""
    B = _rand(n, seed)
    mean, var = exact.z4_enumeration(B)
    assert abs(mean - np.trace(B)) < 1e-12 * n
    assert abs(var - exact.z4_variance(B)) < 1e-11 * var


def test_z4_sample_variance_matches_closed_form():
    """4096 Z4 samples of z^H A^-1 z at 2^4: sample mean/variance inside 5-sigma bands."""
    dims = (2, 2, 2, 2)
    U = synth.random_su3_links(dims, 0.5, 1)
    A = wilson.dense(U, dims, -0.4)
    tr, Ainv = exact.trace_inverse_lu(A)
    N = A.shape[0]
    Z = np.stack([noise.z0_vector(5, r, N) for r in range(4096)], axis=1)
    t = np.einsum("ij,ij->j", np.conj(Z), Ainv @ Z)
    v = exact.z4_variance(Ainv)
    assert abs(t.mean() - tr) < 5.0 * np.sqrt(v / len(t))
    dev = np.abs(t - t.mean()) ** 2
    assert abs(dev.mean() - v) < 5.0 * dev.std() / np.sqrt(len(t))


@pytest.mark.parametrize("k", [0, 1, 4, 10, 19])
def test_theorem1_matches_direct_deflated_variance(k):
    B = _rand(20, 7)
    direct = exact.z4_variance(exact.deflated_remainder(B, k))
    assert abs(exact.theorem1_variance(B, k) - direct) < 1e-10 * max(1.0, direct)
    diff = exact.z4_variance(B) - direct
    assert abs(exact.theorem1_difference(B, k) - diff) < 1e-9 * max(1.0, abs(diff))


def test_paper_3x3_example_outcomes():
    rows = []
    with open(os.path.join(GOLDEN, "example_3x3_section2.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                s, lo, hi, what = line.split()
                rows.append((float(s), float(lo), float(hi), what))
    assert len(rows) == 7
    for s, lo, hi, what in rows:
        ds = np.geomspace(lo, hi, 41)
        r = np.array([exact.example_3x3(d, s) for d in ds])   # Var(A)/Var(A_R)
        if what == "no_reduction":
            assert np.all(r <= 1.0 + 1e-12), (s, lo, hi)
        elif what == "reduction":
            assert np.all(r[1:] > 1.0), (s, lo, hi)
        else:
            assert np.all(np.abs(r - 1.0) < 1e-4), (s, lo, hi)


def test_triplets_are_smallest_singular_triplets():
    dims = (2, 2, 2, 4)
    U = synth.random_su3_links(dims, 0.8, 3)
    A = wilson.dense(U, dims, -0.7)
    V, lam, sig = deflation.smallest_triplets(A, 12)
    sv = np.sort(np.linalg.svd(A, compute_uv=False))
    assert np.allclose(sig, sv[:12], rtol=1e-12)
    # A^H A v = sigma^2 v and V orthonormal
    assert np.abs(A.conj().T @ (A @ V) - V * sig ** 2).max() < 1e-12
    assert np.abs(V.conj().T @ V - np.eye(12)).max() < 1e-12


def _small_problem(dims=(2, 2, 2, 2), eps=0.5, m0=-0.4, seed=1000):
    U = synth.random_su3_links(dims, eps, seed)
    A = wilson.explicit(U, dims, m0)
    AH = wilson.explicit_dagger(U, dims, m0)
    Ad = A.toarray()
    tr, Ainv = exact.trace_inverse_lu(Ad)
    return U, A, AH, Ad, tr, Ainv


def test_full_deflation_gives_exact_trace():
    """k = N: D = A^-1, every sample vanishes and Trace = T_D = Tr(A^-1)."""
    U, A, AH, Ad, tr, Ainv = _small_problem()
    N = Ad.shape[0]
    V, lam, sig = deflation.smallest_triplets(Ad, N)
    Z = np.stack([noise.z0_vector(1, r, N) for r in range(8)], axis=1)
    out = estimator.deflated_hp(AH, lambda Z: solve.dense_solve(Ad, Z), Z, V, sig)
    assert abs(out["T_D"] - tr) < 1e-11 * abs(tr)
    assert np.abs(out["t"]).max() < 1e-10 * abs(tr)
    assert abs(out["trace"][-1] - tr) < 1e-11 * abs(tr)


def test_complete_probing_is_exact_any_deflation_space():
    """4^4 with 256 colours x 12 dilution probes every entry: the estimate is
    exact for any z0 -- and, by linearity of the trace, for ANY (V, sigma)."""
    dims = (4, 4, 4, 4)
    U, A, AH, Ad, tr, Ainv = _small_problem(dims)
    N = Ad.shape[0]
    Z = noise.noise_vectors(dims, 9, 0, 256, True, 0, 3072)
    solve_fn = lambda Z: Ainv @ Z
    out = estimator.deflated_hp(AH, solve_fn, Z, group=12)
    assert abs(out["trace"][-1] - tr) < 1e-12 * abs(tr)
    V = synth.random_orthonormal(N, 10, 4)
    sig = np.linspace(0.3, 2.0, 10)
    out = estimator.deflated_hp(AH, solve_fn, Z, V, sig, group=12)
    assert abs(out["trace"][-1] - tr) < 1e-12 * abs(tr)
    # T_D is exactly the trace of the deflated operator D = V Lambda^-1 V^H A^H
    D = deflation.deflation_operator(AH, V, sig)
    assert abs(out["T_D"] - np.trace(D)) < 1e-12 * abs(np.trace(D))


def test_deterministic_hp_estimate_at_a_closing():
    """With z0 = 1 and all c vectors of a level, the estimate is the sum of the
    A^-1 entries joining same-colour sites (diagonal blocks' spin-colour traces
    included) -- the probing identity behind Section 1's description of HP."""
    dims = (4, 4, 4, 4)
    U, A, AH, Ad, tr, Ainv = _small_problem(dims)
    N = Ad.shape[0]
    c = np.repeat(noise.hp_colour(dims, 32), 12)
    H = noise.hadamard_entry(c[:, None], np.arange(32)[None, :]).astype(np.complex128)
    est = np.mean(np.einsum("ij,ij->j", H.conj(), Ainv @ H))
    same = (c[:, None] == c[None, :])
    assert abs(est - np.sum(Ainv[same])) < 1e-12 * abs(est)


def test_deflation_with_exact_triplets_matches_theorem1():
    """Deflating A^-1 with its k largest triplets (= A's k smallest) through the
    paper's T_D / quadrature form removes exactly the variance Theorem 2.1 gives."""
    U, A, AH, Ad, tr, Ainv = _small_problem()
    k = 24
    V, lam, sig = deflation.smallest_triplets(Ad, k)
    D = deflation.deflation_operator(AH, V, sig)
    assert abs(exact.z4_variance(Ainv - D) - exact.theorem1_variance(Ainv, k)) < 1e-9 * exact.z4_variance(Ainv)


def test_cgnr_reaches_tolerance():
    dims = (4, 4, 4, 4)
    U, A, AH, Ad, tr, Ainv = _small_problem(dims)
    Z = noise.noise_vectors(dims, 2, 0, 16, False, 0, 4)
    Y, it, res = solve.cgnr(A, Z, tol=1e-13)
    assert np.all(res <= 1e-13)
    assert np.abs(Y - Ainv @ Z).max() < 1e-11 * np.abs(Y).max()


def test_jackknife_of_mean_equals_textbook_variance_of_mean():
    x = np.random.default_rng(0).standard_normal(40) + 1j * np.random.default_rng(1).standard_normal(40)
    m, v = estimator.jackknife_mean(x)
    assert abs(m - x.mean()) < 1e-15
    assert abs(v - estimator.sample_variance(x) / len(x)) < 1e-14


def test_deflated_quadrature_equals_gamma5_form():
    """With V from gamma5 A, the paper's z^H V Lambda^-1 V^H A^H z equals
    z^H V diag(1/lambda) V^H gamma5 z (both evaluated here in FP64)."""
    U, A, AH, Ad, tr, Ainv = _small_problem((2, 2, 2, 4))
    N = Ad.shape[0]
    V, lam, sig = deflation.smallest_triplets(Ad, 16)
    Z = noise.noise_vectors((2, 2, 2, 4), 4, 1, 16, False, 0, 16)
    d_paper = deflation.quadrature(AH, V, sig, Z)
    d_g5 = deflation.quadrature_gamma5(V, lam, Z)
    assert np.abs(d_paper - d_g5).max() < 1e-12 * np.abs(d_paper).max()
    assert abs(deflation.T_D(AH, V, sig) - deflation.T_D_gamma5(V, lam)) < 1e-12 * abs(deflation.T_D(AH, V, sig))


def test_gamma5_form_unbiased_for_any_deflation_space():
    """Complete probing at 4^4: T_D_gamma5 + mean(t) = Tr(A^-1) for a random
    V and random signed lambda (trace linearity)."""
    dims = (4, 4, 4, 4)
    U, A, AH, Ad, tr, Ainv = _small_problem(dims)
    N = Ad.shape[0]
    V = synth.random_orthonormal(N, 12, 8)
    lam = np.linspace(-1.5, 1.7, 12) + 0.05
    Z = noise.noise_vectors(dims, 4, 0, 256, True, 0, 3072)
    t = np.einsum("ij,ij->j", np.conj(Z), Ainv @ Z) - deflation.quadrature_gamma5(V, lam, Z)
    est = deflation.T_D_gamma5(V, lam) + t.sum() / 256
    assert abs(est - tr) < 1e-11 * abs(tr)


def test_galerkin_deflation_pins():
    """Galerkin deflation D = V (V^H g5 A V)^-1 V^H g5: equals the literal Lambda form for exact
    eigenvectors; for ANY basis (rounded to BF16, or a random one) D A is the identity on
    span(V), and T_D = Tr(D)."""
    from oracle import deflation, wilson
    from paper_1603_05988_gb300 import synth
    dims, m0 = (2, 2, 2, 4), -0.4
    U = synth.random_su3_links(dims, 0.5, 44)
    Ad = wilson.explicit(U, dims, m0).toarray()
    AH = wilson.explicit_dagger(U, dims, m0)
    V, lam, sig = deflation.smallest_triplets(Ad, 10)
    D, TD, G = deflation.galerkin(Ad, V)
    assert np.allclose(G, np.diag(lam), atol=1e-12)
    assert abs(TD - deflation.T_D(AH, V, sig)) <= 1e-12 * abs(TD)
    Z = np.eye(Ad.shape[0])[:, :7] * (1 + 1j)
    d, _ = deflation.galerkin_terms(Ad, V, Z)
    assert np.allclose(d, [deflation.quadrature(AH, V, sig, Z[:, j]) for j in range(7)], rtol=1e-11)
    rng = np.random.default_rng(2)
    for W in (deflation.bf16_round(V), V @ (rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10)))):
        D, TD, _ = deflation.galerkin(Ad, W)
        assert np.allclose(D @ (Ad @ W), W, atol=1e-9 * np.abs(W).max())
        assert abs(TD - np.trace(D)) <= 1e-10 * abs(TD)


def test_bf16_round_is_round_to_nearest_even():
    from oracle import deflation
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -3.14159265, 1e-3])
    r = deflation.bf16_round(x + 0j).real
    assert r[0] == 1.0
    assert r[1] == 1.0                       # exactly half an ulp (2^-7 at 1): tie, to the even mantissa
    assert r[3] == 1.0                       # a quarter ulp rounds down
    assert r[2] == 1.0 + 2 ** -7             # three quarters of an ulp rounds up
    assert abs(r[4] + 3.140625) < 1e-12      # 8-bit mantissa
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x))
