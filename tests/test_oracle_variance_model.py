"""Pins of the variance model (Theorem 2, Remark 4, Corollary) and of the W_d
distance diagnostic (Section 6.2) of the oracle."""
import itertools

import numpy as np
import pytest

from oracle import noise, variance_model as vm


@pytest.mark.parametrize("hermitian", [False, True])
@pytest.mark.parametrize("k", [0, 4, 10])
def test_theorem2_by_monte_carlo_over_haar_singular_vectors(hermitian, k):
    """The theorem's hypothesis made literal: B = U Sigma V^H with Haar U, V
    (V = U when Hermitian); the average exact Z4 variance of the deflated
    B_R over many draws matches E Var to a few standard errors."""
    rng = np.random.default_rng(10 + k + 100 * hermitian)
    N = 24
    sig = np.sort(rng.uniform(0.1, 3.0, N))[::-1]
    vals = []
    for _ in range(1500):
        U = vm.haar_unitary(N, rng)
        W = U if hermitian else vm.haar_unitary(N, rng)
        vals.append(vm.z4_variance((U[:, k:] * sig[k:]) @ W[:, k:].conj().T))
    vals = np.array(vals)
    se = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - vm.expected_variance(sig, k, hermitian)) <= 5 * se + 1e-3 * vals.mean()


def test_remark4_undeflated_closed_forms():
    rng = np.random.default_rng(3)
    sig = np.sort(rng.uniform(0.5, 2.0, 30))[::-1]
    N = len(sig)
    mu0, V0 = sig.mean(), sig.var()
    assert np.isclose(vm.expected_variance(sig, 0, False), (N - 1) * (V0 + mu0 ** 2), rtol=1e-13)
    assert np.isclose(vm.expected_variance(sig, 0, True), N ** 2 * V0 / (N + 1), rtol=1e-13)


def test_corollary_nonhermitian_ratio_never_above_one():
    rng = np.random.default_rng(4)
    for _ in range(50):
        sig = np.sort(rng.lognormal(0, 1.5, 40))[::-1]
        r = [vm.variance_ratio(sig, k) for k in range(40)]
        assert all(x <= 1 + 1e-12 for x in r)
        # equal to (sum of the tail's squares) / (sum of all squares)
        assert np.isclose(r[7], np.sum(sig[7:] ** 2) / np.sum(sig ** 2), rtol=1e-12)


def test_z4_variance_by_enumeration():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    u = np.array([1, 1j, -1, -1j])
    vals = np.array([np.vdot(u[list(c)], B @ u[list(c)]) for c in itertools.product(range(4), repeat=5)])
    assert np.isclose(vals.mean(), np.trace(B), rtol=1e-12)
    assert np.isclose(np.mean(np.abs(vals - vals.mean()) ** 2), vm.z4_variance(B), rtol=1e-12)


def _rows_of_distance_function(dims, rows, f):
    V = int(np.prod(dims))
    out = []
    for i in rows:
        r = np.zeros(12 * V)
        for s in range(V):
            r[12 * s:12 * s + 12] = f(vm.site_distance(dims, i // 12, s))
        out.append(r)
    return out


def test_wd_of_a_distance_function():
    """B_ij = f(dist(site i, site j)) for every dof pair: W_d = 12 f(d)^2 (d > 0),
    11 f(0)^2 at d = 0 (the diagonal entry excluded)."""
    dims = (4, 4, 2, 4)
    f = lambda d: 2.0 ** (-d)
    rows = [0, 17, 200, 383]
    W = vm.wd(_rows_of_distance_function(dims, rows, f), rows, dims, 6)
    ref = np.array([11 * f(0) ** 2] + [12 * f(d) ** 2 for d in range(1, 7)])
    assert np.allclose(W, ref, rtol=1e-13)


def test_wd_probing_masks_short_distances():
    """With the probing mask of 32 colours no pair at distance 1, 2 or 3 shares a
    colour (the paper's 'first 3 distances'), and 16 colours leave distance 1 only."""
    dims = (8, 8, 8, 8)
    f = lambda d: 1.0 / (1 + d)
    rows = [5, 12 * 1234 + 3, 12 * 4000 + 11]
    B = _rows_of_distance_function(dims, rows, f)
    W32 = vm.wd(B, rows, dims, 5, ncolors=32)
    assert np.all(W32[1:4] == 0) and W32[4] > 0
    W16 = vm.wd(B, rows, dims, 3, ncolors=16)
    assert W16[1] == 0 and W16[2] > 0
