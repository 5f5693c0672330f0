"""Pins of the oracle's counter-based random SU(3) gauge field (oracle.gauge).

Each check compares with something the definition or the mathematics fixes:
the Gaussian law of the Box-Muller normals, the second moments of a Gaussian
Hermitian traceless matrix, scipy's matrix exponential, unitarity and unit
determinant, and the first-order expansion for small eps.
"""
import numpy as np
import pytest
from scipy import linalg, stats

from oracle import gauge


def test_box_muller_normals_are_standard_gaussian():
    n = gauge.normals(11, np.repeat(np.arange(2500), 4), np.tile(np.arange(4), 2500)).ravel()
    assert abs(n.mean()) < 4 * 1 / np.sqrt(n.size)
    assert abs(n.var() - 1.0) < 4 * np.sqrt(2.0 / n.size)
    assert stats.kstest(n, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair and neighbouring pairs are uncorrelated
    m = gauge.normals(12, np.arange(20000), np.zeros(20000))
    c = np.corrcoef(m.T)
    assert np.abs(c - np.eye(20)).max() < 5 / np.sqrt(20000)


def test_generator_is_hermitian_traceless_with_gaussian_moments():
    n = 20000
    H = gauge.hermitian_generators(3, np.arange(n), np.full(n, 2))
    assert np.abs(H - np.conj(np.swapaxes(H, 1, 2))).max() == 0.0
    assert np.abs(np.trace(H, axis1=1, axis2=2)).max() < 1e-14
    # H_ab = (G_ab + conj G_ba)/2 off the diagonal: E|H_ab|^2 = 1;
    # H_aa = Re G_aa - mean: E H_aa^2 = 1 - 1/3
    off = np.abs(H[:, 0, 1]) ** 2
    assert abs(off.mean() - 1.0) < 5 * off.std() / np.sqrt(n)
    d = H[:, 1, 1].real ** 2
    assert abs(d.mean() - 2.0 / 3.0) < 5 * d.std() / np.sqrt(n)


@pytest.mark.parametrize("eps", [0.5, 0.8, 3.0])
def test_links_equal_scipy_expm_and_are_special_unitary(eps):
    sites, mu = np.arange(64), np.arange(64) % 4
    U = gauge.links_at(7, eps, sites, mu)
    H = gauge.hermitian_generators(7, sites, mu)
    for q in range(0, 64, 7):
        assert np.abs(U[q] - linalg.expm(1j * eps * H[q])).max() < 1e-13
    I = np.eye(3)
    assert np.abs(np.einsum("nab,ncb->nac", U, np.conj(U)) - I).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-13


def test_small_eps_is_first_order_in_h():
    sites, mu = np.arange(32), np.zeros(32)
    H = gauge.hermitian_generators(5, sites, mu)
    eps = 1e-6
    U = gauge.links_at(5, eps, sites, mu)
    assert np.abs(U - (np.eye(3) + 1j * eps * H)).max() < 10 * eps ** 2 * np.abs(H).max() ** 2
    assert np.abs(gauge.links_at(5, 0.0, sites, mu) - np.eye(3)).max() < 1e-14   # W W^H = 1 to rounding


def test_field_is_a_pure_function_of_seed_site_and_direction():
    dims = (2, 2, 2, 4)
    U = gauge.random_su3_links(dims, 0.8, 9)
    pick = np.array([3, 17, 31])
    for mu in range(4):
        assert np.array_equal(gauge.links_at(9, 0.8, pick, np.full(3, mu)), U[pick, mu])
    assert not np.allclose(gauge.random_su3_links(dims, 0.8, 10), U)
