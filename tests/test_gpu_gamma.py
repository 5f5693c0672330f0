"""GPU parity of the Gamma-insertion traces Tr(Gamma A^-1) (end of Section 5.2)
against the oracle's literal-form estimator, on identical noise."""
import numpy as np
import pytest

from oracle import deflation, exact, gamma_insertion as gi, noise, wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu

GAMMAS = [0, 1, 5, 10, 12, 15]


@pytest.fixture(scope="module")
def dtr():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_05988_gb300 import dtr as _dtr
    return _dtr


@pytest.fixture(scope="module")
def c4(dtr):
    dims, m0 = (4, 4, 4, 4), -0.4
    U = synth.random_su3_links(dims, 0.5, 1000)
    A = wilson.explicit(U, dims, m0)
    Ad = A.toarray()
    tr, Ainv = exact.trace_inverse_lu(Ad)
    V, lam, sig = deflation.smallest_triplets(Ad, 32)
    lat = dtr.make_lattice(dims)
    return dict(dims=dims, m0=m0, AH=wilson.explicit_dagger(U, dims, m0), Ad=Ad, Ainv=Ainv, V=V, lam=lam, sig=sig,
                lat=lat, g=dtr.gauge_from_host(lat, U), N=Ad.shape[0])


def _check(out, refs, tol_t=1e-8):
    for q, n in enumerate(GAMMAS):
        got, ref = out["gamma"][q], refs[n]
        assert got["n"] == n
        scale = max(np.abs(ref["t"]).max(), 1.0)
        assert np.abs(got["samples"].ravel() - ref["t"]).max() <= tol_t * scale, n
        assert abs(got["T_D"] - ref["T_D"]) <= 1e-11 * max(abs(ref["T_D"]), 1.0), n


@pytest.mark.parametrize("lanes", [1, 3])
def test_gamma_traces_hp_blocks_match_oracle(dtr, c4, lanes):
    """HP blocks (16 colours): V^H Gamma^H z from code-transformed per-colour sums."""
    c = c4
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=6, n_z0=3, ncolors=16, nvec=16, block=16, gammas=GAMMAS, lanes=lanes,
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    refs = {}
    for n in GAMMAS:
        ts = []
        for r in range(3):
            Z = noise.noise_vectors(c["dims"], 6, r, 16, False, 0, 16)
            o = gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, Z, gi.clifford(n), c["V"], c["sig"])
            ts.append(o["t"])
            T_D = o["T_D"]
        refs[n] = {"t": np.concatenate(ts), "T_D": T_D}
    _check(out, refs)
    # Gamma_0 = 1 reproduces the plain estimator's samples and trace
    assert np.abs(out["gamma"][0]["samples"] - out["samples"]).max() <= 1e-12 * np.abs(out["samples"]).max()
    assert abs(out["gamma"][0]["trace"] - out["trace"]) <= 1e-12 * abs(out["trace"])
    assert abs(out["gamma"][0]["T_D"] - out["T_D"]) <= 1e-12 * abs(out["T_D"])


def test_gamma_traces_plain_noise_match_oracle(dtr, c4):
    """Plain Z4 noise (no probing): the generic projection of Gamma^H Z."""
    c = c4
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=2, n_z0=8, ncolors=1, nvec=1, block=8, gammas=GAMMAS,
                         solve=dtr.solve_params(tol=1e-12))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    Z = np.stack([noise.z0_vector(2, r, c["N"]) for r in range(8)], axis=1)
    refs = {}
    for n in GAMMAS:
        o = gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, Z, gi.clifford(n), c["V"], c["sig"])
        refs[n] = {"t": o["t"], "T_D": o["T_D"]}
    _check(out, refs)


def test_gamma_traces_without_deflation(dtr, c4):
    c = c4
    p = dtr.trace_params(seed=4, n_z0=2, ncolors=16, nvec=16, block=16, gammas=[3, 15],
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], None, p)
    for q, n in enumerate([3, 15]):
        ts = []
        for r in range(2):
            Z = noise.noise_vectors(c["dims"], 4, r, 16, False, 0, 16)
            ts.append(gi.deflated_hp_gamma(c["AH"], lambda Z: c["Ainv"] @ Z, Z, gi.clifford(n))["t"])
        ref = np.concatenate(ts)
        assert np.abs(out["gamma"][q]["samples"].ravel() - ref).max() <= 1e-8 * np.abs(ref).max()
        assert out["gamma"][q]["T_D"] == 0


def test_gamma_traces_complete_probing_exact(dtr, c4):
    """256 colours x 12-fold dilution probe every diagonal entry of Gamma A^-1:
    each estimate equals the dense Tr(Gamma A^-1), with the deflation space reused."""
    c = c4
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=13, n_z0=1, ncolors=256, nvec=256, dilute12=True, block=64, gammas=GAMMAS,
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    scale = abs(np.trace(c["Ainv"]))
    for q, n in enumerate(GAMMAS):
        exact_tr = np.trace(gi.dense(gi.clifford(n), c["N"]) @ c["Ainv"])
        assert abs(out["gamma"][q]["trace"] - exact_tr) <= 1e-9 * scale, (n, out["gamma"][q]["trace"], exact_tr)
