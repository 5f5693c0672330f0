"""GPU checks of the variance-model inputs and of the W_d diagnostic against the oracle."""
import numpy as np
import pytest

from oracle import deflation, exact, variance_model as vm, wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


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
    Ad = wilson.explicit(U, dims, m0).toarray()
    tr, Ainv = exact.trace_inverse_lu(Ad)
    V, lam, sig = deflation.smallest_triplets(Ad, 32)
    lat = dtr.make_lattice(dims)
    return dict(dims=dims, m0=m0, Ad=Ad, Ainv=Ainv, V=V, lam=lam, lat=lat, g=dtr.gauge_from_host(lat, U), N=Ad.shape[0])


DOFS = [0, 37, 400, 1111, 2047, 3071]


@pytest.mark.parametrize("deflate,ncolors", [(False, 0), (True, 0), (False, 16), (True, 16)])
def test_wd_matches_oracle_rows(dtr, c4, deflate, ncolors):
    from paper_1603_05988_gb300 import variance
    c = c4
    D = dtr.defl_create(c["lat"], c["V"], c["lam"]) if deflate else None
    W = variance.wd_diagnostic(c["g"], c["m0"], DOFS, 8, defl=D, ncolors=ncolors)
    B = c["Ainv"]
    if deflate:   # A_D^-1 = V Lambda^-1 V^H g5 with the signed eigenvalues of g5 A
        g5 = np.tile(np.array([1] * 6 + [-1] * 6), c["N"] // 12)
        B = B - (c["V"] / c["lam"]) @ (c["V"].conj().T * g5[None, :])
    ref = vm.wd([B[i] for i in DOFS], DOFS, c["dims"], 8, ncolors=ncolors)
    assert np.allclose(W, ref, rtol=1e-8, atol=1e-12 * ref.max())
    if ncolors == 16:
        assert W[1] < 1e-20 * ref.max() + 1e-300   # 16 colours: no same-colour pair at distance 1


def test_frobenius_estimate_and_model_inputs(dtr, c4):
    """frob2 of a trace run estimates ||A^-1||_F^2 without bias; the library's
    Theorem 2 curve from (||A^-1||_F^2, top singular values) equals the oracle's
    formula on the full spectrum."""
    from paper_1603_05988_gb300 import variance
    c = c4
    p = dtr.trace_params(seed=12, n_z0=24, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], None, p)
    F = float(np.sum(np.abs(c["Ainv"]) ** 2))
    assert abs(out["frob2"] - F) <= 5 * out["frob2_err"] + 1e-9 * F
    S = np.linalg.svd(c["Ainv"], compute_uv=False)
    top = variance.sigma_from_lambda(c["lam"])
    assert np.allclose(top, S[:32], rtol=1e-9)
    ev = variance.expected_variance(F, top, c["N"])
    ref = np.array([vm.expected_variance(S, k) for k in range(33)])
    assert np.allclose(ev, ref, rtol=1e-9)
    k, curve = variance.predict_k(F, top, c["N"], t_vector=1.0, t_per_k=1e-3)
    assert 0 <= k <= 32 and curve[k] == curve.min()
