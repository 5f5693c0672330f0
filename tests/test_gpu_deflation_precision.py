"""GPU parity of the deflation space stored in BF16 and of the Galerkin (Gram)
correction against the oracle (same rounded V on both sides)."""
import numpy as np
import pytest

from oracle import deflation, exact, gamma_insertion as gi, noise, wilson
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
    N = Ad.shape[0]
    g5 = np.tile(np.array([1.0] * 6 + [-1.0] * 6), N // 12)
    return dict(dims=dims, m0=m0, Ad=Ad, Ainv=Ainv, V=V, lam=lam, lat=lat, g=dtr.gauge_from_host(lat, U), N=N, g5=g5)


def _zblock(c, seed, n):
    import torch
    Z = noise.noise_vectors(c["dims"], seed, 0, 16, False, 0, n)
    return Z, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()


def test_bf16_storage_matches_rounded_oracle(dtr, c4):
    """V stored in BF16: d_j, T_D and x0 equal the eigenvalue-form values for the
    BF16-rounded V (every kernel widens the stored values exactly)."""
    c = c4
    Vr = deflation.bf16_round(c["V"])
    D = dtr.defl_create(c["lat"], c["V"], c["lam"], prec="bf16")
    Z, z = _zblock(c, 3, 8)
    d, C, x0 = dtr.deflate_project(D, z, want_coeff=True, want_x0=True)
    Dm = (Vr / c["lam"]) @ (Vr.conj().T * c["g5"][None, :])
    d_ref = np.einsum("ij,ij->j", np.conj(Z), Dm @ Z)
    assert np.abs(d.cpu().numpy() - d_ref).max() <= 1e-11 * np.abs(d_ref).max()
    assert abs(D.T_D() - np.trace(Dm)) <= 1e-11 * abs(np.trace(Dm))
    assert np.abs(x0.cpu().numpy().T - Dm @ Z).max() <= 1e-11 * np.abs(Dm @ Z).max()


def test_gram_equals_eigenvalue_form_for_exact_pairs(dtr, c4):
    c = c4
    D0 = dtr.defl_create(c["lat"], c["V"], c["lam"])
    D1 = dtr.defl_create(c["lat"], c["V"], c["lam"]).gram(c["g"], c["m0"])
    Z, z = _zblock(c, 4, 8)
    d0, _, _ = dtr.deflate_project(D0, z)
    d1, _, _ = dtr.deflate_project(D1, z)
    assert np.abs(d1.cpu().numpy() - d0.cpu().numpy()).max() <= 1e-9 * np.abs(d0.cpu().numpy()).max()
    assert abs(D1.T_D() - D0.T_D()) <= 1e-10 * abs(D0.T_D())


@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_gram_matches_oracle_galerkin(dtr, c4, prec):
    """Rounded V + Galerkin correction: T_D, d_j, x0, the HP trace samples and a
    Gamma trace's T_D equal the oracle's Galerkin deflation of the same rounded V."""
    c = c4
    Vr = deflation.bf16_round(c["V"]) if prec == "bf16" else c["V"].astype(np.complex64).astype(np.complex128)
    Dg, TD, _ = deflation.galerkin(c["Ad"], Vr)
    D = dtr.defl_create(c["lat"], c["V"], c["lam"], prec=prec).gram(c["g"], c["m0"])
    assert abs(D.T_D() - TD) <= 1e-9 * abs(TD)
    Z, z = _zblock(c, 5, 8)
    d, _, x0 = dtr.deflate_project(D, z, want_x0=True)
    d_ref = np.einsum("ij,ij->j", np.conj(Z), Dg @ Z)
    assert np.abs(d.cpu().numpy() - d_ref).max() <= 1e-9 * np.abs(d_ref).max()
    assert np.abs(x0.cpu().numpy().T - Dg @ Z).max() <= 1e-9 * np.abs(Dg @ Z).max()
    p = dtr.trace_params(seed=8, n_z0=2, ncolors=16, nvec=16, block=16, gammas=[15],
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    for r in range(2):
        Zr = noise.noise_vectors(c["dims"], 8, r, 16, False, 0, 16)
        t_ref = np.einsum("ij,ij->j", np.conj(Zr), c["Ainv"] @ Zr) - np.einsum("ij,ij->j", np.conj(Zr), Dg @ Zr)
        assert np.abs(out["samples"][r] - t_ref).max() <= 1e-8 * np.abs(t_ref).max()
    G5 = gi.dense(gi.clifford(15), c["N"])
    td5 = np.trace(G5 @ Dg)
    assert abs(out["gamma"][0]["T_D"] - td5) <= 1e-9 * max(abs(td5), 1.0)


@pytest.mark.parametrize("dims,k,b,R", [((4, 4, 4, 4), 32, 16, 32), ((8, 8, 8, 8), 200, 16, 16),
                                        ((4, 4, 4, 8), 64, 3, 6), ((4, 4, 4, 8), 64, 5, 10),
                                        ((4, 4, 4, 4), 100, 32, 32), ((4, 4, 4, 4), 32, 64, 64)])
def test_tensor_core_contraction_matches_oracle(dtr, dims, k, b, R):
    """Plain Z4 blocks (one vector per run, blocks spanning runs) with a BF16
    deflation space take the tensor-core contraction (BF16 operands, FP32
    accumulation per dof chunk, FP64 across chunks): the per-sample deflation
    terms match the oracle's gamma5 form for the same rounded V to FP32
    accumulation accuracy, and T_D is exact."""
    lat = dtr.make_lattice(dims)
    U = synth.random_su3_links(dims, 0.5, 1000)
    g = dtr.gauge_from_host(lat, U)
    V = synth.random_orthonormal(lat.N, k, 7)
    lam = np.where(np.arange(k) % 2 == 0, 1.0, -1.0) * np.linspace(0.7, 1.6, k)
    D = dtr.defl_create(lat, V, lam, prec="bf16")
    p = dtr.trace_params(seed=5, n_z0=R, ncolors=1, nvec=1, block=b,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    n0 = dtr.tensor_core_contractions()
    out = dtr.trace_estimate(g, -0.4, D, p, want_replay=True)
    assert dtr.tensor_core_contractions() - n0 == (R + b - 1) // b    # one per block
    Vr = deflation.bf16_round(V)
    Z = np.stack([noise.z0_vector(5, r, lat.N) for r in range(R)], axis=1)
    d_ref = deflation.quadrature_gamma5(Vr, lam, Z)
    d_gpu = out["replay"][:, 0, :].sum(axis=1)
    assert np.abs(d_gpu - d_ref).max() <= 2e-5 * np.abs(d_ref).max()
    assert abs(D.T_D() - deflation.T_D_gamma5(Vr, lam)) <= 1e-12 * np.sum(1 / np.abs(lam))
