"""GPU parity of the half-storage mixed solvers (DTR_SOLVER_MIXED_F16 / _BF16):
inner BiCGStab with its Krylov vectors stored in FP16 or BF16, FP32 arithmetic,
inside the FP64 defect-correction loop.

The storage precision only changes the path to the answer: the outer loop
stops on the FP64 true residual, so every check below is the same one the
FP64 and FP32-inner solvers meet (true residual <= tol recomputed by the
oracle; per-vector z^H A^-1 z within 1e-8 relative after solves to 1e-10).
"""
import numpy as np
import pytest

from oracle import noise, wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu

HALF = ["mixed_f16", "mixed_bf16"]


@pytest.fixture(scope="module")
def dtr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1603_05988_gb300 import dtr as _dtr
    return _dtr


def _setup(dtr, dims, eps, m0, seed):
    U = synth.random_su3_links(dims, eps, seed)
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    return U, lat, g


@pytest.mark.parametrize("solver", HALF)
@pytest.mark.parametrize("dims,nrhs,graph", [((4, 4, 4, 4), 16, True), ((4, 4, 4, 4), 16, False),
                                             ((8, 8, 8, 8), 16, True),
                                             ((4, 4, 4, 4), 3, True),     # block 4: the 4-column path
                                             ((4, 4, 4, 4), 2, True)])    # block 2: per-element path
def test_half_solve_true_residual(dtr, solver, dims, nrhs, graph):
    import torch
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 3, 2, 16, False, 0, nrhs)
    z = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    p = dtr.solve_params(tol=1e-10, solver=solver, graph=graph)
    y, st = dtr.solve_batch(g, -0.4, z, params=p)
    Y = y.cpu().numpy().T
    A = wilson.explicit(U, dims, -0.4)
    res = np.linalg.norm(Z - A @ Y, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.all(res <= 1e-10), res
    assert all(s["converged"] for s in st)
    # the half-storage inner solves stop at the storage's floor: more than one cycle
    assert max(s["restarts"] for s in st) >= 2


@pytest.mark.parametrize("solver", HALF)
def test_half_graph_matches_host_loop(dtr, solver):
    """Graph-driven and host-driven defect correction run the same kernels in the
    same order: bit-identical solutions and counts."""
    import torch
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 7, 1, 16, False, 0, 16)
    z = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    outs = []
    for graph in (False, True):
        y, st = dtr.solve_batch(g, -0.4, z, params=dtr.solve_params(tol=1e-10, solver=solver, graph=graph))
        outs.append((y.cpu().numpy(), [s["iterations"] for s in st], [s["restarts"] for s in st]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]


def test_half_solver_needs_persistent_engine(dtr):
    import torch
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    z = torch.from_numpy(np.ascontiguousarray(noise.noise_vectors(dims, 1, 0, 1, False, 0, 2).T)).cuda()
    with pytest.raises(dtr.DtrError) as e:
        dtr.solve_batch(g, -0.4, z, params=dtr.solve_params(tol=1e-10, solver="mixed_f16", engine="kernels"))
    assert e.value.code == dtr.DTR_EINVAL


@pytest.mark.parametrize("solver", HALF)
def test_half_trace_samples_match_oracle(dtr, solver):
    """Undeflated 16-colour HP estimate on 4^4: each sample z^H A^-1 z against the
    oracle's LU solve, 1e-8 relative (solves to 1e-10, cond ~ 11)."""
    dims, m0 = (4, 4, 4, 4), -0.4
    U, lat, g = _setup(dtr, dims, 0.5, m0, 1000)
    p = dtr.trace_params(seed=11, n_z0=2, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-10, solver=solver))
    out = dtr.trace_estimate(g, m0, None, p)
    assert out["all_converged"] and out["max_true_residual"] <= 1e-10
    Ainv = np.linalg.inv(wilson.dense(U, dims, m0))
    for r in range(2):
        Zr = noise.noise_vectors(dims, 11, r, 16, False, 0, 16)
        t_ref = np.einsum("ij,ij->j", np.conj(Zr), Ainv @ Zr)
        assert np.abs(out["samples"][r] - t_ref).max() <= 1e-8 * np.abs(t_ref).max()


def test_dslash_double_float_matches_oracle(dtr):
    """The double-float stencil of the outer-residual update (FP32 input, links split
    into FP32 hi + lo, exact products and sums) against the FP64 oracle on the same
    FP32-rounded input: within 1e-13 of the output's scale, while the plain FP32
    stencil is ~1e-7 off (so the check tells the two apart)."""
    import torch
    dims, m0 = (4, 4, 4, 8), -0.6
    U, lat, g = _setup(dtr, dims, 0.7, m0, 1001)
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((3, lat.N)) + 1j * rng.standard_normal((3, lat.N)))
    X = X.astype(np.complex64).astype(np.complex128)
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    ref = wilson.apply(U, dims, m0, X.T).T
    scale = np.abs(ref).max()
    err_df = np.abs(dtr.dslash(g, m0, x, prec="df32").cpu().numpy() - ref).max() / scale
    err_32 = np.abs(dtr.dslash(g, m0, x, prec="f32").cpu().numpy() - ref).max() / scale
    assert err_df <= 1e-13, err_df
    assert err_32 >= 1e-9, err_32


def test_half_inner_iterations_follow_fp32_storage(dtr):
    """At the same inner tolerance the FP16-stored inner BiCGStab takes the steps of
    the FP32-stored one: the same number of defect-correction cycles per column and
    iteration counts within rounding noise.  Its right-hand side is scaled to
    ||r32||^2 = 12 V, so the first step needs rho = rhat^H r0 = 12 V; a solver that
    started from rho = 1 (the FP32 scale) would take a near-zero first step in
    every cycle, about one wasted iteration per cycle and column (+10% here)."""
    import torch
    dims, m0 = (8, 8, 8, 8), -0.6
    U, lat, g = _setup(dtr, dims, 0.8, m0, 5)
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((8, lat.N)) + 1j * rng.standard_normal((8, lat.N))
    z = torch.from_numpy(Z).cuda()
    its, cyc = {}, {}
    for solver in ("mixed_f32", "mixed_f16"):
        p = dtr.solve_params(tol=1e-10, solver=solver, graph=False, inner_tol=3e-4)
        y, st = dtr.solve_batch(g, m0, z, params=p)
        assert all(s["converged"] for s in st)
        its[solver] = np.array([s["iterations"] for s in st])
        cyc[solver] = [s["restarts"] for s in st]
    assert cyc["mixed_f16"] == cyc["mixed_f32"], cyc
    assert np.abs(its["mixed_f16"] - its["mixed_f32"]).max() <= 3, its
    assert its["mixed_f16"].sum() <= 1.05 * its["mixed_f32"].sum(), its
