"""Certification of the mixed solvers' true residual when the solution is much
larger than the right-hand side.

The mixed solvers compute their certifying residual r = z - A y with the
stencil in double-float arithmetic, whose error grows like 1e-13 ||y|| / ||z||;
where ||y|| / ||z|| exceeds 30 the library takes the FP64 stencil for that
residual instead.  Here the free Wilson field at a small mass m0 = 0.02 and a
constant right-hand side (the zero-momentum mode, singular value m0) give
||y|| / ||z|| = 1 / m0 = 50, beside a random right-hand side in the same block
(||y|| / ||z|| of a few).  Every column must meet 1e-10 in the true residual the
oracle recomputes in FP64, and the constant column's solution must equal z / m0.
"""
import numpy as np
import pytest

from oracle import wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("solver", ["mixed_f32", "mixed_f16"])
@pytest.mark.parametrize("graph", [True, False])
def test_solution_dominated_columns_are_certified(solver, graph):
    import torch
    from paper_1603_05988_gb300 import dtr
    dims, m0 = (4, 4, 4, 4), 0.02
    U = synth.random_su3_links(dims, 0.0, 1)  # eps 0: unit links, the free field
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    rng = np.random.default_rng(7)
    spinor = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    Z = np.empty((lat.N, 2), dtype=np.complex128)
    Z[:, 0] = np.tile(spinor, lat.V)  # constant field: A z = m0 z
    Z[:, 1] = rng.standard_normal(lat.N) + 1j * rng.standard_normal(lat.N)
    p = dtr.solve_params(tol=1e-10, solver=solver, graph=graph)
    y, st = dtr.solve_batch(g, m0, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p)
    Y = y.cpu().numpy().T
    A = wilson.explicit(U, dims, m0)
    res = np.linalg.norm(Z - A @ Y, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.all(res <= 1e-10), res
    assert all(s["converged"] for s in st)
    assert np.linalg.norm(Y[:, 0]) / np.linalg.norm(Z[:, 0]) > 30
    assert np.abs(Y[:, 0] - Z[:, 0] / m0).max() <= 1e-8 * np.abs(Z[:, 0] / m0).max()
