"""GPU checks of the learned preconditioner and the FGMRES solver.

* network forward and gradient through the C ABI against the oracle's plain
  numpy network (same BF16-rounded weights, inputs rounded to FP32);
* training on (residual, error) pairs produced by the library's own solver
  lowers the loss;
* FGMRES (with and without the network) reaches the true-residual tolerance,
  the trained network cuts the Arnoldi steps, and the trace estimated through
  the FGMRES path matches the oracle.
"""
import numpy as np
import pytest

from oracle import convnet, deflation, estimator, exact, noise, wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dtr():
    import torch
    assert torch.cuda.is_available()
    from paper_1603_05988_gb300 import dtr as _dtr
    return _dtr


def _c64(x):
    return x.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("dims,nrhs", [((2, 2, 2, 2), 1), ((2, 2, 2, 4), 3)])
def test_net_forward_matches_oracle(dtr, act, dims, nrhs):
    import torch
    lat = dtr.make_lattice(dims)
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=3)
    rng = np.random.default_rng(5)
    X = _c64(rng.standard_normal((lat.N, nrhs)) + 1j * rng.standard_normal((lat.N, nrhs)))
    y = net.apply(torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T
    Ws = [w.astype(np.float64) for w in net.weights(bf16_rounded=True)]
    ref, _, _ = convnet.forward(Ws, X, dims, act)
    assert np.abs(y - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("residual", [False, True])
def test_net_gradient_matches_oracle(dtr, act, residual):
    import torch
    dims = (2, 2, 2, 4)
    lat = dtr.make_lattice(dims)
    U = synth.random_su3_links(dims, 0.5, 21)
    g = dtr.gauge_from_host(lat, U)
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=4)
    rng = np.random.default_rng(6)
    X = _c64(rng.standard_normal((lat.N, 2)) + 1j * rng.standard_normal((lat.N, 2)))
    E = _c64(rng.standard_normal((lat.N, 2)) + 1j * rng.standard_normal((lat.N, 2)))
    loss, grad = net.train_step(torch.from_numpy(np.ascontiguousarray(X.T)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(E.T)).cuda(), step=False, want_grad=True,
                                gauge=g if residual else None, m0=-0.4)
    Ws = [w.astype(np.float64) for w in net.weights(bf16_rounded=True)]
    if residual:
        L, grads = convnet.residual_loss_and_grad(Ws, X, wilson.explicit(U, dims, -0.4),
                                                  wilson.explicit_dagger(U, dims, -0.4), dims, act)
    else:
        L, grads = convnet.loss_and_grad(Ws, X, E, dims, act)
    assert abs(loss - L) <= 1e-4 * abs(L)
    for l in range(4):
        assert np.abs(grad[l] - grads[l]).max() <= 1e-3 * np.abs(grads[l]).max(), l


@pytest.fixture(scope="module")
def trained(dtr):
    """4^4 with weak disorder (eps 0.2) and a small mass (m0 -0.15, ill
    conditioned): a translation-invariant network that sees no links can
    approximate the propagator here.  Trained on 16 x 8 independent
    (residual, error) pairs from the library's own solves, residual loss."""
    from paper_1603_05988_gb300 import learned
    dims, m0 = (4, 4, 4, 4), -0.15
    U = synth.random_su3_links(dims, 0.2, 1000)
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    net = dtr.Net(lat, act=0, init_scale=1.0 / (4.0 + m0), noise=1e-3, seed=1)
    hist = learned.train(net, g, m0, steps=200, batch=8, lr=3e-4, pool=16)
    return dict(dims=dims, m0=m0, U=U, lat=lat, g=g, net=net, hist=hist)


def test_training_lowers_loss(trained):
    h = trained["hist"]
    assert np.mean(h[-10:]) < 0.5 * np.mean(h[:5]), (h[:5], h[-10:])


@pytest.mark.parametrize("use_net", [False, True])
def test_fgmres_reaches_tolerance(dtr, trained, use_net):
    import torch
    t = trained
    Z = noise.noise_vectors(t["dims"], 77, 3, 16, False, 0, 8)
    p = dtr.solve_params(tol=1e-10, solver="fgmres_net", net=t["net"] if use_net else None, gmres_m=16)
    y, st = dtr.solve_batch(t["g"], t["m0"], torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p)
    Y = y.cpu().numpy().T
    A = wilson.explicit(t["U"], t["dims"], t["m0"])
    res = np.linalg.norm(Z - A @ Y, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.all(res <= 1e-10), res


def test_trained_network_cuts_arnoldi_steps(dtr, trained):
    """The gain test: FGMRES steps to 1e-10 with the trained network versus
    the unpreconditioned FGMRES on the same right-hand sides (held-out noise).
    A CPU run of the same training with scipy GMRES gave 141 vs 501 steps."""
    import torch
    t = trained
    Z = noise.noise_vectors(t["dims"], 78, 4, 16, False, 0, 16)
    z = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    its = {}
    for name, net in (("plain", None), ("learned", t["net"])):
        p = dtr.solve_params(tol=1e-10, solver="fgmres_net", net=net, gmres_m=16)
        y, st = dtr.solve_batch(t["g"], t["m0"], z, params=p)
        its[name] = np.mean([s["iterations"] for s in st])
    assert its["learned"] < 0.6 * its["plain"], its


def test_trace_through_fgmres_matches_oracle(dtr, trained):
    t = trained
    A = wilson.explicit(t["U"], t["dims"], t["m0"])
    AH = wilson.explicit_dagger(t["U"], t["dims"], t["m0"])
    Ad = A.toarray()
    tr, Ainv = exact.trace_inverse_lu(Ad)
    V, lam, sig = deflation.smallest_triplets(Ad, 16)
    D = dtr.defl_create(t["lat"], V, lam)
    p = dtr.trace_params(seed=5, n_z0=2, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-12, solver="fgmres_net", net=t["net"]))
    out = dtr.trace_estimate(t["g"], t["m0"], D, p)
    for r in range(2):
        Z = noise.noise_vectors(t["dims"], 5, r, 16, False, 0, 16)
        ref = estimator.deflated_hp(AH, lambda Z: Ainv @ Z, Z, V, sig)
        assert np.abs(out["samples"][r] - ref["t"]).max() <= 1e-8 * np.abs(ref["t"]).max()
        assert abs(out["trace_runs"][r] - ref["trace"][-1]) <= 1e-10 * abs(ref["trace"][-1])
