"""GPU checks of the learned preconditioner and the FGMRES solver.

* network forward and gradient through the C ABI against the oracle's plain
  numpy network (same BF16-rounded weights, inputs rounded to FP32), for the
  FP32 CUDA-core kernels at FP32 tolerances and for the tensor-core kernels
  (BF16 layer inputs and gradients) at tolerances derived from BF16 rounding,
  including one-layer cases that isolate a single convolution on ragged tiles;
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
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=3, precision="f32")
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
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=4, precision="f32")
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


def _bf16(x):
    return deflation.bf16_round(x)


def _one_layer_weights(rng, scale=0.1):
    """Layer 0 random (BF16-exact values), layers 1-3 the identity at the centre offset:
    the network's output is then layer 0's convolution, rounded to BF16 once per
    stored layer input (the identity layers copy BF16 values exactly)."""
    W = np.zeros((4, 81, 24, 24), dtype=np.float32)
    W[0] = rng.standard_normal((81, 24, 24)) * scale
    W[0] = deflation.bf16_round(W[0].astype(np.float64)).real.astype(np.float32)
    for l in range(1, 4):
        W[l, 40] = np.eye(24)
    return W


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("dims,nrhs", [((2, 2, 2, 4), 1), ((12, 20, 4, 10), 3), ((8, 16, 2, 6), 2)])
def test_tc_single_convolution_matches_oracle(dtr, act, dims, nrhs):
    """One tensor-core convolution on tiles of 8 x 16 sites with ragged x, y and t
    edges: y = round_bf16(W_0 * round_bf16(x)) (act 0), or the leaky ReLU applied
    three times to the rounded layer-0 output (act 1: every stored layer input is
    phi of the previous output, and phi scales negatives by 1/4 exactly).  The
    oracle evaluates W_0 on the same BF16-rounded input in FP64; the bound is half
    a BF16 ulp (2^-9 relative) of the stored output plus FP32 accumulation."""
    import torch
    lat = dtr.make_lattice(dims)
    rng = np.random.default_rng(11)
    net = dtr.Net(lat, act=act, weights=_one_layer_weights(rng))
    X = rng.standard_normal((lat.N, nrhs)) + 1j * rng.standard_normal((lat.N, nrhs))
    Xq = _bf16(X)
    y = net.apply(torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T
    W0 = net.weights(bf16_rounded=True)[0].astype(np.float64)
    h = convnet.conv(W0, convnet.to_real(Xq, dims))
    for _ in range(3 if act else 0):
        h = convnet.phi(h, act)
    ref = convnet.to_complex(h, dims)
    err = np.abs(y.real - ref.real) + np.abs(y.imag - ref.imag)
    bound = 2.0 ** -8 * (np.abs(ref.real) + np.abs(ref.imag)) + 1e-5 * np.abs(ref).max()
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("act", [0, 1])
def test_tc_network_forward_matches_oracle(dtr, act):
    """Four random layers on the tensor cores against the FP64 oracle: each of the
    four stored layer inputs is rounded to BF16 (2^-9 relative), so the output
    agrees to a few parts in 10^3 of its maximum."""
    import torch
    dims, nrhs = (8, 16, 2, 4), 2
    lat = dtr.make_lattice(dims)
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=3)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((lat.N, nrhs)) + 1j * rng.standard_normal((lat.N, nrhs))
    y = net.apply(torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T
    Ws = [w.astype(np.float64) for w in net.weights(bf16_rounded=True)]
    ref, _, _ = convnet.forward(Ws, X, dims, act)
    assert np.abs(y - ref).max() <= 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("act", [0, 1])
@pytest.mark.parametrize("residual", [False, True])
def test_tc_gradient_matches_oracle(dtr, act, residual):
    """Loss and weight gradients with BF16 layer inputs and BF16 back-propagated
    gradients (tensor-core forward, backward-data and weight-gradient convolutions)
    against the FP64 oracle.  Up to seven BF16 roundings (2^-9 relative each: four
    stored layer inputs, the loss gradient, two back-propagated gradients) reach a
    layer-0 gradient entry, a sum of ~2e3 products, so entries carry ~0.5% random
    relative error and the largest deviation among 46,656 entries a few times that:
    the bounds are 1.5e-2 in Frobenius norm and 4e-2 of the largest entry.  With the
    leaky ReLU the kernel decides phi'(h) from its own BF16-rounded h: where |h| is
    within the rounding error of zero (a few per mille of the entries) the kernel and
    the FP64 oracle take opposite branches and the gradient there differs by a factor
    of four, so the lower layers' gradients move by a few percent; the bounds for
    act = 1 are 6e-2 and 1.5e-1.  A wrong offset, transpose or a missing mask (half
    the entries off by 4x) gives errors of order one."""
    import torch
    dims = (8, 16, 2, 4)
    lat = dtr.make_lattice(dims)
    U = synth.random_su3_links(dims, 0.5, 21)
    g = dtr.gauge_from_host(lat, U)
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=4)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((lat.N, 2)) + 1j * rng.standard_normal((lat.N, 2))
    E = rng.standard_normal((lat.N, 2)) + 1j * rng.standard_normal((lat.N, 2))
    loss, grad = net.train_step(torch.from_numpy(np.ascontiguousarray(X.T)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(E.T)).cuda(), step=False, want_grad=True,
                                gauge=g if residual else None, m0=-0.4)
    Ws = [w.astype(np.float64) for w in net.weights(bf16_rounded=True)]
    if residual:
        L, grads = convnet.residual_loss_and_grad(Ws, X, wilson.explicit(U, dims, -0.4),
                                                  wilson.explicit_dagger(U, dims, -0.4), dims, act)
    else:
        L, grads = convnet.loss_and_grad(Ws, X, E, dims, act)
    assert abs(loss - L) <= 1e-2 * abs(L)
    fro, mx = (6e-2, 1.5e-1) if act else (1.5e-2, 4e-2)
    for l in (3, 2, 1, 0):  # the last layer's gradient needs no backward-data convolution
        d = grad[l] - grads[l]
        assert np.linalg.norm(d) <= fro * np.linalg.norm(grads[l]), (l, np.linalg.norm(d) / np.linalg.norm(grads[l]))
        assert np.abs(d).max() <= mx * np.abs(grads[l]).max(), (l, np.abs(d).max() / np.abs(grads[l]).max())


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_network_precision_switch(dtr, precision):
    """The two kernel sets compute the same network: outputs agree to BF16 accuracy."""
    import torch
    dims = (8, 16, 2, 4)
    lat = dtr.make_lattice(dims)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((lat.N, 2)) + 1j * rng.standard_normal((lat.N, 2))
    x = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    net = dtr.Net(lat, act=1, init_scale=0.5, noise=0.05, seed=3, precision=precision)
    y1 = net.apply(x).cpu().numpy()
    net.set_precision("f32" if precision == "bf16" else "bf16")
    y2 = net.apply(x).cpu().numpy()
    assert np.abs(y1 - y2).max() <= 1e-2 * np.abs(y2).max()
    with pytest.raises(dtr.DtrError):
        net.set_precision("f64")


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
