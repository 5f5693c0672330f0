"""Pins of the oracle's 4D convolutional network: finite differences for the
weight gradient, the adjoint identity for the transposed stencil, and the
identity network."""
import numpy as np
import pytest

from oracle import convnet


def _rand_weights(seed, scale=0.05):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((81, 24, 24)) * scale for _ in range(4)]


def test_adjoint_identity():
    dims = (2, 2, 2, 4)
    rng = np.random.default_rng(0)
    W = rng.standard_normal((81, 24, 24))
    a = rng.standard_normal((2, 4, 2, 2, 2, 24))
    g = rng.standard_normal((2, 4, 2, 2, 2, 24))
    lhs = np.sum(convnet.conv(W, a) * g)
    rhs = np.sum(a * convnet.conv_transpose(W, g))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_identity_network_scales_input():
    dims = (2, 2, 2, 2)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(12 * 16) + 1j * rng.standard_normal(12 * 16)
    y, _, _ = convnet.forward(convnet.identity_weights(0.3), x, dims, act=0)
    assert np.allclose(y, 0.3 * x)
    # leaky activation: positive homogeneity M(a x) = a M(x), a > 0
    Ws = _rand_weights(2)
    y1, _, _ = convnet.forward(Ws, x, dims, act=1)
    y2, _, _ = convnet.forward(Ws, 2.5 * x, dims, act=1)
    assert np.allclose(y2, 2.5 * y1)


def test_conv_single_offset_is_a_shift():
    """A weight only at offset o moves the field by d(o): out(s) = in(s + d(o))."""
    dims = (4, 2, 2, 2)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((1, 2, 2, 2, 4, 24))
    o = 1 + 3 * 1 + 9 * 1 + 27 * 1 + 1  # dx = +1, others 0
    W = np.zeros((81, 24, 24))
    W[o] = np.eye(24)
    out = convnet.conv(W, a)
    assert np.allclose(out[..., 0, :], a[..., 1, :]) and np.allclose(out[..., 3, :], a[..., 0, :])


@pytest.mark.parametrize("act", [0, 1])
def test_weight_gradient_by_finite_differences(act):
    dims = (2, 2, 2, 2)
    rng = np.random.default_rng(4 + act)
    N = 12 * 16
    x = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    e = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    Ws = _rand_weights(7, 0.2)
    L, grads = convnet.loss_and_grad(Ws, x, e, dims, act)
    h = 1e-6
    for l, (o, co, ci) in [(0, (40, 3, 5)), (1, (0, 7, 2)), (2, (80, 23, 0)), (3, (13, 1, 1)), (3, (40, 10, 11))]:
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[l][o, co, ci] += h
        Wm[l][o, co, ci] -= h
        Lp, _ = convnet.loss_and_grad(Wp, x, e, dims, act)
        Lm, _ = convnet.loss_and_grad(Wm, x, e, dims, act)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grads[l][o, co, ci]) < 1e-6 * max(1.0, abs(fd)), (l, o, co, ci, fd, grads[l][o, co, ci])


def test_residual_loss_gradient_by_finite_differences():
    from oracle import wilson
    from paper_1603_05988_gb300 import synth
    dims = (2, 2, 2, 2)
    U = synth.random_su3_links(dims, 0.5, 3)
    A = wilson.explicit(U, dims, -0.4)
    AH = wilson.explicit_dagger(U, dims, -0.4)
    rng = np.random.default_rng(8)
    N = 12 * 16
    x = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    Ws = _rand_weights(9, 0.2)
    L, grads = convnet.residual_loss_and_grad(Ws, x, A, AH, dims, 1)
    h = 1e-6
    for l, (o, co, ci) in [(0, (40, 2, 9)), (2, (5, 11, 3)), (3, (77, 0, 23))]:
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[l][o, co, ci] += h
        Wm[l][o, co, ci] -= h
        fd = (convnet.residual_loss_and_grad(Wp, x, A, AH, dims, 1)[0]
              - convnet.residual_loss_and_grad(Wm, x, A, AH, dims, 1)[0]) / (2 * h)
        assert abs(fd - grads[l][o, co, ci]) < 1e-6 * max(1.0, abs(fd))
