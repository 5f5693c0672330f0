"""4D convolutional network of the learned preconditioner (oracle; test infrastructure).

The paper does not name its linear solver (the solve step of Algorithm 1); the library
adds an FGMRES solver right-preconditioned by a small network M ~ A^-1.  This
module is the plain reference of that network, used to check the CUDA
forward and backward kernels:

  * a field's 12 complex dofs per site are 24 real channels, channel 2c + p =
    real (p = 0) / imaginary (p = 1) part of dof c = 3*spin + colour;
  * layer l: out(s, co) = sum_o sum_ci W_l[o, co, ci] * in(s + d(o), ci), with
    d(o) = (dx-1, dy-1, dz-1, dt-1) for o = ((dt*3 + dz)*3 + dy)*3 + dx, periodic;
  * y = W_3 * phi(W_2 * phi(W_1 * phi(W_0 * x))), phi = identity (act 0) or
    leaky ReLU with slope 1/4 (act 1);
  * loss over columns j: L = sum_j |y_j - e_j|^2 / |e_j|^2.

Backward is written out by the chain rule (transposed, reflected stencil for
the input gradient; site sums of products for the weight gradient) and pinned
by finite differences in the tests.
"""
import numpy as np

NOFF = 81
NCH = 24


def displacement(o):
    d = []
    for _ in range(4):
        d.append(o % 3 - 1)
        o //= 3
    return d  # (dx, dy, dz, dt)


def to_real(x, dims):
    """(N,) or (N, nrhs) complex -> (nrhs, Lt, Lz, Ly, Lx, 24) real."""
    X = x if x.ndim == 2 else x[:, None]
    nr = X.shape[1]
    lx, ly, lz, lt = dims
    C = X.T.reshape(nr, lt, lz, ly, lx, 12)
    out = np.empty(C.shape[:-1] + (24,))
    out[..., 0::2] = C.real
    out[..., 1::2] = C.imag
    return out


def to_complex(R, dims):
    nr = R.shape[0]
    C = R[..., 0::2] + 1j * R[..., 1::2]
    return C.reshape(nr, -1).T


def _shift(a, d):
    """a(s + d) for a of shape (nrhs, Lt, Lz, Ly, Lx, ch)."""
    dx, dy, dz, dt = d
    out = a
    for shift, ax in ((dx, 4), (dy, 3), (dz, 2), (dt, 1)):
        if shift:
            out = np.roll(out, -shift, axis=ax)
    return out


def conv(W, a):
    """out(s, co) = sum_o sum_ci W[o, co, ci] a(s + d(o), ci)."""
    out = np.zeros(a.shape[:-1] + (W.shape[1],))
    for o in range(NOFF):
        out += _shift(a, displacement(o)) @ W[o].T
    return out


def conv_transpose(W, g):
    """Adjoint of conv: out(t, ci) = sum_o sum_co W[o, co, ci] g(t - d(o), co)."""
    out = np.zeros(g.shape[:-1] + (W.shape[2],))
    for o in range(NOFF):
        d = [-v for v in displacement(o)]
        out += _shift(g, d) @ W[o]
    return out


def phi(u, act):
    return np.where(u < 0, 0.25 * u, u) if act else u


def dphi(u, act):
    return np.where(u < 0, 0.25, 1.0) if act else np.ones_like(u)


def forward(Ws, x, dims, act):
    """Return y (complex, same shape as x) and the pre-activations."""
    a = to_real(x, dims)
    hs = [a]
    h = conv(Ws[0], a)
    for l in range(1, len(Ws)):
        hs.append(h)
        h = conv(Ws[l], phi(h, act))
    y = to_complex(h, dims)
    return (y if x.ndim == 2 else y[:, 0]), hs, h


def loss_and_grad(Ws, x, e, dims, act):
    """L = sum_j |y_j - e_j|^2 / |e_j|^2 and dL/dW_l (list of (81, 24, 24))."""
    y, hs, hout = forward(Ws, x, dims, act)
    E = to_real(e, dims)
    nr = E.shape[0]
    e2 = np.array([np.sum(E[j] ** 2) for j in range(nr)])
    diff = hout - E
    L = float(sum(np.sum(diff[j] ** 2) / e2[j] for j in range(nr)))
    g = np.stack([2.0 * diff[j] / e2[j] for j in range(nr)])
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        inp = hs[l] if l == 0 else phi(hs[l], act)
        gW = np.zeros_like(Ws[l])
        for o in range(NOFF):
            sh = _shift(inp, displacement(o))
            gW[o] = g.reshape(-1, g.shape[-1]).T @ sh.reshape(-1, sh.shape[-1])
        grads[l] = gW
        if l > 0:
            g = conv_transpose(Ws[l], g) * dphi(hs[l], act)
    return L, grads


def residual_loss_and_grad(Ws, x, A, AH, dims, act):
    """Residual-weighted loss of right preconditioning, L = sum_j |A y_j - x_j|^2 / |x_j|^2
    with y = M x, and dL/dW (dL/dy = 2 A^H (A y - x) / |x|^2, then the same backward)."""
    y, hs, hout = forward(Ws, x, dims, act)
    X = x if x.ndim == 2 else x[:, None]
    Y = y if y.ndim == 2 else y[:, None]
    q = A @ Y - X
    nx = np.sum(np.abs(X) ** 2, axis=0)
    L = float(np.sum(np.sum(np.abs(q) ** 2, axis=0) / nx))
    g = to_real(AH @ (2.0 * q / nx), dims)
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        inp = hs[l] if l == 0 else phi(hs[l], act)
        gW = np.zeros_like(Ws[l])
        for o in range(NOFF):
            sh = _shift(inp, displacement(o))
            gW[o] = g.reshape(-1, g.shape[-1]).T @ sh.reshape(-1, sh.shape[-1])
        grads[l] = gW
        if l > 0:
            g = conv_transpose(Ws[l], g) * dphi(hs[l], act)
    return L, grads


def identity_weights(scale0=1.0, L=4):
    Ws = []
    for l in range(L):
        W = np.zeros((NOFF, NCH, NCH))
        W[40] = np.eye(NCH) * (scale0 if l == 0 else 1.0)
        Ws.append(W)
    return Ws
