"""Wilson-Dirac matrix A (oracle; test infrastructure).

Operator (the workload definition for the paper's Dirac matrix, Section 6:
N = 12 V, a nearest-neighbour operator on a periodic 4D lattice):

  (A psi)(x) = (4 + m0) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
                            + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]

Links U has shape (V, 4, 3, 3): U[site, mu, a, b] is row a, column b of
U_mu(site).  Two independent codings are given -- an explicit sparse matrix
assembled from Kronecker blocks and a matrix-free apply built on array rolls
-- so that each checks the other.  A^H is taken literally as the conjugate
transpose of the explicit matrix (the paper's Algorithm 1 applies A^H; no
gamma5 identity is used here).
"""
import numpy as np
import scipy.sparse as sp

from . import gamma as _gamma
from . import lattice as _lat


def explicit(U, dims, m0):
    """Sparse CSR matrix A (N x N, complex128) assembled block by block.

    Block (x, y) is kron(S, C) with S the 4x4 spin matrix and C the 3x3
    colour matrix, because dof index = 3*spin + colour within a site.
    Duplicate (x, y) pairs (extent-2 directions) are summed by the COO->CSR
    conversion, as the operator definition requires.
    """
    V = _lat.volume(dims)
    N = 12 * V
    g = _gamma.gammas()
    eye4 = np.eye(4, dtype=np.complex128)
    rows, cols, vals = [], [], []
    site = np.arange(V)
    base_r = (12 * site)[:, None, None] + np.arange(12)[None, :, None]
    for mu in range(4):
        fwd = _lat.neighbour(dims, mu, +1)
        bwd = _lat.neighbour(dims, mu, -1)
        # forward hop: -1/2 (1 - gamma_mu) (x) U_mu(x), column block x+mu
        S = eye4 - g[mu]
        blk = -0.5 * np.einsum("ab,xcd->xacbd", S, U[:, mu]).reshape(V, 12, 12)
        r = np.broadcast_to(base_r, (V, 12, 12))
        c = (12 * fwd)[:, None, None] + np.arange(12)[None, None, :]
        rows.append(r.ravel()); cols.append(np.broadcast_to(c, (V, 12, 12)).ravel()); vals.append(blk.ravel())
        # backward hop: -1/2 (1 + gamma_mu) (x) U_mu(x-mu)^H, column block x-mu
        S = eye4 + g[mu]
        Ub = np.conj(np.transpose(U[bwd, mu], (0, 2, 1)))
        blk = -0.5 * np.einsum("ab,xcd->xacbd", S, Ub).reshape(V, 12, 12)
        c = (12 * bwd)[:, None, None] + np.arange(12)[None, None, :]
        rows.append(r.ravel()); cols.append(np.broadcast_to(c, (V, 12, 12)).ravel()); vals.append(blk.ravel())
    diag = np.arange(N)
    rows.append(diag); cols.append(diag); vals.append(np.full(N, 4.0 + m0, dtype=np.complex128))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()


def explicit_dagger(U, dims, m0):
    """A^H as the literal conjugate transpose of the explicit matrix."""
    return explicit(U, dims, m0).conj().T.tocsr()


def apply(U, dims, m0, psi):
    """Matrix-free A psi for psi of shape (N,) or (N, nrhs).

    Coded independently of `explicit`: the field is reshaped to
    (Lt, Lz, Ly, Lx, 4, 3[, nrhs]) and neighbours are taken with np.roll.
    """
    lx, ly, lz, lt = dims
    single = psi.ndim == 1
    P = psi.reshape(12 * _lat.volume(dims), -1)
    nr = P.shape[1]
    f = P.reshape(lt, lz, ly, lx, 4, 3, nr)
    Ul = U.reshape(lt, lz, ly, lx, 4, 3, 3)
    axis_of_mu = {0: 3, 1: 2, 2: 1, 3: 0}
    g = _gamma.gammas()
    eye4 = np.eye(4, dtype=np.complex128)
    out = (4.0 + m0) * f
    for mu in range(4):
        ax = axis_of_mu[mu]
        Umu = Ul[:, :, :, :, mu]
        # psi(x + mu): roll by -1 brings site x+mu to position x
        fp = np.roll(f, -1, axis=ax)
        hop = np.einsum("tzyxab,tzyxsbr->tzyxsar", Umu, fp)
        out = out - 0.5 * np.einsum("st,TZYXtar->TZYXsar", eye4 - g[mu], hop)
        # psi(x - mu) and U_mu(x - mu)^H
        fm = np.roll(f, +1, axis=ax)
        Um = np.roll(Umu, +1, axis=ax)
        hop = np.einsum("tzyxba,tzyxsbr->tzyxsar", np.conj(Um), fm)
        out = out - 0.5 * np.einsum("st,TZYXtar->TZYXsar", eye4 + g[mu], hop)
    out = out.reshape(P.shape)
    return out[:, 0] if single else out


def gamma5_vec(psi):
    """gamma_5 applied to a spinor field (N,) or (N, nrhs), via the 4x4 matrix."""
    single = psi.ndim == 1
    P = psi.reshape(-1, 4, 3, psi.shape[1] if not single else 1)
    out = np.einsum("st,vtcr->vscr", _gamma.gamma5(), P).reshape(-1, P.shape[-1])
    return out[:, 0] if single else out


def dense(U, dims, m0):
    """Dense A (small lattices only)."""
    return explicit(U, dims, m0).toarray()


def apply_at(U, dims, m0, psi, sites):
    """(A psi) at the listed sites only, written from the operator's definition one
    direction at a time (a third coding, for lattices too large for the whole-field
    forms): returns (len(sites), 12[, nrhs]) with rows 3 spin + colour."""
    single = psi.ndim == 1
    P = psi.reshape(12 * _lat.volume(dims), -1)
    nr = P.shape[1]
    sites = np.asarray(sites, dtype=np.int64)
    c = _lat.coords(dims)[sites]                      # (S, 4) as (x, y, z, t)
    g = _gamma.gammas()
    eye4 = np.eye(4, dtype=np.complex128)

    def spinor(s):                                    # (S, 4, 3, nr)
        idx = (12 * s[:, None] + np.arange(12)[None, :])
        return P[idx].reshape(len(s), 4, 3, nr)

    out = (4.0 + m0) * spinor(sites)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        cb = c.copy()
        cb[:, mu] = (cb[:, mu] - 1) % dims[mu]
        sf = _lat.site_index(cf, dims)
        sb = _lat.site_index(cb, dims)
        Uf = U[sites, mu]                             # U_mu(x)
        Ub = U[sb, mu]                                # U_mu(x - mu)
        hop_f = np.einsum("kab,ksbr->ksar", Uf, spinor(sf))
        hop_b = np.einsum("kba,ksbr->ksar", np.conj(Ub), spinor(sb))
        out = out - 0.5 * np.einsum("st,ktar->ksar", eye4 - g[mu], hop_f)
        out = out - 0.5 * np.einsum("st,ktar->ksar", eye4 + g[mu], hop_b)
    out = out.reshape(len(sites), 12, nr)
    return out[:, :, 0] if single else out
