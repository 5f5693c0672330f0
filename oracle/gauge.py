"""Counter-based random SU(3) gauge field (oracle; test infrastructure).

The paper's gauge ensembles (Section 6) are not available; a seeded random
field stands in.  The links follow the workload definition U = exp(i eps H),
H a Gaussian Hermitian traceless 3 x 3 matrix, drawn as a pure function of
(seed, site, mu) so that a CPU and a GPU implementation can each compute the
same field from this definition:

  * Philox4x64-10 (Salmon et al., SC'11) with key (seed, 1) and counter
    (site, mu, c, 0) for c = 0..4; each 64-bit output word w gives the
    uniform u = ((w >> 11) + 1/2) 2^-53 in (0, 1).
  * Box-Muller on the word pairs (0, 1) and (2, 3) of each counter:
    r = sqrt(-2 ln u_even), normals (r cos 2 pi u_odd, r sin 2 pi u_odd), so
    counter c yields normals n_4c .. n_4c+3; n_0 .. n_17 are used.
  * G_ab = n_2(3a+b) + i n_2(3a+b)+1; H = (G + G^H)/2 - (Tr H / 3) 1.
  * U = exp(i eps H), here through the Hermitian eigendecomposition
    H = W diag(w) W^H: U = W diag(exp(i eps w)) W^H (a different route from a
    power series, so agreement with another implementation is a real check).

Layout: U[site, mu, a, b], site = x + Lx (y + Ly (z + Lz t)).
"""
import numpy as np

from . import philox as _philox


def normals(seed, sites, mu):
    """(len(sites), 20) standard normals of the links (sites[i], mu[i])."""
    sites = np.asarray(sites, dtype=np.uint64)
    mu = np.asarray(mu, dtype=np.uint64)
    n = sites.shape[0]
    out = np.empty((n, 20))
    key = np.array([seed, 1], dtype=np.uint64)
    for c in range(5):
        ctr = np.zeros((n, 4), dtype=np.uint64)
        ctr[:, 0] = sites
        ctr[:, 1] = mu
        ctr[:, 2] = np.uint64(c)
        w = _philox.philox4x64_10(ctr, key)
        u = ((w >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        for p in range(2):
            r = np.sqrt(-2.0 * np.log(u[:, 2 * p]))
            th = 2.0 * np.pi * u[:, 2 * p + 1]
            out[:, 4 * c + 2 * p] = r * np.cos(th)
            out[:, 4 * c + 2 * p + 1] = r * np.sin(th)
    return out


def hermitian_generators(seed, sites, mu):
    """H (n, 3, 3): the traceless Hermitian matrices of the listed links."""
    g = normals(seed, sites, mu)[:, :18]
    G = (g[:, 0::2] + 1j * g[:, 1::2]).reshape(-1, 3, 3)
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real
    return H - (tr / 3.0)[:, None, None] * np.eye(3)


def links_at(seed, eps, sites, mu):
    """U_mu(x) = exp(i eps H) (n, 3, 3) for the listed (site, mu) pairs."""
    H = hermitian_generators(seed, sites, mu)
    w, W = np.linalg.eigh(H)
    return np.einsum("nab,nb,ncb->nac", W, np.exp(1j * eps * w), np.conj(W))


def random_su3_links(dims, eps, seed):
    """The whole field, (V, 4, 3, 3) complex128."""
    V = int(np.prod(dims))
    sites = np.repeat(np.arange(V), 4)
    mu = np.tile(np.arange(4), V)
    return links_at(seed, eps, sites, mu).reshape(V, 4, 3, 3)
