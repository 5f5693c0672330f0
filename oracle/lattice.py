"""4D periodic lattice indexing (oracle; test infrastructure).

Conventions (shared with the library's C ABI as a documented layout, not as
code):
  site  = x + Lx*(y + Ly*(z + Lz*t))           (x fastest)
  dof i = 12*site + 3*spin + colour             (Section 1: 12 dof per site)
  mu    = 0, 1, 2, 3  <->  x, y, z, t
"""
import numpy as np


def volume(dims):
    return int(np.prod(dims))


def coords(dims):
    """(V, 4) int64 array of (x, y, z, t) for every site in site order."""
    lx, ly, lz, lt = dims
    s = np.arange(volume(dims), dtype=np.int64)
    x = s % lx
    y = (s // lx) % ly
    z = (s // (lx * ly)) % lz
    t = s // (lx * ly * lz)
    return np.stack([x, y, z, t], axis=1)


def site_index(c, dims):
    """Inverse of coords: periodic wrap applied."""
    lx, ly, lz, lt = dims
    x = c[..., 0] % lx
    y = c[..., 1] % ly
    z = c[..., 2] % lz
    t = c[..., 3] % lt
    return x + lx * (y + ly * (z + lz * t))


def neighbour(dims, mu, step):
    """Site index of x + step*mu_hat for every site x (periodic)."""
    c = coords(dims).copy()
    c[:, mu] += step
    return site_index(c, dims)


def manhattan(dims, s1, s2):
    """Periodic Manhattan (taxicab) distance between site arrays s1 and s2."""
    c1 = coords(dims)[s1]
    c2 = coords(dims)[s2]
    d = np.abs(c1 - c2)
    L = np.asarray(dims)
    d = np.minimum(d, L - d)
    return d.sum(axis=-1)
