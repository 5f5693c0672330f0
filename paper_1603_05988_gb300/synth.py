"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This module holds none of the estimator's arithmetic: it only draws the
inputs the method consumes.  The paper's two 32^3x64 clover-Wilson gauge
ensembles (Section 6) are not available, so random SU(3) gauge fields stand
in for them:

    G_ab = g1 + i g2,  g1, g2 ~ N(0, 1) i.i.d.   (numpy Generator, Philox bit
                                                   generator keyed by the seed)
    H    = (G + G^H)/2 - Tr(.)/3 I                (Hermitian, traceless)
    U    = W diag(exp(i eps w)) W^H               (H = W diag(w) W^H)

so U = exp(i eps H) is exactly unitary with det U = exp(i eps Tr H) = 1 up to
rounding.  Layout: U[site, mu, a, b], site = x + Lx*(y + Ly*(z + Lz*t)).

Named workloads (lattice, eps, m0, noise, deflation) follow the five workload
configurations of the estimator: 4^4, 8^4, 16^3x32 and 32^3x64 (the fifth, the
learned preconditioner, reuses the 16^3x32 one).
"""
from dataclasses import dataclass, field

import numpy as np


def random_su3_links(dims, eps, seed):
    """(V, 4, 3, 3) complex128 links U = exp(i eps H) with H Gaussian Hermitian traceless."""
    V = int(np.prod(dims))
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    g = rng.standard_normal((V, 4, 3, 3, 2))
    G = g[..., 0] + 1j * g[..., 1]
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real
    H = H - (tr / 3.0)[..., None, None] * np.eye(3)
    w, W = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("...ab,...b,...cb->...ac", W, ph, np.conj(W))
    return np.ascontiguousarray(U)


def unit_links(dims):
    """Free field: every link the 3x3 identity."""
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def random_orthonormal(N, k, seed):
    """N x k complex matrix with orthonormal columns (QR of a Gaussian matrix)."""
    rng = np.random.Generator(np.random.Philox(key=int(seed) + 77))
    X = rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k))
    Q, _ = np.linalg.qr(X)
    return Q


def disjoint_orthonormal(N, k, seed, support=256):
    """N x k complex matrix with exactly orthonormal columns that is cheap at any N:
    column m is supported on its own random set of `support` dofs with Z4 phases,
    scaled by 1/sqrt(support).  Stands in for a deflation space where only the
    projection arithmetic is under test (the estimator is unbiased for any V)."""
    if k * support > N:
        raise ValueError("k * support must not exceed N")
    rng = np.random.Generator(np.random.Philox(key=int(seed) + 91))
    idx = rng.choice(N, size=k * support, replace=False).reshape(k, support)
    ph = np.array([1, 1j, -1, -1j])[rng.integers(0, 4, size=(k, support))]
    V = np.zeros((N, k), dtype=np.complex128)
    for m in range(k):
        V[idx[m], m] = ph[m] / np.sqrt(support)
    return V


@dataclass
class Workload:
    name: str
    dims: tuple
    eps: float
    m0: float
    n_z0: int            # number of z0 runs (independent Z4 vectors)
    ncolors: int         # hierarchical-probing colours per z0 (1 = plain MC)
    block: int           # right-hand sides per launch
    k: int               # deflation vectors
    defl_prec: str       # storage precision of V
    tol: float = 1e-10
    gauge_seed: int = 1000
    noise_seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def V(self):
        return int(np.prod(self.dims))

    @property
    def N(self):
        return 12 * self.V

    @property
    def nrhs_total(self):
        return self.n_z0 * self.ncolors


WORKLOADS = {
    # 4^4, m0=-0.4, eps=0.5, 64 Z4 vectors (plain MC), k=32 from dense SVD
    "wilson4x4x4x4_mc64_k32": Workload("wilson4x4x4x4_mc64_k32", (4, 4, 4, 4), 0.5, -0.4,
                                       n_z0=64, ncolors=1, block=64, k=32, defl_prec="f64",
                                       gauge_seed=1000),
    # 8^4, eps=0.7, m0=-0.6, 256 z0 x 16-colour HP, blocks of 16 RHS, k=100 FP64
    "wilson8x8x8x8_hp16x256_k100": Workload("wilson8x8x8x8_hp16x256_k100", (8, 8, 8, 8), 0.7, -0.6,
                                            n_z0=256, ncolors=16, block=16, k=100, defl_prec="f64",
                                            gauge_seed=1001),
    # 16^3x32, eps=0.8, m0=-0.75, 512 HP x 4 z0, blocks of 32, k=200 FP32
    "wilson16x16x16x32_hp512x4_k200": Workload("wilson16x16x16x32_hp512x4_k200", (16, 16, 16, 32), 0.8, -0.75,
                                               n_z0=4, ncolors=512, block=32, k=200, defl_prec="f32",
                                               gauge_seed=1002),
    # 32^3x64, eps=0.8, m0=-0.78, 512 HP x 8 z0, k=1000 BF16
    "wilson32x32x32x64_hp512x8_k1000": Workload("wilson32x32x32x64_hp512x8_k1000", (32, 32, 32, 64), 0.8, -0.78,
                                                n_z0=8, ncolors=512, block=32, k=1000, defl_prec="bf16",
                                                gauge_seed=1003),
}
