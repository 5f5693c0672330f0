"""Dirac gamma matrices in the chiral basis (oracle; test infrastructure).

The paper (Section 1, the Dirac operator as a 4D differential operator with 4
spin x 3 colour degrees of freedom per site) fixes no gamma basis.  Reading
taken here, as in the Wilson-Dirac operator definition used for the
workloads: the chiral basis

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   k = 1, 2, 3  (mu = x, y, z)
    gamma_4 = [[0, I], [I, 0]]                                (mu = t)
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)

Spin index 0..3 is the row/column index of these 4x4 matrices.  The exact
trace is basis independent; single samples z^H A^-1 z are not, so the CUDA
library must use the same basis (it does, independently coded).
"""
import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


def gammas():
    """Return [gamma_x, gamma_y, gamma_z, gamma_t] as 4x4 complex128 arrays."""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = [_block(z, -1j * s, 1j * s, z) for s in SIGMA]
    g.append(_block(z, one, one, z))
    return g


def gamma5():
    """gamma_5 as the product gamma_1 gamma_2 gamma_3 gamma_4 (not hard-coded)."""
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]
