"""Philox4x64-10 counter-based generator (oracle; test infrastructure).

Written from the published definition of the Philox family (J. K. Salmon,
M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 4-word counter and 2-word key, ten rounds, each round a
pair of 64x64->128 bit multiplications whose high halves are xor-ed with the
other counter words and the round key, the key bumped by the Weyl constants
between rounds.  Vectorised over counters with numpy uint64; the 128-bit
product is formed from 32-bit halves.

The paper draws z0 with randi([0,3]) (Algorithm 1); a counter-based
generator makes that draw a pure function of (seed, z0 run, dof index) so the
CPU and GPU sides can each compute it from the definition.
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def mulhilo64(a, b):
    """Return (hi, lo) of the 128-bit product a*b for uint64 arrays."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & _M32, a >> _S32
    b0, b1 = b & _M32, b >> _S32
    with np.errstate(over="ignore"):
        p00 = a0 * b0
        p01 = a0 * b1
        p10 = a1 * b0
        p11 = a1 * b1
        mid = (p00 >> _S32) + (p01 & _M32) + (p10 & _M32)
        hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
        lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """ctr: (..., 4) uint64, key: (..., 2) uint64 -> (..., 4) uint64."""
    ctr = np.array(ctr, dtype=np.uint64, copy=True)
    key = np.array(key, dtype=np.uint64, copy=True)
    c0, c1, c2, c3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0, k1 = np.broadcast_to(key[..., 0], c0.shape).copy(), np.broadcast_to(key[..., 1], c0.shape).copy()
    for r in range(10):
        if r > 0:
            with np.errstate(over="ignore"):
                k0 = k0 + W0
                k1 = k1 + W1
        hi0, lo0 = mulhilo64(M0, c0)
        hi1, lo1 = mulhilo64(M1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)
