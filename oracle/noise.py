"""Z4 noise, hierarchical-probing colourings and Hadamard vectors (oracle).

Section 1 (Z4 vectors: entries uniform in {+1, -1, +i, -i}); Section 5.2 and
Algorithm 1 (z0 = exp(i*pi*randi([0,3])/2), z = z0 .* z_h with z_h
the next hierarchical-probing vector, a permuted Hadamard vector over a
nested distance-2^l colouring of the lattice).

Readings (the paper defers the HP construction to its reference [HP 2013]):
  * z0 code of dof i in run r: Philox4x64-10 with key (seed, 0) and counter
    (i // 128, r, 0, 0); the 256 output bits hold 2-bit codes of 128
    consecutive dofs, word w = (i % 128) // 32, bit offset 2*(i % 32).
    Code q means z0(i) = i^q, i.e. 1, i, -1, -i for q = 0, 1, 2, 3.
  * Colouring, nested by construction: colour bit 0 = parity of x+y+z+t
    (2 colours, red-black); then for l = 0, 1, ...: append bits
    ((y>>l)&1, (z>>l)&1, (t>>l)&1) (x 8 colours), then append the parity of
    sum_mu (x_mu >> (l+1)) (x 2 colours).  Colour counts 2, 16, 32, 256, 512,
    4096, 8192, ...  Each colour is the coarser colour plus higher bits, so
    colour mod c_coarse is the coarser colouring.
  * Hadamard (Sylvester, natural order): H[c, j] = (-1)^popcount(c & j).
    For j < c_coarse it depends on c mod c_coarse only, so the first c_coarse
    vectors of a finer level are exactly the coarser level's vectors: the
    nesting Section 1 requires.
  * Optional 12-fold spin-colour dilution multiplies by delta(a, i mod 12);
    right-hand side q then maps to (Hadamard column j, dof type a) =
    (q // 12, q % 12).
"""
import numpy as np

from . import lattice as _lat
from . import philox as _philox

Z4_VALUES = np.array([1.0, 1.0j, -1.0, -1.0j], dtype=np.complex128)


def z0_codes(seed, run, N):
    """2-bit Z4 codes (uint8, values 0..3) of z0 for run `run`, dofs 0..N-1."""
    nblk = (N + 127) // 128
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    ctr[:, 1] = np.uint64(run)
    key = np.array([seed, 0], dtype=np.uint64)
    words = _philox.philox4x64_10(ctr, key)  # (nblk, 4)
    i = np.arange(N)
    blk = i // 128
    w = (i % 128) // 32
    sh = (2 * (i % 32)).astype(np.uint64)
    return ((words[blk, w] >> sh) & np.uint64(3)).astype(np.uint8)


def z0_codes_at(seed, run, idx):
    """z0 codes at the listed dof indices only (the same counter-based stream as
    z0_codes, evaluating just the 128-dof blocks that hold them): for fields too
    large to draw whole."""
    idx = np.asarray(idx, dtype=np.int64)
    blocks, inv = np.unique(idx // 128, return_inverse=True)
    ctr = np.zeros((len(blocks), 4), dtype=np.uint64)
    ctr[:, 0] = blocks.astype(np.uint64)
    ctr[:, 1] = np.uint64(run)
    key = np.array([seed, 0], dtype=np.uint64)
    words = _philox.philox4x64_10(ctr, key)
    w = (idx % 128) // 32
    sh = (2 * (idx % 32)).astype(np.uint64)
    return ((words[inv, w] >> sh) & np.uint64(3)).astype(np.uint8)


def z0_vector(seed, run, N):
    """z0 = exp(i*pi*q/2) written exactly as 1, i, -1, -i (the draw of z0 in Algorithm 1)."""
    return Z4_VALUES[z0_codes(seed, run, N)]


def valid_ncolors(ncolors):
    n = 1
    seq = [1]
    if ncolors == 1:
        return True
    n = 2
    seq.append(n)
    while n < ncolors:
        n *= 8
        seq.append(n)
        if n >= ncolors:
            break
        n *= 2
        seq.append(n)
    return ncolors in seq


def colour_period(ncolors):
    """Period (in lattice units, every direction) of the colouring pattern.

    Periodic lattices whose extents are not multiples of this would break the
    distance property across the boundary, so callers reject them.
    """
    if not valid_ncolors(ncolors):
        raise ValueError("ncolors must be 1, 2, 16, 32, 256, 512, ...")
    if ncolors == 1:
        return 1
    n, period, level = 2, 2, 0
    while n < ncolors:
        n *= 8
        period = max(period, 2 ** (level + 1))
        if n >= ncolors:
            break
        n *= 2
        period = 2 ** (level + 2)
        level += 1
    return period


def hp_colour(dims, ncolors):
    """Colour of each site (int64 array of length V) for `ncolors` colours."""
    if not valid_ncolors(ncolors):
        raise ValueError("ncolors must be 1, 2, 16, 32, 256, 512, ...")
    c = _lat.coords(dims)
    x, y, z, t = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    V = len(x)
    if ncolors == 1:
        return np.zeros(V, dtype=np.int64)
    col = (x + y + z + t) % 2
    n = 2
    level = 0
    while n < ncolors:
        col = col + n * (((y >> level) & 1) + 2 * ((z >> level) & 1) + 4 * ((t >> level) & 1))
        n *= 8
        if n >= ncolors:
            break
        col = col + n * (((x >> (level + 1)) + (y >> (level + 1)) + (z >> (level + 1)) + (t >> (level + 1))) % 2)
        n *= 2
        level += 1
    return col


def hadamard_entry(c, j):
    """Sylvester Hadamard entry H[c, j] = (-1)^popcount(c & j) (integer arrays)."""
    v = np.bitwise_and(np.asarray(c, dtype=np.int64), np.asarray(j, dtype=np.int64))
    pc = np.zeros_like(v)
    while np.any(v):
        pc += v & 1
        v = v >> 1
    return 1 - 2 * (pc % 2)


def noise_vectors(dims, seed, run, ncolors, dilute12, q0, nrhs):
    """Columns q0..q0+nrhs-1 of the probing sequence for z0 run `run`.

    Returns an (N, nrhs) complex128 array with entries in {0, +-1, +-i}:
      z_q(i) = z0_run(i) * H[colour(site(i)), j] * [a == i mod 12 if dilute12]
    with (j, a) = (q // 12, q % 12) when diluted, else j = q.
    """
    V = _lat.volume(dims)
    N = 12 * V
    z0 = z0_vector(seed, run, N)
    col = np.repeat(hp_colour(dims, ncolors), 12)  # colour of each dof's site
    out = np.zeros((N, nrhs), dtype=np.complex128)
    dof_type = np.arange(N) % 12
    for k in range(nrhs):
        q = q0 + k
        j = q // 12 if dilute12 else q
        h = hadamard_entry(col, j)
        z = z0 * h
        if dilute12:
            z = np.where(dof_type == (q % 12), z, 0.0)
        out[:, k] = z
    return out
