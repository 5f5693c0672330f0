"""Pins of the oracle's noise, colouring and Hadamard generators."""
import numpy as np
import pytest

from oracle import lattice, noise, philox


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((123456789, 987), (2**64 - 1, 5, 7, 9)),      # carry out of counter word 0
    ((2**64 - 1, 2**63), (17, 2**64 - 1, 3, 0)),
    ((42, 0), (1000, 3, 0, 0)),
])
def test_philox_matches_numpy_bit_generator(key, ctr):
    """numpy's Philox bit generator is Philox4x64-10; it increments the
    counter before each block, so its first block is our counter + 1."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(8)
    c = list(ctr)
    outs = []
    for _ in range(2):
        # 256-bit increment with carry
        for w in range(4):
            c[w] = (c[w] + 1) % 2**64
            if c[w] != 0:
                break
        outs.append(philox.philox4x64_10(np.array(c, dtype=np.uint64), np.array(key, dtype=np.uint64)))
    assert np.array_equal(np.concatenate(outs), ref)


def test_z4_codes_uniform_and_independent():
    N = 12 * 4096
    codes = np.concatenate([noise.z0_codes(7, r, N) for r in range(4)])
    n = len(codes)
    counts = np.bincount(codes, minlength=4)
    chi2 = np.sum((counts - n / 4) ** 2 / (n / 4))
    assert chi2 < 20.0                       # 3 d.o.f.: p ~ 1.7e-4
    # pairs of consecutive codes: 16 cells, 15 d.o.f.
    pairs = codes[:-1] * 4 + codes[1:]
    pc = np.bincount(pairs, minlength=16)
    chi2p = np.sum((pc - (n - 1) / 16) ** 2 / ((n - 1) / 16))
    assert chi2p < 45.0                      # 15 d.o.f.: p ~ 8e-5
    # different runs and different seeds differ
    assert not np.array_equal(noise.z0_codes(7, 0, 1024), noise.z0_codes(7, 1, 1024))
    assert not np.array_equal(noise.z0_codes(7, 0, 1024), noise.z0_codes(8, 0, 1024))
    # values are exactly the fourth roots of unity
    z = noise.z0_vector(7, 0, 1000)
    assert np.all(np.abs(z) == 1.0) and np.all(z ** 4 == 1.0)


@pytest.mark.parametrize("ncolors,expect", [(2, 2), (16, 2), (32, 4), (256, 4), (512, 8)])
def test_hp_min_same_colour_distance(ncolors, expect):
    """Section 6.2: 32 HP vectors remove distances 1, 2, 3 (closing at
    distance 4); 512 the next closing.  Brute force over all same-colour pairs on 8^4."""
    dims = (8, 8, 8, 8)
    col = noise.hp_colour(dims, ncolors)
    assert len(np.unique(col)) == ncolors
    c = lattice.coords(dims)
    L = np.array(dims)
    best = 10 ** 9
    for colour in range(ncolors):
        m = c[col == colour]
        d = np.abs(m[:, None, :] - m[None, :, :])
        d = np.minimum(d, L - d).sum(axis=2)
        d[np.arange(len(m)), np.arange(len(m))] = 10 ** 9
        best = min(best, int(d.min()))
    assert best == expect


def test_hp_colouring_nested():
    dims = (8, 8, 8, 8)
    seq = [1, 2, 16, 32, 256, 512]
    for a, b in zip(seq[:-1], seq[1:]):
        assert np.array_equal(noise.hp_colour(dims, b) % a, noise.hp_colour(dims, a))


def test_hadamard_orthogonal_and_nested():
    n = 64
    c = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    H = noise.hadamard_entry(c, j)
    assert np.array_equal(H.T @ H, n * np.eye(n, dtype=np.int64))
    # first m columns depend only on c mod m (nesting of probing spaces)
    for m in (2, 16, 32):
        assert np.array_equal(H[:, :m], H[c[:, 0] % m][:, :m])


def test_colour_period_rejects_incompatible_dims():
    assert noise.colour_period(32) == 4
    assert noise.colour_period(512) == 8
    with pytest.raises(ValueError):
        noise.colour_period(3)


def test_probing_vector_structure():
    dims = (4, 4, 4, 4)
    N = 12 * lattice.volume(dims)
    Z = noise.noise_vectors(dims, 3, 2, 16, False, 0, 16)
    z0 = noise.z0_vector(3, 2, N)
    # column 0 is z0 itself (H[., 0] = 1)
    assert np.array_equal(Z[:, 0], z0)
    # Z^H Z / N -> probing projector: columns are orthogonal
    G = Z.conj().T @ Z
    assert np.allclose(G, N * np.eye(16))
    Zd = noise.noise_vectors(dims, 3, 2, 2, True, 0, 24)
    assert np.count_nonzero(Zd) == N * 24 // 12


@pytest.mark.parametrize("N,seed,run", [(3072, 0, 0), (49152, 2**63 + 5, 17), (1 << 20, 9, 3)])
def test_z0_codes_at_matches_whole_field(N, seed, run):
    """The restricted evaluation draws the same codes as the whole-field one at
    any index set (including repeats, block edges and the last dof)."""
    rng = np.random.default_rng(N)
    idx = np.concatenate([rng.integers(0, N, size=500), [0, 127, 128, N - 1, N - 1, 31, 32]])
    assert np.array_equal(noise.z0_codes_at(seed, run, idx), noise.z0_codes(seed, run, N)[idx])
