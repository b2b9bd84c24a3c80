"""Pins for the oracle's radial distribution functions (Appendix A) that do
not come from the oracle itself: exact coordination shells of a simple cubic
lattice with rock-salt charges (counts from a brute-force enumeration of
integer vectors), a numpy histogram of FP64 minimum-image distances, the
ideal-gas limit g -> 1, and permutation / charge-flip symmetries."""
import math

import numpy as np
import pytest

import oracle
import rbsog_inputs as I


def _r3(m):
    """Number of integer vectors v with |v|^2 = m (brute force)."""
    k = int(math.isqrt(m))
    return sum(1 for a in range(-k, k + 1) for b in range(-k, k + 1) for c in range(-k, k + 1)
               if a * a + b * b + c * c == m)


def _rocksalt(n, a):
    idx = np.arange(n ** 3)
    ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
    x = (np.stack([ix, iy, iz], axis=1) + 0.5) * a
    q = np.where((ix + iy + iz) % 2 == 0, 1.0, -1.0)
    return q, x


def test_rocksalt_lattice_shells_exact():
    """n = 10 sites per edge, spacing a: shell m (distance a sqrt(m) < L/2)
    holds N r3(m) / 2 unordered pairs, all unlike for odd m and split evenly
    between ++ and -- for even m (the parity of a sum of squares is the parity
    of the Manhattan length)."""
    n, a, nbins = 10, 1.26, 64
    L = n * a
    q, x = _rocksalt(n, a)
    N = n ** 3
    counts, g, edges = oracle.rdf(q, x, L, nbins)
    per = 2 * nbins / n                     # bins per lattice spacing
    expected = np.zeros((3, nbins), dtype=np.int64)
    for m in range(1, 25):
        r3 = _r3(m)
        if r3 == 0:
            continue
        pos = math.sqrt(m) * per
        assert abs(pos - round(pos)) > 1e-3    # shell well inside a bin
        b = int(pos)
        if m % 2:
            expected[1, b] += N * r3 // 2
        else:
            expected[0, b] += N * r3 // 4
            expected[2, b] += N * r3 // 4
    # bins below the last one see only the shells m <= 24
    np.testing.assert_array_equal(counts[:, :nbins - 1].astype(np.int64), expected[:, :nbins - 1])
    # first shell: 6 unlike neighbours per site
    b1 = int(per)
    assert counts[1, b1] == 3 * N
    # g at the first shell from the closed form of the shell volume
    dr = L / (2 * nbins)
    shell = 4 * math.pi / 3 * ((b1 + 1) ** 3 - b1 ** 3) * dr ** 3
    assert g[1, b1] == pytest.approx(3 * N / ((N / 2) * (N / 2) / L ** 3 * shell), rel=1e-13)


def test_counts_match_numpy_histogram_of_fp64_distances():
    rng = np.random.Generator(np.random.PCG64(7))
    N, L, nbins = 700, 14.0, 128
    x = rng.uniform(0, L, size=(N, 3))
    q = rng.choice([-1.0, 1.0], size=N)
    counts, _, edges = oracle.rdf(q, x, L, nbins)
    iu, ju = np.triu_indices(N, 1)
    d = x[iu] - x[ju]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(axis=1))
    t = (q[iu] < 0).astype(int) + (q[ju] < 0).astype(int)
    keep = r < L / 2
    for k in range(3):
        h, _ = np.histogram(r[keep & (t == k)], bins=edges)
        # quantising positions to L 2^-32 moves distances by ~1e-9: only a pair
        # within that of a bin edge could change bins
        assert np.abs(h - counts[k].astype(np.int64)).sum() <= 2, k


def test_ideal_gas_limit():
    """Uniform random positions: g(r) -> 1 (within Poisson noise) for every
    sign pair, including the N^2 normalisation of like pairs."""
    rng = np.random.Generator(np.random.PCG64(3))
    N, L, nbins = 6000, 30.0, 16
    x = rng.uniform(0, L, size=(N, 3))
    q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])
    counts, g, _ = oracle.rdf(q, x, L, nbins)
    for t in range(3):
        c = counts[t, 4:].astype(float)
        rel = (g[t, 4:] - 1.0) * np.sqrt(c)      # ~ N(0, 1) per bin
        assert np.all(np.abs(rel) < 5.0), (t, rel)
        assert abs(g[t, 4:].mean() - 1.0) < 0.01


def test_permutation_and_charge_flip_symmetry():
    q, x, _ = I.electrolyte(1000, 12.6, seed=5)
    c0, _, _ = oracle.rdf(q, x, 12.6, 64)
    perm = np.random.Generator(np.random.PCG64(1)).permutation(1000)
    c1, _, _ = oracle.rdf(q[perm], x[perm], 12.6, 64)
    np.testing.assert_array_equal(c0, c1)
    c2, _, _ = oracle.rdf(-q, x, 12.6, 64)
    np.testing.assert_array_equal(c0[[2, 1, 0]], c2)
    # every pair closer than L/2 is counted once
    assert int(c0.sum()) > 0


def test_rejects_bad_bin_counts():
    q, x, _ = I.electrolyte(8, 9.0, seed=1)
    for nb in (8, 100, 8192):
        with pytest.raises(ValueError):
            oracle.rdf(q, x, 9.0, nb)
