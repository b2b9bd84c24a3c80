"""Pins of the oracle's near field, far field, self energy and cell list.

  * textbook Ewald summation (an independent split of 1/r) for energy and
    forces, with its own forces checked by finite differences;
  * the NaCl Madelung constant;
  * central finite differences of the oracle's own energies (sign and factor
    of Eq. 3.9, read as -grad U);
  * O(N^2) brute force for the cell list and neighbour counts;
  * per-k invariants of the random-batch force (Eq. 3.24): zero net force,
    no self force;
  * Lemma 1: unbiasedness of Eq. 3.24 and its variance (Eq. 4.8, read with
    |k|^2 inside the sum)."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import ewald, nacl, prod_sog, tight_sog

MADELUNG_NACL = 1.747564594633182  # rock-salt Madelung constant (nearest-neighbour units)


def _system(sog, L, rc=3.0, wca=False):
    return O.System((L, L, L), sog, rc, 1.0, 1.0 if wca else 0.0, 1.0 if wca else 0.0)


def _total(sys_, q, x, m=None, S=0.0):
    f, e = O.forces(sys_, q, x, S=S, m=m)
    return f, e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"], e


def test_ewald_reference_is_self_consistent():
    """The test's Ewald forces are -grad of its own energy."""
    q, x = I.random_neutral(8, 6.0, seed=1, min_dist=0.8)
    U, f = ewald(q, x, 6.0)
    h = 1e-5
    for i, d in ((0, 0), (3, 2), (5, 1)):
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        fd = -(ewald(q, xp, 6.0)[0] - ewald(q, xm, 6.0)[0]) / (2 * h)
        assert f[i, d] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.slow
def test_total_matches_ewald_tight():
    """Near + exact far - self with the b = 1.218 set (eps ~ 4e-11, untruncated)
    reproduces tinfoil Ewald energy and forces of a random neutral system."""
    sog = tight_sog(O)
    L = 12.6
    q, x = I.random_neutral(40, L, seed=11, min_dist=0.8)
    sys_ = _system(sog, L)
    f, U, _ = _total(sys_, q, x)
    Ue, fe = ewald(q, x, L)
    assert U == pytest.approx(Ue, rel=1e-9)
    rms = np.sqrt(np.sum((f - fe) ** 2) / np.sum(fe ** 2))
    assert rms < 1e-8


def test_total_matches_ewald_production():
    """The production set (eps ~ 1e-5, M = 36) agrees with Ewald at the
    1e-5 level for an electrolyte snapshot."""
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=5)
    sub = np.r_[0:60]
    q, x = q[sub], x[sub]
    q = q - q.mean()       # exactly neutral subset
    sys_ = _system(sog, L)
    f, U, _ = _total(sys_, q, x)
    Ue, fe = ewald(q, x, L)
    assert U == pytest.approx(Ue, rel=2e-5)
    rms = np.sqrt(np.sum((f - fe) ** 2) / np.sum(fe ** 2))
    assert rms < 5e-5


@pytest.mark.parametrize("tight", [True, False])
def test_madelung_nacl(tight):
    """Rock salt, 6^3 ions, spacing a = 1.5 (box 9 = 3 r_c): energy per ion
    pair is -1.7475645946 / a."""
    a = 1.5
    q, x = nacl(6, a)
    sog = tight_sog(O) if tight else prod_sog(O)
    sys_ = _system(sog, 9.0)
    _, U, _ = _total(sys_, q, x)
    per_pair = U / (len(q) / 2)
    tol = 1e-9 if tight else 3e-5
    assert per_pair == pytest.approx(-MADELUNG_NACL / a, rel=tol)


def test_like_charges_repel_unlike_attract():
    sog = prod_sog(O)
    L = 12.6
    q = np.array([1.0, 1.0, -1.0, -1.0])
    x = np.array([[2.0, 2.0, 2.0], [3.2, 2.0, 2.0], [8.0, 8.0, 8.0], [9.1, 8.0, 8.0]])
    f, _, _ = _total(_system(sog, L), q, x)
    assert f[0, 0] < 0 < f[1, 0]
    assert f[2, 0] < 0 < f[3, 0]
    # beyond r_c the pair acts only through the far field: check its sign too
    x2 = np.array([[2.0, 2.0, 2.0], [6.0, 2.0, 2.0], [2.0, 8.0, 8.0], [6.0, 8.0, 8.0]])
    q2 = np.array([1.0, 1.0, -1.0, -1.0])
    ff, _ = O.far_exact(_system(sog, L), q2, x2)
    assert ff[0, 0] < 0 < ff[1, 0]


def _fd(fun, x, i, d, h):
    """Fourth-order central difference of -dU/dx[i, d]."""
    def at(t):
        xx = x.copy()
        xx[i, d] += t
        return fun(xx)
    return -(8 * (at(h) - at(-h)) - (at(2 * h) - at(-2 * h))) / (12 * h)


def test_near_force_is_minus_grad_energy():
    """Eq. 3.9 near line read as -grad of U_N (bracket 1/r^3 - 2 sum w/s^2 e^{..}),
    WCA included."""
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=2)
    sys_ = _system(sog, L, wca=True)
    f, _, _, _ = O.near(sys_, q, x)

    def U(xx):
        _, un, uw, _ = O.near(sys_, q, xx)
        return un + uw

    for i, d in ((3, 0), (100, 1), (777, 2)):
        fd = _fd(U, x, i, d, 1e-4)
        assert f[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_far_exact_force_is_minus_grad_energy():
    """Eq. 3.9 far line with the sign of -grad U*_F."""
    sog = prod_sog(O)
    L = 12.6
    q, x = I.random_neutral(16, L, seed=4, min_dist=0.8)
    sys_ = _system(sog, L)
    f, _ = O.far_exact(sys_, q, x)
    for i, d in ((0, 0), (7, 1), (15, 2)):
        fd = _fd(lambda xx: O.far_exact(sys_, q, xx)[1], x, i, d, 1e-4)
        assert f[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_self_energy_closed_form():
    """Eq. 3.8 holds for the unmodified w_0; with the C0 w_0 the self energy
    is (1/2) F_M(0) sum q^2."""
    sog = O.SOG(1.5, 0.8, 0.0, 20)
    sog.omega[0] = sog.omega_bsa0
    sys_ = _system(sog, 12.6)
    q = np.array([1.0, -1.0, 2.0, -2.0])
    b, sg, M = 1.5, 0.8, 20
    printed = (b - b ** (-M)) * math.log(b) / (math.sqrt(2 * math.pi * sg ** 2) * (b - 1)) * np.sum(q ** 2)
    assert O.self_energy(sys_, q) == pytest.approx(printed, rel=1e-13)


def test_cell_list_matches_binning():
    """Cells of side h = L / floor(L / r_c): particle i goes to floor(x / h)
    per axis, members of a cell in increasing index (a stable sort of the
    cell ids), cell_start the prefix sum of the counts."""
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=3)
    nc, cell_of, start, perm = O.cell_list(x, (L, L, L), 3.0)
    assert list(nc) == [4, 4, 4]
    h = L / 4
    c = np.minimum(np.floor(x / h).astype(int), 3)
    ref = (c[:, 2] * 4 + c[:, 1]) * 4 + c[:, 0]
    assert np.array_equal(cell_of, ref)
    assert np.array_equal(perm, np.argsort(ref, kind="stable"))
    assert np.array_equal(start, np.r_[0, np.cumsum(np.bincount(ref, minlength=64))])
    # a cuboid box with unequal cell counts per axis
    Lv = (9.3, 12.0, 15.1)
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, size=(500, 3)) * np.array(Lv)
    nc, cell_of, start, perm = O.cell_list(x, Lv, 3.0)
    n3 = np.floor(np.array(Lv) / 3.0).astype(int)
    assert list(nc) == list(n3)
    c = np.minimum(np.floor(x / (np.array(Lv) / n3)).astype(int), n3 - 1)
    ref = (c[:, 2] * n3[1] + c[:, 1]) * n3[0] + c[:, 0]
    assert np.array_equal(cell_of, ref)
    assert np.array_equal(perm, np.argsort(ref, kind="stable"))


def test_neighbour_counts_match_bruteforce():
    """Cell-list traversal finds exactly the pairs with |r_ij| < r_c of an
    O(N^2) minimum-image scan (same FP64 decision), and the same forces."""
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=6)
    sys_ = _system(sog, L, wca=True)
    fc, unc, uwc, nbc = O.near(sys_, q, x, "cells")
    fd, und, uwd, nbd = O.near(sys_, q, x, "direct")
    d = x[:, None, :] - x[None, :, :]
    d = d - L * np.rint(d / L)
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    np.fill_diagonal(r2, np.inf)
    cnt = np.sum(r2 < 9.0, axis=1)
    assert np.array_equal(nbc, cnt)
    assert np.array_equal(nbd, cnt)
    assert np.allclose(fc, fd, rtol=1e-12, atol=1e-12)
    assert unc == pytest.approx(und, rel=1e-13)
    assert 40 < cnt.mean() < 75      # ~ (4/3) pi 27 * 0.5 = 56.5 at density 0.5


def test_rb_per_k_zero_net_force_and_no_self_force():
    """Im(rho* rho) = 0 makes the random-batch force sum to zero for every k;
    a lone charge feels no far force from itself."""
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=8)
    sys_ = _system(sog, L)
    S = sys_.S()
    for m in ([1, 0, 0], [3, -2, 5], [-7, 1, 1]):
        f, _, _ = O.far_rb(sys_, q, x, S, np.array([m]))
        assert np.all(np.abs(f.sum(0)) <= 1e-12 * np.abs(f).sum())
    f1, _, _ = O.far_rb(sys_, np.array([1.0]), np.array([[1.0, 2.0, 3.0]]), S, np.array([[2, 1, 0]]))
    assert np.all(f1 == 0.0)


def test_rho_matches_direct_sum():
    rng = np.random.default_rng(0)
    q = rng.normal(size=50)
    x = rng.uniform(0, 10, size=(50, 3))
    m = rng.integers(-9, 10, size=(7, 3))
    r = O.rho(q, x, (10.0, 11.0, 12.0), m)
    k = 2 * np.pi * m / np.array([10.0, 11.0, 12.0])
    ref = (q[:, None] * np.exp(1j * (x @ k.T))).sum(0)
    assert np.allclose(r, ref, rtol=1e-13, atol=1e-12)


def _enumerate(sog, L):
    kcut = 2 * math.sqrt(math.log(1e18)) / sog.s[0]
    mm = int(math.ceil(kcut * L / (2 * math.pi)))
    r1 = np.arange(-mm, mm + 1)
    m = np.stack(np.meshgrid(r1, r1, r1, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / L) ** 2, axis=1)
    p = np.zeros(len(m))
    for l in range(sog.M + 1):
        p += sog.omega[l] * sog.s[l] ** 3 * np.exp(-sog.s[l] ** 2 * k2 / 4)
    return m, k2, p


@pytest.mark.slow
def test_rb_unbiased_and_lemma1_variance():
    """Lemma 1: with k drawn iid from F~(k)/(pi^{3/2} S), the mean of Eq. 3.24
    is the exact far force and E|Xi_i|^2 = (1/P)[pi^{3/2} S q_i^2/V^2
    sum_k F~(k) |k|^2 Im(e^{-ik.r_i} rho)^2 - |F_i|^2]; also E U*_RB = U*."""
    sog = prod_sog(O)
    L = 12.6
    V = L ** 3
    q, x, _ = I.electrolyte(1000, L, seed=9)
    sel = np.r_[0:48]
    q, x = q[sel] - q[sel].mean(), x[sel]
    sys_ = _system(sog, L)
    S = sys_.S()
    F_ex, U_ex = O.far_exact(sys_, q, x)
    m, k2, p = _enumerate(sog, L)
    pmf = p / p.sum()
    rng = np.random.default_rng(2022)
    K, P = 3000, 8
    Fs = np.zeros((K, len(q), 3))
    Us = np.zeros(K)
    for t in range(K):
        ms = m[rng.choice(len(m), size=P, p=pmf)]
        Fs[t], Us[t], _ = O.far_rb(sys_, q, x, S, ms)
    mean = Fs.mean(0)
    # Lemma 1 variance from the full sum over k
    k = 2 * math.pi * m / L
    rho = (q[:, None] * np.exp(1j * (x @ k.T))).sum(0)
    th = x @ k.T
    im = np.cos(th) * rho.imag[None, :] - np.sin(th) * rho.real[None, :]
    ft = math.pi ** 1.5 * p
    var_th = (math.pi ** 1.5 * S * q ** 2 / V ** 2 * ((ft * k2)[None, :] * im ** 2).sum(1)
              - np.sum(F_ex ** 2, axis=1)) / P
    var_emp = np.sum((Fs - F_ex[None]) ** 2, axis=(0, 2)) / K
    assert np.allclose(var_emp, var_th, rtol=0.15)
    # unbiasedness: standardised error of the mean
    z = np.sum((mean - F_ex) ** 2, axis=1) / (var_th / K)   # E z = 1 per particle
    assert 0.6 < np.mean(z) < 1.4
    assert Us.mean() == pytest.approx(U_ex, abs=4 * Us.std() / math.sqrt(K))


def test_rb_variance_scales_as_one_over_P():
    """Theorem 2: the random-batch variance is O(1/P)."""
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=10)
    sel = np.r_[0:32]
    q, x = q[sel] - q[sel].mean(), x[sel]
    sys_ = _system(sog, L)
    S = sys_.S()
    F_ex, _ = O.far_exact(sys_, q, x)
    m, _, p = _enumerate(sog, L)
    pmf = p / p.sum()
    rng = np.random.default_rng(7)
    v = {}
    for P in (4, 32):
        errs = []
        for _ in range(600):
            ms = m[rng.choice(len(m), size=P, p=pmf)]
            f, _, _ = O.far_rb(sys_, q, x, S, ms)
            errs.append(np.sum((f - F_ex) ** 2))
        v[P] = np.mean(errs)
    assert v[4] / v[32] == pytest.approx(8.0, rel=0.25)
