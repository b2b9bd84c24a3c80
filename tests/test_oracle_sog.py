"""Pins of the oracle's sum-of-Gaussians decomposition and Fourier-side
quantities against the paper's printed numbers and closed forms.

Covers: Eq. 2.5 (bilateral series), Eq. 2.6 (pointwise error bound),
Eqs. 2.8-2.11 (u-series weights, C0/C1 solve), Table 1, Eq. 3.5 (F~),
Eqs. 3.16-3.17 (S and H), Eq. 3.22 (proposal masses)."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.stats import norm

import oracle as O
from tests._util import B_PROD, M_PROD, prod_sog, table1, untruncated_M


@pytest.mark.parametrize("row", [r for r in table1() if r["reproducible"]], ids=lambda r: f"b={r['b']}")
def test_table1_rows_reproduced(row):
    """Table 1 rows 1 and 3: the joint C0/C1 solve at r_c = 10 gives the
    printed sigma and w0 multiplier to 9 digits."""
    s = O.SOG.solve(row["b"], 10.0, untruncated_M(row["b"]))
    assert s.sigma == pytest.approx(row["sigma"], rel=1e-9)
    assert s.omega0 / s.omega_bsa0 == pytest.approx(row["w0"], rel=1e-9)


def test_table1_eps_column_is_pointwise_bound():
    """The eps column of Table 1 is 2 sqrt(2) exp(-pi^2 / (2 ln b)) (Eq. 2.6)
    to the printed digits; row 5 prints 3.389e-11 where the formula gives
    3.889e-11 (one transposed digit)."""
    rows = table1()
    for r in rows[:4]:
        eps = 2 * math.sqrt(2) * math.exp(-math.pi ** 2 / (2 * math.log(r["b"])))
        assert eps == pytest.approx(r["eps"], rel=2e-3)
    eps5 = 2 * math.sqrt(2) * math.exp(-math.pi ** 2 / (2 * math.log(rows[4]["b"])))
    assert eps5 == pytest.approx(3.889e-11, rel=1e-3)


@pytest.mark.parametrize("b", [2.0, 1.62976708826776469, B_PROD])
def test_bsa_pointwise_error_bound(b):
    """Eq. 2.6: the relative error of the bilateral series (Eq. 2.5) is
    bounded by, and asymptotically equal to, 2 sqrt(2) e^{-pi^2/(2 ln b)}."""
    bound = 2 * math.sqrt(2) * math.exp(-math.pi ** 2 / (2 * math.log(b)))
    rs = np.exp(np.linspace(math.log(0.5), math.log(50.0), 300))
    err = max(abs(1 - r * O.bsa(b, 1.0, r)) for r in rs)
    assert err <= 1.01 * bound
    assert err >= 0.95 * bound


def test_bsa_matches_gamma_integral_at_fine_b():
    """For b -> 1 the quadrature Eq. 2.5 of the integral Eq. 2.4 is exact:
    at b = 1.1 the error bound is 1e-20, so r * BSA(r) = 1 to rounding."""
    for r in (0.3, 1.0, 7.0):
        assert r * O.bsa(1.1, 0.7, r) == pytest.approx(1.0, abs=1e-13)


def test_c0_c1_conditions_hold_for_solve():
    """The solved (sigma, w0) make N = 1/r - F_M continuous with a
    continuous derivative at r_c (Eqs. 2.10-2.11, C1 read with +)."""
    for b, rc in ((2.0, 10.0), (B_PROD, 3.0), (1.3, 2.5)):
        M = untruncated_M(b)
        s = O.SOG.solve(b, rc, M)
        assert rc * s.F(rc)[0] == pytest.approx(1.0, abs=1e-13)
        assert 1.0 + rc * rc * s.dF(rc)[0] == pytest.approx(0.0, abs=1e-11)


def test_solve_is_scale_covariant():
    """sigma scales with r_c and w0/w0_bsa is invariant, so Table 1 row 3
    maps to r_c = 3 by sigma -> 0.3 sigma."""
    a = O.SOG.solve(B_PROD, 10.0, untruncated_M(B_PROD))
    c = O.SOG.solve(B_PROD, 3.0, untruncated_M(B_PROD))
    assert c.sigma == pytest.approx(0.3 * a.sigma, rel=1e-12)
    assert c.omega0 / c.omega_bsa0 == pytest.approx(a.omega0 / a.omega_bsa0, rel=1e-12)


def test_weights_follow_eq_2_9():
    """w_l / w_{l+1} = b and s_{l+1} / s_l = b, s_0 = sqrt(2) sigma,
    w_1 = sqrt(2/pi) ln b / (b sigma)."""
    s = O.SOG(1.7, 0.9, 0.5, 10)
    assert np.allclose(s.omega[1:-1] / s.omega[2:], 1.7, rtol=1e-14)
    assert np.allclose(s.s[1:] / s.s[:-1], 1.7, rtol=1e-14)
    assert s.s[0] == pytest.approx(math.sqrt(2) * 0.9, rel=1e-15)
    assert s.omega[1] == pytest.approx(math.sqrt(2 / math.pi) * math.log(1.7) / (1.7 * 0.9), rel=1e-14)
    assert s.omega[0] == 0.5


def test_production_kernel_accuracy():
    """The production set (Table 1 row 3 at r_c = 3, M = 36) approximates
    1/r with relative error <= 1e-4 on [r_c, 128] and ~ Eq. 2.6 near r_c."""
    s = prod_sog(O)
    rs = np.linspace(3.0, 128.0, 1500)
    err = np.abs(rs * s.F(rs) - 1.0)
    assert err.max() <= 1e-4
    assert err[rs <= 12.6].max() <= 2e-5


@pytest.mark.parametrize("sw", [(0.7, 0.9), (1.5, 0.3), (4.0, 0.05)])
def test_ftilde_is_fourier_transform(sw):
    """Eq. 3.5 for one Gaussian: the radial inverse transform
    (1/(2 pi^2 r)) int_0^inf F~(k) k sin(kr) dk returns w e^{-r^2/s^2}."""
    s_w, w = sw
    g = O.SOG(2.0, s_w / math.sqrt(2), w, 0)          # single Gaussian, s_0 = s_w
    kmax = 14.0 / s_w
    for r in (0.2, 1.0, 2.5):
        val, _ = integrate.quad(lambda k: g.ftilde(k * k)[0] * k * math.sin(k * r), 0, kmax,
                                limit=400, epsabs=1e-14, epsrel=1e-12)
        val /= 2 * math.pi ** 2 * r
        assert val == pytest.approx(w * math.exp(-r * r / s_w ** 2), rel=1e-9, abs=1e-14)


def test_ftilde_sums_over_gaussians():
    s = prod_sog(O)
    for k2 in (0.1, 1.0, 9.0):
        parts = sum(O.SOG(2.0, s.s[l] / math.sqrt(2), s.omega[l], 0).ftilde(k2)[0] for l in range(s.M + 1))
        assert s.ftilde(k2)[0] == pytest.approx(parts, rel=1e-13)


@pytest.mark.parametrize("ratio", [0.05, 0.3, 1.0, 2.5])
def test_H_poisson_dual(ratio):
    """Eq. 3.17: direct theta sum equals its Poisson dual (read without the
    printed pi^2 in the dual exponent)."""
    L = 10.0
    s = ratio * L
    assert O.H(s, L, 0) == pytest.approx(O.H(s, L, 1), rel=1e-14)


@pytest.mark.parametrize("L", [(12.6, 12.6, 12.6), (10.0, 12.0, 15.0)])
def test_S_equals_lattice_sum(L):
    """Eq. 3.16: S = pi^{-3/2} sum_{k != 0} F~(k), checked by brute-force
    summation over the integer lattice."""
    s = prod_sog(O)
    L = np.array(L)
    kcut = 2 * math.sqrt(math.log(1e20)) / s.s[0]
    mm = np.ceil(kcut * L / (2 * math.pi)).astype(int)
    axes = [np.arange(-mm[d], mm[d] + 1) for d in range(3)]
    m = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / L) ** 2, axis=1)
    # pi^{-3/2} F~(k) = sum_l w_l s_l^3 exp(-s_l^2 k^2 / 4)
    tot = 0.0
    for l in range(s.M + 1):
        tot += np.sum(s.omega[l] * s.s[l] ** 3 * np.exp(-s.s[l] ** 2 * k2 / 4))
    assert s.S(L) == pytest.approx(tot, rel=1e-12)


@pytest.mark.parametrize("L", [12.6, 128.0])
def test_proposal_masses(L):
    """Eq. 3.22: q(m) is the N(0, (L/(s_0 pi))^2/2) density integrated over
    [m - 1/2, m + 1/2]; the masses sum to one."""
    s = prod_sog(O)
    s0 = s.s[0]
    sd = L / (math.sqrt(2) * math.pi * s0)
    K = int(12 * sd) + 3
    ms = range(-K, K + 1)
    q = np.array([O.proposal_q1(m, s0, L) for m in ms])
    ref = np.array([norm.cdf((m + 0.5) / sd) - norm.cdf((m - 0.5) / sd) for m in ms])
    assert q.sum() == pytest.approx(1.0, abs=1e-13)
    assert np.allclose(q, ref, rtol=1e-9, atol=1e-15)
