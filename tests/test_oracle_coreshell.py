"""Pins of the oracle's core-shell near-field kernel (Sec. 3.4, Eqs.
3.25-3.26): the Taylor core stays within the alternating-series bound of
its first omitted term, the bit-indexed shell table within the linear
interpolation bound h^2/8 max|g''| plus the FP32 rounding of r^2 that picks
the bin, and with many terms and index bits the whole near field converges
to the direct Gaussian sums."""
import math

import numpy as np
import pytest

import oracle as O
from tests._util import prod_sog


def _sys(L=20.0):
    sog = prod_sog(O)
    return O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0), sog


def _exact(sog, r2):
    r = math.sqrt(r2)
    G = np.sum(sog.omega / sog.s ** 2 * np.exp(-r2 / sog.s ** 2))
    F = np.sum(sog.omega * np.exp(-r2 / sog.s ** 2))
    return 1.0 / (r2 * r) - 2.0 * G, 1.0 / r - F


@pytest.mark.parametrize("Q", [4, 8, 10])
def test_core_taylor_within_first_omitted_term(Q):
    s, sog = _sys()
    cs = O.coreshell(1.0, Q=Q)
    for r2 in np.linspace(0.05, 0.999, 60):
        g, n = O.coreshell_eval(s, cs, r2)
        ge, ne = _exact(sog, r2)
        # per Gaussian the series of e^{-x} alternates with decreasing terms
        # (x = r^2/s^2 < 1 < Q + 1): the error is below the first omitted one
        bg = 2.0 * np.sum(sog.omega / sog.s ** 2 * (r2 / sog.s ** 2) ** Q / math.factorial(Q))
        bn = np.sum(sog.omega * (r2 / sog.s ** 2) ** (Q + 1) / math.factorial(Q + 1))
        assert abs(g - ge) <= bg * (1 + 1e-9) + 1e-13 * ge
        assert abs(n - ne) <= bn * (1 + 1e-9) + 1e-13 * ne


@pytest.mark.parametrize("b_man", [6, 8, 10])
def test_shell_table_within_interpolation_bound(b_man):
    s, sog = _sys()
    cs = O.coreshell(1.0, b_man=b_man)
    for r2 in np.linspace(1.0, 8.999, 400):
        g, n = O.coreshell_eval(s, cs, r2)
        ge, ne = _exact(sog, r2)
        h = 2.0 ** (math.floor(math.log2(r2)) - b_man)          # bin width in u = r^2
        # |g''(u)| <= (15/4) u^{-7/2} + 2 sum w/s^6 and |n''| <= (3/4) u^{-5/2}
        # + sum w/s^4, on the bin (u >= its lower end); the FP32 value of u
        # that picks the bin is within 2^-24 u of u
        u0 = 2.0 ** math.floor(math.log2(r2)) * (1 + math.floor((r2 / 2.0 ** math.floor(math.log2(r2)) - 1)
                                                               * 2 ** b_man) / 2 ** b_man)
        d2g = 15 / 4 * u0 ** -3.5 + 2 * np.sum(sog.omega / sog.s ** 6)
        d2n = 3 / 4 * u0 ** -2.5 + np.sum(sog.omega / sog.s ** 4)
        d1g = 1.5 * u0 ** -2.5 + 2 * np.sum(sog.omega / sog.s ** 4)
        d1n = 0.5 * u0 ** -1.5 + np.sum(sog.omega / sog.s ** 2)
        du = 2.0 ** -24 * r2
        assert abs(g - ge) <= h * h / 8 * d2g + d1g * du + 1e-14
        assert abs(n - ne) <= h * h / 8 * d2n + d1n * du + 1e-14


def test_coreshell_near_field_converges_to_direct_sums():
    import rbsog_inputs as I
    N, L = 1000, 12.6
    q, x, _ = I.electrolyte(N, L, seed=9)
    s, sog = _sys(L)
    xw = O.wrap(x, s.L)
    fd, und, uwd, _ = O.near(s, q, xw, method="direct")
    fc, unc, uwc = O.near_coreshell(s, q, xw, O.coreshell(1.0, Q=16, b_exp=2, b_man=16))
    assert np.linalg.norm(fc - fd) <= 1e-6 * np.linalg.norm(fd)
    assert abs(unc - und) <= 1e-9 * N          # U_near is a sum with cancellation: per particle
    assert uwc == uwd                                         # WCA is not tabulated
    f8, un8, _ = O.near_coreshell(s, q, xw, O.coreshell(1.0))  # the defaults: Q = 10, 2 + 8 index bits
    assert np.linalg.norm(f8 - fd) <= 2e-5 * np.linalg.norm(fd)
    assert abs(un8 - und) <= 1e-6 * N


def test_table_must_reach_the_cutoff():
    s, _ = _sys()
    with pytest.raises(ValueError):
        O.coreshell_eval(s, O.coreshell(0.5, b_exp=2), 8.0)   # 4 octaves from 0.25 end at 4 < 9
    g, _ = O.coreshell_eval(s, O.coreshell(0.5, b_exp=3), 8.0)
    assert math.isfinite(g)
    with pytest.raises(ValueError):
        O.coreshell_eval(s, O.coreshell(1.0), 9.0)           # r = r_c is outside
