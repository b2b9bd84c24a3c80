"""Pins of the oracle's per-Gaussian independent sampling (the variant the
paper describes after the mixture sampler, Sec. 3.3): the shares S_l add up to
the normaliser S of Eq. 3.16; the frequencies of each stratum follow the
exact normalised Gaussian pmf over k != 0 (chi-square over |m|^2 bins, zero
mode never drawn, signs symmetric); the weighted estimator is unbiased for the
exact far energy and force; with equal weights S/P it is the mixture
estimator."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog

L3 = (12.6, 12.6, 12.6)


def _exact_pmf_bins(s, L, edges):
    """P(|m|^2 in [edges[i], edges[i+1])) under p(m) ~ exp(-(pi s/L)^2 |m|^2), m != 0."""
    x = (math.pi * s / L) ** 2
    jm = int(math.ceil(math.sqrt(60.0 / x)))
    r = np.arange(-jm, jm + 1)
    w1 = np.exp(-x * r * r)
    m2 = (r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2).ravel()
    w = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :]).ravel()
    keep = m2 > 0
    m2, w = m2[keep], w[keep] / w[keep].sum()
    return np.histogram(m2, bins=edges, weights=w)[0]


def test_shares_sum_to_the_normaliser():
    sog = prod_sog(O)
    for L in (L3, (10.0, 14.0, 21.5)):
        pe, P_l, S_l = O.pg_plan(sog, L, 64)
        S = sog.S(np.array(L))
        assert S_l.sum() == pytest.approx(S, rel=1e-12)
        tot = S_l.sum()
        act = S_l > 1e-16 * tot
        assert np.array_equal(P_l[act], np.ceil(64 * S_l[act] / tot).astype(int))
        assert (P_l[~act] == 0).all() and pe == P_l.sum() and 64 <= pe <= 64 + act.sum()


def test_strata_follow_the_exact_gaussian_pmf():
    from scipy.stats import chi2
    sog = prod_sog(O)
    P, n_sets = 64, 3000
    pe, P_l, _ = O.pg_plan(sog, L3, P)
    m, st = O.pg_kseq(sog, L3, P, seed=11, set0=5, n_sets=n_sets)
    assert not np.any(np.all(m == 0, axis=1))
    for l in np.nonzero(P_l)[0]:
        ml = m[st == l]
        assert len(ml) == n_sets * P_l[l]
        for d in range(3):                       # signs are symmetric
            nz = ml[:, d] != 0
            if nz.sum() > 200:
                frac = (ml[nz, d] > 0).mean()
                assert abs(frac - 0.5) < 5 * 0.5 / math.sqrt(nz.sum())
        m2 = np.sum(ml.astype(np.int64) ** 2, axis=1)
        q = np.quantile(m2, np.linspace(0, 1, 16))
        edges = np.unique(np.concatenate([[1], q[1:-1].round(), [m2.max() + 1, 10 ** 9]]))
        p = _exact_pmf_bins(sog.s[l], L3[0], edges)
        obs = np.histogram(m2, bins=edges)[0]
        exp = p * len(m2)
        ok = exp > 5
        stat = np.sum((obs[ok] - exp[ok]) ** 2 / exp[ok])
        assert stat < chi2.ppf(0.9999, max(ok.sum() - 1, 1)), (l, stat, obs, exp)
        assert obs[~ok].sum() <= max(5 * exp[~ok].sum(), 10)


def test_weighted_estimator_is_unbiased():
    sog = prod_sog(O)
    N, L = 1000, 12.6
    q, x, _ = I.electrolyte(N, L, seed=3)
    s = O.System(L3, sog, 3.0, 1.0, 0.0, 0.0)
    x = O.wrap(x, s.L)
    f_ex, U_ex = O.far_exact(s, q, x)
    P, n_sets = 64, 400
    c = O.pg_weights(sog, L3, P)
    pe = len(c)
    m, _ = O.pg_kseq(sog, L3, P, seed=12, set0=0, n_sets=n_sets)
    Us, Fs = [], []
    for t in range(n_sets):
        f, U = O.far_rb_w(s, q, x, m[t * pe:(t + 1) * pe], c)
        Us.append(U)
        Fs.append(f[:8])
    Us, Fs = np.array(Us), np.array(Fs)
    se = Us.std(ddof=1) / math.sqrt(n_sets)
    assert abs(Us.mean() - U_ex) < 4.5 * se, (Us.mean(), U_ex, se)
    fse = Fs.std(axis=0, ddof=1) / math.sqrt(n_sets)
    z = np.abs(Fs.mean(axis=0) - f_ex[:8]) / fse
    assert z.max() < 5.0, z.max()


def test_equal_weights_give_the_mixture_estimator():
    sog = prod_sog(O)
    N, L = 1000, 12.6
    q, x, _ = I.electrolyte(N, L, seed=4)
    s = O.System(L3, sog, 3.0, 1.0, 0.0, 0.0)
    x = O.wrap(x, s.L)
    m = O.kseq(sog, s.L, seed=2, n_chains=1, chain_len=48)[:48]
    S = s.S()
    f0, U0, _ = O.far_rb(s, q, x, S, m)
    f1, U1 = O.far_rb_w(s, q, x, m, np.full(48, S / 48))
    assert U1 == pytest.approx(U0, rel=1e-13)
    assert np.allclose(f1, f0, rtol=1e-12, atol=1e-13 * np.abs(f0).max())
