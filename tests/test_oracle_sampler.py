"""Pins of the oracle's counter-based generator and Metropolis-Hastings
frequency sampler (Sec. 3.3, Eqs. 3.18-3.22; Algorithm 1 line 2).

The generator is checked against numpy's Philox4x64-10, an independent
implementation of the same published algorithm; the sampler by a chi-square
test of its (thinned) output against the exact target F~(k)/(pi^{3/2} S)."""
import math

import numpy as np
import pytest
from scipy.stats import chi2

import oracle as O
from tests._util import prod_sog


@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([5, 7, 9, 11], [123, 456]),
                                     ([2**64 - 2, 2**63, 1, 2**40], [2**64 - 1, 99]),
                                     ([123456789, 1, 0, 0], [0xDEADBEEF, 3])])
def test_philox_matches_numpy(ctr, key):
    """numpy.random.Philox(counter=c, key=k) emits the block for counter c+1."""
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    c1 = list(ctr)
    c1[0] += 1
    for i in range(4):          # carry into the next word
        if c1[i] >= 2**64:
            c1[i] -= 2**64
            if i < 3:
                c1[i + 1] += 1
        else:
            break
    assert O.philox4x64_10(c1, key) == ref


def exact_pmf(sog, L):
    """Target P_k = F~(k) / (pi^{3/2} S) over a box holding all but 1e-16 of the mass."""
    L = np.asarray(L, float)
    kcut = 2 * math.sqrt(math.log(1e18)) / sog.s[0]
    mm = np.ceil(kcut * L / (2 * math.pi)).astype(int)
    axes = [np.arange(-mm[d], mm[d] + 1) for d in range(3)]
    m = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / L) ** 2, axis=1)
    p = np.zeros(len(m))
    for l in range(sog.M + 1):
        p += sog.omega[l] * sog.s[l] ** 3 * np.exp(-sog.s[l] ** 2 * k2 / 4)
    S = sog.S(L)
    return m, k2, p / S, p.sum() / S


@pytest.mark.parametrize("L", [(12.6, 12.6, 12.6), (10.0, 12.0, 15.0)])
def test_mh_chain_matches_target_chi2(L):
    sog = prod_sog(O)
    m, k2, pmf, tot = exact_pmf(sog, L)
    assert tot == pytest.approx(1.0, abs=1e-12)
    n_chains, chain_len, thin = 64, 8000, 10
    seq = O.kseq(sog, L, seed=20220527, n_chains=n_chains, chain_len=chain_len)
    seq = seq.reshape(n_chains, chain_len, 3)[:, ::thin, :].reshape(-1, 3)
    assert not np.any(np.all(seq == 0, axis=1))
    # bins of equal target mass along k^2, then the individual vectors of the
    # smallest shell, so that both the radial law and the angular symmetry count
    Lv = np.asarray(L, float)
    ks = np.sum((2 * math.pi * seq / Lv) ** 2, axis=1)
    order = np.argsort(k2, kind="stable")
    cum = np.cumsum(pmf[order])
    nb = 30
    edges_idx = np.searchsorted(cum, np.linspace(0, 1, nb + 1)[1:-1])
    edges = np.unique(k2[order][edges_idx])
    obs = np.bincount(np.searchsorted(edges, ks, side="right"), minlength=len(edges) + 1)
    exp_ = np.bincount(np.searchsorted(edges, k2, side="right"), weights=pmf,
                       minlength=len(edges) + 1) * len(seq)
    assert np.all(obs[exp_ == 0] == 0)
    obs, exp_ = obs[exp_ > 0], exp_[exp_ > 0]
    stat = np.sum((obs - exp_) ** 2 / exp_)
    p_radial = chi2.sf(stat, len(exp_) - 1)
    small = np.where(k2 == k2.min())[0]
    obs_s = np.array([np.sum(np.all(seq == m[i], axis=1)) for i in small])
    exp_s = pmf[small] * len(seq)
    stat_s = np.sum((obs_s - exp_s) ** 2 / exp_s)
    p_small = chi2.sf(stat_s, len(small))
    assert p_radial > 1e-3, (stat, len(exp_))
    assert p_small > 1e-3, (obs_s, exp_s)


def test_kseq_is_concatenated_chains():
    """Algorithm 1's sequence is chain c in entries [c*len, (c+1)*len)."""
    sog = prod_sog(O)
    L = (12.6, 12.6, 12.6)
    seq = O.kseq(sog, L, seed=7, n_chains=5, chain_len=300)
    for c in range(5):
        ch, it = O.mh_chain(sog, L, seed=7, chain=c, length=300)
        assert np.array_equal(seq[c * 300:(c + 1) * 300], ch)
        assert it >= 300


def test_acceptance_rate_in_expected_range():
    """Independence MH with the widest-Gaussian proposal accepts about half
    the proposals at these boxes (a broken ratio drives this to 0 or 1)."""
    sog = prod_sog(O)
    for L, lo, hi in ((12.6, 0.45, 0.7), (128.0, 0.4, 0.65)):
        ch, it = O.mh_chain(sog, (L, L, L), seed=3, chain=0, length=20000)
        moves = np.sum(np.any(ch[1:] != ch[:-1], axis=1)) / (len(ch) - 1)
        assert lo < moves < hi, moves
