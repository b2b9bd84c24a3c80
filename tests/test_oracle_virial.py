"""Pins of the oracle's configurational virial W_ab = -dU/d eps_ab (r -> (1 +
eps) r for positions and box, r_c and the SOG fixed):

  * diagonal: central differences of the total energy (near + WCA + exact
    far) under stretching one axis of the box and the positions;
  * off-diagonal: central differences of the pair energy under a shear of
    the pair separations (the pairs within r_c do not change for a small
    shear), and the symmetry of the tensor;
  * the random-batch far estimator averages to the exact far virial over
    iid k-sets drawn from F~(k)/(pi^{3/2} S)."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog


def _sys(sog, L, wca=True):
    Lv = tuple(L) if not isinstance(L, (int, float)) else (L,) * 3
    return O.System(Lv, sog, 3.0, 1.0, 1.0 if wca else 0.0, 1.0 if wca else 0.0)


def _energy_exact(sog, L, q, x):
    s = _sys(sog, L)
    _, e = O.forces(s, q, O.wrap(x, s.L), S=0.0, m=None)
    return e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"]


def _small():
    q, x, _ = I.electrolyte(1000, 12.6, seed=9)
    sel = np.r_[0:64]
    return q[sel] - q[sel].mean(), x[sel]


def test_diagonal_is_minus_the_energy_derivative_under_axis_stretch():
    sog = prod_sog(O)
    L = 12.6
    q, x = _small()
    W = O.virial(_sys(sog, L), q, O.wrap(x, (L,) * 3))
    h = 1e-6
    for a in range(3):
        sc = np.ones(3)
        sc[a] = 1 + h
        Up = _energy_exact(sog, tuple(L * sc), q, x * sc)
        sc[a] = 1 - h
        Um = _energy_exact(sog, tuple(L * sc), q, x * sc)
        assert W[a, a] == pytest.approx(-(Up - Um) / (2 * h), rel=2e-6, abs=1e-8)


def test_off_diagonal_is_minus_the_pair_energy_derivative_under_shear():
    sog = prod_sog(O)
    L = 12.6
    q, x, _ = I.electrolyte(1000, L, seed=3)
    s = _sys(sog, L, wca=False)
    xw = O.wrap(x, s.L)
    # near-field pairs and their minimum-image separations
    n = len(q)
    d = xw[:, None, :] - xw[None, :, :]
    d -= L * np.round(d / L)
    iu = np.triu_indices(n, 1)
    dd = d[iu]
    r = np.linalg.norm(dd, axis=1)
    keep = r < 2.9                                   # a margin below r_c: no pair crosses it
    dd, qq = dd[keep], (q[:, None] * q[None, :])[iu][keep]

    def U(eps, a, b):
        e = dd.copy()
        e[:, a] += eps * dd[:, b]
        rr = np.linalg.norm(e, axis=1)
        return np.sum(qq * (1.0 / rr - sog.F(rr)))

    # the oracle's near virial over the same pairs: cutoff lowered to 2.9
    s29 = O.System((L,) * 3, sog, 2.9, 1.0, 0.0, 0.0)
    Wn = O.virial(s29, q, xw, S=0.0, m=np.ones((1, 3)))      # S = 0: the far estimator adds nothing
    h = 1e-6
    for a, b in ((0, 1), (1, 2), (2, 0), (1, 0)):
        fd = -(U(h, a, b) - U(-h, a, b)) / (2 * h)
        assert Wn[a, b] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert np.allclose(Wn, Wn.T, rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_random_batch_far_virial_is_unbiased():
    sog = prod_sog(O)
    L = 12.6
    q, x = _small()
    s = _sys(sog, L, wca=False)
    xw = O.wrap(x, s.L)
    S = s.S()
    s0 = O.System((L,) * 3, sog, 1e-3, 1.0, 0.0, 0.0)   # r_c -> 0: far part only
    W_ex = O.virial(s0, q, xw)
    kcut = 2 * math.sqrt(math.log(1e18)) / sog.s[0]
    mm = int(math.ceil(kcut * L / (2 * math.pi)))
    r1 = np.arange(-mm, mm + 1)
    m = np.stack(np.meshgrid(r1, r1, r1, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / L) ** 2, axis=1)
    p = np.zeros(len(m))
    for l in range(sog.M + 1):
        p += sog.omega[l] * sog.s[l] ** 3 * np.exp(-sog.s[l] ** 2 * k2 / 4)
    pmf = p / p.sum()
    rng = np.random.default_rng(7)
    K, P = 2000, 8
    Ws = np.array([O.virial(s0, q, xw, S=S, m=m[rng.choice(len(m), size=P, p=pmf)]) for _ in range(K)])
    mean, err = Ws.mean(0), Ws.std(0) / math.sqrt(K)
    assert np.all(np.abs(mean - W_ex) <= 4 * err + 1e-12)
