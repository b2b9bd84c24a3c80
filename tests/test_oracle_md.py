"""Pins of the oracle's velocity-Verlet driver (Algorithm 1): second-order
energy conservation, time reversibility, the Berendsen rescale, and the
order in which the pre-sampled frequency sequence is consumed."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog


def _sys(L=12.6):
    return O.System((L, L, L), prod_sog(O), 3.0, 1.0, 1.0, 1.0)


def _etot(es):
    return np.array([e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"] + e["K"] for e in es])


def _small_state():
    q, x, v = I.electrolyte(1000, 12.6, seed=12)
    sel = np.r_[0:60]
    return q[sel] - q[sel].mean(), x[sel], v[sel]


@pytest.mark.slow
def test_nve_energy_error_is_second_order():
    """With the exact far sum, the energy fluctuation of velocity Verlet over
    a fixed time shrinks ~4x when dt halves."""
    sys_ = _sys()
    q, x, v = _small_state()
    amp = {}
    for dt, n in ((0.004, 10), (0.002, 20)):
        _, _, _, es = O.md(sys_, q, x, v, 0.0, 0, None, n, dt)
        E = _etot(es)
        f0, e0 = O.forces(sys_, q, O.wrap(x, sys_.L))
        E0 = e0["U_near"] + e0["U_far"] - e0["U_self"] + e0["U_wca"] + 0.5 * np.sum(v * v)
        amp[dt] = np.max(np.abs(E - E0))
    assert amp[0.004] / amp[0.002] == pytest.approx(4.0, rel=0.3)


def test_time_reversible():
    """Forward n steps, flip v, n steps with the k-sets in reverse order
    returns to the start (random-batch far field)."""
    sys_ = _sys()
    q, x, v = _small_state()
    S = sys_.S()
    P, n = 20, 6
    ks = O.kseq(sys_.sog, sys_.L, seed=5, n_chains=1, chain_len=P * (n + 1)).reshape(n + 1, P, 3)
    x1, v1, f1, _ = O.md(sys_, q, x, v, S, P, ks.reshape(-1, 3), n, 0.002)
    # backward: start with the force of the last k-set at x1, then use k-sets n-1 .. 0
    back = ks[::-1][1:].reshape(-1, 3)
    x2, v2, _, _ = O.md(sys_, q, x1, -v1, S, P, back, n, 0.002, f=f1)
    dx = x2 - O.wrap(x, sys_.L)
    dx -= sys_.L * np.rint(dx / sys_.L)
    assert np.max(np.abs(dx)) < 1e-11
    assert np.max(np.abs(v2 + v)) < 1e-10


def test_berendsen_relaxes_temperature():
    """v <- v sqrt(1 + dt/tau (T0/T - 1)) pulls T toward T0 at rate 1/tau."""
    sys_ = _sys()
    q, x, v = _small_state()
    v = v * math.sqrt(3.0)          # start near T = 3
    S = sys_.S()
    P, n = 10, 5
    ks = O.kseq(sys_.sog, sys_.L, seed=1, n_chains=1, chain_len=P * (n + 1))
    _, _, _, es = O.md(sys_, q, x, v, S, P, ks, n, 0.002, T0=1.0, tau=0.004)
    T = [e["T"] for e in es]
    assert T[-1] < T[0] < 3.2
    assert T[-1] < 1.6


def test_kseq_consumed_one_set_per_force():
    """Force evaluation t uses entries [tP, (t+1)P) of the sequence: a run
    split in two with the force carried over equals the run in one piece."""
    sys_ = _sys()
    q, x, v = _small_state()
    S = sys_.S()
    P = 16
    ks = O.kseq(sys_.sog, sys_.L, seed=9, n_chains=2, chain_len=P * 3)   # 6 sets
    xa, va, fa, _ = O.md(sys_, q, x, v, S, P, ks, 5, 0.002)
    xb, vb, fb, _ = O.md(sys_, q, x, v, S, P, ks[:3 * P], 2, 0.002)
    xc, vc, fc, _ = O.md(sys_, q, xb, vb, S, P, ks[3 * P:], 3, 0.002, f=fb)
    assert np.array_equal(xa, xc) and np.array_equal(va, vc) and np.array_equal(fa, fc)
