"""Pins of the oracle's heat flux and Green-Kubo heat conductivity
(Appendix A).

- Einstein-Helfand: for pair forces (near field + WCA) the heat flux times V
  is the time derivative of the energy moment D = sum_i r_i e_i along the
  Newtonian flow, taken here by central differences of states advanced to
  second order; a dropped 1/2, a reversed r_ij, v_i for v_i + v_j or a
  missing kinetic term each fail it.
- Sum rules: the per-atom energies add up to the total energy of the force
  routine (near, WCA, random-batch far, minus self, plus kinetic) and the
  per-atom virials to the pair-scan virial tensor (near + random-batch far),
  both computed by other oracle functions pinned elsewhere (finite
  differences of the energy).
- Closed forms for two particles (WCA only; an ion pair's far energy on one
  frequency).
- The Green-Kubo autocorrelation equals numpy's FFT autocorrelation summed
  over the three components, and a constant flux gives |J|^2 at every lag."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog


def _cluster(n, L, seed):
    """n ions (+-1) in a ball of radius 3.5 at the box centre, kept 0.9
    apart, with Maxwell velocities at T = 1."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-3.5, 3.5, 3)
        if np.dot(p, p) > 3.5 ** 2:
            continue
        if all(np.dot(p - o, p - o) > 0.81 for o in pts):
            pts.append(p)
    x = np.array(pts) + L / 2
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    v = rng.normal(0, 1, (n, 3))
    return q, x, v


def test_einstein_helfand_near_field():
    """J V = d/dt sum_i r_i e_i for the near-field + WCA dynamics of an
    isolated cluster (no far term, positions never wrap)."""
    sog = prod_sog(O)
    L = 30.0
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    q, x, v = _cluster(24, L, seed=3)
    mass = 1.3
    J, e, W = O.heat_flux(s, q, x, v, mass)
    f, _, _, _ = O.near(s, q, x, "direct")
    a = f / mass

    def D(xx, vv):
        _, ee, _ = O.heat_flux(s, q, xx, vv, mass)
        return np.sum(xx * ee[:, None], axis=0)

    def dD_dt(h):   # central difference over states advanced to second order: O(h^2)
        return (D(x + h * v + 0.5 * h * h * a, v + h * a) - D(x - h * v + 0.5 * h * h * a, v - h * a)) / (2 * h)

    dD = (4.0 * dD_dt(1e-4) - dD_dt(2e-4)) / 3.0      # Richardson: O(h^4)
    V = L ** 3
    assert np.abs(J * V - dD).max() <= 1e-6 * np.abs(dD).max()
    assert np.abs(dD).max() > 1.0           # a non-trivial flux


def test_per_atom_sums_equal_the_totals():
    sog = prod_sog(O)
    N, L, P = 1000, 12.6, 64
    q, x, v = I.electrolyte(N, L, seed=12)
    s = O.System((L,) * 3, sog, 3.0, 1.2, 1.0, 1.0)
    m = O.kseq(sog, s.L, seed=4, n_chains=1, chain_len=P)[:P]
    mass = 1.0
    J, e, W = O.heat_flux(s, q, x, v, mass, S=s.S(), m=m)
    _, en = O.forces(s, q, x, S=s.S(), m=m)
    K = 0.5 * mass * np.sum(v * v)
    U = en["U_near"] + en["U_wca"] + en["U_far"] - en["U_self"]
    assert e.sum() == pytest.approx(U + K, rel=1e-12)
    Wref = O.virial(s, q, x, S=s.S(), m=m)
    assert np.abs(W.sum(0) - Wref).max() <= 1e-11 * np.abs(Wref).max()
    assert np.allclose(W, np.transpose(W, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(W).max())
    # J is the per-atom energies and virials contracted with the velocities
    Jref = (np.sum(e[:, None] * v, axis=0) + np.einsum("iab,ib->a", W, v)) / L ** 3
    assert np.allclose(J, Jref, rtol=1e-12, atol=1e-15)


def test_two_particles_closed_form():
    """Two neutral WCA particles inside the WCA range: J V = sum e_i v_i +
    1/2 (f_12 . (v_1 + v_2)) r_12 with e_i = m v_i^2 / 2 + u(r) / 2."""
    sog = prod_sog(O)
    L = 12.0
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    x = np.array([[5.0, 6.0, 6.0], [6.05, 6.2, 5.9]])
    v = np.array([[0.3, -1.1, 0.7], [-0.4, 0.2, 1.5]])
    q = np.zeros(2)
    J, e, W = O.heat_flux(s, q, x, v, 1.0)
    r = x[0] - x[1]
    r2 = r @ r
    sr6 = (1.0 / r2) ** 3
    u = 4 * (sr6 * sr6 - sr6) + 1.0
    f12 = 24 * (2 * sr6 * sr6 - sr6) / r2 * r
    e_ref = 0.5 * np.sum(v * v, axis=1) + 0.5 * u
    JV = e_ref[0] * v[0] + e_ref[1] * v[1] + 0.5 * (f12 @ (v[0] + v[1])) * r
    assert np.allclose(e, e_ref, rtol=1e-13)
    assert np.allclose(J * L ** 3, JV, rtol=1e-12)


def test_ion_pair_far_energy_on_one_frequency():
    """e_i's far part on one frequency m: (c/2) q_i Re(e^{-i k.r_i} rho)
    = (c/2) q_i (q_i + q_j cos(k.(r_j - r_i))), c = lB pi^{3/2} S / V."""
    sog = prod_sog(O)
    L = 12.0
    lB = 0.8
    s = O.System((L,) * 3, sog, 3.0, lB, 0.0, 0.0)
    x = np.array([[1.0, 2.0, 3.0], [7.5, 8.0, 2.0]])      # beyond r_c: no near pair
    v = np.zeros((2, 3))
    q = np.array([1.0, -1.0])
    m = np.array([[1, 2, -1]], dtype=np.int32)
    S = s.S()
    _, e_far, W_far = O.heat_flux(s, q, x, v, 1.0, S=S, m=m)
    _, e0, _ = O.heat_flux(s, q, x, v, 1.0)
    k = 2 * math.pi * m[0] / L
    c = lB * math.pi ** 1.5 * S / L ** 3
    ref = 0.5 * c * q * (q + q[::-1] * np.cos((x[::-1] - x) @ k))
    assert np.allclose(e_far - e0, ref, rtol=1e-12)


def test_green_kubo_heat_matches_fft_autocorrelation():
    rng = np.random.default_rng(7)
    n, max_lag, dt, V, T = 3000, 200, 0.01, 125.0, 1.7
    J = np.zeros((n, 3))
    for t in range(1, n):                       # an AR(1) flux per component
        J[t] = 0.95 * J[t - 1] + rng.normal(0, 1, 3)
    acf, C = O.green_kubo_heat(J, dt, V, T, max_lag)
    ref = np.zeros(max_lag)
    for c in range(3):
        f = np.fft.rfft(J[:, c], 2 * n)
        full = np.fft.irfft(f * np.conj(f))[:n]
        ref += full[:max_lag] / (n - np.arange(max_lag))
    assert np.allclose(acf, ref, rtol=1e-10)
    integral = dt * (0.5 * ref[0] + ref[1:max_lag - 1].sum() + 0.5 * ref[max_lag - 1])
    assert C == pytest.approx(V / (3 * T * T) * integral, rel=1e-10)
    Jc = np.tile([0.5, -1.0, 2.0], (50, 1))
    acf, C = O.green_kubo_heat(Jc, 0.1, 8.0, 2.0, 10)
    assert np.allclose(acf, 5.25, rtol=1e-14)
    assert C == pytest.approx(8.0 / (3 * 4.0) * 5.25 * 9 * 0.1, rel=1e-13)
