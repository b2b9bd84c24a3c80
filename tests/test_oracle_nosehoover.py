"""Pins of the oracle's Nose-Hoover thermostat (symmetric Trotter splitting,
thermostat mass Q = g T0 tau^2, g = 3N - 3): a force-free system follows the
continuous Nose-Hoover equations for (K, xi, eta), integrated here by scipy,
to second order in dt; an interacting fluid conserves U + K + U_th with a
drift that falls as dt^2; a large thermostat mass gives velocity Verlet; and
the kinetic temperature settles at the bath temperature."""
import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog


def _free(n, L, seed):
    rng = np.random.default_rng(seed)
    q = np.zeros(n)
    x = rng.uniform(0, L, (n, 3))
    v = rng.normal(0, 1, (n, 3))
    s = O.System((L,) * 3, prod_sog(O), 3.0, 1.0, 0.0, 0.0)    # no forces
    return q, x, v, s


def _nh_ode(K0, g, T0, Q, t_end, t_eval):
    from scipy.integrate import solve_ivp

    def rhs(_, y):
        K, xi, _eta = y
        return [-2.0 * xi * K, (2.0 * K - g * T0) / Q, xi]

    r = solve_ivp(rhs, (0.0, t_end), [K0, 0.0, 0.0], t_eval=t_eval, rtol=1e-12, atol=1e-12, method="DOP853")
    return r.y


def test_force_free_system_follows_the_nose_hoover_equations():
    n, m, T0, tau = 200, 1.5, 2.0, 0.3
    q, x, v, s = _free(n, 15.0, 8)
    g = 3.0 * n - 3.0
    Q = g * T0 * tau * tau
    K0 = 0.5 * m * float(np.sum(v * v))
    t_end = 2.0
    errs = []
    for dt in (0.02, 0.01):
        nst = int(round(t_end / dt))
        _, v1, _, es = O.md(s, q, x, v, 1.0, 1, np.ones((nst + 1, 3)), nst, dt, mass=m, T0=T0, tau=tau,
                            thermostat=2)
        t = dt * np.arange(1, nst + 1)            # each step advances the thermostat by dt
        K_ode, xi_ode, eta_ode = _nh_ode(K0, g, T0, Q, t_end, t)
        K = np.array([e["K"] for e in es])
        Uth = np.array([e["U_th"] for e in es])
        Uth_ode = 0.5 * Q * xi_ode ** 2 + g * T0 * eta_ode
        errs.append(max(np.abs(K - K_ode).max(), np.abs(Uth - Uth_ode).max()) / K0)
        # velocities are one common factor times the initial ones
        lam = v1[0, 0] / v[0, 0]
        assert np.allclose(v1, lam * v, rtol=1e-12, atol=0)
        assert 0.5 * m * float(np.sum(v1 * v1)) == pytest.approx(K[-1], rel=1e-12)
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0, errs          # second order


def _wca_fluid(N, L, seed):
    qe, x, v = I.electrolyte(N, L, seed=seed)
    s = O.System((L,) * 3, prod_sog(O), 3.0, 1.0, 1.0, 1.0)
    return np.zeros(N), O.wrap(x, s.L), v, s


def test_extended_energy_is_conserved_to_second_order():
    N, L = 512, 10.0
    q, x, v, s = _wca_fluid(N, L, 31)
    drift = []
    for dt in (0.004, 0.002):
        nst = int(round(0.4 / dt))
        _, _, _, es = O.md(s, q, x, v, 1.0, 1, np.ones((nst + 1, 3)), nst, dt, T0=1.6, tau=0.05, thermostat=2)
        H = np.array([e["U_wca"] + e["K"] + e["U_th"] for e in es])
        K = np.array([e["K"] for e in es])
        assert K.max() - K.min() > 0.05 * K[0]            # the thermostat does work
        drift.append(np.abs(H - H[0]).max() / K[0])
    assert drift[0] < 2e-3, drift
    assert drift[0] / drift[1] > 2.5, drift


def test_large_thermostat_mass_is_velocity_verlet():
    N, L = 1000, 12.6
    qe, xe, ve = I.electrolyte(N, L, seed=4)
    sog = prod_sog(O)
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    P = 32
    ks = O.kseq(sog, s.L, seed=2, n_chains=1, chain_len=6 * P)[:6 * P]
    xa, va, _, _ = O.md(s, qe, xe, ve, s.S(), P, ks, 5, 0.002)
    xb, vb, _, eb = O.md(s, qe, xe, ve, s.S(), P, ks, 5, 0.002, T0=1.0, tau=1e9, thermostat=2)
    d = xa - xb
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-9
    assert abs(eb[-1]["U_th"]) < 1e-6


def test_temperature_settles_at_the_bath_temperature():
    N, L = 512, 10.0
    q, x, v, s = _wca_fluid(N, L, 33)                  # T = 1
    nst = 1500
    _, _, _, es = O.md(s, q, x, v, 1.0, 1, np.ones((nst + 1, 3)), nst, 0.004, T0=1.8, tau=0.05, thermostat=2)
    T = np.array([e["T"] for e in es])
    assert abs(T[nst // 2:].mean() - 1.8) < 0.05, T[nst // 2:].mean()
