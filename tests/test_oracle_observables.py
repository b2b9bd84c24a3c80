"""Pins of the oracle's Appendix A observables: MSD and VACF of free
particles are the ballistic closed forms (through many boundary crossings);
the time-origin set and normalisation match closed forms for polynomial
trajectories; the VACF of force-free Langevin dynamics decays as c1^t; the
pressure tensor of an ideal gas is the kinetic tensor over V and otherwise
adds the pinned virial; the Green-Kubo autocorrelation equals numpy's FFT
(Wiener-Khinchin) autocorrelation and its trapezoid integral."""
import math

import numpy as np
import pytest

import oracle as O
from tests._util import prod_sog


def test_free_particles_are_ballistic_across_the_boundary():
    rng = np.random.default_rng(3)
    n, F, L, dts = 400, 40, np.array([7.0, 9.0, 11.0]), 0.5
    r0 = rng.uniform(0, 1, (n, 3)) * L
    v = rng.normal(0, 1.5, (n, 3))                # up to ~0.7 L per frame: many crossings, all < L/2
    v = np.clip(v, -0.45 * L.min() / dts, 0.45 * L.min() / dts)
    xs = np.stack([O.wrap(r0 + v * (f * dts), L) for f in range(F)])
    vs = np.broadcast_to(v, (F, n, 3)).copy()
    msd, vacf, cnt = O.msd_vacf(xs, vs, L, 25, origin_every=3)
    v2 = float(np.mean(np.sum(v * v, axis=1)))
    t = np.arange(25) * dts
    assert np.allclose(msd, v2 * t * t, rtol=1e-10, atol=1e-10)
    assert np.allclose(vacf, v2, rtol=1e-12)
    assert list(cnt) == [len(range(0, F - lag, 3)) for lag in range(25)]


def test_origin_set_and_normalisation_on_polynomial_paths():
    rng = np.random.default_rng(4)
    n, F, n_lags, every = 30, 11, 6, 3
    a = rng.uniform(-1e-3, 1e-3, n)
    c = rng.normal(0, 1, n)
    xs = np.zeros((F, n, 3))
    vs = np.zeros((F, n, 3))
    for f in range(F):
        xs[f, :, 0] = 50.0 + a * f * f           # inside the box, no wrap
        vs[f, :, 1] = c * (f + 1)
    msd, vacf, cnt = O.msd_vacf(xs, vs, 100.0, n_lags, origin_every=every)
    for lag in range(n_lags):
        origins = [o for o in range(0, F, every) if o + lag < F]
        assert cnt[lag] == len(origins)
        m_ref = np.mean(a * a) * np.mean([(2 * o * lag + lag * lag) ** 2 for o in origins])
        v_ref = np.mean(c * c) * np.mean([(o + 1) * (o + lag + 1) for o in origins])
        assert msd[lag] == pytest.approx(m_ref, rel=1e-12, abs=1e-300)
        assert vacf[lag] == pytest.approx(v_ref, rel=1e-12)


def test_force_free_langevin_vacf_decays_geometrically():
    rng = np.random.default_rng(5)
    n, L = 4000, 40.0
    q = np.zeros(n)
    x = rng.uniform(0, L, (n, 3))
    T0, m, dt, tau = 1.3, 1.0, 0.05, 0.5
    v = rng.normal(0, math.sqrt(T0 / m), (n, 3))
    s = O.System((L,) * 3, prod_sog(O), 3.0, 1.0, 0.0, 0.0)
    xs, vs = [x], [v]
    for t in range(12):
        x, v, _, _ = O.md(s, q, x, v, 1.0, 1, np.ones((2, 3)), 1, dt, mass=m, T0=T0, tau=tau, thermostat=1,
                          seed=9, step0=t)
        xs.append(x)
        vs.append(v)
    _, vacf, _ = O.msd_vacf(np.stack(xs), np.stack(vs), L, 8, origin_every=1)
    c1 = math.exp(-dt / tau)
    ref = 3 * T0 / m * c1 ** np.arange(8)
    assert np.allclose(vacf, ref, rtol=0, atol=0.03 * ref[0])


def test_pressure_is_kinetic_plus_virial():
    rng = np.random.default_rng(6)
    n, L, m = 200, 10.0, 1.7
    q = np.zeros(n)
    x = rng.uniform(0, L, (n, 3))
    v = rng.normal(0, 1, (n, 3))
    s0 = O.System((L,) * 3, prod_sog(O), 3.0, 1.0, 0.0, 0.0)      # ideal gas
    Pt = O.pressure(s0, q, x, v, m, 0.0, np.ones((1, 3)))
    assert np.allclose(Pt, m * v.T @ v / L ** 3, rtol=1e-13, atol=0)
    import rbsog_inputs as I
    qe, xe, ve = I.electrolyte(1000, 12.6, seed=7)
    sog = prod_sog(O)
    s = O.System((12.6,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    ks = O.kseq(sog, s.L, seed=2, n_chains=1, chain_len=32)[:32]
    xe = O.wrap(xe, s.L)
    Pt = O.pressure(s, qe, xe, ve, 1.0, s.S(), ks)
    W = O.virial(s, qe, xe, s.S(), ks)
    assert np.allclose(Pt * 12.6 ** 3 - ve.T @ ve, W, rtol=1e-12, atol=1e-9)


def test_green_kubo_matches_fft_autocorrelation():
    rng = np.random.default_rng(8)
    n, lag, dt, V, T = 600, 50, 0.01, 123.0, 1.4
    # a correlated series: AR(1) per component with distinct means
    Pt = np.zeros((n, 3, 3))
    e = rng.normal(0, 1, (n, 3, 3))
    for s in range(1, n):
        Pt[s] = 0.9 * Pt[s - 1] + e[s]
    Pt += np.arange(9).reshape(3, 3)
    acf, Cv = O.green_kubo(Pt, dt, V, T, lag)
    ref = np.zeros(lag)
    for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]:
        y = Pt[:, a, b] - Pt[:, a, b].mean()
        fy = np.fft.rfft(y, 2 * n)
        r = np.fft.irfft(fy * np.conj(fy), 2 * n)[:lag]
        ref += r / (n - np.arange(lag))
    assert np.allclose(acf, ref, rtol=1e-10, atol=1e-12)
    assert Cv == pytest.approx(V / (6 * T) * dt * (ref.sum() - 0.5 * (ref[0] + ref[-1])), rel=1e-10)
