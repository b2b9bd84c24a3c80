"""Pins of the oracle's Langevin dynamics (BAOAB splitting; the paper's
theory uses Langevin dynamics, Sec. 4): the noise is numpy's Philox4x64-10
block for the documented key and counter through Box-Muller; one step of a
force-free system is exactly v' = c1 v + c2 z; a force-free system relaxes
to the Maxwell velocity variance T0/m; and vanishing friction gives
velocity Verlet."""
import math

import numpy as np
import pytest

import oracle as O
from tests._util import prod_sog

KEY1 = 2 ** 63 + 1


def _numpy_noise(seed, t, i):
    # numpy's Philox with counter c emits the block for counter c + 1
    bg = np.random.Philox(counter=np.array([t - 1 if t > 0 else 2 ** 64 - 1, i if t > 0 else i - 1, 0, 0],
                                           dtype=np.uint64),
                          key=np.array([seed, KEY1], dtype=np.uint64))
    r = [int(v) for v in bg.random_raw(4)]
    u = [(v >> 11) / 2.0 ** 53 for v in r]
    r01 = math.sqrt(-2.0 * math.log(1.0 - u[0]))
    r23 = math.sqrt(-2.0 * math.log(1.0 - u[2]))
    return np.array([r01 * math.cos(2 * math.pi * u[1]), r01 * math.sin(2 * math.pi * u[1]),
                     r23 * math.cos(2 * math.pi * u[3])])


@pytest.mark.parametrize("seed,t,i", [(7, 1, 0), (123456789, 5, 999), (2 ** 40 + 3, 17, 12345)])
def test_noise_is_philox_through_box_muller(seed, t, i):
    assert np.allclose(O.langevin_noise(seed, t, i), _numpy_noise(seed, t, i), rtol=0, atol=1e-14)


def _free(n, L, seed):
    rng = np.random.default_rng(seed)
    q = np.zeros(n)
    x = rng.uniform(0, L, (n, 3))
    v = rng.normal(0, 1, (n, 3))
    sog = prod_sog(O)
    s = O.System((L,) * 3, sog, 3.0, 1.0, 0.0, 0.0)    # no charges, no WCA: no forces
    return q, x, v, s


def test_one_force_free_step_is_the_ou_update():
    q, x, v, s = _free(50, 12.0, 3)
    dt, tau, T0, m, seed, step0 = 0.01, 0.2, 1.3, 2.0, 99, 41
    x1, v1, _, _ = O.md(s, q, x, v, 1.0, 1, np.ones((2, 3)), 1, dt, mass=m, T0=T0, tau=tau, thermostat=1,
                        seed=seed, step0=step0)
    c1 = math.exp(-dt / tau)
    c2 = math.sqrt((1 - c1 * c1) * T0 / m)
    z = np.array([_numpy_noise(seed, step0, i) for i in range(len(q))])
    v_ref = c1 * v + c2 * z
    assert np.allclose(v1, v_ref, rtol=0, atol=1e-13)
    x_ref = O.wrap(x + 0.5 * dt * v + 0.5 * dt * v_ref, s.L)
    d = x1 - x_ref
    d -= s.L[0] * np.round(d / s.L[0])
    assert np.abs(d).max() < 1e-12


def test_force_free_velocities_relax_to_maxwell():
    q, x, v, s = _free(3000, 40.0, 5)
    v = 3.0 * v                                          # start far from T0
    T0, m = 1.5, 1.0
    _, v1, _, es = O.md(s, q, x, v, 1.0, 1, np.ones((401, 3)), 400, 0.01, mass=m, T0=T0, tau=0.1, thermostat=1,
                        seed=11)
    var = np.mean(v1 ** 2)
    assert var == pytest.approx(T0 / m, rel=0.03)
    assert es[-1]["T"] == pytest.approx(T0, rel=0.03)


def test_vanishing_friction_is_velocity_verlet():
    import rbsog_inputs as I
    N, L = 1000, 12.6
    qe, xe, ve = I.electrolyte(N, L, seed=4)
    sog = prod_sog(O)
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    P = 32
    ks = O.kseq(sog, s.L, seed=2, n_chains=1, chain_len=6 * P)[:6 * P]
    xa, va, _, _ = O.md(s, qe, xe, ve, s.S(), P, ks, 5, 0.002)
    xb, vb, _, _ = O.md(s, qe, xe, ve, s.S(), P, ks, 5, 0.002, tau=1e15, thermostat=1, seed=1)
    d = xa - xb
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-9
