"""Langevin dynamics (BAOAB; Philox noise keyed by seed and step counter) on
the device against the oracle: trajectories agree step by step (FP64 to
1e-10; FP32C, whose noise is drawn in FP32, to FP32 level), a system gives
the same bits alone and in a batch, and the kinetic temperature relaxes to
the bath temperature."""
import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import oracle_kseq, prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _params(Pk, L, P, prec, n_ksets, seed=5, tau=0.05, T0=1.5, dt=0.002):
    sog = prod_sog(O)
    return Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=n_ksets, seed=seed,
                          precision=prec, tau_T=tau, T_target=T0, dt=dt, thermostat="langevin"), sog


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 2e-6)])
def test_langevin_trajectory_matches_oracle(prec, tol):
    Pk, dev = _setup()
    N, L, P, steps = 1000, 12.6, 32, 5
    q, x, v = I.electrolyte(N, L, seed=21)
    p, sog = _params(Pk, L, P, prec, steps + 1)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    ks = oracle_kseq(O, g, sog, L, p.seed, steps + 1)
    g.step(steps)
    xg, vg, _, st = g.state()
    assert st == steps
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    xo, vo, _, es = O.md(s, q, O.wrap(x, s.L), v, s.S(), P, ks, steps, 0.002, T0=1.5, tau=0.05, thermostat=1,
                         seed=p.seed, step0=0)
    d = xg.cpu().numpy() - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= tol * L
    assert np.linalg.norm(vg.cpu().numpy() - vo) <= tol * 10 * np.linalg.norm(vo)


def test_langevin_system_same_alone_and_in_a_batch():
    Pk, dev = _setup()
    systems = [(1000, 12.6), (2000, 15.874)]
    params = [_params(Pk, L, 64, "fp32c", 12, seed=40 + i)[0] for i, (N, L) in enumerate(systems)]
    states = [I.electrolyte(N, L, seed=60 + i) for i, (N, L) in enumerate(systems)]
    b = Pk.Batch([N for N, _ in systems], params, device=0)
    for i, st in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in st))
    b.step(8)
    for i, (N, L) in enumerate(systems):
        g = Pk.RBSOG(N, params[i], device=0)
        g.set_state(*(torch.tensor(a, device=dev) for a in states[i]))
        g.step(8)
        for u, w in zip(g.state()[:3], b.state(i)[:3]):
            assert torch.equal(u, w)
        g.close()
    b.close()


def test_langevin_temperature_relaxes_to_the_bath():
    Pk, dev = _setup()
    N, L = 4998, 21.5
    q, x, v = I.electrolyte(N, L, seed=22)             # T = 1
    p, _ = _params(Pk, L, 64, "fp32c", 302, tau=0.02, T0=2.0, dt=0.001)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    temps = []
    for _ in range(6):
        g.step(50)
        temps.append(g.energies()["T"])
    g.close()
    assert abs(np.mean(temps[3:]) - 2.0) < 0.1, temps
