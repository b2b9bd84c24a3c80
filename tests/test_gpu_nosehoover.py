"""Nose-Hoover dynamics on the device against the oracle: trajectories and
the thermostat energy U_th agree step by step (FP64 to 1e-10, FP32C to FP32
level), the thermostat variables survive a batch and a re-set state starts
them at zero again."""
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
                          precision=prec, tau_T=tau, T_target=T0, dt=dt, thermostat="nose-hoover"), sog


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 2e-6)])
def test_nose_hoover_trajectory_matches_oracle(prec, tol):
    Pk, dev = _setup()
    N, L, P, steps = 1000, 12.6, 32, 6
    q, x, v = I.electrolyte(N, L, seed=23)
    p, sog = _params(Pk, L, P, prec, steps + 1)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    ks = oracle_kseq(O, g, sog, L, p.seed, steps + 1)
    g.step(steps)
    xg, vg, _, st = g.state()
    e = g.energies()
    assert st == steps
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    xo, vo, _, es = O.md(s, q, O.wrap(x, s.L), v, s.S(), P, ks, steps, 0.002, T0=1.5, tau=0.05, thermostat=2)
    d = xg.cpu().numpy() - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= tol * L
    assert np.linalg.norm(vg.cpu().numpy() - vo) <= tol * 10 * np.linalg.norm(vo)
    assert es[-1]["U_th"] != 0.0
    assert abs(e["U_th"] - es[-1]["U_th"]) <= tol * 10 * es[-1]["K"]
    assert e["K"] == pytest.approx(es[-1]["K"], rel=tol * 10)


def test_nose_hoover_state_in_a_batch_and_reset():
    Pk, dev = _setup()
    systems = [(1000, 12.6), (2000, 15.874)]
    params = [_params(Pk, L, 64, "fp32c", 40, seed=40 + i, T0=1.2 + 0.5 * i)[0] for i, (N, L) in
              enumerate(systems)]
    states = [I.electrolyte(N, L, seed=70 + i) for i, (N, L) in enumerate(systems)]
    b = Pk.Batch([N for N, _ in systems], params, device=0)
    for i, st in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in st))
    b.step(4)
    b.step(4)                       # the thermostat state carries across calls
    for i, (N, L) in enumerate(systems):
        g = Pk.RBSOG(N, params[i], device=0)
        g.set_state(*(torch.tensor(a, device=dev) for a in states[i]))
        g.step(8)
        for u, w in zip(g.state()[:3], b.state(i)[:3]):
            assert torch.equal(u, w)
        assert g.energies()["U_th"] == b.energies(i)["U_th"] != 0.0
        g.close()
    b.close()


def test_set_state_restarts_the_thermostat():
    """Without Coulomb terms the trajectory does not depend on which k-sets
    are drawn, so a re-set context must repeat a fresh one bit for bit."""
    Pk, dev = _setup()
    N, L = 1000, 12.6
    st = I.electrolyte(N, L, seed=80)
    p, _ = _params(Pk, L, 16, "fp64", 20)
    p.coulomb_prefactor = 0.0
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in st))
    g.step(5)
    assert g.energies()["U_th"] != 0.0
    g.set_state(*(torch.tensor(a, device=dev) for a in st))
    assert g.energies()["U_th"] == 0.0
    g.step(3)
    h = Pk.RBSOG(N, p, device=0)
    h.set_state(*(torch.tensor(a, device=dev) for a in st))
    h.step(3)
    for u, w in zip(g.state()[:3], h.state()[:3]):
        assert torch.equal(u, w)
    assert g.energies()["U_th"] == h.energies()["U_th"]
    g.close()
    h.close()
