"""Appendix A observables on the device against the oracle: MSD and VACF
over time origins (FP64 MD sampled every two steps; free flight across many
box crossings against the ballistic closed form), the pressure tensor, and
the Green-Kubo autocorrelation and integral of a pressure series (host and
device input)."""
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


def test_msd_vacf_match_oracle_trajectory():
    Pk, dev = _setup()
    N, L, P, every, n_samp, n_lags, every_o = 1000, 12.6, 32, 2, 12, 6, 2
    q, x, v = I.electrolyte(N, L, seed=51)
    sog = prod_sog(O)
    steps = every * (n_samp - 1)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=steps + 1, seed=4,
                       precision="fp64")
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    ks = oracle_kseq(O, g, sog, L, 4, steps + 1)
    g.observe_start(n_lags, every_o)
    g.observe_sample()
    for _ in range(n_samp - 1):
        g.step(every)
        g.observe_sample()
    msd, vacf, cnt = g.observe_result()
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    xo, vo, fo = O.wrap(x, s.L), v.copy(), None
    xs, vs = [xo], [vo]
    used = 0
    for c in range(n_samp - 1):
        k0 = used * P
        xo, vo, fo, _ = O.md(s, q, xo, vo, s.S(), P, ks[k0:], every, p.dt, f=fo)
        used += every + (1 if c == 0 else 0)
        xs.append(xo)
        vs.append(vo)
    mo, vco, co = O.msd_vacf(np.stack(xs), np.stack(vs), s.L, n_lags, origin_every=every_o)
    assert np.array_equal(cnt, co)
    assert np.allclose(msd[1:], mo[1:], rtol=1e-8, atol=0)
    assert msd[0] == 0.0
    assert np.allclose(vacf, vco, rtol=1e-9, atol=0)


@pytest.mark.parametrize("every_o", [1, 3])
def test_free_flight_msd_is_ballistic(every_o):
    Pk, dev = _setup()
    N, L, dt, per = 2000, 15.874, 0.01, 5
    rng = np.random.default_rng(9)
    q, x, _ = I.electrolyte(N, L, seed=52)
    v = np.clip(rng.normal(0.0, 30.0, (N, 3)), -100.0, 100.0)    # < L/2 per sample, many crossings
    p = Pk.make_params(L, 16, lB=0.0, wca_sigma=0.0, wca_eps=0.0, dt=dt, n_ksets=300, precision="fp64")
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    n_lags = 12
    g.observe_start(n_lags, every_o)
    g.observe_sample()
    for _ in range(30):
        g.step(per)
        g.observe_sample()
    msd, vacf, cnt = g.observe_result()
    g.close()
    v2 = float(np.mean(np.sum(v * v, axis=1)))
    t = np.arange(n_lags) * per * dt
    assert np.allclose(msd, v2 * t * t, rtol=1e-9, atol=1e-12)
    assert np.allclose(vacf, v2, rtol=1e-12)
    assert list(cnt) == [len(range(0, 31 - lag, every_o)) for lag in range(n_lags)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-6)])
def test_pressure_matches_oracle(prec, tol):
    Pk, dev = _setup()
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=53)
    sog = prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=2, seed=3, precision=prec,
                       mass=1.3)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    m = O.kseq(sog, (L,) * 3, seed=7, n_chains=1, chain_len=P)[:P]
    Pt = g.pressure(m)
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    Po = O.pressure(s, q, O.wrap(x, s.L), v, 1.3, s.S(), m)
    assert np.linalg.norm(Pt - Po) <= tol * np.linalg.norm(Po), (Pt, Po)
    assert np.array_equal(Pt, Pt.T)


@pytest.mark.parametrize("on_device", [False, True])
def test_green_kubo_matches_oracle(on_device):
    Pk, dev = _setup()
    rng = np.random.default_rng(10)
    n, lag = 5000, 400
    Pt = np.zeros((n, 3, 3))
    e = rng.normal(0, 1, (n, 3, 3))
    for s in range(1, n):
        Pt[s] = 0.95 * Pt[s - 1] + e[s]
    Pt = 0.5 * (Pt + Pt.transpose(0, 2, 1)) + 3.0 * np.eye(3)
    ser = torch.tensor(Pt.reshape(n, 9), device=dev) if on_device else Pt
    acf, Cg = Pk.binding.rbsog_green_kubo(ser, 0.005, 812.0, 1.1, lag)
    acf_o, Co = O.green_kubo(Pt, 0.005, 812.0, 1.1, lag)
    assert np.allclose(acf, acf_o, rtol=1e-10, atol=1e-12 * abs(acf_o[0]))
    assert Cg == pytest.approx(Co, rel=1e-10)


def test_observer_argument_checks():
    Pk, dev = _setup()
    B = Pk.binding
    q, x, v = I.electrolyte(1000, 12.6, seed=54)
    g = Pk.RBSOG(1000, Pk.make_params(12.6, 16, n_ksets=3), device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    with pytest.raises(B.RBSOGError):
        B.rbsog_observe_sample(g.ctx)              # before start
    with pytest.raises(B.RBSOGError):
        g.observe_start(0, 1)
    with pytest.raises(B.RBSOGError):
        g.observe_start(65, 1)                     # more than 64 origins kept
    g.observe_start(64, 1)
    g.observe_sample()
    msd, vacf, cnt = g.observe_result()
    assert cnt[0] == 1 and cnt[1:].sum() == 0 and msd[0] == 0.0
    g.close()
    with pytest.raises(B.RBSOGError):
        B.rbsog_green_kubo(np.zeros((10, 9)), 0.1, 1.0, 1.0, 11)


def test_observables_need_a_single_system():
    Pk, dev = _setup()
    B = Pk.binding
    systems = [(1000, 12.6), (2000, 15.874)]
    params = [Pk.make_params(L, 16, n_ksets=3, seed=5 + i) for i, (_, L) in enumerate(systems)]
    b = Pk.Batch([N for N, _ in systems], params, device=0)
    for i, (N, L) in enumerate(systems):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in I.electrolyte(N, L, seed=90 + i)))
    with pytest.raises(B.RBSOGError):
        B.rbsog_observe_start(b.ctx, 8, 1)
    with pytest.raises(B.RBSOGError):
        B.rbsog_compute_pressure(b.ctx, np.ones((16, 3), dtype=np.int32))
    b.close()
