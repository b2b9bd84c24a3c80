"""Batched and served systems against the FP64 oracle, not only against
their own runs alone: every system of an autotuned batch of uneven sizes and
Bjerrum lengths, and a job admitted into a running server, follows the
oracle's velocity-Verlet trajectory (Algorithm 1) on its own k-sequence.

Bars as for a single system: FP64 positions within 1e-11, forces within
1e-10 RMS relative and 1e-9 per particle, energies within 1e-10; FP32C
positions within 1e-6, forces within 1e-4 RMS relative and per particle,
total energy within 1e-5."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import PP_FP32C, PP_FP64, per_particle_rel, prod_sog, rms_rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P = 64
# (N, L, Bjerrum length, seed, Berendsen tau): uneven sizes, l_B over the
# replica workload's range [0.7, 1.5]
SYSTEMS = [(1000, 12.6, 0.7, 3, 0.0), (4998, 21.5, 1.5, 4, 0.05), (2000, 15.874, 1.0, 5, 0.0),
           (10648, 27.7, 1.2, 6, 0.0)]


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _params(Pk, sog, L, lB, seed, prec, nsets, tau):
    return Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, lB=lB, seed=seed,
                          n_ksets=nsets, precision=prec, tau_T=tau, T_target=1.0)


def _oracle_run(sog, N, L, lB, seed, tau, state, steps):
    """The oracle's trajectory on the oracle's own sampling of the k-sequence
    (chains of 256, Philox key (seed, chain)), independent of the device."""
    q, x, v = state
    s = O.System((L,) * 3, sog, 3.0, lB, 1.0, 1.0)
    n_chains = -(-(steps + 1) * P // 256)
    ks = O.kseq(sog, s.L, seed=seed, n_chains=n_chains, chain_len=256)
    return O.md(s, q, x, v, s.S(), P, ks, steps, 0.001, tau=tau)


def _compare(prec, L, got, ref, tag):
    xg, vg, fg, eg = got
    xo, vo, fo, eo = ref
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    err = rms_rel(fg, fo)
    worst = per_particle_rel(fg, fo)[1]
    U = eg["U_near"] + eg["U_far"] - eg["U_self"] + eg["U_wca"]
    Uo = eo["U_near"] + eo["U_far"] - eo["U_self"] + eo["U_wca"]
    if prec == "fp64":
        assert np.abs(dx).max() < 1e-11, tag
        assert np.abs(vg - vo).max() < 1e-9, tag
        assert err < 1e-10 and worst < PP_FP64, (tag, err, worst)
        for k in ("U_near", "U_far", "U_wca", "K"):
            assert eg[k] == pytest.approx(eo[k], rel=1e-10, abs=1e-10), (tag, k)
    else:
        assert np.abs(dx).max() < 1e-6, tag
        assert err < 1e-4 and worst < PP_FP32C, (tag, err, worst)
        assert abs(U - Uo) <= 1e-5 * abs(Uo), tag


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_autotuned_batch_matches_oracle(prec):
    Pk, dev = _setup()
    sog = prod_sog(O)
    steps = 6
    states = [I.electrolyte(N, L, seed=700 + i) for i, (N, L, _, _, _) in enumerate(SYSTEMS)]
    params = [_params(Pk, sog, L, lB, seed, prec, steps + 1, tau) for (N, L, lB, seed, tau) in SYSTEMS]
    b = Pk.Batch([s[0] for s in SYSTEMS], params, device=0)
    for i, st in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in st))
    Pk.binding.rbsog_batch_autotune(b.ctx, 2)
    b.step(steps)
    for i, (N, L, lB, seed, tau) in enumerate(SYSTEMS):
        xg, vg, fg, nstep = b.state(i)
        assert nstep == steps
        got = (xg.cpu().numpy(), vg.cpu().numpy(), fg.cpu().numpy(), b.energies(i))
        xo, vo, fo, es = _oracle_run(sog, N, L, lB, seed, tau, states[i], steps)
        _compare(prec, L, got, (xo, vo, fo, es[-1]), (prec, i))
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_job_admitted_mid_run_matches_oracle(prec):
    """A server with two slots runs job A; job B is submitted after A's first
    quantum and joins the running batch.  Both finish on the oracle's
    trajectory."""
    Pk, dev = _setup()
    sog = prod_sog(O)
    jobs = [(2000, 15.874, 1.2, 31, 0.0, 9), (4998, 21.5, 0.8, 32, 0.05, 5)]   # + steps
    states = [I.electrolyte(j[0], j[1], seed=800 + i) for i, j in enumerate(jobs)]
    params = [_params(Pk, sog, j[1], j[2], j[3], prec, j[5] + 1, j[4]) for j in jobs]
    srv = Pk.Server(max_jobs=2, mem_budget_bytes=8 << 30, quantum=3, device=0)
    ids = [srv.submit(params[0], *states[0], nsteps=jobs[0][5])]
    act, _, _ = srv.advance()
    assert act == 1
    ids.append(srv.submit(params[1], *states[1], nsteps=jobs[1][5]))
    for _ in range(50):
        act, wait, _ = srv.advance()
        if act == 0 and wait == 0:
            break
    for i, jid in enumerate(ids):
        N, L, lB, seed, tau, steps = jobs[i]
        st, x, v, f, e, done = srv.result(jid)
        assert st == 2 and done == steps
        xo, vo, fo, es = _oracle_run(sog, N, L, lB, seed, tau, states[i], steps)
        _compare(prec, L, (x, v, f, e), (xo, vo, fo, es[-1]), (prec, i))
        srv.release(jid)
    srv.close()
