"""Serving engine: jobs of uneven size and length, submitted at different
times into a server with fewer slots than jobs, each finish with exactly the
trajectory they follow when run alone (same parameters and seed), whatever
joined or left the batch while they ran."""
import numpy as np
import pytest

import rbsog_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (N, L, lB, seed, steps)
JOBS = [(1000, 12.6, 0.7, 3, 9), (4998, 21.5, 1.5, 4, 5), (2000, 15.874, 1.0, 5, 13),
        (10648, 27.7, 1.2, 6, 7), (1000, 12.6, 1.0, 7, 3), (3456, 18.9, 0.9, 8, 11)]


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _params(Pk, L, lB, seed, prec, steps, tau=0.0):
    return Pk.make_params(L, 64, lB=lB, seed=seed, n_ksets=steps + 1, precision=prec, tau_T=tau, T_target=1.0)


def _alone(Pk, dev, job, p, state):
    N = job[0]
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in state))
    g.step(job[4])
    x, v, f, step = (a.cpu().numpy() if hasattr(a, "cpu") else a for a in g.state())
    e = g.energies()
    g.close()
    return x, v, f, e, step


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_served_jobs_equal_alone_bitwise(prec):
    Pk, dev = _setup()
    states = [I.electrolyte(j[0], j[1], seed=500 + i) for i, j in enumerate(JOBS)]
    params = [_params(Pk, j[1], j[2], j[3], prec, j[4], tau=0.05 if i % 3 == 1 else 0.0)
              for i, j in enumerate(JOBS)]
    srv = Pk.Server(max_jobs=3, mem_budget_bytes=8 << 30, quantum=4, device=0)
    ids = [srv.submit(params[i], *states[i], nsteps=JOBS[i][4]) for i in range(4)]
    peak_active = 0
    rounds = 0
    while True:
        act, wait, _ = srv.advance()
        peak_active = max(peak_active, act)
        rounds += 1
        if rounds == 2:     # late arrivals join a running batch
            ids += [srv.submit(params[i], *states[i], nsteps=JOBS[i][4]) for i in range(4, len(JOBS))]
        if rounds > 2 and act == 0 and wait == 0:
            break
        assert rounds < 100
    assert peak_active == 3
    for i, jid in enumerate(ids):
        st, x, v, f, e, steps = srv.result(jid)
        assert st == 2 and steps == JOBS[i][4]
        xa, va, fa, ea, sa = _alone(Pk, dev, JOBS[i], params[i], states[i])
        assert sa == steps
        for a, b in ((xa, x), (va, v), (fa, f)):
            assert np.array_equal(a, b), (prec, i)
        assert ea == e, (prec, i)
        srv.release(jid)
    srv.close()


def test_server_memory_budget_limits_admission():
    """A budget that holds one job at a time serialises the queue (FIFO)."""
    Pk, dev = _setup()
    jobs = [JOBS[0], JOBS[4]]
    states = [I.electrolyte(j[0], j[1], seed=600 + i) for i, j in enumerate(jobs)]
    params = [_params(Pk, j[1], j[2], j[3], "fp32c", j[4]) for j in jobs]
    # footprint of one 1000-particle, 64-frequency job is well under 4 MiB
    srv = Pk.Server(max_jobs=8, mem_budget_bytes=int(0.75 * 2 * 1000 * 256 + 2 * 64 * 4096), quantum=2,
                    device=0)
    ids = [srv.submit(params[i], *states[i], nsteps=jobs[i][4]) for i in range(2)]
    seen = []
    for _ in range(50):
        act, wait, _ = srv.advance()
        seen.append((act, wait))
        if act == 0 and wait == 0:
            break
    assert max(a for a, _ in seen) == 1
    assert seen[0] == (1, 1)
    for i, jid in enumerate(ids):
        st, x, *_ = srv.result(jid)
        assert st == 2
        xa = _alone(Pk, dev, jobs[i], params[i], states[i])[0]
        assert np.array_equal(xa, x)
    srv.close()


def test_server_rejects_invalid_jobs():
    Pk, dev = _setup()
    B = Pk.binding
    q, x, v = I.electrolyte(1000, 12.6, seed=1)
    p = _params(Pk, 12.6, 1.0, 1, "fp32c", 5)
    srv = Pk.Server(max_jobs=2, mem_budget_bytes=1 << 20, quantum=2, device=0)
    with pytest.raises(B.RBSOGError):
        srv.submit(p, q, x, v, nsteps=0)
    big = I.electrolyte(64000, 50.4, seed=2)
    with pytest.raises(B.RBSOGError):
        srv.submit(_params(Pk, 50.4, 1.0, 1, "fp32c", 5), *big, nsteps=5)
    p_other = _params(Pk, 12.6, 1.0, 1, "fp32c", 5)
    p_other.P = 32                                 # the server's jobs share P (set by the first job)
    jid = srv.submit(p, q, x, v, nsteps=5)
    with pytest.raises(B.RBSOGError):
        srv.submit(p_other, q, x, v, nsteps=5)
    assert srv.result(jid)[0] == 0
    with pytest.raises(B.RBSOGError):
        srv.release(jid)           # not finished
    for _ in range(20):
        srv.advance()
        if srv.result(jid)[0] == 2:
            break
    assert srv.result(jid)[0] == 2
    srv.release(jid)
    srv.close()


def test_server_cancel_waiting_and_running():
    """Cancelling a waiting job drops it from the queue; cancelling a running
    job freezes it at once; the other jobs still finish with their alone
    trajectories."""
    Pk, dev = _setup()
    B = Pk.binding
    jobs = [JOBS[0], JOBS[2], JOBS[4]]
    states = [I.electrolyte(j[0], j[1], seed=700 + i) for i, j in enumerate(jobs)]
    params = [_params(Pk, j[1], j[2], j[3], "fp32c", j[4]) for j in jobs]
    srv = Pk.Server(max_jobs=2, mem_budget_bytes=8 << 30, quantum=2, device=0)
    ids = [srv.submit(params[i], *states[i], nsteps=jobs[i][4]) for i in range(3)]
    act, wait, _ = srv.advance()             # jobs 0 and 1 run, job 2 waits
    assert (act, wait) == (2, 1)
    srv.cancel(ids[2])                        # waiting
    srv.cancel(ids[1])                        # running
    assert srv.result(ids[1])[0] == 3 and srv.result(ids[2])[0] == 3
    with pytest.raises(B.RBSOGError):
        srv.cancel(ids[1])
    for _ in range(50):
        act, wait, _ = srv.advance()
        if act == 0 and wait == 0:
            break
    st, x, *_ = srv.result(ids[0])
    assert st == 2
    assert np.array_equal(x, _alone(Pk, dev, jobs[0], params[0], states[0])[0])
    for jid in ids:
        srv.release(jid)
    srv.close()


@pytest.mark.parametrize("thermostat", ["langevin", "nose-hoover"])
def test_served_thermostatted_jobs_equal_alone(thermostat):
    """Langevin noise (keyed by the step counter) and the Nose-Hoover
    variables (kept with the energies) move with a job when the server
    re-batches it: each job still ends with its alone trajectory."""
    Pk, dev = _setup()
    jobs = [JOBS[0], JOBS[2], JOBS[4], JOBS[5]]
    states = [I.electrolyte(j[0], j[1], seed=800 + i) for i, j in enumerate(jobs)]
    params = []
    for j in jobs:
        p = _params(Pk, j[1], j[2], j[3], "fp32c", j[4], tau=0.05)
        p.thermostat = {"langevin": 1, "nose-hoover": 2}[thermostat]
        params.append(p)
    srv = Pk.Server(max_jobs=2, mem_budget_bytes=8 << 30, quantum=3, device=0)
    ids = [srv.submit(params[i], *states[i], nsteps=jobs[i][4]) for i in range(len(jobs))]
    for _ in range(100):
        act, wait, _ = srv.advance()
        if act == 0 and wait == 0:
            break
    for i, jid in enumerate(ids):
        st, x, v, f, e, steps = srv.result(jid)
        assert st == 2 and steps == jobs[i][4]
        xa, va, fa, ea, sa = _alone(Pk, dev, jobs[i], params[i], states[i])
        for a, b in ((xa, x), (va, v), (fa, f)):
            assert np.array_equal(a, b), (thermostat, i)
        assert ea == e, (thermostat, i)
        srv.release(jid)
    srv.close()
