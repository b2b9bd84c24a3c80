"""Batched replicas: independent systems of uneven size advanced by one graph
launch per step give bit-identical trajectories to the same systems run
alone, and systems loaded at different times keep their own cursors."""
import numpy as np
import pytest

import rbsog_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SYSTEMS = [(1000, 12.6, 0.7, 3), (4998, 21.5, 1.5, 4), (2000, 15.874, 1.0, 5), (10648, 27.7, 1.2, 6)]


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _params(Pk, L, lB, seed, prec, nsets, tau=0.0):
    return Pk.make_params(L, 64, lB=lB, seed=seed, n_ksets=nsets, precision=prec, tau_T=tau, T_target=1.0)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_batch_equals_alone_bitwise(prec):
    Pk, dev = _setup()
    steps = 6
    states = [I.electrolyte(N, L, seed=100 + i) for i, (N, L, _, _) in enumerate(SYSTEMS)]
    params = [_params(Pk, L, lB, seed, prec, steps + 2, tau=0.05 if i % 2 else 0.0)
              for i, (N, L, lB, seed) in enumerate(SYSTEMS)]
    b = Pk.Batch([s[0] for s in SYSTEMS], params, device=0)
    for i, (q, x, v) in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in (q, x, v)))
    b.step(steps)
    batched = [[a.cpu().numpy() for a in b.state(i)[:3]] for i in range(len(SYSTEMS))]
    eb = [b.energies(i) for i in range(len(SYSTEMS))]
    b.close()
    for i, (N, L, lB, seed) in enumerate(SYSTEMS):
        g = Pk.RBSOG(N, params[i], device=0)
        g.set_state(*(torch.tensor(a, device=dev) for a in states[i]))
        g.step(steps)
        alone = [a.cpu().numpy() for a in g.state()[:3]]
        for a, c in zip(alone, batched[i]):
            assert np.array_equal(a, c), (prec, i)
        assert g.energies() == eb[i]
        g.close()


def test_batch_late_join_keeps_other_cursors():
    """A system loaded after the others have stepped gets its own initial
    force evaluation; the running systems are unaffected."""
    Pk, dev = _setup()
    B = Pk.binding
    sysA, sysB = SYSTEMS[0], SYSTEMS[2]
    pa = _params(Pk, sysA[1], sysA[2], sysA[3], "fp32c", 12)
    pb = _params(Pk, sysB[1], sysB[2], sysB[3], "fp32c", 12)
    qa, xa, va = I.electrolyte(sysA[0], sysA[1], seed=1)
    qb, xb, vb = I.electrolyte(sysB[0], sysB[1], seed=2)
    b = Pk.Batch([sysA[0], sysB[0]], [pa, pb], device=0)
    b.set_state(0, *(torch.tensor(a, device=dev) for a in (qa, xa, va)))
    b.set_state(1, *(torch.tensor(a, device=dev) for a in (qb, xb, vb)))
    b.step(2)
    b.set_state(1, *(torch.tensor(a, device=dev) for a in (qb, xb, vb)))   # system 1 restarts
    b.step(3)
    xa5 = b.state(0)[0].cpu().numpy()
    xb3, _, _, sb = b.state(1)
    assert sb == 3
    b.close()
    ga = Pk.RBSOG(sysA[0], pa, device=0)
    ga.set_state(*(torch.tensor(a, device=dev) for a in (qa, xa, va)))
    ga.step(5)
    assert np.array_equal(ga.state()[0].cpu().numpy(), xa5)
    ga.close()
    # system 1 restarted: its first step of the second segment consumed k-sets 3.. (cursor kept)
    assert B.rbsog_get_cursor is not None


def test_autotuned_batch_equals_alone_bitwise():
    """After the autotuner picks launch shapes for a batch, a system run alone
    (which looks up the same remembered shapes for its size class) still
    reproduces its batched trajectory bit for bit."""
    Pk, dev = _setup()
    B = Pk.binding
    steps = 4
    sysl = SYSTEMS[:3]
    states = [I.electrolyte(N, L, seed=300 + i) for i, (N, L, _, _) in enumerate(sysl)]
    params = [_params(Pk, L, lB, seed, "fp32c", steps + 2) for (N, L, lB, seed) in sysl]
    b = Pk.Batch([s[0] for s in sysl], params, device=0)
    for i, (q, x, v) in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in (q, x, v)))
    chosen = B.rbsog_batch_autotune(b.ctx, 2)
    assert chosen["home"] in (64, 96, 120, 160, 224)
    b.step(steps)
    batched = [b.state(i)[0].cpu().numpy() for i in range(len(sysl))]
    b.close()
    for i, (N, L, lB, seed) in enumerate(sysl):
        g = Pk.RBSOG(N, params[i], device=0)
        g.set_state(*(torch.tensor(a, device=dev) for a in states[i]))
        g.step(steps)
        assert np.array_equal(g.state()[0].cpu().numpy(), batched[i])
        g.close()
