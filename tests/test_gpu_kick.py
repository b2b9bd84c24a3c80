"""The velocity-Verlet kicks of a step, whichever kernel runs them (FP32C
fuses the second half kick into the far-force scatter; FP64 and contexts
with a boundary term use the kick kernel): after one step from stored forces
F0 with new forces F1, v = v0 + dt/2m (F0 + F1) and K = (m/2) sum v^2."""
import numpy as np
import pytest

import rbsog_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec,boundary", [("fp32c", 0), ("fp32c", 1), ("fp64", 0)])
def test_one_step_applies_both_half_kicks_once(prec, boundary):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    dev = torch.device("cuda:0")
    N, L, dt, m = 4998, 21.5, 0.002, 1.7
    q, x, v = I.electrolyte(N, L, seed=71)
    p = Pk.make_params(L, 64, n_ksets=4, seed=3, precision=prec, dt=dt, mass=m, boundary=boundary)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    f0 = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    B.rbsog_compute_forces(g.ctx, None, f0)          # k-set 0: the step's first half kick uses these
    g.step(1)                                          # k-set 1 at the drifted positions
    _, v1, f1, st = g.state()
    e = g.energies()
    g.close()
    assert st == 1
    v_ref = v + dt / (2 * m) * (f0.cpu().numpy() + f1.cpu().numpy())
    assert np.abs(v1.cpu().numpy() - v_ref).max() <= 1e-13 * np.abs(v_ref).max()
    K = 0.5 * m * float(np.sum(v1.cpu().numpy() ** 2))
    assert e["K"] == pytest.approx(K, rel=1e-6 if prec == "fp32c" else 1e-12)
