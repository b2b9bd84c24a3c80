"""Zero-frequency (boundary) terms on the device (Sec. 3.2, Eqs. 3.14 and
3.15) against the oracle: total forces with the term (FP64 to 1e-10, FP32C
to 1e-4 RMS relative), the term's energy, and per-system gating in a batch
(a system with the term and one without give the bits they give alone)."""
import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _params(Pk, L, P, prec, kind, n_ksets=2, seed=3):
    sog = prod_sog(O)
    return Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=n_ksets, seed=seed,
                          precision=prec, boundary=kind), sog


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-4)])
@pytest.mark.parametrize("kind", [1, 2])
def test_boundary_term_forces_and_energy_match_oracle(prec, tol, kind):
    Pk, dev = _setup()
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=31)
    p, sog = _params(Pk, L, P, prec, kind)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(torch.tensor(q, device=dev), torch.tensor(x, device=dev))
    m = O.kseq(sog, (L,) * 3, seed=5, n_chains=1, chain_len=P)[:P]
    f = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    e = Pk.binding.rbsog_compute_forces(g.ctx, m, f)
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    xw = O.wrap(x, s.L)
    fo, eo = O.forces(s, q, xw, S=s.S(), m=m)
    Ub, fb = O.boundary(q, xw, s.L, kind)
    assert np.linalg.norm(fb) > 1e-3 * np.linalg.norm(fo)       # well above the FP32C tolerance
    fo = fo + fb
    err = np.linalg.norm(f.cpu().numpy() - fo) / np.linalg.norm(fo)
    assert err < tol, err
    assert e["U_bound"] == pytest.approx(Ub, rel=1e-12 if prec == "fp64" else 1e-9)


def test_boundary_term_is_per_system_in_a_batch():
    Pk, dev = _setup()
    systems = [(1000, 12.6, 1), (2000, 15.874, 0), (1000, 12.6, 2)]
    states = [I.electrolyte(N, L, seed=70 + i) for i, (N, L, _) in enumerate(systems)]
    params = [_params(Pk, L, 64, "fp32c", k, n_ksets=12, seed=4 + i)[0] for i, (N, L, k) in enumerate(systems)]
    b = Pk.Batch([N for N, _, _ in systems], params, device=0)
    for i, st in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in st))
    b.step(8)
    for i, (N, L, kind) in enumerate(systems):
        g = Pk.RBSOG(N, params[i], device=0)
        g.set_state(*(torch.tensor(a, device=dev) for a in states[i]))
        g.step(8)
        xa, va, fa, _ = g.state()
        xb, vb, fb, _ = b.state(i)
        for u, w in ((xa, xb), (va, vb), (fa, fb)):
            assert torch.equal(u, w), (i, kind)
        ea, eb = g.energies(), b.energies(i)
        assert ea == eb
        assert (ea["U_bound"] != 0.0) == (kind != 0)
        g.close()
    b.close()
