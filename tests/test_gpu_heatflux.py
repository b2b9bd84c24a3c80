"""Heat flux and Green-Kubo heat conductivity (Appendix A) through the C
ABI against the oracle: the device heat flux of a state (FP64 for both
precisions) within 1e-9 relative of the oracle's, with and without the far
term, at sizes spanning several blocks and a ragged tail; the conductivity
integral of a seeded flux series within 1e-12."""
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


@pytest.mark.parametrize("N,L,P,lB", [(1000, 12.6, 100, 1.0), (4998, 21.5, 37, 1.3), (64000, 50.4, 200, 0.7)])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_heat_flux_matches_oracle(N, L, P, lB, prec):
    Pk, dev = _setup()
    sog = prod_sog(O)
    q, x, v = I.electrolyte(N, L, seed=N + 3, T=1.5)
    mass = 1.7
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, lB=lB, mass=mass, n_ksets=2,
                       precision=prec)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    s = O.System((L,) * 3, sog, 3.0, lB, 1.0, 1.0)
    m = O.kseq(sog, s.L, seed=31, n_chains=2, chain_len=(P + 1) // 2)[:P]
    xw = O.wrap(x, s.L)
    for mm in (m, None):
        J = g.heat_flux(mm)
        Jo, _, _ = O.heat_flux(s, q, xw, v, mass, S=s.S(), m=mm)
        assert np.linalg.norm(J - Jo) <= 1e-9 * np.linalg.norm(Jo), (mm is None, J, Jo)
    g.close()


def test_heat_flux_rejects_batches_and_boundary_terms():
    Pk, dev = _setup()
    q, x, v = I.electrolyte(1000, 12.6, seed=2)
    g = Pk.RBSOG(1000, Pk.make_params(12.6, 16, n_ksets=2, boundary="spherical"), device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    with pytest.raises(Pk.binding.RBSOGError):
        g.heat_flux(None)
    g.close()
    b = Pk.Batch([1000, 1000], [Pk.make_params(12.6, 16, n_ksets=2)] * 2, device=0)
    for i in range(2):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in (q, x, v)))
    with pytest.raises(Pk.binding.RBSOGError):
        Pk.binding.rbsog_compute_heat_flux(b.ctx, None)
    b.close()


@pytest.mark.parametrize("on_device", [False, True])
def test_green_kubo_heat_matches_oracle(on_device):
    Pk, dev = _setup()
    rng = np.random.default_rng(17)
    n, max_lag, dt, V, T = 5000, 700, 0.005, 2000.0, 1.2
    J = np.zeros((n, 3))
    for t in range(1, n):
        J[t] = 0.97 * J[t - 1] + rng.normal(0, 0.1, 3)
    ser = torch.tensor(J, device=dev) if on_device else J
    acf, C = Pk.binding.rbsog_green_kubo_heat(ser, dt, V, T, max_lag)
    acf_o, C_o = O.green_kubo_heat(J, dt, V, T, max_lag)
    assert np.allclose(acf, acf_o, rtol=1e-12, atol=1e-15)
    assert C == pytest.approx(C_o, rel=1e-12)
