"""The configurational virial tensor on the device (near field + WCA in FP64
from the cell list, far field as the random-batch estimator on a k-set)
against the oracle: FP64 contexts to 1e-10, FP32C contexts (whose rho(k) is
the FP32 compensated sweep) to 1e-6, relative to the tensor's norm."""
import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-6)])
def test_virial_matches_oracle(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    dev = torch.device("cuda:0")
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=41)
    sog = prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=2, seed=3, precision=prec)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    m = O.kseq(sog, (L,) * 3, seed=6, n_chains=1, chain_len=P)[:P]
    W = Pk.binding.rbsog_compute_virial(g.ctx, m)
    g.step(1)                                           # the step path is unaffected by the cell rebuild
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    Wo = O.virial(s, q, O.wrap(x, s.L), S=s.S(), m=m)
    assert np.linalg.norm(W - Wo) <= tol * np.linalg.norm(Wo), (W, Wo)
    assert np.array_equal(W, W.T)
