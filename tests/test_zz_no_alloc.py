"""The allocation-free structure-factor entry point (rbsog_rho_noalloc),
called through the C ABI, agrees with the context-based rbsog_rho on two
calls in a row.

It exists for callers that cannot allocate device memory where they need
rho(k) (work being recorded into a stream capture, hosts whose allocator must
not be re-entered): it keeps its scratch in a fixed device array inside the
library.  This file is collected last so that a failure here leaves every
other test already run."""
import numpy as np
import pytest

import rbsog_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_rho_noalloc_matches_rho_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    dev = torch.device("cuda:0")
    N, L = 4998, 21.5
    q, x, v = I.electrolyte(N, L, seed=21)
    g = Pk.RBSOG(N, Pk.make_params(L, 8, n_ksets=2, precision="fp64"), device=0)
    g.set_state(torch.tensor(q, device=dev), torch.tensor(x, device=dev), torch.tensor(v, device=dev))
    rng = np.random.default_rng(5)
    qd = torch.tensor(q, device=dev)
    xd = torch.tensor(x, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for P in (77, 500):            # two calls in a row, different sizes
        m = rng.integers(-40, 41, size=(P, 3)).astype(np.int32)
        ref = np.zeros((P, 2))
        B.rbsog_rho(g.ctx, m, ref)
        md = torch.tensor(m, device=dev)
        out = torch.full((P, 2), float("nan"), dtype=torch.float64, device=dev)
        B.rbsog_rho_noalloc(qd, xd, (L, L, L), md, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.sum(np.abs(q))
    with pytest.raises(B.RBSOGError):
        m = np.zeros((B.RBSOG_NOALLOC_MAX_P + 1, 3), dtype=np.int32)
        B.rbsog_rho_noalloc(qd, xd, (L, L, L), torch.tensor(m, device=dev),
                            torch.zeros((m.shape[0], 2), dtype=torch.float64, device=dev), stream)
    g.close()
