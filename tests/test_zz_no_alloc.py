"""The allocation-free structure-factor entry point (rbsog_rho_noalloc),
called through the C ABI, agrees with the context-based rbsog_rho and with
the FP64 oracle on two calls in a row.

It exists for callers that cannot allocate device memory where they need
rho(k) (work being recorded into a stream capture, hosts whose allocator must
not be re-entered): it keeps its scratch in a fixed device array inside the
library.  This file is collected last so that a failure here leaves every
other test already run."""
import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def test_rho_noalloc_matches_rho_twice():
    Pk, dev = _setup()
    B = Pk.binding
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
        orc = O.rho(q, O.wrap(x, (L,) * 3), (L, L, L), m)
        assert np.abs(got[:, 0] + 1j * got[:, 1] - orc).max() <= 1e-12 * np.sum(np.abs(q))
    with pytest.raises(B.RBSOGError):
        m = np.zeros((B.RBSOG_NOALLOC_MAX_P + 1, 3), dtype=np.int32)
        B.rbsog_rho_noalloc(qd, xd, (L, L, L), torch.tensor(m, device=dev),
                            torch.zeros((m.shape[0], 2), dtype=torch.float64, device=dev), stream)
    g.close()


def test_rho_noalloc_many_tiles_against_oracle():
    """n = 150,001 is above 64 groups x 1024-particle tiles and not a
    multiple of the tile, so every block loops over several tiles and the
    last tile is ragged; two calls in a row, P up to the stated maximum."""
    _, dev = _setup()
    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    N, L = 150001, 84.35
    rng = np.random.default_rng(9)
    x = rng.uniform(-L, 2 * L, size=(N, 3))          # any real positions
    q = rng.choice([-1.0, 1.0], size=N)
    qd = torch.tensor(q, device=dev)
    xd = torch.tensor(x, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for P in (B.RBSOG_NOALLOC_MAX_P, 33):
        m = rng.integers(-60, 61, size=(P, 3)).astype(np.int32)
        out = torch.full((P, 2), float("nan"), dtype=torch.float64, device=dev)
        B.rbsog_rho_noalloc(qd, xd, (L, L, L), torch.tensor(m, device=dev), out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        sel = np.arange(0, P, max(1, P // 64))        # oracle on a sample of the frequencies
        orc = O.rho(q, O.wrap(x, (L,) * 3), (L, L, L), m[sel])
        assert np.abs(got[sel, 0] + 1j * got[sel, 1] - orc).max() <= 1e-12 * np.sum(np.abs(q))


def test_rho_noalloc_rejects_host_and_mis_shaped_buffers():
    """The binding refuses what would hand the kernel a host pointer or a
    buffer shorter than P rows, before any device work."""
    _, dev = _setup()
    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    n, P, L = 100, 8, (10.0, 10.0, 10.0)
    q = torch.zeros(n, dtype=torch.float64, device=dev)
    x = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    m = torch.ones((P, 3), dtype=torch.int32, device=dev)
    out = torch.zeros((P, 2), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        B.rbsog_rho_noalloc(q.cpu().numpy(), x, L, m, out)
    with pytest.raises(ValueError):
        B.rbsog_rho_noalloc(q, x, L, m, out[: P - 1])
    with pytest.raises(ValueError):
        B.rbsog_rho_noalloc(q, x.float(), L, m, out)
    with pytest.raises(ValueError):
        B.rbsog_rho_noalloc(q, x, L, m.long(), out)
