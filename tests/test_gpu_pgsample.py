"""Per-Gaussian independent sampling on the device against the oracle: the
k-sequence is bit-exact (the sampler's decisions are taken in the same FP64
arithmetic on both sides), batches pad shorter sets with weight-0 entries,
and a force evaluation on a pre-sampled set, each frequency weighted by its
Gaussian's S_l / P_l, matches the oracle's weighted estimator (FP64 to
1e-10, FP32C to FP32 level)."""
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


def _params(Pk, L, P, prec, n_ksets, seed=5):
    sog = prod_sog(O)
    return Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=n_ksets, seed=seed,
                          precision=prec, sampler="per-gaussian"), sog


@pytest.mark.parametrize("L,P,seed", [((12.6,) * 3, 64, 5), ((15.0, 21.5, 30.0), 200, 2 ** 40 + 7)])
def test_kseq_is_bit_exact(L, P, seed):
    Pk, dev = _setup()
    N = 1000
    q, x, v = I.electrolyte(N, min(L), seed=1)
    p, sog = _params(Pk, L, P, "fp64", 40, seed=seed)
    g = Pk.RBSOG(N, p, device=0)
    pe, _, _ = O.pg_plan(sog, L, P)
    assert g.info()[0].P_set == pe
    ks = g.kseq(0, 40)
    g.close()
    mo, _ = O.pg_kseq(sog, L, P, seed, 0, 40)
    assert np.array_equal(ks, mo)


def test_batch_pads_shorter_sets():
    Pk, dev = _setup()
    B = Pk.binding
    boxes = [(12.6,) * 3, (30.0, 30.0, 30.0)]
    sog = prod_sog(O)
    params = [_params(Pk, L, 64, "fp64", 6, seed=9 + i)[0] for i, L in enumerate(boxes)]
    pes = [O.pg_plan(sog, L, 64)[0] for L in boxes]
    b = Pk.Batch([1000, 1000], params, device=0)
    Pb = max(pes)
    for i, L in enumerate(boxes):
        out = np.zeros((6 * Pb, 3), dtype=np.int32)
        B.rbsog_batch_get_kseq(b.ctx, i, 0, 6, out)
        mo, _ = O.pg_kseq(sog, L, 64, 9 + i, 0, 6)
        out = out.reshape(6, Pb, 3)
        assert np.array_equal(out[:, :pes[i]].reshape(-1, 3), mo)
        assert (out[:, pes[i]:] == np.array([1, 0, 0])).all()
    b.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-4)])
def test_weighted_forces_match_oracle(prec, tol):
    Pk, dev = _setup()
    N, L, P = 4998, 21.5, 96
    q, x, v = I.electrolyte(N, L, seed=61)
    p, sog = _params(Pk, L, P, prec, 3, seed=17)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    f = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    Pk.binding.rbsog_compute_forces(g.ctx, None, f)             # set 0
    e = Pk.binding.rbsog_compute_forces(g.ctx, None, f)         # set 1
    fg = f.cpu().numpy()
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    xw = O.wrap(x, s.L)
    pe, _, _ = O.pg_plan(sog, s.L, P)
    m, _ = O.pg_kseq(sog, s.L, P, 17, 1, 1)
    c = O.pg_weights(sog, s.L, P)
    ff, Uf = O.far_rb_w(s, q, xw, m, c)
    fn, Un, Uw = O.near(s, q, xw)[:3]
    fo = fn + ff
    assert e["U_far"] == pytest.approx(Uf, rel=tol)
    err = np.sqrt(np.mean(np.sum((fg - fo) ** 2, axis=1)) / np.mean(np.sum(fo ** 2, axis=1)))
    assert err <= tol, err
    # the far part alone: remove the near field to see the weights act
    err_far = np.sqrt(np.mean(np.sum((fg - fn - ff) ** 2, axis=1)) / np.mean(np.sum(ff ** 2, axis=1)))
    assert err_far <= 10 * tol, err_far


def test_mixed_samplers_rejected():
    Pk, dev = _setup()
    B = Pk.binding
    p0 = _params(Pk, 12.6, 32, "fp64", 2)[0]
    p1 = Pk.make_params(12.6, 32, n_ksets=2)
    sog = prod_sog(O)
    p1.sigma, p1.omega0, p1.M = sog.sigma, sog.omega0, sog.M
    with pytest.raises(B.RBSOGError):
        Pk.Batch([1000, 1000], [p0, p1], device=0)
