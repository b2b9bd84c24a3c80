"""Parity at the full size of the 1,048,576-ion workload (L = 128, r_c = 3),
in the launch configuration the benchmark times: the oracle evaluates the
whole force for P = 100 and a sample of 20,000 particles for P = 500 and
2000 (rho(k) always over all particles).  Each case checks the global RMS
relative error and the worst per-particle error."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import PP_FP32C, PP_FP64, per_particle_rel, prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rms_rel(a, b):
    return math.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, L = 1048576, 128.0
    q, x, v = I.electrolyte(N, L, seed=2024)
    sog = prod_sog(O)
    s = O.System((L, L, L), sog, 3.0, 1.0, 1.0, 1.0)
    return N, L, q, O.wrap(x, s.L), v, sog, s


@pytest.mark.parametrize("P,full", [(100, True), (500, False), (2000, False)])
@pytest.mark.parametrize("prec,tol", [("fp32c", 1e-4), ("fp64", 1e-10)])
def test_full_size_forces(big, P, full, prec, tol):
    import paper_2205_13824_gb300 as Pk
    N, L, q, x, v, sog, s = big
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=2, seed=1,
                       precision=prec)
    g = Pk.RBSOG(N, p, device=0)
    d = torch.device("cuda:0")
    g.set_state(torch.tensor(q, device=d), torch.tensor(x, device=d), torch.tensor(v, device=d))
    if prec == "fp32c" and P == 500:
        Pk.binding.rbsog_batch_autotune(g.ctx, 2)   # the benchmark's launch shapes for this workload
    m = O.kseq(sog, s.L, seed=77, n_chains=8, chain_len=(P + 7) // 8)[:P]
    f = torch.zeros((N, 3), dtype=torch.float64, device=d)
    e = Pk.binding.rbsog_compute_forces(g.ctx, m, f)
    fg = f.cpu().numpy()
    assert np.isfinite(fg).all()
    if full:
        fo, eo = O.forces(s, q, x, S=s.S(), m=m)
        err = rms_rel(fg, fo)
        for k in ("U_near", "U_far", "U_wca"):
            assert e[k] == pytest.approx(eo[k], rel=(1e-10 if prec == "fp64" else 1e-5))
    else:
        idx = np.random.default_rng(P).choice(N, size=20000, replace=False)
        fo = O.forces_sample(s, q, x, s.S(), m, idx)
        fg = fg[idx]
        err = rms_rel(fg, fo)
    med, worst = per_particle_rel(fg, fo)
    print(f"N={N} P={P} {prec}: rms rel force err {err:.3e}, per particle median {med:.3e} max {worst:.3e}")
    assert err < tol
    assert worst < (PP_FP64 if prec == "fp64" else PP_FP32C)
    g.close()
