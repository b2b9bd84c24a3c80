"""Degenerate and boundary inputs through the C ABI against the oracle: the
smallest system (one ion pair), a system with every charge zero (only WCA
acts), and particles sitting exactly on cell boundaries and on the box faces,
for both precisions."""
import math

import numpy as np
import pytest

import oracle as O
from tests._util import prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _forces(Pk, dev, q, x, L, P, prec, m):
    sog = prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=2, seed=3, precision=prec)
    g = Pk.RBSOG(len(q), p, device=0)
    g.set_state(torch.tensor(q, device=dev), torch.tensor(x, device=dev))
    f = torch.zeros((len(q), 3), dtype=torch.float64, device=dev)
    e = Pk.binding.rbsog_compute_forces(g.ctx, m, f)
    g.close()
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    fo, eo = O.forces(s, q, O.wrap(x, s.L), S=s.S(), m=m)
    return f.cpu().numpy(), e, fo, eo


def _m(L, P, seed=1):
    sog = prod_sog(O)
    return O.kseq(sog, (L,) * 3, seed=seed, n_chains=1, chain_len=P)[:P]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-4)])
def test_single_ion_pair(prec, tol):
    Pk, dev = _setup()
    L = 10.0
    q = np.array([1.0, -1.0])
    x = np.array([[2.0, 3.0, 4.0], [3.3, 3.5, 4.2]])
    m = _m(L, 16)
    f, e, fo, eo = _forces(Pk, dev, q, x, L, 16, prec, m)
    assert np.allclose(f.sum(0), 0.0, atol=1e-9)               # equal and opposite
    assert np.linalg.norm(f - fo) <= tol * np.linalg.norm(fo)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-4)])
def test_all_charges_zero(prec, tol):
    Pk, dev = _setup()
    L = 12.6
    n = 10
    idx = np.arange(n ** 3)
    x = (np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) + 0.5) * (L / n)
    x += np.random.default_rng(2).uniform(-0.1, 0.1, x.shape)   # WCA overlaps at spacing ~1.06
    q = np.zeros(n ** 3)
    m = _m(L, 32)
    f, e, fo, eo = _forces(Pk, dev, q, x, L, 32, prec, m)
    assert e["U_near"] == 0.0 and e["U_far"] == 0.0 and e["U_self"] == 0.0
    assert e["U_wca"] == pytest.approx(eo["U_wca"], rel=1e-5)
    assert np.linalg.norm(f - fo) <= tol * np.linalg.norm(fo)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-4)])
def test_particles_on_cell_boundaries_and_box_faces(prec, tol):
    """Coordinates exactly at multiples of the cell side (both the r_c and the
    1.1 r_c grids of the two paths) and at 0 and just below L."""
    Pk, dev = _setup()
    L = 13.2
    rng = np.random.default_rng(5)
    n = 1000
    x = rng.uniform(0, L, size=(n, 3))
    sides = [L / math.floor(L / 3.0), L / math.floor(L / 3.3)]
    for k in range(200):
        h = sides[k % 2]
        x[k, k % 3] = h * rng.integers(0, int(L / h))        # on a cell face
    x[200:210, 0] = 0.0
    x[210:220, 1] = np.nextafter(L, 0.0)
    # keep particles apart so that WCA forces stay moderate: drop close pairs
    # by moving them along z
    from scipy.spatial import cKDTree
    for _ in range(20):
        pairs = cKDTree(x, boxsize=L).query_pairs(0.85)
        if not pairs:
            break
        for a, b in pairs:
            x[b, 2] = (x[b, 2] + 0.9) % L
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    m = _m(L, 64)
    f, e, fo, eo = _forces(Pk, dev, q, x, L, 64, prec, m)
    assert np.linalg.norm(f - fo) <= tol * np.linalg.norm(fo)
