"""Radial distribution functions on the device (Appendix A) against the
oracle: pair counts bit-exact (every bin decision is exact integer
arithmetic on positions quantised to L 2^-32), g(r) to rounding; and the
64,000-ion NVT run with the RDF, the FP32C force error against the FP64 path
on the same frequency set, and the temperature taken every 100 steps."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import PP_FP32C, per_particle_rel, prod_sog

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_13824_gb300 as Pk
    return Pk, torch.device("cuda:0")


def _ctx(Pk, N, L, P=64, prec="fp32c", nsets=4, tau=0.0, seed=3):
    sog = prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=nsets, seed=seed,
                       precision=prec, tau_T=tau, T_target=1.0)
    return Pk.RBSOG(N, p, device=0), sog


def _rocksalt(n, a):
    idx = np.arange(n ** 3)
    ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
    x = (np.stack([ix, iy, iz], axis=1) + 0.5) * a
    q = np.where((ix + iy + iz) % 2 == 0, 1.0, -1.0)
    return q, x


@pytest.mark.parametrize("N,L,nbins", [(1000, 12.6, 64), (4998, 21.5, 256), (216, 9.0, 16),
                                       (10648, 27.7, 4096)])
def test_rdf_counts_bit_exact(N, L, nbins):
    Pk, dev = _setup()
    q, x, v = I.electrolyte(N, L, seed=N + 1)
    g, _ = _ctx(Pk, N, L)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    c_gpu, g_gpu = g.rdf(nbins)
    c_o, g_o, _ = O.rdf(q, x, L, nbins)
    np.testing.assert_array_equal(c_gpu, c_o)
    np.testing.assert_allclose(g_gpu, g_o, rtol=1e-13, atol=0)
    g.close()


def test_rdf_rocksalt_shells_and_neutral_sites():
    """Lattice shells land in single bins with N r3(m)/2 pairs; neutral sites
    (q = 0) are skipped; ragged tail (N not a multiple of the 256-site tile)."""
    Pk, dev = _setup()
    n, a, nbins = 10, 1.26, 64
    L = n * a
    q, x = _rocksalt(n, a)
    q = q.copy()
    q[[3, 17]] = 0.0            # one + and one - site become neutral (17 is odd parity)
    assert q.sum() == 0
    g, _ = _ctx(Pk, n ** 3, L)
    g.set_state(*(torch.tensor(arr, device=dev) for arr in (q, x)))
    c_gpu, _ = g.rdf(nbins)
    c_o, _, _ = O.rdf(q, x, L, nbins)
    np.testing.assert_array_equal(c_gpu, c_o)
    b1 = int(2 * nbins / n)
    assert c_gpu[1, b1] == 3 * n ** 3 - 12 + (1 if np.linalg.norm(x[3] - x[17]) < 1.3 else 0)
    g.close()


def test_rdf_after_dynamics_and_in_batch():
    """Systems inside a batch give the oracle's counts for their seeded
    positions; after the integrator has moved them (wrapped or not), each
    system's counts equal those of a single-system context loaded with the
    positions read back (the batch reads the system's current positions)."""
    Pk, dev = _setup()
    systems = [(1000, 12.6), (2000, 15.874)]
    params, states = [], []
    sog = prod_sog(O)
    for i, (N, L) in enumerate(systems):
        params.append(Pk.make_params(L, 64, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=30,
                                     seed=5 + i, precision="fp32c"))
        states.append(I.electrolyte(N, L, seed=40 + i))
    b = Pk.Batch([N for N, _ in systems], params, device=0)
    for i, st in enumerate(states):
        b.set_state(i, *(torch.tensor(a, device=dev) for a in st))
    for i, (N, L) in enumerate(systems):
        c_gpu, _ = b.rdf(i, 128)
        c_o, _, _ = O.rdf(states[i][0], states[i][1], L, 128)
        np.testing.assert_array_equal(c_gpu, c_o)
    b.step(20)
    for i, (N, L) in enumerate(systems):
        x = b.state(i)[0]
        c_b, g_b = b.rdf(i, 128)
        g1, _ = _ctx(Pk, N, L)
        g1.set_state(torch.tensor(states[i][0], device=dev), x)
        c_1, g_1 = g1.rdf(128)
        g1.close()
        np.testing.assert_array_equal(c_b, c_1)
    b.close()


def test_rdf_rejects_bad_arguments():
    Pk, dev = _setup()
    B = Pk.binding
    q, x, v = I.electrolyte(1000, 12.6, seed=1)
    g, _ = _ctx(Pk, 1000, 12.6)
    with pytest.raises(B.RBSOGError):
        g.rdf(64)                 # no state yet
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    for nb in (8, 100, 8192):
        with pytest.raises(B.RBSOGError):
            g.rdf(nb)
    g.close()
    p = Pk.make_params((12.6, 12.6, 14.0), 64, n_ksets=2)
    h = Pk.RBSOG(1000, p, device=0)
    h.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    with pytest.raises(B.RBSOGError):
        h.rdf(64)                 # not a cubic box
    h.close()


def test_nvt_64000_ions_checkpoints():
    """N = 64,000, L = 50.4, P = 200, Berendsen T0 = 1, FP32C, 1,000 steps.
    The initial state's RDF counts are bit-exact against the oracle.  Every
    100 steps: the FP32C force at the trajectory's positions against the FP64
    path (itself within 1e-10 of the oracle in the parity tests) on the same
    frequency set, over all ions, below 1e-4 RMS relative and per particle;
    finite energies; the temperature relaxes towards T0."""
    Pk, dev = _setup()
    N, L, P = 64000, 50.4, 200
    q, x, v = I.electrolyte(N, L, seed=2022)
    g, sog = _ctx(Pk, N, L, P=P, nsets=1001, tau=0.1, seed=77)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    c_gpu, _ = g.rdf(256)
    c_o, _, _ = O.rdf(q, x, L, 256)
    np.testing.assert_array_equal(c_gpu, c_o)
    chk32, _ = _ctx(Pk, N, L, P=P, nsets=1, seed=1)
    chk64, _ = _ctx(Pk, N, L, P=P, prec="fp64", nsets=1, seed=1)
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    m = O.kseq(sog, s.L, seed=123, n_chains=4, chain_len=P // 4)[:P]
    f32 = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    f64 = torch.zeros_like(f32)
    temps, energies = [], []
    for c in range(10):
        g.step(100)
        xg, vg, _, step = g.state()
        assert step == 100 * (c + 1)
        e = g.energies()
        temps.append(e["T"])
        energies.append(e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"] + e["K"])
        assert all(math.isfinite(val) for val in e.values())
        if c % 3 == 0 or c == 9:
            c_gpu, g_gpu = g.rdf(256)
        for chk, f in ((chk32, f32), (chk64, f64)):
            chk.set_state(torch.tensor(q, device=dev), xg)
            Pk.binding.rbsog_compute_forces(chk.ctx, m, f)
        a, b = f32.cpu().numpy(), f64.cpu().numpy()
        err = math.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))
        assert err < 1e-4, (c, err)
        assert per_particle_rel(a, b)[1] < PP_FP32C, c
    # unlike ions attract: the +- RDF peaks above 1 near contact, ++ stays below it
    b_contact = int(1.1 / (L / 512))
    assert g_gpu[1, b_contact - 3: b_contact + 6].max() > 1.2
    assert g_gpu[0, b_contact - 3: b_contact + 6].max() < g_gpu[1, b_contact - 3: b_contact + 6].max()
    assert abs(temps[-1] - 1.0) < 0.1, temps
    print("T every 100 steps:", [f"{t:.4f}" for t in temps])
    print("E every 100 steps:", [f"{u:.2f}" for u in energies])
    g.close()
    chk32.close()
    chk64.close()
