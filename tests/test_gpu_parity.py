"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs and the same frequency sets.

Bars: integer work bit-exact (sampled sequence, cell list, neighbour
counts); FP64 forces within 1e-10 RMS relative of the oracle; FP32C forces
within 1e-4 RMS relative (the precision target), energies reported."""
import math

import numpy as np
import pytest

import oracle as O
import rbsog_inputs as I
from tests._util import B_PROD, M_PROD, PP_FP32C, PP_FP64, per_particle_rel, prod_sog, untruncated_M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _lib():
    import paper_2205_13824_gb300 as P
    return P


def rms_rel(a, b):
    return math.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))


def make(N, L, P, prec="fp64", n_ksets=4, seed=11, chain_len=0, sog=None, wca=True, lB=1.0,
         tau=0.0, dt=0.001):
    Pk = _lib()
    sog = sog or prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=n_ksets,
                       seed=seed, chain_len=chain_len, precision=prec, lB=lB,
                       wca_sigma=1.0 if wca else 0.0, wca_eps=1.0 if wca else 0.0, tau_T=tau,
                       dt=dt)
    return Pk.RBSOG(N, p, device=0), sog


def osys(L, sog, wca=True, lB=1.0):
    Lv = (L,) * 3 if isinstance(L, (int, float)) else tuple(L)
    return O.System(Lv, sog, 3.0, lB, 1.0 if wca else 0.0, 1.0 if wca else 0.0)


def to_dev(*arrs):
    d = _dev()
    return [torch.tensor(a, device=d) for a in arrs]


# ------------------------------------------------------------------ sampler

@pytest.mark.parametrize("L,P,nsets,chain", [(12.6, 100, 11, 64), (50.4, 200, 7, 0), (128.0, 500, 5, 256),
                                             ((10.0, 12.0, 15.0), 37, 9, 50)])
def test_kseq_bit_exact(L, P, nsets, chain):
    """The device Metropolis-Hastings chains emit exactly the oracle's
    sequence (same Philox streams, same FP64 decisions)."""
    _dev()
    Lv = (L,) * 3 if isinstance(L, (int, float)) else L
    N = 1000
    g, sog = make(N, Lv, P, n_ksets=nsets, seed=20240601, chain_len=chain)
    info, _, _ = g.info()
    ks_gpu = g.kseq(0, nsets)
    ks_orc = O.kseq(sog, Lv, seed=20240601, n_chains=info.n_chains, chain_len=info.chain_len)
    assert np.array_equal(ks_gpu, ks_orc[: nsets * P])
    g.close()


def test_sog_solve_and_S_match_oracle():
    _dev()
    Pk = _lib()
    for L in (12.6, 128.0):
        p = Pk.make_params(L, 10, n_ksets=1)      # sigma <= 0: library solves C0/C1
        g = Pk.RBSOG(1000, p, device=0)
        info, om, s = g.info()
        ref = O.SOG.solve(B_PROD, 3.0, untruncated_M(B_PROD))
        # the C1 root is found from a residual with cancellation (1 + r_c^2 F'),
        # whose FP64 rounding depends on the summation order: the two
        # independent solvers agree to ~1e-11 in sigma, not to the last bit
        assert info.sigma == pytest.approx(ref.sigma, rel=1e-10)
        assert info.omega0 == pytest.approx(ref.omega0, rel=1e-10)
        tr = O.SOG(B_PROD, ref.sigma, ref.omega0, M_PROD)
        assert np.allclose(om, tr.omega, rtol=1e-10)
        assert np.allclose(s, tr.s, rtol=1e-10)
        assert info.S == pytest.approx(tr.S((L, L, L)), rel=1e-10)
        g.close()


# --------------------------------------------------------------- cell list

def _device_cells(start, perm, ncell):
    """Cell of every particle as the device's (cell_start, perm) list it."""
    cell = np.full(len(perm), -1, dtype=np.int64)
    for c in range(ncell):
        cell[perm[start[c]:start[c + 1]]] = c
    return cell


def _fixed_x(x, L):
    return np.clip(np.floor(x[:, 0] * (4294967296.0 / L)), 0.0, 4294967295.0).astype(np.uint64)


@pytest.mark.parametrize("N,L", [(1000, 12.6), (4998, 21.5), (64000, 50.4), (2, 9.0), (10, 20.0),
                                 ("faces", 13.2)])
def test_cell_list_and_neighbours_bit_exact(N, L):
    """Cell membership against the oracle's plain binning (floor(x / h) per
    axis): every cell holds the same set of particles, so cell_start is
    bit-exact.  The device decides the cell by floor(x * (n / L)); the two
    rules can only part for a coordinate within a few ulp of a cell face,
    where the particle may sit in either neighbouring cell along that axis
    (allowed, and counted: the "faces" case puts 300 coordinates on faces).
    Neighbour counts are bit-exact against the oracle's O(N^2) scan or cell
    traversal.  The kernel's own order inside a cell (fixed-point x, then
    index) is checked as an invariant of the device list."""
    _dev()
    if N == "faces":
        rng = np.random.default_rng(5)
        N = 1200
        x = rng.uniform(0, L, size=(N, 3))
        h = L / math.floor(L / 3.0)
        for k in range(300):
            x[k, k % 3] = h * rng.integers(0, int(L / h))
        q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
        v = np.zeros_like(x)
    elif N in (2, 10):       # degenerate: a lone pair; a box of mostly empty cells
        q, x = I.random_neutral(N, L, seed=4, min_dist=0.9)
        v = np.zeros_like(x)
    else:
        q, x, v = I.electrolyte(N, L, seed=3)
    g, sog = make(N, L, 8)
    g.set_state(*to_dev(q, x, v))
    xw = O.wrap(x, (L,) * 3)
    nc, cell_o, start_o, perm_o = O.cell_list(xw, (L, L, L), 3.0)
    ncell = int(np.prod(nc))
    start = np.zeros(ncell + 1, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    nbr = np.zeros(N, dtype=np.int32)
    _lib().binding.rbsog_get_cells(g.ctx, start, perm, nbr)
    assert np.array_equal(np.sort(perm), np.arange(N))          # a permutation
    cell_d = _device_cells(start, perm, ncell)
    diff = np.nonzero(cell_d != cell_o)[0]
    nx, ny = int(nc[0]), int(nc[1])
    h = L / np.asarray(nc, float)
    for i in diff:                                              # face particles only
        cd = np.array([cell_d[i] % nx, (cell_d[i] // nx) % ny, cell_d[i] // (nx * ny)])
        co = np.array([cell_o[i] % nx, (cell_o[i] // nx) % ny, cell_o[i] // (nx * ny)])
        ax = np.nonzero(cd != co)[0]
        assert len(ax) == 1 and abs(int(cd[ax[0]]) - int(co[ax[0]])) == 1, i
        face = max(cd[ax[0]], co[ax[0]]) * h[ax[0]]
        assert abs(xw[i, ax[0]] - face) <= 4 * np.finfo(float).eps * L, i
    if N != 1200:
        assert len(diff) == 0
    if len(diff) == 0:
        assert np.array_equal(start, start_o[: ncell + 1])
    # (every particle's device cell equals its oracle cell but for the face
    # particles above, so every cell holds the same set of members)
    key = (_fixed_x(xw, L) << np.uint64(32)) | np.arange(N, dtype=np.uint64)
    ks, cs = key[perm], cell_d[perm]                            # device order in a cell
    same = cs[1:] == cs[:-1]
    assert np.all(ks[1:][same] > ks[:-1][same])
    if N <= 5000:
        _, _, _, nbr_o = O.near(osys(L, sog), q, xw, "direct")
    else:
        _, _, _, nbr_o = O.near(osys(L, sog), q, xw, "cells")
    assert np.array_equal(nbr, nbr_o)
    g.close()


# ------------------------------------------------------------------- rho(k)

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 2e-6)])
def test_rho_matches_oracle(prec, tol):
    _dev()
    N, L = 4998, 21.5
    q, x, v = I.electrolyte(N, L, seed=5)
    g, sog = make(N, L, 8, prec=prec)
    g.set_state(*to_dev(q, x, v))
    rng = np.random.default_rng(1)
    m = rng.integers(-40, 41, size=(77, 3)).astype(np.int32)
    out = np.zeros((77, 2))
    _lib().binding.rbsog_rho(g.ctx, m, out)
    ref = O.rho(q, O.wrap(x, (L,) * 3), (L, L, L), m)
    err = np.abs(out[:, 0] + 1j * out[:, 1] - ref)
    assert err.max() <= tol * np.sum(np.abs(q))
    g.close()


# ------------------------------------------------------------------- forces

CASES = [
    # N, L, P: the 1,000-ion electrolyte; a ragged size (not a multiple of
    # any tile, P not a multiple of 32); a 64,000-ion box; 3 cells per side
    (1000, 12.6, 100),
    (4998, 21.5, 37),
    (64000, 50.4, 200),
    (216, 9.0, 64),
]


@pytest.mark.parametrize("N,L,P", CASES)
def test_forces_fp64_match_oracle(N, L, P):
    _dev()
    q, x, v = I.electrolyte(N, L, seed=N)
    g, sog = make(N, L, P)
    g.set_state(*to_dev(q, x, v))
    s = osys(L, sog)
    m = O.kseq(sog, s.L, seed=99, n_chains=4, chain_len=(P + 3) // 4)[:P]
    f_gpu = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    e = _lib().binding.rbsog_compute_forces(g.ctx, m, f_gpu)
    xw = O.wrap(x, s.L)
    f_o, e_o = O.forces(s, q, xw, S=s.S(), m=m)          # every particle
    fg = f_gpu.cpu().numpy()
    assert rms_rel(fg, f_o) < 1e-10
    assert per_particle_rel(fg, f_o)[1] < PP_FP64
    for k in ("U_near", "U_far", "U_self", "U_wca"):
        assert e[k] == pytest.approx(e_o[k], rel=1e-10, abs=1e-10)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_forces_in_a_cuboid_box_match_oracle(prec):
    """A cuboid box (three different sides): per-dimension cell sides,
    fixed-point scales, image shifts and stencil windows, against the
    oracle on the same k-set."""
    _dev()
    B = _lib().binding
    a = 1.26
    n = (8, 10, 16)
    L = tuple(float(k * a) for k in n)
    rng = np.random.default_rng(42)
    grid = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1).reshape(-1, 3)
    x = (grid + 0.5) * a + rng.uniform(-0.2, 0.2, size=grid.shape)
    N = x.shape[0]
    q = np.where(rng.permutation(N) % 2 == 0, 1.0, -1.0)
    P = 48
    g, sog = make(N, L, P, prec=prec, n_ksets=2, seed=5)
    g.set_state(*to_dev(q, x))
    s = osys(L, sog)
    m = O.kseq(sog, s.L, seed=9, n_chains=4, chain_len=P // 4)[:P]
    f = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    B.rbsog_compute_forces(g.ctx, m, f)
    fo, _ = O.forces(s, q, O.wrap(x, s.L), S=s.S(), m=m)
    fg = f.cpu().numpy()
    g.close()
    if prec == "fp64":
        assert rms_rel(fg, fo) < 1e-10
        assert per_particle_rel(fg, fo)[1] < PP_FP64
    else:
        assert rms_rel(fg, fo) < 1e-4
        assert per_particle_rel(fg, fo)[1] < PP_FP32C


@pytest.mark.parametrize("N,L,P", CASES)
def test_forces_fp32c_within_target(N, L, P):
    _dev()
    q, x, v = I.electrolyte(N, L, seed=N)
    g, sog = make(N, L, P, prec="fp32c")
    g.set_state(*to_dev(q, x, v))
    s = osys(L, sog)
    m = O.kseq(sog, s.L, seed=99, n_chains=4, chain_len=(P + 3) // 4)[:P]
    f_gpu = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    e = _lib().binding.rbsog_compute_forces(g.ctx, m, f_gpu)
    xw = O.wrap(x, s.L)
    f_o, e_o = O.forces(s, q, xw, S=s.S(), m=m)          # every particle
    fg = f_gpu.cpu().numpy()
    err = rms_rel(fg, f_o)
    med, worst = per_particle_rel(fg, f_o)
    U = e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"]
    U_o = e_o["U_near"] + e_o["U_far"] - e_o["U_self"] + e_o["U_wca"]
    print(f"FP32C N={N} P={P}: rms rel force err {err:.3e}, per particle median {med:.3e} "
          f"max {worst:.3e}, rel energy err {abs(U - U_o) / abs(U_o):.3e}")
    assert abs(U - U_o) <= 1e-5 * abs(U_o)
    assert err < 1e-4
    assert worst < PP_FP32C
    g.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-5)])
def test_folded_sets_equal_the_full_sum(prec, tol):
    """A sampled set is folded into its runs of repeated frequencies, each
    evaluated once and weighted by its length; the forces and energies equal
    those of the same P frequencies given explicitly (no folding), and both
    match the oracle on that set."""
    _dev()
    N, L, P = 4998, 21.5, 200
    q, x, v = I.electrolyte(N, L, seed=77)
    g, sog = make(N, L, P, prec=prec, n_ksets=3, seed=123)
    g.set_state(*to_dev(q, x, v))
    info, _, _ = g.info()
    m = O.kseq(sog, (L,) * 3, seed=123, n_chains=info.n_chains, chain_len=info.chain_len)[:P]
    assert np.array_equal(g.kseq(0, 1), m)     # the device's first set is the oracle's
    runs = 1 + int(np.sum(np.any(m[1:] != m[:-1], axis=1)))
    assert runs < 0.75 * P                    # the chain repeats states: the set folds
    B = _lib().binding
    f_fold = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    e_fold = B.rbsog_compute_forces(g.ctx, None, f_fold)      # next set of the sequence: folded
    f_full = torch.zeros_like(f_fold)
    e_full = B.rbsog_compute_forces(g.ctx, m, f_full)         # the same P frequencies, explicit
    a, b = f_fold.cpu().numpy(), f_full.cpu().numpy()
    assert rms_rel(a, b) < tol
    for k in ("U_near", "U_far", "U_wca"):
        assert e_fold[k] == pytest.approx(e_full[k], rel=tol)
    s = osys(L, sog)
    f_o, e_o = O.forces(s, q, O.wrap(x, s.L), S=s.S(), m=m)
    assert rms_rel(a, f_o) < (1e-10 if prec == "fp64" else 1e-4)
    assert e_fold["U_far"] == pytest.approx(e_o["U_far"], rel=(1e-10 if prec == "fp64" else 1e-5))
    g.close()


def test_far_force_sums_to_zero_and_no_nan():
    """Per k-set the random-batch force has zero sum (Im rho* rho = 0) and
    the near force obeys Newton 3, so the total force sums to ~0."""
    _dev()
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=9)
    for prec, tol in (("fp64", 1e-11), ("fp32c", 1e-5)):
        g, sog = make(N, L, P, prec=prec, n_ksets=3)
        g.set_state(*to_dev(q, x, v))
        f = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
        _lib().binding.rbsog_compute_forces(g.ctx, None, f)
        fn = f.cpu().numpy()
        assert np.isfinite(fn).all()
        assert np.abs(fn.sum(0)).max() <= tol * np.abs(fn).sum(1).mean() * math.sqrt(N)
        g.close()


# ------------------------------------------------------------------- dynamics

@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_md_trajectory_matches_oracle(prec):
    """One force evaluation + 10 velocity-Verlet steps on the 1,000-ion
    electrolyte with the pre-sampled sequence (Algorithm 1)."""
    _dev()
    N, L, P, steps = 1000, 12.6, 100, 10
    q, x, v = I.electrolyte(N, L, seed=1)
    g, sog = make(N, L, P, prec=prec, n_ksets=steps + 1, seed=42, chain_len=100)
    g.set_state(*to_dev(q, x, v))
    g.step(steps)
    xg, vg, fg, nstep = g.state()
    assert nstep == steps
    info, _, _ = g.info()
    s = osys(L, sog)
    ks = O.kseq(sog, s.L, seed=42, n_chains=info.n_chains, chain_len=info.chain_len)
    xo, vo, fo, es = O.md(s, q, x, v, s.S(), P, ks, steps, 0.001)
    dx = xg.cpu().numpy() - xo
    dx -= L * np.rint(dx / L)
    if prec == "fp64":
        assert np.abs(dx).max() < 1e-11
        assert np.abs(vg.cpu().numpy() - vo).max() < 1e-9
        assert rms_rel(fg.cpu().numpy(), fo) < 1e-10
        assert per_particle_rel(fg.cpu().numpy(), fo)[1] < PP_FP64
        e = g.energies()
        assert e["K"] == pytest.approx(es[-1]["K"], rel=1e-10)
        assert e["U_far"] == pytest.approx(es[-1]["U_far"], rel=1e-10)
    else:
        assert np.abs(dx).max() < 1e-6
        assert rms_rel(fg.cpu().numpy(), fo) < 1e-4
        assert per_particle_rel(fg.cpu().numpy(), fo)[1] < PP_FP32C
    g.close()


def test_fp32c_neighbour_lists_over_rebuilds():
    """FP32C with neighbour lists: 80 steps at T = 4 (particles cross the
    skin/2 displacement many times, so lists are rebuilt during the run) stay
    on the oracle's trajectory; a small box (L = 9, fewer than 3 cells of
    r_c + skin per side) takes the cell-stencil path and matches too."""
    _dev()
    for N, L, P, steps in ((1000, 12.6, 100, 80), (216, 9.0, 64, 40)):
        q, x, v = I.electrolyte(N, L, seed=11, T=4.0)
        g, sog = make(N, L, P, prec="fp32c", n_ksets=steps + 1, seed=21, chain_len=50)
        g.set_state(*to_dev(q, x, v))
        g.step(steps)
        xg, vg, fg, nstep = g.state()
        assert nstep == steps
        info, _, _ = g.info()
        s = osys(L, sog)
        ks = O.kseq(sog, s.L, seed=21, n_chains=info.n_chains, chain_len=info.chain_len)
        xo, vo, fo, es = O.md(s, q, x, v, s.S(), P, ks, steps, 0.001)
        dx = xg.cpu().numpy() - xo
        dx -= L * np.rint(dx / L)
        assert np.abs(dx).max() < 1e-5, (N, np.abs(dx).max())
        assert rms_rel(fg.cpu().numpy(), fo) < 1e-4
        moved = np.abs(((xo - x) + L / 2) % L - L / 2).max()
        assert moved > 0.15 or N == 216        # beyond half the skin (0.15 at r_c = 3)
        # the last step of a call computes the energies (the others leave the
        # pair energies out): all of them match the oracle's last step
        e = g.energies()
        for k in ("U_near", "U_far", "U_wca", "K"):
            assert e[k] == pytest.approx(es[-1][k], rel=1e-4, abs=1e-3), k
        assert e["U_wca"] > 0.0
        g.close()


def test_neighbour_list_overflow_is_reported():
    """A cluster far denser than the box's mean density overflows the
    neighbour-list capacity (sized from the mean): the force evaluation fails
    with RBSOG_ENUMERIC instead of dropping pairs."""
    _dev()
    B = _lib().binding
    L = 20.0
    # 1000 particles on a lattice of spacing 0.8 in one corner (density ~2),
    # 512 on a lattice of spacing 1.2 elsewhere: mean density 0.19
    dense = np.stack(np.meshgrid(*[np.arange(10)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.8 + 1.0
    sparse = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3) * 1.2 + 10.3
    x = np.concatenate([dense, sparse]).astype(np.float64)
    N = x.shape[0]
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    g, _ = make(N, L, 32, prec="fp32c", n_ksets=2, seed=1)
    g.set_state(*to_dev(q, x))
    f = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    with pytest.raises(B.RBSOGError, match="neighbour list"):
        B.rbsog_compute_forces(g.ctx, None, f)
    g.close()


def test_fp64_dense_cluster_in_staged_chunks_matches_oracle():
    """FP64 cell stencil on the dense-corner configuration: the corner's rows
    exceed the shared-memory staging chunk (sized from the mean density), so
    later chunks add to the first, and the small system splits the stencil
    rows over the block's warps; forces match the oracle per particle."""
    _dev()
    B = _lib().binding
    L, P = 20.0, 32
    dense = np.stack(np.meshgrid(*[np.arange(10)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.8 + 1.0
    sparse = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3) * 1.2 + 10.3
    x = np.concatenate([dense, sparse]).astype(np.float64)
    N = x.shape[0]
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    g, sog = make(N, L, P, prec="fp64", n_ksets=2, seed=1)
    g.set_state(*to_dev(q, x))
    s = osys(L, sog)
    m = O.kseq(sog, s.L, seed=3, n_chains=4, chain_len=P // 4)[:P]
    f = torch.zeros((N, 3), dtype=torch.float64, device=_dev())
    B.rbsog_compute_forces(g.ctx, m, f)
    fo, _ = O.forces(s, q, O.wrap(x, s.L), S=s.S(), m=m)
    fg = f.cpu().numpy()
    g.close()
    assert math.sqrt(np.sum((fg - fo) ** 2) / np.sum(fo ** 2)) < 1e-10
    assert per_particle_rel(fg, fo)[1] < PP_FP64


def test_berendsen_matches_oracle():
    _dev()
    N, L, P, steps = 1000, 12.6, 50, 6
    q, x, v = I.electrolyte(N, L, seed=2, T=2.0)
    g, sog = make(N, L, P, n_ksets=steps + 1, seed=5, chain_len=50, tau=0.01)
    g.set_state(*to_dev(q, x, v))
    g.step(steps)
    xg, vg, fg, _ = g.state()
    info, _, _ = g.info()
    s = osys(L, sog)
    ks = O.kseq(sog, s.L, seed=5, n_chains=info.n_chains, chain_len=info.chain_len)
    xo, vo, fo, es = O.md(s, q, x, v, s.S(), P, ks, steps, 0.001, T0=1.0, tau=0.01)
    assert np.abs(vg.cpu().numpy() - vo).max() < 1e-9
    assert g.energies()["T"] == pytest.approx(es[-1]["T"], rel=1e-10)
    g.close()


@pytest.mark.parametrize("steps,T", [(5, 1.0), (60, 4.0)])
def test_graph_replay_equals_eager_launches(steps, T):
    """The CUDA-graph step and the eager (profiled) step give identical bits;
    the longer, hotter run moves particles past half the skin, so the
    captured step's conditional rebuild node fires inside the graph."""
    _dev()
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=8, T=T)
    out = []
    for prof in (False, True):
        g, _ = make(N, L, P, prec="fp32c", n_ksets=steps + 1, seed=3)
        _lib().binding.rbsog_set_profiling(g.ctx, prof)
        g.set_state(*to_dev(q, x, v))
        g.step(steps)
        xg, vg, fg, _ = g.state()
        out.append((xg.cpu().numpy(), vg.cpu().numpy(), fg.cpu().numpy()))
        if prof:
            rep = _lib().binding.rbsog_get_profile(g.ctx)
            assert rep["far_scatter_fp32c"][0] == steps + 1
            assert "near_fp32c" in rep and "list_build" in rep
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    if steps == 60:                # a particle moved past skin/2 = r_c/20: lists were rebuilt in the graph
        d = out[0][0] - x
        d -= L * np.round(d / L)
        assert np.sqrt((d ** 2).sum(1)).max() > 3.0 / 20


def test_checkpoint_resume_is_bit_exact():
    """6 steps in one run equal 3 steps, a checkpoint (x, v, f, cursor,
    step) through host memory, a fresh context and 3 more steps: bit for bit
    in FP64; in FP32C the restarted run builds fresh neighbour lists at the
    restart, whose order changes the FP32 rounding of the pair sums only."""
    _dev()
    B = _lib().binding
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=8)
    for prec in ("fp64", "fp32c"):
        g, _ = make(N, L, P, prec=prec, n_ksets=8, seed=3)
        g.set_state(*to_dev(q, x, v))
        g.step(6)
        ref = [a.cpu().numpy() for a in g.state()[:3]]
        g.close()
        g, _ = make(N, L, P, prec=prec, n_ksets=8, seed=3)
        g.set_state(*to_dev(q, x, v))
        g.step(3)
        xs, vs, fs = (np.zeros((N, 3)) for _ in range(3))
        step = B.rbsog_get_state(g.ctx, xs, vs, fs)
        cur = B.rbsog_get_cursor(g.ctx)
        assert (step, cur) == (3, 4)
        g.close()
        g, _ = make(N, L, P, prec=prec, n_ksets=8, seed=3)
        B.rbsog_set_state(g.ctx, q, xs, vs)
        B.rbsog_restore(g.ctx, fs, cur, step)
        g.step(3)
        out = [a.cpu().numpy() for a in g.state()[:3]]
        assert g.state()[3] == 6
        if prec == "fp64":
            for a, b in zip(ref, out):
                assert np.array_equal(a, b)
        else:
            assert np.abs(out[0] - ref[0]).max() < 1e-10
            assert np.abs(out[1] - ref[1]).max() < 1e-7
            assert rms_rel(out[2], ref[2]) < 1e-5
        g.close()


def test_fused_kick_drift_equals_separate_steps():
    """In NVE on neighbour lists a call of several steps lets each step's
    scatter run the next step's kick-drift; the state and energies equal,
    bit for bit, those of one-step calls (each a whole step) and of the
    eager launches, including steps with list rebuilds."""
    _dev()
    N, L, P, steps = 4998, 21.5, 64, 30
    q, x, v = I.electrolyte(N, L, seed=18, T=4.0)
    out = []
    for mode in ("fused", "single", "eager"):
        g, _ = make(N, L, P, prec="fp32c", n_ksets=steps + 2, seed=6)
        _lib().binding.rbsog_set_profiling(g.ctx, mode == "eager")
        g.set_state(*to_dev(q, x, v))
        if mode == "single":
            for _ in range(steps):
                g.step(1)
        else:
            g.step(steps)
        st = [a.cpu().numpy() for a in g.state()[:3]]
        out.append((st, g.energies(), g.info()[0].list_builds))
        g.close()
    assert out[0][2] > 1                      # lists were rebuilt during the run
    for st, e, nb in out[1:]:
        for a, b in zip(out[0][0], st):
            assert np.array_equal(a, b)
        assert e == out[0][1]
        assert nb == out[0][2]


def test_runs_are_deterministic():
    _dev()
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=8)
    res = []
    for _ in range(2):
        g, _ = make(N, L, P, prec="fp32c", n_ksets=4, seed=3)
        g.set_state(*to_dev(q, x, v))
        g.step(3)
        res.append(g.state()[2].cpu().numpy())
        g.close()
    assert np.array_equal(res[0], res[1])


# ------------------------------------------------------------------- errors

def test_invalid_arguments_are_rejected():
    _dev()
    Pk = _lib()
    B = Pk.binding
    ctx = B.rbsog_create(100, 0, None)
    bad = [dict(L=5.0), dict(b=1.0), dict(P=0), dict(M=200), dict(precision=7), dict(r_c=7.0, L=12.0)]
    for kw in bad:
        args = dict(L=12.6, P=10, n_ksets=1)
        args.update(kw)
        with pytest.raises(B.RBSOGError) as ei:
            B.rbsog_set_params(ctx, Pk.make_params(**args))
        assert ei.value.status == 1
    with pytest.raises(B.RBSOGError) as ei:
        B.rbsog_step(ctx, 1)
    assert ei.value.status == 4
    B.rbsog_set_params(ctx, Pk.make_params(12.6, 10, n_ksets=2))
    q = np.ones(100)
    x = np.random.default_rng(0).uniform(0, 12.6, (100, 3))
    with pytest.raises(B.RBSOGError) as ei:
        B.rbsog_set_state(ctx, q, x, None)                 # not neutral
    assert ei.value.status == 1
    q[::2] = -1
    B.rbsog_set_state(ctx, q, x, None)                     # host pointers work too
    with pytest.raises(B.RBSOGError) as ei:
        B.rbsog_step(ctx, 5)                               # only 2 k-sets sampled
    assert ei.value.status == 1
    B.rbsog_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("nsteps,with_f,where", [(1, True, "pinned"), (3, True, "device"), (2, False, "pinned")])
def test_step_io_equals_the_composed_calls(prec, nsteps, with_f, where):
    """rbsog_step_io (state in, steps, state out in one call) gives the bits
    of rbsog_set_state + rbsog_restore + rbsog_step + rbsog_get_state, from a
    mid-run checkpoint (with forces) or from positions alone."""
    _dev()
    import torch
    B = _lib().binding
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=12)
    if with_f:
        g, _ = make(N, L, P, prec=prec, n_ksets=12, seed=3)
        g.set_state(*to_dev(q, x, v))
        g.step(4)
        x, v, f = (a.cpu().numpy() for a in g.state()[:3])
        cur, step = B.rbsog_get_cursor(g.ctx), 4
        g.close()
    else:
        f, cur, step = None, 0, 0

    def buf(a):
        t = torch.tensor(a) if a is not None else None
        if t is None:
            return None
        return t.pin_memory() if where == "pinned" else t.cuda()

    ref, _ = make(N, L, P, prec=prec, n_ksets=12, seed=3)
    B.rbsog_set_state(ref.ctx, q, x, v)
    if with_f:
        B.rbsog_restore(ref.ctx, f, cur, step)
    B.rbsog_step(ref.ctx, nsteps)
    xr, vr, fr = (np.zeros((N, 3)) for _ in range(3))
    sr = B.rbsog_get_state(ref.ctx, xr, vr, fr)
    er = B.rbsog_get_energies(ref.ctx)
    ref.close()

    g, _ = make(N, L, P, prec=prec, n_ksets=12, seed=3)
    xo, vo, fo = (buf(np.zeros((N, 3))) for _ in range(3))
    B.rbsog_step_io(g.ctx, buf(q), buf(x), buf(v), buf(f), cur, step, nsteps, xo, vo, fo)
    torch.cuda.synchronize()
    for a, b in ((xr, xo), (vr, vo), (fr, fo)):
        assert np.array_equal(a, b.cpu().numpy())
    xs = np.zeros((N, 3))
    assert B.rbsog_get_state(g.ctx, xs) == sr
    assert np.array_equal(xs, xr)
    assert B.rbsog_get_energies(g.ctx) == er
    # the same buffers in and out (the bench's end-to-end loop)
    xb, vb, fb = buf(xr), buf(vr), buf(fr)
    B.rbsog_step_io(g.ctx, buf(q), xb, vb, fb, B.rbsog_get_cursor(g.ctx), sr, 1, xb, vb, fb)
    assert np.all(np.isfinite(xb.cpu().numpy()))
    with pytest.raises(B.RBSOGError):
        B.rbsog_step_io(g.ctx, buf(q), xb, vb, fb, 0, 0, 0, xb, vb, fb)   # nsteps < 1
    with pytest.raises(B.RBSOGError):
        B.rbsog_step_io(g.ctx, buf(q), xb, vb, fb, 12, 0, 1, xb, vb, fb)  # no k-set left
    g.close()


def test_fp32c_lists_need_an_accurate_combined_table():
    """The list path takes G and F from one combined table.  An SOG set whose
    narrowest Gaussian is narrow against the table step (sigma = 0.3) makes
    that table inaccurate, so such a set runs on the cell stencil (which
    falls back to exp + Taylor sums by its own check) and still matches the
    oracle; the production set runs on lists.  The cell grid tells which:
    side r_c + skin with lists, r_c without."""
    _dev()
    B = _lib().binding
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=13)
    narrow = O.SOG(B_PROD, 0.3, 1.0, M_PROD)
    narrow = O.SOG(B_PROD, 0.3, narrow.omega_bsa0, M_PROD)
    for sog, nc in ((prod_sog(O), math.floor(L / 3.3)), (narrow, math.floor(L / 3.0))):
        g, _ = make(N, L, P, prec="fp32c", n_ksets=2, seed=3, sog=sog)
        g.set_state(*to_dev(q, x, v))
        info, _, _ = g.info()
        assert tuple(info.ncell) == (nc,) * 3
        m = O.kseq(sog, (L,) * 3, seed=7, n_chains=1, chain_len=P)[:P]
        import torch
        f = torch.zeros((N, 3), dtype=torch.float64, device="cuda:0")
        B.rbsog_compute_forces(g.ctx, m, f)
        s = osys(L, sog)
        fo, _ = O.forces(s, q, O.wrap(x, s.L), S=s.S(), m=m)
        err = np.linalg.norm(f.cpu().numpy() - fo) / np.linalg.norm(fo)
        assert err < 1e-4, (sog.sigma, err)
        g.close()


def test_fp32c_coreshell_kernel_matches_the_oracle_scheme():
    """The paper's core-shell kernel (Sec. 3.4) on the list path: total
    forces and near energy against the oracle's core-shell near field (same
    10 Taylor terms, 2 + 8 index bits, r_in) plus its far field, to the FP32C
    tolerance; the scheme itself stays close to the direct Gaussian sums."""
    _dev()
    import torch
    Pk = _lib()
    B = Pk.binding
    N, L, P = 4998, 21.5, 64
    q, x, v = I.electrolyte(N, L, seed=17)
    sog = prod_sog(O)
    p = Pk.make_params(L, P, sigma=sog.sigma, omega0=sog.omega0, M=sog.M, n_ksets=8, seed=3, precision="fp32c",
                       near_kernel="coreshell", r_in=1.0)
    g = Pk.RBSOG(N, p, device=0)
    g.set_state(*to_dev(q, x, v))
    m = O.kseq(sog, (L,) * 3, seed=9, n_chains=1, chain_len=P)[:P]
    f = torch.zeros((N, 3), dtype=torch.float64, device="cuda:0")
    e = B.rbsog_compute_forces(g.ctx, m, f)
    s = osys(L, sog)
    xw = O.wrap(x, s.L)
    fo, eo = O.forces(s, q, xw, S=s.S(), m=m)
    fnd, und, _, _ = O.near(s, q, xw, method="cells")
    fnc, unc, _ = O.near_coreshell(s, q, xw, O.coreshell(1.0, Q=10, b_exp=2, b_man=8))
    f_cs = fo - fnd + fnc
    err = np.linalg.norm(f.cpu().numpy() - f_cs) / np.linalg.norm(f_cs)
    assert err < 1e-4, err
    assert abs(e["U_near"] - unc) <= 1e-5 * N
    assert np.linalg.norm(fnc - fnd) <= 1e-5 * np.linalg.norm(fnd)    # the scheme vs the direct sums
    B.rbsog_set_profiling(g.ctx, True)
    g.step(2)
    assert "near_fp32c_coreshell" in B.rbsog_get_profile(g.ctx)
    g.close()
    bad = Pk.make_params(L, P, n_ksets=2, precision="fp64", near_kernel="coreshell")
    with pytest.raises(B.RBSOGError):
        Pk.RBSOG(N, bad, device=0)
