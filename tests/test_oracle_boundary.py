"""Pins of the oracle's zero-frequency (boundary) terms (Sec. 3.2):

  * the spherical term (Eq. 3.14) is what a lattice sum taken in growing
    spheres of images adds to the tinfoil Ewald energy (an independent
    Ewald written in the tests);
  * the planar term (Eq. 3.15) is what a sum taken plate by plate (images
    summed over ever wider discs in the xy plane, a few layers in z) adds;
  * both equal the k -> 0 limit of Eq. 3.13 written as a pair sum,
    -(pi/V) sum_ij q_i q_j (k.r_ij)^2 / k^2 averaged over directions or taken
    along z (neutral systems);
  * the forces are minus the gradients of the energies."""
import math

import numpy as np
import pytest

import oracle as O
from tests._util import ewald


def _system(n, L, seed):
    rng = np.random.default_rng(seed)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    x = rng.uniform(0.0, L, size=(n, 3))
    return q, x


def _image_energies(q, x, L, n_img):
    """Energy of the cell with each image cell n (pairs i, j; i = j skipped
    for n = 0), one value per image."""
    d = x[:, None, :] - x[None, :, :]
    e = np.zeros(len(n_img))
    for i in range(len(q)):
        for j in range(len(q)):
            r = np.linalg.norm(d[i, j][None, :] + n_img * L, axis=1)
            if i == j:
                r[np.all(n_img == 0, axis=1)] = np.inf
            e += 0.5 * q[i] * q[j] / r
    return e


def test_spherical_term_is_the_spherical_lattice_sum_minus_tinfoil():
    L = 5.0
    q, x = _system(4, L, 3)
    R = 40
    r1 = np.arange(-R, R + 1)
    n = np.stack(np.meshgrid(r1, r1, r1, indexing="ij"), -1).reshape(-1, 3)
    n = n[np.sum(n * n, axis=1) <= R * R]
    U_sph = np.sum(_image_energies(q, x, L, n))
    U_tin, _ = ewald(q, x, L)
    U0, _ = O.boundary(q, x, L, 1)
    assert abs(U_sph - (U_tin + U0)) < 1e-6 * abs(U_tin + U0)
    assert abs(U_sph - U_tin) > 0.05 * abs(U_tin)          # the term is not small here


def test_planar_term_is_the_plate_by_plate_lattice_sum_minus_tinfoil():
    L = 5.0
    q, x = _system(4, L, 3)

    def plates(R, Z):
        r1 = np.arange(-R, R + 1)
        nxy = np.stack(np.meshgrid(r1, r1, indexing="ij"), -1).reshape(-1, 2)
        nxy = nxy[np.sum(nxy * nxy, axis=1) <= R * R]
        tot = 0.0
        for nz in range(-Z, Z + 1):
            n = np.concatenate([nxy, np.full((len(nxy), 1), nz)], axis=1)
            tot += np.sum(_image_energies(q, x, L, n))
        return tot

    # discs of radius R: the partial sums approach their limit as 1/R
    U_pl = 2.0 * plates(300, 2) - plates(150, 2)
    U_tin, _ = ewald(q, x, L)
    U0, _ = O.boundary(q, x, L, 2)
    assert abs(U_pl - (U_tin + U0)) < 1e-4 * abs(U_tin + U0)
    U0s, _ = O.boundary(q, x, L, 1)
    assert abs(U_pl - (U_tin + U0s)) > 0.1 * abs(U_tin)   # not the spherical term


@pytest.mark.parametrize("kind", [1, 2])
def test_boundary_terms_equal_the_k_to_zero_pair_sum(kind):
    L = (9.0, 11.0, 13.0)
    q, x = _system(40, 9.0, 5)
    V = L[0] * L[1] * L[2]
    d = x[:, None, :] - x[None, :, :]
    qq = q[:, None] * q[None, :]
    if kind == 1:
        avg = np.sum(d * d, axis=2) / 3.0       # direction average of (k.r)^2 / k^2
    else:
        avg = d[:, :, 2] ** 2                    # k along z
    U_pair = -math.pi / V * np.sum(qq * avg)
    U0, _ = O.boundary(q, x, L, kind, lB=1.0)
    assert U0 == pytest.approx(U_pair, rel=1e-12)
    U1, _ = O.boundary(q, x, L, kind, lB=0.7)
    assert U1 == pytest.approx(0.7 * U0, rel=1e-15)
    # neutral: a common shift of all positions changes nothing
    U2, _ = O.boundary(q, x + np.array([0.3, -1.1, 2.5]), L, kind)
    assert U2 == pytest.approx(U0, rel=1e-12)


@pytest.mark.parametrize("kind", [1, 2])
def test_boundary_force_is_minus_grad_energy(kind):
    L = 10.0
    q, x = _system(10, L, 7)
    _, f = O.boundary(q, x, L, kind)
    h = 1e-5
    for i in (0, 3, 8):
        for dd in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, dd] += h
            xm[i, dd] -= h
            fd = -(O.boundary(q, xp, L, kind)[0] - O.boundary(q, xm, L, kind)[0]) / (2 * h)
            assert f[i, dd] == pytest.approx(fd, rel=1e-7, abs=1e-10)
    assert np.allclose(f.sum(0), 0.0, atol=1e-12)   # neutral: no net force
    U0, f0 = O.boundary(q, x, L, 0)
    assert U0 == 0.0 and not f0.any()
