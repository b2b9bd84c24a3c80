"""Shared helpers for the tests: parameter sets and a textbook Ewald sum.

The Ewald routines here are an independent check of the oracle (a different
kernel split of 1/r), written from the standard Ewald formulas."""
from __future__ import annotations

import math
import os

import numpy as np
from scipy.special import erfc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Table 1, row 3 (eps ~ 1.1e-5); production kernel of the electrolyte runs.
B_PROD = 1.48783512395703226
# Table 1, row 5 b value (eps ~ 4e-11); used for tight checks.
B_TIGHT = 1.21812525709410644
M_PROD = 36


def untruncated_M(b: float) -> int:
    """Number of terms after which b^{-l} < 1e-40 (the series is untruncated
    for any FP64 purpose)."""
    return int(math.ceil(40 * math.log(10) / math.log(b)))


def table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            b, sg, w0, eps, M, ok = line.split()
            rows.append(dict(b=float(b), sigma=float(sg), w0=float(w0), eps=float(eps), M=int(M),
                             reproducible=bool(int(ok))))
    return rows


def prod_sog(O, rc=3.0, M=M_PROD, b=B_PROD):
    """Solve sigma, w0 with the untruncated series, then keep l = 0..M."""
    s = O.SOG.solve(b, rc, untruncated_M(b))
    return O.SOG(b, s.sigma, s.omega0, M)


def tight_sog(O, rc=3.0):
    s = O.SOG.solve(B_TIGHT, rc, untruncated_M(B_TIGHT))
    return O.SOG(B_TIGHT, s.sigma, s.omega0, untruncated_M(B_TIGHT))


def ewald(q, x, L, tol=1e-17):
    """Tinfoil Ewald energy and forces of point charges in a cubic box L
    (alpha = 6/L, real-space images within one box, reciprocal sum over
    exp(-k^2/4alpha^2) > tol)."""
    q = np.asarray(q, float)
    x = np.asarray(x, float)
    n = len(q)
    V = L ** 3
    alpha = 6.0 / L
    U = 0.0
    f = np.zeros((n, 3))
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], float) * L
    for i in range(n):
        d = x[i][None, None, :] - x[None, :, :] + shifts[:, None, :]   # r_i - r_j + nL
        r = np.linalg.norm(d, axis=2)
        mask = r > 0
        rr = np.where(mask, r, 1.0)
        qq = q[i] * q[None, :]
        e = np.where(mask, erfc(alpha * rr) / rr, 0.0)
        U += 0.5 * np.sum(qq * e)
        g = np.where(mask, (erfc(alpha * rr) / rr + 2 * alpha / math.sqrt(math.pi)
                            * np.exp(-(alpha * rr) ** 2)) / rr ** 2, 0.0)
        f[i] += np.sum((qq * g)[:, :, None] * d, axis=(0, 1))
    kcut = 2 * alpha * math.sqrt(math.log(1 / tol))
    mm = int(math.ceil(kcut * L / (2 * math.pi)))
    r1 = np.arange(-mm, mm + 1)
    m = np.stack(np.meshgrid(r1, r1, r1, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k = 2 * math.pi * m / L
    k2 = np.sum(k * k, axis=1)
    keep = k2 <= kcut ** 2
    k, k2 = k[keep], k2[keep]
    g = np.exp(-k2 / (4 * alpha ** 2)) / k2
    th = x @ k.T                                   # [n, K]
    rho = (q[:, None] * np.exp(1j * th)).sum(0)    # [K]
    U += 2 * math.pi / V * np.sum(g * np.abs(rho) ** 2)
    im = np.cos(th) * rho.imag[None, :] - np.sin(th) * rho.real[None, :]
    f += -(4 * math.pi / V) * q[:, None] * ((g[None, :] * im) @ k)
    U -= alpha / math.sqrt(math.pi) * np.sum(q ** 2)
    return U, f


def nacl(n_side: int, a: float):
    """Rock-salt lattice with n_side^3 ions (n_side even), spacing a."""
    idx = np.array([[i, j, k] for i in range(n_side) for j in range(n_side) for k in range(n_side)])
    q = np.where(idx.sum(1) % 2 == 0, 1.0, -1.0)
    return q, (idx + 0.5) * a


def rms_rel(a, b):
    """Global RMS relative error sqrt(sum |a_i - b_i|^2 / sum |b_i|^2)."""
    return math.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))


def per_particle_rel(a, b):
    """Per-particle relative force errors |a_i - b_i| / (|b_i| + median_j |b_j|):
    the median in the denominator keeps particles whose force nearly cancels
    from reading as large relative errors, while one particle off by a
    fraction of a typical force still shows.  Returns (median, max)."""
    nb = np.linalg.norm(b, axis=1)
    e = np.linalg.norm(a - b, axis=1) / (nb + np.median(nb))
    return float(np.median(e)), float(e.max())


# per-particle bars: FP64 within 1e-9 of a typical force at every particle;
# FP32C within 1e-4 (the combined near table's worst case is 6.1e-7 of G(0),
# the far field's 24-bit angles and hardware sin/cos about 1e-6 per term)
PP_FP64 = 1e-9
PP_FP32C = 1e-4


def oracle_kseq(O, g, sog, L, seed, nsets):
    """The oracle's own sampling of the first nsets k-sets for a device
    context's chain layout (seed, chains of chain_len); it is the input the
    oracle's trajectory takes, and it equals the device's sequence bit for
    bit (checked here as well)."""
    info = g.info()[0]
    Lv = (L,) * 3 if isinstance(L, (int, float)) else tuple(L)
    ks = O.kseq(sog, Lv, seed=seed, n_chains=info.n_chains, chain_len=info.chain_len)
    P = info.P_set
    assert np.array_equal(g.kseq(0, nsets), ks[: nsets * P])
    return ks
