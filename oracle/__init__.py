"""FP64 CPU oracle for the RBSOG force evaluation (arXiv:2205.13824).

TEST INFRASTRUCTURE ONLY.  This package is the reference the CUDA path is
checked against: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
product package ``paper_2205_13824_gb300`` and never imports it.

The arithmetic lives in ``rbsog_oracle.c`` (plain C, FP64, OpenMP over
independent outer loops); this module compiles it on first use and exposes
numpy-level wrappers.  Every wrapper names the passage of the paper it follows
in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbsog_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborcl.so")
_lock = threading.Lock()
_lib = None

_d = C.c_double
_i32 = C.c_int32
_i64 = C.c_int64
_u64 = C.c_uint64
_pd = C.POINTER(C.c_double)
_pi32 = C.POINTER(C.c_int32)


class OrcSys(C.Structure):
    _fields_ = [("L", _d * 3), ("M", _i32), ("omega", _pd), ("s", _pd), ("rc", _d),
                ("lB", _d), ("wca_sigma", _d), ("wca_eps", _d)]


class OrcCoreShell(C.Structure):
    _fields_ = [("r_in", _d), ("Q", _i32), ("b_exp", _i32), ("b_man", _i32)]


class OrcEnergies(C.Structure):
    _fields_ = [("U_near", _d), ("U_far", _d), ("U_self", _d), ("U_wca", _d), ("K", _d), ("T", _d),
                ("U_th", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborcl.so`` (gcc, -O2, OpenMP,
    no FP contraction so x86 and Arm hosts agree bit for bit)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "rbsog_oracle.h")))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_sog_coeffs.argtypes = [_d, _d, _i32, _pd, _pd]
            for fn in ("orc_sog_F", "orc_sog_dF"):
                getattr(L, fn).argtypes = [_pd, _pd, _i32, _d]
                getattr(L, fn).restype = _d
            L.orc_sog_omega0.argtypes = [_d, _d, _i32, _d]
            L.orc_sog_omega0.restype = _d
            L.orc_sog_solve.argtypes = [_d, _d, _i32, _pd, _pd]
            L.orc_sog_solve.restype = C.c_int
            L.orc_bsa.argtypes = [_d, _d, _d]
            L.orc_bsa.restype = _d
            L.orc_ftilde.argtypes = [_pd, _pd, _i32, _d]
            L.orc_ftilde.restype = _d
            L.orc_H.argtypes = [_d, _d, C.c_int]
            L.orc_H.restype = _d
            L.orc_S.argtypes = [_pd, _pd, _i32, _pd]
            L.orc_S.restype = _d
            L.orc_proposal_q1.argtypes = [_i32, _d, _d]
            L.orc_proposal_q1.restype = _d
            L.orc_philox4x64_10.argtypes = [C.POINTER(_u64), C.POINTER(_u64), C.POINTER(_u64)]
            L.orc_mh_chain.argtypes = [_pd, _pd, _i32, _pd, _u64, _u64, _i64, _pi32]
            L.orc_mh_chain.restype = _i64
            L.orc_kseq.argtypes = [_pd, _pd, _i32, _pd, _u64, _i64, _i64, _pi32]
            L.orc_kseq.restype = _i64
            L.orc_wrap.argtypes = [_i64, _pd, _pd]
            L.orc_cell_list.argtypes = [_i64, _pd, _pd, _d, _pi32, _pi32, _pi32, _pi32]
            L.orc_cell_list.restype = C.c_int
            near = [_i64, _pd, _pd, C.POINTER(OrcSys), _pd, _pd, _pd, _pi32]
            L.orc_near_direct.argtypes = near
            L.orc_near_cells.argtypes = near
            L.orc_near_cells.restype = C.c_int
            L.orc_far_exact.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _d, _pd, _pd]
            L.orc_far_exact.restype = _i64
            L.orc_rho.argtypes = [_i64, _pd, _pd, _pd, _i32, _pi32, _pd]
            L.orc_far_rb.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _pd, _pd, _pd]
            L.orc_forces_sample.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _i64,
                                            C.POINTER(_i64), _pd]
            L.orc_forces_sample.restype = C.c_int
            L.orc_self_energy.argtypes = [_i64, _pd, C.POINTER(OrcSys)]
            L.orc_self_energy.restype = _d
            L.orc_coreshell_eval.argtypes = [C.POINTER(OrcSys), C.POINTER(OrcCoreShell), _d, C.POINTER(_d),
                                             C.POINTER(_d)]
            L.orc_coreshell_eval.restype = C.c_int
            L.orc_near_coreshell.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), C.POINTER(OrcCoreShell), _pd,
                                             C.POINTER(_d), C.POINTER(_d)]
            L.orc_near_coreshell.restype = C.c_int
            L.orc_virial.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _pd]
            L.orc_virial.restype = C.c_int
            L.orc_boundary.argtypes = [_i64, _pd, _pd, _pd, _d, _i32, _pd]
            L.orc_boundary.restype = _d
            L.orc_forces.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _pd,
                                     C.POINTER(OrcEnergies)]
            L.orc_forces.restype = C.c_int
            L.orc_md.argtypes = [_i64, _pd, _pd, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _i64,
                                 _d, _d, _d, _d, C.c_int, C.POINTER(OrcEnergies)]
            L.orc_md.restype = C.c_int
            L.orc_md_thermo.argtypes = [_i64, _pd, _pd, _pd, _pd, C.POINTER(OrcSys), _d, _i32, _pi32, _i64,
                                        _d, _d, _d, _d, C.c_int, C.POINTER(OrcEnergies), _i32, _u64, _i64]
            L.orc_md_thermo.restype = C.c_int
            L.orc_langevin_noise.argtypes = [_u64, _i64, _i64, _pd]
            L.orc_rdf_counts.argtypes = [_i64, _pd, _pd, _d, _i32, C.POINTER(_u64)]
            L.orc_rdf_counts.restype = C.c_int
            L.orc_rdf_g.argtypes = [C.POINTER(_u64), _i32, _d, _i64, _i64, _pd]
            L.orc_msd_vacf.argtypes = [_i64, _i64, _pd, _pd, _pd, _i32, _i32, _pd, _pd, C.POINTER(_i64)]
            L.orc_msd_vacf.restype = C.c_int
            L.orc_pressure.argtypes = [_i64, _pd, _pd, _pd, _d, C.POINTER(OrcSys), _d, _i32, _pi32, _pd]
            L.orc_pressure.restype = C.c_int
            L.orc_green_kubo.argtypes = [_i64, _pd, _d, _d, _d, _i32, _pd, C.POINTER(_d)]
            L.orc_green_kubo.restype = C.c_int
            L.orc_heat_flux.argtypes = [_i64, _pd, _pd, _pd, _d, C.POINTER(OrcSys), _d, _i32, _pi32, _pd, _pd,
                                        _pd]
            L.orc_heat_flux.restype = C.c_int
            L.orc_green_kubo_heat.argtypes = [_i64, _pd, _d, _d, _d, _i32, _pd, C.POINTER(_d)]
            L.orc_green_kubo_heat.restype = C.c_int
            L.orc_pg_plan.argtypes = [_pd, _pd, _i32, _pd, _i32, _pi32, _pd]
            L.orc_pg_plan.restype = _i32
            L.orc_pg_kseq.argtypes = [_pd, _pd, _i32, _pd, _i32, _u64, _i64, _i64, _pi32, _pi32]
            L.orc_pg_kseq.restype = C.c_int
            L.orc_far_rb_w.argtypes = [_i64, _pd, _pd, C.POINTER(OrcSys), _i32, _pi32, _pd, _pd, C.POINTER(_d)]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            L.orc_set_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a, ct=_pd):
    return a.ctypes.data_as(ct)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- SOG (Sec. 2)

class SOG:
    """Sum-of-Gaussians far kernel F_M(r) = sum_{l=0}^{M} w_l exp(-r^2/s_l^2)
    (Eqs. 2.8-2.9) with the C0/C1-tuned narrowest weight w_0 (Eq. 2.11)."""

    def __init__(self, b: float, sigma: float, omega0: float, M: int):
        self.b, self.sigma, self.omega0, self.M = float(b), float(sigma), float(omega0), int(M)
        self.omega = np.zeros(M + 1)
        self.s = np.zeros(M + 1)
        lib().orc_sog_coeffs(self.b, self.sigma, self.M, _p(self.omega), _p(self.s))
        self.omega_bsa0 = float(self.omega[0])
        self.omega[0] = self.omega0

    @classmethod
    def solve(cls, b: float, rc: float, M: int) -> "SOG":
        sig, w0 = _d(), _d()
        rc_ = lib().orc_sog_solve(float(b), float(rc), int(M), C.byref(sig), C.byref(w0))
        if rc_ != 0:
            raise ValueError("no C0/C1 root for these (b, r_c, M)")
        return cls(b, sig.value, w0.value, M)

    def F(self, r):
        return np.array([lib().orc_sog_F(_p(self.omega), _p(self.s), self.M, float(x))
                         for x in np.atleast_1d(r)])

    def dF(self, r):
        return np.array([lib().orc_sog_dF(_p(self.omega), _p(self.s), self.M, float(x))
                         for x in np.atleast_1d(r)])

    def ftilde(self, k2):
        return np.array([lib().orc_ftilde(_p(self.omega), _p(self.s), self.M, float(x))
                         for x in np.atleast_1d(k2)])

    def S(self, L):
        L = _f64(L)
        return lib().orc_S(_p(self.omega), _p(self.s), self.M, _p(L))


def sog_omega0(b, sigma, M, rc):
    return lib().orc_sog_omega0(float(b), float(sigma), int(M), float(rc))


def bsa(b, sigma, r):
    return lib().orc_bsa(float(b), float(sigma), float(r))


def H(s, L, dual=-1):
    return lib().orc_H(float(s), float(L), int(dual))


def proposal_q1(m, s0, Ld):
    return lib().orc_proposal_q1(int(m), float(s0), float(Ld))


# ----------------------------------------------------------- sampler (Sec. 3.3)

def philox4x64_10(ctr, key):
    c = (_u64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (_u64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (_u64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def mh_chain(sog: SOG, L, seed: int, chain: int, length: int):
    L = _f64(L)
    out = np.zeros((length, 3), dtype=np.int32)
    it = lib().orc_mh_chain(_p(sog.omega), _p(sog.s), sog.M, _p(L), int(seed), int(chain),
                            int(length), _p(out, _pi32))
    if it < 0:
        raise RuntimeError("MH chain failed to start")
    return out, int(it)


def kseq(sog: SOG, L, seed: int, n_chains: int, chain_len: int):
    """Frequency sequence of Algorithm 1 from n_chains independent chains."""
    L = _f64(L)
    out = np.zeros((n_chains * chain_len, 3), dtype=np.int32)
    it = lib().orc_kseq(_p(sog.omega), _p(sog.s), sog.M, _p(L), int(seed), int(n_chains),
                        int(chain_len), _p(out, _pi32))
    if it < 0:
        raise RuntimeError("MH chain failed to start")
    return out


# ------------------------------------------------------------ forces (Sec. 3)

class System:
    """Box, SOG kernel, cutoff and pair parameters for the force routines."""

    def __init__(self, L, sog: SOG, rc: float, lB: float = 1.0, wca_sigma: float = 0.0,
                 wca_eps: float = 0.0):
        self.L = _f64(L)
        self.sog = sog
        self.rc, self.lB = float(rc), float(lB)
        self.c = OrcSys((_d * 3)(*self.L), sog.M, _p(sog.omega), _p(sog.s), self.rc, self.lB,
                        float(wca_sigma), float(wca_eps))

    @property
    def V(self):
        return float(np.prod(self.L))

    def S(self):
        return self.sog.S(self.L)


def wrap(x, L):
    x = _f64(x).copy()
    L = _f64(L)
    lib().orc_wrap(x.shape[0], _p(x), _p(L))
    return x


def cell_list(x, L, rc):
    x = _f64(x)
    L = _f64(L)
    n = x.shape[0]
    nc = np.zeros(3, dtype=np.int32)
    ncmax = int(np.prod(np.maximum(np.floor(L / rc), 1)))
    cell_of = np.zeros(n, dtype=np.int32)
    start = np.zeros(ncmax + 1, dtype=np.int32)
    perm = np.zeros(n, dtype=np.int32)
    if lib().orc_cell_list(n, _p(x), _p(L), float(rc), _p(nc, _pi32), _p(cell_of, _pi32),
                           _p(start, _pi32), _p(perm, _pi32)) != 0:
        raise ValueError("fewer than 3 cells per side")
    return nc, cell_of, start, perm


def near(sys_: System, q, x, method="cells"):
    q, x = _f64(q), _f64(x)
    n = x.shape[0]
    f = np.zeros((n, 3))
    un, uw = _d(), _d()
    nbr = np.zeros(n, dtype=np.int32)
    if method == "direct":
        lib().orc_near_direct(n, _p(q), _p(x), C.byref(sys_.c), _p(f), C.byref(un), C.byref(uw),
                              _p(nbr, _pi32))
    else:
        if lib().orc_near_cells(n, _p(q), _p(x), C.byref(sys_.c), _p(f), C.byref(un),
                                C.byref(uw), _p(nbr, _pi32)) != 0:
            raise ValueError("fewer than 3 cells per side")
    return f, un.value, uw.value, nbr


def coreshell(r_in: float, Q: int = 10, b_exp: int = 2, b_man: int = 8) -> OrcCoreShell:
    """Parameters of the core-shell near-field kernel (Sec. 3.4)."""
    return OrcCoreShell(float(r_in), int(Q), int(b_exp), int(b_man))


def coreshell_eval(sys_: System, cs: OrcCoreShell, r2: float):
    """(g, n): the scheme's force factor and pair energy kernel at r^2."""
    g, n = _d(), _d()
    if lib().orc_coreshell_eval(C.byref(sys_.c), C.byref(cs), float(r2), C.byref(g), C.byref(n)) != 0:
        raise ValueError("r^2 outside [0, r_c^2) or the table does not reach r_c^2")
    return g.value, n.value


def near_coreshell(sys_: System, q, x, cs: OrcCoreShell):
    """Near field (+ WCA) with the core-shell kernel: (f, U_near, U_wca)."""
    q, x = _f64(q), _f64(x)
    f = np.zeros_like(x)
    un, uw = _d(), _d()
    if lib().orc_near_coreshell(x.shape[0], _p(q), _p(x), C.byref(sys_.c), C.byref(cs), _p(f), C.byref(un),
                                C.byref(uw)) != 0:
        raise ValueError("the core-shell table does not reach r_c^2")
    return f, un.value, uw.value


def far_exact(sys_: System, q, x, tol=1e-16):
    q, x = _f64(q), _f64(x)
    f = np.zeros((x.shape[0], 3))
    U = _d()
    lib().orc_far_exact(x.shape[0], _p(q), _p(x), C.byref(sys_.c), float(tol), _p(f), C.byref(U))
    return f, U.value


def rho(q, x, L, m):
    q, x, L, m = _f64(q), _f64(x), _f64(L), _i32a(m)
    out = np.zeros((m.shape[0], 2))
    lib().orc_rho(x.shape[0], _p(q), _p(x), _p(L), m.shape[0], _p(m, _pi32), _p(out))
    return out[:, 0] + 1j * out[:, 1]


def far_rb(sys_: System, q, x, S, m):
    q, x, m = _f64(q), _f64(x), _i32a(m)
    f = np.zeros((x.shape[0], 3))
    U = _d()
    r = np.zeros((m.shape[0], 2))
    lib().orc_far_rb(x.shape[0], _p(q), _p(x), C.byref(sys_.c), float(S), m.shape[0],
                     _p(m, _pi32), _p(f), C.byref(U), _p(r))
    return f, U.value, r[:, 0] + 1j * r[:, 1]


def forces_sample(sys_: System, q, x, S, m, idx):
    """Random-batch total force on the particles idx only (rho over all)."""
    q, x, m = _f64(q), _f64(x), _i32a(m)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = np.zeros((len(idx), 3))
    if lib().orc_forces_sample(x.shape[0], _p(q), _p(x), C.byref(sys_.c), float(S), m.shape[0],
                               _p(m, _pi32), len(idx), _p(idx, C.POINTER(_i64)), _p(f)) != 0:
        raise ValueError("fewer than 3 cells per side")
    return f


def self_energy(sys_: System, q):
    q = _f64(q)
    return lib().orc_self_energy(q.shape[0], _p(q), C.byref(sys_.c))


def virial(sys_: System, q, x, S=0.0, m=None):
    """Configurational virial tensor W[3, 3] = -dU/d eps: near (+ WCA) plus
    the random-batch far estimator on k-set m, or the exact far sum (m None)."""
    q, x = _f64(q), _f64(x)
    W = np.zeros(9)
    if m is None:
        lib().orc_virial(x.shape[0], _p(q), _p(x), C.byref(sys_.c), float(S), 0, None, _p(W))
    else:
        m = _i32a(m)
        lib().orc_virial(x.shape[0], _p(q), _p(x), C.byref(sys_.c), float(S), m.shape[0], _p(m, _pi32), _p(W))
    return W.reshape(3, 3)


def pg_plan(sog: SOG, L, P: int):
    """Per-Gaussian sampling plan: (P_eff, P_l[M + 1], S_l[M + 1])."""
    Lv = _f64(np.broadcast_to(np.asarray(L, float), (3,)).copy())
    P_l = np.zeros(sog.M + 1, dtype=np.int32)
    S_l = np.zeros(sog.M + 1)
    pe = lib().orc_pg_plan(_p(sog.omega), _p(sog.s), sog.M, _p(Lv), int(P), _p(P_l, _pi32), _p(S_l))
    if pe < 0:
        raise ValueError("sampling table too long")
    return int(pe), P_l, S_l


def pg_kseq(sog: SOG, L, P: int, seed: int, set0: int, n_sets: int):
    """Per-Gaussian k-sets: (m[n_sets * P_eff, 3], stratum[n_sets * P_eff])."""
    pe, _, _ = pg_plan(sog, L, P)
    Lv = _f64(np.broadcast_to(np.asarray(L, float), (3,)).copy())
    m = np.zeros((n_sets * pe, 3), dtype=np.int32)
    st = np.zeros(n_sets * pe, dtype=np.int32)
    if lib().orc_pg_kseq(_p(sog.omega), _p(sog.s), sog.M, _p(Lv), int(P), int(seed), int(set0), int(n_sets),
                         _p(m, _pi32), _p(st, _pi32)):
        raise ValueError("sampling table too long")
    return m, st


def pg_weights(sog: SOG, L, P: int):
    """Weight S_l / P_l of every frequency of one per-Gaussian set (length P_eff)."""
    pe, P_l, S_l = pg_plan(sog, L, P)
    return np.concatenate([np.full(P_l[l], S_l[l] / P_l[l]) for l in range(sog.M + 1) if P_l[l] > 0])


def far_rb_w(sys_: System, q, x, m, c):
    """Eq. 3.24 with per-frequency weights c (c = S / P everywhere is far_rb); returns (f, U)."""
    q, x = _f64(q), _f64(x)
    m = _i32a(m)
    c = _f64(c)
    f = np.zeros_like(x)
    U = _d(0.0)
    lib().orc_far_rb_w(x.shape[0], _p(q), _p(x), C.byref(sys_.c), m.shape[0], _p(m, _pi32), _p(c), _p(f),
                       C.byref(U))
    return f, U.value


def msd_vacf(x_frames, v_frames, L, n_lags: int, origin_every: int = 1):
    """Appendix A's MSD and VACF over frames x[f, n, 3] (folded positions)
    and v[f, n, 3], averaged over particles and the time origins 0,
    origin_every, ...; returns (msd[n_lags], vacf[n_lags], count[n_lags])."""
    x, v = _f64(x_frames), _f64(v_frames)
    Lv = _f64(np.broadcast_to(np.asarray(L, float), (3,)).copy())
    msd, vacf = np.zeros(n_lags), np.zeros(n_lags)
    cnt = np.zeros(n_lags, dtype=np.int64)
    if lib().orc_msd_vacf(x.shape[1], x.shape[0], _p(x), _p(v), _p(Lv), int(n_lags), int(origin_every),
                          _p(msd), _p(vacf), cnt.ctypes.data_as(C.POINTER(_i64))):
        raise ValueError("bad sizes")
    return msd, vacf, cnt


def pressure(sys_: System, q, x, v, mass, S, m):
    """Pressure tensor (1/V) sum (m v v + r f) of Appendix A, the virial part
    the random-batch estimate on k-set m (or exact for m None)."""
    q, x, v = _f64(q), _f64(x), _f64(v)
    Pt = np.zeros(9)
    if m is None:
        rc_ = lib().orc_pressure(x.shape[0], _p(q), _p(x), _p(v), float(mass), C.byref(sys_.c), float(S), 0,
                                 None, _p(Pt))
    else:
        m = _i32a(m)
        rc_ = lib().orc_pressure(x.shape[0], _p(q), _p(x), _p(v), float(mass), C.byref(sys_.c), float(S),
                                 m.shape[0], _p(m, _pi32), _p(Pt))
    if rc_:
        raise ValueError("fewer than 3 cells per side")
    return Pt.reshape(3, 3)


def green_kubo(P_series, dt, V, T, max_lag):
    """Green-Kubo viscosity of Appendix A from a pressure-tensor series
    [n, 3, 3]; returns (acf[max_lag] summed over a <= b, C)."""
    Pt = _f64(np.asarray(P_series, float).reshape(-1, 9))
    acf = np.zeros(int(max_lag))
    Cv = _d(0.0)
    if lib().orc_green_kubo(Pt.shape[0], _p(Pt), float(dt), float(V), float(T), int(max_lag), _p(acf),
                            C.byref(Cv)):
        raise ValueError("bad sizes")
    return acf, Cv.value


def heat_flux(sys_: System, q, x, v, mass, S=0.0, m=None):
    """Heat flux of Appendix A (orc_heat_flux in the C source): returns
    (J[3], per-atom energies e[n], per-atom virials W[n, 3, 3]); m None: no
    far term (near field, WCA, kinetic and self terms only)."""
    q, x, v = _f64(q), _f64(x), _f64(v)
    n = x.shape[0]
    J = np.zeros(3)
    e = np.zeros(n)
    W = np.zeros((n, 9))
    if m is None:
        rc_ = lib().orc_heat_flux(n, _p(q), _p(x), _p(v), float(mass), C.byref(sys_.c), 0.0, 0, None, _p(J),
                                  _p(e), _p(W))
    else:
        m = _i32a(m)
        rc_ = lib().orc_heat_flux(n, _p(q), _p(x), _p(v), float(mass), C.byref(sys_.c), float(S), m.shape[0],
                                  _p(m, _pi32), _p(J), _p(e), _p(W))
    if rc_:
        raise ValueError("fewer than 3 cells per side")
    return J, e, W.reshape(n, 3, 3)


def green_kubo_heat(J_series, dt, V, T, max_lag):
    """Green-Kubo heat conductivity of Appendix A from a heat-flux series
    [n, 3]; returns (acf[max_lag], C)."""
    J = _f64(np.asarray(J_series, float).reshape(-1, 3))
    acf = np.zeros(int(max_lag))
    Cv = _d(0.0)
    if lib().orc_green_kubo_heat(J.shape[0], _p(J), float(dt), float(V), float(T), int(max_lag), _p(acf),
                                 C.byref(Cv)):
        raise ValueError("bad sizes")
    return acf, Cv.value


def boundary(q, x, L, kind: int, lB: float = 1.0):
    """Zero-frequency term (Sec. 3.2): kind 1 spherical (Eq. 3.14), 2
    planar along z (Eq. 3.15), 0 tinfoil.  Returns (U0, force [n, 3])."""
    q, x = _f64(q), _f64(x)
    Lv = _f64(np.broadcast_to(np.asarray(L, float), (3,)).copy())
    f = np.zeros_like(x)
    U = lib().orc_boundary(q.shape[0], _p(q), _p(x), _p(Lv), float(lB), int(kind), _p(f))
    return U, f


def forces(sys_: System, q, x, S=0.0, m=None):
    """Total force and energies; m = None uses the exact far sum."""
    q, x = _f64(q), _f64(x)
    n = x.shape[0]
    f = np.zeros((n, 3))
    e = OrcEnergies()
    if m is None:
        rc_ = lib().orc_forces(n, _p(q), _p(x), C.byref(sys_.c), 0.0, 0, None, _p(f), C.byref(e))
    else:
        m = _i32a(m)
        rc_ = lib().orc_forces(n, _p(q), _p(x), C.byref(sys_.c), float(S), m.shape[0],
                               _p(m, _pi32), _p(f), C.byref(e))
    if rc_ != 0:
        raise ValueError("fewer than 3 cells per side")
    return f, e.as_dict()


def langevin_noise(seed: int, t: int, i: int):
    z = np.zeros(3)
    lib().orc_langevin_noise(int(seed), int(t), int(i), _p(z))
    return z


def md(sys_: System, q, x, v, S, P, kseq_, nsteps, dt, mass=1.0, T0=1.0, tau=0.0, f=None, thermostat=0,
       seed=0, step0=0):
    """Velocity-Verlet run of Algorithm 1; returns (x, v, f, per-step energies).
    P = 0 uses the exact far sum (kseq_ ignored).  thermostat 1 (tau > 0):
    Langevin dynamics in the BAOAB splitting with noise keyed by seed and the
    step counter (starting at step0)."""
    q = _f64(q)
    x = _f64(x).copy()
    v = _f64(v).copy()
    n = x.shape[0]
    have = f is not None
    f = _f64(f).copy() if have else np.zeros((n, 3))
    es = (OrcEnergies * max(int(nsteps), 1))()
    ks = _i32a(kseq_ if kseq_ is not None else np.zeros((1, 3)))
    rc_ = lib().orc_md_thermo(n, _p(q), _p(x), _p(v), _p(f), C.byref(sys_.c), float(S), int(P),
                              _p(ks, _pi32), int(nsteps), float(dt), float(mass), float(T0), float(tau),
                              int(have), es, int(thermostat), int(seed), int(step0))
    if rc_ != 0:
        raise ValueError("fewer than 3 cells per side")
    return x, v, f, [es[t].as_dict() for t in range(int(nsteps))]


def rdf(q, x, L, nbins):
    """Appendix A: pair-distance histograms by sign pair (rows ++, +-, --) on
    [0, L/2) and the g(r) estimate; returns (counts[3, nbins] uint64,
    g[3, nbins], bin edges[nbins + 1])."""
    q, x = _f64(q), _f64(x)
    counts = np.zeros((3, nbins), dtype=np.uint64)
    if lib().orc_rdf_counts(x.shape[0], _p(q), _p(x), float(L), int(nbins), _p(counts, C.POINTER(_u64))):
        raise ValueError("nbins must be a power of two in [16, 4096] and L > 0")
    g = np.zeros((3, nbins))
    lib().orc_rdf_g(_p(counts, C.POINTER(_u64)), int(nbins), float(L), int((q > 0).sum()), int((q < 0).sum()),
                    _p(g))
    return counts, g, np.arange(nbins + 1) * (float(L) / (2 * nbins))


def num_threads():
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> int:
    """Threads for the oracle's parallel loops; returns the previous count."""
    return int(lib().orc_set_num_threads(int(n)))
