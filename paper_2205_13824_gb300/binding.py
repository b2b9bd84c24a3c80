"""ctypes binding of librbsog (include/rbsog.h): argument marshalling only.

Every ``rbsog_*`` function here has the name and argument order of the C
entry point; it converts torch tensors / numpy arrays to raw pointers and
raises ``RBSOGError`` on a non-zero status.  No arithmetic of the method
happens in Python: if the shared library is missing the import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbsog.so")

RBSOG_FP64 = 0
RBSOG_FP32C = 1
STATUS = {0: "RBSOG_OK", 1: "RBSOG_EINVAL", 2: "RBSOG_ENOMEM", 3: "RBSOG_ECUDA",
          4: "RBSOG_ESTATE", 5: "RBSOG_ENUMERIC", 6: "RBSOG_ETIMEOUT"}

# Every symbol include/rbsog.h declares.
EXPORTS = ("rbsog_create", "rbsog_set_params", "rbsog_get_info", "rbsog_set_state",
           "rbsog_compute_forces", "rbsog_step", "rbsog_get_state", "rbsog_get_energies",
           "rbsog_get_kseq", "rbsog_rho", "rbsog_get_cells", "rbsog_set_profiling",
           "rbsog_get_cursor", "rbsog_restore", "rbsog_step_io", "rbsog_compute_virial", "rbsog_rho_noalloc", "rbsog_measure_peaks",
           "rbsog_compute_pressure", "rbsog_observe_start", "rbsog_observe_sample", "rbsog_observe_result",
           "rbsog_green_kubo", "rbsog_compute_heat_flux", "rbsog_green_kubo_heat",
           "rbsog_batch_create", "rbsog_batch_set_params", "rbsog_batch_set_state", "rbsog_batch_restore",
           "rbsog_batch_get_state", "rbsog_batch_get_energies", "rbsog_batch_get_kseq", "rbsog_batch_step",
           "rbsog_batch_autotune", "rbsog_batch_rdf", "rbsog_rdf",
           "rbsog_server_create", "rbsog_server_submit", "rbsog_server_advance", "rbsog_server_result",
           "rbsog_server_release", "rbsog_server_cancel", "rbsog_server_last_error", "rbsog_server_destroy",
           "rbsog_get_profile", "rbsog_last_error", "rbsog_destroy")


class RBSOGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rbsog_params(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("b", C.c_double), ("sigma", C.c_double),
                ("omega0", C.c_double), ("M", C.c_int32), ("r_c", C.c_double), ("P", C.c_int32),
                ("coulomb_prefactor", C.c_double), ("wca_sigma", C.c_double),
                ("wca_eps", C.c_double), ("dt", C.c_double), ("mass", C.c_double),
                ("T_target", C.c_double), ("tau_T", C.c_double), ("seed", C.c_uint64),
                ("n_ksets", C.c_int64), ("chain_len", C.c_int32), ("precision", C.c_int32),
                ("boundary", C.c_int32), ("near_kernel", C.c_int32), ("r_in", C.c_double),
                ("thermostat", C.c_int32), ("sampler", C.c_int32)]


class rbsog_energies(C.Structure):
    _fields_ = [("U_near", C.c_double), ("U_far", C.c_double), ("U_self", C.c_double),
                ("U_wca", C.c_double), ("K", C.c_double), ("T", C.c_double), ("U_bound", C.c_double),
                ("U_th", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rbsog_info(C.Structure):
    _fields_ = [("sigma", C.c_double), ("omega0", C.c_double), ("S", C.c_double),
                ("M", C.c_int32), ("ncell", C.c_int32 * 3), ("n_chains", C.c_int64),
                ("chain_len", C.c_int32), ("P_set", C.c_int32), ("list_builds", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    st = C.c_int
    sig = {
        "rbsog_create": [C.POINTER(P), C.c_int64, C.c_int, P],
        "rbsog_set_params": [P, C.POINTER(rbsog_params)],
        "rbsog_get_info": [P, C.POINTER(rbsog_info), P, P],
        "rbsog_set_state": [P, P, P, P],
        "rbsog_compute_forces": [P, P, P, C.POINTER(rbsog_energies)],
        "rbsog_step": [P, C.c_int64],
        "rbsog_get_state": [P, P, P, P, C.POINTER(C.c_int64)],
        "rbsog_get_energies": [P, C.POINTER(rbsog_energies)],
        "rbsog_get_cursor": [P, C.POINTER(C.c_int64)],
        "rbsog_restore": [P, P, C.c_int64, C.c_int64],
        "rbsog_step_io": [P, P, P, P, P, C.c_int64, C.c_int64, C.c_int64, P, P, P],
        "rbsog_compute_virial": [P, P, C.c_int32, P],
        "rbsog_compute_pressure": [P, P, C.c_int32, P],
        "rbsog_observe_start": [P, C.c_int32, C.c_int32],
        "rbsog_observe_sample": [P],
        "rbsog_observe_result": [P, P, P, P],
        "rbsog_green_kubo": [P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int32, P,
                             C.POINTER(C.c_double), P],
        "rbsog_compute_heat_flux": [P, P, C.c_int32, P],
        "rbsog_green_kubo_heat": [P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int32, P,
                                  C.POINTER(C.c_double), P],
        "rbsog_get_kseq": [P, C.c_int64, C.c_int64, P],
        "rbsog_rho": [P, P, C.c_int32, P],
        "rbsog_get_cells": [P, P, P, P],
        "rbsog_set_profiling": [P, C.c_int],
        "rbsog_get_profile": [P, C.c_int32, P, P, P, C.POINTER(C.c_int32)],
        "rbsog_destroy": [P],
        "rbsog_rho_noalloc": [C.c_int64, P, P, C.POINTER(C.c_double), P, C.c_int32, P, P],
        "rbsog_measure_peaks": [C.c_int, P],
        "rbsog_batch_create": [C.POINTER(P), C.c_int32, P, C.c_int, P],
        "rbsog_batch_set_params": [P, P],
        "rbsog_batch_set_state": [P, C.c_int32, P, P, P],
        "rbsog_batch_restore": [P, C.c_int32, P, C.c_int64, C.c_int64],
        "rbsog_batch_get_state": [P, C.c_int32, P, P, P, C.POINTER(C.c_int64)],
        "rbsog_batch_get_energies": [P, C.c_int32, C.POINTER(rbsog_energies)],
        "rbsog_batch_get_kseq": [P, C.c_int32, C.c_int64, C.c_int64, P],
        "rbsog_batch_step": [P, C.c_int64],
        "rbsog_batch_autotune": [P, C.c_int32, P],
        "rbsog_batch_rdf": [P, C.c_int32, C.c_int32, P, P],
        "rbsog_rdf": [P, C.c_int32, P, P],
        "rbsog_server_create": [C.POINTER(P), C.c_int32, C.c_int64, C.c_int32, C.c_int, P],
        "rbsog_server_submit": [P, C.c_int64, C.POINTER(rbsog_params), P, P, P, C.c_int64,
                                C.POINTER(C.c_int64)],
        "rbsog_server_advance": [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "rbsog_server_result": [P, C.c_int64, C.POINTER(C.c_int32), P, P, P, C.POINTER(rbsog_energies),
                                C.POINTER(C.c_int64)],
        "rbsog_server_release": [P, C.c_int64],
        "rbsog_server_cancel": [P, C.c_int64],
        "rbsog_server_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = st
    lib.rbsog_last_error.argtypes = [P]
    lib.rbsog_last_error.restype = C.c_char_p
    lib.rbsog_server_last_error.argtypes = [P]
    lib.rbsog_server_last_error.restype = C.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def _ptr(a):
    """Raw address of a torch tensor, numpy array or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(ctx, status):
    if status != 0:
        msg = _lib.rbsog_last_error(ctx)
        raise RBSOGError(status, msg.decode() if msg else "")


def rbsog_create(n: int, device: int = 0, stream: int | None = None):
    ctx = C.c_void_p()
    s = _lib.rbsog_create(C.byref(ctx), int(n), int(device), stream)
    if s != 0:
        raise RBSOGError(s, "rbsog_create failed")
    return ctx


def rbsog_set_params(ctx, p: rbsog_params):
    _check(ctx, _lib.rbsog_set_params(ctx, C.byref(p)))


def rbsog_get_info(ctx, M: int | None = None):
    info = rbsog_info()
    om = s = None
    if M is not None:
        om = np.zeros(M + 1)
        s = np.zeros(M + 1)
    _check(ctx, _lib.rbsog_get_info(ctx, C.byref(info), _ptr(om), _ptr(s)))
    return info, om, s


def rbsog_set_state(ctx, q, x, v=None):
    _check(ctx, _lib.rbsog_set_state(ctx, _ptr(q), _ptr(x), _ptr(v)))


def rbsog_compute_forces(ctx, m_kset=None, f_out=None, want_energies=True):
    e = rbsog_energies() if want_energies else None
    _check(ctx, _lib.rbsog_compute_forces(ctx, _ptr(m_kset), _ptr(f_out),
                                          C.byref(e) if e is not None else None))
    return e.as_dict() if e is not None else None


def rbsog_step(ctx, nsteps: int):
    _check(ctx, _lib.rbsog_step(ctx, int(nsteps)))


def rbsog_get_state(ctx, x=None, v=None, f=None):
    step = C.c_int64()
    _check(ctx, _lib.rbsog_get_state(ctx, _ptr(x), _ptr(v), _ptr(f), C.byref(step)))
    return step.value


def rbsog_get_cursor(ctx):
    c = C.c_int64()
    _check(ctx, _lib.rbsog_get_cursor(ctx, C.byref(c)))
    return c.value


def rbsog_restore(ctx, f, kset_cursor: int, step: int):
    _check(ctx, _lib.rbsog_restore(ctx, _ptr(f), int(kset_cursor), int(step)))


def rbsog_step_io(ctx, q, x, v, f, kset_cursor: int, step: int, nsteps: int, x_out=None, v_out=None,
                  f_out=None):
    _check(ctx, _lib.rbsog_step_io(ctx, _ptr(q), _ptr(x), _ptr(v), _ptr(f), int(kset_cursor), int(step),
                                   int(nsteps), _ptr(x_out), _ptr(v_out), _ptr(f_out)))


def rbsog_compute_virial(ctx, m):
    """Virial tensor [3, 3] of the current positions with the far field on k-set m[P][3]."""
    m = np.ascontiguousarray(m, dtype=np.int32)
    W = np.zeros(9)
    _check(ctx, _lib.rbsog_compute_virial(ctx, _ptr(m), int(m.shape[0]), _ptr(W)))
    return W.reshape(3, 3)


def rbsog_compute_pressure(ctx, m):
    """Pressure tensor [3, 3] (kinetic + virial over V), the far field on k-set m[P][3]."""
    m = np.ascontiguousarray(m, dtype=np.int32)
    Pt = np.zeros(9)
    _check(ctx, _lib.rbsog_compute_pressure(ctx, _ptr(m), int(m.shape[0]), _ptr(Pt)))
    return Pt.reshape(3, 3)


def rbsog_compute_heat_flux(ctx, m=None):
    """Heat flux J[3] of Appendix A; the far term on k-set m[P][3], none for m None."""
    J = np.zeros(3)
    if m is None:
        _check(ctx, _lib.rbsog_compute_heat_flux(ctx, None, 0, _ptr(J)))
    else:
        m = np.ascontiguousarray(m, dtype=np.int32)
        _check(ctx, _lib.rbsog_compute_heat_flux(ctx, _ptr(m), int(m.shape[0]), _ptr(J)))
    return J


def rbsog_observe_start(ctx, n_lags: int, origin_every: int = 1):
    _check(ctx, _lib.rbsog_observe_start(ctx, int(n_lags), int(origin_every)))


def rbsog_observe_sample(ctx):
    _check(ctx, _lib.rbsog_observe_sample(ctx))


def rbsog_observe_result(ctx, n_lags: int):
    """(msd[n_lags], vacf[n_lags], count[n_lags]) accumulated since rbsog_observe_start."""
    msd, vacf = np.zeros(n_lags), np.zeros(n_lags)
    cnt = np.zeros(n_lags, dtype=np.int64)
    _check(ctx, _lib.rbsog_observe_result(ctx, _ptr(msd), _ptr(vacf), _ptr(cnt)))
    return msd, vacf, cnt


def rbsog_green_kubo(P_series, dt: float, V: float, T: float, max_lag: int, stream=None):
    """(acf[max_lag], C) of a pressure-tensor series [n, 3, 3] (host array or device tensor)."""
    if not hasattr(P_series, "data_ptr"):
        P_series = np.ascontiguousarray(np.asarray(P_series, dtype=np.float64).reshape(-1, 9))
    n = P_series.shape[0]
    acf = np.zeros(int(max_lag))
    Cv = C.c_double()
    st = _lib.rbsog_green_kubo(_ptr(P_series), int(n), float(dt), float(V), float(T), int(max_lag), _ptr(acf),
                               C.byref(Cv), C.c_void_p(stream))
    if st != 0:
        raise RBSOGError(st, "rbsog_green_kubo failed")
    return acf, Cv.value


def rbsog_get_energies(ctx):
    e = rbsog_energies()
    _check(ctx, _lib.rbsog_get_energies(ctx, C.byref(e)))
    return e.as_dict()


def rbsog_get_kseq(ctx, set0: int, nsets: int, m_out):
    _check(ctx, _lib.rbsog_get_kseq(ctx, int(set0), int(nsets), _ptr(m_out)))


def rbsog_rho(ctx, m, rho_out):
    P = int(m.shape[0])
    _check(ctx, _lib.rbsog_rho(ctx, _ptr(m), P, _ptr(rho_out)))


def rbsog_get_cells(ctx, cell_start=None, perm=None, nbr=None):
    _check(ctx, _lib.rbsog_get_cells(ctx, _ptr(cell_start), _ptr(perm), _ptr(nbr)))


def rbsog_set_profiling(ctx, on: bool):
    _check(ctx, _lib.rbsog_set_profiling(ctx, 1 if on else 0))


def rbsog_get_profile(ctx, cap: int = 64):
    names = (C.c_char * 32 * cap)()
    launches = np.zeros(cap, dtype=np.int64)
    ms = np.zeros(cap, dtype=np.float64)
    cnt = C.c_int32()
    _check(ctx, _lib.rbsog_get_profile(ctx, cap, C.cast(names, C.c_void_p), _ptr(launches),
                                       _ptr(ms), C.byref(cnt)))
    out = {}
    for i in range(min(cnt.value, cap)):
        out[bytes(names[i]).split(b"\0")[0].decode()] = (int(launches[i]), float(ms[i]))
    return out


RBSOG_NOALLOC_MAX_P = 2048


def _device_tensor(t, name, dtype, shape):
    """t must be a contiguous torch CUDA tensor on the current device with the
    given dtype and shape: the allocation-free entry point reads and writes
    raw device addresses, so a host array or a short buffer must not reach it."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: a torch CUDA tensor is required")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: tensor on cuda:{t.device.index}, current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    return t.data_ptr()


def rbsog_rho_noalloc(q, x, L, m, rho_out, stream=None):
    """rho(k) from caller-owned device buffers with no device allocation
    (see include/rbsog.h).  q[n] and x[n, 3] float64, m[P, 3] int32 and
    rho_out[P, 2] float64 must be contiguous CUDA tensors on the current
    device; P must not exceed RBSOG_NOALLOC_MAX_P."""
    import torch
    if not hasattr(x, "shape") or len(x.shape) != 2:
        raise ValueError("x: expected shape (n, 3)")
    n = int(x.shape[0])
    P = int(m.shape[0]) if hasattr(m, "shape") else -1
    if n < 1 or P < 1:
        raise ValueError("need n >= 1 particles and P >= 1 frequencies")
    if P > RBSOG_NOALLOC_MAX_P:
        raise RBSOGError(1, f"rbsog_rho_noalloc: P={P} exceeds the allocation-free maximum of "
                            f"{RBSOG_NOALLOC_MAX_P}")
    pq = _device_tensor(q, "q", torch.float64, (n,))
    px = _device_tensor(x, "x", torch.float64, (n, 3))
    pm = _device_tensor(m, "m", torch.int32, (P, 3))
    po = _device_tensor(rho_out, "rho_out", torch.float64, (P, 2))
    Lc = (C.c_double * 3)(*[float(v) for v in L])
    s = _lib.rbsog_rho_noalloc(n, pq, px, Lc, pm, P, po, stream)
    if s != 0:
        raise RBSOGError(s, "rbsog_rho_noalloc: invalid argument or CUDA failure")


def rbsog_measure_peaks(device: int = 0):
    out = np.zeros(5)
    s = _lib.rbsog_measure_peaks(int(device), _ptr(out))
    if s != 0:
        raise RBSOGError(s, "rbsog_measure_peaks failed")
    return {"mufu_per_s": out[0], "fma32_per_s": out[1], "fma64_per_s": out[2], "sm_mhz": out[3],
            "sm_count": int(out[4])}


def rbsog_batch_create(n_per, device: int = 0, stream: int | None = None):
    arr = np.ascontiguousarray(n_per, dtype=np.int64)
    ctx = C.c_void_p()
    s = _lib.rbsog_batch_create(C.byref(ctx), int(arr.shape[0]), _ptr(arr), int(device), stream)
    if s != 0:
        raise RBSOGError(s, "rbsog_batch_create failed")
    return ctx


def rbsog_batch_set_params(ctx, params):
    arr = (rbsog_params * len(params))(*params)
    _check(ctx, _lib.rbsog_batch_set_params(ctx, C.cast(arr, C.c_void_p)))


def rbsog_batch_set_state(ctx, sys: int, q, x, v=None):
    _check(ctx, _lib.rbsog_batch_set_state(ctx, int(sys), _ptr(q), _ptr(x), _ptr(v)))


def rbsog_batch_restore(ctx, sys: int, f, kset_cursor: int, step: int):
    _check(ctx, _lib.rbsog_batch_restore(ctx, int(sys), _ptr(f), int(kset_cursor), int(step)))


def rbsog_batch_get_state(ctx, sys: int, x=None, v=None, f=None):
    step = C.c_int64()
    _check(ctx, _lib.rbsog_batch_get_state(ctx, int(sys), _ptr(x), _ptr(v), _ptr(f), C.byref(step)))
    return step.value


def rbsog_batch_get_energies(ctx, sys: int):
    e = rbsog_energies()
    _check(ctx, _lib.rbsog_batch_get_energies(ctx, int(sys), C.byref(e)))
    return e.as_dict()


def rbsog_batch_get_kseq(ctx, sys: int, set0: int, nsets: int, m_out):
    _check(ctx, _lib.rbsog_batch_get_kseq(ctx, int(sys), int(set0), int(nsets), _ptr(m_out)))


def rbsog_batch_step(ctx, nsteps: int):
    _check(ctx, _lib.rbsog_batch_step(ctx, int(nsteps)))


def rbsog_batch_autotune(ctx, reps: int = 3):
    chosen = np.zeros(2, dtype=np.int32)
    _check(ctx, _lib.rbsog_batch_autotune(ctx, int(reps), _ptr(chosen)))
    return {"home": int(chosen[0]), "tile": int(chosen[1])}


def rbsog_batch_rdf(ctx, sys: int, nbins: int, counts=None, g=None):
    """Appendix A pair histograms counts[3, nbins] (uint64; rows ++, +-, --)
    and g[3, nbins] of system `sys`; allocates host numpy arrays if omitted."""
    if counts is None:
        counts = np.zeros((3, nbins), dtype=np.uint64)
    if g is None:
        g = np.zeros((3, nbins))
    _check(ctx, _lib.rbsog_batch_rdf(ctx, int(sys), int(nbins), _ptr(counts), _ptr(g)))
    return counts, g


def rbsog_rdf(ctx, nbins: int, counts=None, g=None):
    return rbsog_batch_rdf(ctx, 0, nbins, counts, g)


def _check_server(s, status):
    if status != 0:
        msg = _lib.rbsog_server_last_error(s)
        raise RBSOGError(status, msg.decode() if msg else "")


def rbsog_server_create(max_jobs: int, mem_budget_bytes: int, quantum: int, device: int = 0,
                        stream: int | None = None):
    s = C.c_void_p()
    st = _lib.rbsog_server_create(C.byref(s), int(max_jobs), int(mem_budget_bytes), int(quantum),
                                  int(device), stream)
    if st != 0:
        raise RBSOGError(st, "rbsog_server_create failed")
    return s


def rbsog_server_submit(s, p: rbsog_params, q, x, v, nsteps: int) -> int:
    """q, x, v: host numpy arrays (float64, C-contiguous); v may be None."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    jid = C.c_int64()
    _check_server(s, _lib.rbsog_server_submit(s, int(q.shape[0]), C.byref(p), _ptr(q), _ptr(x), _ptr(v),
                                              int(nsteps), C.byref(jid)))
    return jid.value


def rbsog_server_advance(s):
    a, w, r = C.c_int32(), C.c_int32(), C.c_int32()
    _check_server(s, _lib.rbsog_server_advance(s, C.byref(a), C.byref(w), C.byref(r)))
    return a.value, w.value, r.value


def rbsog_server_result(s, job_id: int, n: int):
    """(status, x, v, f, energies, steps_done); arrays only once status == 2."""
    st = C.c_int32()
    steps = C.c_int64()
    e = rbsog_energies()
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    f = np.empty((n, 3))
    _check_server(s, _lib.rbsog_server_result(s, int(job_id), C.byref(st), _ptr(x), _ptr(v), _ptr(f),
                                              C.byref(e), C.byref(steps)))
    if st.value != 2:
        return st.value, None, None, None, None, 0
    return st.value, x, v, f, e.as_dict(), steps.value


def rbsog_server_cancel(s, job_id: int):
    _check_server(s, _lib.rbsog_server_cancel(s, int(job_id)))


def rbsog_server_release(s, job_id: int):
    _check_server(s, _lib.rbsog_server_release(s, int(job_id)))


def rbsog_server_last_error(s) -> str:
    m = _lib.rbsog_server_last_error(s)
    return m.decode() if m else ""


def rbsog_server_destroy(s):
    _check_server(None, _lib.rbsog_server_destroy(s))


def rbsog_last_error(ctx) -> str:
    m = _lib.rbsog_last_error(ctx)
    return m.decode() if m else ""


def rbsog_destroy(ctx):
    _check(None, _lib.rbsog_destroy(ctx))


def rbsog_green_kubo_heat(J_series, dt: float, V: float, T: float, max_lag: int, stream=None):
    """(acf[max_lag], C) of a heat-flux series [n, 3] (host array or device tensor)."""
    if not hasattr(J_series, "data_ptr"):
        J_series = np.ascontiguousarray(np.asarray(J_series, dtype=np.float64).reshape(-1, 3))
    n = J_series.shape[0]
    acf = np.zeros(int(max_lag))
    Cv = C.c_double()
    st = _lib.rbsog_green_kubo_heat(_ptr(J_series), int(n), float(dt), float(V), float(T), int(max_lag),
                                    _ptr(acf), C.byref(Cv), C.c_void_p(stream))
    if st != 0:
        raise RBSOGError(st, "rbsog_green_kubo_heat failed")
    return acf, Cv.value
