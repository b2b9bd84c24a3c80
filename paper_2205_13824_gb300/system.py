"""Thin torch-facing wrapper over the C ABI: one RBSOG system on one GPU.

All arithmetic runs in librbsog's kernels; this class only owns the context
handle, builds the parameter struct and hands tensor pointers through."""
from __future__ import annotations

from . import binding as B

# Table 1, row 3 of the paper (b with eps ~ 1.1e-5); M = 36 keeps the SOG
# relative error below 1e-4 out to r = 128 at r_c = 3.
DEFAULT_B = 1.48783512395703226
DEFAULT_M = 36


def make_params(L, P, r_c=3.0, b=DEFAULT_B, sigma=0.0, omega0=0.0, M=DEFAULT_M, lB=1.0,
                wca_sigma=1.0, wca_eps=1.0, dt=0.001, mass=1.0, T_target=1.0, tau_T=0.0,
                seed=1, n_ksets=1, chain_len=0, precision="fp64", boundary=0, near_kernel=0,
                r_in=0.0, thermostat=0, sampler=0) -> B.rbsog_params:
    if isinstance(L, (int, float)):
        L = (float(L),) * 3
    p = B.rbsog_params()
    p.L = (B.C.c_double * 3)(*[float(v) for v in L])
    p.b, p.sigma, p.omega0, p.M = float(b), float(sigma), float(omega0), int(M)
    p.r_c, p.P = float(r_c), int(P)
    p.coulomb_prefactor = float(lB)
    p.wca_sigma, p.wca_eps = float(wca_sigma), float(wca_eps)
    p.dt, p.mass, p.T_target, p.tau_T = float(dt), float(mass), float(T_target), float(tau_T)
    p.seed, p.n_ksets, p.chain_len = int(seed), int(n_ksets), int(chain_len)
    p.precision = {"fp64": B.RBSOG_FP64, "fp32c": B.RBSOG_FP32C}[precision] \
        if isinstance(precision, str) else int(precision)
    p.boundary = {"tinfoil": 0, "spherical": 1, "planar": 2}[boundary] \
        if isinstance(boundary, str) else int(boundary)
    p.near_kernel = {"table": 0, "coreshell": 1}[near_kernel] \
        if isinstance(near_kernel, str) else int(near_kernel)
    p.r_in = float(r_in)
    p.thermostat = {"berendsen": 0, "langevin": 1, "nose-hoover": 2}[thermostat] \
        if isinstance(thermostat, str) else int(thermostat)
    p.sampler = {"mixture": 0, "per-gaussian": 1}[sampler] if isinstance(sampler, str) else int(sampler)
    return p


class RBSOG:
    """One periodic system of n point charges advanced by velocity Verlet
    with the random batch sum-of-Gaussians force (Algorithm 1)."""

    def __init__(self, n: int, params: B.rbsog_params, device: int = 0, stream=None):
        import torch
        self.n = int(n)
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = B.rbsog_create(self.n, self.device, stream)
        self.params = params
        B.rbsog_set_params(self.ctx, params)

    def info(self):
        info, om, s = B.rbsog_get_info(self.ctx, self.params.M)
        return info, om, s

    def set_state(self, q, x, v=None):
        B.rbsog_set_state(self.ctx, q, x, v)

    def forces(self, m=None, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        e = B.rbsog_compute_forces(self.ctx, m, out)
        return out, e

    def step(self, nsteps: int):
        B.rbsog_step(self.ctx, nsteps)

    def state(self):
        import torch
        dev = f"cuda:{self.device}"
        x = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        v = torch.empty_like(x)
        f = torch.empty_like(x)
        step = B.rbsog_get_state(self.ctx, x, v, f)
        return x, v, f, step

    def energies(self):
        return B.rbsog_get_energies(self.ctx)

    def rdf(self, nbins: int = 256):
        """(counts[3, nbins], g[3, nbins]) by sign pair ++, +-, -- on [0, L/2)."""
        return B.rbsog_rdf(self.ctx, nbins)

    def pressure(self, m):
        """Pressure tensor [3, 3] of Appendix A, the far virial on k-set m[P][3]."""
        return B.rbsog_compute_pressure(self.ctx, m)

    def heat_flux(self, m=None):
        """Heat flux J[3] of Appendix A, the far term on k-set m[P][3]."""
        return B.rbsog_compute_heat_flux(self.ctx, m)

    def observe_start(self, n_lags: int, origin_every: int = 1):
        """Start MSD/VACF accumulation; the current state is frame 0 of the next sample."""
        self._obs_lags = int(n_lags)
        B.rbsog_observe_start(self.ctx, n_lags, origin_every)

    def observe_sample(self):
        B.rbsog_observe_sample(self.ctx)

    def observe_result(self):
        """(msd, vacf, count) per lag in samples."""
        return B.rbsog_observe_result(self.ctx, self._obs_lags)

    def kseq(self, set0: int, nsets: int):
        import numpy as np
        out = np.zeros((nsets * self.info()[0].P_set, 3), dtype=np.int32)
        B.rbsog_get_kseq(self.ctx, set0, nsets, out)
        return out

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.rbsog_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent systems of uneven size advanced together: one CUDA graph
    launch per step covers every system (see rbsog_batch_* in rbsog.h)."""

    def __init__(self, n_per, params, device: int = 0, stream=None):
        import torch
        self.n_per = [int(n) for n in n_per]
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = B.rbsog_batch_create(self.n_per, self.device, stream)
        self.params = list(params)
        B.rbsog_batch_set_params(self.ctx, self.params)

    def set_state(self, sys, q, x, v=None):
        B.rbsog_batch_set_state(self.ctx, sys, q, x, v)

    def restore(self, sys, f, kset_cursor, step):
        B.rbsog_batch_restore(self.ctx, sys, f, kset_cursor, step)

    def step(self, nsteps: int):
        B.rbsog_batch_step(self.ctx, nsteps)

    def state(self, sys):
        import torch
        n = self.n_per[sys]
        dev = f"cuda:{self.device}"
        x = torch.empty((n, 3), dtype=torch.float64, device=dev)
        v = torch.empty_like(x)
        f = torch.empty_like(x)
        step = B.rbsog_batch_get_state(self.ctx, sys, x, v, f)
        return x, v, f, step

    def energies(self, sys):
        return B.rbsog_batch_get_energies(self.ctx, sys)

    def rdf(self, sys, nbins: int = 256):
        return B.rbsog_batch_rdf(self.ctx, sys, nbins)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.rbsog_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of MD jobs (see rbsog_server_* in rbsog.h): jobs are
    queued with submit(), admitted while a slot is free and their memory
    footprint fits, advanced together by advance(), and retired when done."""

    def __init__(self, max_jobs=64, mem_budget_bytes=64 << 30, quantum=50, device: int = 0, stream=None):
        import torch
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.s = B.rbsog_server_create(max_jobs, mem_budget_bytes, quantum, self.device, stream)
        self.n_of = {}

    def submit(self, params, q, x, v=None, nsteps=1) -> int:
        jid = B.rbsog_server_submit(self.s, params, q, x, v, nsteps)
        self.n_of[jid] = len(q)
        return jid

    def advance(self):
        """(active, waiting, retired this call)."""
        return B.rbsog_server_advance(self.s)

    def result(self, jid):
        return B.rbsog_server_result(self.s, jid, self.n_of[jid])

    def cancel(self, jid):
        B.rbsog_server_cancel(self.s, jid)

    def release(self, jid):
        B.rbsog_server_release(self.s, jid)
        self.n_of.pop(jid, None)

    def close(self):
        if getattr(self, "s", None) is not None:
            B.rbsog_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
