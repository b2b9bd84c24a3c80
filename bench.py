#!/usr/bin/env python
"""Throughput benchmark of the RBSOG velocity-Verlet step.

Workload (default): the 1,048,576-ion 1:1 electrolyte (L = 128, number
density 0.5, r_c = 3, P = 500 frequencies per step, SOG b = 1.4878, M = 36),
FP32C path.  One "step" is the whole hot path: half kick + drift, cell-list
build, near field, rho(k) sweep and combine, far-field scatter, half kick and
the fixed-order energy reductions.  Inputs are resident in HBM when the timed
region starts; the state (~0.2 GB) is larger than L2.

Prints ONE JSON line (rank 0).  With --gpus N > 1 (torchrun, one process per
GPU) every rank advances its own independent replica (weak scaling, no data
collective); the timed region is bracketed by barriers and the slowest rank's
time is used.

--impl reference times the FP64 CPU oracle (the checker the CUDA path is
validated against) on the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at N=1M (FP32-comp vs FP64 path, same error); p50/p99 job latency"
N_DEF, L_DEF, P_DEF = 1048576, 128.0, 500


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--L", type=float, default=L_DEF)
    ap.add_argument("--P", type=int, default=P_DEF)
    ap.add_argument("--quick", action="store_true", help="skip the FP64 path, P sweep and CPU baseline")
    return ap.parse_args()


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time); identity on a single process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_value(n_per_rank, world, seconds_per_step):
    """Particle-steps per second of the whole job: every rank advances its own
    replica of n_per_rank particles (weak scaling)."""
    return world * n_per_rank / seconds_per_step


def reference_rank_runs(rank):
    """The oracle arm runs on rank 0 only; other ranks exit without work."""
    return rank == 0


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    return rank, world, local, dist


class Clocks:
    """nvidia-smi sampler of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


def electrolyte_state(N, L, seed):
    import rbsog_inputs as I
    return I.electrolyte(N, L, seed=seed)


# ncu summaries (profiles/) holding the DRAM traffic of a kernel at this
# workload, with the hash of the kernel source they were taken from
PROFILE_OF = {"near": ("near_fp32c_lists_electrolyte_N1048576.md", "k_verlet.cu"),
              "rho_sweep": ("rho_sweep_fp32c_electrolyte_N1048576_P500.md", "k_far.cu"),
              "far_scatter": ("far_scatter_fp32c_electrolyte_N1048576_P500.md", "k_far.cu"),
              "list_build": ("list_build_fp32c_electrolyte_N1048576.md", "k_verlet.cu")}


def profiled_fields(kernel, N, P):
    """(DRAM bytes per launch, limiter) from the committed ncu summary, or
    (None, None) when the summary is for another workload or the kernel
    source changed since."""
    import hashlib
    import re
    for key, (fname, src) in PROFILE_OF.items():
        if not kernel.startswith(key):
            continue
        if N != N_DEF or (key not in ("near", "list_build") and P != P_DEF):
            return None, None
        try:
            txt = open(os.path.join(ROOT, "profiles", fname)).read()
            cur = hashlib.sha256(open(os.path.join(ROOT, "paper_2205_13824_gb300", "csrc", src), "rb")
                                 .read()).hexdigest()[:16]
        except OSError:
            return None, None
        m = re.search(r"traffic_bytes_per_launch: (\d+)", txt)
        h = re.search(r"sha256 prefix `([0-9a-f]+)`", txt)
        lim = re.search(r"`limiter: ([^`]+)`", txt)
        if h and h.group(1) == cur:
            return (int(m.group(1)) if m else None), (lim.group(1) + " (ncu)" if lim else None)
        return None, None
    return None, None


def distinct_per_set(ks, P):
    """Mean number of runs of equal consecutive frequencies per k-set: the
    frequencies the far-field kernels evaluate once the sets are folded."""
    import numpy as np
    m = np.asarray(ks).reshape(-1, P, 3)
    starts = np.any(m[:, 1:] != m[:, :-1], axis=2).sum(axis=1) + 1
    return float(starts.mean())


def roofline_for(name, launches, ms_total, N, L, P, rc, meas, hbm_gbs, lists=False, P_eval=None):
    """Algorithmic work of one launch over its average CUDA-event duration,
    against the rate measured on this GPU by rbsog_measure_peaks.  P_eval:
    frequencies per set the far-field kernels evaluate (the distinct runs of
    a folded set), P when None."""
    t = ms_total / launches / 1e3
    traffic, limiter = profiled_fields(name, N, P)
    out = {"kernel": name, "ms_per_launch": t * 1e3, "traffic": traffic}
    if limiter:
        out["limiter"] = limiter
    if name.startswith(("rho_sweep", "far_scatter")):
        # one (particle, evaluated frequency) term = one sin + one cos on the MUFU pipe
        Pe = P if P_eval is None else P_eval
        achieved = N * Pe / t / 1e9
        peak = meas["mufu_per_s"] / 2 / 1e9
        out.update(bound="alu", achieved=achieved, peak=peak, unit="Gsincos/s", frac=achieved / peak,
                   peak_basis="measured MUFU sin+cos rate / 2 (rbsog_measure_peaks)",
                   work=f"N x {Pe:.1f} evaluated frequencies per set (P = {P} sampled)")
        return out
    if name.startswith("list_build"):
        # per rebuild: a distance test (8 FP32 ops: 3 differences, 3 for r^2,
        # 2 compares) for every candidate of the particle's x-windows in the
        # 9 rows of cells around it (cells of side >= r_l = 1.1 r_c); the
        # expected count follows from the window geometry, averaged over the
        # particle's place in its cell
        import numpy as np
        rl = 1.1 * rc
        n = math.floor(L / rl)
        h = L / n
        g = np.random.default_rng(1).uniform(0.0, h, size=(100000, 2))
        per = 0.0
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                b2 = rl * rl - (g[:, 0] ** 2 if dy else 0.0) - (g[:, 1] ** 2 if dz else 0.0)
                per += float(np.mean(2.0 * np.sqrt(np.maximum(b2, 0.0))))
        cand = (N / L ** 3) * h * h * per
        achieved = N * 8.0 * cand / t / 1e12
        peak = meas["fma32_per_s"] / 1e12
        out.update(bound="alu", achieved=achieved, peak=peak, unit="Top/s", frac=achieved / peak,
                   peak_basis="measured FP32 FMA issue rate; work = 8 FP32 ops per candidate of the per-particle "
                              f"x-windows ({cand:.0f} per particle), per rebuild")
        return out
    if name.startswith("near"):
        # FP32 instruction-equivalents: 8 per candidate distance test, 50 per
        # pair inside r_c with the pair energies, 36 without them (the list
        # force leaves them out on every step but the last of a call; MUFU
        # ops counted once).  Candidates: the particles within r_c + skin of
        # the neighbour-list method (skin = r_c / 10), or the 27-cell stencil
        # when the step runs without lists
        pairs = 4.0 / 3.0 * math.pi * rc ** 3 * N / L ** 3
        if lists:
            cand = 4.0 / 3.0 * math.pi * (1.1 * rc) ** 3 * N / L ** 3
            basis = "candidate test within r_c + skin"
        else:
            cand = 27.0 * N / math.floor(L / rc) ** 3
            basis = "candidate test over the 27-cell stencil"
        per_pair = 36.0 if lists else 50.0
        ops = N * (8.0 * cand + per_pair * pairs)
        achieved = ops / t / 1e12
        peak = meas["fma32_per_s"] / 1e12
        out.update(bound="alu", achieved=achieved, peak=peak, unit="Top/s", frac=achieved / peak,
                   peak_basis="measured FP32 FMA issue rate (rbsog_measure_peaks); work = 8 FP32 ops per "
                              + basis + f" + {per_pair:.0f} per pair within r_c"
                              + (" (forces only: the pair energies are left out on all steps but the last "
                                 "of a call)" if lists else ""))
        return out
    achieved = N * 64 / t / 1e9
    out.update(bound="hbm", achieved=achieved, peak=hbm_gbs, unit="GB/s", frac=achieved / hbm_gbs)
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def rel_errors(f, fo, e=None, eo=None):
    """RMS relative force error, per-particle median and max of
    |F_i - F_ref,i| / (|F_ref,i| + median_j |F_ref,j|), and the relative
    error of the total potential energy U_near + U_far - U_self + U_wca."""
    import numpy as np
    nb = np.linalg.norm(fo, axis=1)
    pp = np.linalg.norm(f - fo, axis=1) / (nb + np.median(nb))
    out = {"rms_rel_force": float(np.sqrt(np.sum((f - fo) ** 2) / np.sum(fo ** 2))),
           "per_particle_median": float(np.median(pp)), "per_particle_max": float(pp.max())}
    if e is not None and eo is not None:
        U = e["U_near"] + e["U_far"] - e["U_self"] + e["U_wca"]
        Uo = eo["U_near"] + eo["U_far"] - eo["U_self"] + eo["U_wca"]
        out["rel_energy"] = abs(U - Uo) / abs(Uo)
    return out


def sig(v, digits=4):
    """Round floats (recursively) to a few significant digits for the JSON line."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}")
    if isinstance(v, dict):
        return {k: sig(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [sig(x, digits) for x in v]
    return v


def run_ours(args, rank, world, local, dist):
    import numpy as np
    import torch

    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    N, L, P, K, W = args.N, args.L, args.P, args.steps, args.warmup
    q, x, v = electrolyte_state(N, L, seed=2024 + rank)
    n_e2e = max(3, min(K, 10))
    n_long = 0 if args.quick else 220
    need = W + 2 * K + n_e2e + n_long + 8
    p32 = Pk.make_params(L, P, n_ksets=need, seed=17 + rank, precision="fp32c")
    g = Pk.RBSOG(N, p32, device=local)
    tq, tx, tv = (torch.tensor(a, device=dev) for a in (q, x, v))
    g.set_state(tq, tx, tv)
    P_eval = distinct_per_set(g.kseq(0, need), P)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # roofline denominators on this GPU: the best of three runs, so that a
    # run slowed by a clock dip does not lower the peak
    runs = [B.rbsog_measure_peaks(local) for _ in range(3)]
    meas = {k: max(r[k] for r in runs) for k in runs[0]}
    tuned = B.rbsog_batch_autotune(g.ctx, 3)    # launch shapes for this workload
    g.step(W)                                   # warm-up (builds the step graph)
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    builds0 = g.info()[0].list_builds
    clk = Clocks(local)
    with clk:
        barrier()
        e0.record(stream)
        g.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / K
    clocks = clk.summary()
    ms = max_over_ranks([ms], dist, dev)[0]
    rebuilds_in_window = g.info()[0].list_builds - builds0

    # a longer graph-replayed window: the neighbour-list rebuild interval and
    # the per-step time with rebuilds in their long-run proportion
    amort = None
    if n_long:
        b0 = g.info()[0].list_builds
        e0.record(stream)
        g.step(n_long)
        e1.record(stream)
        torch.cuda.synchronize()
        nb = g.info()[0].list_builds - b0
        ms_long = e0.elapsed_time(e1) / n_long
        amort = {"steps": n_long, "rebuilds": nb, "steps_per_rebuild": (n_long / nb) if nb else None,
                 "ms_per_step": ms_long, "value": whole_job_value(N, world, ms_long / 1e3)}

    # per-kernel CUDA-event timing over K more steps (eager launches)
    B.rbsog_set_profiling(g.ctx, True)
    barrier()
    b_prof = g.info()[0].list_builds
    e0.record(stream)
    g.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_prof = e0.elapsed_time(e1) / K
    prof = B.rbsog_get_profile(g.ctx)
    B.rbsog_set_profiling(g.ctx, False)
    rebuilds_prof = g.info()[0].list_builds - b_prof
    # the near field runs on neighbour lists (built at least once so far)
    lists = g.info()[0].list_builds > 0
    # kernels every graph-replayed step launches; the cell-list and list-build
    # kernels sit in a conditional graph node and run only on rebuild steps
    # (every ~22 steps here), so they are not counted
    gated = ("cell_bin", "cell_scan", "cell_scatter", "cell_order_gather", "list_build")
    launches_per_step = sum(c for k, (c, _) in prof.items() if not k.startswith(gated)) / K
    if lists:
        launches_per_step += 1   # the one-thread kernel that sets the rebuild node's condition
    gpu_launches = int(round(launches_per_step * K))
    if "kick_drift" in prof and lists:
        # NVE on neighbour lists: in the graph-replayed call each step's
        # scatter runs the next step's kick-drift, so the call launches one
        # kick-drift kernel instead of one per step
        gpu_launches -= K - 1
    if rebuilds_in_window:
        # kernels of one rebuild: the cell-list and list-build launches of the
        # profiled rebuilds per rebuild (one launch each, the scan two)
        per_build = sum(c for k, (c, _) in prof.items() if k.startswith(gated)) / max(1, rebuilds_prof)
        gpu_launches += int(round(per_build * rebuilds_in_window))

    # end to end through the C ABI from pinned host buffers: per step the
    # state (q, x, v, f) goes host->device, one step runs, (x, v, f) comes
    # back, in one rbsog_step_io call (the state lives in host memory)
    hq = torch.tensor(q).pin_memory()
    xs, vs, fs = (torch.empty((N, 3), dtype=torch.float64).pin_memory() for _ in range(3))
    step0 = B.rbsog_get_state(g.ctx, xs, vs, fs)
    cur = B.rbsog_get_cursor(g.ctx)
    barrier()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        B.rbsog_step_io(g.ctx, hq, xs, vs, fs, cur + i, step0 + i, 1, xs, vs, fs)
    t_e2e = (time.perf_counter() - t0) / n_e2e
    h2d = hq.numel() * 8 + 3 * xs.numel() * 8
    d2h = 3 * xs.numel() * 8
    t_e2e = max_over_ranks([t_e2e], dist, dev)[0]
    g.close()

    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6686.1)
    top = max(prof.items(), key=lambda kv: kv[1][1])
    roof = roofline_for(top[0], top[1][0], top[1][1], N, L, P, 3.0, meas, hbm, lists, P_eval)
    roof_far = [roofline_for(k, c, t, N, L, P, 3.0, meas, hbm, P_eval=P_eval) for k, (c, t) in prof.items()
                if k.startswith(("rho_sweep", "far_scatter"))]
    roof_near = [roofline_for(k, c, t, N, L, P, 3.0, meas, hbm, lists) for k, (c, t) in prof.items()
                 if k.startswith("near")]
    # profiled steps launch the build kernels only on a rebuild: the profiled
    # time over those launches is the time per rebuild
    roof_build = [roofline_for(k, c, t, N, L, P, 3.0, meas, hbm, lists)
                  for k, (c, t) in prof.items() if k.startswith("list_build")]
    tot = sum(tt for _, tt in prof.values())
    kernels = {k: {"launches": c, "ms_per_launch": t / c, "share": t / tot}
               for k, (c, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    value = whole_job_value(N, world, ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"1:1 electrolyte N={N} L={L:g} r_c=3 P={P} FP32C", "N": N, "L": L,
                   "P": P, "r_c": 3.0, "sog": "b=1.48783512395703226 M=36 (Table 1 row 3 at r_c=3)",
                   "precision": "fp32c", "l2": "inputs larger than L2 (state ~0.2 GB per replica)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single system",
                   "autotuned": tuned},
        "e2e": {"value": whole_job_value(N, world, t_e2e), "unit": "particle-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "clocks": clocks,
    }
    head = {"fp32c": {"value": value, "ms_per_step": ms, "rebuilds_in_window": rebuilds_in_window,
                      "P": P, "P_evaluated_per_set": P_eval}}
    if amort:
        head["fp32c"]["long_window"] = amort
    extras = {}
    if not args.quick and rank == 0:
        extras = run_extras(args, q, x, v, dev)
        line["cpu_baseline"] = extras.pop("cpu_baseline")
    line.update({
        "gpu_launches_note": "graph-replayed steps: the kernels outside the conditional rebuild node, plus the "
                             "cell-list and list-build kernels of the rebuilds inside the window",
        "roofline_far_field": sig(roof_far),
        "roofline_near_field": sig(roof_near),
        "roofline_list_build": sig(roof_build),
        "near_field_method": "neighbour lists, skin r_c/10, rebuilt on a displacement test" if lists
                             else "cell stencil",
        "measured_peaks": sig({"mufu_per_s": meas["mufu_per_s"], "fma32_per_s": meas["fma32_per_s"],
                               "fma64_per_s": meas["fma64_per_s"], "sm_mhz": meas["sm_mhz"],
                               "sm_count": meas.get("sm_count")}),
        "kernels": sig(kernels, 3),
        "ms_per_step_eager_profiled": ms_prof,
    })
    hl = extras.pop("headline", {})
    line.update(sig(extras))
    head.update(hl)
    head["far_field_frac"] = {r["kernel"]: sig(r["frac"], 3) for r in roof_far}
    head["near_field_frac"] = {r["kernel"]: sig(r["frac"], 3) for r in roof_near}
    head["list_build_frac"] = {r["kernel"]: sig(r.get("frac"), 3) for r in roof_build}
    # the compact summary goes last, so that it survives when only the end
    # of a long line is kept
    line["headline"] = sig(head)
    return line, rank


def run_extras(args, q, x, v, dev):
    """FP64 comparator path at the same workload; the FP32C and FP64 forces
    and energies on one k-set against the FP64 oracle (timed on the host
    cores: the CPU baseline); the P sweep of the FP32C path; the options."""
    import numpy as np
    import torch

    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    N, L, P = args.N, args.L, args.P
    out = {}
    tq, tx, tv = (torch.tensor(a, device=dev) for a in (q, x, v))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    base, m, f_o, e_o = cpu_baseline(N, L, P, q, x, v)
    out["cpu_baseline"] = base
    K64 = max(2, min(args.steps, 5))
    g64 = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=K64 + 4, seed=17, precision="fp64"), device=dev.index)
    g32 = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=4, seed=17, precision="fp32c"), device=dev.index)
    g64.set_state(tq, tx, tv)
    g32.set_state(tq, tx, tv)
    f64 = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    f32 = torch.zeros_like(f64)
    e64 = B.rbsog_compute_forces(g64.ctx, m, f64)
    e32 = B.rbsog_compute_forces(g32.ctx, m, f32)
    f64n, f32n = f64.cpu().numpy(), f32.cpu().numpy()
    err32 = rel_errors(f32n, f_o, e32, e_o)
    err64 = rel_errors(f64n, f_o, e64, e_o)
    err32_64 = rel_errors(f32n, f64n, e32, e64)
    g32.close()
    g64.step(1)
    torch.cuda.synchronize()
    e0.record(st)
    g64.step(K64)
    e1.record(st)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / K64
    g64.close()
    out["fp64_path"] = {"value": N / (ms64 / 1e3), "unit": "particle-steps/s", "ms_per_step": ms64,
                        "steps": K64, "dtype": "f64"}
    acc = {"k_set": f"one k-set of P={P} from the oracle's sampler, initial state of the workload",
           "particles": N, "fp32c_vs_oracle": err32, "fp64_vs_oracle": err64, "fp32c_vs_fp64_gpu": err32_64}
    out["accuracy"] = acc
    out["headline"] = {"fp64": {"value": N / (ms64 / 1e3), "ms_per_step": ms64},
                       "fp32c_vs_oracle": err32, "fp64_vs_oracle": {k: err64[k] for k in ("rms_rel_force",
                                                                                         "per_particle_max",
                                                                                         "rel_energy")}}
    sweep = {}
    for Ps in (100, 500, 2000):
        if Ps == P:
            continue
        g = Pk.RBSOG(N, Pk.make_params(L, Ps, n_ksets=args.steps + 8, seed=19, precision="fp32c"),
                     device=dev.index)
        g.set_state(tq, tx, tv)
        g.step(2)
        torch.cuda.synchronize()
        e0.record(st)
        g.step(args.steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1) / args.steps
        sweep[str(Ps)] = {"value": N / (ms_s / 1e3), "ms_per_step": ms_s}
        g.close()
    out["fp32c_P_sweep"] = sweep
    # the FP64 path at the other two batch sizes (a few steps: about 0.1 s each)
    sweep64 = {}
    for Ps in (100, 2000):
        if Ps == P:
            continue
        g = Pk.RBSOG(N, Pk.make_params(L, Ps, n_ksets=K64 + 4, seed=19, precision="fp64"), device=dev.index)
        g.set_state(tq, tx, tv)
        g.step(1)
        torch.cuda.synchronize()
        e0.record(st)
        g.step(K64)
        e1.record(st)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1) / K64
        sweep64[str(Ps)] = {"value": N / (ms_s / 1e3), "ms_per_step": ms_s, "steps": K64}
        g.close()
    out["fp64_P_sweep"] = sweep64
    # the zero-frequency term of a spherical or planar boundary (Sec. 3.2) on
    # the same workload: step time with it, and its own kernels' time
    bnd = {}
    for kind, name in ((1, "spherical"), (2, "planar")):
        g = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=args.steps + 8, seed=19, precision="fp32c", boundary=kind),
                     device=dev.index)
        g.set_state(tq, tx, tv)
        g.step(2)
        torch.cuda.synchronize()
        e0.record(st)
        g.step(args.steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1) / args.steps
        B.rbsog_set_profiling(g.ctx, True)
        g.step(3)
        torch.cuda.synchronize()
        prof_b = B.rbsog_get_profile(g.ctx)
        bnd[name] = {"value": N / (ms_b / 1e3), "ms_per_step": ms_b,
                     "boundary_kernels_ms": prof_b["boundary"][1] / prof_b["boundary"][0]}
        g.close()
    out["fp32c_boundary_terms"] = bnd
    # the paper's core-shell near-field kernel (Sec. 3.4) in place of the
    # combined table, r_in = r_c / 3
    g = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=args.steps + 8, seed=19, precision="fp32c",
                                   near_kernel="coreshell"), device=dev.index)
    g.set_state(tq, tx, tv)
    g.step(2)
    torch.cuda.synchronize()
    e0.record(st)
    g.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms_c = e0.elapsed_time(e1) / args.steps
    B.rbsog_set_profiling(g.ctx, True)
    g.step(3)
    torch.cuda.synchronize()
    prof_c = B.rbsog_get_profile(g.ctx)
    near_c = prof_c["near_fp32c_coreshell"]
    out["fp32c_coreshell_near"] = {"value": N / (ms_c / 1e3), "ms_per_step": ms_c,
                                   "near_ms": near_c[1] / near_c[0]}
    g.close()
    out.update(run_dynamics_extras(args, tq, tx, tv, dev))
    out["small_configs"] = run_small_configs(dev)
    rep = run_replicas(dev)
    out["batched_replicas"] = rep
    srv = run_serving(dev)
    out["serving"] = srv
    cb = srv["continuous_batching"]
    out["headline"]["replicas"] = {"value": rep["value"], "ms_per_step": rep["ms_per_step"], "steps": rep["steps"]}
    out["headline"]["serving"] = {"jobs": srv["jobs"], "p50_s": cb["latency_p50_s"], "p99_s": cb["latency_p99_s"],
                                  "served_particle_steps_per_s": cb["served_particle_steps_per_s"],
                                  "fp64_one_at_a_time_p50_s": srv["one_at_a_time_fp64"]["latency_p50_s"],
                                  "fp64_one_at_a_time_p99_s": srv["one_at_a_time_fp64"]["latency_p99_s"],
                                  "sub_saturation_rate_per_s": srv["sub_saturation"]["arrival_rate_per_s"],
                                  "sub_saturation_p50_s": srv["sub_saturation"]["latency_p50_s"],
                                  "sub_saturation_p99_s": srv["sub_saturation"]["latency_p99_s"]}
    return out


def run_small_configs(dev):
    """The two smaller workloads as specified.  1,000-ion electrolyte (L =
    12.6, P = 100), FP64: one force evaluation and 10 velocity-Verlet steps,
    timed, with the forces after the 10 steps against the oracle's trajectory
    on the oracle's own sequence (the CPU-baseline leg's oracle).  64,000-ion
    electrolyte (L = 50.4, P = 200), FP32C, 1,000 Berendsen steps at T0 = 1:
    every 100 steps the FP32C force at the trajectory's positions against the
    FP64 path on one k-set (RMS relative and worst particle), the total
    energy and T; the same run through the FP64 path, and 1,000 NVE steps in
    both precisions from the same start, for the energies side by side."""
    import numpy as np
    import torch

    import paper_2205_13824_gb300 as Pk
    import rbsog_inputs as I
    B = Pk.binding
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    # 1,000 ions, FP64: 10 steps against the oracle's trajectory, then the
    # steady-state step time on the same system
    N, L, P, steps = 1000, 12.6, 100, 10
    q, x, v = I.electrolyte(N, L, seed=1)
    p = Pk.make_params(L, P, n_ksets=steps + 1, seed=7, precision="fp64")
    g = Pk.RBSOG(N, p, device=dev.index)
    g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
    info = g.info()[0]
    g.step(steps)
    xg, _, fg, _ = (a.cpu().numpy() if hasattr(a, "cpu") else a for a in g.state())
    kseq_dev = g.kseq(0, steps + 1)
    g.close()
    base, ks, xo, fo = cpu_baseline_small(q, x, v, L, P, steps, info.n_chains, info.chain_len)
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    reps = 200

    def steady_ms(prec):
        h = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=steps * (reps + 1) + 1, seed=7, precision=prec),
                     device=dev.index)
        h.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
        B.rbsog_batch_autotune(h.ctx, 3)   # launch shapes for this size (state untouched)
        h.step(steps)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            h.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        h.close()
        return e0.elapsed_time(e1) / (reps * steps)
    ms = steady_ms("fp64")
    ms32 = steady_ms("fp32c")
    out["electrolyte_N1000_fp64"] = {
        "ms_per_step": ms, "value": N / (ms / 1e3), "unit": "particle-steps/s",
        "timing": f"{reps} calls of {steps} steps each, after autotuning and a first call",
        "vs_oracle_after_10_steps": dict(rel_errors(fg, fo), max_position_diff=float(np.abs(dx).max()),
                                         same_k_sequence=bool(np.array_equal(kseq_dev, ks[: len(kseq_dev)]))),
        "cpu_baseline": base,
        "fp32c": {"ms_per_step": ms32, "value": N / (ms32 / 1e3)},
        "note": "the FP64 near field of 1,000 ions splits each block's cell-stencil rows over its four warps; "
                "it stays bound by the latency of this GPU's FP64 units (64 blocks), not by their rate"}
    # 64,000 ions, FP32C, 1,000 Berendsen steps; NVE drift
    N, L, P = 64000, 50.4, 200
    q, x, v = I.electrolyte(N, L, seed=2022)
    tq, tx, tv = (torch.tensor(a, device=dev) for a in (q, x, v))
    g = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=1001, seed=77, precision="fp32c", tau_T=0.1), device=dev.index)
    g.set_state(tq, tx, tv)
    c32 = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=1, seed=1, precision="fp32c"), device=dev.index)
    c64 = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=1, seed=1, precision="fp64"), device=dev.index)
    m = c64.kseq(0, 1)
    f32 = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    f64 = torch.zeros_like(f32)
    rows, t_steps = [], 0.0
    for c in range(10):
        e0.record(st)
        g.step(100)
        e1.record(st)
        torch.cuda.synchronize()
        t_steps += e0.elapsed_time(e1)
        xg = g.state()[0]
        en = g.energies()
        for ctx, f in ((c32, f32), (c64, f64)):
            ctx.set_state(tq, xg)
            B.rbsog_compute_forces(ctx.ctx, m, f)
        err = rel_errors(f32.cpu().numpy(), f64.cpu().numpy())
        rows.append({"step": 100 * (c + 1), "rms_rel_force_vs_fp64": err["rms_rel_force"],
                     "per_particle_max_vs_fp64": err["per_particle_max"], "T": en["T"],
                     "E_total": en["U_near"] + en["U_far"] - en["U_self"] + en["U_wca"] + en["K"]})
    counts, gr = g.rdf(256)
    g.close()
    c32.close()
    c64.close()
    # the same 1,000 NVT steps through the FP64 path, and 1,000 NVE steps in
    # both precisions: energies every 100 steps side by side
    runs = {}
    for name, prec, tau in (("nvt_fp64", "fp64", 0.1), ("nve_fp32c", "fp32c", 0.0), ("nve_fp64", "fp64", 0.0)):
        h = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=1001, seed=77, precision=prec, tau_T=tau), device=dev.index)
        h.set_state(tq, tx, tv)
        es = []
        for c in range(10):
            h.step(100)
            en = h.energies()
            es.append(en["U_near"] + en["U_far"] - en["U_self"] + en["U_wca"] + en["K"])
        h.close()
        runs[name] = es
    e32 = [r["E_total"] for r in rows]
    energy = {
        "nvt_fp32c_E_every_100_steps": e32, "nvt_fp64_E_every_100_steps": runs["nvt_fp64"],
        "nvt_max_rel_E_diff_fp32c_vs_fp64": max(abs(a - b) / abs(b) for a, b in zip(e32, runs["nvt_fp64"])),
        "nvt_rel_E_change_steps_100_to_1000": (e32[-1] - e32[0]) / abs(e32[0]),
        "nve_fp32c_E_every_100_steps": runs["nve_fp32c"], "nve_fp64_E_every_100_steps": runs["nve_fp64"],
        "nve_max_rel_E_diff_fp32c_vs_fp64": max(abs(a - b) / abs(b) for a, b in
                                                zip(runs["nve_fp32c"], runs["nve_fp64"])),
        "nve_note": "without a thermostat the random-batch force noise heats the system (the method is "
                    "analysed under a thermostat); both precisions follow the same energies"}
    b = int(1.1 / (L / 512))
    out["electrolyte_N64000_fp32c_nvt"] = {"steps": 1000, "ms_per_step": t_steps / 1000,
                                           "value": N / (t_steps / 1000 / 1e3), "every_100_steps": rows,
                                           "rdf_contact_peak": {"++": float(gr[0, b - 3:b + 6].max()),
                                                                "+-": float(gr[1, b - 3:b + 6].max())},
                                           "energy": energy}
    return out


def run_dynamics_extras(args, tq, tx, tv, dev):
    """Step time with the Langevin and Nose-Hoover thermostats and with the
    per-Gaussian sampler on the same workload; the cost of the Appendix A
    observables beside the step (one MSD/VACF sample with 8 origins, one
    pressure tensor, one Green-Kubo integral of a 10^4-sample series)."""
    import torch

    import paper_2205_13824_gb300 as Pk
    B = Pk.binding
    N, L, P = args.N, args.L, args.P
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    out = {}

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for name, kw in (("fp32c_langevin", {"tau_T": 0.1, "thermostat": "langevin"}),
                     ("fp32c_nose_hoover", {"tau_T": 0.1, "thermostat": "nose-hoover"}),
                     ("fp32c_per_gaussian_sampler", {"sampler": "per-gaussian"})):
        g = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=args.steps + 8, seed=19, precision="fp32c", **kw),
                     device=dev.index)
        g.set_state(tq, tx, tv)
        g.step(2)
        ms_t = timed(lambda: g.step(args.steps), 1) / args.steps
        out[name] = {"value": N / (ms_t / 1e3), "unit": "particle-steps/s", "ms_per_step": ms_t}
        if "sampler" in kw:
            out[name]["P_set"] = int(g.info()[0].P_set)
        g.close()
    g = Pk.RBSOG(N, Pk.make_params(L, P, n_ksets=args.steps + 8, seed=19, precision="fp32c"), device=dev.index)
    g.set_state(tq, tx, tv)
    g.observe_start(64, 8)
    for _ in range(64):
        g.observe_sample()
    ms_obs = timed(g.observe_sample, 20)
    m = g.kseq(0, 1)
    g.pressure(m)
    t0 = time.perf_counter()
    g.pressure(m)
    ms_p = (time.perf_counter() - t0) * 1e3
    g.heat_flux(m)
    t0 = time.perf_counter()
    g.heat_flux(m)
    ms_h = (time.perf_counter() - t0) * 1e3
    g.close()
    ser = torch.randn((10000, 9), dtype=torch.float64, device=dev)
    B.rbsog_green_kubo(ser, 0.01, 1.0, 1.0, 1000)
    t0 = time.perf_counter()
    B.rbsog_green_kubo(ser, 0.01, 1.0, 1.0, 1000)
    ms_gk = (time.perf_counter() - t0) * 1e3
    out["observables"] = {"msd_vacf_sample_ms": ms_obs, "msd_vacf_origins": 8,
                          "pressure_tensor_ms": ms_p, "heat_flux_ms": ms_h, "green_kubo_ms": ms_gk,
                          "green_kubo_series": "10000 samples x 1000 lags"}
    return out


def serve_trace(Pk, trace, states, P, max_jobs, quantum, budget):
    """Replay a job trace in real time through one server: jobs are
    submitted when their arrival time has passed; latency = completion -
    arrival (wall clock)."""
    srv = Pk.Server(max_jobs=max_jobs, mem_budget_bytes=budget, quantum=quantum)
    lat, pending = [], {}
    nxt = 0
    t0 = time.perf_counter()
    while nxt < len(trace) or pending:
        now = time.perf_counter() - t0
        while nxt < len(trace) and trace[nxt]["t"] <= now:
            j = trace[nxt]
            p = Pk.make_params(j["L"], P, seed=j["seed"], n_ksets=j["steps"] + 1, precision="fp32c")
            pending[srv.submit(p, *states[nxt], nsteps=j["steps"])] = j["t"]
            nxt += 1
        if not pending:
            time.sleep(max(0.0, trace[nxt]["t"] - now))
            continue
        _, _, retired = srv.advance()
        if retired:
            done = time.perf_counter() - t0
            for jid in list(pending):
                if srv.result(jid)[0] == 2:
                    lat.append(done - pending.pop(jid))
                    srv.release(jid)
    span = time.perf_counter() - t0
    srv.close()
    return lat, span


def fifo_latencies(arrivals, service):
    """Latencies of one FIFO server with the given arrival and service times."""
    free, lat = 0.0, []
    for a, s in zip(arrivals, service):
        start = max(a, free)
        free = start + s
        lat.append(free - a)
    return lat


SERVE_JOBS, SERVE_RATE, SERVE_BUDGET = 200, 50.0, 150 * 10 ** 9
# a second, sub-saturation trace: an arrival rate whose offered load stays
# below what the engine serves, so that latency is service, not queueing
SERVE_SUB_JOBS, SERVE_SUB_RATE = 80, 8.0


def run_serving(dev, n_jobs=SERVE_JOBS, P=200):
    """The serving workload as specified: Poisson arrivals at 50 jobs/s, N
    log-uniform in [500, 200000] at density 0.5, steps uniform in [100,
    10000], P = 200, FP32C, device-memory budget 150 GB; a seeded trace of
    n_jobs jobs replayed in real time through continuous batching.  The
    offered load exceeds what one GPU serves, so a second trace at 8 jobs/s
    (offered about 1.1e9 particle-steps/s) gives the latencies below
    saturation.  Against
    it: the same jobs one at a time in FP64, FIFO in arrival order, with each
    job's service time = its step count x its own FP64 step time measured on
    the device (the job's state, 5 graph-replayed steps after one warm-up);
    the full FP64 runs would take hours, so this part is extrapolated per job
    and labelled so."""
    import numpy as np
    import torch

    import paper_2205_13824_gb300 as Pk
    import rbsog_inputs as I
    trace = I.job_trace(n_jobs, seed=11, rate=SERVE_RATE, n_min=500, n_max=200000, steps_min=100,
                        steps_max=10000)
    out = {"jobs": n_jobs, "arrival_rate_per_s": SERVE_RATE, "P": P, "N_range": [500, 200000],
           "steps_range": [100, 10000], "mem_budget_bytes": SERVE_BUDGET, "precision": "fp32c",
           "trace": "rbsog_inputs.job_trace(seed=11)", "quantum_steps": 50}
    states = [I.electrolyte(j["N"], j["L"], seed=j["seed"] % 100000) for j in trace]
    work = sum(j["N"] * j["steps"] for j in trace)
    out["offered_particle_steps_per_s"] = work / trace[-1]["t"]
    warm = I.job_trace(1, seed=5, rate=50.0, n_min=500, n_max=2000, steps_min=5, steps_max=5)
    serve_trace(Pk, [dict(warm[0], t=0.0)], [I.electrolyte(warm[0]["N"], warm[0]["L"], seed=1)], P, 4, 5,
                SERVE_BUDGET)
    lat, span = serve_trace(Pk, trace, states, P, 128, 50, SERVE_BUDGET)
    lat = np.sort(np.array(lat))
    out["continuous_batching"] = {"max_jobs": 128, "makespan_s": span, "served_particle_steps_per_s": work / span,
                                  "latency_p50_s": float(np.percentile(lat, 50)),
                                  "latency_p99_s": float(np.percentile(lat, 99)), "completed": int(lat.size)}
    # the sub-saturation point: the same recipe at a lower arrival rate
    trace2 = I.job_trace(SERVE_SUB_JOBS, seed=12, rate=SERVE_SUB_RATE, n_min=500, n_max=200000, steps_min=100,
                         steps_max=10000)
    states2 = [I.electrolyte(j["N"], j["L"], seed=j["seed"] % 100000) for j in trace2]
    work2 = sum(j["N"] * j["steps"] for j in trace2)
    lat2, span2 = serve_trace(Pk, trace2, states2, P, 128, 50, SERVE_BUDGET)
    lat2 = np.sort(np.array(lat2))
    out["sub_saturation"] = {"jobs": SERVE_SUB_JOBS, "arrival_rate_per_s": SERVE_SUB_RATE,
                             "trace": "rbsog_inputs.job_trace(seed=12)",
                             "offered_particle_steps_per_s": work2 / trace2[-1]["t"], "makespan_s": span2,
                             "served_particle_steps_per_s": work2 / span2,
                             "latency_p50_s": float(np.percentile(lat2, 50)),
                             "latency_p99_s": float(np.percentile(lat2, 99)), "completed": int(lat2.size)}
    # FP64 one job at a time: every job's own FP64 step time on the device
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    t_meas = time.perf_counter()
    for j, (q, x, v) in zip(trace, states):
        g = Pk.RBSOG(j["N"], Pk.make_params(j["L"], P, seed=j["seed"], n_ksets=8, precision="fp64"))
        g.set_state(*(torch.tensor(a, device=dev) for a in (q, x, v)))
        g.step(1)
        e0.record(st)
        g.step(5)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1) / 5)
        g.close()
    t_meas = time.perf_counter() - t_meas
    service = [m * j["steps"] / 1e3 for m, j in zip(ms, trace)]
    lat64 = np.sort(np.array(fifo_latencies([j["t"] for j in trace], service)))
    free = 0.0
    for a_, s_ in zip([j["t"] for j in trace], service):
        free = max(a_, free) + s_
    out["one_at_a_time_fp64"] = {
        "basis": "FIFO in arrival order; service = steps x the job's own FP64 step time, measured on the "
                 "device over 5 steps of each job (extrapolated to its step count)",
        "measure_s": t_meas, "makespan_s": free, "served_particle_steps_per_s": work / free,
        "latency_p50_s": float(np.percentile(lat64, 50)), "latency_p99_s": float(np.percentile(lat64, 99)),
        "fp64_ms_per_step_median": float(np.median(ms))}
    return out


def run_replicas(dev, n_sys=256, P=200, K=500, W=5):
    """Batched replicas as specified: n_sys independent electrolytes, N
    log-uniform in [1000, 100000], density 0.5, Bjerrum length uniform in
    [0.7, 1.5], P = 200, FP32C, all advanced by one graph launch per step
    (autotuned shapes), timed over 500 steps."""
    import torch

    import paper_2205_13824_gb300 as Pk
    import rbsog_inputs as I
    B = Pk.binding
    Ns, Ls, lBs = I.replica_sizes(n_sys, seed=4)
    params = [Pk.make_params(float(Ls[i]), P, lB=float(lBs[i]), seed=1000 + i, n_ksets=W + K + 4,
                             precision="fp32c") for i in range(n_sys)]
    b = Pk.Batch([int(n) for n in Ns], params, device=dev.index)
    for i in range(n_sys):
        q, x, v = I.electrolyte(int(Ns[i]), float(Ls[i]), seed=5000 + i)
        b.set_state(i, torch.tensor(q, device=dev), torch.tensor(x, device=dev), torch.tensor(v, device=dev))
    tuned = B.rbsog_batch_autotune(b.ctx, 2)
    b.step(W)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step(K)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    total = int(sum(int(n) for n in Ns))
    b.close()
    return {"value": total / (ms / 1e3), "unit": "particle-steps/s", "ms_per_step": ms, "steps": K,
            "n_sys": n_sys, "particles": total, "P": P, "launches_per_step": "one graph launch",
            "autotuned": tuned}


def cpu_baseline(N, L, P, q, x, v):
    """The FP64 oracle, as it stands, on the host cores: one full force
    evaluation (near field over its cell list + random-batch far field with
    rho(k) over all particles; the cost of one velocity-Verlet step) of the
    whole workload on a k-set from the oracle's own sampler.  Returns the
    baseline record, that k-set and the oracle's forces and energies (the
    reference the GPU paths' errors are measured against)."""
    import numpy as np

    import oracle as O
    sog = O.SOG.solve(1.48783512395703226, 3.0, 232)
    sog = O.SOG(sog.b, sog.sigma, sog.omega0, 36)
    s = O.System((L, L, L), sog, 3.0, 1.0, 1.0, 1.0)
    S = s.S()
    m = O.kseq(sog, s.L, seed=5, n_chains=8, chain_len=(P + 7) // 8)[:P]
    xw = O.wrap(x, s.L)
    t0 = time.perf_counter()
    f_o, e_o = O.forces(s, q, xw, S=S, m=m)
    dt = time.perf_counter() - t0
    # one host core on a 65,536-particle sample of the same electrolyte (the
    # oracle's cost per particle-step does not depend on N)
    ns = min(N, 65536)
    Ls = L * (ns / N) ** (1.0 / 3.0)
    q1, x1, v1 = electrolyte_state(ns, Ls, seed=2025)
    s1 = O.System((Ls, Ls, Ls), sog, 3.0, 1.0, 1.0, 1.0)
    ks1 = O.kseq(sog, s1.L, seed=5, n_chains=8, chain_len=(P + 7) // 8)
    old = O.set_num_threads(1)
    t1 = time.perf_counter()
    O.md(s1, q1, x1, v1, s1.S(), P, ks1, 1, 0.001, f=np.zeros_like(x1))
    dt1 = time.perf_counter() - t1
    O.set_num_threads(old)
    base = {"value": N / dt, "unit": "particle-steps/s", "cores": O.num_threads(),
            "kind": "oracle", "sample": f"one full FP64 force evaluation (near cells + random-batch far, "
                                        f"P={P}) of the N={N} workload",
            "seconds": dt,
            "one_core": {"value": ns / dt1, "unit": "particle-steps/s", "cores": 1, "seconds": dt1,
                         "sample": f"1 full step of a {ns}-particle sample at the same density and P={P}"}}
    return base, m, f_o, e_o


def cpu_baseline_small(q, x, v, L, P, steps, n_chains, chain_len):
    """The FP64 oracle on the 1,000-ion electrolyte: `steps` velocity-Verlet
    steps from the initial state on the oracle's own sampling of the
    k-sequence for the GPU context's chain layout, timed on the host cores.
    Returns the baseline record, that sequence and the final positions and
    forces."""
    import oracle as O
    sog = O.SOG.solve(1.48783512395703226, 3.0, 232)
    sog = O.SOG(sog.b, sog.sigma, sog.omega0, 36)
    s = O.System((L,) * 3, sog, 3.0, 1.0, 1.0, 1.0)
    ks = O.kseq(sog, s.L, seed=7, n_chains=n_chains, chain_len=chain_len)
    t0 = time.perf_counter()
    xo, _, fo, _ = O.md(s, q, x, v, s.S(), P, ks, steps, 0.001)
    dt = time.perf_counter() - t0
    base = {"value": len(q) * steps / dt, "unit": "particle-steps/s", "cores": O.num_threads(),
            "kind": "oracle", "sample": f"initial force + {steps} FP64 steps of the {len(q)}-ion system, P={P}",
            "seconds": dt}
    return base, ks, xo, fo


def run_reference(args, rank, world, sample=65536):
    """Oracle arm, bounded per step: each step is one full FP64 velocity-
    Verlet step of the oracle (near field over its cell list, random-batch
    far field with rho(k) over all particles, P frequencies) on a sample of
    the workload: the same electrolyte at the same density with `sample`
    particles (the oracle's cost per particle-step does not depend on N:
    pairs per particle and P are the same).  Value: particle-steps per second
    on the host cores of rank 0."""
    import oracle as O
    N, L, P, K, W = args.N, args.L, args.P, args.steps, args.warmup
    ns = min(N, sample)
    Ls = L * (ns / N) ** (1.0 / 3.0)
    q, x, v = electrolyte_state(ns, Ls, seed=2024)
    sog = O.SOG.solve(1.48783512395703226, 3.0, 232)
    sog = O.SOG(sog.b, sog.sigma, sog.omega0, 36)
    s = O.System((Ls, Ls, Ls), sog, 3.0, 1.0, 1.0, 1.0)
    S = s.S()
    ks = O.kseq(sog, s.L, seed=5, n_chains=16, chain_len=(P * (W + K + 1) + 15) // 16)
    x, v, f, _ = O.md(s, q, x, v, S, P, ks, 0, 0.001)      # initial forces
    used = 1
    if W:
        x, v, f, _ = O.md(s, q, x, v, S, P, ks[used * P:], W, 0.001, f=f)
        used += W
    t0 = time.perf_counter()
    x, v, f, _ = O.md(s, q, x, v, S, P, ks[used * P:], K, 0.001, f=f)
    el = time.perf_counter() - t0
    val = ns * K / el
    smalls = oracle_small_configs(O, sog)
    return {"metric": METRIC, "value": val, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"1:1 electrolyte N={N} L={L:g} r_c=3 P={P}", "N": N, "L": L, "P": P},
            "cpu_baseline": {"value": val, "unit": "particle-steps/s", "cores": O.num_threads(),
                             "kind": "oracle",
                             "sample": f"{K} full FP64 oracle steps of the same electrolyte at density 0.5 "
                                       f"with {ns} particles (L={Ls:.3f}), P={P}, on the host cores"},
            "e2e": {"value": val, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "oracle_configs": smalls}


def oracle_small_configs(O, sog):
    """The oracle on the smaller workloads, timed on the host cores: the
    1000-ion electrolyte (L = 12.6, P = 100) for one force evaluation and 10
    velocity-Verlet steps, the 64,000-ion one (L = 50.4, P = 200) for one
    force evaluation and 10 steps, and one force evaluation per P in
    {100, 500, 2000} on a 65,536-ion sample of the 1,048,576-ion workload
    (L scaled to density 0.5; per particle-step, so it extrapolates to the
    full size)."""
    out = {}
    for name, n, L, P in (("N1000_L12.6_P100", 1000, 12.6, 100), ("N64000_L50.4_P200", 64000, 50.4, 200)):
        q, x, v = electrolyte_state(n, L, seed=7)
        s = O.System((L, L, L), sog, 3.0, 1.0, 1.0, 1.0)
        ks = O.kseq(sog, s.L, seed=5, n_chains=8, chain_len=(P * 11 + 7) // 8)
        t0 = time.perf_counter()
        x, v, f, _ = O.md(s, q, x, v, s.S(), P, ks, 0, 0.001)
        t1 = time.perf_counter()
        O.md(s, q, x, v, s.S(), P, ks[P:], 10, 0.001, f=f)
        t2 = time.perf_counter()
        out[name] = {"force_eval_s": t1 - t0, "steps": 10, "particle_steps_per_s": n * 10 / (t2 - t1)}
    ns = 65536
    Ls = 128.0 * (ns / 1048576) ** (1.0 / 3.0)
    q, x, v = electrolyte_state(ns, Ls, seed=9)
    s = O.System((Ls, Ls, Ls), sog, 3.0, 1.0, 1.0, 1.0)
    for P in (100, 500, 2000):
        ks = O.kseq(sog, s.L, seed=5, n_chains=8, chain_len=(P + 7) // 8)
        t0 = time.perf_counter()
        O.md(s, q, x, v, s.S(), P, ks, 0, 0.001)
        el = time.perf_counter() - t0
        out[f"N1048576_P{P}_sample65536"] = {"force_eval_s": el, "particle_steps_per_s": ns / el,
                                             "extrapolated_full_step_s": el * 1048576 / ns}
    out["cores"] = O.num_threads()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if not reference_rank_runs(rank):
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    rank, world, local, dist = dist_setup(args)
    line, rank = run_ours(args, rank, world, local, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
