"""Throughput of the bulb-model radial step on GB300 (beam-updates/s = beams x RK stage evaluations / s).

Workload (default): the large two-flavour multi-angle bulb, 1000 energies x 2000 angles x (nu, nubar)
= 4,000,000 beams, FP32 per-beam precession with FP64 moment reduction and step control,
Dormand-Prince 5(4), matter r^-3 profile, starting at the neutrino sphere r = 11 km.  A bench step is
one radial step attempt (7 passes over all beams, 6 stage evaluations); the same workload on the
plain FP64 path is timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs an independent replica of the workload (weak scaling; the single
instance's moment reduction has no cross-GPU exchange here).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from bulb_inputs import workload_2f_large  # noqa: E402

BYTES_PER_BEAM_STAGE = {("mixed", "dp45"): 14.0, ("fp64", "dp45"): 28.0,
                        ("mixed", "rk4"): 15.0, ("fp64", "rk4"): 30.0}
L2_BYTES = 129 * 1024 * 1024
# DRAM traffic of one timed launch of the step kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of an 8-step launch after the L2 flush).  It holds only for that launch size and for the kernel
# code it was taken on, identified by kernel_code_hash(); otherwise the benchmark reports null.
STEP_TRAFFIC = {"bytes_per_launch": 51212800 + 173520640, "steps_per_launch": 8,
                "code_sha256": "384a7fc295b4893c6b375e919685cf6890297471778ed692739cffb47e9a3cb5"}
KERNEL_SOURCES = ["step_kernel.cuh", "xflat_internal.cuh", "kernels_2f.cu"]
# Warp instructions of one radial step of the same kernel code (smsp__inst_executed.sum of one ncu
# capture of a one-step launch, which also carries the launch's first set-up, so a step inside a
# longer launch issues a little less): with the step time and the sampled SM clock it gives the
# kernel's place under its instruction-issue ceiling (4 warp instructions per clock per SM).
STEP_INSTRUCTIONS = {"warp_inst_per_step": 132219345, "code_sha256": STEP_TRAFFIC["code_sha256"]}


def issue_roofline(ms_per_step, sm_mhz, n_sm):
    """Issue-rate roofline of the step kernel, or None when the recorded count belongs to other code."""
    if kernel_code_hash() != STEP_INSTRUCTIONS["code_sha256"] or not sm_mhz:
        return None
    achieved = STEP_INSTRUCTIONS["warp_inst_per_step"] / (ms_per_step * 1e-3)
    peak = 4.0 * n_sm * sm_mhz * 1e6
    return {"achieved": achieved, "peak": peak, "unit": "warp-inst/s", "frac": achieved / peak,
            "warp_inst_per_step": STEP_INSTRUCTIONS["warp_inst_per_step"],
            "note": "ncu warp-instruction count of a one-step launch of this kernel code; peak = 4 per clock "
                    "per SM at the median sampled SM clock"}


def kernel_code_hash():
    """SHA-256 of the step kernel's code: the sources with comments and blank lines removed, so a
    comment edit does not invalidate the recorded counters but any code change does."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1912_10596_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].strip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def step_traffic(steps_per_launch):
    ok = kernel_code_hash() == STEP_TRAFFIC["code_sha256"] and steps_per_launch == STEP_TRAFFIC["steps_per_launch"]
    return STEP_TRAFFIC["bytes_per_launch"] if ok else None
METRIC = "beam-updates/s (beams x RK stages)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)


def bench_config(xf, wl, precision):
    return xf.config_from_workload(wl, precision=precision, steps_per_launch=1,
                                   rtol=1e-6 if precision == "mixed" else 1e-9,
                                   atol=1e-6 if precision == "mixed" else 1e-9)


def launch_chunks(steps, per_launch):
    """Split `steps` radial steps into persistent launches of at most `per_launch` steps."""
    out = []
    while steps > 0:
        out.append(min(per_launch, steps))
        steps -= out[-1]
    return out


def time_device_steps(xf, torch, wl, precision, steps, warmup, flush, shape=None, per_launch=1):
    """Time exactly `steps` radial steps, run as persistent launches of up to `per_launch` steps
    with the L2 flushed before every launch.  Returns (ms per launch, launch sizes, beam-stage
    updates per step, stats, solver)."""
    stream = torch.cuda.current_stream()
    cfg = bench_config(xf, wl, precision)
    if shape is not None:
        cfg.block_size, cfg.blocks_per_sm = shape
    cfg.cuda_stream = stream.cuda_stream
    s = xf.Solver(cfg)
    s.set_spectra(wl.spectra())
    s.advance([wl.r1], max_steps=1)                          # first step: sets the target
    for _ in range(max(0, warmup - 1)):
        s.advance(None, max_steps=1)
    torch.cuda.synchronize()
    st0 = s.stats()
    chunks = launch_chunks(steps, per_launch)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    for (e0, e1), n in zip(evs, chunks):
        flush(); e0.record(stream)
        s.advance(None, max_steps=n)
        e1.record(stream)
    torch.cuda.synchronize()
    st1 = s.stats()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    if st1.status != 0:
        raise RuntimeError(f"device status {st1.status}")
    bsu = (st1.beam_stage_updates - st0.beam_stage_updates) / steps
    acc = st1.accepted - st0.accepted
    s.timed_accepted_fraction = acc / max(1, acc + st1.rejected - st0.rejected)
    return ms, chunks, bsu, st1, s


def time_more_steps(torch, s, steps, flush, per_launch):
    """Time `steps` further radial steps of an existing solver (launches of up to per_launch steps,
    the L2 flushed before each).  Returns (ms per step, beam-stage updates per step, accepted
    steps, attempted steps)."""
    stream = torch.cuda.current_stream()
    st0 = s.stats()
    chunks = launch_chunks(steps, per_launch)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    for (e0, e1), n in zip(evs, chunks):
        flush(); e0.record(stream)
        s.advance(None, max_steps=n)
        e1.record(stream)
    torch.cuda.synchronize()
    st1 = s.stats()
    if st1.status != 0:
        raise RuntimeError(f"device status {st1.status}")
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    acc = st1.accepted - st0.accepted
    att = acc + st1.rejected - st0.rejected
    return ms / steps, (st1.beam_stage_updates - st0.beam_stage_updates) / steps, acc, att


def repeat_stats(torch, s, steps, repeats, flush, per_launch):
    """Median, minimum and maximum of `repeats` timings of `steps` steps each."""
    runs = [time_more_steps(torch, s, steps, flush, per_launch) for _ in range(repeats)]
    ms = [r[0] for r in runs]
    return {"repeats": repeats, "steps_per_repeat": steps, "ms_per_step_median": statistics.median(ms),
            "ms_per_step_min": min(ms), "ms_per_step_max": max(ms),
            "beam_stage_updates_per_step": runs[0][1],
            "accepted_fraction": sum(r[2] for r in runs) / max(1, sum(r[3] for r in runs))}


def e2e_steps(xf, torch, s, wl, steps):
    """Through the public API with host buffers: state in from pinned host memory, one step,
    per-beam survival probabilities back to the host, every step."""
    nb = wl.n_beams
    host_state = torch.empty((3, nb), dtype=torch.float64, pin_memory=True)
    pee_host = torch.empty(nb, dtype=torch.float64, pin_memory=True)
    s.get_rho(xf.LAYOUT_NATIVE)                                 # warm the staging buffer
    state0 = s.get_rho(xf.LAYOUT_NATIVE)
    host_state.copy_(torch.from_numpy(state0))
    r = s.stats().r_km
    import ctypes
    torch.cuda.synchronize()
    st_a = s.stats()
    t0 = time.perf_counter()
    for _ in range(steps):
        xf.xflat_set_rho(s.h, ctypes.c_void_p(host_state.data_ptr()), 0, xf.LAYOUT_NATIVE, r)
        s.advance([wl.r1], max_steps=1)
        xf.xflat_pee(s.h, ctypes.c_void_p(pee_host.data_ptr()), None)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st_b = s.stats()
    # every call of the loop restarts from the same state at the same radius: count its stages
    # (the stats accumulate over the calls; a set_rho is not a stage)
    bsu = st_b.beam_stage_updates - st_a.beam_stage_updates
    return bsu / dt, host_state.numel() * 8, pee_host.numel() * 8


def cpu_baseline(seconds=12.0, impl_steps=None):
    """The FP64 oracle as it stands, on a bounded sample of the same workload: all 1000 energy bins
    and 20 of the 2000 angle bins (the first 20; 40,000 beams), Dormand-Prince steps from r = 11 km."""
    from oracle.physics import Bulb, Grid
    from oracle.integrate import dp45_step
    wl = workload_2f_large("fp64")
    g = Grid.from_workload(wl)
    sub = Grid(E=g.E, u=g.u[:20], du=g.du[:20], N=g.N)
    wl.n_angle = 20
    b = Bulb(wl, grid=sub)
    Y = b.initial_state()
    r, h = 11.0, 1e-9
    k1 = b.rhs(r, Y)
    n, t0 = 0, time.perf_counter()
    while (impl_steps is None and time.perf_counter() - t0 < seconds) or (impl_steps is not None and n < impl_steps):
        Y5, err, k7 = dp45_step(b.rhs, r, Y, h, k1, wl.atol, wl.rtol)
        n += 1
    dt = time.perf_counter() - t0
    beams = 2 * 20 * wl.n_energy
    return beams * 6 * n / dt, n, dt, beams


def _cpu_worker(seconds):
    v, n, dt, beams = cpu_baseline(seconds)
    return v, n


def cpu_baseline_all_cores(seconds=12.0):
    """The same bounded oracle sample run as independent copies on every host core at once (the
    oracle's beams are coupled through the moments at every stage, so one sample does not split
    across processes): the summed rate of the copies, with the process count."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        res = pool.map(_cpu_worker, [seconds] * n)
    return sum(v for v, _ in res), n, sum(k for _, k in res)


def matched_error(xf, torch, log=None):
    """Mixed and batched forms against the plain FP64 path at matched survival-probability error.

    Each candidate integrates the same window from the initial condition; its error is the largest
    |P_ee - P_ee,ref| over every beam against the FP64 DP45 run at rtol = atol = 1e-9 (the GPU FP64
    path, itself pinned to the oracle at 1e-10).  The speedup at 1e-4 is the time of the fastest
    FP64 candidate whose error is within 1e-4 over that of the fastest mixed candidate within 1e-4.
    Windows (no matter, so that the collective flavour evolution of the small case's physics
    happens inside them): the 4M-beam grid over 100 -> 110 km; the 64 batched instances over
    100 -> 101 km, the mixed form all instances in one persistent launch per chunk of steps, the
    FP64 path one instance after another; the three-flavour grid (256 E x 512 u) over
    100 -> 102 km."""
    from bulb_inputs import Workload, batched_workloads, workload_3f_fp64
    stream = torch.cuda.current_stream()

    def run(wls, precision, integrator, tol, r0, r1, per_instance):
        groups = [[w] for w in wls] if per_instance else [wls]
        ms, acc, rej, pees = 0.0, 0, 0, []
        for grp in groups:
            cfgs = [xf.config_from_workload(w, precision=precision, integrator=integrator, rtol=tol,
                                            atol=tol, h0_km=1e-3, steps_per_launch=64) for w in grp]
            for c in cfgs:
                c.cuda_stream = stream.cuda_stream
            sv = xf.Solver(cfgs)
            for i, w in enumerate(grp):
                sv.set_spectra(w.spectra(), inst=i)
            sv.reset(r0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if len(grp) == 1:
                sv.evolve(r0, r1)
            else:
                sv.evolve_batch([r1] * len(grp))
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            for i in range(len(grp)):
                st = sv.stats(inst=i)
                acc, rej = acc + st.accepted, rej + st.rejected
                pees.append(sv.pee(inst=i)[0])
            sv.close()
        return ms, acc, rej, np.concatenate(pees)

    def compare(name, wls, r0, r1, batched):
        ref_ms, ra, rr, ref = run(wls, "fp64", "dp45", 1e-9, r0, r1, True)
        rows = [{"form": "fp64 dp45 rtol 1e-9 (reference)", "precision": "fp64", "ms": ref_ms,
                 "accepted": ra, "rejected": rr, "max_abs_dpee": 0.0}]
        plan = [("fp64", "dp45", 1e-6, True), ("fp64", "lie_adaptive", 1e-6, True),
                ("mixed", "dp45", 1e-6, not batched), ("mixed", "lie_adaptive", 1e-6, not batched)]
        for prec, integ, tol, per in plan:
            ms, a, r, pee = run(wls, prec, integ, tol, r0, r1, per)
            rows.append({"form": f"{prec} {integ} rtol {tol:g}" + (" (all instances in one launch)" if not per else ""),
                         "precision": prec, "ms": ms, "accepted": a, "rejected": r,
                         "max_abs_dpee": float(np.abs(pee - ref).max())})
            if log:
                log(json.dumps(rows[-1]))
        ok64 = [x["ms"] for x in rows if x["precision"] == "fp64" and x["max_abs_dpee"] <= 1e-4]
        okmx = [x["ms"] for x in rows if x["precision"] == "mixed" and x["max_abs_dpee"] <= 1e-4]
        return {"window_km": [r0, r1], "beams": int(sum(w.n_beams for w in wls)), "instances": len(wls),
                "pee_change": float(np.abs(ref - 1.0).max()), "runs": rows,
                "speedup_at_1e-4": (min(ok64) / min(okmx)) if ok64 and okmx else None}

    big = workload_2f_large("mixed")
    big.matter = "none"
    single = compare("4M", [big], 100.0, 110.0, False)
    batch = [w for w in batched_workloads()]
    for w in batch:
        w.matter = "none"
    batched = compare("batched", batch, 100.0, 101.0, True)
    wl3 = workload_3f_fp64()
    wl3.matter = "none"
    three = compare("3f", [wl3], 100.0, 102.0, False)
    return single, batched, three


def compare_integrators():
    """Accuracy against cost of the integrators on the 4096-beam case (64 E x 32 u, FP64) over a
    window of strong collective evolution (100 -> 110 km): the exponential midpoint rule (the
    paper's kind of scheme: exact Eq. U propagators with a mid-point rule and adaptive steps),
    Dormand-Prince 5(4) and the fixed-step commutator-free Lie RK4, against a DP45 reference at
    rtol = atol = 1e-12.  One JSON line per run: max |P_ee - P_ee,ref| over all beams, stage
    evaluations, accepted / rejected steps, device time (CUDA events around xflat_evolve)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_1912_10596_gb300 import xflat as xf
    from bulb_inputs import workload_2f_small_fp64
    wl = workload_2f_small_fp64()
    r0, r1 = 100.0, 110.0

    def run(integrator, **over):
        cfg = xf.config_from_workload(wl, integrator=integrator, **over)
        cfg.cuda_stream = torch.cuda.current_stream().cuda_stream
        s = xf.Solver(cfg)
        s.set_spectra(wl.spectra())
        s.reset(r0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        s.evolve(r0, r1)
        e1.record()
        torch.cuda.synchronize()
        pee, _ = s.pee()
        st = s.stats()
        return pee, st, e0.elapsed_time(e1)

    ref, _, _ = run("dp45", rtol=1e-12, atol=1e-12, h0_km=1e-3)
    plan = [("exp_midpoint", dict(rtol=t, atol=t, h0_km=1e-3)) for t in (1e-4, 1e-5, 1e-6, 1e-7)]
    plan += [("dp45", dict(rtol=t, atol=t, h0_km=1e-3)) for t in (1e-6, 1e-7, 1e-8, 1e-9, 1e-10)]
    plan += [("lie_rk4", dict(fixed_dr_km=(r1 - r0) / n)) for n in (250, 500, 1000, 2000, 4000)]
    plan += [("rk4", dict(fixed_dr_km=(r1 - r0) / n)) for n in (250, 500, 1000, 2000, 4000)]
    for integ, over in plan:
        pee, st, ms = run(integ, **over)
        print(json.dumps({"integrator": integ, **{k: v for k, v in over.items() if k != "atol"},
                          "max_abs_dpee": float(np.abs(pee - ref).max()), "stage_evals": int(st.stage_evals),
                          "accepted": int(st.accepted), "rejected": int(st.rejected), "device_ms": ms,
                          "workload": wl.name, "window_km": [r0, r1]}))


def measure_configs(only=None):
    """Device rates of the other workloads (they are parity-test configurations, not benchmark
    lines): CUDA events on the launching stream, the L2 flushed before every timed launch.  One
    JSON line per workload: beam-stage updates per second, time per step, and the algorithmic
    bytes per beam-stage over the launch time against the measured HBM copy bandwidth.

    * 4096-beam case (64 E x 32 u, FP64): commutator RK4 with its step (0.0945 km) over 100 -> 200 km,
      and Lie RK4 (CF4) over the whole 11 -> 200 km in 2000 steps;
    * three flavours (256 E x 512 u, FP64 DP45, both hierarchies): a window of steps from 11 km;
    * 64 batched instances (mixed DP45, about 29 M beams): a window of steps from 11 km, one
      persistent launch per chunk for all instances;
    * adjoint (200 E x 400 u, FP64 RK4, 5000 steps over 100 -> 300 km, checkpoints every 64 steps):
      time per gradient;
    * extended bulb model, 100 E x 10 phi x 2000 u (4M beams, mixed DP45): a window of steps."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_1912_10596_gb300 import xflat as xf
    from bulb_inputs import (Workload, workload_2f_small_fp64, workload_3f_fp64, batched_workloads,
                             workload_adjoint)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    hbm, peak_kind = _peaks()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def line(name, beams, bsu, ms, steps, bpbs, **extra):
        rate = bsu / (ms / 1e3)
        out = {"workload": name, "beams": beams, "beam_stage_updates": bsu, "device_ms": ms,
               "ms_per_step": ms / steps if steps else None, "beam_updates_per_s": rate,
               "bytes_per_beam_stage": bpbs,
               "hbm_frac": (bpbs * rate / 1e9) / hbm if bpbs else None, "peak": f"{hbm} GB/s ({peak_kind})"}
        out.update(extra)
        print(json.dumps(out), flush=True)

    def solver(cfgs, spectra):
        for c in cfgs:
            c.cuda_stream = stream.cuda_stream
        sv = xf.Solver(cfgs)
        for i, N in enumerate(spectra):
            sv.set_spectra(N, inst=i)
        return sv

    def window(sv, r1s, steps, per_launch=8, warmup=3):
        """Time `steps` steps of every instance from its current radius (launches of per_launch
        steps, L2 flushed before each); returns (ms, beam-stage updates)."""
        sv.advance(r1s, max_steps=1)
        for _ in range(warmup - 1):
            sv.advance(None, max_steps=1)
        torch.cuda.synchronize()
        b0 = sv.stats(0).beam_stage_updates                  # the handle's total over its instances
        ms = 0.0
        for n in launch_chunks(steps, per_launch):
            flush_l2(flush_buf)
            e0, e1 = ev(), ev()
            e0.record(stream)
            sv.advance(None, max_steps=n)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        st = [sv.stats(i) for i in range(sv.n_inst)]
        if any(x.status != 0 for x in st):
            raise RuntimeError("device status " + str([x.status for x in st]))
        return ms, st[0].beam_stage_updates - b0

    def want(name):
        return only is None or only == name

    # 4096-beam case: whole radial ranges, one xflat_evolve each (warm-up run first)
    wl = workload_2f_small_fp64()
    h = (wl.r1 - wl.r0) / wl.n_steps
    for integ, r0 in (("rk4", 100.0), ("lie_rk4", wl.r0)) if want("small") else ():
        sv = solver([xf.config_from_workload(wl, integrator=integ, fixed_dr_km=h)], [wl.spectra()])
        for rep in range(2):
            sv.reset(r0)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            sv.evolve(r0, wl.r1)
            e1.record(stream)
            torch.cuda.synchronize()
        st = sv.stats()
        steps = int(st.accepted)
        line(f"{wl.name} ({integ}, {r0:g} -> {wl.r1:g} km)", wl.n_beams, st.beam_stage_updates,
             e0.elapsed_time(e1), steps, 30.0, passes_per_step=4,
             us_per_pass=1e3 * e0.elapsed_time(e1) / (4 * steps))
        sv.close()

    # three flavours, both hierarchies
    for dm31 in (2.4e-3, -2.4e-3) if want("3f") else ():
        wl = workload_3f_fp64(dm31)
        sv = solver([xf.config_from_workload(wl)], [wl.spectra()])
        ms, bsu = window(sv, [wl.r1], 16)
        line(wl.name, wl.n_beams, bsu, ms, 16, 84.0, window="16 DP45 steps from 11 km")
        sv.close()

    # 64 batched instances
    if want("batched"):
        wls = batched_workloads()
        sv = solver([xf.config_from_workload(w) for w in wls], [w.spectra() for w in wls])
        ms, bsu = window(sv, [w.r1 for w in wls], 16)
        total = sum(w.n_beams for w in wls)
        line("batched 64 instances (seed 0x5EED0003)", total, bsu, ms, 16, 14.0,
             window="16 DP45 steps of every instance from 11 km", state_bytes=12 * total,
             block_size=sv.stats().block_size, blocks=sv.stats().grid_blocks)
        sv.close()
    # extended bulb model in the shape of the paper's runs (energies x azimuthal x polar bins,
    # Sec. 4.2): 100 E x 10 phi x 2000 u x (nu, nubar) = 4M beams, mixed DP45, four moments
    if want("extended"):
        wl = Workload(name="bulb2f_ext_100E_10phi_2000u_mixed_dp45", n_energy=100, n_angle=2000,
                      matter="power_law", r0=11.0, r1=500.0, integrator="dp45", precision="mixed",
                      rtol=1e-6, atol=1e-6)
        sv = solver([xf.config_from_workload(wl, n_phi=10)], [wl.spectra()])
        ms, bsu = window(sv, [wl.r1], 16)
        nb = sv.nbeams()
        line(wl.name, nb, bsu, ms, 16, 14.0, window="16 DP45 steps from 11 km",
             block_size=sv.stats().block_size, blocks=sv.stats().grid_blocks)
        sv.close()
    # the configured radial ranges from r = R with the adaptive exact propagators: the 4M-beam case
    # (mixed at rtol 1e-6 over all of 11 -> 500 km; FP64 at 1e-6 and 1e-9 for a bounded wall time)
    # and the three-flavour case over 11 -> 1000 km (mixed; FP64 for a bounded wall time), and the
    # explicit DP45 step near R for comparison (mixed 4M beams; FP64 three flavours)
    if want("range") or only == "range3f":
        from bulb_inputs import workload_2f_large
        budget = 30.0

        def range_run(wl, precision, integrator, tol, r1, n_per_launch=64):
            cfg = xf.config_from_workload(wl, precision=precision, integrator=integrator, rtol=tol, atol=tol,
                                          h0_km=1e-9, steps_per_launch=n_per_launch)
            sv = solver([cfg], [wl.spectra()])
            sv.reset(wl.r0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0, e1 = ev(), ev()
            e0.record(stream)
            sv.advance([r1], max_steps=n_per_launch)
            marks = []
            while True:
                sv.advance(None, max_steps=n_per_launch)
                torch.cuda.synchronize()
                st = sv.stats()
                marks.append((round(time.perf_counter() - t0, 3), st.r_km, int(st.accepted), int(st.rejected)))
                if st.r_km >= r1 or st.status or time.perf_counter() - t0 > budget:
                    break
            e1.record(stream)
            torch.cuda.synchronize()
            st = sv.stats()
            pee, mean = sv.pee()
            out = {"workload": wl.name, "integrator": integrator, "precision": precision, "rtol": tol,
                   "beams": wl.n_beams, "r_start_km": wl.r0, "r_reached_km": st.r_km, "r_target_km": r1,
                   "accepted": int(st.accepted), "rejected": int(st.rejected), "status": int(st.status),
                   "device_ms": e0.elapsed_time(e1), "wall_s": time.perf_counter() - t0,
                   "beam_stage_updates": int(st.beam_stage_updates), "pee_min": float(pee.min()),
                   "pee_mean": float(mean), "progress": marks[:: max(1, len(marks) // 10)]}
            print(json.dumps(out), flush=True)
            sv.close()

        def range_run_batch(wls, precision, integrator, tol, n_per_launch=64):
            """All instances of a batch in one handle, each to its own configured end radius."""
            cfgs = [xf.config_from_workload(w, precision=precision, integrator=integrator, rtol=tol, atol=tol,
                                            h0_km=1e-9, steps_per_launch=n_per_launch) for w in wls]
            sv = solver(cfgs, [w.spectra() for w in wls])
            sv.reset(wls[0].r0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0, e1 = ev(), ev()
            e0.record(stream)
            sv.advance([w.r1 for w in wls], max_steps=n_per_launch)
            while True:
                done = sv.advance(None, max_steps=n_per_launch)
                sts = [sv.stats(i) for i in range(len(wls))]
                if done or any(x.status for x in sts) or time.perf_counter() - t0 > budget:
                    break
            e1.record(stream)
            torch.cuda.synchronize()
            sts = [sv.stats(i) for i in range(len(wls))]
            pmin = min(float(sv.pee(inst=i)[0].min()) for i in range(len(wls)))
            out = {"workload": f"batched {len(wls)} instances (seed 0x5EED0003)", "integrator": integrator,
                   "precision": precision, "rtol": tol, "beams": int(sum(w.n_beams for w in wls)),
                   "r_start_km": wls[0].r0, "r_reached_km_min": min(x.r_km for x in sts),
                   "r_target_km": wls[0].r1, "instances_done": sum(1 for x, w in zip(sts, wls) if x.r_km >= w.r1),
                   "accepted_sum": int(sum(x.accepted for x in sts)), "rejected_sum": int(sum(x.rejected for x in sts)),
                   "accepted_max": int(max(x.accepted for x in sts)), "status": [int(x.status) for x in sts if x.status],
                   "device_ms": e0.elapsed_time(e1), "wall_s": time.perf_counter() - t0, "pee_min": pmin}
            print(json.dumps(out), flush=True)
            sv.close()

        if only == "range3f":
            # the three-flavour configured range alone (normal hierarchy, mixed): a short command
            # for profiling the three-flavour exponential kernel
            wl3 = workload_3f_fp64()
            range_run(wl3, "mixed", "lie_adaptive", 1e-6, wl3.r1)
            return
        big = workload_2f_large("mixed")
        range_run(big, "mixed", "lie_adaptive", 1e-6, big.r1)
        range_run(big, "fp64", "lie_adaptive", 1e-6, big.r1)
        range_run(big, "fp64", "lie_adaptive", 1e-9, big.r1)
        range_run(big, "mixed", "dp45", 1e-6, big.r1, n_per_launch=256)
        # three flavours, both hierarchies: the adaptive exact propagators (3 x 3 Eq. U by
        # eigen-decomposition) over the whole 11 -> 1000 km, and explicit DP45 from R for comparison
        for dm31 in (2.4e-3, -2.4e-3):
            wl3 = workload_3f_fp64(dm31)
            range_run(wl3, "mixed", "lie_adaptive", 1e-6, wl3.r1)
            range_run(wl3, "fp64", "lie_adaptive", 1e-6, wl3.r1)
        wl3 = workload_3f_fp64()
        range_run(wl3, "fp64", "dp45", 1e-9, wl3.r1, n_per_launch=256)
        # the 64 batched instances over their configured 11 -> 300 km in one handle
        range_run_batch(batched_workloads(), "mixed", "lie_adaptive", 1e-6)
    if not want("adjoint"):
        return

    # adjoint
    wl = workload_adjoint()
    r0, r1 = 100.0, 300.0
    sv = solver([xf.config_from_workload(wl, fixed_dr_km=(r1 - r0) / wl.n_steps)], [wl.spectra()])
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv.adjoint(r0, r1, wl.n_steps, 64)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    fwd = wl.n_beams * 4 * wl.n_steps
    line(f"{wl.name} ({r0:g} -> {r1:g} km, K = 64)", wl.n_beams, fwd, 1e3 * dt, wl.n_steps, None,
         seconds_per_gradient=dt, note="beam_stage_updates counts the forward stages only; the "
         "gradient also recomputes every segment and runs the adjoint sweep (wall clock around xflat_adjoint)")
    sv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-matched", action="store_true",
                    help="skip the speedups at matched survival-probability error")
    ap.add_argument("--repeats", type=int, default=5, help="repeats behind the median timings")
    ap.add_argument("--steps-per-launch", type=int, default=8,
                    help="radial steps per persistent launch in the timed region (L2 flushed before each)")
    ap.add_argument("--compare-integrators", action="store_true",
                    help="accuracy against cost of the integrators on the 4096-beam case instead of the benchmark")
    ap.add_argument("--configs", action="store_true",
                    help="device rates of the other workloads (small, three-flavour, batched, adjoint) instead of the benchmark")
    ap.add_argument("--only", choices=["small", "3f", "batched", "extended", "adjoint", "range", "range3f"],
                    help="with --configs: measure one of the workloads")
    args = ap.parse_args()
    if args.compare_integrators:
        compare_integrators()
        return
    if args.configs:
        measure_configs(args.only)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    wl = workload_2f_large("mixed")

    if args.impl == "reference":
        if rank != 0:
            return
        per_step = []
        for _ in range(args.warmup):
            cpu_baseline(impl_steps=1)
        for _ in range(args.steps):
            v, n, dt, beams = cpu_baseline(impl_steps=1)
            per_step.append(dt)
        value = 2 * 20 * wl.n_energy * 6 * args.steps / sum(per_step)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "beam-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(per_step) / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl.name, "beams": wl.n_beams, "integrator": "dp45",
                           "r_start_km": 11.0, "sample_beams": 2 * 20 * wl.n_energy},
                "cpu_baseline": {"value": value, "unit": "beam-updates/s", "cores": 1, "kind": "oracle",
                                 "sample": "FP64 numpy oracle, Dormand-Prince steps at r = 11 km on 1000 E x first 20 of 2000 u bins x (nu, nubar)"},
                "e2e": {"value": value, "unit": "beam-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_1912_10596_gb300 import xflat as xf
    from paper_1912_10596_gb300 import shard

    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    flush = lambda: flush_l2(flush_buf)  # noqa: E731

    shape = None
    if not args.no_tune:
        from paper_1912_10596_gb300 import autotune
        shape = autotune.tune(xf, [bench_config(xf, wl, "mixed")], [wl.spectra()], [wl.r1],
                              log=lambda m: print(m, file=sys.stderr))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    spl = max(1, args.steps_per_launch)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, chunks, bsu, st, solver = time_device_steps(xf, torch, wl, "mixed", args.steps, args.warmup,
                                                        flush, shape, spl)
        rep_main = repeat_stats(torch, solver, max(200, args.steps), args.repeats, flush, spl)
    clocks = clk.summary()
    t_ms = shard.max_over_ranks(sum(ms))                      # the slowest rank's time
    value = world * bsu * args.steps / (t_ms / 1e3)
    hbm, peak_kind = _peaks()
    # algorithmic bytes of all timed launches over their summed CUDA-event durations (= per launch
    # bytes over the mean launch duration when the launches are equal)
    achieved = BYTES_PER_BEAM_STAGE[("mixed", "dp45")] * bsu * args.steps / (sum(ms) / 1e3) / 1e9

    # accepted-only rate: the stages of accepted steps only (a rejected DP45 attempt evaluates 6
    # stages too); the all-attempt rate is `value`
    acc_frac = solver.timed_accepted_fraction
    fp64 = None
    if not args.no_fp64:
        k64 = max(20, args.steps // 4)
        ms64, _, bsu64, st64, s64 = time_device_steps(xf, torch, wl, "fp64", k64, args.warmup, flush,
                                                      None, spl)
        v64 = bsu64 * k64 / (sum(ms64) / 1e3)
        rep64 = repeat_stats(torch, s64, k64, args.repeats, flush, spl)
        fp64 = {"value": v64, "unit": "beam-updates/s", "ms_per_step": sum(ms64) / k64,
                "repeats": rep64,
                "speedup_mixed_vs_fp64_per_step": (bsu * args.steps / (sum(ms) / 1e3)) / v64}
        s64.close()
    e2e = None
    if not args.no_e2e:
        k_e2e = max(20, args.steps // 4)
        runs = [e2e_steps(xf, torch, solver, wl, k_e2e) for _ in range(args.repeats)]
        v_e2e = statistics.median(r[0] for r in runs)
        e2e = {"value": world * v_e2e, "unit": "beam-updates/s", "h2d_bytes_per_step": runs[0][1],
               "d2h_bytes_per_step": runs[0][2], "steps_per_repeat": k_e2e, "repeats": args.repeats,
               "median_of_repeats": True}
    matched = None
    if rank == 0 and not args.no_matched:
        single, batched, three = matched_error(xf, torch, log=lambda m: print(m, file=sys.stderr))
        matched = {"speedup_mixed_vs_fp64_at_1e-4": single["speedup_at_1e-4"],
                   "speedup_batched_vs_fp64_at_1e-4": batched["speedup_at_1e-4"],
                   "speedup_mixed_vs_fp64_at_1e-4_three_flavours": three["speedup_at_1e-4"],
                   "single": single, "batched": batched, "three_flavours": three}
    cpu = None
    if rank == 0 and not args.no_cpu:
        v, n, dt, beams = cpu_baseline()
        v_all, nproc, n_all = cpu_baseline_all_cores()
        cpu = {"value": v, "unit": "beam-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"FP64 numpy oracle, {n} Dormand-Prince steps at r = 11 km on 1000 E x first 20 of 2000 u bins x (nu, nubar) = {beams} beams, {dt:.1f} s",
               "all_cores": {"value": v_all, "unit": "beam-updates/s", "cores": nproc, "nproc": nproc,
                             "sample": f"the same sample as {nproc} independent processes (spawn), 12 s each, {n_all} steps in all"}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "beam-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "beams": wl.n_beams, "integrator": "dp45",
                       "precision": "mixed: f32 per-beam algebra and moment contributions, FP64-accurate (exact integer) moment sums, exact max error norm, f64 step control",
                       "r_start_km": 11.0, "stage_evals_per_step": bsu / wl.n_beams,
                       "steps_per_launch": spl,
                       "l2": f"flushed before every timed launch of up to {spl} steps (write of a 258 MB buffer)",
                       "grid_blocks": st.grid_blocks, "block_size": st.block_size,
                       "autotuned_shape": list(shape) if shape else None},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": step_traffic(spl),
                         "note": f"{BYTES_PER_BEAM_STAGE[('mixed', 'dp45')]} algorithmic B per beam-stage "
                                 f"({BYTES_PER_BEAM_STAGE[('mixed', 'dp45')] * bsu * spl / 1e9:.2f} GB per {spl}-step launch); "
                                 f"traffic = DRAM bytes per {spl}-step launch; peak {peak_kind}",
                         "issue": issue_roofline(t_ms / args.steps, (clocks or {}).get("sm_mhz"),
                                                 torch.cuda.get_device_properties(0).multi_processor_count)},
            "accepted_value": value * acc_frac,
            "repeats": rep_main,
            "clocks": clocks,
            "gpu_launches": len(chunks),
            "matched_error": matched,
            "speedup_mixed_vs_fp64_at_1e-4": matched["speedup_mixed_vs_fp64_at_1e-4"] if matched else None,
            "speedup_batched_vs_fp64_at_1e-4": matched["speedup_batched_vs_fp64_at_1e-4"] if matched else None,
            "fp64_path": fp64,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
