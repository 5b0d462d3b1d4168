"""Launch-shape autotuner for the persistent step kernel.

For one workload it times a few radial steps for every candidate (threads per block, resident
blocks per SM) -- which also selects the kernel's register budget, see csrc/kernels_2f.cu -- and
returns the fastest.  Results are cached per (GPU, workload signature) in _build/autotune.json.
All timing runs through the library's own launches (xflat_advance) with CUDA events.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_build", "autotune.json")

# (block_size, blocks_per_sm): 768 or 512 resident threads per SM
CANDIDATES_MIXED_2F = [(256, 3), (256, 2), (512, 1), (128, 6), (128, 4)]
CANDIDATES_OTHER = [(256, 1), (128, 2)]


def _signature(cfg, n_inst, gpu):
    return (f"{gpu}|nf{cfg.n_flavor}|p{cfg.precision}|i{cfg.integrator}|"
            f"E{cfg.n_energy}|u{cfg.n_angle}|n{n_inst}")


def _time(xf, torch, cfgs, spectra, r_end, steps, warmup):
    stream = torch.cuda.current_stream()
    for c in cfgs:
        c.cuda_stream = stream.cuda_stream
        c.steps_per_launch = 1
    s = xf.Solver(cfgs)
    for i, N in enumerate(spectra):
        s.set_spectra(N, inst=i)
    s.advance(r_end, max_steps=1)
    for _ in range(warmup):
        s.advance(None, max_steps=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        s.advance(None, max_steps=1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = s.stats()
    s.close()
    return ms, st.status


def tune(xf, cfgs, spectra, r_end, steps=6, warmup=2, use_cache=True, log=None):
    """Return (block_size, blocks_per_sm) of the fastest candidate for these instance configs."""
    import torch

    gpu = torch.cuda.get_device_name()
    key = _signature(cfgs[0], len(cfgs), gpu)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except Exception:
            cache = {}
    if key in cache:
        return tuple(cache[key]["best"])
    mixed2f = cfgs[0].precision == xf.MIXED and cfgs[0].n_flavor == 2
    cands = CANDIDATES_MIXED_2F if mixed2f else CANDIDATES_OTHER
    results = {}
    for bs, bps in cands:
        trial = []
        for c in cfgs:
            t = xf.xflat_config.from_buffer_copy(c)
            t.block_size, t.blocks_per_sm = bs, bps
            trial.append(t)
        try:
            ms, status = _time(xf, torch, trial, spectra, r_end, steps, warmup)
        except xf.XflatError:
            continue
        if status == 0:
            results[f"{bs}x{bps}"] = ms
            if log:
                log(f"autotune {key}: block {bs} x {bps}/SM: {ms:.4f} ms/step")
    best = min(results, key=results.get)
    best_t = tuple(int(x) for x in best.split("x"))
    cache[key] = {"best": best_t, "ms_per_step": results}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return best_t
