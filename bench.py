"""Benchmark: DFSPH particle-steps/s on the large rigid-coupling dam break (1.2M fluid
particles, 3 floating boxes, CFL dt <= 1e-3 s, 0.1 % density and divergence tolerance).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  The timed region is K CUDA-graph steps on the library's
stream, bracketed by CUDA events; `e2e` repeats the measurement through the C ABI with
each step's result (positions) copied to pinned host memory; `roofline` reports the
dominant kernel from a second pass of eager, CUDA-event-timed steps; `cpu_baseline` times
the CPU oracle on a bounded sample.  With N > 1 (torchrun) every rank runs an
independent replica of the scene (the scene does not shard; scaling is weak).

Secondary sections of the same line (rank 0; `--no-learned`, `--no-batched` skip them):
`learned_vs_plain` (the warm-start network trained in the run, then zero / previous-step /
learned warm starts on the 8k and the 1.2M dam breaks and the 64-scene batch),
`batched_64_scenes` (sharded over the ranks), `wcsph_1.2M`, `solvers_8k` (DFSPH, PCISPH,
WCSPH), `viscous_column_250k` (implicit viscosity), `coupling_1.2M` (weak vs strong) and
`post_processing_1.2M`.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DFSPH particle-steps/s at 0.1% density error, learned vs plain; %HBM peak"
UNIT = "particle-steps/s"
WORKLOAD = ("dam break with two-way rigid coupling: 125x98x98 = 1,200,500 fluid particles "
            "(r = 0.005 m) in a 2x1x1 m one-layer tank, 3 rigid boxes (0.1 m, 500 kg/m^3), "
            "CFL dt <= 1e-3 s, eta = 0.1% density / 0.1% divergence")

# Algorithmic bytes per fluid particle of each kernel: the particle's own state read and
# written once (neighbour data is reused on chip; the neighbour lists are an
# implementation choice and not counted), plus the boundary particles' state once.
ALGO_BYTES = {
    "dens_pass_a": 44, "div_pass_a": 44,        # x, v, rho, alpha, kappa_sum -> kappa/rho, kappa_sum
    "dens_pass_b": 40, "div_pass_b": 40,        # x, kappa/rho, v -> v
    "dens_warm_pass_b": 40, "div_warm_pass_b": 40,
    "density_alpha": 52,                        # x, v, kappa_v_prev -> rho, alpha, counts, kappa_v, kappa/rho
    "nonpressure": 56,                          # x, v, rho -> v*, rho, kappa_sum, kappa0, kappa/rho
    "warm_density": 48,                         # x, v*, rho, kappa_prev -> kappa0, kappa_sum, kappa/rho
}
BOUNDARY_BYTES = 16                             # x_b, Psi_b per boundary particle and sweep
# DRAM bytes (read + write) per launch measured by ncu on this workload at 1 thread per
# particle, gather batch 4 and cell size h (1 + 2^-8), for the kernels as they are built
# now (the roofline's `traffic`; null for any other kernel or configuration).  Filled from
# the committed captures (profiles/*_dam_break_1.2M.md); a kernel changed since its capture
# has no entry.
TRAFFIC = {("density_alpha", 1, 4, 27): 82.70e6 + 169.47e6,
           ("dens_pass_a", 1, 4, 27): 211.59e6 + 4.72e6,
           ("dens_pass_b", 1, 4, 27): 199.69e6 + 4.33e6}
# L1 data-pipe (LSU) wavefronts per launch measured by ncu in the same captures
# (l1tex__data_pipe_lsu_wavefronts, per-SM average x 152 SMs).  The pipe takes one wavefront per
# SM per cycle, so over the live launch time this is the fraction of the roof that binds the
# neighbour gathers.
L1_WAVEFRONTS = {("density_alpha", 1, 4, 27): 617053.83 * 152,
                 ("dens_pass_a", 1, 4, 27): 203077.14 * 152,
                 ("dens_pass_b", 1, 4, 27): 124865.32 * 152}
# FP32 operations per neighbour pair in the list sweeps (distance, spline gradient, dot)
FLOPS_PER_PAIR = {"dens_pass_a": 26, "div_pass_a": 24, "dens_pass_b": 22, "div_pass_b": 22,
                  "dens_warm_pass_b": 22, "div_warm_pass_b": 22, "nonpressure": 30,
                  "warm_density": 26, "density_alpha": 40}
# extra FP32 operations per fluid particle outside the pair sums: the density sweep's
# candidate tests (about 216 per particle at 8 flop each: 3 differences, 3 products, 2 sums)
FLOPS_PER_PARTICLE = {"density_alpha": 216 * 8}
# the kernels reported with a roofline of their own (the step's three largest)
ROOFLINE_KERNELS = ("density_alpha", "dens_pass_a", "dens_pass_b")
# launches per step of a kernel in the timed region, from the solver iteration counts
# (the eager timing pass runs later steps, whose iteration counts differ)
PER_DENSITY_ITERATION = ("dens_pass_a", "dens_pass_b", "dens_check")
PER_DIVERGENCE_ITERATION = ("div_pass_a", "div_pass_b", "div_check")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    def __init__(self, path, index=0):
        self.path = path
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(desc, steps=2):
    """The oracle on the host cores: `steps` steps of the full workload with every core
    (OpenMP), and one step of the reference arm's scaled copy on one thread."""
    import oracle
    oracle.build()
    o = oracle.Scene(desc)
    t = time.perf_counter()
    for _ in range(steps):
        o.step(0.0)
    el = time.perf_counter() - t
    n = len(desc["fluid_x"])
    cores = oracle.num_threads()
    d1 = reference_sample()
    o1 = oracle.Scene(d1)
    oracle.set_num_threads(1)
    try:
        t = time.perf_counter()
        o1.step(0.0)
        el1 = time.perf_counter() - t
    finally:
        oracle.set_num_threads(cores)
    n1 = len(d1["fluid_x"])
    return {"value": n * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d oracle steps of the full %d-particle workload from its initial state "
                      "(FP64, OpenMP, %.1f s)" % (steps, n, el),
            "single_thread": {"value": n1 / el1, "unit": UNIT, "cores": 1,
                              "sample": "1 oracle step of a %d-particle scaled copy of the workload "
                                        "from its initial state (FP64, %.1f s)" % (n1, el1)}}


def learned_vs_plain():
    """Train the warm-start network on the GPU from the solver's own states (200k samples
    from 500 steps of seeded 0.5M-1.2M-particle dam breaks) and compare the zero,
    previous-step and learned warm starts on the 8k-particle dam break (100 steps, fixed
    dt = 4e-4 s) at the 0.1 % tolerance and at 0.001 %, and on the 1.2M-particle rigid dam
    break (200 steps from rest, CFL dt, 0.1 %)."""
    import time as _t
    from paper_2403_11156_gb300 import scenes, warmstart
    t = _t.perf_counter()
    f, y = warmstart.generate_dataset(200_000, 500)
    t_data = _t.perf_counter() - t
    t = _t.perf_counter()
    params, hist = warmstart.train(f, y, epochs=30)
    t_train = _t.perf_counter() - t
    out = {"samples": int(f.shape[0]), "data_s": round(t_data, 3), "train_s": round(t_train, 3),
           "train_loss_first": float(hist[0]), "train_loss_last": float(hist[-1])}
    # the learned start also runs gated: held back (previous-step start instead) in a step
    # whose previous density solve sat at the 2-iteration floor
    for tag, eta in (("eta_1e-3", 1e-3), ("eta_1e-5", 1e-5)):
        desc = scenes.dam_break_small(eta_density=eta, eta_divergence=eta)
        out[tag] = warmstart.compare_warm_starts(desc, params, steps=100, gate=2)
    big = scenes.dam_break_rigid()
    out["dam_break_1.2M_rigid"] = warmstart.compare_warm_starts(big, params, steps=200, gate=2)
    for mode in out["dam_break_1.2M_rigid"].values():
        mode["particle_steps_per_s"] = len(big["fluid_x"]) / (mode["ms_per_step"] / 1000.0)
    for res in (out["eta_1e-3"], out["eta_1e-5"], out["dam_break_1.2M_rigid"]):
        # the solves' iteration floor: at least 2 density and 1 divergence iterations per step
        res["iteration_floor"] = {"density": 2, "divergence": 1}
        p = res["previous"]
        for key in ("learned", "learned_gated"):
            l = res[key]
            res[key + "_over_previous"] = {
                "density_iteration_ratio": p["density_iters_per_step"] / l["density_iters_per_step"],
                "solver_iteration_ratio": (p["density_iters_per_step"] + p["divergence_iters_per_step"]) /
                                          (l["density_iters_per_step"] + l["divergence_iters_per_step"]),
                "time_ratio": p["ms_per_step"] / l["ms_per_step"]}
    return out, params


def learned_headline(desc, params, steps, warmup, autotune, stream, gate=0):
    """The benchmark workload with the learned warm start, over the same region as the
    plain `value`: `warmup` untimed graph steps from the same initial state, then `steps`
    graph steps timed with CUDA events on the library stream."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    d = dict(desc)
    d["warm_start"] = scenes.WARM_LEARNED
    d["learned_gate"] = gate
    n = len(d["fluid_x"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with sph.Context(d, stream=stream, autotune=autotune) as g:
        g.sph_set_mlp(params)
        g.sph_steps(warmup, 0.0)
        g.sph_synchronize(raise_on_error=False)
        s0 = g.sph_get_stats()
        torch.cuda.synchronize()
        a.record(stream)
        g.sph_steps(steps, 0.0)
        b.record(stream)
        torch.cuda.synchronize()
        status = g.sph_synchronize(raise_on_error=False)
        s1 = g.sph_get_stats()
    ms = a.elapsed_time(b) / steps
    return {"value": n / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "mean_density_iters": (s1["total_dens_iters"] - s0["total_dens_iters"]) / steps,
            "mean_divergence_iters": (s1["total_div_iters"] - s0["total_div_iters"]) / steps,
            "final_density_error": s1["dens_err"], "status": sph.STATUS_NAMES[status],
            "learned_gate": gate}


def batched_learned(params, steps=200):
    """The 64-scene batch (as in batched_throughput) with the previous-step and the learned
    warm starts: 200 graph steps after 5 warm-up steps (the first steps from rest sit at the
    minimum iteration counts under either start); ms per step and mean iterations."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    out = {}
    for name, mode, gate in (("previous", scenes.WARM_PREVIOUS, 0), ("learned", scenes.WARM_LEARNED, 0),
                             ("learned_gated", scenes.WARM_LEARNED, 2)):
        ds = scenes.batch_dam_break()
        for d in ds:
            d["warm_start"] = mode
            d["learned_gate"] = gate
        nf = sum(len(d["fluid_x"]) for d in ds)
        stream = torch.cuda.Stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with sph.Context(ds, stream=stream, autotune=True) as g:
            if mode == scenes.WARM_LEARNED:
                g.sph_set_mlp(params)
            g.sph_steps(5, 0.0)
            g.sph_synchronize(raise_on_error=False)
            s0 = [g.sph_get_stats(k) for k in range(len(ds))]
            a.record(stream)
            g.sph_steps(steps, 0.0)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / steps
            s1 = [g.sph_get_stats(k) for k in range(len(ds))]
        dens = [(y["total_dens_iters"] - x["total_dens_iters"]) / steps for x, y in zip(s0, s1)]
        div = [(y["total_div_iters"] - x["total_div_iters"]) / steps for x, y in zip(s0, s1)]
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": nf / (ms / 1000.0),
                     "mean_density_iters": float(np.mean(dens)), "max_density_iters": float(np.max(dens)),
                     "mean_divergence_iters": float(np.mean(div))}
    out["time_ratio"] = out["previous"]["ms_per_step"] / out["learned"]["ms_per_step"]
    out["gated_time_ratio"] = out["previous"]["ms_per_step"] / out["learned_gated"]["ms_per_step"]
    return out


def batched_throughput(steps=30, rank=0, world=1, barrier=lambda: None):
    """64 independent dam breaks (20k-200k particles, log-uniform, seed 5) in one autotuned
    context: every kernel of a step covers all scenes in one launch.  With several GPUs each rank
    steps its share of the scenes (largest first onto the least-loaded rank) and the
    whole-job rate is the sum of particles over the slowest rank's time.  Returns
    particle-steps/s of the batch and, on one GPU, of the same scenes stepped one at a
    time (8 of them, scaled)."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    from paper_2403_11156_gb300.sharding import reduce_timing, shard_scenes
    ds_all = scenes.batch_dam_break()
    mine = shard_scenes([len(d["fluid_x"]) for d in ds_all], world)[rank]
    ds = [ds_all[k] for k in mine]
    nf = sum(len(d["fluid_x"]) for d in ds)
    stream = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with sph.Context(ds, stream=stream, autotune=True) as g:
        tuning = g.sph_get_tuning()
        g.sph_steps(5, 0.0)
        g.sph_synchronize(raise_on_error=False)
        barrier()
        torch.cuda.synchronize()
        a.record(stream)
        g.sph_steps(steps, 0.0)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = a.elapsed_time(b) / steps
        st = [g.sph_get_stats(k) for k in range(len(ds))]
    ms, nf_all = reduce_timing(ms, nf, world, device="cuda")
    out = {"scenes": len(ds_all), "fluid_particles": int(nf_all), "ranks": world, "ms_per_step": ms,
           "autotune": {k: tuning[k] for k in ("tuned", "from_cache", "gather_batch", "cell_factor", "lanes")},
           "particle_steps_per_s": nf_all / (ms / 1000.0),
           "density_iters_range": [min(x["dens_iters"] for x in st), max(x["dens_iters"] for x in st)]}
    if world > 1:
        return out
    single_ms, single_n = 0.0, 0
    for k in range(0, len(ds), 8):
        with sph.Context(ds[k], stream=stream) as g:
            g.sph_steps(5, 0.0)
            g.sph_synchronize(raise_on_error=False)
            a.record(stream)
            g.sph_steps(steps, 0.0)
            b.record(stream)
            torch.cuda.synchronize()
            single_ms += a.elapsed_time(b) / steps
            single_n += len(ds[k]["fluid_x"])
    out["one_at_a_time_particle_steps_per_s"] = single_n / (single_ms / 1000.0)
    return out


def viscous_column_time(steps=300):
    """The 250k-particle high-viscosity column (nu = 0.1 m^2/s, implicit viscosity by
    matrix-free CG to 1e-4 relative residual every step) falling onto a plane: 300 graph
    steps from rest; ms per step, CG and solver iterations per step."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    d = scenes.viscous_column()
    n = len(d["fluid_x"])
    stream = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cg = []
    with sph.Context(d, stream=stream) as g:
        g.sph_steps(3, 0.0)
        g.sph_synchronize(raise_on_error=False)
        s0 = g.sph_get_stats()
        ms = 0.0
        for _ in range(steps // 10):
            a.record(stream)
            g.sph_steps(10, 0.0)
            b.record(stream)
            st = g.sph_get_stats()              # synchronises
            ms += a.elapsed_time(b)
            cg.append(st["cg_iters"])
        s1 = g.sph_get_stats()
    k = (steps // 10) * 10
    return {"fluid_particles": n, "boundary_particles": len(d["boundary_x"]), "steps": k,
            "ms_per_step": ms / k, "particle_steps_per_s": n * k / (ms / 1000.0),
            "cg_iters_last_step_mean": float(np.mean(cg)),
            "density_iters_per_step": (s1["total_dens_iters"] - s0["total_dens_iters"]) / k,
            "divergence_iters_per_step": (s1["total_div_iters"] - s0["total_div_iters"]) / k,
            "dt": s1["dt"], "status_flags": s1["flags"]}


def coupling_comparison(steps=500):
    """The 1.2M-particle rigid dam break with weak and with strong two-way coupling: 500
    graph steps from rest (the boxes fall about 0.4 s before they sit in the flow); ms per
    step, solver iterations per step and the boxes' final speeds."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    out = {}
    for name, mode in (("weak", scenes.COUPLING_WEAK), ("strong", scenes.COUPLING_STRONG)):
        d = scenes.dam_break_rigid(rigid_coupling=mode)
        n = len(d["fluid_x"])
        stream = torch.cuda.Stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with sph.Context(d, stream=stream) as g:
            g.sph_steps(3, 0.0)
            g.sph_synchronize(raise_on_error=False)
            s0 = g.sph_get_stats()
            a.record(stream)
            g.sph_steps(steps, 0.0)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / steps
            s1 = g.sph_get_stats()
            bodies = g.sph_read_bodies()
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": n / (ms / 1000.0),
                     "density_iters_per_step": (s1["total_dens_iters"] - s0["total_dens_iters"]) / steps,
                     "divergence_iters_per_step": (s1["total_div_iters"] - s0["total_div_iters"]) / steps,
                     "box_speeds": [float(np.linalg.norm(bd[7:10])) for bd in bodies]}
    return out


def wcsph_step_time(steps=50):
    """The same 1.2M-particle dam break (without the boxes) under the WCSPH pressure solver
    (Sec. 3.4.1), the algorithm of the paper's only timing table (Table 1, whose particle
    count is not stated), at its acoustic step: milliseconds per step."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    d = scenes.dam_break_rigid(n_boxes=0)
    d.update(scenes.wcsph_parameters(98 * 2 * d["radius"], d["radius"]))
    nf = len(d["fluid_x"])
    stream = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with sph.Context(d, stream=stream) as g:
        g.sph_steps(5, 0.0)
        g.sph_synchronize(raise_on_error=False)
        a.record(stream)
        g.sph_steps(steps, 0.0)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        st = g.sph_get_stats()
    return {"fluid_particles": nf, "dt": float(d["dt_max"]), "ms_per_step": ms,
            "particle_steps_per_s": nf / (ms / 1000.0), "status_flags": int(st["flags"]),
            "paper_table1_context": "Taichi CUDA WCSPH on A100: 0.0401 s/step, particle count not stated"}


def solver_comparison(seconds=0.04):
    """The 8,000-particle dam break under the three pressure solvers the paper implements,
    each at its own step (DFSPH and PCISPH 4e-4 s at the 0.1 % density tolerance, WCSPH its
    acoustic step), over the same simulated time: iterations per step and GPU milliseconds
    per simulated second."""
    import torch
    from paper_2403_11156_gb300 import scenes, sph
    out = {}
    for name, d in (("dfsph", scenes.dam_break_small()), ("pcisph", scenes.dam_break_pcisph()),
                    ("wcsph", scenes.dam_break_wcsph())):
        dt = float(d["dt_max"])
        steps = max(1, int(round(seconds / dt)))
        stream = torch.cuda.Stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with sph.Context(d, stream=stream) as g:
            a.record(stream)
            g.sph_steps(steps, dt)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            st = g.sph_get_stats()
        out[name] = {"dt": dt, "steps": steps, "ms_per_step": ms / steps,
                     "ms_per_simulated_second": ms / (steps * dt),
                     "density_iters_per_step": st["total_dens_iters"] / steps,
                     "divergence_iters_per_step": st["total_div_iters"] / steps,
                     "final_density_error": st["dens_err"]}
    return out


def post_processing(g, desc, stream):
    """Phase three (Sec. 4.3) on the benchmark scene's final state: the volume-fraction
    field on a grid of spacing r over the tank, its 0.5 iso-surface, and a height map at
    r/2 pixels; milliseconds of each (CUDA events)."""
    import torch
    from paper_2403_11156_gb300 import sph
    r = desc["radius"]
    lo, hi = desc["domain_min"], desc["domain_max"]
    dims = [int((hi[a] - lo[a]) / r) + 1 for a in range(3)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        field = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
        w, h = int((hi[0] - lo[0]) / (r / 2)), int((hi[1] - lo[1]) / (r / 2))
        img = torch.empty((h, w), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        ev[0].record(stream)
        g.sph_surface_field(lo, r, dims, out=field)
        ev[1].record(stream)
        tris = sph.sph_surface_mesh(field, lo, r, 0.5, stream=stream)
        ev[2].record(stream)
        g.sph_render_heightmap(lo[:2], (lo[0] + w * r / 2, lo[1] + h * r / 2), w, h, r, out=img)
        ev[3].record(stream)
        torch.cuda.synchronize()
    return {"grid": dims, "field_ms": ev[0].elapsed_time(ev[1]), "mesh_ms": ev[1].elapsed_time(ev[2]),
            "triangles": int(len(tris)), "height_map": [w, h], "height_map_ms": ev[2].elapsed_time(ev[3])}


def reference_sample():
    from paper_2403_11156_gb300 import scenes
    # the same construction scaled to 80 x 64 x 64 = 327,680 particles (tank 0.64x), so that
    # a full --steps K --warmup W run of the oracle ends within a few minutes
    return scenes.dam_break_rigid(n=(80, 64, 64), tank=(1.28, 0.64, 0.64))


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    # the host's cores, however the process was launched (torchrun sets OMP_NUM_THREADS=1)
    oracle.set_num_threads(len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    d = reference_sample()
    o = oracle.Scene(d)
    for _ in range(args.warmup):
        o.step(0.0)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.step(0.0)
    el = time.perf_counter() - t
    n = len(d["fluid_x"])
    v = n * args.steps / el
    sample = ("oracle (FP64 C, OpenMP) stepping a %d-particle scaled copy of the workload "
              "(same r, tolerances, CFL and rigid boxes; tank 1.28x0.64x0.64 m)" % n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--timing-steps", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default 27-cell stencil and gather batch instead of autotuning")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the secondary workloads (64-scene batch, WCSPH, solver comparison, viscous column, "
                         "weak vs strong coupling, post-processing)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-vs-plain warm-start comparison")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2403_11156_gb300 import build, scenes, sph
    from paper_2403_11156_gb300.sharding import reduce_timing

    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    desc = scenes.dam_break_rigid()
    n_fluid = len(desc["fluid_x"])
    stream = torch.cuda.Stream()
    g = sph.Context(desc, stream=stream, autotune=not args.no_autotune)
    tuning = g.sph_get_tuning()
    g.sph_steps(args.warmup, 0.0)
    g.sph_synchronize()

    # ---- timed region: K graph-launched steps (inputs resident; the scene's working set
    # of ~0.5 GB per step is larger than L2, so no flush is needed between steps)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = g.sph_launch_count()
    it0 = g.sph_get_stats()
    clocks = ClockSampler("/tmp/bench_clocks_%d.csv" % rank, local)
    with clocks:
        barrier()
        torch.cuda.synchronize()
        start.record(stream)
        g.sph_steps(args.steps, 0.0)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = start.elapsed_time(stop)
    status = g.sph_synchronize(raise_on_error=False)
    it1 = g.sph_get_stats()
    launches = g.sph_launch_count() - l0
    ms, units = reduce_timing(ms, n_fluid * args.steps, world, device="cuda")
    value = units / (ms / 1000.0)

    # ---- end to end through the C ABI: the same K steps from the same initial state on a
    # second context (same, cached tuning).  Every step is enqueued with its host dt and
    # its result, all positions in original particle order, is read into page-locked host
    # memory by sph_read_state (on_device = 3: unpermuted on the library stream, copied on
    # the library's copy stream while the next step runs).  The host keeps one read in
    # flight: after enqueuing step k and its read it waits (sph_read_wait, keep = 1) until
    # step k - 1's positions are on the host, and it reuses a host buffer only after that.
    # The scene is resident on the device (uploaded once at create, outside the timed
    # region); per step the host supplies dt (4 B) and receives 12 B per particle.
    pinned = [torch.empty((n_fluid, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    e2e_steps = args.steps
    g2 = sph.Context(desc, stream=stream, autotune=not args.no_autotune)
    g2.sph_steps(args.warmup, 0.0)
    g2.sph_synchronize()
    barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(e2e_steps):
        g2.sph_step(0.0)
        g2.sph_read_state_host(0, x=pinned[k % 2], sync=False)
        g2.sph_read_wait(1)                         # step k - 1's positions are on the host
    g2.sph_read_wait(0)
    e2e_wall = time.perf_counter() - t
    x_e2e = pinned[(e2e_steps - 1) % 2].numpy().copy()
    g2.close()
    e2e_ms, e2e_units = reduce_timing(e2e_wall * 1000.0, n_fluid * e2e_steps, world, device="cuda")
    e2e = {"value": e2e_units / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": 4,
           "d2h_bytes_per_step": 12 * n_fluid,
           "path": "sph_step + sph_read_state(on_device = 3) into page-locked host memory, sph_read_wait(keep = 1)",
           "last_positions_finite": bool(np.all(np.isfinite(x_e2e)))}

    # ---- kernel breakdown: eager steps with CUDA events around every launch (graph kernel
    # nodes cannot be bracketed by events).  Per-launch times come from these steps; the
    # time per step of each kernel weights them by its launches per step in the timed
    # region (solver passes by that region's mean iteration counts), which picks the
    # dominant kernel of the timed region's regime.
    g.sph_set_mode(graph=False, timing=True)
    g.sph_kernel_times(reset=True)
    it_t0 = g.sph_get_stats()
    g.sph_steps(args.timing_steps, 0.0)
    g.sph_synchronize(raise_on_error=False)
    it_t1 = g.sph_get_stats()
    kt = g.sph_kernel_times(reset=True)
    g.sph_set_mode(graph=True, timing=False)
    dens_per_step = (it1["total_dens_iters"] - it0["total_dens_iters"]) / args.steps
    div_per_step = (it1["total_div_iters"] - it0["total_div_iters"]) / args.steps
    per_step_launch = {}
    for k_name, (n_launch, _) in kt.items():
        if k_name in PER_DENSITY_ITERATION:
            per_step_launch[k_name] = dens_per_step
        elif k_name in PER_DIVERGENCE_ITERATION:
            per_step_launch[k_name] = div_per_step
        else:
            per_step_launch[k_name] = n_launch / args.timing_steps
    per_step_ms = {k_name: v[1] / v[0] * per_step_launch[k_name] for k_name, v in kt.items() if v[0]}
    total_ms = sum(per_step_ms.values())
    n_b = len(desc["boundary_x"])
    hbm, sm_max, peak_src = load_peaks()
    sm_mhz = clocks.summary().get("sm_mhz") or sm_max
    cfg_key = (tuning.get("lanes"), tuning.get("gather_batch"),
               27 if float(tuning.get("cell_factor", 0.0)) > 0.75 else 125)
    nn_mean = float(g.sph_read_field(sph.FIELD_NN_FLUID).mean())

    def roofline(name):
        n_launch, k_ms = kt[name]
        per_launch_s = k_ms / n_launch / 1000.0
        algo = ALGO_BYTES.get(name, 48) * n_fluid + BOUNDARY_BYTES * n_b
        achieved_gbs = algo / per_launch_s / 1e9
        r = {"kernel": name, "bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
             "frac": achieved_gbs / hbm, "traffic": TRAFFIC.get((name,) + cfg_key),
             "peak_source": ("%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src if peak_src == "measured"
                             else "fallback 6.8 TB/s"),
             "algorithmic_bytes_per_launch": algo, "avg_launch_us": per_launch_s * 1e6,
             "launches_per_step": per_step_launch[name],
             "share_of_step": per_step_ms[name] / total_ms if total_ms else None}
        if r["traffic"]:
            # the DRAM rate the launch sustains: ncu's bytes per launch over the live time
            r["traffic_gbs"] = r["traffic"] / per_launch_s / 1e9
            r["traffic_frac"] = r["traffic_gbs"] / hbm
        wf = L1_WAVEFRONTS.get((name,) + cfg_key)
        if wf:
            r["l1"] = {"wavefronts_per_launch": wf, "peak_wavefronts_per_s": 152 * sm_mhz * 1e6,
                       "frac": wf / per_launch_s / (152 * sm_mhz * 1e6)}
        if name in FLOPS_PER_PAIR:
            # ALU view: counted FP32 flops (pairs at the step's mean neighbour count, plus
            # the density sweep's candidate tests) over the FP32 peak at the sampled clock
            flops = (FLOPS_PER_PAIR[name] * nn_mean + FLOPS_PER_PARTICLE.get(name, 0)) * n_fluid
            r["alu"] = {"achieved_tflops": flops / per_launch_s / 1e12,
                        "peak_tflops": fp32_peak_tflops(sm_mhz), "pairs_per_particle": nn_mean}
            r["alu"]["frac"] = r["alu"]["achieved_tflops"] / r["alu"]["peak_tflops"]
        return r

    top_name = max(per_step_ms.items(), key=lambda t: t[1])[0]
    roof = roofline(top_name)
    rooflines = {k_name: roofline(k_name) for k_name in ROOFLINE_KERNELS if k_name in kt}
    breakdown = {k_name: {"launches_timing_pass": kt[k_name][0], "launches_per_step": round(per_step_launch[k_name], 3),
                          "us_per_launch": round(1000.0 * kt[k_name][1] / kt[k_name][0], 2),
                          "ms_per_step": round(v, 4), "share": round(v / total_ms, 4)}
                 for k_name, v in sorted(per_step_ms.items(), key=lambda t: -t[1])}

    d_it = it1["total_dens_iters"] - it0["total_dens_iters"]
    v_it = it1["total_div_iters"] - it0["total_div_iters"]
    post = None
    if rank == 0 and not args.no_batched:
        post = post_processing(g, desc, stream)
    learned = None
    learned_line = None
    if rank == 0 and not args.no_learned:
        learned, params = learned_vs_plain()
        # the metric's other half: the same workload and timed region with the learned start
        learned_line = learned_headline(desc, params, args.steps, args.warmup, not args.no_autotune, stream)
        plain_iters = (d_it + v_it) / args.steps
        learned_iters = learned_line["mean_density_iters"] + learned_line["mean_divergence_iters"]
        learned_line["over_plain"] = {
            "value_ratio": learned_line["value"] / value,
            "density_iteration_ratio": (d_it / args.steps) / max(learned_line["mean_density_iters"], 1e-9),
            "solver_iteration_ratio": plain_iters / max(learned_iters, 1e-9)}
        if not args.no_batched:
            learned["batched_64_scenes"] = batched_learned(params)
    batched = None
    if not args.no_batched:
        batched = batched_throughput(rank=rank, world=world, barrier=barrier)
    wcsph = None
    solvers = None
    column = None
    coupling = None
    if rank == 0 and not args.no_batched:
        wcsph = wcsph_step_time()
        solvers = solver_comparison()
        column = viscous_column_time()
        coupling = coupling_comparison()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g.close()
        cpu = cpu_baseline(desc)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fluid_particles": n_fluid, "boundary_particles": n_b,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "warm_start": "previous-step kappa (plain DFSPH)",
                   "l2": "working set per step > L2 (129 MB); no flush",
                   "mean_density_iters": d_it / args.steps, "mean_divergence_iters": v_it / args.steps,
                   "final_density_error": it1["dens_err"], "dt": it1["dt"], "status": sph.STATUS_NAMES[status],
                   "autotune": tuning},
        "clocks": clocks.summary(), "gpu_launches": int(launches), "e2e": e2e, "roofline": roof,
        "rooflines": rooflines, "kernels": breakdown, "cpu_baseline": cpu, "learned": learned_line,
        "learned_vs_plain": learned,
        "batched_64_scenes": batched,
        "wcsph_1.2M": wcsph,
        "viscous_column_250k": column,
        "coupling_1.2M": coupling,
        "solvers_8k": solvers,
        "post_processing_1.2M": post,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
