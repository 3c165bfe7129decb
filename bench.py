#!/usr/bin/env python3
"""Throughput of the SPH strength step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32k|fp64] [--scale S]

Workload: the 2,000,000-particle basalt impact (1.8M target + 0.2M impactor
at 5 km/s and 45 degrees, Tillotson basalt with strength, radial g field),
seeded and synthetic. One step is the whole hot path: drift, cell list
(Morton keys, radix sort, permutation), density / smoothing-length solve,
EOS + yield + radial return, the full-stress pair loop with its finalize,
and the kicks with rescaling and FP64 reductions.

Metric: particle-steps/s = particles x steps / device time of the K timed
steps (whole job over all ranks; with N > 1 every rank runs its own
replica of the impact, no data-path collective). The state (~450 MB) is far
larger than L2, so no flush is needed between steps.

The JSON line also carries: e2e (the same metric through sph_step_host with
pinned host buffers, copies inside the timed region), roofline (the
dominant kernel's algorithmic FLOP/s over the FP32 or FP64 ALU peak from
unit counts and clock, beside the measured FMA peak), cpu_baseline (the
FP64 C oracle stepping the whole impact on every host core, plus one thread
on a bounded sub-volume) and the SM clocks sampled during the timed region.
--impl reference times the oracle itself, whole FP64 steps of the same
impact on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FLOPs per in-range pair, counted term by term from the
# formulas as the oracle writes them out (Eq. 1 and 3 for the density, one
# evaluation; Eq. 4-8 and 18-21 with du/dt|_H for the forces), an add, sub,
# mul, div or sqrt counting 1; factors that belong to one particle
# (P/(Omega rho^2), S/(Omega rho^2), 1/(Omega rho), kernel normalisation)
# are formed once per particle and not counted per pair. The kernels
# contract the force terms and execute fewer operations; candidate
# rejection, compensation and index work are not counted either way.
FLOPS_DENSITY_PAIR = 27
FLOPS_FORCE_PAIR = 209
# B300 unit counts: 128 FP32 lanes per SM, 2 FLOP per FMA, at the 2032 MHz
# maximum clock (the SM count is read from the device); FP64 at the nominal
# 1.25 TFLOP/s.
FP32_LANES, MAX_MHZ = 128, 2032.0
FP64_NOMINAL_TFLOPS = 1.25

# DRAM bytes (read + write) per particle per launch of the FP32 pair kernels,
# from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` on the
# 600k-particle impact (bench.py --scale 0.3 --spans 1,2; profiles/ has the
# command) and scaled by particles. Keyed by a hash of the kernel's sources: once the
# kernel changes the figure no longer applies and traffic is reported null.
KERNEL_SOURCES = {"k_forces": ("sph_forces.cu", "sph_pair.cuh", "sph_internal.cuh",
                                "sph_kick.cuh"),
                  "k_density": ("sph_density.cu", "sph_pair.cuh", "sph_internal.cuh")}
TRAFFIC_PER_PARTICLE = {"k_forces": (182.1, "d40545feba64"),
                        "k_density": (64.2, "59345c92f537")}


def source_hash(kernel: str) -> str:
    import hashlib
    m = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2603_19764_b300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:12]


def traffic_per_launch(kernel: str, n: int, precision: int):
    if precision != 1 or kernel not in TRAFFIC_PER_PARTICLE:
        return None
    per, h = TRAFFIC_PER_PARTICLE[kernel]
    return per * n if source_hash(kernel) == h else None


def fp32_peak_tflops(mhz: float, n_sm: int) -> float:
    return n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(mhz: float) -> float:
    return FP64_NOMINAL_TFLOPS * mhz / MAX_MHZ


# --------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the timed region starts once the sampler has written its first row
        t0 = time.time()
        while time.time() - t0 < 3.0 and os.path.getsize(self.f.name) == 0:
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(mhz)}


# ------------------------------------------------------------ ranks
def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of every rank's value (the job takes as long as its
    slowest rank); the identity on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the
    slowest rank's time (replicas: each rank steps its own copy)."""
    return world * units_per_rank * steps / seconds


# ------------------------------------------------------------ workloads
def make_workload(scale: float, precision: int):
    from paper_2603_19764_b300 import workloads as wl
    return wl.impact(int(1_800_000 * scale), int(200_000 * scale), precision=precision)


def contact_subvolume(w, n_sub: int) -> dict:
    """The n_sub particles nearest the initial contact point of the impact."""
    a = w.arrays
    x = np.stack([a["x"], a["y"], a["z"]], 1)
    nt = w.systems[0][1] if w.systems else w.n
    imp = a["id"] >= int(round(0.9 * nt))
    c_t, c_i = x[~imp].mean(0), x[imp].mean(0)
    r_t = np.sqrt(((x[~imp] - c_t) ** 2).sum(1)).max()
    r_i = np.sqrt(((x[imp] - c_i) ** 2).sum(1)).max()
    contact = c_t + (c_i - c_t) * r_t / (r_t + r_i)
    d = np.sqrt(((x - contact) ** 2).sum(1))
    sel = np.argsort(d, kind="stable")[:n_sub]
    sel.sort()
    sub = {k: v[sel].copy() for k, v in a.items()}
    sub["id"] = np.arange(sel.size, dtype=np.int64)
    return sub


def sampled_error(sim, w, p, precision: int, nsample: int = 1000, seed: int = 7) -> dict:
    """Oracle comparison on nsample particles of the current GPU state."""
    import oracle
    sim.forces_strength()
    g = sim.to_numpy()
    idx = np.sort(np.random.default_rng(seed).choice(w.n, nsample, replace=False))
    rho, _, cnt = oracle.density_given_h(p, g, idx=idx)
    st, S = oracle.eos_yield(p, w.materials, g)
    out, _ = oracle.forces(p, w.materials, st, S=S, idx=idx)
    derr = 0.0
    for f in ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz"):
        scale = float(np.max(np.abs(g[f]))) or 1.0
        derr = max(derr, float(np.max(np.abs(g[f][idx] - out[f][idx]))) / scale)
    return {"sample": nsample, "rho_rel_max": float(np.max(np.abs(g["rho"][idx] / rho - 1))),
            "counts_exact": bool(np.array_equal(cnt, g["nngb"][idx])),
            "deriv_maxnorm_rel": derr,
            "tolerance": {"rho_rel": 1e-5 if precision else 1e-6,
                          "deriv_maxnorm_rel": 1e-4 if precision else 1e-9}}


def oracle_rate(w, arrays: dict, budget_s: float, max_steps: int,
                fixed_steps: int | None = None, warmup: int = 0) -> dict:
    """The FP64 C oracle, as it stands, stepping `arrays` (a state of w's
    system) with its adaptive dt; derivatives are formed and `warmup` steps
    taken before the clock starts."""
    import oracle
    p = dict(w.params, h_tol=1e-10)
    st, info = oracle.derivatives(p, w.materials, arrays)
    for _ in range(warmup):
        st, infos = oracle.step(p, w.materials, st, info["dt_next"])
        info = infos[-1]
    steps, t0 = 0, time.perf_counter()
    while True:
        st, infos = oracle.step(p, w.materials, st, info["dt_next"])
        info = infos[-1]
        steps += 1
        el = time.perf_counter() - t0
        if fixed_steps is not None:
            if steps >= fixed_steps:
                break
        elif el >= budget_s or steps >= max_steps:
            break
    n = arrays["x"].shape[0]
    return {"value": n * steps / el, "steps": steps, "particles": n, "seconds": el}


def cpu_baseline(w, budget_s: float = 15.0, max_steps: int = 3, n_single: int = 20_000,
                 single_budget_s: float = 5.0) -> dict:
    """The oracle on the machine's host cores: full steps of the whole workload
    on every core, and one thread on the particles nearest the contact
    point (a bounded sample: one thread would take minutes per full step)."""
    import oracle
    nth = oracle.threads()
    full = oracle_rate(w, w.arrays, budget_s, max_steps)
    oracle.set_threads(1)
    try:
        one = oracle_rate(w, contact_subvolume(w, min(n_single, w.n)), single_budget_s, 20)
    finally:
        oracle.set_threads(nth)
    return {"value": full["value"], "unit": "particle-steps/s", "cores": nth, "kind": "oracle",
            "seconds": full["seconds"],
            "sample": "%d FP64 oracle steps (OpenMP, %d threads) of the whole %d-particle impact"
                      % (full["steps"], nth, full["particles"]),
            "single_thread": {"value": one["value"], "unit": "particle-steps/s", "cores": 1,
                              "sample": "%d FP64 oracle steps (one thread) of the %d particles "
                                        "of the impact nearest the contact point"
                                        % (one["steps"], one["particles"])}}


# --------------------------------------------------------------- arms
def run_reference(args, rank: int, world: int):
    """The oracle as it stands, timed on the host cores: W untimed and then
    K timed FP64 steps of the whole impact (every particle, adaptive dt), so
    ms_per_step is a measured step of the same workload as the GPU arm."""
    if rank != 0:
        return
    w = make_workload(args.scale, 1)
    import oracle
    r = oracle_rate(w, w.arrays, 0.0, 0, fixed_steps=max(1, args.steps), warmup=args.warmup)
    cb = {"value": r["value"], "unit": "particle-steps/s", "cores": oracle.threads(),
          "kind": "oracle",
          "sample": "%d FP64 oracle steps (OpenMP, %d threads) of the whole %d-particle impact, "
                    "after %d untimed" % (r["steps"], oracle.threads(), r["particles"],
                                          args.warmup)}
    line = {"metric": "SPH+strength particle-steps/s (2M part.), chosen vs plain form at stated error",
            "value": cb["value"], "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": r["steps"], "warmup": args.warmup,
            "ms_per_step": 1e3 * r["seconds"] / r["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "basalt impact 1.8M+0.2M particles, 5 km/s, 45 deg",
                       "particles": r["particles"], "precision": "fp64 oracle",
                       "dt": "adaptive, Eq. 38-39 (dt_next of the previous step)"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_plain(w, dev, snapshot: dict, dts: list, warmup: int = 3, graph: bool = True) -> dict:
    """The plain FP64 form doing the chosen form's timed work: it starts
    from the same state (`snapshot`, the chosen form's caller arrays at the
    start of its timed steps, derivatives included) and takes the same step
    sizes `dts`, replayed from a CUDA graph like the chosen form. Warm-up
    steps (graph capture) run from the snapshot too; the state is then put
    back in place, so the graph's pointers stay valid."""
    import torch
    from paper_2603_19764_b300 import sph
    p = dict(w.params, precision=0, h_tol=1e-10)
    sim = sph.Simulation(snapshot, w.materials, p, device=str(dev))
    if graph:
        sim.set_graph(True)
    for k in range(warmup):
        sim.step(dts[k % len(dts)])
    torch.cuda.synchronize(dev)
    for f, t in sim.t.items():
        t.copy_(torch.as_tensor(snapshot[f]).to(dev))
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for dt in dts:
        sim.step(dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    sim.close()
    return {"value": w.n * len(dts) / (ms / 1e3), "unit": "particle-steps/s",
            "ms_per_step": ms / len(dts), "steps": len(dts), "precision": "fp64",
            "graph": graph, "work": "same start state and step sizes as the timed chosen steps"}


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist
    from paper_2603_19764_b300 import build, sph

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    precision = 1 if args.precision == "fp32k" else 0
    w = make_workload(args.scale, precision)
    p = dict(w.params, precision=precision, h_tol=1e-6 if precision else 1e-10)
    sim = sph.Simulation(w.arrays, w.materials, p, device=str(dev))
    sim.prime()
    # the chosen form: group spans tuned on the first steps, then the step
    # replayed from a CUDA graph
    if args.spans:
        sim.set_spans(*[int(v) for v in args.spans.split(",")])
    elif args.tune > 0:
        sim.autotune(args.tune)
        while sim.tune_info()["steps_left"] > 0:   # spans, then staging depths
            sim.step(0.0)
    if not args.no_graph:
        sim.set_graph(True)
    for _ in range(args.warmup):
        sim.step(0.0)
    # start state of the timed steps, for the plain form's identical work
    snapshot = sim.to_numpy() if (rank == 0 and precision == 1 and not args.no_plain) else None
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [sim.step(0.0) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, world, dev)
    # phase times (for the roofline) from direct launches of the same
    # form: steps replayed from a graph carry no phase events
    sim.set_graph(False)
    sim.set_timing(True)
    for _ in range(max(3, min(args.steps, 10))):
        sim.step(0.0)
    phases = sim.phase_times()
    sim.set_timing(False)
    tune_rep = sim.tune_info()
    ms_step = ms / args.steps
    value = job_rate(w.n, world, args.steps, ms / 1e3)

    # roofline of the dominant kernel (by CUDA-event phase time)
    nsteps = max(phases["steps"], 1)
    pairs_f = statistics.mean(i["pairs_force"] for i in infos)
    pairs_d = statistics.mean(i["pairs_density"] for i in infos)
    t_force = phases["forces"] / nsteps
    t_dens = phases["density"] / nsteps
    if t_force >= t_dens:
        kname, flops, tk = "k_forces", FLOPS_FORCE_PAIR * pairs_f, t_force
    else:
        kname, flops, tk = "k_density", FLOPS_DENSITY_PAIR * pairs_d, t_dens
    achieved = flops / (tk / 1e3) / 1e12
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(MAX_MHZ, n_sm) if precision else fp64_peak_tflops(MAX_MHZ)
    fma = {"fp32": sph.measure_fma_peak(1, 20), "fp64": sph.measure_fma_peak(0, 5)}
    fma_own = fma["fp32" if precision else "fp64"]
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_per_launch(kname, w.n, precision), "traffic_unit": "bytes",
                "peak_basis": ("%s lanes x 2 x %.0f MHz (unit counts)" %
                               ("%dx128 FP32" % n_sm if precision else "FP64 nominal 1.25 TFLOP/s",
                                MAX_MHZ)),
                "kernel_ms": tk, "pairs_per_step": pairs_f if kname == "k_forces" else pairs_d,
                "peak_fma_measured": fma_own["tflops"],
                "frac_of_fma_measured": achieved / fma_own["tflops"]}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        host = sph.HostState(sim.to_numpy())
        if args.copy_chunks:
            sim.set_copy_chunks(args.copy_chunks)
        sim.step_host(host, 0.0)
        torch.cuda.synchronize(dev)
        ne = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(ne):
            r = sim.step_host(host, 0.0)
        te = time.perf_counter() - t0
        te = max_over_ranks(te, world, dev)
        e2e = {"value": job_rate(w.n, world, ne, te), "unit": "particle-steps/s",
               "h2d_bytes_per_step": r["bytes_in"], "d2h_bytes_per_step": r["bytes_out"],
               "steps": ne, "copy_chunks": args.copy_chunks or 8}
    # error of this form against the FP64 oracle on a seeded sample, on the
    # state the timed steps produced (derivatives recomputed as it stands)
    err = None
    if rank == 0 and not args.no_error:
        err = sampled_error(sim, w, p, precision)
    sim.close()

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w)
        cb = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "single_thread")}

    # the plain FP64 form on the same impact, a few steps, for the chosen-vs-plain ratio
    plain = None
    if rank == 0 and args.precision == "fp32k" and not args.no_plain:
        plain = time_plain(w, dev, snapshot, [i["dt"] for i in infos][:args.plain_steps or None],
                           warmup=args.warmup, graph=not args.no_graph)
        snapshot = None

    if rank == 0:
        line = {"metric": "SPH+strength particle-steps/s (2M part.), chosen vs plain form at stated error",
                "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if precision else "f64", "data": "synthetic",
                "config": {"workload": "basalt impact 1.8M+0.2M particles, 5 km/s, 45 deg",
                           "particles": w.n, "precision": args.precision,
                           "dt": "adaptive, Eq. 38-39 (dt_next of the previous step)",
                           "dt_mean": statistics.mean(i["dt"] for i in infos),
                           "l2": "state 450 MB > L2, no flush",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "error": err,
                "tuner": tune_rep, "graph": not args.no_graph,
                "gpu_launches": sum(i["kernel_launches"] for i in infos),
                "plain_fp64": plain,
                "fma_peak_measured": {k: {q: v[q] for q in ("tflops", "ms", "sm_mhz")}
                                      for k, v in fma.items()},
                "clocks": clocks,
                "phases_ms_per_step": {k: (v / nsteps if k != "steps" else v)
                                       for k, v in phases.items()},
                "sweeps": max(i["sweeps"] for i in infos),
                "pairs_per_step": {"density": pairs_d, "force": pairs_f},
                "candidates_per_step": {
                    "density": statistics.mean(i["cand_density"] for i in infos),
                    "force": statistics.mean(i["cand_force"] for i in infos)},
                "groups_per_bucket": {
                    "density": statistics.mean(i["groups_density"] for i in infos) / ((w.n + 31) // 32),
                    "force": statistics.mean(i["groups_force"] for i in infos) / ((w.n + 31) // 32)},
                "energy": {"e_kin": infos[-1]["e_kin"], "e_int": infos[-1]["e_int"],
                           "e_pot": infos[-1]["e_pot"]}}
        print(json.dumps(line), flush=True)


def run_batch(args, rank: int, world: int, local_rank: int):
    """The batched form on the 64-impact sweep, against the same 64 impacts
    stepped one after another by their own contexts (sequential launches).

    Every system steps with its own adaptive dt (its dt_next). Arms: batched FP32 form under
    a CUDA graph with tuned group spans (the chosen form), batched FP64,
    sequential FP32 form, sequential plain FP64. Each arm's value is
    particles x steps / device time of its timed steps.
    """
    import torch
    import torch.distributed as dist
    from paper_2603_19764_b300 import build, sph
    from paper_2603_19764_b300 import workloads as wl

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = wl.impact_batch(64, precision=1, scale=args.batch_scale)
    zeros = np.zeros(len(w.systems))   # every system at its own dt_next
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        out = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), out

    def batched(precision, steps, tune, graph, sampler=None):
        p = dict(w.params, precision=precision, h_tol=1e-6 if precision else 1e-10)
        sim = sph.Simulation(w.arrays, w.materials, p, device=str(dev), systems=w.systems)
        sim.prime()
        sim.set_graph(graph)
        if tune:
            sim.autotune(tune)
            while sim.tune_info()["steps_left"] > 0:   # spans, then staging depths
                sim.step_batch(zeros)
        for _ in range(args.warmup):
            sim.step_batch(zeros)
        if world > 1:
            dist.barrier()
        if sampler:
            sampler.start()
        ms, infos = timed(lambda: sim.step_batch(zeros), steps)
        clocks = sampler.stop() if sampler else None
        rep = sim.tune_info()
        err = sampled_error(sim, w, p, precision) if (rank == 0 and not args.no_error) else None
        sim.close()
        return ms, infos, rep, err, clocks

    def sequential(precision, steps):
        p = dict(w.params, precision=precision, h_tol=1e-6 if precision else 1e-10)
        sims = []
        for k in range(len(w.systems)):
            ws = w.system(k)
            sims.append(sph.Simulation(ws.arrays, ws.materials, p, device=str(dev)))
        for sim in sims:
            sim.prime()
            sim.step(0.0)

        def one():
            return [sim.step(0.0) for sim in sims]
        ms, infos = timed(one, steps)
        for sim in sims:
            sim.close()
        return ms, sum(i["kernel_launches"] for step in infos for i in step)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ms_c, infos, rep, err, clocks = batched(1, args.steps, 2, True, sampler)
    ms_c = max_over_ranks(ms_c, world, dev)
    value = job_rate(w.n, world, args.steps, ms_c / 1e3)
    ks = max(1, min(args.steps, args.plain_steps or 3))
    arms = {}
    if rank == 0:
        ms_b64, _, rep64, err64, _ = batched(0, ks, 2, True)
        arms["batched_fp64"] = {"value": w.n * ks / (ms_b64 / 1e3), "ms_per_step": ms_b64 / ks,
                                "steps": ks, "spans": [rep64["span_density"], rep64["span_forces"]],
                                "error": err64}
        for name, prec in (("sequential_fp32k", 1), ("sequential_fp64_plain", 0)):
            ms_s, nl = sequential(prec, ks)
            arms[name] = {"value": w.n * ks / (ms_s / 1e3), "ms_per_step": ms_s / ks,
                          "steps": ks, "gpu_launches": nl}
        sizes = [c for _, c in w.systems]
        line = {"metric": "SPH+strength particle-steps/s, 64-impact batch, batched vs sequential",
                "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_c / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "64 basalt impacts, targets log-uniform 2k-200k, "
                                       "gamma 0.01-0.5, 1-20 km/s, 0-60 deg, one seed",
                           "particles": w.n, "systems": len(sizes), "smallest": min(sizes),
                           "largest": max(sizes), "precision": "fp32k", "graph": True,
                           "dt": "adaptive per system, Eq. 38-39",
                           "l2": "state > L2, no flush"},
                "tuner": rep, "error": err, "clocks": clocks,
                "gpu_launches": sum(i["kernel_launches"] for i in infos),
                "arms": arms,
                "speedup_vs_sequential_plain": value / arms["sequential_fp64_plain"]["value"],
                "speedup_vs_sequential_same_form": value / arms["sequential_fp32k"]["value"]}
        print(json.dumps(line), flush=True)


def run_learned(args, rank: int, world: int, local_rank: int):
    """The learned smoothing-length guess on the 8M-particle impact.

    Histories: `history_steps` steps of the 1M basalt sphere (plain FP64) and
    of the 2M impact (FP32 form) with recording on, every `record_every`-th
    step kept. The network is trained on the GPU by the library's kernels.
    Then the 8M impact (FP32 form) runs with the previous-H guess, the
    continuity guess and the network guess from the same primed state;
    value = particle-steps/s of the network arm.
    """
    import torch
    import torch.distributed as dist
    from paper_2603_19764_b300 import build, sph
    from paper_2603_19764_b300 import workloads as wl

    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sc = args.learned_scale

    # ---- histories
    t_hist = time.perf_counter()
    Xs, ys, sources = [], [], []
    for name, w, prec in (("basalt sphere 1M, FP64", wl.config(2, scale=sc), 0),
                          ("impact 2M, FP32 form", wl.config(3, scale=sc), 1)):
        p = dict(w.params, precision=prec, h_tol=1e-6 if prec else 1e-10)
        sim = sph.Simulation(w.arrays, w.materials, p, device=str(dev))
        sim.set_learned_h(sph.GUESS_PREVIOUS, record=True)
        sim.prime()
        kept = 0
        for k in range(args.history_steps):
            sim.step(0.0)
            if (k + 1) % args.record_every == 0:
                X, y = sim.learn_samples()
                ok = torch.isfinite(y)
                Xs.append(X[ok].clone())
                ys.append(y[ok].clone())
                kept += 1
        sim.close()
        sources.append({"workload": name, "particles": w.n, "steps": args.history_steps,
                        "kept_steps": kept})
        del w
    X = torch.cat(Xs)
    y = torch.cat(ys)
    del Xs, ys
    torch.cuda.synchronize(dev)
    t_hist = time.perf_counter() - t_hist

    # ---- training on the GPU
    t_train = time.perf_counter()
    net = sph.Mlp(device=str(dev))
    net.set(wl.mlp_init(), np.ones(sph.MLP_NNORM))
    net.fit_norm(X, y)
    L0, _ = net.loss_grad(X, y)
    losses = []
    for ep in range(args.epochs):
        perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(ep))
        losses.append(net.train_epoch(X, y, perm, batch=16384, lr=2e-3))
    L1, _ = net.loss_grad(X, y)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t_train
    nsamples = int(X.shape[0])
    del X, y

    # ---- the 8M impact with each guess
    w = wl.config(5, scale=sc)
    p = dict(w.params, precision=1, h_tol=1e-6)
    arms, states = {}, {}
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    clocks = None
    for name, guess in (("previous", sph.GUESS_PREVIOUS), ("continuity", sph.GUESS_CONTINUITY),
                        ("network", sph.GUESS_NETWORK)):
        sim = sph.Simulation(w.arrays, w.materials, p, device=str(dev))
        sim.set_learned_h(guess, net=net if guess == sph.GUESS_NETWORK else None)
        sim.prime()
        first = sim.step(0.0)
        states[name] = _by_id(sim.to_numpy(), ("id", "h", "nngb", "x", "y", "z"))
        for _ in range(args.warmup):
            sim.step(0.0)
        sim.set_timing(True)
        if world > 1:
            dist.barrier()
        if sampler and name == "network":
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        infos = [sim.step(0.0) for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        if sampler and name == "network":
            clocks = sampler.stop()
        ph = sim.phase_times()
        err = None
        if name == "network" and rank == 0 and not args.no_error:
            err = sampled_error(sim, w, p, 1)
        sim.close()
        nst = max(ph["steps"], 1)
        arms[name] = {"value": w.n * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                      "sweeps_per_particle": statistics.mean(i["sweeps_total"] for i in infos) / w.n,
                      "first_step_sweeps_per_particle": first["sweeps_total"] / w.n,
                      "max_sweeps": max(i["sweeps"] for i in infos),
                      "density_ms_per_step": ph["density"] / nst,
                      "phases_ms_per_step": {k: v / nst for k, v in ph.items() if k != "steps"},
                      "gpu_launches": sum(i["kernel_launches"] for i in infos)}
        if err is not None:
            arms[name]["error"] = err
    # neighbour counts after the exact solve, one step from the same primed
    # state: previous-H guess against the network guess
    a, b = states["previous"], states["network"]
    mism = np.nonzero(a["nngb"] != b["nngb"])[0]
    rel_h = np.abs(b["h"] / a["h"] - 1.0)
    detail = []
    X3 = np.stack([a["x"], a["y"], a["z"]], 1)
    for i in mism[:20]:
        d = np.sqrt(((X3 - X3[i]) ** 2).sum(1))
        q = np.abs(d[np.abs(d / a["h"][i] - 1) < 1e-3] / a["h"][i] - 1)
        detail.append({"id": int(a["id"][i]), "counts": [int(a["nngb"][i]), int(b["nngb"][i])],
                       "h_rel_diff": float(rel_h[i]),
                       "closest_abs_r_over_H_minus_1": float(q.min()) if q.size else None})
    value = arms["network"]["value"]
    if rank == 0:
        line = {"metric": "SPH+strength particle-steps/s (8M impact), learned vs previous-H guess",
                "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": arms["network"]["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64, network bf16", "data": "synthetic",
                "config": {"workload": "basalt impact 7.2M+0.8M particles, 5 km/s, 45 deg",
                           "particles": w.n, "precision": "fp32k", "dt": "adaptive, Eq. 38-39",
                           "l2": "state > L2, no flush"},
                "training": {"sources": sources, "samples": nsamples, "epochs": args.epochs,
                             "batch": 16384, "lr": 2e-3, "loss_before": L0, "loss_after": L1,
                             "epoch_losses": losses, "history_seconds": t_hist,
                             "train_seconds": t_train},
                "arms": arms,
                "sweeps_saved_per_particle": (arms["previous"]["sweeps_per_particle"] -
                                              arms["network"]["sweeps_per_particle"]),
                "speedup_vs_previous": value / arms["previous"]["value"],
                "counts_after_one_step": {"mismatches": int(mism.size), "particles": w.n,
                                          "max_h_rel_diff": float(rel_h.max()),
                                          "detail": detail},
                "clocks": clocks,
                "gpu_launches": arms["network"]["gpu_launches"]}
        print(json.dumps(line), flush=True)
    net.close()


def oracle_error(g: dict, w, p, precision: int, idx=None) -> dict:
    """Derivatives of a GPU state g (rho, omega, H, counts as the GPU left
    them) against the FP64 oracle evaluated on that same state, on the
    particles idx (None = all)."""
    import oracle
    rho, _, cnt = oracle.density_given_h(p, g, idx=idx)
    st, S = oracle.eos_yield(p, w.materials, g)
    out, _ = oracle.forces(p, w.materials, st, S=S, idx=idx)
    sel = np.arange(g["x"].shape[0]) if idx is None else idx
    derr = {}
    for f in ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz"):
        scale = float(np.max(np.abs(g[f]))) or 1.0
        derr[f] = float(np.max(np.abs(g[f][sel] - out[f][sel]))) / scale
    return {"n": int(sel.size), "rho_rel_max": float(np.max(np.abs(g["rho"][sel] / rho - 1))),
            "count_mismatches": int(np.count_nonzero(cnt != g["nngb"][sel])),
            "deriv_maxnorm_rel": max(derr.values()), "deriv_by_field": derr,
            "tolerance": {"rho_rel": 1e-5 if precision else 1e-6,
                          "deriv_maxnorm_rel": 1e-4 if precision else 1e-9}}


def run_drift(args, rank: int, world: int, local_rank: int):
    """Error and conservation of the chosen form over `--drift-steps` steps of
    the impact, beside the plain FP64 form stepped with the same step sizes
    (the FP64 run's adaptive dt, Eq. 38-39, drives both).

    * one-step error: at every `--spot-every`-th step the FP32 form's state
      is copied into a fresh context whose derivatives are recomputed and
      compared with the oracle's on the same state (seeded sample of
      `--spot` particles); at the checkpoints (1, 10, last) on every
      particle. The stepping contexts are never touched by the checks.
    * trajectory: FP32 form against FP64 form, particle by particle.
    * conservation: total energy (kinetic + internal + potential of the
      fixed radial field) of both runs against the start. Linear momentum
      is reported too; the field is external, so it is not conserved."""
    if rank != 0:
        return
    import torch
    from paper_2603_19764_b300 import build, sph
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.scale, 1)
    pa = dict(w.params, precision=1, h_tol=1e-6)
    pb = dict(w.params, precision=0, h_tol=1e-10)
    A = sph.Simulation(w.arrays, w.materials, pa, device=str(dev))
    B = sph.Simulation(w.arrays, w.materials, pb, device=str(dev))
    ia, ib = A.prime(), B.prime()
    A.set_spans(*[int(v) for v in (args.spans or "1,2").split(",")])
    A.set_graph(True)
    m = w.arrays["m"]
    vscale = float(np.sum(m * np.sqrt(w.arrays["vx"] ** 2 + w.arrays["vy"] ** 2
                                      + w.arrays["vz"] ** 2)))

    def energy(i):
        return i["e_kin"] + i["e_int"] + i["e_pot"]

    e0a, e0b = energy(ia), energy(ib)
    ekin0 = ib["e_kin"]
    p0a, p0b = np.array(ia["p"]), np.array(ib["p"])
    keys = ("x", "y", "z", "vx", "vy", "vz", "rho", "u", "h")
    x0 = _by_id(A.to_numpy(), ("x", "y", "z"))
    nsteps = args.drift_steps
    checkpoints = sorted({1, min(10, nsteps), nsteps})
    rng = np.random.default_rng(11)
    spot, full, traj, cons = [], [], [], []
    t_start = time.perf_counter()
    for k in range(1, nsteps + 1):
        ib = B.step(0.0)
        ia = A.step(ib["dt"])
        cons.append({"step": k, "dt": ib["dt"],
                     "dE_fp32k": (energy(ia) - e0a) / ekin0, "dE_fp64": (energy(ib) - e0b) / ekin0,
                     "dp_fp32k": float(np.linalg.norm(np.array(ia["p"]) - p0a)) / vscale,
                     "dp_fp64": float(np.linalg.norm(np.array(ib["p"]) - p0b)) / vscale})
        is_cp = k in checkpoints
        if k % args.spot_every == 0 or is_cp:
            ga = A.to_numpy()
            C = sph.Simulation(ga, w.materials, pa, device=str(dev))
            C.neighbours()
            C.density()
            C.forces_strength()
            gc = C.to_numpy()
            C.close()
            idx = np.sort(rng.choice(w.n, min(args.spot, w.n), replace=False))
            e = oracle_error(gc, w, pa, 1, idx=idx)
            spot.append(dict(step=k, **{q: e[q] for q in ("n", "rho_rel_max", "count_mismatches",
                                                          "deriv_maxnorm_rel")}))
            if is_cp:
                full.append(dict(step=k, **oracle_error(gc, w, pa, 1)))
                a = _by_id(ga, keys)
                b = _by_id(B.to_numpy(), keys)
                disp = max(float(np.max(np.abs(b[q] - x0[q]))) for q in ("x", "y", "z"))
                dx = np.sqrt(sum((a[q] - b[q]) ** 2 for q in ("x", "y", "z")))
                vmax = float(np.max(np.sqrt(b["vx"] ** 2 + b["vy"] ** 2 + b["vz"] ** 2)))
                dv = np.sqrt(sum((a[q] - b[q]) ** 2 for q in ("vx", "vy", "vz")))
                drho = np.abs(a["rho"] / b["rho"] - 1)
                traj.append({"step": k, "max_disp": disp,
                             "dx_max_over_disp": float(dx.max()) / disp,
                             "dx_p99_over_disp": float(np.quantile(dx, 0.99)) / disp,
                             "dv_max_over_vmax": float(dv.max()) / vmax,
                             "dv_p99_over_vmax": float(np.quantile(dv, 0.99)) / vmax,
                             "drho_max": float(drho.max()),
                             "drho_p99": float(np.quantile(drho, 0.99)),
                             "dh_max": float(np.max(np.abs(a["h"] / b["h"] - 1)))})
    A.close()
    B.close()
    line = {"mode": "drift", "workload": "basalt impact 1.8M+0.2M particles, 5 km/s, 45 deg",
            "particles": w.n, "steps": nsteps, "form": "fp32k (spans %s, graph)" % (args.spans or "1,2"),
            "seconds": time.perf_counter() - t_start,
            "dt": "adaptive from the FP64 run, Eq. 38-39, the same for both",
            "spot_error": spot, "full_error": full, "trajectory_fp32k_vs_fp64": traj,
            "conservation": [c for c in cons if c["step"] in checkpoints or c["step"] % 10 == 0],
            "conservation_max": {q: max(abs(c[q]) for c in cons)
                                 for q in ("dE_fp32k", "dE_fp64", "dp_fp32k", "dp_fp64")},
            "units": {"dE": "(E - E0) / E_kin0", "dp": "|p - p0| / sum m|v0|"}}
    print(json.dumps(line), flush=True)


def run_rungs(args, rank: int, world: int, local_rank: int):
    """Hierarchical individual steps against one global step, on the impact
    (FP32 form, graphs): both advance the same physical time, the global
    run with dt = dt_next (Eq. 38-39, the smallest criterion), the rung run
    with big steps of 2^R dt_next, so the particles that need it still step
    dt_next and the rest take 2x to 2^R x longer steps."""
    if rank != 0:
        return
    import torch
    from paper_2603_19764_b300 import build, sph
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.scale, 1)
    R = args.max_rung
    arms = {}
    t_target = None
    # both arms start from one relaxed state: the seeded initial state sheds
    # its transient (radial return of the random stresses, the first shock)
    # in global steps first, so that the rung arm's warm-up does not land
    # every particle on the finest rung
    p0 = dict(w.params, precision=1, h_tol=1e-6)
    sim = sph.Simulation(w.arrays, w.materials, p0, device=str(dev))
    sim.prime()
    for _ in range(args.relax_steps):
        sim.step(0.0)
    start = sim.to_numpy()
    sim.close()
    for name, mr in (("global", 0), ("rungs", R)):
        p = dict(w.params, precision=1, h_tol=1e-6, max_rung=mr)
        sim = sph.Simulation(start, w.materials, p, device=str(dev))
        info = sim.prime()
        e0 = info["e_kin"] + info["e_int"] + info["e_pot"]
        sim.set_spans(1, 2)
        sim.set_graph(True)
        for _ in range(args.warmup):
            info = sim.step((2 ** mr) * info["dt_next"])
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_sim, calls, updates, hist = 0.0, 0, 0, np.zeros(16, np.int64)
        t0 = time.perf_counter()
        ev0.record(stream)
        while True:
            dt = (2 ** mr) * info["dt_next"]
            info = sim.step(dt)
            t_sim += dt
            calls += 1
            updates += info["particle_updates"]
            hist += np.array(info["rung_counts"])
            if (t_target is None and calls >= args.steps) or (t_target is not None and t_sim >= t_target):
                break
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1)
        wall = time.perf_counter() - t0
        if t_target is None:
            t_target = t_sim
        e1 = info["e_kin"] + info["e_int"] + info["e_pot"]
        arms[name] = {"calls": calls, "simulated_s": t_sim, "device_ms": ms, "wall_s": wall,
                      "simulated_per_device_s": t_sim / (ms / 1e3),
                      "particle_updates_per_s": updates / (ms / 1e3),
                      "updates_per_particle_per_sim_s": updates / w.n / t_sim,
                      "rung_share": (hist / max(1, hist.sum())).round(4).tolist()[:max(1, mr + 1)],
                      "dE_over_Ekin0": (e1 - e0) / info["e_kin"]}
        sim.close()
    g, r = arms["global"], arms["rungs"]
    line = {"mode": "rungs", "workload": "basalt impact 1.8M+0.2M particles, 5 km/s, 45 deg",
            "particles": w.n, "max_rung": R, "form": "fp32k, graph",
            "arms": arms,
            "speedup_simulated_time": r["simulated_per_device_s"] / g["simulated_per_device_s"],
            "relax_steps": args.relax_steps, "warmup": args.warmup,
            "note": "same physical time from the same relaxed state; the rung run's big step "
                    "is 2^R dt_next"}
    print(json.dumps(line), flush=True)


def _by_id(g: dict, keys) -> dict:
    order = np.argsort(g["id"], kind="stable")
    return {k: g[k][order] for k in keys}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32k", choices=["fp32k", "fp64"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--copy-chunks", type=int, default=0,
                    help="force-pass launches whose outputs sph_step_host copies back as "
                         "each completes (0: the library's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--tune", type=int, default=2)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--spans", default="", help="density,forces group spans (no tuning)")
    ap.add_argument("--plain-steps", type=int, default=0,
                    help="plain-form steps (0: all of the chosen form's timed steps)")
    ap.add_argument("--workload", default="impact", choices=["impact", "batch64", "learned", "drift", "rungs"])
    ap.add_argument("--max-rung", type=int, default=2)
    ap.add_argument("--relax-steps", type=int, default=20,
                    help="rungs mode: global steps from the seeded state before both arms")
    ap.add_argument("--drift-steps", type=int, default=100)
    ap.add_argument("--spot-every", type=int, default=5)
    ap.add_argument("--spot", type=int, default=10_000)
    ap.add_argument("--history-steps", type=int, default=200)
    ap.add_argument("--record-every", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--learned-scale", type=float, default=1.0)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch64":
            run_batch(args, rank, world, local_rank)
        elif args.workload == "learned":
            run_learned(args, rank, world, local_rank)
        elif args.workload == "drift":
            run_drift(args, rank, world, local_rank)
        elif args.workload == "rungs":
            run_rungs(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
