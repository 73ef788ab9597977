#!/usr/bin/env python3
"""Throughput of deep-potential MD on one B300: energy+force atom-steps/s.

One step = one velocity-Verlet MD step of the whole hot path (neighbour update,
environment, embedding, attention layers, descriptor, fitting, hand-written
backward, force/virial assembly, integration) on the 24,000-atom synthetic
protein-in-water system (1,500-atom H/C/N/O/S blob in 7,500 waters, 57.69 x
57.69 x 72.11 A, 0.1 atoms/A^3) with the attention-family model (embedding
1->32->64->128, 3 attention layers of width 128 with 4 heads, axis 16,
fitting 2048->240->240->240->1, rc 6 A, nmax 120), random N(0, 0.1) weights,
300 K Maxwell-Boltzmann velocities, dt 0.5 fs, lists rebuilt every 10 steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fused|plain]
    python bench.py --impl reference ...      # the FP64 CPU oracle on host cores
    python bench.py --report 1,2,3,4,5        # per-configuration accuracy/drift/latency reports

Prints one JSON line (rank 0).  N > 1 (torchrun) runs N independent replicas,
one per GPU (the model is atom-local; no collective is needed): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import configs as CF, maxwell_boltzmann, normal_blob  # noqa: E402

WORKLOAD = ("protein-in-water 24,000 atoms (1,500-atom blob + 7,500 H2O, 57.69x57.69x72.11 A), "
            "attention family: embedding 1-32-64-128, 3 attention layers (H 128, 4 heads), "
            "axis 16, fitting 2048-240-240-240-1, rc 6 A, nmax 120; NVE dt 0.5 fs, rebuild every 10")
GRAPH_WORKLOAD = ("protein-in-water 24,000 atoms (same system), graph family: node 128, edge 64, "
                  "6 layers, angle channel 40 nearest within 4 A, fitting 128-240-240-240-1, "
                  "rc 6 A, nmax 120; NVE dt 0.5 fs, rebuild every 10")
METRIC = "energy+force atom-steps/s"
FP32_ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # 148 SMs x 128 FP32 lanes x FMA x 2.032 GHz
# DRAM bytes (read + write) per atom of one launch, from an ncu capture of the
# 4,800-atom case (`--system small`); traffic grows with the atoms processed
# (per-atom tiles, lists, gradients), so a launch over N atoms moves N x this.
# These are not measured by this program: they hold for the kernel source whose
# SHA-256 prefix is recorded beside them, and the line reports null otherwise.
NCU_TRAFFIC_PER_ATOM = {"k_af_bwd": (545.724672e6 + 9.589760e6) / 4800,
                        "k_af_fwd": (16.883712e6 + 452.838144e6) / 4800}
NCU_TRAFFIC_SOURCE = ("paper_2602_02234_b300/csrc/fused_af.cu", "313160fdb172cd7c")


def _source_sha(rel):
    import hashlib
    try:
        with open(os.path.join(ROOT, rel), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def traffic_per_atom(kernel):
    """The captured DRAM bytes per atom of `kernel`, or None when the kernel's
    source has changed since the capture."""
    rel, sha = NCU_TRAFFIC_SOURCE
    if kernel not in NCU_TRAFFIC_PER_ATOM or not sha or _source_sha(rel) != sha:
        return None
    return NCU_TRAFFIC_PER_ATOM[kernel]


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ replicas
def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x: a job is as slow as its slowest replica."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ algorithmic work
def af_flops_per_atom(model, n):
    """Algorithmic FLOPs for one atom with n real neighbours, split as
    (forward network, fitting forward + input gradient, backward network);
    padding to 128 rows and the backward's recomputation are excluded."""
    d = model.as_dict()
    e1, e2, m1, m2, H, L = d["e1"], d["e2"], d["m1"], d["m2"], d["hidden"], d["n_layers"]
    emb = 2 * n * (e1 + e1 * e2 + e2 * m1)
    att_fwd = 2 * n * m1 * 3 * H + 4 * n * n * H + 2 * n * H * m1
    att_bwd = 2 * n * m1 * H + 8 * n * n * H + 2 * n * 3 * H * m1
    desc = 2 * 4 * n * m1 + 2 * 4 * m1 * m2
    fit = 2 * (m1 * m2 * d["f1"] + d["f1"] * d["f2"] + d["f2"] * d["f3"] + d["f3"])
    return (emb + L * att_fwd + desc, 2 * fit, emb + L * att_bwd + 2 * desc)


def setup_system(which="protein24k", message_passing=False, family="attention"):
    if which == "small":   # profiling case: same recipe, 4,800 atoms (300-atom blob)
        from synth import cached, protein_in_water
        s = cached(protein_in_water, 4800, 300, (33.74, 33.74, 42.17), CF.SYSTEM_SEED + 1)
    else:
        s = CF.protein24k()
    model = CF.GRAPH_MODEL if family == "graph" else CF.ATTN_MODEL
    if message_passing:
        from dataclasses import replace
        model = replace(model, message_passing=1)
    masses = s.masses
    v0 = maxwell_boltzmann(masses[s.types], 300.0, CF.VELOCITY_SEED)
    return s, model, masses, v0


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    s, model, masses, v0 = setup_system()
    w = normal_blob(oracle.af_weight_count(model), CF.WEIGHT_SEED)
    rng = np.random.default_rng(0)
    per_step = args.ref_sample
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    for _ in range(args.warmup):
        oracle.af_atoms(model, w, s.types, s.coords, s.box, rng.choice(s.n, per_step, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.af_atoms(model, w, s.types, s.coords, s.box, rng.choice(s.n, per_step, replace=False))
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    sample = (f"{per_step} random centre atoms per step (energy + pair gradients of each, FP64 "
              f"C oracle, OpenMP over atoms)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_atoms": s.n},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": threads,
                             "kind": "oracle", "sample": sample, "nproc": os.cpu_count(),
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(seconds=12.0, seconds_1thread=6.0):
    """The oracle as it stands, timed on this host over a bounded random
    sample: OpenMP over every host core, then on one thread."""
    import oracle
    s, model, _, _ = setup_system()
    w = normal_blob(oracle.af_weight_count(model), CF.WEIGHT_SEED)
    rng = np.random.default_rng(1)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def rate(nthreads, batch, budget):
        done = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget:
            oracle.af_atoms(model, w, s.types, s.coords, s.box,
                            rng.choice(s.n, batch, replace=False), nthreads)
            done += batch
        dt = time.perf_counter() - t0
        return done, dt

    done, dt = rate(threads, max(8, threads * 4), seconds)
    done1, dt1 = rate(1, 2, seconds_1thread)
    return {"value": done / dt, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} random centre atoms of the 24,000-atom system in {dt:.1f} s "
                      f"(energy + pair gradients per atom, FP64, OpenMP)",
            "value_1thread": done1 / dt1,
            "sample_1thread": f"{done1} random centre atoms on one thread in {dt1:.1f} s",
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


# ------------------------------------------------------------------ serving
def serving_bench(n_req, seed=7, load=0.9, n_steps=50, capacity=None, mem_budget=0):
    """Continuous batching of independent systems (sizes log-uniform 96..6000,
    50 MD steps each): capacity with every request queued at once (unless
    given), then a Poisson-arrival run at `load` times that capacity.  Returns
    p50/p99 tick (step) latency, request latency and aggregate atom-steps/s.
    mem_budget > 0 caps the device memory of the resident batch (bytes)."""
    import paper_2602_02234_b300 as dp
    from paper_2602_02234_b300 import serve
    from synth import serving_requests

    model = CF.ATTN_MODEL
    desc = dp.model_desc(model, dp.PREC_FUSED, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY)
    w = normal_blob(dp.weight_count(desc), CF.WEIGHT_SEED)
    reqs = serving_requests(n_req, 0.0, seed, n_steps=n_steps)
    masses = reqs[0].system.masses
    vels = [maxwell_boltzmann(masses[r.system.types], 300.0, CF.VELOCITY_SEED + k)
            for k, r in enumerate(reqs)]
    mean_atoms = float(np.mean([r.system.n for r in reqs]))
    kw = {"mem_budget": mem_budget} if mem_budget else {}
    if capacity is None:
        srv = dp.Server(desc, w, masses, max_slots=64, dt_fs=CF.DT_FS, **kw)
        _, st_cap = serve.run(srv, reqs, vels)
        srv.close()
        capacity = st_cap["atom_steps"] / st_cap["wall_s"]
    rate = load * capacity / (mean_atoms * n_steps)
    reqs = serving_requests(n_req, rate, seed, n_steps=n_steps)
    srv = dp.Server(desc, w, masses, max_slots=64, dt_fs=CF.DT_FS, **kw)
    _, st = serve.run(srv, reqs, vels)
    srv.close()
    return {"requests": n_req, "steps_per_request": n_steps, "offered_load": load,
            "arrival_rate_per_s": rate, "capacity_atom_steps_per_s": capacity,
            "p50_step_ms": st["p50_tick_ms"], "p99_step_ms": st["p99_tick_ms"],
            "request_p50_ms": st["request_p50_ms"], "request_p99_ms": st["request_p99_ms"],
            "atom_steps_per_s": st["atom_steps"] / st["wall_s"], "max_resident": st["max_resident"],
            "mem_budget_bytes": mem_budget or None,
            "sizes": "log-uniform 96..6000 atoms, water below 600, 6.25 % blob above"}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2602_02234_b300 as dp

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    graph = args.family == "graph"
    s, model, masses, v0 = setup_system(args.system, args.message_passing, args.family)
    w = normal_blob(dp.weight_count(dp.model_desc(model, dp.PREC_PLAIN_F32)), CF.WEIGHT_SEED)
    stream = torch.cuda.Stream()

    def make(prec):
        return dp.DeepPotential(dp.model_desc(model, prec, skin=CF.SKIN,
                                              rebuild_every=CF.REBUILD_EVERY),
                                s.types, s.box, w, masses=masses, stream=stream)

    forms = []
    fused_name = "mixed_tc_f16" if graph else "fused_f16"
    if args.form in ("auto", "fused"):
        try:
            forms.append((fused_name, make(dp.PREC_FUSED)))
        except dp.DPError as e:
            if args.form == "fused":
                raise
            print(f"# fused form unavailable: {e}", file=sys.stderr)
    if args.form in ("auto", "plain"):
        forms.append(("plain_f32", make(dp.PREC_PLAIN_F32)))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def time_steps(pot, K):
        pot.set_state(s.coords, v0, 0)
        pot.step(args.warmup, CF.DT_FS)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        with ClockSampler(local_rank) as clk:
            with torch.cuda.stream(stream):
                e0.record(stream)
                pot.step(K, CF.DT_FS)
                e1.record(stream)
            e1.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        return ms, clk.summary()

    results = {}
    for name, pot in forms:
        ms, clocks = time_steps(pot, args.steps)
        results[name] = {"ms": ms, "clocks": clocks, "pot": pot}

    main_name = forms[0][0]
    main = results[main_name]
    pot = main["pot"]
    K = args.steps
    value = job_throughput(s.n * K, world, main["ms"] / 1e3)

    # the dominant kernel alone, timed with events on the stream it runs on
    cnt, _, _ = pot.neighbours()
    nreal = np.minimum(cnt, model.nmax)
    parts = None if graph else np.array([af_flops_per_atom(model, int(k)) for k in nreal]).sum(0)
    reps = 5

    def time_network(part_mask):
        pot.enqueue_network(1, part_mask)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            pot.enqueue_network(reps, part_mask)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    pk, pk_kind = peaks()
    if graph:
        # memory-bound: the edge features (pairs x Ed) must be read and written
        # once per layer in the forward and their adjoint once per layer in the
        # backward, a floor under every evaluation's DRAM traffic; the mixed form
        # stores the edge state in 16 bits and its adjoint in FP32
        net_ms = time_network(0)
        kernel_ms = {"network": net_ms}
        alg_bytes = float(model.n_layers * int(nreal.sum()) * model.edge * (2 * 2 + 2 * 4))
        achieved = alg_bytes / (net_ms / 1e3) / 1e9
        peak = pk.get("hbm_gbs", 6400.0)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "graph network phase (all kernels of one evaluation)",
                    "peak_kind": f"HBM copy bandwidth ({pk_kind})",
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "algorithmic_bytes_note": "L x pairs x Ed x (2 x 2 B + 2 x 4 B): the 16-bit edge "
                                              "state read and written per layer forward, its FP32 "
                                              "adjoint read and written per layer backward",
                    "launch_ms": net_ms, "kernel_ms": kernel_ms}
    elif main_name == "fused_f16":
        kernel_ms = {name: time_network(mask) for name, mask in
                     (("k_af_fwd", 1), ("k_fit", 2), ("k_af_bwd", 4))}
        dominant = max(kernel_ms, key=kernel_ms.get)
        flops = float(parts[{"k_af_fwd": 0, "k_fit": 1, "k_af_bwd": 2}[dominant]])
        net_ms = kernel_ms[dominant]
        # each kernel is timed alone (a few back-to-back launches, well under a
        # second), so the burst peak is the one that applies
        peak = pk.get("bf16_tflops", 1800.0)
        bound = "tensor"
        peak_note = (f"dense 16-bit tensor peak, burst ({pk_kind}; the kernel is timed alone; "
                     "the FP16 rate equals the measured BF16 rate, nominal ratio 1)")
        kernel_name = dominant
    else:
        net_ms = time_network(0)
        kernel_ms = {"network": net_ms}
        flops = float(parts.sum())
        peak = FP32_ALU_PEAK_TFLOPS
        bound, peak_note = "alu", "FP32 FFMA: 148 SMs x 128 lanes x 2 x 2.032 GHz (derived)"
        kernel_name = "plain network phase (all kernels of one evaluation)"
    if not graph:
        achieved = flops / (net_ms / 1e3) / 1e12
        if args.message_passing:   # every network part is several launches plus cross-atom steps
            kernel_name += " (message passing: one launch per layer)"
        traffic = traffic_per_atom(kernel_name)
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": traffic * s.n if traffic else None,
                    "traffic_note": "not measured by this run: DRAM bytes per atom from an ncu "
                                    "capture of the same kernel source on 4,800 atoms, times "
                                    "the atoms of one launch (null when the source differs)",
                    "kernel": kernel_name,
                    "peak_kind": peak_note, "algorithmic_flop_per_launch": flops,
                    "launch_ms": net_ms, "kernel_ms": kernel_ms}

    # end to end through the C ABI with pinned host buffers, copies every step
    xh = torch.empty((s.n, 3), dtype=torch.float64, pin_memory=True).numpy()
    vh = torch.empty((s.n, 3), dtype=torch.float64, pin_memory=True).numpy()
    x_now, v_now, _ = pot.get_state()
    xh[:] = x_now
    vh[:] = v_now
    barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        tr = pot.step(1, CF.DT_FS, coords=xh, vel=vh, energies=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_throughput(s.n * K, world, e2e_s), "unit": "atom-steps/s",
           "h2d_bytes_per_step": 2 * xh.nbytes, "d2h_bytes_per_step": 2 * xh.nbytes + tr.nbytes,
           "note": "host wall clock around dp_step(1) with pinned host coords/velocities in and out"}

    n_comp, n_step = pot.kernels_per_step()
    line = {"metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": main["ms"] / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16" if main_name in ("fused_f16", "mixed_tc_f16") else "f32",
            "data": "synthetic",
            "config": {"workload": (GRAPH_WORKLOAD if graph else WORKLOAD)
                       if args.system == "protein24k" else
                       f"small profiling case ({s.n} atoms)", "n_atoms": s.n, "form": main_name,
                       "family": args.family,
                       "message_passing": bool(args.message_passing),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: skin/selection lists and pair gradients "
                             "(~0.4 GB per step) exceed the 126 MB L2"},
            "clocks": main["clocks"], "e2e": e2e, "gpu_launches": n_step * K,
            "roofline": roofline}
    for name in results:
        line[name] = {"value": job_throughput(s.n * K, world, results[name]["ms"] / 1e3),
                      "ms_per_step": results[name]["ms"] / K}
    if fused_name in results and "plain_f32" in results:
        line["fused_vs_plain"] = results["plain_f32"]["ms"] / results[fused_name]["ms"]
        if not graph:
            # the comparison arm's own roofline: its network phase (all plain
            # kernels of one evaluation) against the derived FP32 FFMA peak
            ppot = results["plain_f32"]["pot"]
            ppot.enqueue_network(1, 0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                ppot.enqueue_network(2, 0)
                e1.record(stream)
            e1.synchronize()
            pms = e0.elapsed_time(e1) / 2
            pflops = float(parts.sum())
            line["plain_f32"]["roofline"] = {
                "bound": "alu", "achieved": pflops / (pms / 1e3) / 1e12,
                "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": pflops / (pms / 1e3) / 1e12 / FP32_ALU_PEAK_TFLOPS,
                "kernel": "plain network phase (all kernels of one evaluation)",
                "peak_kind": "FP32 FFMA: 148 SMs x 128 lanes x 2 x 2.032 GHz (derived)",
                "algorithmic_flop_per_launch": pflops, "launch_ms": pms}
    plain_model = not args.message_passing and not graph
    if rank == 0 and args.serving > 0 and args.system == "protein24k" and plain_model:
        line["serving"] = serving_bench(args.serving)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.system == "protein24k" and plain_model:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for name, p in forms:
        p.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ per-configuration reports
def _drift(tr, n_atoms, dt_fs):
    """Total-energy drift of an NVE trace: least-squares slope per atom per ns,
    and the largest excursion from the first value per atom."""
    et = tr.sum(1)
    t_ns = np.arange(len(et)) * dt_fs * 1e-6
    slope = float(np.polyfit(t_ns, et, 1)[0]) if len(et) > 2 else 0.0
    return {"steps": len(et), "slope_eV_per_atom_per_ns": slope / n_atoms,
            "max_excursion_eV_per_atom": float(np.max(np.abs(et - et[0]))) / n_atoms}


def _err(F, Fo, E=None, Eo=None):
    rms = float(np.sqrt(np.mean(Fo ** 2)))
    out = {"max_abs_dF_over_F_rms": float(np.max(np.abs(F - Fo))) / rms,
           "rms_dF_over_F_rms": float(np.sqrt(np.mean((F - Fo) ** 2))) / rms, "F_rms": rms}
    if E is not None:
        out["rel_dE"] = abs(E - Eo) / abs(Eo)
    return out


def _timed_steps(pot, K, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        pot.step(K, CF.DT_FS)
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / K


def report_config(which):
    """One JSON object for configuration `which` (1..5) of the benchmark set."""
    import torch
    import oracle
    import paper_2602_02234_b300 as dp
    stream = torch.cuda.Stream()
    out = {"config": which}
    if which == 1:      # 64 waters, FP64 / FP32 / fused against the oracle, 100 NVE steps
        m, s = CF.WATER64_MODEL, CF.water64()
        w = normal_blob(oracle.af_weight_count(m), CF.WEIGHT_SEED)
        masses = s.masses
        v0 = maxwell_boltzmann(masses[s.types], 300.0, CF.VELOCITY_SEED)
        Eo, _, Fo, _ = oracle.af_compute(m, w, s.types, s.coords, s.box)
        t0 = time.perf_counter()
        xo, vo, epo, eko = oracle.af_md(m, w, s.types, masses, s.coords, v0, s.box, 100, CF.DT_FS)
        out["oracle_md_atom_steps_per_s"] = s.n * 100 / (time.perf_counter() - t0)
        out["oracle_drift"] = _drift(np.stack([epo, eko], 1), s.n, CF.DT_FS)
        for name, prec in (("plain_f64", dp.PREC_PLAIN_F64), ("plain_f32", dp.PREC_PLAIN_F32),
                           ("fused_f16", dp.PREC_FUSED)):
            pot = dp.DeepPotential(dp.model_desc(m, prec), s.types, s.box, w, masses=masses,
                                   stream=stream)
            E, F, V = pot.compute(s.coords)
            x, v = s.coords.copy(), v0.copy()
            tr = pot.step(100, CF.DT_FS, coords=x, vel=v, energies=True)
            pot.set_state(s.coords, v0, 0)
            pot.step(5, CF.DT_FS)
            ms = _timed_steps(pot, 100, stream)
            out[name] = {"vs_oracle": _err(F, Fo, E, Eo), "drift": _drift(tr, s.n, CF.DT_FS),
                         "x_after_100_vs_oracle_max_A": float(np.max(np.abs(x - xo))),
                         "ms_per_step": ms, "atom_steps_per_s": s.n / (ms / 1e3)}
            pot.close()
    elif which == 2:    # 24,000 atoms: NVE drift of the fused and plain forms, force agreement
        s, m, masses, v0 = setup_system()
        w = normal_blob(oracle.af_weight_count(m), CF.WEIGHT_SEED)
        pots = {}
        # 100 steps (50 fs): with random-init weights the system leaves equilibrium
        # within ~100 fs (the potential energy falls by thousands of eV and the
        # integration breaks down for every form), so drift is measured before that
        for name, prec, n_steps in (("fused_f16", dp.PREC_FUSED, 100),
                                    ("plain_f32", dp.PREC_PLAIN_F32, 100)):
            pot = dp.DeepPotential(dp.model_desc(m, prec, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                                   s.types, s.box, w, masses=masses, stream=stream)
            E, F, V = pot.compute(s.coords)
            pot.set_state(s.coords, v0, 0)
            t0 = time.perf_counter()
            tr = pot.step(n_steps, CF.DT_FS, energies=True)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            out[name] = {"drift": _drift(tr, s.n, CF.DT_FS),
                         "atom_steps_per_s_over_run": s.n * n_steps / wall}
            pots[name] = (E, F, pot)
        Ef, Ff, _ = pots["fused_f16"]
        Ep, Fp, _ = pots["plain_f32"]
        out["fused_vs_plain_f32"] = _err(Ff, Fp, Ef, Ep)
        rng = np.random.default_rng(3)
        sample = np.sort(rng.choice(s.n, 48, replace=False))
        Fo = oracle.af_forces_subset(m, w, s.types, s.coords, s.box, sample)
        out["fused_vs_oracle_48_atoms"] = _err(Ff[sample], Fo)
        out["plain_f32_vs_oracle_48_atoms"] = _err(Fp[sample], Fo)
        for _, _, pot in pots.values():
            pot.close()
        # the paper's set-up: the deep potential covers the protein only (DP group)
        mask = np.zeros(s.n, bool)
        mask[: s.blob_atoms] = True
        pot = dp.DeepPotential(dp.model_desc(m, dp.PREC_FUSED, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                               s.types, s.box, w, masses=masses, stream=stream)
        pot.set_group(mask)
        Eg, Fg, _ = pot.compute(s.coords)
        pot.set_state(s.coords, v0, 0)
        pot.step(3, CF.DT_FS)
        ms = _timed_steps(pot, 20, stream)
        Ego, _, Fgo, _ = oracle.af_compute_group(m, w, s.types, s.coords, s.box, mask)
        # four fitting heads on the shared descriptor (energies of all four per step)
        from dataclasses import replace as _replace
        m4 = _replace(m, fit_heads=4)
        w4 = normal_blob(oracle.af_weight_count(m4), CF.WEIGHT_SEED)
        pot4 = dp.DeepPotential(dp.model_desc(m4, dp.PREC_FUSED, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                                s.types, s.box, w4, masses=masses, stream=stream)
        pot4.set_state(s.coords, v0, 0)
        pot4.step(3, CF.DT_FS)
        out["fit_heads_4_fused"] = {"ms_per_step": _timed_steps(pot4, 20, stream),
                                    "head_energies": [float(x) for x in pot4.head_energies()]}
        pot4.close()
        out["dp_group_protein_fused"] = {
            "members": int(mask.sum()), "ms_per_step": ms,
            "member_atom_steps_per_s": int(mask.sum()) / (ms / 1e3),
            "vs_oracle": _err(Fg[mask], Fgo[mask], Eg, Ego)}
        pot.close()
        # cross-atom message passing (atom channel passed between neighbours
        # each layer), plain FP32 against the same path without it
        mm = _replace(m, message_passing=1)
        wm = normal_blob(oracle.af_weight_count(mm), CF.WEIGHT_SEED)
        res_mp = {}
        for name, mdl, wts, prec, K in (
                ("plain_f32", m, w, dp.PREC_PLAIN_F32, 5),
                ("message_passing_plain_f32", mm, wm, dp.PREC_PLAIN_F32, 5),
                ("fused_f16", m, w, dp.PREC_FUSED, 20),
                ("message_passing_fused_f16", mm, wm, dp.PREC_FUSED, 20)):
            pot = dp.DeepPotential(dp.model_desc(mdl, prec, skin=CF.SKIN,
                                                 rebuild_every=CF.REBUILD_EVERY),
                                   s.types, s.box, wts, masses=masses, stream=stream)
            pot.set_state(s.coords, v0, 0)
            pot.step(3, CF.DT_FS)
            res_mp[name] = (_timed_steps(pot, K, stream), pot.compute(s.coords))
            pot.close()
        for form, base in (("plain_f32", "plain_f32"), ("fused_f16", "fused_f16")):
            ms = res_mp["message_passing_" + form][0]
            out["message_passing_" + form] = {
                "ms_per_step": ms, "atom_steps_per_s": s.n / (ms / 1e3),
                "without_messages_ms_per_step": res_mp[base][0],
                "overhead": ms / res_mp[base][0] - 1.0}
        Emf, Fmf, _ = res_mp["message_passing_fused_f16"][1]
        Emp, Fmp, _ = res_mp["message_passing_plain_f32"][1]
        out["message_passing_fused_vs_plain_f32"] = _err(Fmf, Fmp, Emf, Emp)
    elif which == 3:    # graph family at 24,000 atoms
        s, _, masses, v0 = setup_system()
        m = CF.GRAPH_MODEL
        w = normal_blob(oracle.gf_weight_count(m), CF.WEIGHT_SEED)
        res = {}
        for name, prec, K in (("plain_f32", dp.PREC_PLAIN_F32, 5), ("plain_f64", dp.PREC_PLAIN_F64, 2),
                              ("mixed_tc_f16", dp.PREC_FUSED, 5)):
            pot = dp.DeepPotential(dp.model_desc(m, prec, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                                   s.types, s.box, w, masses=masses, stream=stream)
            E, F, V = pot.compute(s.coords)
            pot.set_state(s.coords, v0, 0)
            pot.step(2, CF.DT_FS)
            ms = _timed_steps(pot, K, stream)
            res[name] = (E, F, pot)
            out[name] = {"ms_per_step": ms, "atom_steps_per_s": s.n / (ms / 1e3)}
        E32, F32, _ = res["plain_f32"]
        E64, F64, p64 = res["plain_f64"]
        out["f32_vs_f64"] = _err(F32, F64, E32, E64)
        out["mixed_tc_f16_vs_f64"] = _err(res["mixed_tc_f16"][1], F64, res["mixed_tc_f16"][0], E64)
        rng = np.random.default_rng(11)
        atoms = rng.choice(s.n, 6, replace=False)
        h, worst = 1e-4, 0.0
        for i in atoms:
            for a in range(3):
                xp = s.coords.copy(); xp[i, a] += h
                xm = s.coords.copy(); xm[i, a] -= h
                fd = -(p64.compute(xp)[0] - p64.compute(xm)[0]) / (2 * h)
                worst = max(worst, abs(fd - F64[i, a]))
        out["fd_check"] = {"atoms": len(atoms), "h_A": h, "max_abs_dF_over_F_rms":
                           worst / float(np.sqrt(np.mean(F64 ** 2)))}
        for _, _, pot in res.values():
            pot.close()
        # the attention family on the same system and precision, for the AF/GF ratio
        sa, ma, _, _ = setup_system()
        wa = normal_blob(oracle.af_weight_count(ma), CF.WEIGHT_SEED)
        for name, prec, K in (("af_plain_f32", dp.PREC_PLAIN_F32, 5), ("af_fused_f16", dp.PREC_FUSED, 20)):
            pot = dp.DeepPotential(dp.model_desc(ma, prec, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                                   sa.types, sa.box, wa, masses=masses, stream=stream)
            pot.set_state(sa.coords, v0, 0)
            pot.step(3, CF.DT_FS)
            out[name] = {"ms_per_step": _timed_steps(pot, K, stream)}
            pot.close()
        out["af_over_gf_throughput_f32"] = out["plain_f32"]["ms_per_step"] / out["af_plain_f32"]["ms_per_step"]
    elif which == 4:    # serving: offered-load sweep and a memory-capped run
        first = serving_bench(256, load=0.25)
        cap = first["capacity_atom_steps_per_s"]
        out["sweep"] = [first] + [serving_bench(256, load=ld, capacity=cap)
                                  for ld in (0.5, 0.75, 0.9, 1.0, 1.2)]
        out["memory_capped_2GB"] = serving_bench(256, load=0.9, capacity=cap, mem_budget=2 << 30)
    elif which == 5:    # 100,000 atoms: fused vs plain FP32
        s = CF.protein100k()
        m = CF.ATTN_MODEL
        masses = s.masses
        v0 = maxwell_boltzmann(masses[s.types], 300.0, CF.VELOCITY_SEED)
        w = normal_blob(oracle.af_weight_count(m), CF.WEIGHT_SEED)
        res = {}
        for name, prec, K in (("fused_f16", dp.PREC_FUSED, 50), ("plain_f32", dp.PREC_PLAIN_F32, 3)):
            pot = dp.DeepPotential(dp.model_desc(m, prec, skin=CF.SKIN, rebuild_every=CF.REBUILD_EVERY),
                                   s.types, s.box, w, masses=masses, stream=stream)
            E, F, V = pot.compute(s.coords)
            pot.set_state(s.coords, v0, 0)
            pot.step(3, CF.DT_FS)
            ms = _timed_steps(pot, K, stream)
            out[name] = {"ms_per_step": ms, "atom_steps_per_s": s.n / (ms / 1e3), "steps": K}
            res[name] = (E, F)
            pot.close()
        out["fused_vs_plain"] = out["plain_f32"]["ms_per_step"] / out["fused_f16"]["ms_per_step"]
        out["fused_vs_plain_f32"] = _err(res["fused_f16"][1], res["plain_f32"][1],
                                         res["fused_f16"][0], res["plain_f32"][0])
        rng = np.random.default_rng(5)
        sample = np.sort(rng.choice(s.n, 32, replace=False))
        Fo = oracle.af_forces_subset(m, w, s.types, s.coords, s.box, sample)
        out["fused_vs_oracle_32_atoms"] = _err(res["fused_f16"][1][sample], Fo)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["auto", "fused", "plain"], default="auto")
    ap.add_argument("--ref-sample", type=int, default=48)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=256,
                    help="requests in the continuous-batching measurement (0: skip)")
    ap.add_argument("--system", choices=["protein24k", "small"], default="protein24k",
                    help="small: 4,800-atom box of the same recipe, for profiler captures")
    ap.add_argument("--family", choices=["attention", "graph"], default="attention",
                    help="graph: the graph family's step (mixed tensor-core form and plain FP32; "
                         "no serving or CPU-baseline legs)")
    ap.add_argument("--message-passing", action="store_true",
                    help="the attention family with cross-atom message passing (no serving or "
                         "CPU-baseline legs: its oracle is a whole-system program)")
    ap.add_argument("--report", default="",
                    help="comma-separated configurations (1-5): accuracy, drift, latency, graph "
                         "family, serving sweep, 100k atoms; one JSON line each, no timing contract")
    args = ap.parse_args()
    if args.report:
        for c in args.report.split(","):
            print(json.dumps(report_config(int(c))), flush=True)
        return 0
    args.warmup = max(3, args.warmup)       # timing rule: at least 3 untimed warm-up steps
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
