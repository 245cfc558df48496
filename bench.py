"""Benchmark: free-flight segments per second of the GB300 tracer.

Workload (one step): the silicon-like thin film, 100 nm, diffuse walls,
uniform gradient along z, 3 x 1000 modes at 300 K, 1e7 particles, 40
scattering events / 4096 segments per particle at most, FP32 trajectories
with FP64 tallies.  One step traces every particle from emission to
termination (steps I-VI of the trajectory algorithm) in one le_mc_run.

Printed JSON line (rank 0):
  value        segments/s over the K timed steps, device-timed with CUDA events
               on the launching stream, material tables resident in HBM
  e2e          the same metric through the public C ABI with host descriptors:
               material build + upload, run, read-back, destroy, every step
  roofline     dominant kernel against the ALU-issue peak (bound "alu")
  cpu_baseline the FP64 oracle on this host's cores over a bounded sample
  clocks       nvidia-smi samples taken during the timed region

``--impl reference`` times the FP64 CPU oracle (the reference for this
method) on the same workload and metric, one bounded sample per step.
Under torchrun (--gpus N > 1) each rank traces its own independent instance
(weak scaling, no data-path collective); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_PARTICLES = 10_000_000
METRIC = "free-flight segments/s per GB300 (plain vs batched); p50/p99 latency at 1% std error"
UNIT = "segments/s"
WORKLOAD = ("silicon-like thin film 100 nm, diffuse walls, gradient along z, LA + doubly degenerate TA x 1000 bins (2000 modes) at 300 K, "
            "1e7 particles, K_s=40, K_e=4096, FP32 trajectories / FP64 tallies")

# Algorithmic lane operations per free-flight segment of the film kernel
# (counted from the algorithm, not from the compiled code):
#   Philox4x32-10: 10 rounds x (2 wide multiplies + 2 three-input XORs)  40
#   three uniforms from the random words (shift/or + add)                   6
#   flight length -Lambda ln u (log2 + 2 multiplies)                        3
#   wall distance (select numerator, reciprocal, multiply, compare, min)    7
#   advance x, snap at walls, accumulate L_z                                4
#   new direction (sincos, sqrt pair, three components, selects)           14
#   Eq. 2 mode redraw on scattering (wide multiply, 2 loads, compare,
#     select), weighted by the scattering share of segments (~0.8)          4
#   event counters and termination tests                                    6
OPS_PER_SEGMENT = 84
LANES_PER_SM = 128  # FP32/INT32 lanes issuing one operation per clock

# The other kernels timed here, counted the same way (lane operations from
# the algorithm; a transcendental, reciprocal or square root counts as one):
#   gray slab, walls source, black walls, one mode, 50-bin profile: the film's
#     84 without the Eq. 2 table lookup (one mode: -4), plus the profile: bin
#     range (2 floors, 2 clamps), time per unit x (rcp, mul), two partial-bin
#     and one whole-bin range update of T and q (6 shared FP64 adds, 10
#     products)                                                             +22
OPS_SLAB = 84 - 4 + 22
#   pored film, steady: the film's 84 plus the cylinder (squared norms and the
#     dot product 6, discriminant 2, sqrt, difference, reciprocal, product,
#     clamp, two tests, compare/select 3: 16), two unit-cell faces ahead
#     (select numerator, reciprocal, product, compare, select: 10), y and z
#     advance (2), pore-wall normal and cosine law about it (2 differences, 2
#     products, 6 multiply-adds: 10), outcome selects for the cylinder and the
#     faces (6) and periodic re-insertion (4)                                 +48
OPS_POROUS = 84 + 48
#   pored film with 8 x 8 steady maps: the pored film's segment plus the map
#     cell range (2 products, 2 floors, 2 clamps, 2 reciprocals, per axis an
#     end-point estimate and its exact check: 12) and the deferred job record
#     (12 shared stores); the per-cell work (merge search, interval, two FP64
#     reductions) is not counted, so this fraction is a lower bound       +28
OPS_POROUS_MAPS = OPS_POROUS + 28
#   surface pulse: the pored film's segment plus the segment end time (rcp,
#     multiply-add), the sample index range (2 products, 2 ceilings, 2 clamps,
#     2 compares) and the deferred job record (11 shared stores): +21 per
#     segment; per sample update: owner search (5 shuffles, 5 compares),
#     interpolated position (1 product, 1 multiply-add, 3 multiply-adds), cell
#     (3 products, 3 floors, 6 clamps, 3 index multiply-adds) and the int32
#     reduction: 31
OPS_PULSE_SEG = OPS_POROUS + 21
OPS_PULSE_SAMPLE = 31
BYTES_PULSE_SAMPLE = 4  # one int32 reduction into the grid per sample update


def _sha_kernel_sources():
    """Hash of the film kernel's sources (its body, helpers and parameter
    layout, and the launcher that picks its instance and launch bounds) with
    comments and whitespace removed, so that only edits which can change the
    compiled code invalidate a capture."""
    h = hashlib.sha256()
    for f in ("trace_kernel.cuh", "device_math.cuh", "le_mc_internal.h", "trace_launch.cu"):
        with open(os.path.join(ROOT, "paper_1206_3316_gb300", "csrc", f)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update(re.sub(r"\s+", "", txt).encode())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per launch of the film kernel from the committed ncu summary,
    or None if the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "trace_kernel_film_fp32_1e7.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m_h = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", txt)
    if not m_b or not m_h or m_h.group(1) != _sha_kernel_sources():
        return None
    return float(m_b.group(1))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"le_mc_clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_problem(problem, rank, world):
    """Weak scaling: rank r traces its own independent instance of the
    workload (instance id r of the counter-based stream)."""
    p = W.with_run(problem, instance_id=int(problem["run"].get("instance_id", 0)) * world + rank)
    return p


def max_over_ranks(value, dist):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_baseline(problem, seconds=12.0):
    """The FP64 oracle on this host's cores over a bounded sample of the
    workload (same film, fewer particles)."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    probe = W.with_run(problem, n_particles=20_000, precision="fp64")
    t0 = time.perf_counter()
    r = O.run(probe, n_threads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_particle = dt / 20_000
    n = int(min(max(seconds / per_particle, 20_000), 2 ** 31))
    sample = W.with_run(problem, n_particles=n, precision="fp64")
    t0 = time.perf_counter()
    r = O.run(sample, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": r["segments"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} particles of the same film workload, FP64, {dt:.1f} s on {cores} threads"}


def batched_measurement(P, torch, dev, stream, steps, launch):
    """Plain vs batched on the many-instance workload: 256 silicon-like films,
    thickness log-uniform in [10 nm, 100 um], particle counts log-uniform in
    [1e4, 1e7].  Plain = one le_mc_run per instance, back to back on one
    stream; batched = one persistent launch over all instances (autotuned
    shape, replayed CUDA graph)."""
    probs = W.batched_films(256)
    total = sum(p["run"]["n_particles"] for p in probs)
    mat = P.le_mc_create_material(P.material_desc(probs[0]["material"]))
    geos = [P.le_mc_create_geometry(P.geometry_desc(p["geometry"])) for p in probs]
    rds = [P.run_desc(p["source"], p["run"], launch) for p in probs]

    def plain_pass():
        hs = [P.le_mc_run(mat, g, r, stream) for g, r in zip(geos, rds)]
        return hs

    for h in plain_pass():  # warm-up
        P.le_mc_destroy_run(h)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    hs = plain_pass()
    b.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = a.elapsed_time(b)
    plain_segs = sum(P.le_mc_read_tallies(h)["segments"] for h in hs)
    plain_launches = sum(P.le_mc_read_tallies(h)["kernel_launches"] for h in hs)
    for h in hs:
        P.le_mc_destroy_run(h)
    for g in geos:
        P.le_mc_destroy_geometry(g)
    P.le_mc_destroy_material(mat)

    with P.Batch(probs) as bt:
        cache = os.path.join(ROOT, "_build", "autotune_cache.txt")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        cfg = bt.autotune(stream, cache_path=cache)
        cfg = dict(cfg, use_graph=True)
        bt.set_config(cfg)
        bt.launch(stream)  # capture + warm-up
        bt.wait()
        ms, segs, launches = [], 0, 0
        for _ in range(max(1, min(steps, 5))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.launch(stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
            res = bt.results()
            segs += sum(r["segments"] for r in res)
            launches += res[0]["kernel_launches"]
    batched = segs / (sum(ms) / 1e3)
    plain = plain_segs / (plain_ms / 1e3)
    return {"value": batched, "unit": UNIT, "plain_sequential": plain, "speedup": batched / plain,
            "instances": len(probs), "particles_per_launch": total, "ms_per_launch": statistics.mean(ms),
            "plain_ms_per_pass": plain_ms, "launch": cfg, "graph": True,
            "workload": "256 silicon-like films, L log-uniform [10 nm, 100 um], N log-uniform [1e4, 1e7]",
            "gpu_launches": launches + plain_launches}


def served_measurement(P, seconds, max_slots=16):
    """Served form: Poisson request arrivals (mean 50/s) mixing gray slabs,
    silicon-like films and porous films of random size, T_eq in [100, 400] K,
    target relative std errors 1 % and 0.3 %, particle budgets log-uniform in
    [1e5, 1e8]; requests are admitted by the native server as slots and
    device memory free up.  Latency = completion - submission."""
    reqs = W.served_stream(duration_s=seconds)
    with P.Server(max_slots=max_slots) as srv:
        ids = []
        t0 = time.perf_counter()
        for r in reqs:
            delay = r["arrival_s"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(r["problem"], r["target_rel_err"]))
        srv.wait_all(1800)
        stats = srv.stats()
        res = [srv.poll(i) for i in ids]
    done = [(q, r) for q, r in zip(reqs, res) if r["state"] == "done"]
    first = min(r["submit_s"] for r in res)
    last = max(r["done_s"] for _, r in done)
    out = {"requests": len(reqs), "completed": len(done), "failed": stats["failed"],
           "aggregate_segments_per_s": stats["segments"] / (last - first), "unit": UNIT,
           "arrival_rate_hz": 50.0, "seconds": seconds, "max_slots": max_slots,
           "resident_kernel_launches": stats["kernel_launches"],
           "latency": "completion - submission, over the requests that reached their target; requests "
                      "that spent their particle budget first are counted apart (missed_target)"}
    for target in (0.01, 0.003):
        mine = [(q, r) for q, r in done if q["target_rel_err"] == target]
        met = sorted(r["done_s"] - r["submit_s"] for q, r in mine if r["rel_err"] <= target)
        missed = [r["done_s"] - r["submit_s"] for q, r in mine if r["rel_err"] > target]
        if met:
            out[f"target_{target:g}"] = {
                "met_target": len(met), "missed_target": len(missed),
                "p50_s": met[len(met) // 2], "p99_s": met[min(len(met) - 1, int(0.99 * len(met)))],
                "missed_p50_s": sorted(missed)[len(missed) // 2] if missed else None}
    return out


def config_measurements(P, torch, dev, stream, flush, steps, warmup, peak_ops, peaks):
    """The other workloads of the method, each timed alone with CUDA events on
    its launching stream (trace kernel only, from le_mc_tallies.kernel_ms,
    and the whole le_mc_run step), L2 flushed before every step:
      slab          gray slab, Kn = 1, black walls at T_eq +- 1 K, T(x) and
                    q(x) on 50 bins, 1e8 particles (FP64, the configuration's
                    precision, and FP32 trajectories)
      porous        steady pored film (300 nm, pitch 100 nm, radius 30 nm,
                    silicon-like, K_s 40, K_e 4096), 1e8 particles, FP32
      porous_maps   the same with steady 8 x 8 maps of T and q_z over the unit
                    cell (32 batch groups)
      pulse         surface heat pulse on the 6 x 6-cell pored film, Eq. 3
                    grid 32 x 64 x 64 at 200 samples, 1e8 particles, FP32"""
    out = {}
    cases = [
        ("slab_fp64", W.gray_slab(n_particles=100_000_000, n_bins=50, precision="fp64"), OPS_SLAB, "fp64"),
        ("slab_fp32", W.gray_slab(n_particles=100_000_000, n_bins=50, precision="fp32"), OPS_SLAB, "alu"),
        ("porous", W.porous_film(n_particles=100_000_000), OPS_POROUS, "alu"),
        ("porous_maps", W.porous_film(n_particles=100_000_000, map=(8, 8), n_batch=32), OPS_POROUS_MAPS, "alu"),
        ("pulse", W.porous_pulse(n_particles=100_000_000), OPS_PULSE_SEG, "alu"),
    ]
    sms = P.le_mc_device_info()[0]
    sm_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    for name, prob, ops_seg, bound in cases:
        mat = P.le_mc_create_material(P.material_desc(prob["material"]))
        geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
        try:
            k_steps = max(1, min(steps, 5))
            step_ms, kern_ms, segs, samples, flags, launches = [], [], 0, 0, 0, 0
            for k in range(warmup + k_steps):
                rd = P.run_desc(prob["source"], W.with_run(prob, seed=prob["run"]["seed"] + 7000 + k)["run"])
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h = P.le_mc_run(mat, geo, rd, stream)
                e1.record(stream)
                t = P.le_mc_read_tallies(h)
                if k >= warmup:
                    step_ms.append(e0.elapsed_time(e1))
                    kern_ms.append(t["kernel_ms"])
                    segs += t["segments"]
                    flags |= t["device_flags"]
                    launches += t["kernel_launches"]
                    if prob["run"].get("n_samples", 0) > 0:
                        g = P.le_mc_read_array(h, "grid")
                        samples += int(np.abs(g.astype(np.int64)).sum())
                P.le_mc_destroy_run(h)
        finally:
            P.le_mc_destroy_geometry(geo)
            P.le_mc_destroy_material(mat)
        per_launch_s = statistics.mean(kern_ms) / 1e3
        seg_launch = segs / k_steps
        smp_launch = samples / k_steps
        ops = seg_launch * ops_seg + smp_launch * (OPS_PULSE_SAMPLE if name == "pulse" else 0)
        entry = {"value": segs / (sum(step_ms) / 1e3), "unit": UNIT, "steps": k_steps, "warmup": warmup,
                 "ms_per_step": statistics.mean(step_ms), "kernel_ms_per_launch": 1e3 * per_launch_s,
                 "segments_per_launch": seg_launch, "particles_per_launch": prob["run"]["n_particles"],
                 "device_flags": flags, "gpu_launches": launches}
        if bound == "fp64":
            # FP64 trajectories: the segment's geometric and transcendental
            # operations run on the FP64 units (Philox stays on the integer
            # units); GB300's nominal dense FP64 rate is 1.25 TFLOP/s, i.e.
            # 6.25e11 operations/s counting a fused multiply-add as one (no
            # measured FP64 peak is available)
            peak = 6.25e11
            fp64_ops = seg_launch * (ops_seg - 40)
            entry["roofline"] = {"bound": "fp64", "achieved": fp64_ops / per_launch_s / 1e12, "peak": peak / 1e12,
                                 "unit": "Tops/s", "frac": fp64_ops / per_launch_s / peak,
                                 "ops_per_segment": ops_seg - 40,
                                 "peak_basis": "nominal GB300 dense FP64, 1.25 TFLOP/s (FMA = 2 flops)"}
        else:
            achieved = ops / per_launch_s
            entry["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                                 "unit": "Tops/s", "frac": achieved / peak_ops, "ops_per_segment": ops_seg,
                                 "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes x {sm_hz / 1e6:.0f} MHz"}
        if name == "pulse":
            entry["sample_updates_per_launch"] = smp_launch
            entry["ops_per_sample_update"] = OPS_PULSE_SAMPLE
            hbm = float(peaks.get("hbm_gbs", 6800.0))
            gbs = smp_launch * BYTES_PULSE_SAMPLE / per_launch_s / 1e9
            entry["grid_reductions"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                        "frac": gbs / hbm, "bytes_per_sample_update": BYTES_PULSE_SAMPLE}
        out[name] = entry
    if "porous" in out and "porous_maps" in out:
        out["porous_maps"]["cost_vs_plain"] = (out["porous_maps"]["kernel_ms_per_launch"] /
                                               out["porous"]["kernel_ms_per_launch"])
    return out


def run_reference(args, problem, rank, world):
    """Reference arm: the FP64 CPU oracle, one bounded sample per step."""
    if rank != 0:
        return
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    probe = W.with_run(problem, n_particles=10_000, precision="fp64")
    t0 = time.perf_counter()
    O.run(probe, n_threads=cores)
    per_particle = max(time.perf_counter() - t0, 1e-4) / 10_000
    budget = 150.0 / max(args.steps + args.warmup, 1)  # whole run within a few minutes
    n = int(min(max(budget / per_particle, 10_000), N_PARTICLES))
    sample = W.with_run(problem, n_particles=n, precision="fp64")
    for _ in range(args.warmup):
        O.run(W.with_run(sample, n_particles=min(n, 10_000)), n_threads=cores)
    segs, elapsed = 0, 0.0
    for k in range(args.steps):
        s = W.with_run(sample, seed=sample["run"]["seed"] + k)
        t0 = time.perf_counter()
        r = O.run(s, n_threads=cores)
        elapsed += time.perf_counter() - t0
        segs += r["segments"]
    value = segs / elapsed
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_particles_per_step": n,
                       "note": "FP64 CPU oracle, bounded sample of the workload per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} particles per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n-particles", type=int, default=N_PARTICLES)
    ap.add_argument("--threads-per-block", type=int, default=0, help="0 = library default")
    ap.add_argument("--refill-min", type=int, default=0, help="0 = library default")
    ap.add_argument("--chunk", type=int, default=0, help="0 = library default")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the gray-slab and pored-film (steady, pulse) measurements")
    ap.add_argument("--served-seconds", type=float, default=60.0,
                    help="length of the request stream of the served form (0 = skip)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    problem = W.silicon_film(n_particles=args.n_particles, precision="fp32")

    if args.impl == "reference":
        run_reference(args, problem, rank, world)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1206_3316_gb300 as P
    prob = rank_problem(problem, rank, world)
    launch = {"threads_per_block": args.threads_per_block, "blocks_per_sm": args.blocks_per_sm,
              "refill_min": args.refill_min, "chunk": args.chunk}
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    mat = P.le_mc_create_material(P.material_desc(prob["material"]))
    geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
    rdesc = P.run_desc(prob["source"], prob["run"], launch)

    def step(seed_offset):
        rdesc.seed = prob["run"]["seed"] + seed_offset
        return P.le_mc_run(mat, geo, rdesc, stream)

    for w in range(args.warmup):
        h = step(10_000 + w)
        P.le_mc_read_tallies(h)
        P.le_mc_destroy_run(h)
    torch.cuda.synchronize(dev)

    # ---- device-timed region: K steps, L2 flushed between steps -----------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    handles = []
    sampler = ClockSampler(local_rank if world > 1 else int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or 0))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with sampler:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            handles.append(step(k))
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    segs, kern_ms, launches, flags, kappas = 0, [], 0, 0, []
    e2e_launches = 0
    for h in handles:
        t = P.le_mc_read_tallies(h)
        segs += t["segments"]
        kern_ms.append(t["kernel_ms"])
        launches += t["kernel_launches"]
        flags |= t["device_flags"]
        kappas.append(t["kappa"])
        P.le_mc_destroy_run(h)
    t_dev = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_dev, dist)
    segs_all = sum_over_ranks(segs, dist)
    value = segs_all / t_max

    # ---- end to end through the C ABI, host descriptors and results -------
    e2e_steps = max(3, min(args.steps, 10))
    n_modes = P.le_mc_material_table(P.material_desc(prob["material"]))[0].size
    # le_mc_create_material uploads per mode: (Lambda, v) in FP32 and FP64
    # and three alias tables (emission, Eq. 2, initial condition) of 8 bytes
    h2d = n_modes * (8 + 16 + 3 * 8)
    # le_mc_read_tallies reads sums, counters, queue head and flags, and the
    # long-first list counts (runs of >= 4096 particles)
    d2h = 2 * 8 + 7 * 8 + 2 * 8 + (3 * 4 if args.n_particles >= 4096 else 0)
    e2e_segs = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        m = P.le_mc_create_material(P.material_desc(prob["material"]))
        g = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
        rd = P.run_desc(prob["source"], W.with_run(prob, seed=prob["run"]["seed"] + 500 + k)["run"], launch)
        h = P.le_mc_run(m, g, rd, stream)
        t = P.le_mc_read_tallies(h)
        e2e_segs += t["segments"]
        e2e_launches += t["kernel_launches"]
        P.le_mc_destroy_run(h)
        P.le_mc_destroy_geometry(g)
        P.le_mc_destroy_material(m)
    torch.cuda.synchronize(dev)
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_value = sum_over_ranks(e2e_segs, dist) / e2e_t

    P.le_mc_destroy_geometry(geo)
    P.le_mc_destroy_material(mat)

    peaks, peak_src = _peaks()
    sms, name = P.le_mc_device_info()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sms * LANES_PER_SM * sm_mhz * 1e6
    configs = None
    if not args.no_configs and rank == 0:
        configs = config_measurements(P, torch, dev, stream, flush, args.steps, max(3, args.warmup), peak_ops, peaks)

    if rank != 0:
        dist.destroy_process_group()
        return

    clocks = sampler.summary()
    per_launch_s = statistics.mean(kern_ms) / 1e3
    segs_per_launch = segs / args.steps
    achieved = segs_per_launch * OPS_PER_SEGMENT / per_launch_s
    traffic = _profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_particles": args.n_particles, "form": "plain",
                   "tallies": "per-particle FP32 sums, FP64 accumulation",
                   "l2": "flushed between steps (256 MiB write)",
                   "launch": {"threads_per_block": args.threads_per_block or 512,
                              "blocks_per_sm": args.blocks_per_sm or "occupancy",
                              "refill_min": args.refill_min or 4, "chunk": args.chunk or 256},
                   "kappa_W_per_mK": statistics.mean(kappas), "device": name, "sms": sms,
                   "wall_s_timed_region": wall},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "gpu_launches": e2e_launches},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "trace_kernel_r80<float, PLANES, GRADIENT, all-diffuse>",
                     "ops_per_segment": OPS_PER_SEGMENT,
                     "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz ({peak_src} sm_max_mhz)"},
        "clocks": clocks,
        "device_flags": flags,
    }
    if configs is not None:
        line["configs"] = configs
    if not args.no_batched:
        line["batched"] = batched_measurement(P, torch, dev, stream, args.steps, launch)
        # whole-launch rate (the dominant kernel is the same trace kernel)
        line["batched"]["roofline_frac"] = line["batched"]["value"] * OPS_PER_SEGMENT / peak_ops
    if args.served_seconds > 0:
        line["served"] = served_measurement(P, args.served_seconds)
        # arrival-limited: the stream offers far less work than the GPU can trace
        line["served"]["roofline_frac"] = line["served"]["aggregate_segments_per_s"] * OPS_PER_SEGMENT / peak_ops
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(problem)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
