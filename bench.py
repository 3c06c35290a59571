"""Benchmark of the near-field step on the clustered 512^3 workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step is one pass of the whole hot path over the box: the pair kernel
(nf_forces: work queue, source staging, pair sum, compensated accumulation)
then the FP64 kick-drift with re-binning (nf_kick_drift: kick, drift, stable
radix sort by cell, cell table, work-queue plan).  The metric is near-field
pair interactions per second (one ordered sink-source evaluation per pair,
self pairs included); particles per second per step is reported beside it.
Inputs are resident in HBM when the timed region starts and are larger than
L2 (2.1 GB of positions).  The plain FP32 kernel is timed on the same
positions for comparison, and both are checked against the FP64 oracle on
sampled sinks.

`--impl reference` times the FP64 CPU oracle (the reference of this build) on
the same workload: each step evaluates a bounded sample of sinks.

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (weak scaling; the near-field of one box needs no exchange here);
only the timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "zeldovich512"
METRIC = "near-field Gpair-interactions/s and particles/s/step at 512^3 clustered vs plain FP32 kernel"
UNIT = "Gpair/s"
# FP32 FMA-pipe lane operations per pair at r >= eps (3 sub, 3 for r^2, 4 for the Newton-refined r^-3 in the
# accumulators' scale: y^2, r^2 y^2 - A, y^3, their product; 3 accumulate): the least the law needs for a pair
# outside the softening length, i.e. nearly every pair, and what the kernel executes for such a pair
FMA_OPS_PER_PAIR = 13
PREVIOUS_OPS_PER_PAIR = 14   # the same with the Newton factor 1 + 3e formed on its own (2 ops instead of 1)
BRANCH_FREE_OPS_PER_PAIR = 18   # the same with the law evaluated branch-free, min(r^-3, g(r)), for every pair
ISSUE_OPS_PER_PAIR = 20    # FP32-pipe instructions per pair of the branch-free law issued one lane-op at a time
# DRAM bytes (read + write) of one compensated pair-kernel launch of this workload: the mean of the
# launches inside the bench's steps in the ncu launch list of this workload, valid while nf_pair.cu's code
# (comments removed) hashes to the value below (the record reports null traffic once the code has changed)
PAIR_TRAFFIC_BYTES = 1.18050e10
PAIR_TRAFFIC_SOURCE_SHA256 = "44afd19ae9bd14a9"
FP32_LANES_PER_SM = 128


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"sm_max_mhz": 2032.0}, "fallback"


def _make_workload(name):
    from synth import workload
    return workload(name)


def _oracle_sample(w, b, k, seed):
    """Oracle FP64 forces on k sampled sinks: (acc, sumabs, pairs, seconds, sinks)."""
    import oracle
    rng = np.random.default_rng(seed)
    sinks = np.sort(rng.choice(b.n, k, replace=False)).astype(np.int64)
    t = time.perf_counter()
    acc, sa, pairs = oracle.forces(b, w.eps, sinks, with_sumabs=True)
    return acc, sa, pairs, time.perf_counter() - t, sinks


def _sized_sample(w, b, target_s, seed):
    """A sink count whose oracle pass takes about target_s seconds on this host."""
    k = min(b.n, 20000)
    _, _, _, t, _ = _oracle_sample(w, b, k, seed)
    if t < 0.5 * target_s:
        k = int(min(b.n, k * target_s / max(t, 1e-3)))
    return k


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (bounded sample of sinks per step)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    w = _make_workload(WORKLOAD)
    b = oracle.bin_positions(w.pos, w.cpd, w.box)
    k = args.ref_sinks or _sized_sample(w, b, args.ref_seconds, seed=99)
    times, pairs = [], []
    for s in range(args.warmup + args.steps):
        _, _, p, dt, _ = _oracle_sample(w, b, k, seed=100 + s)
        if s >= args.warmup:
            times.append(dt)
            pairs.append(p)
    value = sum(pairs) / sum(times) / 1e9
    cores = os.cpu_count()
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * sum(times) / len(times), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic (seeded Zel'dovich lattice + Plummer halos)", impl="reference",
                config=dict(workload=f"{WORKLOAD}: N=512^3, CPD=405, R=2, eps=1/50 spacing", sinks_per_step=k),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"{k} uniformly sampled sinks per step, all their near-field pairs"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """Largest value of x over all ranks of the default process group (timing only)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(pairs_per_replica: int, world: int, step_ms: float) -> float:
    """Gpair/s of the whole job: every rank evaluates its own replica in step_ms (the slowest rank's time)."""
    return world * pairs_per_replica / (step_ms * 1e-3) / 1e9


def pair_source_code_hash() -> str:
    """sha256 prefix of nf_pair.cu with its comments and blank lines removed: comment edits keep it."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1810_02916_b300", "csrc", "nf_pair.cu")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()[:16]


def _pair_traffic():
    return PAIR_TRAFFIC_BYTES if pair_source_code_hash() == PAIR_TRAFFIC_SOURCE_SHA256 else None


def _launches_per_step(cpd):
    """Kernels the library launches per step (counted from the code; the ncu launch list agrees).

    forces: pair kernel + partial reduction = 2.
    kick-drift: kick-drift, sort keys and cell counts (2); radix sort, per 8-bit pass a histogram,
    three scan kernels and a scatter (5 x passes); gather (1); cell-start scan (3); plan:
    neighbourhood sizes (occupancy, three window sums, pair total: 5), counter reset (1),
    5 occupancy classes x (count, three scan kernels, emit, advance) (30), lane items (count,
    three scan kernels, emit, advance: 6), source split (count, three scans of three kernels,
    expand: 11), heavy-before-light partition (flags, three scan kernels, scatter: 5).
    """
    ncell = cpd ** 3
    bits = max(1, (ncell - 1).bit_length())
    passes = (bits + 7) // 8
    plan = 5 + 1 + 5 * 6 + 6 + 11 + 5
    kick_drift = 2 + 5 * passes + 1 + 3 + plan
    return 2 + kick_drift


def run(args):
    import torch
    import paper_1810_02916_b300 as nfb

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.Stream()

    w = _make_workload(WORKLOAD)
    nf = nfb.NearField(w.cpd, w.eps, w.box)
    nf.set_stream(stream)
    Xd = torch.from_numpy(w.pos).to(f"cuda:{dev}")
    nf.bin_particles(Xd)
    del Xd
    n = nf.n
    acc_d = torch.empty((n, 4), dtype=torch.float32, device=f"cuda:{dev}")
    # the autotuner picks the sink tiling, split floor and launch shape on the initial state
    # (outside the timed region); the comparison boxes below use the same choice
    tune_s, tune_report = 0.0, "not run (--no-tune)"
    if not args.no_tune:
        t0 = time.perf_counter()
        tune_report = nf.tune()
        tune_s = time.perf_counter() - t0
    tuning = nf.tuning()

    def apply_tuning(box):
        box.set_shape(tuning["warps"], tuning["stage"])
        box.set_tiling(tuning["c4"], tuning["c2"], tuning["c1"], tuning["split_floor"])

    # time step: max|a| dt^2 <= 0.1 eps (so max |v| dt stays far below 0.8 cells)
    with torch.cuda.stream(stream):
        nf.forces(acc_d)
    torch.cuda.synchronize()
    amax = float(acc_d[:, :3].abs().max())
    dt = (0.1 * w.eps / amax) ** 0.5

    def step():
        nf.forces(False)
        nf.kick_drift(dt)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(dev)
    clocks.start()
    nf.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # pairs of each timed step: the count of the plan its force pass runs (read after the
    # previous kick-drift, which has synchronised already; an 8-byte copy)
    step_pairs = [nf.pair_count()]
    e0.record(stream)
    for k in range(args.steps):
        step()
        if k + 1 < args.steps:
            step_pairs.append(nf.pair_count())
    e1.record(stream)
    torch.cuda.synchronize()
    nf.profile(False)
    step_ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    launches, pair_ms = nf.profile_read()
    pair_ms /= max(launches, 1)
    pairs = sum(step_pairs) / len(step_pairs)      # mean pairs per timed step
    t_max = max_over_ranks(step_ms, f"cuda:{dev}") if world > 1 else step_ms
    value = whole_job_rate(pairs, world, t_max)
    pair_kernel_gps = pairs / (pair_ms * 1e-3) / 1e9

    # plain FP32 kernel on the same positions, and accuracy of both on sampled sinks
    import oracle
    extra = {}
    if rank == 0:
        b = oracle.bin_positions(w.pos, w.cpd, w.box)   # layout of the current state differs after steps:
        nf_cmp = nfb.NearField(w.cpd, w.eps, w.box)      # compare on a fresh box of the initial positions
        nf_cmp.set_stream(stream)
        nf_cmp.bin_particles(torch.from_numpy(w.pos).to(f"cuda:{dev}"))
        apply_tuning(nf_cmp)
        pairs0 = nf_cmp.pair_count()
        acc_c = nf_cmp.forces()
        nf_cmp.set_accumulation(nfb.ACC_PLAIN)
        nf_cmp.profile(True)
        for _ in range(3):
            nf_cmp.forces(acc_d)
        k, ms = nf_cmp.profile_read()
        acc_p = nf_cmp.forces()
        nf_cmp.close()
        ref, sa, _, _, sinks = _oracle_sample(w, b, 20000, seed=7)
        ec = oracle.error_stats(acc_c[sinks, :3], ref, sa)
        ep = oracle.error_stats(acc_p[sinks, :3], ref, sa)
        kc = args.cpu_sinks or _sized_sample(w, b, args.cpu_seconds, seed=8)
        _, _, sampled_pairs, cpu_s, _ = _oracle_sample(w, b, kc, seed=9)
        extra = dict(
            compensated=dict(pair_kernel_gpair_s=pair_kernel_gps, error_vs_oracle=ec),
            plain_fp32=dict(pair_kernel_gpair_s=pairs0 / (ms / k * 1e-3) / 1e9, error_vs_oracle=ep,
                            note="initial positions of the workload, before any step"),
            cpu_baseline=dict(value=sampled_pairs / cpu_s / 1e9, unit=UNIT, cores=os.cpu_count(), kind="oracle",
                              sample=f"{kc} uniformly sampled sinks of the workload "
                                     f"({sampled_pairs} pairs, {cpu_s:.1f} s)"),
        )

    # end to end through the C ABI with pinned host buffers: positions in, accelerations out
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        xh = torch.from_numpy(w.pos).pin_memory()
        ah = torch.empty((n, 4), dtype=torch.float32).pin_memory()
        nf_e = nfb.NearField(w.cpd, w.eps, w.box)
        nf_e.set_stream(stream)
        apply_tuning(nf_e)

        def e2e_step():
            nf_e.bin_particles(xh)
            nf_e.forces(ah)
            nf_e.kick_drift(dt)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e_s = (time.perf_counter() - t0) / args.e2e_steps
        nf_e.close()
        e2e = dict(value=pairs0 / e_s / 1e9, unit=UNIT, h2d_bytes_per_step=int(xh.numel() * 8),
                   d2h_bytes_per_step=int(ah.numel() * 4),
                   step="nf_bin_particles(pinned host xyz) + nf_forces(pinned host acc) + nf_kick_drift")

    # secondary: the 64-box batched configuration on this GPU (one persistent launch under a CUDA graph)
    if rank == 0 and world == 1 and args.batched_steps > 0:
        specs = _batched_specs()
        extra["batched"] = _time_batched(specs, list(range(len(specs))), args.batched_steps, 2)

    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_gps = props.multi_processor_count * sm_max * 1e6 * FP32_LANES_PER_SM / FMA_OPS_PER_PAIR / 1e9
    peak14_gps = props.multi_processor_count * sm_max * 1e6 * FP32_LANES_PER_SM / PREVIOUS_OPS_PER_PAIR / 1e9
    issue_peak_gps = props.multi_processor_count * sm_max * 1e6 * FP32_LANES_PER_SM / ISSUE_OPS_PER_PAIR / 1e9
    branch_free_peak_gps = (props.multi_processor_count * sm_max * 1e6 * FP32_LANES_PER_SM /
                            BRANCH_FREE_OPS_PER_PAIR / 1e9)
    if rank == 0:
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=t_max, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
            data="synthetic (seeded Zel'dovich lattice + Plummer halos)",
            config=dict(workload=f"{WORKLOAD}: N=512^3=134217728, CPD=405, R=2, eps=1/50 spacing, "
                                 "Zel'dovich P(k)~k^-1.5 + 2000 Plummer halos",
                        pairs_per_step=pairs, pairs_per_step_note=f"mean over the {args.steps} timed steps, each "
                        "the count of the plan its force pass ran", particles=n, dt=dt,
                        parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                        tuning=dict(tuning, tuner_seconds=round(tune_s, 1),
                                    tuner="nf_tune on the initial state: " + tune_report.split("->")[-1].strip()),
                        l2="inputs larger than L2 (2.1 GB positions, 3.2 GB FP64 sums)"),
            particles_per_s_per_step=world * n / (t_max * 1e-3),
            gpu_launches=_launches_per_step(w.cpd) * args.steps,
            roofline=dict(bound="alu", achieved=pair_kernel_gps, peak=peak_gps, unit=UNIT,
                          frac=pair_kernel_gps / peak_gps, traffic=_pair_traffic(),
                          traffic_note="DRAM read+write bytes of one pair-kernel launch (ncu, same workload); "
                                       "algorithmic bytes: positions 2.15 GB read + FP64 sums 3.22 GB written",
                          frac_14_ops=pair_kernel_gps / peak14_gps,
                          branch_free_frac=pair_kernel_gps / branch_free_peak_gps,
                          issue_convention_frac=pair_kernel_gps / issue_peak_gps,
                          paper_convention_frac=pair_kernel_gps * 23 /
                          (props.multi_processor_count * sm_max * 1e-3 * FP32_LANES_PER_SM * 2),
                          peak_basis=f"FP32 FMA-lane roofline: {props.multi_processor_count} SMs x {sm_max:.0f} MHz "
                                     f"({src}) x 128 lanes / {FMA_OPS_PER_PAIR} FMA-pipe ops per pair (Newtonian "
                                     "pair, one Newton step); frac_14_ops: the same over "
                                     f"{PREVIOUS_OPS_PER_PAIR} ops (the Newton factor formed on its own); "
                                     "branch_free_frac: the same over "
                                     f"{BRANCH_FREE_OPS_PER_PAIR} ops (min(r^-3, g) for every pair); "
                                     f"issue_convention_frac: over {ISSUE_OPS_PER_PAIR} single-lane instructions per "
                                     "pair of the branch-free law; paper_convention_frac: 23 FLOP per pair against "
                                     "the FMA peak (2 FLOP per lane per cycle)"),
            clocks=clk, e2e=e2e, **extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_forces_only(args):
    """Profiling driver: bin one workload, then `--forces-only` force passes (no bench line)."""
    import torch
    import paper_1810_02916_b300 as nfb
    w = _make_workload(args.workload)
    nf = nfb.NearField(w.cpd, w.eps, w.box)
    if args.plain:
        nf.set_accumulation(nfb.ACC_PLAIN)
    nf.bin_particles(torch.from_numpy(w.pos).cuda())
    acc = torch.empty((nf.n, 4), dtype=torch.float32, device="cuda")
    nf.forces(acc)                      # untimed first pass (one-time kernel set-up)
    nf.profile(2 if args.class_profile else True)
    for _ in range(args.forces_only):
        nf.forces(acc)
    k, ms = nf.profile_read()
    pairs = nf.pair_count()
    out = dict(workload=args.workload, launches=k, ms_per_launch=ms / max(k, 1), pairs=pairs,
               gpair_s=pairs / (ms / max(k, 1) * 1e-3) / 1e9)
    if args.class_profile:
        peaks, _ = _peaks()
        out["classes"] = class_table(nf.profile_classes(), pairs * k, k, float(peaks.get("sm_max_mhz", 2032.0)))
    print(json.dumps(out), flush=True)
    return 0


def class_table(raw, pairs_total, launches, sm_mhz, warps_per_sm=24):
    """Per-item-class breakdown of the pair kernel (profile mode 2).

    busy_share: the class's share of the warps' summed busy cycles.  eff: pairs per warp-cycle
    against the FMA-lane bound shared by the resident warps (128 lanes / 13 ops per pair per SM
    cycle over warps_per_sm warps), i.e. how close the class runs to the roofline while it runs.
    Lane items' pairs are the pass's total minus the tiled items' pairs.  busy_over_lifetime: busy
    cycles over the warps' lifetimes (time spent taking items from the queue is the rest);
    lifetime_over_wall: a warp's mean lifetime over one launch's wall time (the idle tail is the rest)."""
    per_warp_bound = FP32_LANES_PER_SM / FMA_OPS_PER_PAIR / warps_per_sm
    classes = {k: v for k, v in raw.items() if isinstance(v, tuple)}
    tiled_pairs = sum(v[2] for k, v in classes.items() if not k.startswith("lane"))
    busy = sum(v[0] for v in classes.values()) or 1
    rows = {}
    for name, (cyc, items, pr) in classes.items():
        if name == "lane items":
            pr = pairs_total - tiled_pairs
        if items == 0:
            continue
        rows[name] = dict(items=items // launches, pairs=pr // launches, busy_share=cyc / busy,
                          pair_share=pr / max(pairs_total, 1),
                          eff=(pr / cyc / per_warp_bound) if cyc else None)
    life = raw["warp_lifetime_cycles"]
    return dict(rows=rows, busy_over_lifetime=busy / max(life, 1), warps=raw["warps"] // launches,
                wall_ms_per_launch=raw["wall_ns"] / 1e6 / launches,
                lifetime_over_wall=life / max(raw["warps"], 1) / (raw["wall_ns"] / launches * 1e-3 * sm_mhz)
                if raw["wall_ns"] else None)


BATCHED_BOXES = 64


def _batched_specs():
    """The batched workload: 64 independent unit boxes, N log-uniform in [32^3, 128^3] (seeded)."""
    from synth import generators as gen
    return gen.batched_boxes(BATCHED_BOXES, gen.rng_for(3))


def shard_boxes(n_boxes: int, rank: int, world: int) -> list[int]:
    """Boxes of one rank: rank, rank + world, rank + 2 world, ...  The boxes are independent, so
    ranks exchange nothing but the timing and the pair totals."""
    return list(range(rank, n_boxes, world))


def batched_job(pairs_local: int, ms_local: float, world: int) -> tuple[int, float, float]:
    """Whole-job (pairs, ms, Gpair/s) of a sharded batch: pairs summed over ranks, the slowest rank's time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(pairs_local)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        pairs = int(round(float(t.item())))
        ms = max_over_ranks(ms_local)
    else:
        pairs, ms = int(pairs_local), float(ms_local)
    return pairs, ms, pairs / (ms * 1e-3) / 1e9


def _time_batched(specs, idx, steps, warmup):
    """Boxes specs[idx] in one persistent launch replayed from a CUDA graph, against one nf_forces
    launch per box on the same boxes (CUDA events on the boxes' stream)."""
    import torch
    import paper_1810_02916_b300 as nfb
    stream = torch.cuda.Stream()
    boxes, outs = [], []
    for i in idx:
        sp = specs[i]
        b = nfb.NearField(sp.cpd, sp.eps)
        b.set_stream(stream)
        b.bin_particles(torch.from_numpy(sp.pos).cuda())
        boxes.append(b)
        outs.append(torch.empty((b.n, 4), dtype=torch.float32, device="cuda"))
    pairs = sum(b.pair_count() for b in boxes)
    n = sum(b.n for b in boxes)
    out = dict(boxes=len(boxes), particles=n, pairs=pairs, steps=steps)
    if not boxes:
        out.update(graph_ms=0.0, per_box_ms=0.0)
        return out
    with torch.cuda.stream(stream):
        nfb.forces_batched(boxes, outs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        nfb.forces_batched(boxes, outs)
    for _ in range(warmup):
        g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / steps
    # one launch per box, same stream
    for b, o in zip(boxes, outs):
        b.forces(o)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for b, o in zip(boxes, outs):
            b.forces(o)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1) / steps
    for b in boxes:
        b.close()
    out.update(graph_ms=ms_graph, graph_gpair_s=pairs / (ms_graph * 1e-3) / 1e9,
               per_box_ms=ms_single, per_box_gpair_s=pairs / (ms_single * 1e-3) / 1e9,
               what="one persistent launch over all boxes replayed from a CUDA graph (graph_*) vs one "
                    "nf_forces launch per box (per_box_*)")
    return out


def run_batched(args):
    """The batched configuration: 64 independent boxes in one persistent launch replayed from a CUDA
    graph.  Under torchrun each rank takes its share of the boxes (shard_boxes) on its own GPU; every
    rank prints its own line and rank 0 the whole job's (pairs summed, slowest rank's time)."""
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")       # only host scalars are reduced
    torch.cuda.set_device(local)
    specs = _batched_specs()
    idx = shard_boxes(len(specs), rank, world)
    r = _time_batched(specs, idx, args.steps, args.warmup)
    print(json.dumps(dict(mode="batched", rank=rank, world=world, boxes_of_rank=idx, **r)), flush=True)
    pairs, ms, gps = batched_job(r["pairs"], r["graph_ms"], world)
    if rank == 0:
        print(json.dumps(dict(mode="batched", n_gpus=world, boxes=len(specs), pairs=pairs, ms=ms, gpair_s=gps,
                              unit=UNIT, scaling="strong", parallelism=f"boxes sharded over {world} rank(s), "
                              "no data exchange")), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_adjoint(args):
    """Secondary measurement: forward forces and the adjoint (VJP) kernel on the 64^3 clustered box."""
    import torch
    import paper_1810_02916_b300 as nfb
    from synth import generators as gen
    w = _make_workload("clustered64")
    nf = nfb.NearField(w.cpd, w.eps, w.box)
    nf.bin_particles(torch.from_numpy(w.pos).cuda())
    W = torch.zeros((nf.n, 4), device="cuda")
    W[:, :3] = torch.from_numpy(gen.cotangent(nf.n, gen.rng_for(5))).float().cuda()
    acc = torch.empty_like(W)
    grad = torch.empty_like(W)
    pairs = nf.pair_count()
    out = dict(mode="adjoint", workload="clustered64", particles=nf.n, pairs=pairs)
    for name, fn in (("forces", lambda: nf.forces(acc)), ("vjp", lambda: nf.vjp(W, grad))):
        for _ in range(args.warmup):
            fn()
        nf.profile(True)
        for _ in range(args.steps):
            fn()
        k, ms = nf.profile_read()
        nf.profile(False)
        out[name] = dict(ms=ms / k, gpair_s=pairs / (ms / k * 1e-3) / 1e9)
    print(json.dumps(out), flush=True)
    return 0


def run_cutoff(args):
    """Secondary measurement: the cut-off mode (dense far cells through sub-cell quadrupoles) on the 512^3
    workload against the exact pass, with both compared to the FP64 oracles on sampled sinks."""
    import torch
    import oracle
    import paper_1810_02916_b300 as nfb
    w = _make_workload(WORKLOAD)
    nf = nfb.NearField(w.cpd, w.eps, w.box)
    nf.bin_particles(torch.from_numpy(w.pos).cuda())
    acc = torch.empty((nf.n, 4), device="cuda")
    exact_pairs = nf.pair_count()
    out = dict(mode="cutoff", workload=WORKLOAD, particles=nf.n, exact_pairs=exact_pairs, n_min=args.cutoff)
    results = {}
    for name, n_min in (("exact", 0), ("cutoff", args.cutoff)):
        nf.set_cutoff(n_min)
        for _ in range(args.warmup):
            nf.forces(acc)
        nf.profile(True)
        for _ in range(args.steps):
            nf.forces(acc)
        k, ms = nf.profile_read()
        nf.profile(False)
        results[name] = acc[:, :3].cpu().numpy().astype(np.float64)
        out[name] = dict(ms=ms / k, exact_pairs_per_s=exact_pairs / (ms / k * 1e-3) / 1e9,
                         direct_pairs=nf.pair_count())
    out["speedup"] = out["exact"]["ms"] / out["cutoff"]["ms"]
    b = oracle.bin_positions(w.pos, w.cpd, w.box)
    rng = np.random.default_rng(11)
    sinks = np.sort(rng.choice(b.n, 4000, replace=False)).astype(np.int64)
    ex = oracle.forces(b, w.eps, sinks)
    cu = oracle.cutoff(b, w.eps, args.cutoff, sinks)
    out["cutoff"]["error_vs_cutoff_oracle"] = oracle.error_stats(results["cutoff"][sinks], cu)
    out["cutoff"]["error_vs_exact_oracle"] = oracle.error_stats(results["cutoff"][sinks], ex)
    out["cutoff_oracle_vs_exact_oracle"] = oracle.error_stats(cu, ex)
    out["exact"]["error_vs_exact_oracle"] = oracle.error_stats(results["exact"][sinks], ex)
    out["unit"] = "Gpair/s (exact pairs / time)"
    nf.close()
    print(json.dumps(out), flush=True)
    return 0


def run_multipoles(args):
    """Secondary measurement: order-8 Cartesian multipoles of every cell of the 256^3 clustered box."""
    import torch
    import paper_1810_02916_b300 as nfb
    w = _make_workload("clustered256")
    nf = nfb.NearField(w.cpd, w.eps, w.box)
    nf.bin_particles(torch.from_numpy(w.pos).cuda())
    T = 165
    out = torch.empty((nf.ncell, T), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        nf.multipoles(8, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        nf.multipoles(8, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps(dict(mode="multipoles", workload="clustered256", order=8, cells=nf.ncell, particles=nf.n,
                          ms=ms, mparticles_s=nf.n / (ms * 1e-3) / 1e6,
                          out_gb=nf.ncell * T * 8 / 1e9)), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default tiling and shape)")
    ap.add_argument("--batched-steps", type=int, default=5,
                    help="graph replays of the 64-box batch reported beside the bench line (0: skip)")
    ap.add_argument("--cpu-sinks", type=int, default=0, help="0: size the sample to --cpu-seconds")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-sinks", type=int, default=0, help="0: size the sample to --ref-seconds")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default=WORKLOAD, help="profiling driver only (with --forces-only)")
    ap.add_argument("--forces-only", type=int, default=0, help="profiling driver: this many force passes")
    ap.add_argument("--cutoff", type=int, default=1024, help="--mode cutoff: n_min of the dense far cells")
    ap.add_argument("--plain", action="store_true", help="profiling driver: plain FP32 accumulation")
    ap.add_argument("--class-profile", action="store_true",
                    help="profiling driver: per-item-class clock sums of the pair kernel")
    ap.add_argument("--mode", default="step", choices=["step", "batched", "adjoint", "multipoles", "cutoff"],
                    help="batched / adjoint: secondary measurements (not the bench line)")
    args = ap.parse_args()
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "adjoint":
        return run_adjoint(args)
    if args.mode == "multipoles":
        return run_multipoles(args)
    if args.mode == "cutoff":
        return run_cutoff(args)
    if args.forces_only:
        return run_forces_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
