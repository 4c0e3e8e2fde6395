"""Throughput benchmark of the hot path on synthetic inputs shaped like the
paper's workloads.  Prints one JSON line (rank 0).

Workloads (``--workload``):
  training_step   (default) full-atom training step, 256 chains x 700 residues,
                  uniform residue types: full-atom forward -> LRMSD forward (to
                  structures built from N(0, 0.1 rad)-perturbed angles) -> LRMSD
                  backward -> full-atom backward.  Unit: residues/s.
  backbone_uneven backbone step over 4096 chains of log-uniform lengths in
                  [50, 1000]: backbone forward -> LRMSD -> backbone backward.
                  Unit: residues/s.
  lrmsd_batch     16384 coordinate-set pairs of U{100..5000} atoms: LRMSD
                  forward + backward.  Unit: atoms/s (atoms of the input side).
  fullatom_short  the training step on 4096 full-atom chains of log-uniform
                  lengths in [16, 128] (short chains: packed several per CTA when
                  the autotuner picks the packed schedule).  Unit: residues/s.
  mixed_batch     the training step on 256 chains x 700 residues where every
                  other chain is backbone-only (residue code 20: N, CA, C), both
                  models in the same persistent launches.  Unit: residues/s.
  length_sweep    scan forward and backward against the paper's O(L^2)
                  backward forms, both models, 32 chains of L = 64 .. 4096.
  backbone_stress precision stress, 64 backbone chains x 10000 residues, the
                  same step as backbone_uneven; reports the coordinate drift and
                  gradient error against the FP64 per-chain form.

The default run (training_step) also times backbone_uneven and lrmsd_batch
with the same protocol and reports them under "workloads" (``--no-extra``
skips them).

``--impl reference`` times the FP64 CPU oracle, as it stands, on a bounded
sample of the same workload instead.

Timing: W warm-up steps, then K timed steps; a step (all its C-ABI calls) is
one CUDA graph replayed between CUDA events on the launching stream, and L2 is
flushed (a 512 MiB write, outside the events) before every step.  Per-call
times (breakdown, roofline) come from a second graph of the same calls with
event-record nodes between them.  Under
torchrun each rank runs its own batch (weak scaling, no data-path collective);
the elapsed time is the max over ranks.
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

METRIC = "residues/s fwd+bwd at FP32 err≤2e-3 Å vs plain FP64 GPU form; HBM roofline %"
METRIC_LRMSD = "atoms/s LRMSD fwd+bwd vs plain FP64 GPU form; HBM roofline %"

DEFAULT_BATCH = {"training_step": 256, "backbone_uneven": 4096, "lrmsd_batch": 16384,
                 "backbone_stress": 64, "length_sweep": 32, "mixed_batch": 256, "fullatom_short": 4096}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a C-ABI
# call's kernels from one ncu capture, per unit processed (residue or atom),
# keyed by (workload, call), with the profile summary that holds the capture.
# An entry is removed when one of its kernels changes after the capture.
TRAFFIC = {
    # (workload, call) -> entries (per-unit DRAM bytes, unit, profile, launch shape of the
    # capture or None if the kernels take none); cold-cache captures of one launch.  The
    # entry whose shape matches the step's launch shape is used.
    # Full-atom kernels captured at 4096 chains x 700 residues (coordinates above L2),
    # scaled by residues processed.
    ("training_step", "fullatom_forward"): [
        (320464128 / 2867200, "residue", "profiles/fa_kernels_training_step_256x700.md",
         "threads=384,res_per_thread=1"),
        (321153024 / 2867200, "residue", "profiles/fa_kernels_training_step_256x700.md",
         "threads=256,res_per_thread=1")],
    ("training_step", "lrmsd_fullatom_backward"): [
        (661773312 / 2867200, "residue", "profiles/fa_kernels_training_step_256x700.md",
         "threads=384,res_per_thread=1"),
        (662446848 / 2867200, "residue", "profiles/fa_kernels_training_step_256x700.md",
         "threads=256,res_per_thread=1")],
    # the uneven backbone batch itself (1302424 residues), shape 256 x 4
    ("backbone_uneven", "backbone_forward"): [
        (19462656 / 1302424, "residue", "profiles/backbone_kernels_backbone_uneven_4096.md",
         "threads=256,res_per_thread=4")],
    ("backbone_uneven", "lrmsd_backbone_backward"): [
        (101150976 / 1302424, "residue", "profiles/backbone_kernels_backbone_uneven_4096.md",
         "threads=256,res_per_thread=4")],
    # LRMSD kernels captured on 4096 pairs (10499521 atoms), scaled by atoms
    ("lrmsd_batch", "lrmsd_forward"): [
        (273839872 / 10499521, "atom", "profiles/lrmsd_kernels_lrmsd_batch_4096.md", None)],
    ("lrmsd_batch", "lrmsd_backward"): [
        (449672960 / 10499521, "atom", "profiles/lrmsd_kernels_lrmsd_batch_4096.md", None)],
}


# --schedule: TPL_SCHED_* of the chain calls
SCHEDULES = {"auto": 0, "longest": 1, "batch": 2, "packed": 3}

# launch shapes of the backbone training-step kernel
STEP_SHAPES = [(128, 4), (256, 4), (256, 2), (128, 2), (512, 2)]


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="tpl", choices=["tpl", "reference"])
    p.add_argument("--workload", default="training_step", choices=sorted(DEFAULT_BATCH))
    p.add_argument("--batch", type=int, default=0, help="chains (or pairs) per GPU; 0 = workload default")
    p.add_argument("--length", type=int, default=700, help="residues per chain (training_step)")
    p.add_argument("--threads", type=int, default=0, help="CTA size of the chain kernels (0 = default)")
    p.add_argument("--res-per-thread", type=int, default=0, help="residues per thread (0 = default)")
    p.add_argument("--bwd", default="coords", choices=["coords", "recompute", "quadratic"],
                   help="chain backward: read the forward's coordinates, rebuild frames, or (backbone) "
                        "the paper's O(L^2) sums from the coordinates")
    p.add_argument("--fusion", default="backward", choices=["step", "backward", "none"],
                   help="training step: fused step (full atom: two calls; backbone: one call), fused backward (three calls), "
                        "or separate calls (four)")
    p.add_argument("--unfused", action="store_true", help="same as --fusion none")
    p.add_argument("--no-autotune", action="store_true",
                   help="use the library's default launch shape instead of the autotuner's pick")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 per-chain comparison")
    p.add_argument("--schedule", default="auto", choices=sorted(SCHEDULES),
                   help="work-list schedule of the chain calls (anything but auto skips the autotuner)")
    p.add_argument("--write-padding", action="store_true",
                   help="chain calls write their outputs' padding every call (default: the bench "
                        "zeroes the output buffers once and passes TPL_FLAG_PADDING_ZEROED)")
    p.add_argument("--no-extra", action="store_true",
                   help="training step only: skip the uneven backbone and LRMSD batch workloads")
    a = p.parse_args(argv)
    if a.batch <= 0:
        a.batch = DEFAULT_BATCH[a.workload]
    if a.unfused:
        a.fusion = "none"
    if a.bwd == "quadratic" and a.workload not in ("backbone_uneven", "backbone_stress"):
        p.error("--bwd quadratic is the backbone comparator (backbone workloads only)")
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device, world):
    """The largest value of x over all ranks (the job's elapsed time).  The
    replicas exchange nothing else: there is no data-path collective."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, world, steps, max_ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank has a batch of its own)."""
    return units_per_rank_step * world * steps / (max_ms * 1e-3)


# ----------------------------------------------------------------------------- host inputs
def make_inputs(args, rank):
    """Seeded host arrays of the workload (one batch per rank)."""
    import workloads

    if args.workload == "fullatom_short":
        rng = workloads.rng_for(7, salt=rank)
        lengths = workloads.lengths_loguniform(args.batch, 16, 128, rng)
        a, seq = workloads.fullatom_inputs(lengths, rng, Lmax=128)
        ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
        return {"angles": a, "seq": seq, "lengths": lengths, "target_angles": ta}
    if args.workload in ("training_step", "mixed_batch"):
        rng = workloads.rng_for(4, salt=rank)
        lengths = np.full(args.batch, args.length, np.int32)
        a, seq = workloads.fullatom_inputs(lengths, rng)
        if args.workload == "mixed_batch":
            seq[1::2] = workloads.BACKBONE_ONLY  # every other chain: the backbone model
        ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
        return {"angles": a, "seq": seq, "lengths": lengths, "target_angles": ta}
    if args.workload == "backbone_uneven":
        rng = workloads.rng_for(2, salt=rank)
        lengths = workloads.lengths_loguniform(args.batch, 50, 1000, rng)
        a = workloads.backbone_angles(lengths, rng, Lmax=workloads.pad_to(1000))
        ta = workloads.perturb_angles(a, lengths, rng)
        return {"angles": a, "lengths": lengths, "target_angles": ta}
    if args.workload == "backbone_stress":
        rng = workloads.rng_for(5, salt=rank)
        lengths = np.full(args.batch, 10000, np.int32)
        a = workloads.backbone_angles(lengths, rng)
        ta = workloads.perturb_angles(a, lengths, rng)
        return {"angles": a, "lengths": lengths, "target_angles": ta}
    rng = workloads.rng_for(3, salt=rank)
    x, y, n = workloads.lrmsd_clouds(args.batch, 100, 5000, rng)
    return {"input": x, "target": y, "num_atoms": n}


def describe(args, world):
    B = args.batch
    if args.workload == "training_step":
        return (METRIC, "residues/s", {
            "workload": f"full-atom training step, {B} chains x {args.length} residues per GPU, "
                        "uniform residue types, phi/psi/chi ~ U[-pi,pi], omega = pi; forward -> "
                        "LRMSD to N(0,0.1 rad)-perturbed targets -> backward",
            "global_batch": B * world, "seq_len": args.length})
    if args.workload == "fullatom_short":
        return (METRIC, "residues/s", {
            "workload": f"full-atom training step, {B} chains per GPU, lengths log-uniform in [16,128], "
                        "uniform residue types; forward -> LRMSD to N(0,0.1 rad)-perturbed targets -> backward",
            "global_batch": B * world, "seq_len": 128})
    if args.workload == "mixed_batch":
        return (METRIC, "residues/s", {
            "workload": f"mixed training step, {B} chains x {args.length} residues per GPU, every other "
                        "chain backbone-only (N, CA, C), the rest uniform residue types; forward -> "
                        "LRMSD to N(0,0.1 rad)-perturbed targets -> backward, one launch per call",
            "global_batch": B * world, "seq_len": args.length})
    if args.workload == "backbone_uneven":
        return (METRIC, "residues/s", {
            "workload": f"backbone step, {B} chains per GPU, lengths log-uniform in [50,1000], "
                        "phi/psi ~ U[-pi,pi], omega = pi; forward -> LRMSD to "
                        "N(0,0.1 rad)-perturbed targets -> backward",
            "global_batch": B * world, "seq_len": "logU[50,1000]"})
    if args.workload == "backbone_stress":
        return (METRIC, "residues/s", {
            "workload": f"backbone precision stress, {B} chains x 10000 residues per GPU, "
                        "phi/psi ~ U[-pi,pi], omega = pi; forward -> LRMSD to "
                        "N(0,0.1 rad)-perturbed targets -> backward",
            "global_batch": B * world, "seq_len": 10000})
    return (METRIC_LRMSD, "atoms/s", {
        "workload": f"LRMSD batch, {B} pairs per GPU, atoms U{{100..5000}}, N(0,15 A) clouds, "
                    "target = rotated + N(0,10 A) shift + N(0,0.5 A) noise; forward + backward",
        "global_batch": B * world})


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle arm
def oracle_step(args, d, n):
    """One step of the FP64 CPU oracle, as it stands, on the first n chains (or
    pairs) of the batch.  Returns (seconds, units processed)."""
    import oracle

    s = slice(0, n)
    if args.workload in ("training_step", "mixed_batch", "fullatom_short"):
        a, seq, L, ta = d["angles"][s], d["seq"][s], d["lengths"][s], d["target_angles"][s]
        Amax = oracle.max_atoms(seq, L)
        t0 = time.perf_counter()
        tgt, na = oracle.fullatom_forward(ta, seq, L, Amax)
        c, na = oracle.fullatom_forward(a, seq, L, Amax)
        oracle.lrmsd_forward(c, tgt, na)
        g = oracle.lrmsd_backward(np.full(n, 1.0 / n), c, tgt, na)
        oracle.fullatom_backward(a, seq, L, g)
        return time.perf_counter() - t0, int(L.sum())
    if args.workload in ("backbone_uneven", "backbone_stress"):
        a, L, ta = d["angles"][s], d["lengths"][s], d["target_angles"][s]
        t0 = time.perf_counter()
        tgt = oracle.backbone_forward(ta, L)
        c = oracle.backbone_forward(a, L)
        na = 3 * L
        oracle.lrmsd_forward(c, tgt, na)
        g = oracle.lrmsd_backward(np.full(n, 1.0 / n), c, tgt, na)
        oracle.backbone_backward(a, L, g)
        return time.perf_counter() - t0, int(L.sum())
    x, y, na = d["input"][s], d["target"][s], d["num_atoms"][s]
    t0 = time.perf_counter()
    oracle.lrmsd_forward(x, y, na)
    oracle.lrmsd_backward(np.ones(n), x, y, na)
    return time.perf_counter() - t0, int(na.sum())


def oracle_count(args, d, budget_s):
    """How many chains (pairs) make one oracle step of about budget_s seconds."""
    t1, _ = oracle_step(args, d, 1)
    total = len(next(iter(d.values())))
    return int(max(1, min(total, budget_s / max(t1, 1e-3))))


def cpu_baseline(args, d, unit, budget_s=12.0):
    import oracle

    oracle.build()
    n = oracle_count(args, d, budget_s)
    t, units = oracle_step(args, d, n)
    total = len(next(iter(d.values())))
    return {"value": units / t, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {total} chains/pairs of the workload, one full step in "
                      f"{t:.1f} s, single thread"}


def run_reference_sweep(args):
    """The oracle's backward (the paper's O(L^2) lever sums, FP64, one thread)
    on one chain per length of the sweep, each length bounded to a few seconds."""
    import time

    import oracle
    import workloads

    oracle.build()
    rows, total = [], 0.0
    for L in SWEEP_LENGTHS:
        if total > 60.0:
            break
        rng = workloads.rng_for(6, salt=L)
        lengths = np.full(1, L, np.int32)
        a = workloads.backbone_angles(lengths, rng)
        g = workloads.upstream_grad((1, 3 * L, 3), rng)
        t0 = time.perf_counter()
        oracle.backbone_backward(a, lengths, g)
        t1 = time.perf_counter()
        fa, seq = workloads.fullatom_inputs(lengths, rng)
        Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
        gf = workloads.upstream_grad((1, Amax, 3), rng)
        oracle.fullatom_backward(fa, seq, lengths, gf)
        t2 = time.perf_counter()
        rows.append({"L": L, "backbone_backward_ms": 1e3 * (t1 - t0), "fullatom_backward_ms": 1e3 * (t2 - t1)})
        total += t2 - t0
    last = rows[-1]
    value = last["L"] / (last["fullatom_backward_ms"] * 1e-3)
    line = {
        "impl": "reference", "metric": "fullatom_backward_residues_per_s_at_longest", "value": value,
        "unit": "residues/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": last["fullatom_backward_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "length_sweep", "batch": 1, "lengths": [r["L"] for r in rows]},
        "sweep": rows,
        "cpu_baseline": {"value": value, "unit": "residues/s", "cores": 1, "kind": "oracle",
                         "sample": "one chain per length, single thread, lengths until 60 s"},
        "e2e": {"value": value, "unit": "residues/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "length_sweep":
        run_reference_sweep(args)
        return
    import oracle

    oracle.build()
    d = make_inputs(args, 0)
    metric, unit, config = describe(args, 1)
    # the whole run stays near two minutes whatever --steps is
    n = oracle_count(args, d, 120.0 / (args.steps + 1))
    for _ in range(min(args.warmup, 1)):
        oracle_step(args, d, n)
    times, units = [], 0
    for _ in range(args.steps):
        t, u = oracle_step(args, d, n)
        times.append(t)
        units += u
    value = units / sum(times)
    config["sample_chains"] = n
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": f"first {n} chains/pairs of the workload per step, single thread"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- GPU workloads
def lrmsd_forward_kernels(tpl, P):
    """Kernels of tpl_lrmsd_forward for P pairs on this device (the library's plan)."""
    return ["lrmsd_pair_kernel"] * tpl.tpl_lrmsd_forward_launches(P)


class Step:
    """The C-ABI calls of one step with their bookkeeping.

    shape    launch shape of the chain kernels ("threads=.." [",res_per_thread=.."])

    calls    [(name, fn)] in launch order
    launches {name: kernels of ours per call}
    kernels  {name: [kernel names]}
    alg      {name: algorithmic bytes per call}
    units    units (residues or atoms) per step
    h2d      [(device tensor, pinned host tensor)] inputs of a step
    h2d_late {index in h2d: index of the first call that reads it} for inputs
             the first call does not read (their copies overlap the calls before)
    d2h      (pinned host tensor, device tensor) the step's result
    fp64     callable -> dict (errors vs the FP64 per-chain GPU form, its throughput)
    """


def cold_pick(torch, dev, cands, tuned, calls_for, reps=20, labels=("autotuned", "default")):
    """The fastest of the candidate options for a step made of calls_for(o),
    each captured as a CUDA graph and timed with L2 flushed before every
    replay (the protocol of the timed region)."""
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    times = []
    for o in cands:
        for c in calls_for(o):
            c()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for c in calls_for(o):
                c()
        best = None
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None or t < best else best
        times.append(best)
        del g
    i = int(np.argmin(times))
    tuned = dict(tuned, cold_ms=dict(zip(labels, times)), chosen=labels[i])
    return cands[i], tuned


def setup_training_step(args, tpl, torch, dev, d):
    import workloads

    a, seq, lengths, ta = d["angles"], d["seq"], d["lengths"], d["target_angles"]
    B, Lmax = a.shape[0], a.shape[2]
    Amax = workloads.pad_to(tpl.fullatom_max_atoms(seq, lengths))
    opts = tpl.Opts(threads=args.threads, res_per_thread=args.res_per_thread, schedule=SCHEDULES[args.schedule],
                    bwd_mode=tpl.BWD_FROM_COORDS if args.bwd == "coords" else tpl.BWD_RECOMPUTE)
    A = torch.from_numpy(a).to(dev)
    S = torch.from_numpy(seq).to(dev)
    Ln = torch.from_numpy(lengths).to(dev)
    TA = torch.from_numpy(ta).to(dev)
    coords = torch.empty((B, Amax, 3), device=dev)
    target = torch.empty((B, Amax, 3), device=dev)
    na = torch.empty((B,), dtype=torch.int32, device=dev)
    na_t = torch.empty_like(na)
    lr = torch.empty((B,), device=dev)
    wgt = torch.full((B,), 1.0 / B, device=dev)  # d(mean LRMSD)/d(LRMSD_b)
    gcoords = torch.empty_like(coords)
    gang = torch.empty_like(A)
    fa_ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=dev)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, Amax), dtype=torch.uint8, device=dev)
    tpl.tpl_fullatom_forward(TA, S, Ln, target, na_t, fa_ws, opts)  # target structures
    torch.cuda.synchronize()
    n_atoms = int(na_t.sum().item())
    tuned = None
    gtune = None
    if not args.no_autotune and not args.threads and args.schedule == "auto":
        if args.bwd == "coords" and args.fusion == "backward":
            # the three calls of the timed step
            opts, tms = tpl.tpl_fullatom_lrmsd_autotune(A, S, Ln, coords, na, target, wgt, lr, lr_ws, gang, fa_ws)
            tuned = {"threads": opts.threads, "res_per_thread": opts.res_per_thread, "schedule": opts.schedule,
                     "step_ms": tms}
        else:
            gtune = torch.randn((B, Amax, 3), device=dev)
            opts, tms = tpl.tpl_fullatom_autotune(A, S, Ln, coords, na, gtune, gang, fa_ws,
                                                  bwd_mode=opts.bwd_mode)
            tuned = {"threads": opts.threads, "res_per_thread": opts.res_per_thread, "schedule": opts.schedule,
                     "fwd_bwd_ms": tms}

    if tuned is not None:
        # the autotuner times warm replays; this step is timed with L2 flushed,
        # so its pick is checked against the library default under that protocol
        opts, tuned = cold_pick(torch, dev, [opts, tpl.Opts(bwd_mode=opts.bwd_mode)], tuned, lambda o: [
            lambda: tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, o),
            lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws),
            lambda: tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, coords, target, wgt, lr_ws, gang, fa_ws, o)]
            if args.bwd == "coords" and args.fusion == "backward" else [
            lambda: tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, o),
            lambda: tpl.tpl_fullatom_backward(A, S, Ln, coords, gtune, gang, fa_ws, o)])
    if not args.write_padding:
        # buffers live across steps: zeroed once here, the calls skip their padding
        opts.flags = tpl.FLAG_PADDING_ZEROED
        coords.zero_()
        gang.zero_()
    st = Step()
    st.shape = f"threads={opts.threads or 384},res_per_thread={opts.res_per_thread or 1}"
    res = int(lengths.sum())
    st.kernels = {"fullatom_forward": ["schedule_kernel", "fa_fwd_kernel"],
                  "lrmsd_forward": lrmsd_forward_kernels(tpl, B)}
    st.alg = {"fullatom_forward": res * (28 + 1) + 12 * n_atoms, "lrmsd_forward": 24 * n_atoms}
    st_ws = None
    if args.fusion == "step" and args.bwd == "coords":
        # forward with the LRMSD moments in its tiles, then per chain the eigen-solve
        # and the residual pass (LRMSD out); backward with the LRMSD gradient
        # formed inside (one workspace for both)
        st_ws = torch.empty(tpl.tpl_fullatom_lrmsd_workspace_size(B, Lmax), dtype=torch.uint8, device=dev)
        st.calls = [
            ("lrmsd_step_forward",
             lambda: tpl.tpl_fullatom_lrmsd_forward(A, S, Ln, target, coords, na, lr, st_ws, opts)),
            ("lrmsd_step_backward",
             lambda: tpl.tpl_fullatom_lrmsd_backward(S, Ln, coords, target, wgt, gang, st_ws, opts)),
        ]
        st.kernels = {"lrmsd_step_forward": ["schedule_kernel", "fa_fwd_kernel", "lrmsd_parts_kernel"],
                      "lrmsd_step_backward": ["fa_bwd_coords_kernel"]}
        # forward: angles and sequence in, coordinates out, target read for the moments;
        # backward: angles and sequence in, angle gradient out, coordinates and target read
        st.alg = {"lrmsd_step_forward": res * (28 + 1) + 24 * n_atoms,
                  "lrmsd_step_backward": res * (28 + 1 + 28) + 24 * n_atoms}
    elif args.fusion == "none" or args.bwd != "coords":
        bwd_kernel = "fa_bwd_coords_kernel" if args.bwd == "coords" else "fa_bwd_kernel"
        st.calls = [
            ("fullatom_forward", lambda: tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, opts)),
            ("lrmsd_forward", lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws)),
            ("lrmsd_backward", lambda: tpl.tpl_lrmsd_backward(wgt, coords, target, na, gcoords, lr_ws)),
            ("fullatom_backward",
             lambda: tpl.tpl_fullatom_backward(A, S, Ln, coords, gcoords, gang, fa_ws, opts)),
        ]
        st.kernels.update({"lrmsd_backward": ["lrmsd_grad_kernel"], "fullatom_backward": [bwd_kernel]})
        st.alg.update({"lrmsd_backward": 36 * n_atoms, "fullatom_backward": res * (28 + 1 + 28) + 12 * n_atoms})
    else:
        # LRMSD backward formed inside the full-atom backward (no coordinate-gradient tensor)
        st.calls = [
            ("fullatom_forward", lambda: tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, opts)),
            ("lrmsd_forward", lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws)),
            ("lrmsd_fullatom_backward",
             lambda: tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, coords, target, wgt, lr_ws, gang, fa_ws, opts)),
        ]
        st.kernels["lrmsd_fullatom_backward"] = ["fa_bwd_coords_kernel"]
        # angles 28 + sequence 1 in, angle gradient 28 out per residue; coordinates and target 24 per atom
        st.alg["lrmsd_fullatom_backward"] = res * (28 + 1 + 28) + 24 * n_atoms
    st.launches = {k: len(v) for k, v in st.kernels.items()}
    st.units = res
    st.atoms = n_atoms
    st.extra_config = {"atoms_per_gpu": n_atoms, "threads": opts.threads or "default",
                       "res_per_thread": opts.res_per_thread or "default",
                       "output_padding": "written every call" if args.write_padding else "zeroed once",
                       "fullatom_backward": args.bwd, "autotuned": tuned,
                       "fusion": {2: "fused step: forward with LRMSD moments + eigen-solve; backward with "
                                     "LRMSD gradient, residuals and LRMSD",
                                  3: "LRMSD backward formed inside the full-atom backward",
                                  4: "separate calls"}[len(st.calls)]}
    tgt_host = target.cpu().pin_memory()
    st.h2d = [(A, torch.from_numpy(a).pin_memory()), (S, torch.from_numpy(seq).pin_memory()),
              (Ln, torch.from_numpy(lengths).pin_memory()), (target, tgt_host)]
    if st.calls[0][0] == "fullatom_forward":
        st.h2d_late = {3: 1}  # the target is first read by the LRMSD forward
    st.outputs = {"coords": coords, "target": target, "num_atoms": na, "lrmsd": lr, "grad_angles": gang,
                  "weights": wgt}
    st.d2h = (torch.empty((B,), dtype=torch.float32).pin_memory(), lr)

    def fp64():
        A64 = torch.from_numpy(a.astype(np.float64)).to(dev)
        c64 = torch.zeros((B, Amax, 3), dtype=torch.float64, device=dev)
        t64 = torch.zeros_like(c64)
        na64 = torch.zeros((B,), dtype=torch.int32, device=dev)
        lr64 = torch.zeros((B,), dtype=torch.float64, device=dev)
        state = torch.zeros((B, 16), dtype=torch.float64, device=dev)
        gc = torch.zeros_like(c64)
        ga = torch.zeros_like(A64)
        w = torch.full((B,), 1.0 / B, dtype=torch.float64, device=dev)
        # the FP64 form gets the FP32 step's own target so only the step's arithmetic differs
        t64.copy_(target.double())

        def step64():
            tpl.tpl_fullatom_forward_ref64(A64, S, Ln, c64, na64)
            tpl.tpl_lrmsd_forward_ref64(c64, t64, na64, lr64, state)
            tpl.tpl_lrmsd_backward_ref64(w, c64, t64, na64, state, gc)
            tpl.tpl_fullatom_backward_ref64(A64, S, Ln, c64, gc, ga)

        ms = time_once(torch, step64)
        return {"fp64_gpu_form": {"value": res / (ms * 1e-3), "unit": "residues/s", "ms_per_step": ms},
                "errors_vs_fp64_gpu": errors(torch, coords, c64, gang, ga, lr, lr64)}

    st.fp64 = fp64
    return st


def setup_backbone_uneven(args, tpl, torch, dev, d):
    a, lengths, ta = d["angles"], d["lengths"], d["target_angles"]
    B, Lmax = a.shape[0], a.shape[2]
    opts = tpl.Opts(threads=args.threads, res_per_thread=args.res_per_thread, schedule=SCHEDULES[args.schedule],
                    bwd_mode=tpl.BWD_FROM_COORDS if args.bwd == "coords" else tpl.BWD_RECOMPUTE)
    A = torch.from_numpy(a).to(dev)
    Ln = torch.from_numpy(lengths).to(dev)
    na_host = (3 * lengths).astype(np.int32)
    na = torch.from_numpy(na_host).to(dev)
    coords = torch.empty((B, 3 * Lmax, 3), device=dev)
    target = torch.empty_like(coords)
    lr = torch.empty((B,), device=dev)
    wgt = torch.full((B,), 1.0 / B, device=dev)
    gcoords = torch.empty_like(coords)
    gang = torch.empty_like(A)
    bb_ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=dev)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, 3 * Lmax), dtype=torch.uint8, device=dev)
    tpl.tpl_backbone_forward(torch.from_numpy(ta).to(dev), Ln, target, bb_ws, opts)
    torch.cuda.synchronize()
    tuned = None
    step_fused = args.fusion == "step" and args.bwd == "coords"
    st_ws = None
    if step_fused:
        st_ws = torch.empty(tpl.tpl_backbone_lrmsd_workspace_size(B, Lmax), dtype=torch.uint8, device=dev)
        if opts.res_per_thread == 0 and opts.threads == 0:
            opts.threads, opts.res_per_thread = 128, 4
    if not args.no_autotune and not args.threads and not args.res_per_thread and args.schedule == "auto":
        if step_fused:
            # the training-step shapes, timed as the step is timed
            cands = [tpl.Opts(threads=t, res_per_thread=k, schedule=tpl.SCHED_PACKED) for t, k in STEP_SHAPES]
            opts, tuned = cold_pick(torch, dev, cands, {}, lambda o: [
                lambda: tpl.tpl_backbone_lrmsd_step(A, Ln, target, wgt, coords, lr, gang, st_ws, o)],
                labels=[f"{t}x{k}" for t, k in STEP_SHAPES])
        elif args.bwd == "coords" and not args.unfused:
            # the three calls of the timed step
            opts, tms = tpl.tpl_backbone_lrmsd_autotune(A, Ln, coords, target, na, wgt, lr, lr_ws, gang, bb_ws)
            tuned = {"threads": opts.threads, "res_per_thread": opts.res_per_thread,
                     "schedule": opts.schedule, "step_ms": tms}
        else:
            gtune = torch.randn((B, 3 * Lmax, 3), device=dev)
            opts, tms = tpl.tpl_backbone_autotune(A, Ln, coords, gtune, gang, bb_ws, bwd_mode=opts.bwd_mode)
            tuned = {"threads": opts.threads, "res_per_thread": opts.res_per_thread,
                     "schedule": opts.schedule, "fwd_bwd_ms": tms}
    n_atoms = int(na_host.sum())
    res = int(lengths.sum())

    if not args.write_padding:
        opts.flags = tpl.FLAG_PADDING_ZEROED
        coords.zero_()
        gang.zero_()
    st = Step()
    st.shape = f"threads={opts.threads or 128},res_per_thread={opts.res_per_thread or 4}"
    st.kernels = {"backbone_forward": ["schedule_kernel", "bb_fwd_kernel"],
                  "lrmsd_forward": lrmsd_forward_kernels(tpl, B)}
    st.alg = {"backbone_forward": 48 * res, "lrmsd_forward": 24 * n_atoms}
    if step_fused:
        # one call: whole chains in one CTA each (pack or one tile); longer
        # chains add the eigen-solve and backward launches
        st.calls = [("lrmsd_step",
                     lambda: tpl.tpl_backbone_lrmsd_step(A, Ln, target, wgt, coords, lr, gang, st_ws, opts))]
        tile = opts.threads * opts.res_per_thread
        st.kernels = {"lrmsd_step": ["schedule_kernel", "bb_step_kernel"] +
                      (["lrmsd_solve_tiles_kernel", "bb_bwd_kernel"] if Lmax > tile else [])}
        # angles 12 in, angle gradient 12 out per residue; target 12 in, coordinates 12 out per atom
        st.alg = {"lrmsd_step": 24 * res + 24 * n_atoms}
    elif args.unfused or args.bwd != "coords":
        st.calls = [
            ("backbone_forward", lambda: tpl.tpl_backbone_forward(A, Ln, coords, bb_ws, opts)),
            ("lrmsd_forward", lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws)),
            ("lrmsd_backward", lambda: tpl.tpl_lrmsd_backward(wgt, coords, target, na, gcoords, lr_ws)),
            ("backbone_backward",
             lambda: tpl.tpl_backbone_backward(A, Ln, coords, gcoords, gang, bb_ws, opts)),
        ]
        st.kernels.update({"lrmsd_backward": ["lrmsd_grad_kernel"], "backbone_backward": ["bb_bwd_kernel"]})
        st.alg.update({"lrmsd_backward": 36 * n_atoms, "backbone_backward": 60 * res})
        if args.bwd == "quadratic":
            # the paper's O(L^2) sums of Eq. 2, one thread per atom (comparator)
            st.calls[3] = ("backbone_backward",
                           lambda: tpl.tpl_backbone_backward_quadratic(Ln, coords, gcoords, gang))
            st.kernels["backbone_backward"] = ["bb_bwd_quadratic_kernel"]
    else:
        st.calls = [
            ("backbone_forward", lambda: tpl.tpl_backbone_forward(A, Ln, coords, bb_ws, opts)),
            ("lrmsd_forward", lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws)),
            ("lrmsd_backbone_backward",
             lambda: tpl.tpl_backbone_backward_lrmsd(A, Ln, coords, target, wgt, lr_ws, gang, bb_ws, opts)),
        ]
        st.kernels["lrmsd_backbone_backward"] = ["bb_bwd_kernel"]
        # angles 12 in, gradient 12 out per residue; coordinates and target 24 per atom
        st.alg["lrmsd_backbone_backward"] = 24 * res + 24 * n_atoms
    st.launches = {k: len(v) for k, v in st.kernels.items()}
    st.units = res
    st.atoms = n_atoms
    st.extra_config = {"atoms_per_gpu": n_atoms, "threads": opts.threads or "default",
                       "res_per_thread": opts.res_per_thread or "default",
                       "output_padding": "written every call" if args.write_padding else "zeroed once",
                       "backbone_backward": args.bwd,
                       "autotuned": tuned,
                       "lrmsd_backward": "separate call" if len(st.calls) == 4 else
                                         "formed inside the backbone backward" if len(st.calls) == 3 else
                                         "one training-step call"}
    st.h2d = [(A, torch.from_numpy(a).pin_memory()), (Ln, torch.from_numpy(lengths).pin_memory()),
              (na, torch.from_numpy(na_host).pin_memory()), (target, target.cpu().pin_memory())]
    if step_fused:  # one call reads everything; the atom counts are not an input
        st.h2d = [st.h2d[0], st.h2d[1], st.h2d[3]]
        st.h2d_late = {}
    else:
        st.h2d_late = {2: 1, 3: 1}  # atom counts and target are first read by the LRMSD forward
    st.outputs = {"coords": coords, "target": target, "lrmsd": lr, "grad_angles": gang, "weights": wgt}
    st.d2h = (torch.empty((B,), dtype=torch.float32).pin_memory(), lr)

    def fp64():
        A64 = torch.from_numpy(a.astype(np.float64)).to(dev)
        c64 = torch.zeros((B, 3 * Lmax, 3), dtype=torch.float64, device=dev)
        t64 = target.double()
        lr64 = torch.zeros((B,), dtype=torch.float64, device=dev)
        state = torch.zeros((B, 16), dtype=torch.float64, device=dev)
        gc = torch.zeros_like(c64)
        ga = torch.zeros_like(A64)
        w = torch.full((B,), 1.0 / B, dtype=torch.float64, device=dev)

        def step64():
            tpl.tpl_backbone_forward_ref64(A64, Ln, c64)
            tpl.tpl_lrmsd_forward_ref64(c64, t64, na, lr64, state)
            tpl.tpl_lrmsd_backward_ref64(w, c64, t64, na, state, gc)
            tpl.tpl_backbone_backward_ref64(A64, Ln, c64, gc, ga)

        ms = time_once(torch, step64)
        return {"fp64_gpu_form": {"value": res / (ms * 1e-3), "unit": "residues/s", "ms_per_step": ms},
                "errors_vs_fp64_gpu": errors(torch, coords, c64, gang, ga, lr, lr64,
                                             prefix_atoms=3000 if Lmax > 1000 else None)}

    st.fp64 = fp64
    return st


def setup_lrmsd_batch(args, tpl, torch, dev, d):
    x, y, n = d["input"], d["target"], d["num_atoms"]
    P, Nmax = x.shape[0], x.shape[1]
    X = torch.from_numpy(x).to(dev)
    Y = torch.from_numpy(y).to(dev)
    NA = torch.from_numpy(n).to(dev)
    lr = torch.empty((P,), device=dev)
    up = torch.ones((P,), device=dev)
    gx = torch.empty_like(X)
    ws = torch.empty(tpl.tpl_lrmsd_workspace_size(P, Nmax), dtype=torch.uint8, device=dev)
    n_atoms = int(n.sum())

    st = Step()
    st.shape = None
    st.calls = [("lrmsd_forward", lambda: tpl.tpl_lrmsd_forward(X, Y, NA, lr, ws)),
                ("lrmsd_backward", lambda: tpl.tpl_lrmsd_backward(up, X, Y, NA, gx, ws))]
    st.kernels = {"lrmsd_forward": lrmsd_forward_kernels(tpl, P),
                  "lrmsd_backward": ["lrmsd_grad_kernel"]}
    st.launches = {k: len(v) for k, v in st.kernels.items()}
    st.alg = {"lrmsd_forward": 24 * n_atoms, "lrmsd_backward": 36 * n_atoms}
    st.units = n_atoms
    st.atoms = n_atoms
    st.extra_config = {"atoms_per_gpu": n_atoms, "Nmax": Nmax}
    st.h2d = [(X, torch.from_numpy(x).pin_memory()), (Y, torch.from_numpy(y).pin_memory()),
              (NA, torch.from_numpy(n).pin_memory())]
    st.outputs = {"lrmsd": lr, "grad_input": gx, "weights": up}
    st.d2h = (torch.empty((P,), dtype=torch.float32).pin_memory(), lr)

    def fp64():
        X64, Y64 = X.double(), Y.double()
        lr64 = torch.zeros((P,), dtype=torch.float64, device=dev)
        state = torch.zeros((P, 16), dtype=torch.float64, device=dev)
        g64 = torch.zeros_like(X64)
        up64 = torch.ones((P,), dtype=torch.float64, device=dev)

        def step64():
            tpl.tpl_lrmsd_forward_ref64(X64, Y64, NA, lr64, state)
            tpl.tpl_lrmsd_backward_ref64(up64, X64, Y64, NA, state, g64)

        ms = time_once(torch, step64)
        g32 = gx.double().reshape(P, -1)
        g6 = g64.reshape(P, -1)
        grad_rel = float(((g32 - g6).norm(dim=1) / g6.norm(dim=1).clamp_min(1e-300)).max().item())
        return {"fp64_gpu_form": {"value": n_atoms / (ms * 1e-3), "unit": "atoms/s", "ms_per_step": ms},
                "errors_vs_fp64_gpu": {"lrmsd_max_abs_A": float((lr.double() - lr64).abs().max().item()),
                                       "grad_rel_max": grad_rel}}

    st.fp64 = fp64
    return st


def time_once(torch, fn):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def errors(torch, c32, c64, g32, g64, lr32, lr64, prefix_atoms=None):
    """Max-abs coordinate error, per-chain relative angle-gradient error (max over
    chains) and max-abs LRMSD error of the FP32 step against the FP64 form.
    With prefix_atoms, also the coordinate error over the first prefix_atoms
    atoms of every chain (the drift along long chains)."""
    B = c32.shape[0]
    a = g32.double().reshape(B, -1)
    b = g64.reshape(B, -1)
    dc = (c32.double() - c64).abs()
    out = {"coord_max_abs_A": float(dc.max().item()),
           "grad_rel_max": float(((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-300)).max().item()),
           "lrmsd_max_abs_A": float((lr32.double() - lr64).abs().max().item())}
    if prefix_atoms is not None:
        out[f"coord_max_abs_first_{prefix_atoms}_atoms_A"] = float(dc[:, :prefix_atoms].max().item())
    return out


SETUP = {"training_step": setup_training_step, "mixed_batch": setup_training_step,
         "fullatom_short": setup_training_step,
         "backbone_uneven": setup_backbone_uneven,
         "backbone_stress": setup_backbone_uneven, "lrmsd_batch": setup_lrmsd_batch}


# ----------------------------------------------------------------------------- GPU arm
def measure(args, workload, tpl, torch, dev, rank, world, local, flush):
    """Times one workload's step (a CUDA graph of its C-ABI calls) and its
    end-to-end form; returns the fields of its JSON line."""
    sub = argparse.Namespace(**vars(args))
    if workload != args.workload:  # an extra workload of the default run: its own defaults
        sub.workload, sub.batch, sub.threads, sub.res_per_thread = workload, DEFAULT_BATCH[workload], 0, 0
    d = make_inputs(sub, rank)
    st = SETUP[workload](sub, tpl, torch, dev, d)
    metric, unit, config = describe(sub, world)
    names = [n for n, _ in st.calls]
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        for _, c in st.calls:
            c()
    torch.cuda.synchronize()
    status = tpl.tpl_get_status()
    if status != 0:
        raise SystemExit(f"device status 0x{status:x} after the warm-up steps ({workload})")
    # the whole step is one CUDA graph (forward -> LRMSD -> backward), replayed
    # between CUDA events; a second graph with event-record nodes between the
    # calls gives the per-call times (its extra nodes make it a little slower,
    # so it is used for the breakdown and the roofline, not for the value)
    nc = len(st.calls)
    step_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(step_graph):
        for _, c in st.calls:
            c()
    split_ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(nc + 1)]
    split_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(split_graph):
        for i, (_, c) in enumerate(st.calls):
            split_ev[i].record()
            c()
        split_ev[nc].record()
    torch.cuda.synchronize()

    def step():
        step_graph.replay()

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    total_ms = max_over_ranks(float(step_ms.sum()), dev, world)
    value = job_throughput(st.units, world, args.steps, total_ms)

    # per-call times from the split graph (same inputs, L2 flushed before each step)
    n_split = min(args.steps, 500)
    per = np.zeros((n_split, nc))
    for k in range(n_split):
        flush.zero_()
        split_graph.replay()
        split_ev[nc].synchronize()
        per[k] = [split_ev[i].elapsed_time(split_ev[i + 1]) for i in range(nc)]

    # roofline of the dominant call (per-unit bytes x units per launch / mean event time)
    mean_ms = per.mean(axis=0)
    dom = names[int(np.argmax(mean_ms))]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = st.alg[dom] / (mean_ms[names.index(dom)] * 1e-3) / 1e9
    # a capture at the step's launch shape (or one that takes no shape)
    tr = next((e for e in TRAFFIC.get((workload, dom), []) if e[3] is None or e[3] == st.shape), None)
    traffic = None
    if tr is not None:
        traffic = tr[0] * (st.atoms if tr[1] == "atom" else st.units)
    roofline = {"bound": "hbm", "kernel": "+".join(st.kernels[dom]), "call": dom,
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": tr[2] if tr else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "alg_bytes": st.alg[dom]}
    step_bytes = sum(st.alg.values())

    # end to end: pinned host inputs -> device, the step, result -> host
    h2d = sum(h.numel() * h.element_size() for _, h in st.h2d)
    host_out, dev_out = st.d2h
    d2h = host_out.numel() * host_out.element_size()

    # One graph per end-to-end step: the copies of the inputs the first call
    # needs, the calls, the copy of the result back; inputs read only by later
    # calls are copied on a second stream that joins before their first reader.
    late = getattr(st, "h2d_late", {})
    join_at = min(late.values()) if late else None
    side = torch.cuda.Stream(dev)
    e2e_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(e2e_graph):
        cap = torch.cuda.current_stream(dev)
        joined = None
        if late:
            fork = torch.cuda.Event()
            fork.record(cap)
            side.wait_event(fork)
            with torch.cuda.stream(side):
                for i in sorted(late):
                    dv, h = st.h2d[i]
                    dv.copy_(h, non_blocking=True)
                joined = torch.cuda.Event()
                joined.record(side)
        for i, (dv, h) in enumerate(st.h2d):
            if i not in late:
                dv.copy_(h, non_blocking=True)
        for i, (_, c) in enumerate(st.calls):
            if joined is not None and i == join_at:
                cap.wait_event(joined)
            c()
        host_out.copy_(dev_out, non_blocking=True)

    def e2e_step():
        e2e_graph.replay()

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    n_e2e = min(args.steps, 200)
    e_ms = 0.0
    for _ in range(n_e2e):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    e_ms = max_over_ranks(e_ms, dev, world)
    e2e_value = job_throughput(st.units, world, n_e2e, e_ms)

    # the e2e loop rewrote the inputs with the same values: the FP32 outputs the
    # FP64 comparison reads are those of the last step
    extra = {}
    if rank == 0 and not args.no_fp64:
        extra = st.fp64()
    config.update({"parallelism": f"replicas x{world}", "l2": "flushed (512 MiB write) before every step"})
    config.update(st.extra_config)
    out = {
        "metric": metric, "value": value, "unit": unit, "ms_per_step": total_ms / args.steps,
        "config": config,
        "breakdown_ms": dict(zip(names, [float(x) for x in mean_ms])),
        "breakdown_source": "graph of the step with event nodes between the calls",
        "step_alg_bytes": step_bytes,
        "step_gbs": step_bytes / (total_ms / args.steps * 1e-3) / 1e9,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": sum(st.launches.values()) * args.steps,
        "clocks": clk,
    }
    out.update(extra)
    return out, d, unit


# The default run (the training step) also times these workloads, each with
# the same protocol, and reports them under "workloads".
EXTRA_WORKLOADS = ("backbone_uneven", "lrmsd_batch")


# ----------------------------------------------------------------------------- length sweep
SWEEP_LENGTHS = (64, 128, 256, 512, 1024, 2048, 4096)


def _flushed_ms(torch, fn, flush, reps):
    """Median of reps launches of fn, each after an L2 flush, timed with CUDA
    events on the current stream."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _slope(ls, ts):
    """Least-squares exponent of t ~ L^k over the sweep's upper half."""
    h = len(ls) // 2
    x, y = np.log(np.array(ls[h:], float)), np.log(np.array(ts[h:], float))
    return float(np.polyfit(x, y, 1)[0]) if len(x) >= 2 else None


def run_length_sweep(args):
    """The scan forward and backward against the paper's O(L^2) backward forms
    (Eq. 2 summed per (angle, atom); Eq. 1 depth first), for both models, at
    growing chain length and a fixed batch: the shapes of the paper's timing
    figures.  Inputs are seeded synthetic chains of one length."""
    import torch

    import paper_1812_01108_gb300 as tpl
    import workloads

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tpl.load_library()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    B, reps = args.batch, max(3, args.steps)
    sweep = []
    clocks = ClockSampler(local)
    clocks.start()
    for L in SWEEP_LENGTHS:
        rng = workloads.rng_for(6, salt=L)
        lengths = np.full(B, L, np.int32)
        Ln = torch.from_numpy(lengths).to(dev)
        row = {"L": L}
        # backbone
        a = workloads.backbone_angles(lengths, rng)
        A = torch.from_numpy(a).to(dev)
        c = torch.zeros((B, 3 * L, 3), device=dev)
        g = torch.from_numpy(workloads.upstream_grad((B, 3 * L, 3), rng)).to(dev)
        ga = torch.zeros_like(A)
        gq = torch.zeros_like(A)
        ws = torch.empty(tpl.tpl_backbone_workspace_size(B, L), dtype=torch.uint8, device=dev)
        o = tpl.Opts(bwd_mode=tpl.BWD_FROM_COORDS)
        row["backbone_forward_ms"] = _flushed_ms(torch, lambda: tpl.tpl_backbone_forward(A, Ln, c, ws, o), flush, reps)
        row["backbone_backward_scan_ms"] = _flushed_ms(
            torch, lambda: tpl.tpl_backbone_backward(A, Ln, c, g, ga, ws, o), flush, reps)
        row["backbone_backward_quadratic_ms"] = _flushed_ms(
            torch, lambda: tpl.tpl_backbone_backward_quadratic(Ln, c, g, gq), flush, reps)
        torch.cuda.synchronize()
        row["backbone_scan_vs_quadratic_rel"] = float(torch.linalg.vector_norm(ga - gq) /
                                                      torch.linalg.vector_norm(gq))
        del A, c, g, ga, gq, ws
        # full atom
        fa, seq = workloads.fullatom_inputs(lengths, rng)
        Amax = workloads.pad_to(tpl.fullatom_max_atoms(seq, lengths))
        A = torch.from_numpy(fa).to(dev)
        S = torch.from_numpy(seq).to(dev)
        c = torch.zeros((B, Amax, 3), device=dev)
        na = torch.zeros((B,), dtype=torch.int32, device=dev)
        g = torch.from_numpy(workloads.upstream_grad((B, Amax, 3), rng)).to(dev)
        ga = torch.zeros_like(A)
        gq = torch.zeros_like(A)
        ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, L), dtype=torch.uint8, device=dev)
        row["atoms_per_chain"] = int(tpl.fullatom_max_atoms(seq, lengths))
        row["fullatom_forward_ms"] = _flushed_ms(
            torch, lambda: tpl.tpl_fullatom_forward(A, S, Ln, c, na, ws, o), flush, reps)
        row["fullatom_backward_scan_ms"] = _flushed_ms(
            torch, lambda: tpl.tpl_fullatom_backward(A, S, Ln, c, g, ga, ws, o), flush, reps)
        row["fullatom_backward_quadratic_ms"] = _flushed_ms(
            torch, lambda: tpl.tpl_fullatom_backward_quadratic(S, Ln, c, g, gq), flush, reps)
        torch.cuda.synchronize()
        row["fullatom_scan_vs_quadratic_rel"] = float(torch.linalg.vector_norm(ga - gq) /
                                                      torch.linalg.vector_norm(gq))
        del A, S, c, na, g, ga, gq, ws
        torch.cuda.empty_cache()
        sweep.append(row)
    clk = clocks.stop()
    ls = [r["L"] for r in sweep]
    exps = {k[:-3]: _slope(ls, [r[k] for r in sweep]) for k in sweep[0] if k.endswith("_ms")}
    last = sweep[-1]
    ms = last["fullatom_forward_ms"] + last["fullatom_backward_scan_ms"]
    line = {
        "metric": "fullatom_fwd_bwd_residues_per_s_at_longest", "value": B * last["L"] / (ms * 1e-3),
        "unit": "residues/s", "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "length_sweep", "batch": B, "lengths": list(SWEEP_LENGTHS),
                   "backward_input": "forward coordinates", "l2": "flushed before every timed call"},
        "sweep": sweep, "time_exponent_upper_half": exps, "clocks": clk,
        # per length and timed repetition: backbone forward 2 (work list, scan),
        # scan backward 1, quadratic 1; full atom the same
        "gpu_launches": 8 * reps * len(SWEEP_LENGTHS),
    }
    if rank == 0:
        print(json.dumps(line))


def run_tpl(args):
    import torch

    import paper_1812_01108_gb300 as tpl
    from paper_1812_01108_gb300 import build as tpl_build

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        tpl_build.build()
    if world > 1:
        dist.barrier()
    tpl.load_library()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    main_out, d, unit = measure(args, args.workload, tpl, torch, dev, rank, world, local, flush)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, d, unit)
    extras = {}
    if args.workload == "training_step" and not args.no_extra:
        for w in EXTRA_WORKLOADS:
            torch.cuda.empty_cache()
            out, _, _ = measure(args, w, tpl, torch, dev, rank, world, local, flush)
            extras[w] = out
    if rank == 0:
        line = {
            "metric": main_out["metric"], "value": main_out["value"], "unit": main_out["unit"],
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main_out["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        }
        line.update({k: v for k, v in main_out.items() if k not in line})
        line["cpu_baseline"] = cpu
        if extras:
            line["workloads"] = extras
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "length_sweep":
        run_length_sweep(args)
    else:
        run_tpl(args)


if __name__ == "__main__":
    main()
