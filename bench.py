"""Throughput benchmark of the hot path: one step = full-atom forward -> LRMSD
forward (to perturbed target structures) -> LRMSD backward -> full-atom
backward, on synthetic inputs shaped like the paper's workloads.

Default workload: the training-step shape, 256 chains x 700 residues with
uniformly random residue types (the largest full-atom configuration).  Prints
one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.

Timing: W warm-up steps, then K timed steps; each timed step is bracketed by
CUDA events on the launching stream, and L2 is flushed (a 512 MiB write)
before every step outside the timed interval.  Under torchrun each rank runs
its own batch (weak scaling, no data-path collective); the elapsed time is the
max over ranks.
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="tpl", choices=["tpl", "reference"])
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--length", type=int, default=700)
    p.add_argument("--threads", type=int, default=0, help="CTA size of the chain kernels (0 = default)")
    p.add_argument("--bwd", default="coords", choices=["coords", "recompute"],
                   help="full-atom backward: read the forward's coordinates or rebuild frames")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 per-chain comparison")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(B, L, rank):
    import workloads

    rng = workloads.rng_for(4, salt=rank)
    lengths = np.full(B, L, np.int32)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    return a, seq, lengths, ta


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
def oracle_sample(a, seq, lengths, ta, n_chains):
    """The FP64 CPU oracle, as it stands, on the first n_chains of the batch: one full step."""
    import oracle

    s = slice(0, n_chains)
    Amax = oracle.max_atoms(seq[s], lengths[s])
    t0 = time.perf_counter()
    tgt, na = oracle.fullatom_forward(ta[s], seq[s], lengths[s], Amax)
    c, na = oracle.fullatom_forward(a[s], seq[s], lengths[s], Amax)
    oracle.lrmsd_forward(c, tgt, na)
    g = oracle.lrmsd_backward(np.full(n_chains, 1.0 / n_chains), c, tgt, na)
    oracle.fullatom_backward(a[s], seq[s], lengths[s], g)
    return time.perf_counter() - t0


def cpu_baseline(a, seq, lengths, ta, budget_s=12.0):
    import oracle

    oracle.build()
    t1 = oracle_sample(a, seq, lengths, ta, 1)
    n = int(max(1, min(len(lengths), budget_s / max(t1, 1e-3))))
    t = oracle_sample(a, seq, lengths, ta, n)
    res = int(lengths[:n].sum())
    return {"value": res / t, "unit": "residues/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} of {len(lengths)} chains x {int(lengths[0])} residues, one full step "
                      f"(forward, LRMSD forward+backward, backward) in {t:.1f} s, single thread"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    a, seq, lengths, ta = make_workload(args.batch, args.length, 0)
    import oracle

    oracle.build()
    t1 = oracle_sample(a, seq, lengths, ta, 1)
    # the whole run stays near two minutes whatever --steps is
    per_step = 120.0 / (args.steps + 1)
    n = int(max(1, min(args.batch, per_step / max(t1, 1e-3))))
    for _ in range(min(args.warmup, 1)):
        oracle_sample(a, seq, lengths, ta, n)
    times = [oracle_sample(a, seq, lengths, ta, n) for _ in range(args.steps)]
    res = int(lengths[:n].sum())
    value = res * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "residues/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"full-atom training step, {args.batch} chains x {args.length} "
                               "residues (forward, LRMSD forward+backward, backward)",
                   "sample_chains": n},
        "cpu_baseline": {"value": value, "unit": "residues/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} chains per step of the same workload, single thread"},
        "e2e": {"value": value, "unit": "residues/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- GPU arm
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

    B, L = args.batch, args.length
    a, seq, lengths, ta = make_workload(B, L, rank)
    import workloads

    Amax = workloads.pad_to(max(tpl.fullatom_max_atoms(seq, lengths), tpl.fullatom_max_atoms(seq, lengths)))
    Lmax = a.shape[2]
    opts = tpl.Opts(threads=args.threads,
                    bwd_mode=tpl.BWD_FROM_COORDS if args.bwd == "coords" else tpl.BWD_RECOMPUTE)

    # device-resident inputs
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
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    names = ["fullatom_forward", "lrmsd_forward", "lrmsd_backward", "fullatom_backward"]
    # our kernels per call: schedule + forward; moments + solve + residual; gradient; backward
    launches = {"fullatom_forward": 2, "lrmsd_forward": 3, "lrmsd_backward": 1, "fullatom_backward": 1}

    calls = [
        lambda: tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, opts),
        lambda: tpl.tpl_lrmsd_forward(coords, target, na, lr, lr_ws),
        lambda: tpl.tpl_lrmsd_backward(wgt, coords, target, na, gcoords, lr_ws),
        lambda: tpl.tpl_fullatom_backward(A, S, Ln, coords, gcoords, gang, fa_ws, opts),
    ]
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        for c in calls:
            c()
    torch.cuda.synchronize()
    assert tpl.tpl_get_status() == 0
    # one CUDA graph per C-ABI call: replays cost the host a few microseconds, so
    # the events below see GPU time, not Python launch overhead
    graphs = []
    for c in calls:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            c()
        graphs.append(g)
    torch.cuda.synchronize()

    def step(ev=None):
        for i, g in enumerate(graphs):
            if ev is not None:
                ev[i].record(stream)
            g.replay()
        if ev is not None:
            ev[4].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(args.steps)])
    step_ms = per.sum(axis=1)
    total_ms = float(step_ms.sum())
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    residues = int(lengths.sum())
    value = residues * world * args.steps / (total_ms * 1e-3)

    # algorithmic bytes per launch (per-unit figures x units per launch)
    n_atoms = int(na.sum().item())
    alg = {
        "fullatom_forward": residues * (28 + 1) + 12 * n_atoms,
        "lrmsd_forward": 24 * n_atoms,
        "lrmsd_backward": 36 * n_atoms,
        "fullatom_backward": residues * (28 + 1 + 28) + 12 * n_atoms,
    }
    mean_ms = per.mean(axis=0)
    dom = int(np.argmax(mean_ms))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg[names[dom]] / (mean_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "alg_bytes": alg[names[dom]]}
    step_bytes = sum(alg.values())

    # end to end: pinned host inputs -> device, the step, loss -> host
    pa = torch.from_numpy(a).pin_memory()
    ps = torch.from_numpy(seq).pin_memory()
    pl = torch.from_numpy(lengths).pin_memory()
    tgt_host = target.cpu().pin_memory()
    loss_host = torch.empty((B,), dtype=torch.float32).pin_memory()
    h2d = pa.numel() * 4 + ps.numel() + pl.numel() * 4 + tgt_host.numel() * 4
    d2h = loss_host.numel() * 4

    def e2e_step():
        A.copy_(pa, non_blocking=True)
        S.copy_(ps, non_blocking=True)
        Ln.copy_(pl, non_blocking=True)
        target.copy_(tgt_host, non_blocking=True)
        step()
        loss_host.copy_(lr, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = 0.0
    for _ in range(min(args.steps, 200)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_ms = float(t.item())
    e2e_value = residues * world * min(args.steps, 200) / (e_ms * 1e-3)

    extra = {}
    if rank == 0 and not args.no_fp64:
        extra = fp64_comparison(tpl, torch, dev, a, seq, lengths, Amax, coords, gang, ta)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(a, seq, lengths, ta)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "residues/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"full-atom training step, {B} chains x {L} residues per GPU, "
                                   "uniform residue types, phi/psi/chi ~ U[-pi,pi], omega = pi; "
                                   "forward -> LRMSD to N(0,0.1 rad)-perturbed targets -> backward",
                       "global_batch": B * world, "seq_len": L, "parallelism": f"replicas x{world}",
                       "atoms_per_gpu": n_atoms, "l2": "flushed (512 MiB write) before every step",
                       "threads": args.threads or "default", "fullatom_backward": args.bwd},
            "breakdown_ms": dict(zip(names, [float(x) for x in mean_ms])),
            "step_alg_bytes": step_bytes,
            "step_gbs": step_bytes / (total_ms / args.steps * 1e-3) / 1e9,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "residues/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": sum(launches.values()) * args.steps,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def fp64_comparison(tpl, torch, dev, a, seq, lengths, Amax, coords32, gang32, ta):
    """Errors of the FP32 step against the plain FP64 per-chain GPU form, and that
    form's own throughput on the same workload."""
    B, _, Lmax = a.shape
    A64 = torch.from_numpy(a.astype(np.float64)).to(dev)
    S = torch.from_numpy(seq).to(dev)
    Ln = torch.from_numpy(lengths).to(dev)
    c64 = torch.zeros((B, Amax, 3), dtype=torch.float64, device=dev)
    t64 = torch.zeros_like(c64)
    na = torch.zeros((B,), dtype=torch.int32, device=dev)
    lr = torch.zeros((B,), dtype=torch.float64, device=dev)
    st = torch.zeros((B, 16), dtype=torch.float64, device=dev)
    gc = torch.zeros_like(c64)
    ga = torch.zeros_like(A64)
    w = torch.full((B,), 1.0 / B, dtype=torch.float64, device=dev)
    tpl.tpl_fullatom_forward_ref64(torch.from_numpy(ta.astype(np.float64)).to(dev), S, Ln, t64, na)

    def step64():
        tpl.tpl_fullatom_forward_ref64(A64, S, Ln, c64, na)
        tpl.tpl_lrmsd_forward_ref64(c64, t64, na, lr, st)
        tpl.tpl_lrmsd_backward_ref64(w, c64, t64, na, st, gc)
        tpl.tpl_fullatom_backward_ref64(A64, S, Ln, c64, gc, ga)

    step64()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step64()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    coord_err = float((coords32.double() - c64).abs().max().item())
    g32 = gang32.double().reshape(B, -1)
    g64 = ga.reshape(B, -1)
    grad_rel = float(((g32 - g64).norm(dim=1) / g64.norm(dim=1).clamp_min(1e-300)).max().item())
    return {"fp64_gpu_form": {"value": int(lengths.sum()) / (ms * 1e-3), "unit": "residues/s",
                              "ms_per_step": ms},
            "errors_vs_fp64_gpu": {"coord_max_abs_A": coord_err, "grad_rel_max": grad_rel}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_tpl(args)


if __name__ == "__main__":
    main()
