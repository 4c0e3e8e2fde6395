"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Each rank runs a replica on a batch of its own (weak scaling); the ranks
exchange only the elapsed time, reduced with MAX, and the whole-job value
counts the units of every rank.  The reference arm runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import bench

rank, world, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
args = bench.parse()
d = bench.make_inputs(args, rank)
# batch identity: a digest of this rank's inputs, gathered on every rank
dig = float(np.asarray(d["angles"], np.float64).sum())
got = [None] * world
dist.all_gather_object(got, (rank, dig, d["angles"].shape, int(d["lengths"].sum())))
elapsed = 10.0 + 5.0 * rank          # a slower rank 1
mx = bench.max_over_ranks(elapsed, torch.device("cpu"), world)
units = int(d["lengths"].sum())
val = bench.job_throughput(units, world, 3, mx)
if rank == 0:
    print(json.dumps({{"got": [[g[0], g[1], list(g[2]), g[3]] for g in got], "max": mx, "value": val,
                      "units": units}}))
dist.barrier()
dist.destroy_process_group()
"""


def _launch(argv, script, world=2):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", script, *argv], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


@pytest.mark.parametrize("workload", ["training_step", "backbone_uneven"])
def test_two_rank_replicas_reduce_time_with_max(workload):
    outs = _launch(["--workload", workload, "--batch", "4", "--length", "32"],
                   WORKER.format(root=ROOT))
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert outs[1].strip() == ""                      # only rank 0 prints
    (r0, d0, s0, u0), (r1, d1, s1, u1) = line["got"]
    assert (r0, r1) == (0, 1)
    assert s0 == s1                                   # same shapes per rank
    assert d0 != d1                                   # but independent batches
    assert line["max"] == 15.0                        # the slowest rank's time
    assert np.isclose(line["value"], line["units"] * 2 * 3 / 15.0e-3)


def test_reference_arm_runs_on_rank0_only():
    script = ("import sys; sys.path.insert(0, %r); import bench; bench.main()" % ROOT)
    port = _free_port()
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r = subprocess.run([sys.executable, "-c", script, "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--batch", "2", "--length", "16"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and r.stdout.strip() == ""
