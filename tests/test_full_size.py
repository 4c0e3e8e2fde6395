"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (autotuned launch shape, fused LRMSD backward, one step of the bench's
own calls), on sampled chains and pairs that the FP64 oracle computes one by
one on the same inputs.

  training step  256 chains x 700 residues, full atom
  uneven batch   4096 backbone chains, lengths log-uniform in [50, 1000]
  LRMSD batch    16384 pairs of U{100..5000} atoms
"""
import numpy as np
import pytest
import torch

import bench
import oracle
import paper_1812_01108_gb300 as tpl
from tests.gpu_util import host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

COORD_TOL, GRAD_TOL, LRMSD_TOL = 2e-3, 1e-4, 1e-5


def _one_step(workload):
    d_ = require_gpu()
    tpl.tpl_get_status()  # reads and clears what earlier tests left in the status word
    args = bench.parse(["--workload", workload])
    d = bench.make_inputs(args, 0)
    st = bench.SETUP[workload](args, tpl, torch, d_, d)
    for _, c in st.calls:
        c()
    torch.cuda.synchronize()
    assert tpl.tpl_get_status() == 0
    return d, {k: host(v) for k, v in st.outputs.items()}


def test_training_step_256x700_sampled_chains():
    d, o = _one_step("training_step")
    a, seq, L, ta = d["angles"], d["seq"], d["lengths"], d["target_angles"]
    for b in (0, 1, 97, 255):
        s = slice(b, b + 1)
        c64, n64 = oracle.fullatom_forward(a[s], seq[s], L[s], o["coords"].shape[1])
        t64, _ = oracle.fullatom_forward(ta[s], seq[s], L[s], o["coords"].shape[1])
        assert o["num_atoms"][b] == n64[0]
        assert np.abs(o["coords"][s] - c64).max() <= COORD_TOL
        assert np.abs(o["target"][s] - t64).max() <= COORD_TOL
        # LRMSD and its chained gradient on the GPU's own FP32 coordinates
        x, y = o["target"][s], o["coords"][s]
        assert abs(o["lrmsd"][b] - oracle.lrmsd_forward(y, x, n64)[0]) <= LRMSD_TOL
        g = oracle.lrmsd_backward(o["weights"][s].astype(np.float64), y, x, n64)
        assert rel_err(o["grad_angles"][s], oracle.fullatom_backward(a[s], seq[s], L[s], g)) <= GRAD_TOL


def test_uneven_backbone_4096_sampled_chains():
    d, o = _one_step("backbone_uneven")
    a, L, ta = d["angles"], d["lengths"], d["target_angles"]
    order = np.argsort(L)
    picks = sorted(set([int(order[0]), int(order[1]), int(order[-1]), int(order[-2])] +
                       [int(i) for i in np.random.default_rng(5).choice(len(L), 12, replace=False)]))
    for b in picks:
        s = slice(b, b + 1)
        assert np.abs(o["coords"][s] - oracle.backbone_forward(a[s], L[s])).max() <= COORD_TOL
        assert np.abs(o["target"][s] - oracle.backbone_forward(ta[s], L[s])).max() <= COORD_TOL
        x, y, n = o["target"][s], o["coords"][s], 3 * L[s]
        assert abs(o["lrmsd"][b] - oracle.lrmsd_forward(y, x, n)[0]) <= LRMSD_TOL
        g = oracle.lrmsd_backward(o["weights"][s].astype(np.float64), y, x, n)
        assert rel_err(o["grad_angles"][s], oracle.backbone_backward(a[s], L[s], g)) <= GRAD_TOL


def test_lrmsd_batch_16384_sampled_pairs():
    d, o = _one_step("lrmsd_batch")
    x, y, n = d["target"], d["input"], d["num_atoms"]
    picks = np.random.default_rng(6).choice(len(n), 48, replace=False)
    picks = np.concatenate([picks, [int(np.argmin(n)), int(np.argmax(n))]])
    w = o["weights"].astype(np.float64)
    for p in picks:
        s = slice(p, p + 1)
        assert abs(o["lrmsd"][p] - oracle.lrmsd_forward(y[s], x[s], n[s])[0]) <= LRMSD_TOL
        assert rel_err(o["grad_input"][s], oracle.lrmsd_backward(w[s], y[s], x[s], n[s])) <= GRAD_TOL
