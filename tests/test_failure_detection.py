"""Failure detection without a GPU fault.

A cross-CTA signal that never arrives (a flag that nothing sets) must end
the bounded wait with TPL_STATUS_TIMEOUT, and the context must stay usable:
the next calls run and give correct results.  Bad data that the host cannot
see (a length outside [0, Lmax]) becomes a status bit as well.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1812_01108_gb300 as tpl
import workloads
from tests.gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu


def _backbone_ok(d):
    rng = workloads.rng_for(0, salt=21)
    lengths = np.array([64, 17, 0, 40], np.int32)
    a = workloads.backbone_angles(lengths, rng, Lmax=64)
    coords = torch.empty((4, 192, 3), device=d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(4, 64), dtype=torch.uint8, device=d)
    tpl.tpl_backbone_forward(dev(a, d), dev(lengths, d), coords, ws)
    torch.cuda.synchronize()
    return np.abs(host(coords) - oracle.backbone_forward(a, lengths)).max()


def test_lost_signal_times_out_and_context_survives():
    d = require_gpu()
    tpl.tpl_get_status()  # clear
    flag = torch.zeros(4, dtype=torch.int32, device=d)
    t0 = time.perf_counter()
    tpl.tpl_selftest_wait_timeout(flag)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert tpl.tpl_get_status() & tpl.STATUS_TIMEOUT
    assert waited < 30.0
    # the context is intact: a normal call afterwards is correct and clean
    assert _backbone_ok(d) < 2e-3
    assert tpl.tpl_get_status() == 0


def test_bad_length_is_a_status_bit_not_a_fault():
    d = require_gpu()
    tpl.tpl_get_status()
    lengths = np.array([64, 70, -3, 10], np.int32)  # 70 > Lmax, -3 < 0
    a = np.zeros((4, 3, 64), np.float32)
    coords = torch.full((4, 192, 3), float("nan"), device=d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(4, 64), dtype=torch.uint8, device=d)
    tpl.tpl_backbone_forward(dev(a, d), dev(lengths, d), coords, ws)
    torch.cuda.synchronize()
    assert tpl.tpl_get_status() & tpl.STATUS_BAD_LENGTH
    assert np.all(np.isfinite(host(coords)))
    assert _backbone_ok(d) < 2e-3
