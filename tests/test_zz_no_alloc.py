"""The allocation-free LRMSD forward (tpl_lrmsd_forward_noalloc).

Some callers can neither allocate device memory nor pass a workspace, so this
entry point keeps its scratch in a fixed array inside the library.  The test
calls it through the C ABI several times in a row (the array keeps the
previous call's contents) and checks each result against the workspace-based
tpl_lrmsd_forward: both paths run the same deterministic kernels, so the
results must be identical.  The calls cover both shapes of the forward's
one-CTA-per-pair kernel: the wide one (a batch that fits one wave) and the
compact one (larger batches), the latter at the documented limit (4096 pairs
of 8192 atoms, every per-pair slot of the array in use).  It collects last so a failure
here leaves every other test already run, and it passes alone in a fresh
process as well as after the others.
"""
import numpy as np
import pytest
import torch

import paper_1812_01108_gb300 as tpl
import workloads
from tests.gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

MAX_PAIRS, MAX_ATOMS = 4096, 8192  # the limits include/tpl.h states


def _with_workspace(X, Y, N):
    P, Nmax, _ = X.shape
    out = torch.full((P,), float("nan"), device=X.device)
    ws = torch.empty(tpl.tpl_lrmsd_workspace_size(P, Nmax), dtype=torch.uint8, device=X.device)
    tpl.tpl_lrmsd_forward(X, Y, N, out, ws)
    return out


def _no_alloc(X, Y, N):
    out = torch.full((X.shape[0],), float("nan"), device=X.device)
    tpl.tpl_lrmsd_forward_noalloc(X, Y, N, out)
    return out


def test_no_alloc_forward_matches_workspace_forward_on_consecutive_calls():
    d = require_gpu()
    rng = np.random.default_rng(20240)
    big = workloads.lrmsd_clouds(MAX_PAIRS, 100, MAX_ATOMS, rng, Nmax=MAX_ATOMS)
    small = workloads.lrmsd_clouds(57, 3, 900, rng)
    big2 = workloads.lrmsd_clouds(MAX_PAIRS, 3, 2000, rng)
    assert tpl.tpl_lrmsd_forward_launches(MAX_PAIRS) == 1 and tpl.tpl_lrmsd_forward_launches(57) == 1
    # compact CTAs at the limit, then wide ones, then compact ones again over
    # the array the first call left behind
    for x, y, n in (big, small, big2):
        X, Y, N = dev(x, d), dev(y, d), dev(n, d)
        got = host(_no_alloc(X, Y, N))
        ref = host(_with_workspace(X, Y, N))
        torch.cuda.synchronize()
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref)
        del X, Y, N


def test_no_alloc_forward_rejects_sizes_beyond_its_limits():
    d = require_gpu()
    # too many atoms per pair
    x = torch.zeros((2, MAX_ATOMS + 4, 3), device=d)
    n = torch.full((2,), MAX_ATOMS + 4, dtype=torch.int32, device=d)
    out = torch.full((2,), 7.0, device=d)
    with pytest.raises(tpl.TplError) as err:
        tpl.tpl_lrmsd_forward_noalloc(x, x, n, out)
    assert err.value.code == 2  # TPL_ERR_BAD_SHAPE
    # too many pairs
    x = torch.zeros((MAX_PAIRS + 1, 8, 3), device=d)
    n = torch.full((MAX_PAIRS + 1,), 8, dtype=torch.int32, device=d)
    out = torch.full((MAX_PAIRS + 1,), 7.0, device=d)
    with pytest.raises(tpl.TplError) as err:
        tpl.tpl_lrmsd_forward_noalloc(x, x, n, out)
    assert err.value.code == 2
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)  # nothing was launched
