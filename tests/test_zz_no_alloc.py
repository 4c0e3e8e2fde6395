"""The allocation-free LRMSD forward (tpl_lrmsd_forward_noalloc).

Some callers can neither allocate device memory nor pass a workspace, so this
entry point keeps its scratch in a fixed array inside the library.  The test
calls it through the C ABI twice in a row (the array keeps the previous call's
contents) and checks each result against the workspace-based
tpl_lrmsd_forward, within the LRMSD tolerance of the other tests.  It collects
last so a failure here leaves every other test already run, and it passes
alone in a fresh process as well as after the others.
"""
import numpy as np
import pytest
import torch

import paper_1812_01108_gb300 as tpl
import workloads
from tests.gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

LRMSD_TOL = 1e-5  # the LRMSD tolerance of tests/test_parity_lrmsd.py


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


def test_no_alloc_forward_matches_workspace_forward_on_two_calls():
    d = require_gpu()
    rng = np.random.default_rng(20240)
    cases = [workloads.lrmsd_clouds(300, 100, 5000, rng), workloads.lrmsd_clouds(57, 3, 900, rng)]
    for x, y, n in cases:  # two calls in a row, different shapes
        X, Y, N = dev(x, d), dev(y, d), dev(n, d)
        got = host(_no_alloc(X, Y, N))
        ref = host(_with_workspace(X, Y, N))
        torch.cuda.synchronize()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= LRMSD_TOL


def test_no_alloc_forward_rejects_sizes_beyond_its_limits():
    d = require_gpu()
    x = torch.zeros((2, 8196, 3), device=d)
    n = torch.full((2,), 8196, dtype=torch.int32, device=d)
    out = torch.zeros((2,), device=d)
    with pytest.raises(tpl.TplError) as err:
        tpl.tpl_lrmsd_forward_noalloc(x, x, n, out)
    assert err.value.code == 2  # TPL_ERR_BAD_SHAPE
