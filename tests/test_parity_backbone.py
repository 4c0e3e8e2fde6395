"""Backbone model (Section 3): FP32 scan kernels and the FP64 per-chain form
against the FP64 CPU oracle, element by element.

Tolerances: coordinates max-abs <= 2e-3 A (the stated FP32 bound for chains up to
1000 residues); angle gradients ||g32 - g64|| / ||g64|| <= 1e-4 per chain; the
FP64 GPU form within 1e-9 A / 1e-9 relative of the oracle (same arithmetic,
different rounding order).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_01108_gb300 as tpl
import workloads
from tests.gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

COORD_TOL = 2e-3
GRAD_TOL = 1e-4

# lengths that span several tiles of every launch shape, with ragged tails,
# empty and single-residue chains
LENGTHS = np.array([0, 1, 2, 3, 5, 63, 64, 65, 127, 255, 256, 257, 511, 700, 1000], np.int32)


def _inputs(lengths, seed, Lmax=None):
    rng = np.random.default_rng(seed)
    a = workloads.backbone_angles(lengths, rng, Lmax=Lmax)
    g = workloads.upstream_grad((len(lengths), 3 * a.shape[2], 3), rng, valid=3 * lengths)
    return a, g


def _run_fp32(a, lengths, g, opts=None, bwd_opts=None, fill=float("nan")):
    d = require_gpu()
    A = dev(a, d)
    Ln = dev(lengths, d)
    B, _, Lmax = a.shape
    coords = torch.full((B, 3 * Lmax, 3), fill, device=d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tpl.tpl_backbone_forward(A, Ln, coords, ws, opts)
    ga = torch.full_like(A, fill)
    tpl.tpl_backbone_backward(A, Ln, coords, dev(g, d), ga, ws, bwd_opts if bwd_opts is not None else opts)
    torch.cuda.synchronize()
    return host(coords), host(ga)


@pytest.fixture(scope="module")
def reference():
    a, g = _inputs(LENGTHS, 11)
    return a, g, oracle.backbone_forward(a, LENGTHS), oracle.backbone_backward(a, LENGTHS, g)


@pytest.mark.parametrize("threads,k", [(128, 2), (64, 1), (64, 4), (256, 4), (512, 2), (128, 1),
                                       (256, 1), (512, 1), (128, 4)])
def test_fp32_scan_matches_oracle(reference, threads, k):
    a, g, c64, g64 = reference
    opts = {"threads": threads, "res_per_thread": k}
    c32, ga32 = _run_fp32(a, LENGTHS, g, opts)
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    # padding written as exact zeros
    for b, L in enumerate(LENGTHS):
        assert np.all(c32[b, 3 * L:] == 0) and np.all(ga32[b, :, L:] == 0)
    assert np.all(ga32[:, 2, 0] == 0)  # omega_0 carries no gradient


@pytest.mark.parametrize("sched", [tpl.SCHED_LONGEST_FIRST, tpl.SCHED_BATCH_ORDER, tpl.SCHED_PACKED])
@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_schedules_and_backward_modes(reference, sched, bwd):
    a, g, c64, g64 = reference
    c32, ga32 = _run_fp32(a, LENGTHS, g, {"schedule": sched}, {"schedule": sched, "bwd_mode": bwd})
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL


@pytest.mark.parametrize("threads,k", [(128, 4), (64, 1), (256, 2), (512, 1)])
@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_packed_short_chains(threads, k, bwd):
    """Many chains of at most one tile: up to 8 whole chains share a tile
    (segmented scans), with empty chains and lengths not a multiple of the
    residues per thread."""
    rng = np.random.default_rng(41)
    lengths = rng.integers(0, 41, size=300).astype(np.int32)
    lengths[:7] = [0, 1, 2, 3, 4, 5, 64]
    a, g = _inputs(lengths, 42, Lmax=64)
    opts = {"threads": threads, "res_per_thread": k, "schedule": tpl.SCHED_PACKED}
    c32, ga32 = _run_fp32(a, lengths, g, opts, dict(opts, bwd_mode=bwd))
    assert np.abs(c32 - oracle.backbone_forward(a, lengths)).max() <= COORD_TOL
    g64 = oracle.backbone_backward(a, lengths, g)
    for b, L in enumerate(lengths):
        assert np.all(c32[b, 3 * L:] == 0) and np.all(ga32[b, :, L:] == 0)
        if L > 1:
            assert rel_err(ga32[b][None], g64[b][None]) <= GRAD_TOL


def test_packed_and_tiled_chains_in_one_batch():
    """Log-uniform lengths: chains longer than a tile use tiles and the
    look-back, the rest are packed."""
    rng = np.random.default_rng(43)
    lengths = workloads.lengths_loguniform(96, 1, 1000, rng)
    a, g = _inputs(lengths, 44, Lmax=1000)
    for bwd in (tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE):
        opts = {"threads": 128, "res_per_thread": 2, "schedule": tpl.SCHED_PACKED}
        c32, ga32 = _run_fp32(a, lengths, g, opts, dict(opts, bwd_mode=bwd))
        assert np.abs(c32 - oracle.backbone_forward(a, lengths)).max() <= COORD_TOL
        assert rel_err(ga32, oracle.backbone_backward(a, lengths, g)) <= GRAD_TOL


def test_results_do_not_depend_on_the_schedule(reference):
    a, g, _, _ = reference
    c1, g1 = _run_fp32(a, LENGTHS, g, {"schedule": tpl.SCHED_LONGEST_FIRST})
    c2, g2 = _run_fp32(a, LENGTHS, g, {"schedule": tpl.SCHED_BATCH_ORDER})
    assert np.array_equal(c1, c2) and np.array_equal(g1, g2)


@pytest.mark.parametrize("sched", [tpl.SCHED_PACKED, tpl.SCHED_LONGEST_FIRST])
@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_padding_flag_changes_nothing_but_the_padding(reference, sched, bwd):
    """FLAG_PADDING_ZEROED: on outputs the caller zeroed, every element equals
    the default call's; on NaN-filled outputs the real residues still do (the
    backward reads no padding of the coordinates) and only padding may differ."""
    a, g, _, _ = reference
    o = {"threads": 128, "res_per_thread": 4, "schedule": sched}
    of = dict(o, flags=tpl.FLAG_PADDING_ZEROED)
    c0, g0 = _run_fp32(a, LENGTHS, g, o, dict(o, bwd_mode=bwd))
    c1, g1 = _run_fp32(a, LENGTHS, g, of, dict(of, bwd_mode=bwd), fill=0.0)
    assert np.array_equal(c0, c1) and np.array_equal(g0, g1)
    c2, g2 = _run_fp32(a, LENGTHS, g, of, dict(of, bwd_mode=bwd))
    for b, L in enumerate(LENGTHS):
        assert np.array_equal(c2[b, :3 * L], c0[b, :3 * L])
        assert np.array_equal(g2[b, :, :L], g0[b, :, :L])


def test_fp64_per_chain_form_matches_oracle(reference):
    d = require_gpu()
    a, g, c64, g64 = reference
    A = dev(a.astype(np.float64), d)
    Ln = dev(LENGTHS, d)
    B, _, Lmax = a.shape
    coords = torch.full((B, 3 * Lmax, 3), float("nan"), dtype=torch.float64, device=d)
    tpl.tpl_backbone_forward_ref64(A, Ln, coords)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_backbone_backward_ref64(A, Ln, coords, dev(g.astype(np.float64), d), ga)
    torch.cuda.synchronize()
    assert np.abs(host(coords) - c64).max() < 1e-9
    assert rel_err(host(ga), g64) < 1e-9


def test_autograd_function_and_gradcheck_direction():
    d = require_gpu()
    lengths = np.array([40, 17], np.int32)
    a, g = _inputs(lengths, 3)
    A = dev(a, d).requires_grad_(True)
    coords = tpl.backbone(A, dev(lengths, d))
    (coords * dev(g, d)).sum().backward()
    g64 = oracle.backbone_backward(a, lengths, g)
    assert rel_err(host(A.grad), g64) <= GRAD_TOL


@pytest.fixture(scope="module")
def reference_o():
    a, g = _inputs(LENGTHS, 61)
    rng = np.random.default_rng(62)
    go = workloads.upstream_grad((len(LENGTHS), a.shape[2], 3), rng, valid=LENGTHS)
    c64, o64 = oracle.backbone_forward_o(a, LENGTHS)
    return a, g, go, c64, o64, oracle.backbone_backward_o(a, LENGTHS, g, go)


@pytest.mark.parametrize("threads,k,sched", [(128, 4, tpl.SCHED_PACKED), (128, 1, tpl.SCHED_PACKED),
                                             (128, 2, tpl.SCHED_LONGEST_FIRST), (256, 4, tpl.SCHED_BATCH_ORDER)])
@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_backbone_with_o_matches_the_oracle(reference_o, threads, k, sched, bwd):
    """The carbonyl O placed in the scan and counted in the backward (O_j after
    C_j), against the oracle; N/CA/C bit-identical to the plain forward."""
    d = require_gpu()
    a, g, go, c64, o64, g64 = reference_o
    B, _, Lmax = a.shape
    A, Ln = dev(a, d), dev(LENGTHS, d)
    opts = {"threads": threads, "res_per_thread": k, "schedule": sched, "bwd_mode": bwd}
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    c = torch.full((B, 3 * Lmax, 3), float("nan"), device=d)
    o = torch.full((B, Lmax, 3), float("nan"), device=d)
    tpl.tpl_backbone_forward_o(A, Ln, c, o, ws, opts)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_backbone_backward_o(A, Ln, c, o, dev(g, d), dev(go, d), ga, ws, opts)
    c_plain = torch.full_like(c, float("nan"))
    ws2 = torch.empty_like(ws)
    tpl.tpl_backbone_forward(A, Ln, c_plain, ws2, opts)
    torch.cuda.synchronize()
    c, o, ga = host(c), host(o), host(ga)
    assert np.array_equal(c, host(c_plain))
    assert np.abs(o - o64).max() <= COORD_TOL and np.abs(c - c64).max() <= COORD_TOL
    assert rel_err(ga, g64) <= GRAD_TOL
    for b, L in enumerate(LENGTHS):
        assert np.all(o[b, L:] == 0) and np.all(ga[b, :, L:] == 0)


def test_backbone_with_o_padding_flag():
    """FLAG_PADDING_ZEROED on the O calls: real residues unchanged on NaN-filled outputs."""
    d = require_gpu()
    lengths = np.array([0, 1, 70, 513, 300], np.int32)
    a, g = _inputs(lengths, 7, Lmax=520)
    rng = np.random.default_rng(8)
    go = workloads.upstream_grad((len(lengths), a.shape[2], 3), rng, valid=lengths)
    B, _, Lmax = a.shape
    A, Ln = dev(a, d), dev(lengths, d)
    out = []
    for flags, fill in ((0, 0.0), (tpl.FLAG_PADDING_ZEROED, float("nan"))):
        opts = {"threads": 128, "res_per_thread": 4, "flags": flags, "bwd_mode": tpl.BWD_FROM_COORDS}
        ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
        c = torch.full((B, 3 * Lmax, 3), fill, device=d)
        o = torch.full((B, Lmax, 3), fill, device=d)
        tpl.tpl_backbone_forward_o(A, Ln, c, o, ws, opts)
        ga = torch.full_like(A, fill)
        tpl.tpl_backbone_backward_o(A, Ln, c, o, dev(g, d), dev(go, d), ga, ws, opts)
        torch.cuda.synchronize()
        out.append((host(c), host(o), host(ga)))
    (c0, o0, g0), (c1, o1, g1) = out
    for b, L in enumerate(lengths):
        assert np.array_equal(c1[b, :3 * L], c0[b, :3 * L]) and np.array_equal(o1[b, :L], o0[b, :L])
        assert np.array_equal(g1[b, :, :L], g0[b, :, :L])
        assert np.all(o0[b, L:] == 0) and np.all(g0[b, :, L:] == 0)


def test_backbone_with_o_autograd_and_rejected_shapes():
    d = require_gpu()
    lengths = np.array([40, 17, 1], np.int32)
    a, g = _inputs(lengths, 5)
    rng = np.random.default_rng(6)
    go = workloads.upstream_grad((3, a.shape[2], 3), rng, valid=lengths)
    A = dev(a, d).requires_grad_(True)
    coords, o = tpl.backbone_with_o(A, dev(lengths, d))
    ((coords * dev(g, d)).sum() + (o * dev(go, d)).sum()).backward()
    assert rel_err(host(A.grad), oracle.backbone_backward_o(a, lengths, g, go)) <= GRAD_TOL
    B, _, Lmax = a.shape
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    with pytest.raises(tpl.TplError):
        tpl.tpl_backbone_forward_o(A.detach(), dev(lengths, d), torch.empty((B, 3 * Lmax, 3), device=d),
                                   torch.empty((B, Lmax, 3), device=d), ws, {"threads": 512, "res_per_thread": 2})


@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_long_chains_precision_stress(bwd):
    """4 chains x 10000 residues (the precision-stress shape at reduced batch).
    The 2e-3 A coordinate bound is stated for chains up to 1000 residues, so at
    10000 the drift is bounded loosely and reported; the angle-gradient bound
    (1e-4 relative) holds at every length."""
    lengths = np.full(4, 10000, np.int32)
    a, g = _inputs(lengths, 5)
    opts = {"threads": 256, "res_per_thread": 4}
    c32, ga32 = _run_fp32(a, lengths, g, opts, dict(opts, bwd_mode=bwd))
    c64 = oracle.backbone_forward(a, lengths)
    drift = np.abs(c32 - c64).max()
    print(f"drift at 10000 residues {drift:.3e} A")
    assert drift < 1e-2, drift
    # first 1000 residues stay inside the bound
    assert np.abs(c32[:, :3000] - c64[:, :3000]).max() <= COORD_TOL
    err = rel_err(ga32, oracle.backbone_backward(a, lengths, g))
    print(f"angle-gradient relative error at 10000 residues {err:.3e}")
    assert err <= GRAD_TOL, err


def test_bad_length_sets_status_without_faulting():
    d = require_gpu()
    tpl.tpl_get_status()  # clear
    lengths = np.array([5, 9999, -3], np.int32)  # > Lmax and < 0
    a, g = _inputs(np.array([5, 8, 0], np.int32), 1, Lmax=8)
    c32, _ = _run_fp32(a, lengths, g)
    st = tpl.tpl_get_status()
    assert st & tpl.STATUS_BAD_LENGTH
    assert np.all(c32[2] == 0)  # negative length treated as empty


def test_backward_without_forward_workspace_flags_and_zeroes():
    d = require_gpu()
    tpl.tpl_get_status()
    lengths = np.array([30, 12], np.int32)
    a, g = _inputs(lengths, 9)
    A, Ln = dev(a, d), dev(lengths, d)
    B, _, Lmax = a.shape
    ws = torch.zeros(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_backbone_backward(A, Ln, None, dev(g, d), ga, ws)
    assert tpl.tpl_get_status() & tpl.STATUS_BAD_WORKSPACE
    assert torch.all(ga == 0)


def test_autotuner_picks_a_valid_shape_and_its_results_match():
    d = require_gpu()
    rng = np.random.default_rng(45)
    lengths = workloads.lengths_loguniform(64, 20, 600, rng)
    a, g = _inputs(lengths, 46, Lmax=600)
    A, Ln, G = dev(a, d), dev(lengths, d), dev(g, d)
    B, _, Lmax = a.shape
    coords = torch.empty((B, 3 * Lmax, 3), device=d)
    ga = torch.empty_like(A)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    best, ms = tpl.tpl_backbone_autotune(A, Ln, coords, G, ga, ws, bwd_mode=tpl.BWD_FROM_COORDS)
    assert ms > 0 and best.threads in (64, 128, 256, 512) and best.res_per_thread in (1, 2, 4)
    assert best.schedule in (tpl.SCHED_PACKED, tpl.SCHED_LONGEST_FIRST)
    c32, ga32 = _run_fp32(a, lengths, g, best)
    assert np.abs(c32 - oracle.backbone_forward(a, lengths)).max() <= COORD_TOL
    assert rel_err(ga32, oracle.backbone_backward(a, lengths, g)) <= GRAD_TOL


def test_lrmsd_step_autotuner_picks_a_valid_shape_and_its_step_matches_the_oracle():
    """tpl_backbone_lrmsd_autotune times forward, LRMSD forward and the fused
    backward per candidate; the step with its pick agrees with the oracle."""
    d = require_gpu()
    rng = np.random.default_rng(49)
    lengths = workloads.lengths_loguniform(64, 20, 600, rng)
    a, _ = _inputs(lengths, 50, Lmax=600)
    ta = workloads.perturb_angles(a, lengths, rng)
    B, _, Lmax = a.shape
    A, Ln = dev(a, d), dev(lengths, d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, 3 * Lmax, 3), device=d)
    tpl.tpl_backbone_forward(dev(ta, d), Ln, tgt, ws)
    coords = torch.zeros_like(tgt)
    na = dev((3 * lengths).astype(np.int32), d)
    lr = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, 3 * Lmax), dtype=torch.uint8, device=d)
    w = dev(np.linspace(-1.0, 2.0, B).astype(np.float32), d)
    ga = torch.empty_like(A)
    best, ms = tpl.tpl_backbone_lrmsd_autotune(A, Ln, coords, tgt, na, w, lr, lr_ws, ga, ws)
    assert ms > 0 and best.threads in (64, 128, 256, 512) and best.res_per_thread in (1, 2, 4)
    assert best.schedule in (tpl.SCHED_PACKED, tpl.SCHED_LONGEST_FIRST)
    assert best.bwd_mode == tpl.BWD_FROM_COORDS
    ga.fill_(float("nan"))
    lr.fill_(float("nan"))
    tpl.tpl_backbone_forward(A, Ln, coords, ws, best)
    tpl.tpl_lrmsd_forward(coords, tgt, na, lr, lr_ws)
    tpl.tpl_backbone_backward_lrmsd(A, Ln, coords, tgt, w, lr_ws, ga, ws, best)
    torch.cuda.synchronize()
    c32, t32 = host(coords), host(tgt)
    assert np.abs(host(lr) - oracle.lrmsd_forward(c32, t32, 3 * lengths)).max() <= 1e-5
    g64 = oracle.lrmsd_backward(host(w).astype(np.float64), c32, t32, 3 * lengths)
    assert rel_err(host(ga), oracle.backbone_backward(a, lengths, g64)) <= GRAD_TOL


@pytest.mark.parametrize("threads,k,sched", [(128, 4, tpl.SCHED_PACKED), (256, 2, tpl.SCHED_LONGEST_FIRST),
                                              (64, 1, tpl.SCHED_PACKED)])
def test_fused_lrmsd_backward_equals_the_two_calls_and_the_oracle(threads, k, sched):
    """tpl_backbone_backward_lrmsd = tpl_lrmsd_backward + tpl_backbone_backward
    (FROM_COORDS), packed and tiled chains, against the oracle chain."""
    d = require_gpu()
    rng = np.random.default_rng(47)
    lengths = workloads.lengths_loguniform(40, 1, 900, rng)
    lengths[:3] = [0, 1, 900]
    a, _ = _inputs(lengths, 48, Lmax=900)
    ta = workloads.perturb_angles(a, lengths, rng)
    B, _, Lmax = a.shape
    A, Ln = dev(a, d), dev(lengths, d)
    opts = {"threads": threads, "res_per_thread": k, "schedule": sched}
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, 3 * Lmax, 3), device=d)
    tpl.tpl_backbone_forward(dev(ta, d), Ln, tgt, ws, opts)
    coords = torch.zeros_like(tgt)
    tpl.tpl_backbone_forward(A, Ln, coords, ws, opts)
    na = dev((3 * lengths).astype(np.int32), d)
    lr = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, 3 * Lmax), dtype=torch.uint8, device=d)
    tpl.tpl_lrmsd_forward(coords, tgt, na, lr, lr_ws)
    w = dev(np.linspace(-1.0, 2.0, B).astype(np.float32), d)
    ga_fused = torch.full_like(A, float("nan"))
    tpl.tpl_backbone_backward_lrmsd(A, Ln, coords, tgt, w, lr_ws, ga_fused, ws, opts)
    gc = torch.empty_like(coords)
    tpl.tpl_lrmsd_backward(w, coords, tgt, na, gc, lr_ws)
    ga_two = torch.full_like(A, float("nan"))
    tpl.tpl_backbone_backward(A, Ln, coords, gc, ga_two, ws, dict(opts, bwd_mode=tpl.BWD_FROM_COORDS))
    torch.cuda.synchronize()
    f = host(ga_fused)
    assert np.all(np.isfinite(f))
    assert rel_err(f, host(ga_two)) <= 1e-5
    g64 = oracle.lrmsd_backward(host(w).astype(np.float64), host(coords), host(tgt), 3 * lengths)
    ga64 = oracle.backbone_backward(a, lengths, g64)
    # a one-residue chain is a rigid N-CA-C triangle: input and target are
    # congruent, LRMSD is zero up to rounding and its gradient is undefined
    m = lengths >= 2
    assert rel_err(f[m], ga64[m]) <= GRAD_TOL
    for b, L in enumerate(lengths):
        assert np.all(f[b, :, L:] == 0)


def _step_inputs(seed, n=40, Lmax=900):
    rng = np.random.default_rng(seed)
    lengths = workloads.lengths_loguniform(n, 1, Lmax, rng)
    lengths[:4] = [0, 1, 2, Lmax]
    a, _ = _inputs(lengths, seed + 1, Lmax=Lmax)
    ta = workloads.perturb_angles(a, lengths, rng)
    return a, ta, lengths


def _run_step(a, ta, lengths, opts, fill=0.0, w=None):
    d = require_gpu()
    B, _, Lmax = a.shape
    A, Ln = dev(a, d), dev(lengths, d)
    tgt = torch.zeros((B, 3 * Lmax, 3), device=d)
    ws0 = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tpl.tpl_backbone_forward(dev(ta, d), Ln, tgt, ws0)
    if w is None:
        w = np.linspace(-1.0, 2.0, B).astype(np.float32)
    W = dev(w, d)
    ws = torch.empty(tpl.tpl_backbone_lrmsd_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    coords = torch.full((B, 3 * Lmax, 3), fill, device=d)
    lr = torch.full((B,), float("nan"), device=d)
    ga = torch.full_like(A, fill)
    tpl.tpl_backbone_lrmsd_step(A, Ln, tgt, W, coords, lr, ga, ws, opts)
    torch.cuda.synchronize()
    return host(coords), host(lr), host(ga), host(tgt), w


@pytest.mark.parametrize("threads,k,sched", [(128, 4, tpl.SCHED_PACKED), (256, 4, tpl.SCHED_PACKED),
                                             (128, 2, tpl.SCHED_LONGEST_FIRST), (512, 2, tpl.SCHED_PACKED),
                                             (256, 2, tpl.SCHED_BATCH_ORDER)])
def test_training_step_matches_the_separate_calls_and_the_oracle(threads, k, sched):
    """tpl_backbone_lrmsd_step: chains done whole in one CTA (packs, one-tile
    chains) and chains of several tiles (tile moments, eigen-solve, backward
    with residual sums) against the three separate calls and the oracle chain
    (Section 3 forward, Section 4 LRMSD and gradient, Eq. 2)."""
    d = require_gpu()
    a, ta, lengths = _step_inputs(51)
    B, _, Lmax = a.shape
    opts = {"threads": threads, "res_per_thread": k, "schedule": sched}
    c, lr, ga, tgt, w = _run_step(a, ta, lengths, opts, fill=float("nan"))
    # the separate calls
    A, Ln = dev(a, d), dev(lengths, d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    c2 = torch.zeros((B, 3 * Lmax, 3), device=d)
    tpl.tpl_backbone_forward(A, Ln, c2, ws, opts)
    na = dev((3 * lengths).astype(np.int32), d)
    lr2 = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, 3 * Lmax), dtype=torch.uint8, device=d)
    T = dev(tgt, d)
    tpl.tpl_lrmsd_forward(c2, T, na, lr2, lr_ws)
    ga2 = torch.zeros_like(A)
    tpl.tpl_backbone_backward_lrmsd(A, Ln, c2, T, dev(w, d), lr_ws, ga2, ws, opts)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(ga)) and np.all(np.isfinite(lr))
    assert np.abs(c - host(c2)).max() <= 1e-4
    assert np.abs(lr - host(lr2)).max() <= 1e-5
    m = lengths >= 2  # a one-residue chain is congruent to its target: no gradient
    # both FP32 paths, their LRMSD moments summed in different orders
    assert rel_err(ga[m], host(ga2)[m]) <= GRAD_TOL
    # the oracle chain
    assert np.abs(c - oracle.backbone_forward(a, lengths)).max() <= COORD_TOL
    assert np.abs(lr - oracle.lrmsd_forward(c, tgt, 3 * lengths)).max() <= 1e-5
    g64 = oracle.lrmsd_backward(w.astype(np.float64), c, tgt, 3 * lengths)
    assert rel_err(ga[m], oracle.backbone_backward(a, lengths, g64)[m]) <= GRAD_TOL
    for b, L in enumerate(lengths):
        assert np.all(c[b, 3 * L:] == 0) and np.all(ga[b, :, L:] == 0)


def test_training_step_padding_flag_and_shape_checks():
    """FLAG_PADDING_ZEROED leaves the real residues unchanged; RECOMPUTE and
    unsupported shapes are rejected before any launch."""
    a, ta, lengths = _step_inputs(53, n=24, Lmax=600)
    o = {"threads": 128, "res_per_thread": 4}
    c0, lr0, g0, _, _ = _run_step(a, ta, lengths, o)
    c1, lr1, g1, _, _ = _run_step(a, ta, lengths, dict(o, flags=tpl.FLAG_PADDING_ZEROED), fill=float("nan"))
    assert np.array_equal(lr0, lr1)
    for b, L in enumerate(lengths):
        assert np.array_equal(c1[b, :3 * L], c0[b, :3 * L]) and np.array_equal(g1[b, :, :L], g0[b, :, :L])
    for bad in ({"bwd_mode": tpl.BWD_RECOMPUTE}, {"threads": 64, "res_per_thread": 1}, {"threads": 512, "res_per_thread": 4}):
        with pytest.raises(tpl.TplError):
            _run_step(a, ta, lengths, bad)


def test_packed_schedule_is_deterministic():
    """The packs come from a stable sort (no atomics decide the order), so the
    packed results are bit-identical from run to run."""
    rng = np.random.default_rng(49)
    lengths = workloads.lengths_loguniform(3000, 1, 800, rng)
    a, g = _inputs(lengths, 50, Lmax=800)
    opts = {"threads": 128, "res_per_thread": 4, "schedule": tpl.SCHED_PACKED}
    c1, g1 = _run_fp32(a, lengths, g, opts, dict(opts, bwd_mode=tpl.BWD_FROM_COORDS))
    _run_fp32(a[:7], lengths[:7], g[:7], opts)  # something else in between
    c2, g2 = _run_fp32(a, lengths, g, opts, dict(opts, bwd_mode=tpl.BWD_FROM_COORDS))
    assert np.array_equal(c1, c2) and np.array_equal(g1, g2)


def _free_omega(a, lengths, rng):
    """omega per residue: trans (pi +- 0.1), cis (0 +- 0.1) or uniform, in thirds."""
    B, _, Lmax = a.shape
    kind = rng.integers(0, 3, size=(B, Lmax))
    om = np.where(kind == 0, np.pi + rng.normal(0, 0.1, (B, Lmax)),
                  np.where(kind == 1, rng.normal(0, 0.1, (B, Lmax)), rng.uniform(-np.pi, np.pi, (B, Lmax))))
    a = a.copy()
    a[:, 2] = (om * (np.arange(Lmax)[None, :] < lengths[:, None])).astype(np.float32)
    return a


@pytest.mark.parametrize("bwd", [tpl.BWD_FROM_COORDS, tpl.BWD_RECOMPUTE])
def test_free_omega_cis_and_trans(bwd):
    """omega is an input (reading 3), not fixed at pi: with cis, trans and
    arbitrary peptide bonds the coordinates, all angle gradients and the omega
    row of the gradient on its own match the oracle."""
    rng = np.random.default_rng(57)
    a, g = _inputs(LENGTHS, 58)
    a = _free_omega(a, LENGTHS, rng)
    c64 = oracle.backbone_forward(a, LENGTHS)
    g64 = oracle.backbone_backward(a, LENGTHS, g)
    c32, ga32 = _run_fp32(a, LENGTHS, g, {"threads": 128, "res_per_thread": 4},
                          {"threads": 128, "res_per_thread": 4, "bwd_mode": bwd})
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    assert rel_err(ga32[:, 2], g64[:, 2]) <= GRAD_TOL
    assert np.all(ga32[:, 2, 0] == 0)


def test_quadratic_comparator_matches_the_scan_and_the_oracle(reference):
    """tpl_backbone_backward_quadratic (the paper's O(L^2) sums of Eq. 2 on the
    GPU) agrees with the oracle and with the suffix-scan backward on the same
    FP32 coordinates; padding and omega_0 are zero."""
    a, g, c64, g64 = reference
    d = require_gpu()
    c32, ga_scan = _run_fp32(a, LENGTHS, g, None, {"bwd_mode": tpl.BWD_FROM_COORDS})
    B, _, Lmax = a.shape
    ga_q = torch.full((B, 3, Lmax), float("nan"), device=d)
    tpl.tpl_backbone_backward_quadratic(dev(LENGTHS, d), dev(c32, d), dev(g, d), ga_q)
    torch.cuda.synchronize()
    gq = host(ga_q)
    assert np.all(np.isfinite(gq))
    assert rel_err(gq, g64) <= GRAD_TOL
    assert rel_err(gq, ga_scan) <= 1e-5
    for b, L in enumerate(LENGTHS):
        assert np.all(gq[b, :, L:] == 0)
    assert np.all(gq[:, 2, 0] == 0)
