"""Full-atom model (Section 2): FP32 scan kernels and the FP64 per-chain form
against the FP64 CPU oracle, element by element.  Tolerances as for the backbone:
coordinates <= 2e-3 A, gradients <= 1e-4 relative per chain, FP64 form 1e-9.
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
LRMSD_TOL = 1e-5
LENGTHS = np.array([0, 1, 2, 31, 64, 255, 256, 257, 350, 513, 700], np.int32)
# launch shapes (threads, residues per thread) of the full-atom kernels
SHAPES = [(128, 1), (256, 1), (384, 1), (128, 2), (192, 2), (64, 4), (192, 4)]
RECOMPUTE_SHAPES = [(128, 1), (256, 1), (384, 1)]  # frames rebuilt from the angles: one residue per thread


def _inputs(lengths, seed, omega_noise=0.0):
    rng = np.random.default_rng(seed)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    if omega_noise:
        a[:, 2] += rng.normal(0, omega_noise, size=a[:, 2].shape).astype(np.float32)
        a *= (np.arange(a.shape[2])[None, :] < lengths[:, None])[:, None, :]
    Amax = workloads.pad_to(max(oracle.max_atoms(seq, lengths), 1))
    g = workloads.upstream_grad((len(lengths), Amax, 3), rng)
    return a, seq, g, Amax


def _run_fp32(a, seq, lengths, g, Amax, opts=None, from_coords=False, fill=float("nan")):
    d = require_gpu()
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    B, _, Lmax = a.shape
    coords = torch.full((B, Amax, 3), fill, device=d)
    na = torch.full((B,), -1, dtype=torch.int32, device=d)
    ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tpl.tpl_fullatom_forward(A, S, Ln, coords, na, ws, opts)
    ga = torch.full_like(A, fill)
    tpl.tpl_fullatom_backward(A, S, Ln, coords if from_coords else None, dev(g, d), ga, ws, opts)
    torch.cuda.synchronize()
    return host(coords), host(na), host(ga)


@pytest.fixture(scope="module")
def reference():
    a, seq, g, Amax = _inputs(LENGTHS, 21, omega_noise=0.2)
    c64, na64 = oracle.fullatom_forward(a, seq, LENGTHS, Amax)
    # the upstream gradient is defined on real atoms only
    g = g * (np.arange(Amax)[None, :] < na64[:, None])[:, :, None]
    g64 = oracle.fullatom_backward(a, seq, LENGTHS, g)
    return a, seq, g.astype(np.float32), Amax, c64, na64, g64


@pytest.mark.parametrize("shape,from_coords", [(s, True) for s in SHAPES] + [(s, False) for s in RECOMPUTE_SHAPES])
def test_fp32_scan_matches_oracle(reference, shape, from_coords):
    a, seq, g, Amax, c64, na64, g64 = reference
    opts = {"threads": shape[0], "res_per_thread": shape[1]}
    c32, na32, ga32 = _run_fp32(a, seq, LENGTHS, g, Amax, opts, from_coords)
    assert np.array_equal(na32, na64)  # atom counts bit-exact
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    for b in range(len(LENGTHS)):
        assert np.all(c32[b, na64[b]:] == 0)
        assert np.all(ga32[b, :, LENGTHS[b]:] == 0)
    # unused chi rows and omega_0 are exactly zero
    for b, L in enumerate(LENGTHS):
        for j in range(L):
            nchi = tpl.residue_table(int(seq[b, j]))[2]
            assert np.all(ga32[b, 3 + nchi:, j] == 0)
        if L:
            assert ga32[b, 2, 0] == 0


@pytest.mark.parametrize("shape,from_coords", [((192, 2), True), ((64, 4), True), ((256, 1), False)])
def test_schedule_independent_and_deterministic(reference, shape, from_coords):
    a, seq, g, Amax, *_ = reference
    o = {"threads": shape[0], "res_per_thread": shape[1]}
    r1 = _run_fp32(a, seq, LENGTHS, g, Amax, dict(o, schedule=tpl.SCHED_LONGEST_FIRST), from_coords)
    r2 = _run_fp32(a, seq, LENGTHS, g, Amax, dict(o, schedule=tpl.SCHED_BATCH_ORDER), from_coords)
    r3 = _run_fp32(a, seq, LENGTHS, g, Amax, dict(o, schedule=tpl.SCHED_BATCH_ORDER), from_coords)
    for x, y, z in zip(r1, r2, r3):
        assert np.array_equal(x, y) and np.array_equal(y, z)


@pytest.mark.parametrize("shape,from_coords", [((384, 1), True), ((192, 2), True), ((256, 1), False)])
def test_padding_flag_changes_nothing_but_the_padding(reference, shape, from_coords):
    """FLAG_PADDING_ZEROED: on outputs the caller zeroed, every element equals
    the default call's; on NaN-filled outputs the real atoms and residues
    still do and only padding may differ."""
    a, seq, g, Amax, c64, na64, _ = reference
    o = {"threads": shape[0], "res_per_thread": shape[1]}
    of = dict(o, flags=tpl.FLAG_PADDING_ZEROED)
    r0 = _run_fp32(a, seq, LENGTHS, g, Amax, o, from_coords)
    r1 = _run_fp32(a, seq, LENGTHS, g, Amax, of, from_coords, fill=0.0)
    assert all(np.array_equal(x, y) for x, y in zip(r0, r1))
    c2, na2, g2 = _run_fp32(a, seq, LENGTHS, g, Amax, of, from_coords)
    assert np.array_equal(na2, na64)
    for b, L in enumerate(LENGTHS):
        assert np.array_equal(c2[b, :na64[b]], r0[0][b, :na64[b]])
        assert np.array_equal(g2[b, :, :L], r0[2][b, :, :L])


def test_fp64_per_chain_form_matches_oracle(reference):
    d = require_gpu()
    a, seq, g, Amax, c64, na64, g64 = reference
    A = dev(a.astype(np.float64), d)
    S, Ln = dev(seq, d), dev(LENGTHS, d)
    B = a.shape[0]
    coords = torch.full((B, Amax, 3), float("nan"), dtype=torch.float64, device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    tpl.tpl_fullatom_forward_ref64(A, S, Ln, coords, na)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward_ref64(A, S, Ln, coords, dev(g.astype(np.float64), d), ga)
    torch.cuda.synchronize()
    assert np.array_equal(host(na), na64)
    assert np.abs(host(coords) - c64).max() < 1e-9
    assert rel_err(host(ga), g64) < 1e-9


def test_backbone_atoms_equal_backbone_kernel():
    # Section 5's cross-check, on the GPU: N/CA/C of the full-atom kernel equal
    # the backbone kernel's within FP32 rounding.
    d = require_gpu()
    lengths = np.array([300, 120], np.int32)
    a, seq, g, Amax = _inputs(lengths, 4)
    c32, na32, _ = _run_fp32(a, seq, lengths, g, Amax, from_coords=True)
    bb = tpl.backbone(dev(np.ascontiguousarray(a[:, :3]), d), dev(lengths, d))
    bb = host(bb)
    for b, L in enumerate(lengths):
        off = 0
        for j in range(L):
            assert np.abs(c32[b, off:off + 3] - bb[b, 3 * j:3 * j + 3]).max() < 1e-3
            off += tpl.residue_table(int(seq[b, j]))[1]


def test_bad_residue_and_too_many_atoms_set_status():
    d = require_gpu()
    tpl.tpl_get_status()
    lengths = np.array([10, 10], np.int32)
    a, seq, g, Amax = _inputs(lengths, 6)
    seq = seq.copy()
    seq[0, 3] = 31
    _run_fp32(a, seq, lengths, g, Amax, from_coords=True)
    assert tpl.tpl_get_status() & tpl.STATUS_BAD_RESIDUE
    seq[0, 3] = 1
    c32, na32, ga32 = _run_fp32(a, seq, lengths, g[:, :12], 12, from_coords=True)  # Amax far too small
    assert tpl.tpl_get_status() & tpl.STATUS_TOO_MANY_ATOMS
    assert np.all(np.isfinite(c32)) and np.all(np.isfinite(ga32))


def test_tiles_whose_atoms_overflow_the_stage_match_the_oracle():
    """Chains of TRP (14 atoms per residue, more than the stage holds per
    residue slot on average) and mixes around it: those tiles write (and the
    backward reads) their atoms without the stage; all tiles match the oracle."""
    rng = np.random.default_rng(71)
    lengths = np.array([700, 383, 200, 129], np.int32)
    a, seq, g, Amax = _inputs(lengths, 72)
    seq = seq.copy()
    seq[0, :] = 17                      # TRP only: every tile overflows
    seq[1, :200] = 17                   # half TRP
    seq[2, ::2] = 17                    # every other residue
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    g = workloads.upstream_grad((len(lengths), Amax, 3), rng)
    c64, na64 = oracle.fullatom_forward(a, seq, lengths, Amax)
    g = (g * (np.arange(Amax)[None, :] < na64[:, None])[:, :, None]).astype(np.float32)
    g64 = oracle.fullatom_backward(a, seq, lengths, g)
    for shape in [(192, 2), (64, 4), (256, 1)]:
        opts = {"threads": shape[0], "res_per_thread": shape[1]}
        c32, na32, ga32 = _run_fp32(a, seq, lengths, g, Amax, opts, from_coords=True)
        assert np.array_equal(na32, na64)
        assert np.abs(c32 - c64).max() <= COORD_TOL
        assert rel_err(ga32, g64) <= GRAD_TOL


def _short_chain_inputs(seed, trp=False):
    """Many chains shorter than a tile (packed several per CTA), empty and
    one-residue chains, and a few chains longer than a tile."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(1, 120, size=48).astype(np.int32)
    lengths[:6] = [0, 1, 2, 383, 384, 700]
    a, seq = workloads.fullatom_inputs(lengths, rng, Lmax=700)
    if trp:  # 14 atoms per residue: packs whose atoms overflow the stage
        seq[:] = 17
    a[:, 2] += rng.normal(0, 0.2, size=a[:, 2].shape).astype(np.float32)
    a *= (np.arange(700)[None, :] < lengths[:, None])[:, None, :]
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    c64, na64 = oracle.fullatom_forward(a, seq, lengths, Amax)
    g = workloads.upstream_grad((len(lengths), Amax, 3), rng)
    g = (g * (np.arange(Amax)[None, :] < na64[:, None])[:, :, None]).astype(np.float32)
    return a, seq, lengths, g, Amax, c64, na64, oracle.fullatom_backward(a, seq, lengths, g)


@pytest.mark.parametrize("shape,trp", [((384, 1), False), ((128, 2), False), ((192, 4), False), ((64, 4), False),
                                       ((384, 1), True), ((128, 2), True)])
def test_packed_short_chains_match_the_oracle(shape, trp):
    """Chains per CTA > 1 in the full-atom kernels (SCHED_PACKED): segmented
    scans, per-chain stores, the backward from the coordinates; with all-TRP
    chains the packs overflow the stage and go straight to global memory."""
    a, seq, lengths, g, Amax, c64, na64, g64 = _short_chain_inputs(81 + shape[0], trp)
    opts = {"threads": shape[0], "res_per_thread": shape[1], "schedule": tpl.SCHED_PACKED}
    c32, na32, ga32 = _run_fp32(a, seq, lengths, g, Amax, opts, from_coords=True)
    assert np.array_equal(na32, na64)
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    for b, L in enumerate(lengths):
        assert np.all(c32[b, na64[b]:] == 0) and np.all(ga32[b, :, L:] == 0)
    # the padding flag: identical real rows on NaN-filled outputs
    c2, na2, g2 = _run_fp32(a, seq, lengths, g, Amax, dict(opts, flags=tpl.FLAG_PADDING_ZEROED), True)
    for b, L in enumerate(lengths):
        assert np.array_equal(c2[b, :na64[b]], c32[b, :na64[b]]) and np.array_equal(g2[b, :, :L], ga32[b, :, :L])


def test_packed_lrmsd_backward_matches_the_oracle():
    """The LRMSD gradient formed inside the packed full-atom backward."""
    d = require_gpu()
    a, seq, lengths, _, Amax, c64, na64, _ = _short_chain_inputs(91)
    rng = np.random.default_rng(92)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    B, _, Lmax = a.shape
    opts = {"threads": 192, "res_per_thread": 2, "schedule": tpl.SCHED_PACKED}
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, Amax, 3), device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    tpl.tpl_fullatom_forward(dev(ta, d), S, Ln, tgt, na, ws, opts)
    c = torch.zeros_like(tgt)
    tpl.tpl_fullatom_forward(A, S, Ln, c, na, ws, opts)
    lr = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, Amax), dtype=torch.uint8, device=d)
    tpl.tpl_lrmsd_forward(c, tgt, na, lr, lr_ws)
    w = dev(np.linspace(-1.0, 2.0, B).astype(np.float32), d)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, c, tgt, w, lr_ws, ga, ws, opts)
    torch.cuda.synchronize()
    gc64 = oracle.lrmsd_backward(host(w).astype(np.float64), host(c), host(tgt), na64)
    g64 = oracle.fullatom_backward(a, seq, lengths, gc64)
    m = lengths >= 2
    assert rel_err(host(ga)[m], g64[m]) <= GRAD_TOL


def test_packed_schedule_needs_the_coordinate_backward():
    """A packed forward with RECOMPUTE is rejected; a backward that rebuilds
    frames on a packed workspace flags it and writes zeros."""
    d = require_gpu()
    a, seq, lengths, g, Amax, *_ = _short_chain_inputs(95)
    B, _, Lmax = a.shape
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    c = torch.zeros((B, Amax, 3), device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    with pytest.raises(tpl.TplError):
        tpl.tpl_fullatom_forward(A, S, Ln, c, na, ws, {"threads": 128, "res_per_thread": 1,
                                                       "schedule": tpl.SCHED_PACKED, "bwd_mode": tpl.BWD_RECOMPUTE})
    tpl.tpl_get_status()
    o = {"threads": 128, "res_per_thread": 1, "schedule": tpl.SCHED_PACKED}
    tpl.tpl_fullatom_forward(A, S, Ln, c, na, ws, o)
    ga = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward(A, S, Ln, None, dev(g, d), ga, ws, dict(o, bwd_mode=tpl.BWD_RECOMPUTE))
    torch.cuda.synchronize()
    assert tpl.tpl_get_status() & tpl.STATUS_BAD_WORKSPACE
    assert np.all(np.isfinite(host(ga)))


def test_recompute_needs_one_residue_per_thread():
    d = require_gpu()
    lengths = np.array([40], np.int32)
    a, seq, g, Amax = _inputs(lengths, 8)
    with pytest.raises(tpl.TplError) as err:
        _run_fp32(a, seq, lengths, g, Amax, {"threads": 192, "res_per_thread": 2}, from_coords=False)
    assert err.value.code == 1  # TPL_ERR_INVALID_ARG


def test_autotuner_picks_a_valid_shape_and_its_results_match(reference):
    d = require_gpu()
    a, seq, g, Amax, c64, na64, g64 = reference
    A, S, Ln, G = dev(a, d), dev(seq, d), dev(LENGTHS, d), dev(g, d)
    B, _, Lmax = a.shape
    coords = torch.empty((B, Amax, 3), device=d)
    na = torch.empty((B,), dtype=torch.int32, device=d)
    ga = torch.empty_like(A)
    ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    best, ms = tpl.tpl_fullatom_autotune(A, S, Ln, coords, na, G, ga, ws, bwd_mode=tpl.BWD_FROM_COORDS)
    assert ms > 0 and (best.threads, best.res_per_thread) in SHAPES
    assert best.schedule in (tpl.SCHED_BATCH_ORDER, tpl.SCHED_LONGEST_FIRST)
    c32, n32, ga32 = _run_fp32(a, seq, LENGTHS, g, Amax, best, from_coords=True)
    assert np.array_equal(n32, na64)
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL


def test_lrmsd_step_autotuner_picks_a_valid_shape_and_its_step_matches_the_oracle():
    """tpl_fullatom_lrmsd_autotune times forward, LRMSD forward and the fused
    backward per candidate; the step with its pick agrees with the oracle."""
    d = require_gpu()
    rng = workloads.rng_for(4, salt=37)
    lengths = np.array([700, 333, 64, 1, 0, 257, 512, 129], np.int32)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    B, _, Lmax = a.shape
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    fa_ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, Amax, 3), device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    tpl.tpl_fullatom_forward(dev(ta, d), S, Ln, tgt, na, fa_ws)
    coords = torch.zeros_like(tgt)
    lr = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, Amax), dtype=torch.uint8, device=d)
    w = dev(np.linspace(0.5, 2.0, B).astype(np.float32), d)
    ga = torch.empty_like(A)
    best, ms = tpl.tpl_fullatom_lrmsd_autotune(A, S, Ln, coords, na, tgt, w, lr, lr_ws, ga, fa_ws)
    assert ms > 0 and (best.threads, best.res_per_thread) in SHAPES
    assert best.schedule in (tpl.SCHED_BATCH_ORDER, tpl.SCHED_LONGEST_FIRST)
    assert best.bwd_mode == tpl.BWD_FROM_COORDS
    ga.fill_(float("nan"))
    lr.fill_(float("nan"))
    tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, best)
    tpl.tpl_lrmsd_forward(coords, tgt, na, lr, lr_ws)
    tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, coords, tgt, w, lr_ws, ga, fa_ws, best)
    torch.cuda.synchronize()
    c32, t32, n32 = host(coords), host(tgt), host(na)
    assert np.abs(host(lr) - oracle.lrmsd_forward(c32, t32, n32)).max() <= 1e-5
    g64 = oracle.lrmsd_backward(host(w).astype(np.float64), c32, t32, n32)
    assert rel_err(host(ga), oracle.fullatom_backward(a, seq, lengths, g64)) <= GRAD_TOL


@pytest.mark.parametrize("shape", [(256, 1), (192, 2), (64, 4)])
def test_fused_lrmsd_backward_equals_the_two_calls_and_the_oracle(shape):
    """tpl_fullatom_backward_lrmsd = tpl_lrmsd_backward + tpl_fullatom_backward
    (FROM_COORDS), against the same chain of oracle calls."""
    d = require_gpu()
    rng = workloads.rng_for(4, salt=31)
    lengths = np.array([700, 333, 64, 1, 0, 257], np.int32)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    B, _, Lmax = a.shape
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    opts = {"threads": shape[0], "res_per_thread": shape[1]}
    fa_ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, Amax, 3), device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    tpl.tpl_fullatom_forward(dev(ta, d), S, Ln, tgt, na, fa_ws, opts)
    coords = torch.zeros_like(tgt)
    tpl.tpl_fullatom_forward(A, S, Ln, coords, na, fa_ws, opts)
    lr = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, Amax), dtype=torch.uint8, device=d)
    tpl.tpl_lrmsd_forward(coords, tgt, na, lr, lr_ws)
    w = dev(np.linspace(0.5, 2.0, B).astype(np.float32), d)
    ga_fused = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, coords, tgt, w, lr_ws, ga_fused, fa_ws, opts)
    gc = torch.empty_like(coords)
    tpl.tpl_lrmsd_backward(w, coords, tgt, na, gc, lr_ws)
    ga_two = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward(A, S, Ln, coords, gc, ga_two, fa_ws, dict(opts, bwd_mode=tpl.BWD_FROM_COORDS))
    torch.cuda.synchronize()
    f, t = host(ga_fused), host(ga_two)
    assert np.all(np.isfinite(f))
    assert rel_err(f, t) <= 1e-5
    # oracle chain on the same FP32 coordinates
    c32, t32, n32 = host(coords), host(tgt), host(na)
    g64 = oracle.lrmsd_backward(host(w).astype(np.float64), c32, t32, n32)
    ga64 = oracle.fullatom_backward(a, seq, lengths, g64)
    assert rel_err(f, ga64) <= GRAD_TOL


@pytest.mark.parametrize("shape", [(384, 1), (192, 2), (64, 4)])
def test_fused_training_step_matches_the_separate_calls_and_the_oracle(shape):
    """tpl_fullatom_lrmsd_forward / _backward (moments in the forward's tiles,
    then per chain the eigen-solve and the residual pass; the LRMSD gradient
    formed in the backward) against
    tpl_fullatom_forward + tpl_lrmsd_forward + tpl_fullatom_backward_lrmsd and
    against the oracle chain on the same FP32 coordinates."""
    d = require_gpu()
    tpl.tpl_get_status()  # reads and clears what earlier tests left in the status word
    rng = workloads.rng_for(4, salt=33)
    lengths = np.array([700, 333, 64, 1, 0, 257, 700, 9], np.int32)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    B, _, Lmax = a.shape
    A, S, Ln = dev(a, d), dev(seq, d), dev(lengths, d)
    opts = {"threads": shape[0], "res_per_thread": shape[1]}
    fa_ws = torch.empty(tpl.tpl_fullatom_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tgt = torch.zeros((B, Amax, 3), device=d)
    na = torch.zeros((B,), dtype=torch.int32, device=d)
    tpl.tpl_fullatom_forward(dev(ta, d), S, Ln, tgt, na, fa_ws, opts)
    w = dev(np.linspace(0.5, 2.0, B).astype(np.float32), d)
    # separate calls
    c1 = torch.zeros_like(tgt)
    tpl.tpl_fullatom_forward(A, S, Ln, c1, na, fa_ws, opts)
    l1 = torch.zeros((B,), device=d)
    lr_ws = torch.empty(tpl.tpl_lrmsd_workspace_size(B, Amax), dtype=torch.uint8, device=d)
    tpl.tpl_lrmsd_forward(c1, tgt, na, l1, lr_ws)
    g1 = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_backward_lrmsd(A, S, Ln, c1, tgt, w, lr_ws, g1, fa_ws, opts)
    # fused step
    st_ws = torch.empty(tpl.tpl_fullatom_lrmsd_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    c2 = torch.full_like(tgt, float("nan"))
    n2 = torch.full((B,), -1, dtype=torch.int32, device=d)
    l2 = torch.full((B,), float("nan"), device=d)
    tpl.tpl_fullatom_lrmsd_forward(A, S, Ln, tgt, c2, n2, l2, st_ws, opts)
    g2 = torch.full_like(A, float("nan"))
    tpl.tpl_fullatom_lrmsd_backward(S, Ln, c2, tgt, w, g2, st_ws, opts)
    torch.cuda.synchronize()
    assert tpl.tpl_get_status() & ~tpl.STATUS_ZERO_LRMSD == 0
    assert np.array_equal(host(c1), host(c2)) and np.array_equal(host(na), host(n2))
    m = lengths >= 2  # one residue or none: congruent structures, LRMSD 0 and no gradient
    assert np.abs(host(l1) - host(l2))[m].max() <= 1e-5
    assert rel_err(host(g2)[m], host(g1)[m]) <= 1e-4
    c32, t32, n32 = host(c2), host(tgt), host(n2)
    assert np.abs(host(l2) - oracle.lrmsd_forward(c32, t32, n32))[m].max() <= LRMSD_TOL
    g64 = oracle.lrmsd_backward(host(w).astype(np.float64), c32, t32, n32)
    ga64 = oracle.fullatom_backward(a, seq, lengths, g64)
    assert rel_err(host(g2)[m], ga64[m]) <= GRAD_TOL
    for b, L in enumerate(lengths):
        assert np.all(host(g2)[b, :, L:] == 0)


def _mixed_inputs(seed):
    """Full-atom chains, backbone-only chains (code 20) and chains that mix
    both residue by residue, in one batch."""
    rng = np.random.default_rng(seed)
    lengths = np.array([0, 1, 37, 256, 257, 500, 700, 129, 64, 3], np.int32)
    Lmax = 700
    a, seq = workloads.fullatom_inputs(lengths, rng, Lmax=Lmax)
    seq[1::3] = 20                      # whole backbone-only chains
    seq[2::3, ::2] = 20                 # every other residue backbone-only
    a[:, 2] += rng.normal(0, 0.2, size=a[:, 2].shape).astype(np.float32)
    a *= (np.arange(Lmax)[None, :] < lengths[:, None])[:, None, :]
    Amax = workloads.pad_to(max(oracle.max_atoms(seq, lengths), 1))
    g = workloads.upstream_grad((len(lengths), Amax, 3), rng)
    return a, seq, lengths, g, Amax


@pytest.mark.parametrize("shape,from_coords", [((384, 1), True), ((192, 2), True), ((64, 4), True),
                                               ((256, 1), False)])
def test_mixed_backbone_and_fullatom_batch(shape, from_coords):
    """One persistent launch over a batch mixing both models (residue code 20
    places N, CA, C only) against the oracle; backbone-only chains also equal
    the backbone kernel's coordinates."""
    d = require_gpu()
    a, seq, lengths, g, Amax = _mixed_inputs(71)
    c64, na64 = oracle.fullatom_forward(a, seq, lengths, Amax)
    g = (g * (np.arange(Amax)[None, :] < na64[:, None])[:, :, None]).astype(np.float32)
    g64 = oracle.fullatom_backward(a, seq, lengths, g)
    c32, na32, ga32 = _run_fp32(a, seq, lengths, g, Amax, {"threads": shape[0], "res_per_thread": shape[1]},
                                from_coords)
    assert np.array_equal(na32, na64)
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    for b, L in enumerate(lengths):
        assert np.all(c32[b, na64[b]:] == 0) and np.all(ga32[b, :, L:] == 0)
    # whole backbone-only chains against the backbone kernel
    bb = [b for b in range(1, len(lengths), 3)]
    ab = np.ascontiguousarray(a[bb, :3])
    cb = host(_backbone_coords(ab, lengths[bb], d))
    for i, b in enumerate(bb):
        n = 3 * lengths[b]
        assert np.abs(c32[b, :n] - cb[i, :n]).max() <= COORD_TOL


def _backbone_coords(a, lengths, d):
    B, _, Lmax = a.shape
    c = torch.zeros((B, 3 * Lmax, 3), device=d)
    ws = torch.empty(tpl.tpl_backbone_workspace_size(B, Lmax), dtype=torch.uint8, device=d)
    tpl.tpl_backbone_forward(dev(a, d), dev(lengths, d), c, ws)
    torch.cuda.synchronize()
    return c


def test_quadratic_comparator_matches_the_scan_and_the_oracle(reference):
    """tpl_fullatom_backward_quadratic (the paper's depth-first O(L^2) sums of
    Eq. 1) against the scan backward and the oracle, chains of every length of
    the reference batch (several CTAs of 18 residues, ragged ends)."""
    d = require_gpu()
    a, seq, g, Amax, c64, na64, g64 = reference
    c32, na32, ga_scan = _run_fp32(a, seq, LENGTHS, g, Amax, {"threads": 256, "res_per_thread": 1}, True)
    ga = torch.full((len(LENGTHS), 7, a.shape[2]), float("nan"), device=d)
    tpl.tpl_fullatom_backward_quadratic(dev(seq, d), dev(LENGTHS, d), dev(c32, d), dev(g, d), ga)
    torch.cuda.synchronize()
    q = host(ga)
    assert np.all(np.isfinite(q))
    assert rel_err(q, g64) <= GRAD_TOL
    assert rel_err(q, ga_scan) <= GRAD_TOL
    for b, L in enumerate(LENGTHS):
        assert np.all(q[b, :, L:] == 0)
        for j in range(L):
            nchi = tpl.residue_table(int(seq[b, j]))[2]
            assert np.all(q[b, 3 + nchi:, j] == 0)
        if L:
            assert q[b, 2, 0] == 0


@pytest.mark.parametrize("from_coords", [False, True])
def test_free_omega_cis_and_trans(from_coords):
    """omega per residue trans (pi +- 0.1), cis (0 +- 0.1) or uniform: the
    coordinates, all angle gradients and the omega row on its own match the
    oracle (omega is an input, reading 3)."""
    rng = np.random.default_rng(59)
    a, seq, g, Amax = _inputs(LENGTHS, 60)
    B, _, Lmax = a.shape
    kind = rng.integers(0, 3, size=(B, Lmax))
    om = np.where(kind == 0, np.pi + rng.normal(0, 0.1, (B, Lmax)),
                  np.where(kind == 1, rng.normal(0, 0.1, (B, Lmax)), rng.uniform(-np.pi, np.pi, (B, Lmax))))
    a[:, 2] = (om * (np.arange(Lmax)[None, :] < LENGTHS[:, None])).astype(np.float32)
    c64, na64 = oracle.fullatom_forward(a, seq, LENGTHS, Amax)
    g = (g * (np.arange(Amax)[None, :] < na64[:, None])[:, :, None]).astype(np.float32)
    g64 = oracle.fullatom_backward(a, seq, LENGTHS, g)
    c32, na32, ga32 = _run_fp32(a, seq, LENGTHS, g, Amax, {"threads": 256}, from_coords)
    assert np.array_equal(na32, na64)
    assert np.abs(c32 - c64).max() <= COORD_TOL
    assert rel_err(ga32, g64) <= GRAD_TOL
    assert rel_err(ga32[:, 2], g64[:, 2]) <= GRAD_TOL
