"""LRMSD (Section 4): FP32 kernels (an FP32 eigen-solve refined once against
the exact T), and the FP64 per-pair form, against the FP64 CPU oracle.  Tolerances: LRMSD max-abs <= 1e-5 A;
gradient ||g32 - g64|| / ||g64|| <= 1e-4 per pair; FP64 form 1e-9.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_01108_gb300 as tpl
import workloads
from tests.gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

LRMSD_TOL = 1e-5
GRAD_TOL = 1e-4


def _clouds(sizes, seed, noise=0.5):
    rng = np.random.default_rng(seed)
    P = len(sizes)
    Nmax = workloads.pad_to(max(max(sizes), 1))
    # full clouds first (non-degenerate), then cut to the requested sizes
    x, y, _ = workloads.lrmsd_clouds(P, Nmax, Nmax, rng, Nmax=Nmax, noise=noise)
    n = np.array(sizes, np.int32)
    mask = (np.arange(Nmax)[None, :] < n[:, None])[:, :, None]
    return (x * mask).astype(np.float32), (y * mask).astype(np.float32), n


def _run(x, y, n, w):
    d = require_gpu()
    X, Y, N = dev(x, d), dev(y, d), dev(n, d)
    P, Nmax, _ = x.shape
    out = torch.full((P,), float("nan"), device=d)
    ws = torch.empty(tpl.tpl_lrmsd_workspace_size(P, Nmax), dtype=torch.uint8, device=d)
    tpl.tpl_lrmsd_forward(X, Y, N, out, ws)
    gi = torch.full_like(X, float("nan"))
    tpl.tpl_lrmsd_backward(dev(w, d), X, Y, N, gi, ws)
    torch.cuda.synchronize()
    return host(out), host(gi)


SIZES = [0, 1, 2, 3, 4, 5, 100, 2047, 2048, 2049, 4095, 4096, 4097, 5000, 777, 3]


def test_matches_oracle_across_chunk_boundaries():
    x, y, n = _clouds(SIZES, 1)
    w = np.linspace(-1, 2, len(SIZES)).astype(np.float32)
    l32, g32 = _run(x, y, n, w)
    l64 = oracle.lrmsd_forward(x, y, n)
    g64 = oracle.lrmsd_backward(w, x, y, n)
    assert np.abs(l32 - l64).max() <= LRMSD_TOL
    # 1-2 atoms: the optimal rotation is not unique, so only the value is compared
    unique = n >= 3
    assert rel_err(g32[unique], g64[unique]) <= GRAD_TOL
    for p, k in enumerate(n):
        assert np.all(g32[p, k:] == 0)


def test_config3_shaped_sample():
    rng = workloads.rng_for(3, salt=7)
    x, y, n = workloads.lrmsd_clouds(48, 100, 5000, rng)
    w = np.ones(48, np.float32)
    l32, g32 = _run(x, y, n, w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL
    assert rel_err(g32, oracle.lrmsd_backward(w, x, y, n)) <= GRAD_TOL


def test_identical_structures_zero_lrmsd_and_flag():
    require_gpu()
    tpl.tpl_get_status()
    x, _, n = _clouds([50, 50], 2)
    y = x.copy()
    l32, g32 = _run(x, y, n, np.ones(2, np.float32))
    assert np.abs(l32).max() < 1e-3
    # rounding may leave a tiny positive LRMSD; the gradient is then bounded
    assert np.all(np.isfinite(g32))


def test_fp64_per_pair_form_matches_oracle():
    d = require_gpu()
    x, y, n = _clouds([10, 500, 3000, 0, 7], 3)
    w = np.array([1.0, 0.5, -2.0, 1.0, 3.0])
    X, Y, N = dev(x.astype(np.float64), d), dev(y.astype(np.float64), d), dev(n, d)
    P = len(n)
    out = torch.zeros((P,), dtype=torch.float64, device=d)
    st = torch.zeros((P, 16), dtype=torch.float64, device=d)
    tpl.tpl_lrmsd_forward_ref64(X, Y, N, out, st)
    gi = torch.full_like(X, float("nan"))
    tpl.tpl_lrmsd_backward_ref64(dev(w, d), X, Y, N, st, gi)
    torch.cuda.synchronize()
    assert np.abs(host(out) - oracle.lrmsd_forward(x, y, n)).max() < 1e-9
    assert rel_err(host(gi), oracle.lrmsd_backward(w, x, y, n)) < 1e-8


def test_autograd_lrmsd():
    d = require_gpu()
    x, y, n = _clouds([300, 40], 4)
    X = dev(x, d).requires_grad_(True)
    l = tpl.lrmsd(X, dev(y, d), dev(n, d))
    l.sum().backward()
    assert rel_err(host(X.grad), oracle.lrmsd_backward(np.ones(2), x, y, n)) <= GRAD_TOL


def test_precision_small_clouds_far_from_origin():
    """The moments are shifted by each pair's first atom and summed in
    double-float, so a cloud far from the origin costs no precision."""
    x, y, n = _clouds([100] * 12 + [5000] * 4, 5)
    off = np.array([300.0, -200.0, 150.0], np.float32)
    mask = (np.arange(x.shape[1])[None, :] < n[:, None])[:, :, None]
    x = ((x + off) * mask).astype(np.float32)
    y = ((y - 2 * off) * mask).astype(np.float32)
    w = np.ones(len(n), np.float32)
    l32, g32 = _run(x, y, n, w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL
    assert rel_err(g32, oracle.lrmsd_backward(w, x, y, n)) <= GRAD_TOL


def test_precision_close_fit():
    """LRMSD near 0.1 A.  The value keeps the 1e-5 A bound.  The gradient is
    the residual y' - U x', a difference of FP32 terms of size |x'| (about 26 A
    here) that ends near LRMSD: its relative error is a few units of
    eps_32 |x'| / LRMSD (eps_32 = 2^-24 relative rounding, |x'| / LRMSD ~ 300),
    so the bound for this case is 10 eps_32 |x'|_rms / min LRMSD."""
    x, y, n = _clouds([100] * 12 + [2000] * 4, 6, noise=0.05)
    w = np.ones(len(n), np.float32)
    l32, g32 = _run(x, y, n, w)
    l64 = oracle.lrmsd_forward(x, y, n)
    assert l64.max() < 0.15
    assert np.abs(l32 - l64).max() <= LRMSD_TOL
    xr = max(float(np.sqrt(((x[p, :k] - x[p, :k].mean(0)) ** 2).sum(1)).mean()) for p, k in enumerate(n))
    bound = 10 * 2.0 ** -24 * xr / float(l64.min())
    assert 1e-4 < bound < 1e-3
    assert rel_err(g32, oracle.lrmsd_backward(w, x, y, n)) <= bound


def test_protein_shaped_pairs():
    """Full-atom chains built from the origin against angle-perturbed copies
    (the training-step pairing), on identical FP32 coordinates."""
    rng = workloads.rng_for(4, salt=11)
    lengths = np.array([700, 350, 128, 64], np.int32)
    a, seq = workloads.fullatom_inputs(lengths, rng)
    ta = workloads.perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    c, n = oracle.fullatom_forward(a, seq, lengths, Amax)
    t, _ = oracle.fullatom_forward(ta, seq, lengths, Amax)
    x, y = t.astype(np.float32), c.astype(np.float32)
    w = np.full(len(n), 0.25, np.float32)
    l32, g32 = _run(x, y, n.astype(np.int32), w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL
    assert rel_err(g32, oracle.lrmsd_backward(w, x, y, n)) <= GRAD_TOL


def test_large_batch_of_small_pairs():
    """Many pairs of a few atoms: the compact CTA shape, most of its threads idle."""
    rng = np.random.default_rng(9)
    P = 8300
    x, y, n = workloads.lrmsd_clouds(P, 3, 40, rng)
    w = rng.normal(size=P).astype(np.float32)
    l32, g32 = _run(x, y, n, w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL
    assert rel_err(g32, oracle.lrmsd_backward(w, x, y, n)) <= GRAD_TOL


# sizes around the atoms a CTA loads per pass (four per thread and group:
# 1024 for the compact shape, 4096 for the wide one) and their halves
CHUNK_SIZES = [0, 1, 2, 3, 4, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2999, 3000, 4095, 4096, 4097]


@pytest.mark.parametrize("P", [200, 600, 2000])
def test_batches_of_every_size_around_the_load_passes(P):
    """Batches that fit one wave of wide CTAs (200) and larger ones (compact
    CTAs), with atom counts around the CTA's load passes, so pairs end in
    every position of a pass."""
    sizes = [CHUNK_SIZES[i % len(CHUNK_SIZES)] for i in range(P)]
    x, y, n = _clouds(sizes, 11 + P)
    w = np.random.default_rng(P).normal(size=P).astype(np.float32)
    l32, g32 = _run(x, y, n, w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL
    unique = n >= 3
    assert rel_err(g32[unique], oracle.lrmsd_backward(w, x, y, n)[unique]) <= GRAD_TOL
    for p, k in enumerate(n):
        assert np.all(g32[p, k:] == 0)


@pytest.mark.parametrize("P", [150, 1500])
def test_two_atom_pairs(P):
    """Two atoms: R has rank one, so the largest eigenvalue of T is exactly
    double and every cofactor of T - lambda I vanishes; the eigen-solve must
    still land in the eigenspace of lambda_max (aligned, not anti-aligned,
    difference vectors), for both CTA shapes (150 pairs fit one wave of wide
    CTAs, 1500 do not)."""
    rng = np.random.default_rng(P + 5)
    x, y, n = workloads.lrmsd_clouds(P, 2, 2, rng)
    w = rng.normal(size=P).astype(np.float32)
    l32, g32 = _run(x, y, n, w)
    assert np.abs(l32 - oracle.lrmsd_forward(x, y, n)).max() <= LRMSD_TOL


def _rot(q):
    q = np.asarray(q, np.float64)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _degenerate_clouds(P, rng, Nmax, extent):
    """Pairs whose optimal rotation is not unique: collinear atoms (any turn
    about the line fits as well: the largest eigenvalue of T is double), evenly
    or unevenly spaced over `extent` A, as exact rigid copies; plus two-fold
    symmetric clouds, as exact copies and with 0.3 A noise."""
    x = np.zeros((P, Nmax, 3), np.float64)
    y = np.zeros_like(x)
    n = np.zeros(P, np.int32)
    for p in range(P):
        k = int(rng.integers(4, Nmax + 1))
        kind = p % 4
        if kind < 2:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            t = np.linspace(-0.5, 0.5, k) if kind == 0 else np.sort(rng.uniform(-0.5, 0.5, k))
            pts = np.outer(t * extent, d) + rng.normal(size=3) * 5
        else:
            k -= k % 2
            half = rng.normal(scale=12.0, size=(k // 2, 3))
            axis = rng.normal(size=3)
            axis /= np.linalg.norm(axis)
            pts = np.concatenate([half, half @ (2 * np.outer(axis, axis) - np.eye(3)).T]) + rng.normal(size=3) * 3
        moved = pts @ _rot(rng.normal(size=4)).T + rng.normal(size=3) * 10
        if kind == 3:
            moved = moved + rng.normal(scale=0.3, size=moved.shape)
        x[p, :k], y[p, :k], n[p] = pts, moved, k
    return x.astype(np.float32), y.astype(np.float32), n


@pytest.mark.parametrize("P,extent", [(16, 60.0), (600, 60.0), (64, 770.0)])
def test_degenerate_largest_eigenvalue(P, extent):
    """Collinear pairs (a double largest eigenvalue) and two-fold symmetric
    pairs: the LRMSD is unique even where the rotation is not, and must match
    the oracle.  P = 600 takes the streaming kernels, P = 16 and 64 one CTA per
    pair.  The exact copies have an LRMSD of rounding size, where the FP32
    rounding of U and of the coordinates alone moves the value by a few units
    of 2^-24 |x'|: the bound is 10 * 2^-24 * max |x' - centroid| of each pair
    (about 1.8e-5 A for the 60 A lines), and never below 1e-5 A."""
    rng = np.random.default_rng(71 + P)
    x, y, n = _degenerate_clouds(P, rng, 512, extent)
    l32, _ = _run(x, y, n, np.ones(P, np.float32))
    l64 = oracle.lrmsd_forward(x, y, n)
    for p in range(P):
        pts = y[p, :n[p]].astype(np.float64)
        bound = max(LRMSD_TOL, 10 * 2.0 ** -24 * np.linalg.norm(pts - pts.mean(0), axis=1).max())
        assert abs(l32[p] - l64[p]) <= bound, (p, l32[p], l64[p], bound)
