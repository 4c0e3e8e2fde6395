"""Pins for the LRMSD oracle (paper Section 4).

Pinned against: the Kabsch/SVD solution from numpy (a library routine), a brute
force rotation search on 5-atom inputs, numpy's symmetric eigen-solver, rigid
invariance, symmetry in its two arguments, and central finite differences.
"""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation

import oracle
import workloads


def _pairs(P=5, n_lo=3, n_hi=40, seed=0, noise=0.5):
    rng = np.random.default_rng(seed)
    x, y, n = workloads.lrmsd_clouds(P, n_lo, n_hi, rng, noise=noise)
    return x.astype(np.float64), y.astype(np.float64), n


def _kabsch(x, y):
    xc = x - x.mean(0)
    yc = y - y.mean(0)
    s = np.linalg.svd(xc.T @ yc, compute_uv=False)
    d = np.sign(np.linalg.det(xc.T @ yc))
    e = (xc ** 2).sum() + (yc ** 2).sum() - 2 * (s[0] + s[1] + d * s[2])
    return np.sqrt(max(e, 0.0) / len(x))


def test_matches_kabsch_svd():
    x, y, n = _pairs(P=8)
    l = oracle.lrmsd_forward(x, y, n)
    for p in range(8):
        assert abs(l[p] - _kabsch(y[p, :n[p]], x[p, :n[p]])) < 1e-10


def test_brute_force_rotation_search_5_atoms():
    rng = np.random.default_rng(1)
    for trial in range(3):
        x = rng.normal(0, 3, size=(5, 3))
        y = Rotation.random(random_state=trial).apply(x) + rng.normal(0, 0.8, size=(5, 3)) + 4.0
        val = oracle.lrmsd_forward(y[None], x[None], [5])[0]
        xc = x - x.mean(0)
        yc = y - y.mean(0)

        def rmsd(rv):
            M = Rotation.from_rotvec(rv).as_matrix()
            return np.sqrt(((xc - yc @ M.T) ** 2).sum() / 5)

        grid = Rotation.random(4000, random_state=100 + trial).as_rotvec()
        vals = np.array([rmsd(r) for r in grid])
        best = min(minimize(rmsd, grid[i], method="Nelder-Mead",
                            options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 20000}).fun
                   for i in np.argsort(vals)[:5])
        assert best >= val - 1e-9
        assert best - val < 1e-6


def test_zero_for_rigid_copy_and_invariance():
    x, y, n = _pairs(P=4, seed=2)
    rot = Rotation.random(4, random_state=3).as_matrix()
    moved = np.einsum("pij,pnj->pni", rot, x) + 7.0
    moved *= (np.arange(x.shape[1])[None, :] < n[:, None])[:, :, None]
    assert np.abs(oracle.lrmsd_forward(moved, x, n)).max() < 1e-6  # sqrt of ~1e-13 rounding
    l1 = oracle.lrmsd_forward(y, x, n)
    y2 = np.einsum("pij,pnj->pni", rot, y) - 3.0
    y2 *= (np.arange(x.shape[1])[None, :] < n[:, None])[:, :, None]
    assert np.allclose(oracle.lrmsd_forward(y2, x, n), l1, atol=1e-10)


def test_symmetric_in_arguments():
    x, y, n = _pairs(P=6, seed=4)
    assert np.allclose(oracle.lrmsd_forward(y, x, n), oracle.lrmsd_forward(x, y, n), atol=1e-10)


def test_rotation_is_proper_and_maps_target_onto_input():
    x, y, n = _pairs(P=5, seed=5)
    l, U, lam = oracle.lrmsd_forward(y, x, n, return_aux=True)
    for p in range(5):
        assert np.allclose(U[p] @ U[p].T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(U[p]) - 1.0) < 1e-12
        xc = x[p, :n[p]] - x[p, :n[p]].mean(0)
        yc = y[p, :n[p]] - y[p, :n[p]].mean(0)
        resid = np.sqrt(((yc - xc @ U[p].T) ** 2).sum() / n[p])
        assert abs(resid - l[p]) < 1e-9


def test_jacobi_matches_numpy_eigh():
    rng = np.random.default_rng(6)
    for _ in range(20):
        A = rng.normal(size=(4, 4))
        A = A + A.T
        ev, V = oracle.sym4_eig(A)
        assert np.allclose(ev, np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(A @ V, V * ev[None, :], atol=1e-11)


def test_gradient_matches_central_differences():
    x, y, n = _pairs(P=3, n_lo=4, n_hi=9, seed=7)
    w = np.array([1.0, -0.5, 2.0])
    gy = oracle.lrmsd_backward(w, y, x, n)
    h = 1e-5
    for p in range(3):
        for i in range(x.shape[1]):
            for k in range(3):
                yp = y.copy(); ym = y.copy()
                yp[p, i, k] += h; ym[p, i, k] -= h
                fd = w[p] * (oracle.lrmsd_forward(yp, x, n)[p] - oracle.lrmsd_forward(ym, x, n)[p]) / (2 * h)
                if i >= n[p]:
                    assert gy[p, i, k] == 0.0
                else:
                    assert abs(fd - gy[p, i, k]) < 1e-6 * (1 + abs(gy).max())
    # translation invariance: gradients sum to zero per pair
    assert np.abs(gy.sum(axis=1)).max() < 1e-12


def test_degenerate_sizes():
    x = np.zeros((3, 4, 3))
    y = np.zeros((3, 4, 3))
    y[1, 0] = [1.0, 2.0, 3.0]
    x[1, 0] = [-1.0, 0.0, 5.0]
    n = np.array([0, 1, 0], np.int32)
    assert np.all(oracle.lrmsd_forward(y, x, n) == 0.0)
    g = oracle.lrmsd_backward(np.ones(3), y, x, n)
    assert np.all(g == 0.0)


def test_collinear_pairs_match_kabsch():
    """Collinear atoms leave the turn about the line free: the largest
    eigenvalue of T is double.  The LRMSD is still unique: zero for a rigid
    copy, and equal to the Kabsch value (numpy SVD) when the second line is
    stretched, which no rotation can undo."""
    rng = np.random.default_rng(19)
    for k in (3, 7, 40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t = np.sort(rng.uniform(-20, 20, k))
        x = np.outer(t, d) + rng.normal(size=3)
        rot = Rotation.from_quat(rng.normal(size=4)).as_matrix()
        y = x @ rot.T + rng.normal(size=3) * 5
        n = np.array([k], np.int32)
        # the closed form sqrt((E0 - 2 lambda) / N) cancels: at a zero LRMSD it
        # leaves about sqrt(few ulp * E0 / N)
        e0n = (((x - x.mean(0)) ** 2).sum() + ((y - y.mean(0)) ** 2).sum()) / k
        assert oracle.lrmsd_forward(y[None], x[None], n)[0] <= np.sqrt(64 * 2.0 ** -52 * e0n)
        ys = 1.1 * y  # stretched copy
        ref = _kabsch(ys, x)
        assert abs(oracle.lrmsd_forward(ys[None], x[None], n)[0] - ref) < 1e-9
