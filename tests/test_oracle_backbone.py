"""Pins for the backbone oracle (paper Section 3).

Each pin checks the oracle against something other than itself: the constants
the paper prints (golden file), geometry measured with independent code, the
chain rule's prefix property, central finite differences, and an independent
rotation-about-an-axis form of the derivative.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.geom import angle, dihedral, dist, read_table, wrap

CONST = {row[0]: (int(row[1]), float(row[2]), float(row[3]))
         for row in read_table("backbone_constants.txt")}
ORDER = ["N", "CA", "C"]


def _random(B=3, L=9, seed=0):
    rng = np.random.default_rng(seed)
    lengths = np.array([L, L - 2, 1][:B], np.int32)
    a = workloads.backbone_angles(lengths, rng, Lmax=L).astype(np.float64)
    return a, lengths


def test_bond_lengths_and_angles_match_printed_constants():
    a, lengths = _random()
    c = oracle.backbone_forward(a, lengths)
    for b, L in enumerate(lengths):
        for i in range(1, 3 * L):
            name = ORDER[i % 3]
            _, theta_c, d = CONST[name]
            assert abs(dist(c[b, i - 1], c[b, i]) - d) < 1e-12
            if i >= 2:
                # R_i's theta = pi - value sets the angle at atom i-1
                assert abs(angle(c[b, i - 2], c[b, i - 1], c[b, i]) - theta_c) < 1e-12


def test_measured_dihedrals_equal_input_angles():
    a, lengths = _random()
    c = oracle.backbone_forward(a, lengths)
    for b, L in enumerate(lengths):
        for i in range(2, 3 * L - 1):
            # dihedral about bond (i-1, i) is the angle of transform R_i
            row = CONST[ORDER[i % 3]][0]
            j = i // 3
            assert abs(wrap(dihedral(*c[b, i - 2:i + 2]) - a[b, row, j])) < 1e-12


def test_first_residue_closed_form_and_origin():
    # R_0 = I: N_0 at the origin; CA_0 = R(phi_0) 0 = (d cos th, 0, -d sin th)
    a = np.zeros((1, 3, 4), np.float32)
    a[0, 0] = [0.3, -1.0, 2.0, 0.5]
    a[0, 1] = [1.1, 0.2, -2.5, 0.0]
    a[0, 2] = np.pi
    c = oracle.backbone_forward(a, [4])
    _, theta_c, d = CONST["CA"]
    th = np.pi - theta_c
    assert np.allclose(c[0, 0], 0.0, atol=0)
    assert np.allclose(c[0, 1], [d * np.cos(th), 0.0, -d * np.sin(th)], atol=1e-15)


def test_all_trans_chain_is_planar_zigzag():
    L = 12
    a = np.full((1, 3, L), np.pi, np.float64)
    c = oracle.backbone_forward(a, [L])
    assert np.abs(c[0, :, 1]).max() < 1e-12
    # trans turns alternate in sign, so bond directions repeat every 6 bonds
    bonds = np.diff(c[0], axis=0)
    assert np.allclose(bonds[6:], bonds[:-6], atol=1e-12)


def test_omega0_is_unused():
    a, lengths = _random()
    a2 = a.copy()
    a2[:, 2, 0] += 0.7
    assert np.array_equal(oracle.backbone_forward(a, lengths), oracle.backbone_forward(a2, lengths))


def test_prefix_property_and_padding():
    a, _ = _random(B=1, L=10)
    full = oracle.backbone_forward(a, [10])
    short = oracle.backbone_forward(a, [6])
    assert np.array_equal(full[0, :18], short[0, :18])
    assert np.all(short[0, 18:] == 0.0)


def test_empty_chain_and_empty_batch():
    a = np.zeros((2, 3, 4))
    c = oracle.backbone_forward(a, [0, 0])
    assert np.all(c == 0)
    g = oracle.backbone_backward(a, [0, 0], np.ones((2, 12, 3)))
    assert np.all(g == 0)
    assert oracle.backbone_forward(np.zeros((0, 3, 4)), np.zeros(0, np.int32)).shape == (0, 12, 3)


def test_gradient_matches_central_differences():
    a, lengths = _random(B=2, L=7, seed=3)
    a = a.astype(np.float64)
    rng = np.random.default_rng(5)
    g = rng.normal(size=(2, 21, 3))
    ga = oracle.backbone_backward(a, lengths, g)
    h = 1e-6
    for b in range(2):
        for r in range(3):
            for j in range(lengths[b]):
                ap = a.copy(); am = a.copy()
                ap[b, r, j] += h; am[b, r, j] -= h
                fd = ((oracle.backbone_forward(ap, lengths)[b] -
                       oracle.backbone_forward(am, lengths)[b]) * g[b]).sum() / (2 * h)
                assert abs(fd - ga[b, r, j]) <= 1e-7 * (1 + abs(ga).max())
    # padding rows and omega_0 carry no gradient
    assert ga[1, :, lengths[1]:].max() == 0 and ga[:, 2, 0].max() == 0


def test_gradient_matches_rotation_about_bond_axis():
    # Independent form: rotating by d(alpha_i) about the bond (i-1 -> i) moves atom k
    # by u_i x (r_k - r_i); dL/dalpha_i = sum_{k>=i} g_k . (u_i x (r_k - r_i)).
    a, lengths = _random(B=2, L=30, seed=7)
    rng = np.random.default_rng(8)
    g = rng.normal(size=(2, 90, 3))
    ga = oracle.backbone_backward(a, lengths, g)
    c = oracle.backbone_forward(a, lengths)
    for b in range(2):
        n = 3 * lengths[b]
        for i in range(1, n):
            u = c[b, i] - c[b, i - 1]
            u /= np.linalg.norm(u)
            torque = np.cross(c[b, i:n] - c[b, i], g[b, i:n]).sum(axis=0)
            row = CONST[ORDER[i % 3]][0]
            assert abs(np.dot(u, torque) - ga[b, row, i // 3]) < 1e-9 * (1 + abs(ga).max())
