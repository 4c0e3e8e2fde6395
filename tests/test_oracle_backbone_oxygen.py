"""Pins for the oracle's backbone carbonyl O (paper Section 3 places N, CA and
C only; the O of residue j is rigid in the frame of C_j after psi_j).

Each pin checks the oracle against something other than itself: the Engh &
Huber C-O bond and CA-C-O angle of the golden geometry file, the IUPAC
dihedral N-CA-C-O = psi + 180 and the peptide-plane geometry measured with
independent code, the full-atom oracle's O on an all-glycine chain (a separate
frame construction, Section 2), and central finite differences of the forward
for the gradient.
"""
import os

import numpy as np

import oracle
import workloads
from tests.geom import GOLDEN, angle, dihedral, dist, wrap

GLY = 7


def _golden(kind, atoms):
    with open(os.path.join(GOLDEN, "sidechain_geometry.txt")) as f:
        for line in f:
            body = line.split("#", 1)[0].split("|", 1)[0].split()
            if body and body[0] == kind and body[1] == "*" and body[2:2 + len(atoms)] == atoms:
                return float(body[2 + len(atoms)])
    raise KeyError((kind, atoms))


def _random(seed=0, lengths=(9, 7, 1, 0), Lmax=12):
    rng = np.random.default_rng(seed)
    lengths = np.array(lengths, np.int32)
    a = workloads.backbone_angles(lengths, rng, Lmax=Lmax).astype(np.float64)
    a[:, 2] += rng.normal(0, 0.3, size=a[:, 2].shape)  # free omega
    a *= (np.arange(Lmax)[None, :] < lengths[:, None])[:, None, :]
    return a, lengths


def test_o_geometry_matches_engh_huber_and_the_peptide_plane():
    a, lengths = _random()
    c, o = oracle.backbone_forward_o(a, lengths)
    c_o = _golden("bond", ["C", "O"])
    ca_c_o = _golden("angle", ["CA", "C", "O"])
    for b, L in enumerate(lengths):
        for j in range(L):
            n, ca, cc = c[b, 3 * j], c[b, 3 * j + 1], c[b, 3 * j + 2]
            assert abs(dist(cc, o[b, j]) - c_o) < 1e-12
            assert abs(np.degrees(angle(ca, cc, o[b, j])) - ca_c_o) < 1e-9
            assert abs(wrap(dihedral(n, ca, cc, o[b, j]) - (a[b, 1, j] + np.pi))) < 1e-12
            if j + 1 < L:  # O in the plane of CA, C and the next N, on the other side of the CA-C axis
                assert abs(wrap(dihedral(c[b, 3 * j + 3], ca, cc, o[b, j]) - np.pi)) < 1e-12
        assert np.all(o[b, L:] == 0)
    # the coordinates are the backbone forward's
    assert np.array_equal(c, oracle.backbone_forward(a, lengths))


def test_o_equals_the_fullatom_glycine_o():
    a, lengths = _random(seed=1)
    _, o = oracle.backbone_forward_o(a, lengths)
    B, _, Lmax = a.shape
    fa = np.zeros((B, 7, Lmax))
    fa[:, :3] = a
    seq = np.full((B, Lmax), GLY, np.uint8)
    cf, na = oracle.fullatom_forward(fa, seq, lengths, 4 * Lmax)
    for b, L in enumerate(lengths):
        assert na[b] == 4 * L
        if L:
            assert np.abs(cf[b, 3:4 * L:4] - o[b, :L]).max() < 1e-10
            assert np.abs(cf[b, 0:4 * L:4] - oracle.backbone_forward(a, lengths)[b, 0:3 * L:3]).max() < 1e-10


def test_gradient_with_o_matches_central_differences():
    a, lengths = _random(seed=2, lengths=(6, 4, 1), Lmax=8)
    rng = np.random.default_rng(7)
    B, _, Lmax = a.shape
    g = rng.normal(size=(B, 3 * Lmax, 3))
    go = rng.normal(size=(B, Lmax, 3))
    ga = oracle.backbone_backward_o(a, lengths, g, go)

    def loss(x, b):
        c, o = oracle.backbone_forward_o(x, lengths)
        return (c[b] * g[b]).sum() + (o[b] * go[b]).sum()

    h = 1e-6
    for b in range(B):
        for r in range(3):
            for j in range(lengths[b]):
                ap = a.copy(); am = a.copy()
                ap[b, r, j] += h; am[b, r, j] -= h
                fd = (loss(ap, b) - loss(am, b)) / (2 * h)
                assert abs(fd - ga[b, r, j]) <= 1e-7 * (1 + np.abs(ga).max())
    assert ga[:, 2, 0].max() == 0 and np.all(ga[1, :, lengths[1]:] == 0)
    # the last residue's psi now moves its O
    assert abs(ga[0, 1, lengths[0] - 1]) > 0
    # without an O gradient it is the plain backward
    assert np.allclose(oracle.backbone_backward_o(a, lengths, g, np.zeros_like(go)),
                       oracle.backbone_backward(a, lengths, g), rtol=0, atol=1e-12)
