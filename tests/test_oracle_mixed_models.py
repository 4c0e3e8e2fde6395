"""Pins for residue code 20 of the full-atom oracle: a residue that places the
Section 3 backbone only (N, CA, C), so that one full-atom batch can hold
backbone-model chains, or chains that mix both models residue by residue.

The pins compare with the backbone oracle (Section 3, itself pinned to the
printed constants and to finite differences), which shares no frame code with
the full-atom graph of Section 2, and with central finite differences of the
full-atom forward on mixed chains.
"""
import numpy as np

import oracle
import workloads

BB = 20


def _angles(lengths, Lmax, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-np.pi, np.pi, size=(len(lengths), 7, Lmax))
    a[:, 2] = np.pi + rng.normal(0, 0.2, size=(len(lengths), Lmax))
    a *= (np.arange(Lmax)[None, :] < np.asarray(lengths)[:, None])[:, None, :]
    return a


def test_code_20_is_the_backbone_residue():
    three, n, nchi, names, groups, _ = oracle.residue_info(BB)
    assert (three, n, nchi) == ("BB", 3, 0)
    assert names == ["N", "CA", "C"] and groups == [0, 1, 2]
    assert oracle.chain_atoms(np.full(5, BB, np.uint8), 5) == 15


def test_backbone_only_chains_equal_the_backbone_model():
    lengths = np.array([9, 4, 1, 0], np.int32)
    Lmax = 12
    a = _angles(lengths, Lmax, 1)
    seq = np.full((4, Lmax), BB, np.uint8)
    c, na = oracle.fullatom_forward(a, seq, lengths, 3 * Lmax)
    cb = oracle.backbone_forward(a[:, :3], lengths)
    assert np.array_equal(na, 3 * lengths)
    assert np.abs(c - cb).max() < 1e-10
    g = np.random.default_rng(2).normal(size=c.shape) * (np.arange(3 * Lmax)[None, :, None] < 3 * lengths[:, None, None])
    ga = oracle.fullatom_backward(a, seq, lengths, g)
    assert np.abs(ga[:, :3] - oracle.backbone_backward(a[:, :3], lengths, g)).max() < 1e-9
    assert np.all(ga[:, 3:] == 0)


def test_mixed_chain_backbone_atoms_and_finite_differences():
    rng = np.random.default_rng(3)
    L, Lmax = 8, 8
    lengths = np.array([L], np.int32)
    seq = rng.integers(0, 21, size=(1, Lmax)).astype(np.uint8)
    seq[0, ::3] = BB
    a = _angles(lengths, Lmax, 4)
    Amax = workloads.pad_to(oracle.max_atoms(seq, lengths))
    c, na = oracle.fullatom_forward(a, seq, lengths, Amax)
    cb = oracle.backbone_forward(a[:, :3], lengths)
    off = 0
    for j in range(L):
        assert np.abs(c[0, off:off + 3] - cb[0, 3 * j:3 * j + 3]).max() < 1e-10
        off += oracle.residue_info(int(seq[0, j]))[1]
    assert off == na[0]
    g = rng.normal(size=c.shape)
    g[0, na[0]:] = 0
    ga = oracle.fullatom_backward(a, seq, lengths, g)
    h = 1e-6
    for r in range(7):
        for j in range(L):
            ap = a.copy(); am = a.copy()
            ap[0, r, j] += h; am[0, r, j] -= h
            fd = ((oracle.fullatom_forward(ap, seq, lengths, Amax)[0] -
                   oracle.fullatom_forward(am, seq, lengths, Amax)[0]) * g).sum() / (2 * h)
            assert abs(fd - ga[0, r, j]) <= 1e-7 * (1 + np.abs(ga).max())
