"""Pins for the full-atom oracle (paper Section 2, and the Section 5 cross-check).

The side-chain geometry is authored (the paper prints none), so the pins are:
heavy-atom counts and chi counts from chemistry, measured chi equal to the input
chi, the printed R' angle with L chirality, N/CA/C identical to the backbone
model (the paper's own FP64 cross-check), rigidity of each group, finite
differences, and an independent rotation-about-an-axis form of Eq. 1.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.geom import angle, dihedral, dist, read_table, wrap

HEAVY = {int(r[0]): (r[1], int(r[2]), int(r[3])) for r in read_table("heavy_atoms.txt")}
CHI = {}
for r in read_table("chi_atoms.txt"):
    CHI.setdefault(r[0], {})[int(r[1])] = r[2:6]
RPRIME_DEG = float(read_table("rprime.txt")[0][0])


def _chain(seq_codes, seed=0, omega=np.pi):
    rng = np.random.default_rng(seed)
    L = len(seq_codes)
    a, _ = workloads.fullatom_inputs(np.array([L], np.int32), rng, Lmax=L, omega=omega)
    s = np.array([seq_codes], np.uint8)
    return a.astype(np.float64), s, np.array([L], np.int32)


def _atoms_by_residue(coords, seq, L):
    out = []
    off = 0
    for j in range(L):
        three, n, nchi, names, groups, r0 = oracle.residue_info(seq[j])
        out.append({nm: coords[off + k] for k, nm in enumerate(names)})
        off += n
    return out


def test_residue_table_matches_chemistry():
    for code in range(20):
        three, n, nchi, names, groups, r0 = oracle.residue_info(code)
        exp_three, exp_n, exp_chi = HEAVY[code]
        assert (three, n, nchi) == (exp_three, exp_n, exp_chi)
        assert names[:4] == ["N", "CA", "C", "O"]
        assert len(set(names)) == n
        # the first atom of every rigid group sits at its frame's origin (Section 2)
        seen = set()
        for k, g in enumerate(groups):
            if g not in seen and g != 2 or names[k] == "C":
                if g not in seen:
                    assert np.allclose(r0[k], 0.0)
            seen.add(g)


def test_measured_chi_equals_input_and_rprime_gives_L_chirality():
    codes = list(range(20)) * 2
    a, s, lengths = _chain(codes, seed=1)
    c, na = oracle.fullatom_forward(a, s, lengths)
    res = _atoms_by_residue(c[0], s[0], len(codes))
    for j, code in enumerate(codes):
        three = HEAVY[code][0]
        at = res[j]
        for k, quad in CHI.get(three, {}).items():
            measured = dihedral(*[at[x] for x in quad])
            assert abs(wrap(measured - a[0, 2 + k, j])) < 1e-10, (three, k)
        if "CB" in at:
            # improper C-N-CA-CB is the R' rotation; L configuration: positive volume
            imp = np.degrees(dihedral(at["C"], at["N"], at["CA"], at["CB"]))
            assert abs(abs(imp) - RPRIME_DEG) < 1e-9
            vol = np.dot(at["N"] - at["CA"], np.cross(at["C"] - at["CA"], at["CB"] - at["CA"]))
            assert vol > 0


def test_backbone_atoms_equal_backbone_model():
    # Section 5 compares the backbone layer with the FP64 full-atom one atom by atom.
    rng = np.random.default_rng(2)
    lengths = np.array([23, 17, 1], np.int32)
    a, s = workloads.fullatom_inputs(lengths, rng)
    a[:, 2] += rng.normal(0, 0.2, size=a[:, 2].shape).astype(np.float32)  # non-trans omega too
    c, na = oracle.fullatom_forward(a, s, lengths)
    bb = oracle.backbone_forward(a[:, :3], lengths)
    for b, L in enumerate(lengths):
        off = 0
        for j in range(L):
            n = HEAVY[int(s[b, j])][1]
            assert np.abs(c[b, off:off + 3] - bb[b, 3 * j:3 * j + 3]).max() < 1e-12
            off += n
        assert na[b] == off
        assert np.all(c[b, off:] == 0)


def test_rigid_groups_keep_internal_geometry_when_angles_change():
    # Section 2: atoms of one rigid group move together; distances inside a group
    # and the covalent bonds between groups do not depend on the angles.
    codes = list(range(20))
    a, s, lengths = _chain(codes, seed=3)
    a2, _, _ = _chain(codes, seed=4)
    c1, _ = oracle.fullatom_forward(a, s, lengths)
    c2, _ = oracle.fullatom_forward(a2, s, lengths)
    r1 = _atoms_by_residue(c1[0], s[0], 20)
    r2 = _atoms_by_residue(c2[0], s[0], 20)
    for j, code in enumerate(codes):
        three, n, nchi, names, groups, r0 = oracle.residue_info(code)
        for x in range(n):
            for y in range(n):
                same = groups[x] == groups[y]
                if same:
                    assert abs(dist(r1[j][names[x]], r1[j][names[y]]) -
                               dist(r2[j][names[x]], r2[j][names[y]])) < 1e-12
        for k, quad in CHI.get(three, {}).items():
            for u, v in ((quad[0], quad[1]), (quad[1], quad[2]), (quad[2], quad[3])):
                assert abs(dist(r1[j][u], r1[j][v]) - dist(r2[j][u], r2[j][v])) < 1e-12
            assert abs(angle(*[r1[j][q] for q in quad[1:]]) -
                       angle(*[r2[j][q] for q in quad[1:]])) < 1e-12
        assert abs(angle(r1[j]["CA"], r1[j]["C"], r1[j]["O"]) -
                   angle(r2[j]["CA"], r2[j]["C"], r2[j]["O"])) < 1e-12


def test_o_is_trans_to_next_n_and_proline_ring_closes():
    codes = [14, 14, 14, 0]
    a, s, lengths = _chain(codes, seed=5)
    c, _ = oracle.fullatom_forward(a, s, lengths)
    r = _atoms_by_residue(c[0], s[0], 4)
    for j in range(3):
        psi_o = dihedral(r[j]["N"], r[j]["CA"], r[j]["C"], r[j]["O"])
        psi_n = dihedral(r[j]["N"], r[j]["CA"], r[j]["C"], r[j + 1]["N"])
        assert abs(wrap(psi_o - psi_n - np.pi)) < 1e-10
        assert abs(dist(r[j]["CD"], r[j]["N"]) - 1.473) < 2e-3


def test_unused_chi_rows_are_ignored():
    a, s, lengths = _chain(list(range(20)), seed=6)
    c, _ = oracle.fullatom_forward(a, s, lengths)
    a2 = a.copy()
    for j in range(20):
        nchi = HEAVY[int(s[0, j])][2]
        a2[0, 3 + nchi:, j] += 1.0
    a2[0, 2, 0] += 0.5  # omega_0 unused as well
    c2, _ = oracle.fullatom_forward(a2, s, lengths)
    assert np.array_equal(c, c2)


def test_gradient_matches_central_differences():
    codes = [1, 17, 14, 11, 7, 12, 8, 0, 9]
    a, s, lengths = _chain(codes, seed=7, omega=np.pi)
    a = a.astype(np.float64)
    a[0, 2] += np.random.default_rng(1).normal(0, 0.3, size=len(codes))
    c, na = oracle.fullatom_forward(a, s, lengths)
    g = np.random.default_rng(9).normal(size=c.shape)
    ga = oracle.fullatom_backward(a, s, lengths, g)
    h = 1e-6
    Amax = c.shape[1]
    for r in range(7):
        for j in range(len(codes)):
            ap = a.copy(); am = a.copy()
            ap[0, r, j] += h; am[0, r, j] -= h
            cp, _ = oracle.fullatom_forward(ap, s, lengths, Amax)
            cm, _ = oracle.fullatom_forward(am, s, lengths, Amax)
            fd = ((cp - cm) * g).sum() / (2 * h)
            assert abs(fd - ga[0, r, j]) <= 1e-7 * (1 + abs(ga).max()), (r, j)
    # unused rows carry exactly zero
    for j, code in enumerate(codes):
        assert np.all(ga[0, 3 + HEAVY[code][2]:, j] == 0)
    assert ga[0, 2, 0] == 0


def test_gradient_matches_rotation_about_bond_axis():
    # dL/dalpha = u . sum_{k downstream} (r_k - p) x g_k with u the bond axis and p on it.
    codes = list(range(20))
    a, s, lengths = _chain(codes, seed=10)
    c, na = oracle.fullatom_forward(a, s, lengths)
    g = np.random.default_rng(11).normal(size=c.shape)
    ga = oracle.fullatom_backward(a, s, lengths, g)
    L = len(codes)
    res = _atoms_by_residue(c[0], s[0], L)
    offs = np.cumsum([0] + [HEAVY[x][1] for x in codes])
    n_tot = offs[-1]

    def contrib(idx, p, u):
        return np.dot(u, np.cross(c[0, idx] - p, g[0, idx]).sum(axis=0))

    scale = 1 + abs(ga).max()
    for j, code in enumerate(codes):
        three, n, nchi, names, groups, r0 = oracle.residue_info(code)
        at = res[j]
        later = np.arange(offs[j + 1], n_tot)
        own = np.arange(offs[j], offs[j + 1])
        # phi: axis N->CA, everything of residue j but N, and later residues
        u = at["CA"] - at["N"]; u /= np.linalg.norm(u)
        idx = np.concatenate([own[1:], later])
        assert abs(contrib(idx, at["CA"], u) - ga[0, 0, j]) < 1e-9 * scale
        # psi: axis CA->C, atoms C, O and later residues
        u = at["C"] - at["CA"]; u /= np.linalg.norm(u)
        idx = np.concatenate([own[2:4], later])
        assert abs(contrib(idx, at["C"], u) - ga[0, 1, j]) < 1e-9 * scale
        # omega_j (j >= 1): axis C_{j-1}->N_j, every atom of residues >= j
        if j >= 1:
            u = at["N"] - res[j - 1]["C"]; u /= np.linalg.norm(u)
            idx = np.arange(offs[j], n_tot)
            assert abs(contrib(idx, at["N"], u) - ga[0, 2, j]) < 1e-9 * scale
        # chi_k: axis (b -> c) of the IUPAC quadruple; atoms beyond c on that branch are
        # those the rotation moves: every side-chain atom whose distance to the axis
        # changes is not needed -- use the atoms that move when chi_k changes.
        for k, quad in CHI.get(three, {}).items():
            u = at[quad[2]] - at[quad[1]]; u /= np.linalg.norm(u)
            a2 = a.copy(); a2[0, 2 + k, j] += 0.5
            c2, _ = oracle.fullatom_forward(a2, s, lengths)
            moved = [offs[j] + t for t in range(n)
                     if np.abs(c2[0, offs[j] + t] - c[0, offs[j] + t]).max() > 1e-9]
            assert abs(contrib(np.array(moved), at[quad[2]], u) - ga[0, 2 + k, j]) < 1e-9 * scale
