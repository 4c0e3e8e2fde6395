"""Pins of the oracle's side-chain geometry (paper Section 2: the rigid
groups' standard-frame coordinates depend only on the residue type, and the
paper prints none of them).

Every bond length and bond angle that the oracle's residue table sets is
measured on structures the oracle builds, for every residue type and random
phi, psi, omega and chi, and compared with tests/golden/sidechain_geometry.txt,
whose values are typed from the bond-length and bond-angle tables of Engh &
Huber (1991), each line naming its atom-type row.  Values the table sets
directly must come out exact (FP64 rounding); ring closures and the angles
between two branches, which follow from the others, within the tolerance the
golden line gives.  Aromatic rings must be planar and the CB centres of ILE and
THR must have the configuration of the natural L amino acids.

A change of one digit in any bond or angle of the oracle's table fails
test_every_table_bond_and_angle_matches_the_golden_values: every side-chain
atom has an exact bond line and an exact angle line (test_golden_covers_every_atom).
"""
import os

import numpy as np
import pytest

import oracle
from tests.geom import GOLDEN, angle, dist

EXACT_A = 1e-10     # Angstrom
EXACT_DEG = 1e-8    # degrees
PLANAR_A = 1e-10


def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "sidechain_geometry.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0]
            body = line.split("|", 1)[0].split()
            if not body:
                continue
            kind, res = body[0], body[1]
            if kind in ("bond", "angle"):
                n = 2 if kind == "bond" else 3
                atoms = body[2:2 + n]
                value, tol = float(body[2 + n]), float(body[3 + n])
            elif kind == "planar":
                atoms, value, tol = body[2:-2], None, 0.0
            elif kind == "chiral":
                atoms, value, tol = body[2:6], body[6], 0.0
            else:
                raise ValueError(f"unknown golden kind {kind!r}")
            rows.append((kind, res, atoms, value, tol))
    return rows


GOLDEN_ROWS = _golden()
TYPES = {oracle.residue_info(c)[0]: c for c in range(20)}


def _built_residues(code, seed):
    """Residue `code` in the middle of ALA-X-ALA with random phi, psi, chi and
    a random (non-trans) omega: {atom name: position}."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-np.pi, np.pi, size=(1, 7, 3))
    a[0, 2] = np.pi + rng.normal(0.0, 0.3, size=3)
    seq = np.array([[0, code, 0]], np.uint8)
    c, na = oracle.fullatom_forward(a, seq, np.array([3], np.int32))
    names = oracle.residue_info(code)[3]
    off = oracle.residue_info(0)[1]
    return {nm: c[0, off + k] for k, nm in enumerate(names)}


def _rows_for(three):
    return [r for r in GOLDEN_ROWS if r[1] in (three, "*")]


def test_golden_names_real_atoms():
    for kind, res, atoms, value, tol in GOLDEN_ROWS:
        types = TYPES.values() if res == "*" else [TYPES[res]]
        for code in types:
            names = oracle.residue_info(code)[3]
            assert all(a in names for a in atoms), (res, atoms)


def test_golden_covers_every_atom():
    """Every side-chain atom of every type has an exact bond line and an exact
    angle line ending at it, and backbone O too: so every bond and angle the
    table sets is pinned."""
    for three, code in TYPES.items():
        names = oracle.residue_info(code)[3]
        rows = _rows_for(three)
        for atom in names[3:]:
            bonds = [r for r in rows if r[0] == "bond" and r[4] == 0 and atom in r[2]]
            angles = [r for r in rows if r[0] == "angle" and r[4] == 0 and atom in (r[2][0], r[2][2])]
            assert bonds and angles, (three, atom)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_every_table_bond_and_angle_matches_the_golden_values(seed):
    for three, code in TYPES.items():
        r = _built_residues(code, seed + 100 * code)
        for kind, res, atoms, value, tol in _rows_for(three):
            if kind == "bond":
                d = dist(r[atoms[0]], r[atoms[1]])
                assert abs(d - value) <= (tol if tol > 0 else EXACT_A), (three, atoms, d, value)
            elif kind == "angle":
                t = np.degrees(angle(r[atoms[0]], r[atoms[1]], r[atoms[2]]))
                assert abs(t - value) <= (tol if tol > 0 else EXACT_DEG), (three, atoms, t, value)


@pytest.mark.parametrize("seed", [3, 4])
def test_aromatic_rings_are_planar_and_chiral_centres_are_natural(seed):
    for three, code in TYPES.items():
        r = _built_residues(code, seed + 100 * code)
        for kind, res, atoms, value, tol in _rows_for(three):
            if kind == "planar":
                p = np.array([r[a] for a in atoms])
                p = p - p.mean(axis=0)
                normal = np.linalg.svd(p)[2][-1]
                assert np.abs(p @ normal).max() <= PLANAR_A, (three, atoms)
            elif kind == "chiral":
                x = r[atoms[0]]
                a, b, c = (r[q] - x for q in atoms[1:])
                # with the three heaviest substituents in CIP order a > b > c,
                # a . (b x c) > 0 is S (L-alanine's CA: N > C > CB gives S)
                vol = float(np.dot(a, np.cross(b, c)))
                assert ("S" if vol > 0 else "R") == value, (three, atoms)


def test_chirality_convention_on_alanine():
    """The sign convention of the chiral rows, checked on a centre whose
    configuration the paper fixes (R' gives L amino acids, Section 2): CA of
    ALA, N > C > CB, is S."""
    r = _built_residues(TYPES["ALA"], 7)
    x = r["CA"]
    assert np.dot(r["N"] - x, np.cross(r["C"] - x, r["CB"] - x)) > 0


# Mistakes planted in a copy of the oracle (built on the CPU in a temporary
# directory): one digit of one table value each -- a side-chain bond, a
# side-chain angle, an aromatic ring bond, a proline ring angle, a value of
# the fitted HIS ring and the backbone O angle.  The pins above must reject
# every one of them.
PLANTED = [
    ('{"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},', '{"CG", 2, "CB", "CA", "N", 1.521, 114.1, 0.0, 1},'),
    ('{"SD", 3, "CG", "CB", "CA", 1.803, 112.7, 0.0, 1},', '{"SD", 3, "CG", "CB", "CA", 1.803, 112.8, 0.0, 1},'),
    ('{"CE1", 2, "CD1", "CG", "CB", 1.382, 121.2, 180.0, 0},', '{"CE1", 2, "CD1", "CG", "CB", 1.383, 121.2, 180.0, 0},'),
    ('{"CD", 1, "CG", "CB", "CA", 1.503, 106.1, 33.0, 0}', '{"CD", 1, "CG", "CB", "CA", 1.503, 106.2, 33.0, 0}'),
    ('{"NE2", 2, "CD2", "CG", "CB", 1.382, 109.6, 180.0, 0}', '{"NE2", 2, "CD2", "CG", "CB", 1.382, 109.7, 180.0, 0}'),
    ("O_ANGLE_DEG = 120.1,", "O_ANGLE_DEG = 120.2,"),
]


@pytest.mark.parametrize("old,new", PLANTED)
def test_a_planted_table_mistake_fails_the_pins(tmp_path, old, new):
    import subprocess
    import sys

    here = os.path.dirname(os.path.abspath(oracle.__file__))
    src = open(os.path.join(here, "tpl_oracle.c")).read()
    assert old in src, old
    bad = tmp_path / "tpl_oracle.c"
    bad.write_text(src.replace(old, new, 1))  # the first residue that has it
    env = dict(os.environ, TPL_ORACLE_SRC=str(bad), TPL_ORACLE_LIB=str(tmp_path / "liboracle.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(root, "tests", "test_oracle_sidechain_geometry.py"),
                        "-k", "not planted"], cwd=root, env=env, capture_output=True, text=True)
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]
