"""Seeded synthetic inputs shaped like the paper's workloads.

The paper benchmarks batches of chains with random amino-acid sequences and
random dihedral angles (Section 5, Figs. 4-6 and 8); there is no dataset to
load.  This module draws such inputs from ``numpy.random.default_rng`` and is
the only code shared by the oracle side and the CUDA side of the tests and the
benchmark.  It holds none of the method's arithmetic: no transforms, no residue
geometry, no LRMSD.  (The one rotation it applies, to make LRMSD targets, is a
library call: ``scipy.spatial.transform.Rotation``.)

Angles are drawn in float64 and cast to float32 once; both sides consume the
same float32 arrays.  Unused chi rows of a residue are drawn too and ignored by
the mapping (the residue type decides which chi rows are read).

Workload recipes (seed = 1812_01108 + index):
  0  backbone, 32 chains x 64 residues; phi, psi ~ U[-pi, pi], omega = pi;
     upstream gradient N(0, 1); LRMSD targets from angles + N(0, 0.1 rad)
  1  full atom, 64 chains, lengths U{128..350}, residue types uniform over 20;
     phi, psi, chi ~ U[-pi, pi], omega = pi
  2  backbone, 4096 chains, lengths round(exp(U[ln 50, ln 1000])), angles as 0
  3  LRMSD, 16384 pairs, N ~ U{100..5000}; x ~ N(0, 15 A); target = Rot(q) x +
     t + eps with q a random unit quaternion, t ~ N(0, 10 A), eps ~ N(0, 0.5 A)
  4  full atom, 256 chains x 700 residues (training-step shape)
  4b backbone precision stress, 64 chains x 10000 residues
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1812_01108
N_RESIDUE_TYPES = 20
BACKBONE_ONLY = 20  # residue code of a residue with its backbone N, CA, C only


def rng_for(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + int(index) + 1000 * int(salt))


def lengths_uniform(B, lo, hi, rng):
    return rng.integers(lo, hi + 1, size=B).astype(np.int32)


def lengths_loguniform(B, lo, hi, rng):
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=B))).astype(np.int32)


def pad_to(n, multiple=4):
    return int(-(-int(n) // multiple) * multiple)


def backbone_angles(lengths, rng, Lmax=None, omega=np.pi):
    """[B,3,Lmax] float32 rows phi, psi, omega; zero past each chain's length."""
    lengths = np.asarray(lengths, np.int32)
    B = lengths.shape[0]
    Lmax = pad_to(max(int(lengths.max()) if B else 1, 1)) if Lmax is None else int(Lmax)
    a = np.zeros((B, 3, Lmax), np.float64)
    a[:, 0] = rng.uniform(-np.pi, np.pi, size=(B, Lmax))
    a[:, 1] = rng.uniform(-np.pi, np.pi, size=(B, Lmax))
    a[:, 2] = omega
    mask = np.arange(Lmax)[None, :] < lengths[:, None]
    a *= mask[:, None, :]
    return a.astype(np.float32)


def fullatom_inputs(lengths, rng, Lmax=None, omega=np.pi):
    """(angles [B,7,Lmax] float32 rows phi, psi, omega, chi1..4; seq [B,Lmax] uint8)."""
    lengths = np.asarray(lengths, np.int32)
    B = lengths.shape[0]
    Lmax = pad_to(max(int(lengths.max()) if B else 1, 1)) if Lmax is None else int(Lmax)
    seq = rng.integers(0, N_RESIDUE_TYPES, size=(B, Lmax)).astype(np.uint8)
    a = np.zeros((B, 7, Lmax), np.float64)
    a[:, 0] = rng.uniform(-np.pi, np.pi, size=(B, Lmax))
    a[:, 1] = rng.uniform(-np.pi, np.pi, size=(B, Lmax))
    a[:, 2] = omega
    a[:, 3:7] = rng.uniform(-np.pi, np.pi, size=(B, 4, Lmax))
    mask = np.arange(Lmax)[None, :] < lengths[:, None]
    a *= mask[:, None, :]
    seq = np.where(mask, seq, 0).astype(np.uint8)
    return a.astype(np.float32), seq


def perturb_angles(angles, lengths, rng, sigma=0.1, rows=(0, 1)):
    """Copy of ``angles`` with N(0, sigma) added to the given rows (targets for LRMSD)."""
    a = np.array(angles, dtype=np.float64, copy=True)
    lengths = np.asarray(lengths)
    mask = np.arange(a.shape[2])[None, :] < lengths[:, None]
    for r in rows:
        a[:, r] += rng.normal(0.0, sigma, size=a[:, r].shape) * mask
    return a.astype(np.float32)


def upstream_grad(shape, rng, valid=None):
    """N(0, 1) upstream gradient, zero on padding rows when ``valid`` [B] atom counts are given."""
    g = rng.normal(0.0, 1.0, size=shape)
    if valid is not None:
        valid = np.asarray(valid)
        g *= (np.arange(shape[1])[None, :] < valid[:, None])[:, :, None]
    return g.astype(np.float32)


def lrmsd_clouds(P, n_lo, n_hi, rng, Nmax=None, sigma=15.0, shift=10.0, noise=0.5):
    """(input [P,Nmax,3], target [P,Nmax,3], num_atoms [P]) float32 clouds, zero padded.

    input = x ~ N(0, sigma); target = Rot(q) x + t + eps.
    """
    from scipy.spatial.transform import Rotation

    n = rng.integers(n_lo, n_hi + 1, size=P).astype(np.int32)
    Nmax = pad_to(int(n.max()) if P else 1) if Nmax is None else int(Nmax)
    x = rng.normal(0.0, sigma, size=(P, Nmax, 3))
    q = rng.normal(size=(P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rot = Rotation.from_quat(q).as_matrix()
    t = rng.normal(0.0, shift, size=(P, 1, 3))
    eps = rng.normal(0.0, noise, size=(P, Nmax, 3))
    y = np.einsum("pij,pnj->pni", rot, x) + t + eps
    mask = (np.arange(Nmax)[None, :] < n[:, None])[:, :, None]
    return (x * mask).astype(np.float32), (y * mask).astype(np.float32), n


# ----------------------------------------------------------------------------- configs
def config0():
    rng = rng_for(0)
    lengths = np.full(32, 64, np.int32)
    a = backbone_angles(lengths, rng)
    g = upstream_grad((32, 3 * a.shape[2], 3), rng, valid=3 * lengths)
    target_angles = perturb_angles(a, lengths, rng)
    return {"name": "backbone 32x64", "angles": a, "lengths": lengths, "grad": g,
            "target_angles": target_angles}


def config1():
    rng = rng_for(1)
    lengths = lengths_uniform(64, 128, 350, rng)
    a, seq = fullatom_inputs(lengths, rng)
    target_angles = perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    return {"name": "full-atom 64 x U{128..350}", "angles": a, "seq": seq, "lengths": lengths,
            "target_angles": target_angles}


def config2(B=4096):
    rng = rng_for(2)
    lengths = lengths_loguniform(B, 50, 1000, rng)
    a = backbone_angles(lengths, rng)
    target_angles = perturb_angles(a, lengths, rng)
    return {"name": f"backbone {B} x logU[50,1000]", "angles": a, "lengths": lengths,
            "target_angles": target_angles}


def config3(P=16384, n_lo=100, n_hi=5000):
    rng = rng_for(3)
    x, y, n = lrmsd_clouds(P, n_lo, n_hi, rng)
    return {"name": f"LRMSD {P} pairs x U{{{n_lo}..{n_hi}}}", "input": x, "target": y,
            "num_atoms": n}


def config4(B=256, L=700):
    rng = rng_for(4)
    lengths = np.full(B, L, np.int32)
    a, seq = fullatom_inputs(lengths, rng)
    target_angles = perturb_angles(a, lengths, rng, rows=(0, 1, 3, 4, 5, 6))
    return {"name": f"full-atom training step {B}x{L}", "angles": a, "seq": seq,
            "lengths": lengths, "target_angles": target_angles}


def config4b(B=64, L=10000):
    rng = rng_for(5)
    lengths = np.full(B, L, np.int32)
    a = backbone_angles(lengths, rng)
    return {"name": f"backbone stress {B}x{L}", "angles": a, "lengths": lengths}
