"""Plain FP64 CPU oracle for the angles -> coordinates mapping, its adjoint and LRMSD.

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA library; only
the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import it.  It shares no code, header, table or constant with the CUDA
path (``tpl_oracle.c`` is compiled by gcc on its own).

Every function takes and returns numpy arrays.  Floating inputs are promoted to
float64 before the call, so an FP32 array handed to both the oracle and the
CUDA library is the same input for both.

Paper sections followed (Derevyanko & Lamoureux 2018, "TorchProteinLibrary"):
  * backbone_forward / backbone_backward: Section 3 (explicit R, atom index rule,
    M_i = R_0 ... R_i, derivative of r_i and the sums of Eq. 2);
  * fullatom_forward / fullatom_backward: Section 2 (transform graph, R', r = M r0,
    Eq. 1);
  * lrmsd_forward / lrmsd_backward: Section 4 (Coutsias-Seok-Dill quaternion method).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, geometry invariants, finite differences, library and brute-force
cross-checks).  The full-atom side-chain geometry is authored (the paper prints
none); every bond and angle of it is pinned against the Engh & Huber (1991)
values typed into tests/golden/sidechain_geometry.txt.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The source and library paths can be redirected (TPL_ORACLE_SRC / TPL_ORACLE_LIB)
# so that a test can build a copy of the oracle with a planted mistake and
# check that the pins catch it.
_SRC = os.environ.get("TPL_ORACLE_SRC", os.path.join(_HERE, "tpl_oracle.c"))
_LIB_PATH = os.environ.get("TPL_ORACLE_LIB", os.path.join(_HERE, "liboracle.so"))
_lock = threading.Lock()
_lib = None

RESIDUES = ("ALA", "ARG", "ASN", "ASP", "CYS", "GLN", "GLU", "GLY", "HIS", "ILE",
            "LEU", "LYS", "MET", "PHE", "PRO", "SER", "THR", "TRP", "TYR", "VAL")


def build(force: bool = False) -> str:
    """Compile ``tpl_oracle.c`` into ``liboracle.so`` with gcc (-O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tpl_oracle.h"))):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", "-I", _HERE, "-o", tmp,
                        _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_backbone_forward.argtypes = [P, P, I, I, P]
            lib.oracle_backbone_backward.argtypes = [P, P, I, I, P, P]
            lib.oracle_backbone_forward_o.argtypes = [P, P, I, I, P, P]
            lib.oracle_backbone_backward_o.argtypes = [P, P, I, I, P, P, P]
            lib.oracle_fullatom_forward.argtypes = [P, P, P, I, I, I, P, P]
            lib.oracle_fullatom_backward.argtypes = [P, P, P, I, I, I, P, P]
            lib.oracle_fullatom_chain_atoms.argtypes = [P, I]
            lib.oracle_residue_info.argtypes = [I, P, P, P]
            lib.oracle_residue_atom.argtypes = [I, I, P, P]
            lib.oracle_residue_atom_r0.argtypes = [I, I, P]
            lib.oracle_lrmsd_forward.argtypes = [P, P, P, I, I, P, P, P]
            lib.oracle_lrmsd_backward.argtypes = [P, P, P, P, I, I, P]
            lib.oracle_sym4_eig.argtypes = [P, P, P]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


# ----------------------------------------------------------------------------- backbone
def backbone_forward(angles, lengths):
    """angles [B,3,Lmax] (phi, psi, omega) -> coords [B,3*Lmax,3]; Section 3."""
    a = _f64(angles)
    ln = _i32(lengths)
    B, _, Lmax = a.shape
    out = np.zeros((B, 3 * Lmax, 3), np.float64)
    _check(_load().oracle_backbone_forward(_p(a), _p(ln), B, Lmax, _p(out)), "backbone_forward")
    return out


def backbone_backward(angles, lengths, grad_coords):
    """dL/d(phi, psi, omega) [B,3,Lmax] from dL/dr [B,3*Lmax,3]; Section 3, Eq. 2."""
    a = _f64(angles)
    ln = _i32(lengths)
    g = _f64(grad_coords)
    B, _, Lmax = a.shape
    out = np.zeros((B, 3, Lmax), np.float64)
    _check(_load().oracle_backbone_backward(_p(a), _p(ln), B, Lmax, _p(g), _p(out)),
           "backbone_backward")
    return out


def backbone_forward_o(angles, lengths):
    """Backbone with the carbonyl O: (coords [B,3*Lmax,3], O [B,Lmax,3]); O_j rigid
    in the frame of C_j after psi_j (bond C-O, angle CA-C-O, dihedral
    N-CA-C-O = psi_j + 180); Section 3 with the full-atom tables' O."""
    a = _f64(angles)
    ln = _i32(lengths)
    B, _, Lmax = a.shape
    out = np.zeros((B, 3 * Lmax, 3), np.float64)
    o = np.zeros((B, Lmax, 3), np.float64)
    _check(_load().oracle_backbone_forward_o(_p(a), _p(ln), B, Lmax, _p(out), _p(o)), "backbone_forward_o")
    return out, o


def backbone_backward_o(angles, lengths, grad_coords, grad_o):
    """Eq. 2 with the O atoms among the moved atoms: dL/d(phi, psi, omega)."""
    a = _f64(angles)
    ln = _i32(lengths)
    g = _f64(grad_coords)
    go = _f64(grad_o)
    B, _, Lmax = a.shape
    out = np.zeros((B, 3, Lmax), np.float64)
    _check(_load().oracle_backbone_backward_o(_p(a), _p(ln), B, Lmax, _p(g), _p(go), _p(out)),
           "backbone_backward_o")
    return out


# ----------------------------------------------------------------------------- full atom
def chain_atoms(seq, length):
    s = _u8(seq)
    n = _load().oracle_fullatom_chain_atoms(_p(s), int(length))
    if n < 0:
        raise ValueError("bad residue code")
    return n


def max_atoms(seq, lengths):
    s = _u8(seq)
    return max([chain_atoms(s[b], int(lengths[b])) for b in range(s.shape[0])] + [0])


def fullatom_forward(angles, seq, lengths, Amax=None):
    """angles [B,7,Lmax] (phi, psi, omega, chi1..4), seq [B,Lmax] -> (coords [B,Amax,3],
    num_atoms [B]); Section 2."""
    a = _f64(angles)
    s = _u8(seq)
    ln = _i32(lengths)
    B, _, Lmax = a.shape
    if Amax is None:
        Amax = max_atoms(s, ln)
    out = np.zeros((B, Amax, 3), np.float64)
    na = np.zeros((B,), np.int32)
    _check(_load().oracle_fullatom_forward(_p(a), _p(s), _p(ln), B, Lmax, Amax, _p(out), _p(na)),
           "fullatom_forward")
    return out, na


def fullatom_backward(angles, seq, lengths, grad_coords):
    """dL/d(angles) [B,7,Lmax] from dL/dr [B,Amax,3]; Section 2, Eq. 1."""
    a = _f64(angles)
    s = _u8(seq)
    ln = _i32(lengths)
    g = _f64(grad_coords)
    B, _, Lmax = a.shape
    Amax = g.shape[1]
    out = np.zeros((B, 7, Lmax), np.float64)
    _check(_load().oracle_fullatom_backward(_p(a), _p(s), _p(ln), B, Lmax, Amax, _p(g), _p(out)),
           "fullatom_backward")
    return out


def residue_info(code):
    """(three-letter name, n_atoms, n_chi, [atom names], [group ids], r0 [n_atoms,3])."""
    lib = _load()
    name = ctypes.create_string_buffer(4)
    na = ctypes.c_int()
    nc = ctypes.c_int()
    _check(lib.oracle_residue_info(int(code), name, ctypes.byref(na), ctypes.byref(nc)),
           "residue_info")
    names, groups = [], []
    r0 = np.zeros((na.value, 3), np.float64)
    for i in range(na.value):
        nm = ctypes.create_string_buffer(8)
        g = ctypes.c_int()
        _check(lib.oracle_residue_atom(int(code), i, nm, ctypes.byref(g)), "residue_atom")
        names.append(nm.value.decode())
        groups.append(g.value)
        _check(lib.oracle_residue_atom_r0(int(code), i, _p(r0[i])), "residue_atom_r0")
    return name.value.decode(), na.value, nc.value, names, groups, r0


# ----------------------------------------------------------------------------- LRMSD
def lrmsd_forward(input, target, num_atoms, return_aux=False):
    """LRMSD(x = target, y = input) per pair; Section 4.  Optionally (U [P,3,3], lambda [P])."""
    y = _f64(input)
    x = _f64(target)
    n = _i32(num_atoms)
    P, Nmax, _ = y.shape
    out = np.zeros((P,), np.float64)
    U = np.zeros((P, 3, 3), np.float64)
    lam = np.zeros((P,), np.float64)
    _check(_load().oracle_lrmsd_forward(_p(y), _p(x), _p(n), P, Nmax, _p(out), _p(U), _p(lam)),
           "lrmsd_forward")
    return (out, U, lam) if return_aux else out


def lrmsd_backward(grad_lrmsd, input, target, num_atoms):
    """dLRMSD/d(input) [P,Nmax,3] scaled by grad_lrmsd [P]; Section 4."""
    gl = _f64(grad_lrmsd)
    y = _f64(input)
    x = _f64(target)
    n = _i32(num_atoms)
    P, Nmax, _ = y.shape
    out = np.zeros((P, Nmax, 3), np.float64)
    _check(_load().oracle_lrmsd_backward(_p(gl), _p(y), _p(x), _p(n), P, Nmax, _p(out)),
           "lrmsd_backward")
    return out


def sym4_eig(A):
    """Cyclic-Jacobi eigen-decomposition of a symmetric 4x4: (evals ascending, evecs columns)."""
    a = _f64(A).reshape(16)
    ev = np.zeros(4, np.float64)
    V = np.zeros(16, np.float64)
    _load().oracle_sym4_eig(_p(a), _p(ev), _p(V))
    return ev, V.reshape(4, 4)
