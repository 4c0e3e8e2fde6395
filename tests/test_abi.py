"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tpl.h declares.  Host-only calls (residue tables, argument checks that
return before any CUDA call) run here without a GPU; no compute is launched.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1812_01108_gb300 import build as tpl_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tpl.h")


@pytest.fixture(scope="module")
def lib():
    path = tpl_build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpl_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_library_targets_sm103a():
    # the build passes a single gencode for compute_103a / sm_103a
    assert tpl_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_residue_tables_bit_exact_with_oracle(lib):
    lib.tpl_residue_table.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.tpl_residue_atom.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    for code in range(21):  # 0..19 amino acids, 20 the backbone-only residue
        three = ctypes.create_string_buffer(4)
        na, nc = ctypes.c_int(), ctypes.c_int()
        assert lib.tpl_residue_table(code, three, ctypes.byref(na), ctypes.byref(nc)) == 0
        o_three, o_n, o_chi, o_names, o_groups, o_r0 = oracle.residue_info(code)
        assert (three.value.decode(), na.value, nc.value) == (o_three, o_n, o_chi)
        for i in range(na.value):
            name = ctypes.create_string_buffer(8)
            grp = ctypes.c_int()
            r0 = (ctypes.c_float * 3)()
            assert lib.tpl_residue_atom(code, i, name, ctypes.byref(grp), r0) == 0
            assert name.value.decode() == o_names[i]
            assert grp.value == o_groups[i]
            # standard-frame positions: independently computed, FP32 vs FP64
            assert np.allclose(np.array(r0[:]), o_r0[i], atol=2e-6), (code, o_names[i])
    assert lib.tpl_residue_table(21, None, None, None) != 0


def test_chain_atom_counts_bit_exact_with_oracle(lib):
    lib.tpl_fullatom_chain_atoms.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.tpl_fullatom_max_atoms.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    rng = np.random.default_rng(0)
    seq = rng.integers(0, 20, size=(7, 40)).astype(np.uint8)
    lengths = np.array([0, 1, 5, 17, 39, 40, 23], np.int32)
    for b in range(7):
        n = lib.tpl_fullatom_chain_atoms(seq[b].ctypes.data_as(ctypes.c_void_p), int(lengths[b]))
        assert n == oracle.chain_atoms(seq[b], lengths[b])
    m = lib.tpl_fullatom_max_atoms(seq.ctypes.data_as(ctypes.c_void_p),
                                   lengths.ctypes.data_as(ctypes.c_void_p), 7, 40)
    assert m == oracle.max_atoms(seq, lengths)
    bad = seq.copy()
    bad[3, 2] = 25
    assert lib.tpl_fullatom_max_atoms(bad.ctypes.data_as(ctypes.c_void_p),
                                      lengths.ctypes.data_as(ctypes.c_void_p), 7, 40) == -1


def test_host_argument_checks_return_before_any_launch(lib):
    P = ctypes.c_void_p
    lib.tpl_backbone_forward.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_size_t, P, P]
    lib.tpl_lrmsd_forward.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_size_t, P]
    lib.tpl_last_error.restype = ctypes.c_char_p
    # negative batch -> TPL_ERR_INVALID_ARG (1)
    assert lib.tpl_backbone_forward(None, None, -1, 4, None, None, 0, None, None) == 1
    assert b"must be >= 0" in lib.tpl_last_error()
    # Lmax not a multiple of 4 -> TPL_ERR_BAD_SHAPE (2)
    assert lib.tpl_backbone_forward(None, None, 1, 6, None, None, 0, None, None) == 2
    # NULL pointer with B > 0 -> TPL_ERR_INVALID_ARG
    assert lib.tpl_backbone_forward(None, None, 1, 8, None, None, 0, None, None) == 1
    # misaligned pointer -> TPL_ERR_MISALIGNED (3)
    assert lib.tpl_backbone_forward(P(16), P(32), 1, 8, P(52), None, 0, None, None) == 3
    # empty batch is a no-op success
    assert lib.tpl_backbone_forward(None, None, 0, 8, None, None, 0, None, None) == 0
    assert lib.tpl_lrmsd_forward(None, None, None, 0, 8, None, None, 0, None) == 0
    assert lib.tpl_lrmsd_forward(None, None, None, 2, 6, None, None, 0, None) == 2
    # launch options: unknown flags, schedule or backward mode -> TPL_ERR_INVALID_ARG
    from paper_1812_01108_gb300 import Opts
    for bad in ({"flags": 0x2}, {"flags": -1}, {"schedule": 9}, {"bwd_mode": 5}, {"threads": -8}):
        assert lib.tpl_backbone_forward(None, None, 1, 8, None, None, 0, ctypes.byref(Opts(**bad)), None) == 1
        assert b"unknown" in lib.tpl_last_error() or b"negative" in lib.tpl_last_error()


def test_workspace_sizes(lib):
    lib.tpl_lrmsd_workspace_size.restype = ctypes.c_size_t
    lib.tpl_backbone_workspace_size.restype = ctypes.c_size_t
    assert lib.tpl_backbone_workspace_size(4096, 1000) >= 4096 * 4
    assert lib.tpl_lrmsd_workspace_size(16384, 5000) >= 16384 * 16 * 4
    assert lib.tpl_lrmsd_workspace_size(16384, 5000) % 256 == 0
