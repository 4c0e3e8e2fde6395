"""GB300 (sm_103a) implementation of the differentiable dihedral-angle ->
Cartesian-coordinate mapping of proteins and of LRMSD, after Derevyanko &
Lamoureux, "TorchProteinLibrary" (2018).

This module is argument marshalling only: every step of the computation runs
in the hand-written CUDA kernels of ``libtpl.so`` (C ABI in ``include/tpl.h``).
PyTorch provides device memory, streams and autograd.  There is no CPU path:
if the library is not built, or a tensor is not on a CUDA device, the calls
raise.

Two layers:
  * ``tpl_*`` functions mirror the C ABI one to one (caller-allocated outputs
    and workspace, the current CUDA stream);
  * ``backbone``, ``fullatom`` and ``lrmsd`` are ``torch.autograd.Function``
    wrappers that allocate outputs and workspaces with PyTorch.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = [
    "TplError", "Opts", "library_path", "load_library", "tpl_backbone_forward",
    "tpl_backbone_backward", "tpl_fullatom_forward", "tpl_fullatom_backward",
    "tpl_lrmsd_forward", "tpl_lrmsd_backward", "tpl_lrmsd_forward_noalloc",
    "tpl_backbone_forward_ref64",
    "tpl_backbone_backward_ref64", "tpl_fullatom_forward_ref64", "tpl_fullatom_backward_ref64",
    "tpl_lrmsd_forward_ref64", "tpl_lrmsd_backward_ref64", "tpl_get_status",
    "tpl_selftest_wait_timeout", "tpl_backbone_autotune", "tpl_fullatom_autotune",
    "tpl_backbone_lrmsd_autotune", "tpl_fullatom_lrmsd_autotune", "tpl_lrmsd_forward_launches",
    "tpl_backbone_backward_quadratic",
    "tpl_fullatom_backward_lrmsd", "tpl_backbone_backward_lrmsd", "tpl_fullatom_lrmsd_workspace_size",
    "tpl_fullatom_lrmsd_forward", "tpl_fullatom_lrmsd_backward", "backbone",
    "fullatom", "lrmsd", "residue_table", "fullatom_max_atoms", "BWD_RECOMPUTE",
    "BWD_FROM_COORDS", "SCHED_LONGEST_FIRST", "SCHED_BATCH_ORDER", "SCHED_PACKED",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtpl.so")
_lib = None
_lock = threading.Lock()

BWD_AUTO, BWD_RECOMPUTE, BWD_FROM_COORDS = 0, 1, 2
SCHED_AUTO, SCHED_LONGEST_FIRST, SCHED_BATCH_ORDER, SCHED_PACKED = 0, 1, 2, 3
STATUS_BAD_RESIDUE, STATUS_BAD_LENGTH, STATUS_TOO_MANY_ATOMS, STATUS_ZERO_LRMSD = 1, 2, 4, 8
STATUS_TIMEOUT, STATUS_BAD_WORKSPACE = 16, 32
FLAG_PADDING_ZEROED = 0x1


class TplError(RuntimeError):
    """A tpl_* call returned a nonzero status."""

    def __init__(self, name, code, message):
        super().__init__(f"{name} failed with status {code}: {message}")
        self.code = code


class Opts(ctypes.Structure):
    """``tpl_opts``: zero fields mean automatic."""

    _fields_ = [("bwd_mode", ctypes.c_int), ("threads", ctypes.c_int),
                ("res_per_thread", ctypes.c_int), ("schedule", ctypes.c_int),
                ("flags", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load ``libtpl.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with paper_1812_01108_gb300.build.build() "
                "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(_LIB_PATH)
        P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        O = ctypes.POINTER(Opts)
        F = ctypes.POINTER(ctypes.c_float)
        sig = {
            "tpl_backbone_workspace_size": ([I, I], Z),
            "tpl_fullatom_workspace_size": ([I, I], Z),
            "tpl_lrmsd_workspace_size": ([I, I], Z),
            "tpl_backbone_forward": ([P, P, I, I, P, P, Z, O, P], I),
            "tpl_backbone_backward": ([P, P, I, I, P, P, P, P, Z, O, P], I),
            "tpl_fullatom_forward": ([P, P, P, I, I, I, P, P, P, Z, O, P], I),
            "tpl_fullatom_backward": ([P, P, P, I, I, I, P, P, P, P, Z, O, P], I),
            "tpl_fullatom_backward_lrmsd": ([P, P, P, I, I, I, P, P, P, P, Z, P, P, Z, O, P], I),
            "tpl_backbone_backward_lrmsd": ([P, P, I, I, P, P, P, P, Z, P, P, Z, O, P], I),
            "tpl_fullatom_lrmsd_workspace_size": ([I, I], Z),
            "tpl_backbone_lrmsd_workspace_size": ([I, I], Z),
            "tpl_backbone_lrmsd_step": ([P, P, I, I, P, P, P, P, P, P, Z, O, P], I),
            "tpl_fullatom_lrmsd_forward": ([P, P, P, I, I, I, P, P, P, P, P, Z, O, P], I),
            "tpl_fullatom_lrmsd_backward": ([P, P, I, I, I, P, P, P, P, P, Z, O, P], I),
            "tpl_lrmsd_forward": ([P, P, P, I, I, P, P, Z, P], I),
            "tpl_lrmsd_backward": ([P, P, P, P, I, I, P, P, Z, P], I),
            "tpl_lrmsd_forward_noalloc": ([P, P, P, I, I, P, P], I),
            "tpl_backbone_forward_ref64": ([P, P, I, I, P, P], I),
            "tpl_backbone_backward_ref64": ([P, P, I, I, P, P, P, P], I),
            "tpl_fullatom_forward_ref64": ([P, P, P, I, I, I, P, P, P], I),
            "tpl_fullatom_backward_ref64": ([P, P, P, I, I, I, P, P, P, P], I),
            "tpl_lrmsd_forward_ref64": ([P, P, P, I, I, P, P, P], I),
            "tpl_lrmsd_backward_ref64": ([P, P, P, P, I, I, P, P, P], I),
            "tpl_residue_table": ([I, P, P, P], I),
            "tpl_residue_atom": ([I, I, P, P, P], I),
            "tpl_fullatom_chain_atoms": ([P, I], I),
            "tpl_fullatom_max_atoms": ([P, P, I, I], I),
            "tpl_get_status": ([P, P], I),
            "tpl_selftest_wait_timeout": ([P, P], I),
            "tpl_backbone_autotune": ([P, P, I, I, P, P, P, P, Z, I, O, F, P], I),
            "tpl_fullatom_autotune": ([P, P, P, I, I, I, P, P, P, P, P, Z, I, O, F, P], I),
            "tpl_lrmsd_forward_launches": ([I], I),
            "tpl_backbone_backward_quadratic": ([P, I, I, P, P, P, P], I),
            "tpl_backbone_forward_o": ([P, P, I, I, P, P, P, Z, O, P], I),
            "tpl_backbone_backward_o": ([P, P, I, I, P, P, P, P, P, P, Z, O, P], I),
            "tpl_fullatom_backward_quadratic": ([P, P, I, I, I, P, P, P, P], I),
            "tpl_backbone_lrmsd_autotune": ([P, P, I, I, P, P, P, P, P, P, Z, P, P, Z, O, F, P], I),
            "tpl_fullatom_lrmsd_autotune": ([P, P, P, I, I, I, P, P, P, P, P, P, Z, P, P, Z, O, F, P], I),
            "tpl_last_error": ([], ctypes.c_char_p),
            "tpl_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(name, code):
    if code != 0:
        raise TplError(name, code, load_library().tpl_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream(t, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return ctypes.c_void_p(s.cuda_stream)


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, Opts):
        return ctypes.byref(opts)
    return ctypes.byref(Opts(**opts))


# ----------------------------------------------------------------------------- C ABI mirror
def tpl_backbone_workspace_size(B, Lmax):
    return int(load_library().tpl_backbone_workspace_size(B, Lmax))


def tpl_fullatom_workspace_size(B, Lmax):
    return int(load_library().tpl_fullatom_workspace_size(B, Lmax))


def tpl_lrmsd_workspace_size(P, Nmax):
    return int(load_library().tpl_lrmsd_workspace_size(P, Nmax))


def tpl_backbone_forward(angles, lengths, coords, workspace, opts=None, stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_backbone_forward", load_library().tpl_backbone_forward(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float32, "coords")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_backbone_backward(angles, lengths, coords, grad_coords, grad_angles, workspace, opts=None,
                          stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_backbone_backward", load_library().tpl_backbone_backward(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(coords), _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_fullatom_forward(angles, seq, lengths, coords, num_atoms, workspace, opts=None, stream=None):
    B, _, Lmax = angles.shape
    Amax = coords.shape[1]
    _check("tpl_fullatom_forward", load_library().tpl_fullatom_forward(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(num_atoms, torch.int32, "num_atoms")),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _opts(opts),
        _stream(angles, stream)))


def tpl_fullatom_backward(angles, seq, lengths, coords, grad_coords, grad_angles, workspace,
                          opts=None, stream=None):
    B, _, Lmax = angles.shape
    Amax = grad_coords.shape[1]
    _check("tpl_fullatom_backward", load_library().tpl_fullatom_backward(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax, _ptr(coords),
        _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_backbone_autotune(angles, lengths, coords, grad_coords, grad_angles, workspace,
                          bwd_mode=0, stream=None):
    """Times forward + backward for every launch shape and schedule on this
    batch; returns (fastest Opts, its milliseconds).  Overwrites coords and
    grad_angles.  Not capturable."""
    B, _, Lmax = angles.shape
    best = Opts()
    ms = ctypes.c_float(0.0)
    _check("tpl_backbone_autotune", load_library().tpl_backbone_autotune(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float32, "coords")),
        _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), int(bwd_mode), ctypes.byref(best),
        ctypes.byref(ms), _stream(angles, stream)))
    return best, ms.value


def tpl_fullatom_autotune(angles, seq, lengths, coords, num_atoms, grad_coords, grad_angles,
                          workspace, bwd_mode=0, stream=None):
    """As tpl_backbone_autotune for the full-atom calls; overwrites coords,
    num_atoms and grad_angles."""
    B, _, Lmax = angles.shape
    Amax = coords.shape[1]
    best = Opts()
    ms = ctypes.c_float(0.0)
    _check("tpl_fullatom_autotune", load_library().tpl_fullatom_autotune(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(num_atoms, torch.int32, "num_atoms")),
        _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), int(bwd_mode), ctypes.byref(best),
        ctypes.byref(ms), _stream(angles, stream)))
    return best, ms.value


def tpl_lrmsd_forward_launches(P):
    """Kernels tpl_lrmsd_forward launches for P pairs on the current device."""
    return int(load_library().tpl_lrmsd_forward_launches(int(P)))


def tpl_backbone_lrmsd_autotune(angles, lengths, coords, target, num_atoms, grad_lrmsd, lrmsd,
                                lrmsd_workspace, grad_angles, workspace, stream=None):
    """Times the LRMSD training step (forward, tpl_lrmsd_forward, fused backward)
    for every launch shape and schedule; returns (fastest Opts, its milliseconds).
    Overwrites coords, lrmsd, lrmsd_workspace and grad_angles.  Not capturable."""
    B, _, Lmax = angles.shape
    best = Opts()
    ms = ctypes.c_float(0.0)
    _check("tpl_backbone_lrmsd_autotune", load_library().tpl_backbone_lrmsd_autotune(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")),
        _ptr(_cuda(lrmsd, torch.float32, "lrmsd")), _ptr(lrmsd_workspace),
        lrmsd_workspace.numel() * lrmsd_workspace.element_size(),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), ctypes.byref(best), ctypes.byref(ms),
        _stream(angles, stream)))
    return best, ms.value


def tpl_fullatom_lrmsd_autotune(angles, seq, lengths, coords, num_atoms, target, grad_lrmsd, lrmsd,
                                lrmsd_workspace, grad_angles, workspace, stream=None):
    """As tpl_backbone_lrmsd_autotune for the full-atom calls; also overwrites
    num_atoms."""
    B, _, Lmax = angles.shape
    Amax = coords.shape[1]
    best = Opts()
    ms = ctypes.c_float(0.0)
    _check("tpl_fullatom_lrmsd_autotune", load_library().tpl_fullatom_lrmsd_autotune(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(num_atoms, torch.int32, "num_atoms")),
        _ptr(_cuda(target, torch.float32, "target")), _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")),
        _ptr(_cuda(lrmsd, torch.float32, "lrmsd")), _ptr(lrmsd_workspace),
        lrmsd_workspace.numel() * lrmsd_workspace.element_size(),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), ctypes.byref(best), ctypes.byref(ms),
        _stream(angles, stream)))
    return best, ms.value


def tpl_backbone_lrmsd_workspace_size(B, Lmax):
    return int(load_library().tpl_backbone_lrmsd_workspace_size(B, Lmax))


def tpl_backbone_lrmsd_step(angles, lengths, target, grad_lrmsd, coords, lrmsd, grad_angles, workspace,
                            opts=None, stream=None):
    """Backbone training step on the LRMSD loss: fills coords, lrmsd and
    grad_angles = d(sum_b grad_lrmsd[b] LRMSD_b) / d(angles) in one call."""
    B, _, Lmax = angles.shape
    _check("tpl_backbone_lrmsd_step", load_library().tpl_backbone_lrmsd_step(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")), _ptr(_cuda(coords, torch.float32, "coords")),
        _ptr(_cuda(lrmsd, torch.float32, "lrmsd")), _ptr(_cuda(grad_angles, torch.float32, "grad_angles")),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_fullatom_lrmsd_workspace_size(B, Lmax):
    return int(load_library().tpl_fullatom_lrmsd_workspace_size(B, Lmax))


def tpl_fullatom_lrmsd_forward(angles, seq, lengths, target, coords, num_atoms, lrmsd_out, workspace, opts=None,
                               stream=None):
    """Fused training step, forward: coordinates, atom counts and the LRMSD
    against ``target``; the rotation and the gradient scale stay in ``workspace``."""
    B, _, Lmax = angles.shape
    Amax = coords.shape[1]
    _check("tpl_fullatom_lrmsd_forward", load_library().tpl_fullatom_lrmsd_forward(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(target, torch.float32, "target")), _ptr(_cuda(coords, torch.float32, "coords")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), _ptr(_cuda(lrmsd_out, torch.float32, "lrmsd")),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_fullatom_lrmsd_backward(seq, lengths, coords, target, grad_lrmsd, grad_angles, workspace, opts=None,
                                stream=None):
    """Fused training step, backward: angle gradients of sum_b grad_lrmsd[b] * LRMSD_b."""
    B, Lmax = seq.shape
    Amax = coords.shape[1]
    _check("tpl_fullatom_lrmsd_backward", load_library().tpl_fullatom_lrmsd_backward(
        _ptr(_cuda(seq, torch.uint8, "seq")), _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")), _ptr(_cuda(grad_angles, torch.float32, "grad_angles")),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _opts(opts), _stream(coords, stream)))


def tpl_backbone_forward_o(angles, lengths, coords, o_coords, workspace, opts=None, stream=None):
    """Backbone forward that also places each residue's carbonyl O (o_coords [B, Lmax, 3])."""
    B, _, Lmax = angles.shape
    _check("tpl_backbone_forward_o", load_library().tpl_backbone_forward_o(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(o_coords, torch.float32, "o_coords")),
        _ptr(workspace), workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_backbone_backward_o(angles, lengths, coords, o_coords, grad_coords, grad_o, grad_angles, workspace,
                            opts=None, stream=None):
    """Backbone backward with the O atoms among the moved atoms (grad_o [B, Lmax, 3])."""
    B, _, Lmax = angles.shape
    _check("tpl_backbone_backward_o", load_library().tpl_backbone_backward_o(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax,
        _ptr(coords), _ptr(o_coords),
        _ptr(_cuda(grad_coords, torch.float32, "grad_coords")), _ptr(_cuda(grad_o, torch.float32, "grad_o")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_backbone_backward_quadratic(lengths, coords, grad_coords, grad_angles, stream=None):
    """The paper's O(L^2) form of the backbone backward (every angle-atom term
    summed directly), a comparator for tpl_backbone_backward."""
    B, _, Lmax = grad_angles.shape
    _check("tpl_backbone_backward_quadratic", load_library().tpl_backbone_backward_quadratic(
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, _ptr(_cuda(coords, torch.float32, "coords")),
        _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _stream(grad_angles, stream)))


def tpl_fullatom_backward_quadratic(seq, lengths, coords, grad_coords, grad_angles, stream=None):
    """The paper's depth-first O(L^2) form of the full-atom backward (each angle
    sums over the atoms it moves), a comparator for tpl_fullatom_backward."""
    B, _, Lmax = grad_angles.shape
    Amax = coords.shape[1]
    _check("tpl_fullatom_backward_quadratic", load_library().tpl_fullatom_backward_quadratic(
        _ptr(_cuda(seq, torch.uint8, "seq")), _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(grad_coords, torch.float32, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _stream(grad_angles, stream)))


def tpl_backbone_backward_lrmsd(angles, lengths, coords, target, grad_lrmsd, lrmsd_workspace,
                                grad_angles, workspace, opts=None, stream=None):
    """Backward of sum_b grad_lrmsd[b] * LRMSD(coords[b], target[b]) to the backbone
    angles in one call."""
    B, _, Lmax = angles.shape
    _check("tpl_backbone_backward_lrmsd", load_library().tpl_backbone_backward_lrmsd(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")), _ptr(lrmsd_workspace),
        lrmsd_workspace.numel() * lrmsd_workspace.element_size(),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_fullatom_backward_lrmsd(angles, seq, lengths, coords, target, grad_lrmsd, lrmsd_workspace,
                                grad_angles, workspace, opts=None, stream=None):
    """Backward of sum_b grad_lrmsd[b] * LRMSD(coords[b], target[b]) to the angles
    in one call (the LRMSD gradient is formed in the kernel)."""
    B, _, Lmax = angles.shape
    Amax = coords.shape[1]
    _check("tpl_fullatom_backward_lrmsd", load_library().tpl_fullatom_backward_lrmsd(
        _ptr(_cuda(angles, torch.float32, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, Amax,
        _ptr(_cuda(coords, torch.float32, "coords")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")), _ptr(lrmsd_workspace),
        lrmsd_workspace.numel() * lrmsd_workspace.element_size(),
        _ptr(_cuda(grad_angles, torch.float32, "grad_angles")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _opts(opts), _stream(angles, stream)))


def tpl_lrmsd_forward(input, target, num_atoms, lrmsd_out, workspace, stream=None):
    P, Nmax, _ = input.shape
    _check("tpl_lrmsd_forward", load_library().tpl_lrmsd_forward(
        _ptr(_cuda(input, torch.float32, "input")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), P, Nmax,
        _ptr(_cuda(lrmsd_out, torch.float32, "lrmsd")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(input, stream)))


def tpl_lrmsd_forward_noalloc(input, target, num_atoms, lrmsd_out, stream=None):
    """LRMSD forward with the library's fixed internal scratch (no workspace).
    The C call uses the scratch array of the current device, so the tensors'
    device is made current for it."""
    P, Nmax, _ = input.shape
    with torch.cuda.device(_cuda(input, torch.float32, "input").device):
        _check("tpl_lrmsd_forward_noalloc", load_library().tpl_lrmsd_forward_noalloc(
            _ptr(input), _ptr(_cuda(target, torch.float32, "target")),
            _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), P, Nmax,
            _ptr(_cuda(lrmsd_out, torch.float32, "lrmsd")), _stream(input, stream)))


def tpl_lrmsd_backward(grad_lrmsd, input, target, num_atoms, grad_input, workspace, stream=None):
    P, Nmax, _ = input.shape
    _check("tpl_lrmsd_backward", load_library().tpl_lrmsd_backward(
        _ptr(_cuda(grad_lrmsd, torch.float32, "grad_lrmsd")),
        _ptr(_cuda(input, torch.float32, "input")), _ptr(_cuda(target, torch.float32, "target")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), P, Nmax,
        _ptr(_cuda(grad_input, torch.float32, "grad_input")), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(input, stream)))


def tpl_backbone_forward_ref64(angles, lengths, coords, stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_backbone_forward_ref64", load_library().tpl_backbone_forward_ref64(
        _ptr(_cuda(angles, torch.float64, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float64, "coords")), _stream(angles, stream)))


def tpl_backbone_backward_ref64(angles, lengths, coords, grad_coords, grad_angles, stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_backbone_backward_ref64", load_library().tpl_backbone_backward_ref64(
        _ptr(_cuda(angles, torch.float64, "angles")), _ptr(_cuda(lengths, torch.int32, "lengths")),
        B, Lmax, _ptr(_cuda(coords, torch.float64, "coords")),
        _ptr(_cuda(grad_coords, torch.float64, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float64, "grad_angles")), _stream(angles, stream)))


def tpl_fullatom_forward_ref64(angles, seq, lengths, coords, num_atoms, stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_fullatom_forward_ref64", load_library().tpl_fullatom_forward_ref64(
        _ptr(_cuda(angles, torch.float64, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, coords.shape[1],
        _ptr(_cuda(coords, torch.float64, "coords")), _ptr(_cuda(num_atoms, torch.int32, "num_atoms")),
        _stream(angles, stream)))


def tpl_fullatom_backward_ref64(angles, seq, lengths, coords, grad_coords, grad_angles, stream=None):
    B, _, Lmax = angles.shape
    _check("tpl_fullatom_backward_ref64", load_library().tpl_fullatom_backward_ref64(
        _ptr(_cuda(angles, torch.float64, "angles")), _ptr(_cuda(seq, torch.uint8, "seq")),
        _ptr(_cuda(lengths, torch.int32, "lengths")), B, Lmax, coords.shape[1],
        _ptr(_cuda(coords, torch.float64, "coords")),
        _ptr(_cuda(grad_coords, torch.float64, "grad_coords")),
        _ptr(_cuda(grad_angles, torch.float64, "grad_angles")), _stream(angles, stream)))


def tpl_lrmsd_forward_ref64(input, target, num_atoms, lrmsd_out, state, stream=None):
    P, Nmax, _ = input.shape
    _check("tpl_lrmsd_forward_ref64", load_library().tpl_lrmsd_forward_ref64(
        _ptr(_cuda(input, torch.float64, "input")), _ptr(_cuda(target, torch.float64, "target")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), P, Nmax,
        _ptr(_cuda(lrmsd_out, torch.float64, "lrmsd")), _ptr(_cuda(state, torch.float64, "state")),
        _stream(input, stream)))


def tpl_lrmsd_backward_ref64(grad_lrmsd, input, target, num_atoms, state, grad_input, stream=None):
    P, Nmax, _ = input.shape
    _check("tpl_lrmsd_backward_ref64", load_library().tpl_lrmsd_backward_ref64(
        _ptr(_cuda(grad_lrmsd, torch.float64, "grad_lrmsd")),
        _ptr(_cuda(input, torch.float64, "input")), _ptr(_cuda(target, torch.float64, "target")),
        _ptr(_cuda(num_atoms, torch.int32, "num_atoms")), P, Nmax,
        _ptr(_cuda(state, torch.float64, "state")),
        _ptr(_cuda(grad_input, torch.float64, "grad_input")), _stream(input, stream)))


def tpl_selftest_wait_timeout(flag, stream=None):
    """Bounded wait on ``flag`` (an int32 CUDA tensor the caller keeps at 0):
    gives up after the poll limit and sets TPL_STATUS_TIMEOUT."""
    import torch

    _check("tpl_selftest_wait_timeout", load_library().tpl_selftest_wait_timeout(
        _ptr(_cuda(flag, torch.int32, "flag")), _stream(flag, stream)))


def tpl_get_status(device=None):
    """Read and clear the device status word (synchronises the current stream)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    out = ctypes.c_int(0)
    _check("tpl_get_status", load_library().tpl_get_status(
        ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream), ctypes.byref(out)))
    return out.value


def residue_table(code):
    """(three-letter name, n_atoms, n_chi, [(atom name, group, r0 xyz)])."""
    lib = load_library()
    three = ctypes.create_string_buffer(4)
    na, nc = ctypes.c_int(), ctypes.c_int()
    _check("tpl_residue_table", lib.tpl_residue_table(code, three, ctypes.byref(na), ctypes.byref(nc)))
    atoms = []
    for i in range(na.value):
        name = ctypes.create_string_buffer(8)
        grp = ctypes.c_int()
        r0 = (ctypes.c_float * 3)()
        _check("tpl_residue_atom", lib.tpl_residue_atom(code, i, name, ctypes.byref(grp), r0))
        atoms.append((name.value.decode(), grp.value, tuple(r0)))
    return three.value.decode(), na.value, nc.value, atoms


def fullatom_max_atoms(seq_host, lengths_host):
    """Smallest Amax for a host (numpy) uint8 sequence batch and int32 lengths."""
    import numpy as np

    s = np.ascontiguousarray(seq_host, dtype=np.uint8)
    ln = np.ascontiguousarray(lengths_host, dtype=np.int32)
    n = load_library().tpl_fullatom_max_atoms(s.ctypes.data_as(ctypes.c_void_p),
                                              ln.ctypes.data_as(ctypes.c_void_p),
                                              s.shape[0], s.shape[1])
    if n < 0:
        raise ValueError("bad residue code or length")
    return n


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------- autograd
class BackboneFn(torch.autograd.Function):
    """Section 3: angles [B,3,Lmax] -> N/CA/C coordinates [B,3*Lmax,3]."""

    @staticmethod
    def forward(ctx, angles, lengths, opts=None):
        B, _, Lmax = angles.shape
        coords = torch.empty((B, 3 * Lmax, 3), dtype=torch.float32, device=angles.device)
        ws = _workspace(tpl_backbone_workspace_size(B, Lmax), angles.device)
        tpl_backbone_forward(angles, lengths, coords, ws, opts)
        # the backward reuses the forward's tile schedule and tile-start frames
        ctx.save_for_backward(angles, lengths, coords, ws)
        ctx.opts = opts
        return coords

    @staticmethod
    def backward(ctx, grad_coords):
        angles, lengths, coords, ws = ctx.saved_tensors
        ga = torch.empty_like(angles)
        tpl_backbone_backward(angles, lengths, coords, grad_coords.contiguous(), ga, ws, ctx.opts)
        return ga, None, None


class BackboneOFn(torch.autograd.Function):
    """Section 3 with each residue's carbonyl O: angles [B,3,Lmax] ->
    (N/CA/C coordinates [B,3*Lmax,3], O [B,Lmax,3])."""

    @staticmethod
    def forward(ctx, angles, lengths, opts=None):
        B, _, Lmax = angles.shape
        coords = torch.empty((B, 3 * Lmax, 3), dtype=torch.float32, device=angles.device)
        o = torch.empty((B, Lmax, 3), dtype=torch.float32, device=angles.device)
        ws = _workspace(tpl_backbone_workspace_size(B, Lmax), angles.device)
        tpl_backbone_forward_o(angles, lengths, coords, o, ws, opts)
        ctx.save_for_backward(angles, lengths, coords, o, ws)
        ctx.opts = opts
        return coords, o

    @staticmethod
    def backward(ctx, grad_coords, grad_o):
        angles, lengths, coords, o, ws = ctx.saved_tensors
        if grad_coords is None:
            grad_coords = torch.zeros_like(coords)
        if grad_o is None:
            grad_o = torch.zeros_like(o)
        ga = torch.empty_like(angles)
        tpl_backbone_backward_o(angles, lengths, coords, o, grad_coords.contiguous(), grad_o.contiguous(), ga,
                                ws, ctx.opts)
        return ga, None, None


class FullAtomFn(torch.autograd.Function):
    """Section 2: angles [B,7,Lmax] + sequence -> heavy-atom coordinates [B,Amax,3]."""

    @staticmethod
    def forward(ctx, angles, seq, lengths, Amax, opts=None):
        B, _, Lmax = angles.shape
        coords = torch.empty((B, Amax, 3), dtype=torch.float32, device=angles.device)
        num_atoms = torch.empty((B,), dtype=torch.int32, device=angles.device)
        ws = _workspace(tpl_fullatom_workspace_size(B, Lmax), angles.device)
        tpl_fullatom_forward(angles, seq, lengths, coords, num_atoms, ws, opts)
        # the backward reads the forward's coordinates (axes and origins of
        # every frame) and its workspace (schedule, each residue's first atom)
        ctx.save_for_backward(angles, seq, lengths, coords, ws)
        ctx.opts = opts
        ctx.mark_non_differentiable(num_atoms)
        return coords, num_atoms

    @staticmethod
    def backward(ctx, grad_coords, _grad_num):
        angles, seq, lengths, coords, ws = ctx.saved_tensors
        ga = torch.empty_like(angles)
        tpl_fullatom_backward(angles, seq, lengths, coords, grad_coords.contiguous(), ga, ws, ctx.opts)
        return ga, None, None, None, None


class LRMSDFn(torch.autograd.Function):
    """Section 4: LRMSD(x = target, y = input) per pair, differentiable in the input."""

    @staticmethod
    def forward(ctx, input, target, num_atoms):
        P, Nmax, _ = input.shape
        out = torch.empty((P,), dtype=torch.float32, device=input.device)
        ws = _workspace(tpl_lrmsd_workspace_size(P, Nmax), input.device)
        tpl_lrmsd_forward(input, target, num_atoms, out, ws)
        ctx.save_for_backward(input, target, num_atoms, ws)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        input, target, num_atoms, ws = ctx.saved_tensors
        g = torch.empty_like(input)
        tpl_lrmsd_backward(grad_out.contiguous().float(), input, target, num_atoms, g, ws)
        return g, None, None


def backbone(angles, lengths, opts=None):
    return BackboneFn.apply(angles, lengths, opts)


def backbone_with_o(angles, lengths, opts=None):
    """Differentiable backbone with carbonyl O: (coords, o)."""
    return BackboneOFn.apply(angles, lengths, opts)


def fullatom(angles, seq, lengths, Amax, opts=None):
    return FullAtomFn.apply(angles, seq, lengths, int(Amax), opts)


def lrmsd(input, target, num_atoms):
    return LRMSDFn.apply(input, target, num_atoms)
