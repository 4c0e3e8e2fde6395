"""Helpers for the GPU parity tests: build/load the library and move arrays."""
import numpy as np
import pytest
import torch

import paper_1812_01108_gb300 as tpl
from paper_1812_01108_gb300 import build as tpl_build

_built = False


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    global _built
    if not _built:
        tpl_build.build()  # fails loudly (no CPU fallback) if nvcc is missing
        tpl.load_library()
        _built = True
    return torch.device("cuda", 0)


def dev(a, device, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    """Per chain ||a - b|| / ||b|| (rows of a batch), max over chains with nonzero b."""
    a = np.asarray(a, np.float64).reshape(a.shape[0], -1)
    b = np.asarray(b, np.float64).reshape(b.shape[0], -1)
    nb = np.linalg.norm(b, axis=1)
    m = nb > 0
    return float((np.linalg.norm(a - b, axis=1)[m] / nb[m]).max()) if m.any() else 0.0
