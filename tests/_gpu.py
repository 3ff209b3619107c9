"""Shared helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    import paper_1004_3354_gb300 as ed
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    return ed


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(x64: np.ndarray, prec, ed, torch):
    """Host float64 vector -> device vector in the sector format (via the library's converter)."""
    d = torch.from_numpy(np.ascontiguousarray(x64)).cuda()
    if prec in ("fp64", ed.ED_PREC_FP64):
        return d
    p = ed.PREC_NAMES.get(prec, prec)
    out = torch.empty(len(x64) * ed.elems_per_value(p), dtype=torch.float32, device="cuda")
    ed.ed_convert(d, ed.ED_PREC_FP64, out, p, len(x64))
    return out


def to_host(v, prec, n, ed, torch):
    p = ed.PREC_NAMES.get(prec, prec)
    if p == ed.ED_PREC_FP64:
        return v.cpu().numpy()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ed.ed_convert(v, p, out, ed.ED_PREC_FP64, n)
    return out.cpu().numpy()


def empty_vec(n, prec, ed, torch, count=1):
    p = ed.PREC_NAMES.get(prec, prec)
    return torch.empty(n * count * ed.elems_per_value(p), dtype=ed.torch_dtype(p), device="cuda")


def rel_err(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
