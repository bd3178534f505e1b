"""Shared helpers of the test suite (no method arithmetic)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F (real or complex; ||b|| = 0 read as 1)."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a = np.asarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.asarray(b, dtype=np.complex128 if cplx else np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def header_symbols():
    """Function names declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names += re.findall(r"^\s*(?:int|const char\*|void)\s+(h2_\w+)\s*\(", txt, flags=re.M)
    return names


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch
