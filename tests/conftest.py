import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def rel_err(x, ref):
    """Per-field normwise errors: (max|x - ref| / max|ref|, ||x - ref||_2 / ||ref||_2).

    Fields whose reference is identically zero report the absolute max error."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64).reshape(5, -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(5, -1)
    out = []
    for b in range(5):
        d = x[b] - ref[b]
        scale = np.max(np.abs(ref[b])) if ref[b].size else 0.0
        mx = np.max(np.abs(d)) if d.size else 0.0
        if scale == 0.0:
            out.append((mx, mx))
            continue
        out.append((mx / scale, np.linalg.norm(d) / np.linalg.norm(ref[b])))
    return out
