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

    Fields whose reference is identically zero report the absolute max error.
    2-D arrays are (fields, points), any number of fields; flat arrays hold
    five fields."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    x = x if x.ndim == 2 else x.reshape(5, -1)
    ref = ref if ref.ndim == 2 else ref.reshape(5, -1)
    assert x.shape == ref.shape, (x.shape, ref.shape)
    out = []
    for b in range(x.shape[0]):
        d = x[b] - ref[b]
        scale = np.max(np.abs(ref[b])) if ref[b].size else 0.0
        mx = np.max(np.abs(d)) if d.size else 0.0
        if scale == 0.0:
            out.append((mx, mx))
            continue
        out.append((mx / scale, np.linalg.norm(d) / np.linalg.norm(ref[b])))
    return out


def eos_banded_theta_ratio(M: int, seed: int):
    """Theta'/Theta_ref per point for tests of the pressure-perturbation forms,
    by blocks of 32 consecutive points (one warp when a CTA covers whole
    elements of 32-point multiples): blocks entirely within |x| <= 1/64, within
    1/64 < |x| <= 1/8, within 1/8 < |x| <= 0.6, and blocks that mix all three."""
    import numpy as np
    rng = np.random.default_rng(seed)
    lo = [(0.0, 1 / 64), (1 / 64, 1 / 8), (1 / 8, 0.6)]
    x = np.empty(M)
    for b0 in range(0, M, 32):
        n = min(32, M - b0)
        band = (b0 // 32) % 4
        bands = [band] * n if band < 3 else list(rng.integers(0, 3, size=n))
        mag = np.array([rng.uniform(*lo[k]) for k in bands])
        x[b0:b0 + n] = mag * rng.choice([-1.0, 1.0], size=n)
    return x