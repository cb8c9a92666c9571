"""Every configuration `bench.py --workload nq-sweep` times, at its full size:
the paper's Nq study (3,538,944 points at Nq = 4, 8, 12, 16; seed 1), in
NUMA_FP64, NUMA_DF64 (N <= 7) and NUMA_MIXED, with five fields and in the
8-field form with three passive tracers, through the same handles and kernels
as the bench.

The oracle's pointwise form evaluates 4000 sampled points (and the first and
last) of each; the bar is the mode's: 1e-12 (FP64), max(1e-12, 16 2^-48
kappa) (double-float, kappa the field's condition number over the whole mesh)
or 1e-5 (mixed) of the field's largest value over the whole mesh.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from bench import NQ_STUDY
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


_WORKLOADS = {}


def study_workload(N):
    if N not in _WORKLOADS:
        _WORKLOADS.clear()   # one study mesh at a time (about 1 GB of host arrays)
        _WORKLOADS[N] = wl.make_workload(N, NQ_STUDY[N], seed=1, tracers=3)
    return _WORKLOADS[N]


@pytest.mark.parametrize("variant", ["fp64", "mixed", "fp64_8fields", "mixed_8fields", "df64",
                                     "df64_8fields"])
@pytest.mark.parametrize("N", sorted(NQ_STUDY))
def test_nq_study_configuration_on_sampled_points(N, variant):
    if variant.startswith("df64") and N > 7:
        pytest.skip("the double-float mode takes N <= 7")
    w8 = study_workload(N)
    w = w8 if variant.endswith("_8fields") else dataclasses.replace(w8, q=w8.q[:5])
    mode = variant.split("_")[0]
    prob = w.problem()
    state = w.q_mixed() if mode == "mixed" else w.q
    with VolumeTerm.from_problem(prob, precision=mode) as vt:
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(state)).cuda()).cpu().numpy()
    out = out.astype(np.float64)
    assert np.all(np.isfinite(out))
    ids = np.concatenate([np.random.default_rng(N).choice(w.M, size=4000, replace=False),
                          [0, w.M - 1]])
    ref = oracle.vol_rhs_points(prob, w.q, ids)
    scale = np.max(np.abs(out), axis=1, keepdims=True)
    tol = 1e-5 if mode == "mixed" else 1e-12
    if mode == "df64":   # the double-float bar: max(1e-12, 16 2^-48 kappa) per field
        tol = np.maximum(1e-12, 16 * 2.0 ** -48 * oracle.condition_numbers(prob, w.q))
    err = np.max(np.abs(out[:, ids] - ref) / scale, axis=1)
    assert np.all(err <= tol), (variant, N, err, tol)
