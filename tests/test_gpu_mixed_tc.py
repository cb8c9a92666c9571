"""GPU tests of the single-evaluation tensor-core sweep (numa_vol_set_sweep with
NUMA_SWEEP_TENSOR_TF32 on a NUMA_MIXED handle of N = 7).

The D sums run as TF32 split products on tcgen05 (heads and tails of the
fluxes and of D, FP32 accumulation in tensor memory).  Bar, as for the
CUDA-core mixed mode: per-field normwise max relative error <= 1e-5 against the
FP64 oracle of the full state; also within 1e-5 of the CUDA-core kernel.  The
persistent grid takes element counts below, at and above one wave of CTAs.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import NumaError, VolumeTerm
from conftest import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def run(prob, q32, sweep="tensor_tf32"):
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        vt.set_sweep(sweep)
        if sweep == "tensor_tf32":
            assert vt.kernel_name == "vol_rhs_mixed_tc_kernel<8>"
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q32)).cuda())
        torch.cuda.synchronize()
        vt.status()
        return out.cpu().numpy().astype(np.float64)


def check(out, ref, tol=TOL, label=""):
    errs = rel_err(out, ref)
    for b, (mx, _) in enumerate(errs):
        assert mx <= tol, f"{label} {wl.FIELD_NAMES[b]}: {mx:.3e}"
    return errs


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (7, 7, 7), (20, 20, 1)])
def test_tensor_sweep_matches_oracle_and_cuda_cores(shape):
    # 1, 6, 343 and 400 elements: below, around and above one wave of the
    # persistent grid (two CTAs per SM)
    w = wl.make_workload(7, shape, seed=70 + shape[0])
    prob = w.problem()
    tc = run(prob, w.q_mixed())
    cc = run(prob, w.q_mixed(), "cuda_cores")
    print(shape, check(tc, oracle.vol_rhs_o2(prob, w.q), label=f"tc {shape}"))
    check(tc, cc, label=f"tc vs cuda cores {shape}")


def test_tensor_sweep_full_size_workload():
    w = wl.bench_full()
    prob = w.problem()
    print("full", check(run(prob, w.q_mixed()), oracle.vol_rhs_o2(prob, w.q), label="full"))


def test_tensor_sweep_zero_perturbation_is_exactly_zero():
    mesh = wl.warped_box(7, (2, 2, 2))
    rho0, rt0 = wl.hydrostatic_reference(mesh.x[2])
    prob = {"N": 7, "Ne": mesh.Ne, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": rho0,
            "rhotheta_ref": rt0, **wl.DRY_AIR.as_dict()}
    q32 = np.zeros((5, mesh.M), dtype=np.float32)
    assert np.all(run(prob, q32) == 0.0)


def test_tensor_sweep_host_path_and_graph_replay_are_bitwise():
    w = wl.make_workload(7, (4, 3, 2), seed=77)
    with VolumeTerm.from_problem(w.problem(), precision="mixed") as vt:
        vt.set_sweep("tensor_tf32")
        q = torch.from_numpy(np.ascontiguousarray(w.q_mixed())).cuda()
        eager = vt.rhs(q)
        torch.cuda.synchronize()
        host = np.empty_like(w.q_mixed())
        vt.rhs_host(w.q_mixed(), host)
        assert np.array_equal(host, eager.cpu().numpy())
        out = torch.empty_like(q)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            vt.rhs(q, out, stream=s)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
        vt.status()


def test_tensor_sweep_is_refused_where_it_does_not_apply():
    w4 = wl.make_workload(4, 1, seed=1)
    w7 = wl.make_workload(7, 1, seed=1)
    with VolumeTerm.from_problem(w4.problem(), precision="mixed") as vt:
        with pytest.raises(NumaError, match="UNSUPPORTED"):
            vt.set_sweep("tensor_tf32")
        assert vt.kernel_name == "vol_rhs_mixed_kernel<5>"
    with VolumeTerm.from_problem(w7.problem(), precision="fp64") as vt:
        with pytest.raises(NumaError, match="UNSUPPORTED"):
            vt.set_sweep("tensor_tf32")
    with VolumeTerm.from_problem(w7.problem(), precision="mixed") as vt:
        vt.set_sweep("tensor_tf32")
        vt.set_sweep("cuda_cores")
        assert vt.kernel_name == "vol_rhs_mixed_kernel<8>"
