"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: the FP64 path must match the oracle to a per-field normwise max
relative error  max|x - x*| / max|x*| <= 1e-12.  The oracle and the kernels
round differently: summation order, FMA contraction, CUDA's pow against the
C library's pow.  The bound absorbs that and nothing larger.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import _lib, build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm, NumaError
from conftest import eos_banded_theta_ratio, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_FP64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _lib.load()


def gpu_rhs(prob, q, stream=None):
    with VolumeTerm.from_problem(prob) as vt:
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        out = vt.rhs(qd, stream=stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def assert_parity(out, ref, tol=TOL_FP64, label=""):
    errs = rel_err(out, ref)
    for b, (mx, rms) in enumerate(errs):
        assert mx <= tol, f"{label} field {wl.FIELD_NAMES[b]}: max rel err {mx:.3e} > {tol}"
    return errs


def test_parity_small_workload():
    # N = 4 (Nq = 5), 8^3 = 512 elements on the warped 10 km box, seed 0.
    w = wl.parity_small()
    prob = w.problem()
    out = gpu_rhs(prob, w.q)
    ref = oracle.vol_rhs_o2(prob, w.q)
    errs = assert_parity(out, ref, label="N=4 512 elements")
    print("max/rms per field", errs)


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 1), (2, 2, 2), (5, 3, 1)])
def test_parity_every_order_and_odd_sizes(N, shape):
    w = wl.make_workload(N, shape, seed=100 + N)
    prob = w.problem()
    assert_parity(gpu_rhs(prob, w.q), oracle.vol_rhs_o2(prob, w.q), label=f"N={N} {shape}")


@pytest.mark.parametrize("N", [3, 7])
def test_parity_across_the_eos_branches(N):
    # Theta'/Theta_ref in each range of the kernel's pressure perturbation,
    # with warps wholly inside one range (9-term series, 15-term series,
    # expm1/log1p) and warps that mix them (the widest form for all lanes).
    w = wl.make_workload(N, (3, 2, 1), seed=40 + N)
    q = w.q.copy()
    q[4] = w.rhotheta_ref * (1.0 + eos_banded_theta_ratio(w.M, seed=N))
    prob = w.problem()
    assert_parity(gpu_rhs(prob, q), oracle.vol_rhs_o2(prob, q), label=f"N={N} EOS branches")


def test_parity_full_size_workload():
    # N = 7 (Nq = 8), 32^3 = 32768 elements (16.8M points), seed 1: the timed
    # workload, against the complete oracle and, on a sample of points, against
    # the oracle's pointwise form.
    w = wl.bench_full()
    prob = w.problem()
    out = gpu_rhs(prob, w.q)
    ref = oracle.vol_rhs_o2(prob, w.q)
    errs = assert_parity(out, ref, label="full size")
    print("max/rms per field", errs)
    ids = np.random.default_rng(5).choice(w.M, size=4000, replace=False)
    ids = np.concatenate([ids, [0, w.M - 1]])
    pts = oracle.vol_rhs_points(prob, w.q, ids)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out[:, ids] - pts) / scale) <= TOL_FP64


def test_zero_perturbation_is_exactly_zero_on_gpu():
    for N in (3, 7):
        mesh = wl.warped_box(N, (3, 2, 2))
        rho0, rt0 = wl.hydrostatic_reference(mesh.x[2])
        q = np.zeros((5, mesh.M))
        q[0], q[4] = rho0, rt0
        prob = {"N": N, "Ne": mesh.Ne, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": rho0,
                "rhotheta_ref": rt0, **wl.DRY_AIR.as_dict()}
        assert np.all(gpu_rhs(prob, q) == 0.0)


def test_manufactured_closed_form_on_gpu():
    # Linear velocity on a non-orthogonal affine mesh: -div(u q_b) in closed form.
    import test_oracle_pins as pins
    for N in (2, 5, 7):
        prob, q, want = pins._manufactured_linear_velocity(N)
        assert_parity(gpu_rhs(prob, q), want, label=f"manufactured N={N}")
        prob, q, want = pins._manufactured_linear_pressure(
            N, wl.Constants(p0=1.0, R=1.0, cp=3.5, grav=2.5))
        out = gpu_rhs(prob, q)
        assert np.all(out[0] == 0) and np.all(out[4] == 0)
        for b in (1, 2, 3):
            assert np.max(np.abs(out[b] - want[b])) <= 1e-12 * np.max(np.abs(want[b]))


def test_paper_units_by_hand_on_gpu():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_units_n1_by_hand.json")))
    mesh = wl.affine_box(1, (1, 1, 1), L=2.0, B=np.eye(3))
    q = np.zeros((5, 8))
    want = np.zeros((5, 8))
    names = ("rho", "U1", "U2", "U3", "Theta")
    for node in range(8):
        env = {"i": node % 2, "j": (node // 2) % 2, "k": node // 4}
        q[:, node] = [eval(gold["state"][f], env) for f in names]
        want[:, node] = [eval(gold["rhs"][f], env) for f in names]
    prob = {"N": 1, "Ne": 1, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": np.zeros(8),
            "rhotheta_ref": np.zeros(8), **wl.PAPER_UNITS.as_dict()}
    assert np.max(np.abs(gpu_rhs(prob, q) - want)) < 1e-15


def test_side_stream_and_determinism():
    w = wl.make_workload(5, (4, 3, 2), seed=9)
    prob = w.problem()
    s = torch.cuda.Stream()
    with VolumeTerm.from_problem(prob) as vt:
        qd = torch.from_numpy(w.q).cuda()
        torch.cuda.synchronize()
        a = vt.rhs(qd, stream=s)
        b = vt.rhs(qd, stream=s)
        s.synchronize()
        assert torch.equal(a, b)
        # host entry point: same kernel, copies included
        h = vt.rhs_host(w.q)
        assert np.array_equal(h, a.cpu().numpy())
        pinned = torch.from_numpy(w.q).pin_memory()
        h2 = vt.rhs_host(pinned)
        assert np.array_equal(h2.numpy(), h)


def test_empty_mesh_is_a_no_op():
    g = [np.zeros(0)] * 9
    with VolumeTerm(3, 0, g, np.zeros(0), np.zeros(0), np.zeros(0), **wl.DRY_AIR.as_dict()) as vt:
        q = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
        out = vt.rhs(q)
        assert out.numel() == 0


def test_invalid_pointers_are_rejected_and_context_survives():
    import ctypes as C
    w = wl.make_workload(3, 2, seed=4)
    prob = w.problem()
    lib = _lib.load()
    with VolumeTerm.from_problem(prob) as vt:
        q = torch.from_numpy(w.q).cuda()
        big = torch.zeros(5 * w.M + 2, dtype=torch.float64, device="cuda")
        out = torch.empty_like(q)
        # misaligned (8-byte offset)
        rc = lib.numa_vol_rhs(vt.handle, C.c_void_p(big.data_ptr() + 8), C.c_void_p(out.data_ptr()), None)
        assert rc == _lib.NUMA_EINVAL
        # overlapping q and rhs
        rc = lib.numa_vol_rhs(vt.handle, C.c_void_p(big.data_ptr()), C.c_void_p(big.data_ptr() + 16), None)
        assert rc == _lib.NUMA_EINVAL
        # host memory where device memory is required
        host = np.zeros(5 * w.M)
        rc = lib.numa_vol_rhs(vt.handle, C.c_void_p(host.ctypes.data), C.c_void_p(out.data_ptr()), None)
        assert rc == _lib.NUMA_EINVAL
        assert b"device pointers" in lib.numa_vol_last_error()
        # the context is intact: a valid call still matches the oracle
        res = vt.rhs(q)
        torch.cuda.synchronize()
        assert_parity(res.cpu().numpy(), oracle.vol_rhs_o2(prob, w.q))
    with pytest.raises(NumaError):   # the double-float mode takes N <= 7
        VolumeTerm(8, 1, [np.ones(729)] * 9, np.ones(729), np.ones(729), np.ones(729),
                   p0=1e5, R=287.0, cp=1004.0, grav=9.8, precision="df64").close()


def test_handles_of_different_orders_interleave():
    ws = [wl.make_workload(N, 2, seed=20 + N) for N in (2, 7, 4)]
    vts = [VolumeTerm.from_problem(w.problem()) for w in ws]
    try:
        outs = [vt.rhs(torch.from_numpy(w.q).cuda()) for vt, w in zip(vts, ws)]
        torch.cuda.synchronize()
        for w, o in zip(ws, outs):
            assert_parity(o.cpu().numpy(), oracle.vol_rhs_o2(w.problem(), w.q))
    finally:
        for vt in vts:
            vt.close()
