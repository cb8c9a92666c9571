"""GPU parity of the 8-field form (passive tracers Q1..Q3 after Theta, the
paper's benchmark form, Sec. 2) in NUMA_FP64 and NUMA_DF64, through the C ABI.

Bar: per-field normwise max relative error <= 1e-12 against the oracle's O2
form, as for the five base fields (double-float: max(1e-12, 16 2^-48 kappa)
per field, kappa the field's condition number from the oracle's error bound).  Properties that hold at any size: tracers
leave the five base fields bit for bit as without them, and a tracer equal to
Theta has Theta's rhs bit for bit (same flux, same arithmetic).
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def gpu_rhs(prob, q):
    with VolumeTerm.from_problem(prob) as vt:
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q)).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("N,T", [(1, 3), (3, 1), (4, 2), (7, 3), (9, 2), (11, 3)])
def test_tracer_parity(N, T):
    w = wl.make_workload(N, (3, 2, 1), seed=400 + N, tracers=T)
    prob = w.problem()
    out = gpu_rhs(prob, w.q)
    assert out.shape == (5 + T, w.M)
    ref = oracle.vol_rhs_o2(prob, w.q)
    for f in range(5 + T):
        mx = np.max(np.abs(out[f] - ref[f])) / np.max(np.abs(ref[f]))
        assert mx <= TOL, (N, T, wl.FIELD_NAMES[f], mx)


@pytest.mark.parametrize("N", [7, 11])
def test_tracers_are_passive_and_theta_copies_match(N):
    w8 = wl.make_workload(N, (2, 2, 1), seed=410 + N, tracers=3)
    w5 = wl.make_workload(N, (2, 2, 1), seed=410 + N)
    q = w8.q.copy()
    q[6] = q[4]                                   # Q2 = Theta
    r8 = gpu_rhs(w8.problem(), q)
    r5 = gpu_rhs(w5.problem(), w5.q)
    assert np.array_equal(r8[:5], r5)
    assert np.array_equal(r8[6], r8[4])


def test_tracer_host_path_full_paper_form():
    # The paper's benchmark element: Nq = 8 with 8 fields, on the host path.
    w = wl.make_workload(7, (4, 3, 2), seed=420, tracers=3)
    prob = w.problem()
    with VolumeTerm.from_problem(prob) as vt:
        dev = vt.rhs(torch.from_numpy(w.q).cuda()).cpu().numpy()
        assert np.array_equal(vt.rhs_host(w.q), dev)
    ref = oracle.vol_rhs_o2(prob, w.q)
    for f in range(8):
        assert np.max(np.abs(dev[f] - ref[f])) <= TOL * np.max(np.abs(ref[f])), f


@pytest.mark.parametrize("N,T", [(2, 3), (4, 1), (7, 3)])
def test_mixed_precision_tracers(N, T):
    # FP32 8-field form (the paper's benchmark precision and field count):
    # every field within the mixed mode's 1e-5 bar of the FP64 oracle.
    w = wl.make_workload(N, (3, 2, 1), seed=440 + N, tracers=T)
    prob = w.problem()
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        if N == 7:
            assert vt.kernel_name == "vol_rhs_mixed_kernel<8>"
        out = vt.rhs(torch.from_numpy(w.q_mixed()).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.vol_rhs_o2(prob, w.q)
    for f in range(5 + T):
        mx = np.max(np.abs(out[f] - ref[f])) / np.max(np.abs(ref[f]))
        assert mx <= 1e-5, (N, T, wl.FIELD_NAMES[f], mx)


def df_rhs(prob, q):
    with VolumeTerm.from_problem(prob, precision="df64") as vt:
        assert vt.kernel_name == f"vol_rhs_df64_kernel<{prob['N'] + 1}>"
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q)).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def df_check(prob, q, out, label):
    ref = oracle.vol_rhs_o2(prob, q)
    kappa = oracle.condition_numbers(prob, q, ref)
    tol = np.maximum(TOL, 16 * 2.0 ** -48 * kappa)
    for f in range(ref.shape[0]):
        mx = np.max(np.abs(out[f] - ref[f])) / np.max(np.abs(ref[f]))
        assert mx <= tol[f], (label, wl.FIELD_NAMES[f], mx, tol[f])


@pytest.mark.parametrize("T", [1, 3])
@pytest.mark.parametrize("N", range(1, 8))
def test_df64_tracer_parity_every_order(N, T):
    # Double-float 8-field form at every order: the oracle's bar per field; the
    # five base fields bit for bit as without tracers; a tracer equal to
    # Theta has Theta's rhs bit for bit.
    w = wl.make_workload(N, (3, 2, 1), seed=440 + N, tracers=T)
    w5 = wl.make_workload(N, (3, 2, 1), seed=440 + N)
    prob = w.problem()
    out = df_rhs(prob, w.q)
    assert out.shape == (5 + T, w.M)
    df_check(prob, w.q, out, f"df64 N={N} T={T}")
    assert np.array_equal(out[:5], df_rhs(w5.problem(), w5.q))
    q = w.q.copy()
    q[5] = q[4]
    assert np.array_equal(df_rhs(prob, q)[5], out[4])


def test_df64_tracers_through_the_fp64_fallback():
    # A tracer value beyond the double-float range (>= 2^41) sends its element
    # to the native FP64 evaluation, tracers included; the other elements stay
    # in double-float.  Both within the bar of the oracle.
    w = wl.make_workload(7, (3, 1, 1), seed=450, tracers=3)
    q = w.q.copy()
    q[6, 100] = 2.0 ** 45
    prob = w.problem()
    df_check(prob, q, df_rhs(prob, q), "df64 fallback")


def test_df64_tracer_host_path_is_bitwise():
    w = wl.make_workload(5, (4, 3, 2), seed=451, tracers=2)
    with VolumeTerm.from_problem(w.problem(), precision="df64") as vt:
        dev = vt.rhs(torch.from_numpy(w.q).cuda()).cpu().numpy()
        assert np.array_equal(vt.rhs_host(w.q), dev)
