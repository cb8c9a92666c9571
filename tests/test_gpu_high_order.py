"""GPU parity of the native FP64 volume term at orders N = 8..15 (Nq up to 16,
the range of the paper's Nq study, Sec. 4, Table 2), through the C ABI.

Same bar as the low orders: per-field normwise max relative error <= 1e-12
against the oracle's O2 form (and, at the study's sizes, against its pointwise
form on sampled points).
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import _lib, build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, Engine, NumaError, VolumeTerm
from conftest import eos_banded_theta_ratio, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12
# The paper's Nq study: 3,538,944 points at every order.
# Mixed precision at N = 8..15: the 1e-5 bar of the mixed mode.
STUDY = {3: (48, 48, 24), 7: (24, 24, 12), 11: (16, 16, 8), 15: (12, 12, 6)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def gpu_rhs(prob, q):
    with VolumeTerm.from_problem(prob) as vt:
        assert vt.kernel_name == f"vol_rhs_high_kernel<{prob['N'] + 1}, double>"
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q)).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def assert_parity(out, ref, label):
    for b, (mx, _) in enumerate(rel_err(out, ref)):
        assert mx <= TOL, f"{label} {wl.FIELD_NAMES[b]}: {mx:.3e}"


@pytest.mark.parametrize("N", range(8, 16))
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 1), (2, 2, 1)])
def test_parity_every_high_order(N, shape):
    w = wl.make_workload(N, shape, seed=200 + N)
    prob = w.problem()
    assert_parity(gpu_rhs(prob, w.q), oracle.vol_rhs_o2(prob, w.q), f"N={N} {shape}")


@pytest.mark.parametrize("N", [8, 11, 15])
def test_high_order_zero_perturbation_is_exactly_zero(N):
    w = wl.make_workload(N, (2, 1, 1), seed=5)
    q = np.zeros_like(w.q)
    q[0], q[4] = w.rho_ref, w.rhotheta_ref
    assert not np.any(gpu_rhs(w.problem(), q))


@pytest.mark.parametrize("N", [11, 15])
def test_high_order_across_the_eos_forms(N):
    w = wl.make_workload(N, (2, 1, 1), seed=300 + N)
    q = w.q.copy()
    q[4] = w.rhotheta_ref * (1.0 + eos_banded_theta_ratio(w.M, seed=N))
    prob = w.problem()
    assert_parity(gpu_rhs(prob, q), oracle.vol_rhs_o2(prob, q), f"N={N} EOS forms")


@pytest.mark.parametrize("N", [11, 15])
def test_study_size_on_sampled_points(N):
    # The paper's Nq study at 3,538,944 points: sampled points against the
    # oracle's pointwise form, scaled by the field's largest sampled value.
    w = wl.make_workload(N, STUDY[N], seed=1)
    prob = w.problem()
    out = gpu_rhs(prob, w.q)
    ids = np.concatenate([np.random.default_rng(N).choice(w.M, size=4000, replace=False),
                          [0, w.M - 1]])
    pts = oracle.vol_rhs_points(prob, w.q, ids)
    scale = np.max(np.abs(out), axis=1, keepdims=True)
    assert np.max(np.abs(out[:, ids] - pts) / scale) <= TOL
    assert np.all(np.isfinite(out))


def test_host_entry_point_and_rejections_at_high_order():
    w = wl.make_workload(9, (3, 1, 1), seed=9)
    prob = w.problem()
    with VolumeTerm.from_problem(prob) as vt:
        dev = vt.rhs(torch.from_numpy(w.q).cuda()).cpu().numpy()
        assert np.array_equal(vt.rhs_host(w.q), dev)
        q = torch.from_numpy(w.q).cuda()
        with Batch("fp64") as b:
            with pytest.raises(NumaError, match="EUNSUPPORTED"):
                b.add(vt, q)
        with Engine("fp64", budget_bytes=1 << 26) as eng:
            with pytest.raises(NumaError, match="EUNSUPPORTED"):
                eng.submit(vt, w.q, np.empty_like(w.q), 1, 0.01)
    with pytest.raises(NumaError, match="EUNSUPPORTED"):
        VolumeTerm.from_problem(prob, precision="df64")


@pytest.mark.parametrize("T", [0, 1, 3])
@pytest.mark.parametrize("N", range(8, 16))
def test_mixed_precision_high_orders(N, T):
    # The FP32 instantiation of the high-order kernel: perturbation state,
    # FP32 sweeps, p' from Theta'; every field within 1e-5 of the FP64 oracle.
    # Every order with 5, 6 and 8 fields: one pass, and the forms whose later
    # fields wait in tensor memory (4 + 1, 4 + 2, 4 + 4, 5 + 1, 5 + 3, 6 + 2,
    # 7 + 1 fields).
    w = wl.make_workload(N, (2, 1, 1), seed=500 + N, tracers=T)
    prob = w.problem()
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        assert vt.kernel_name == f"vol_rhs_high_kernel<{N + 1}, float>"
        out = vt.rhs(torch.from_numpy(w.q_mixed()).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.vol_rhs_o2(prob, w.q)
    for f in range(5 + T):
        mx = np.max(np.abs(out[f] - ref[f])) / np.max(np.abs(ref[f]))
        assert mx <= 1e-5, (N, T, wl.FIELD_NAMES[f], mx)


def test_mixed_high_order_across_the_eos_forms():
    w = wl.make_workload(11, (2, 1, 1), seed=611)
    q = w.q.copy()
    q[4] = w.rhotheta_ref * (1.0 + eos_banded_theta_ratio(w.M, seed=11))
    prob = w.problem()
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        q32 = wl.perturbation_state(q, w.rho_ref, w.rhotheta_ref)
        out = vt.rhs(torch.from_numpy(q32).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.vol_rhs_o2(prob, q)
    for f in range(5):
        assert np.max(np.abs(out[f] - ref[f])) <= 1e-5 * np.max(np.abs(ref[f])), f


@pytest.mark.parametrize("N,shape,T", [(11, (5, 2, 2), 3), (11, (20, 16, 16), 0),
                                       (15, (16, 16, 10), 0)])
def test_mixed_high_order_host_path_is_bitwise(N, shape, T):
    # The host entry point launches the mesh in 16 chunks (first element > 0,
    # each launch with its own end), which bounds the kernel's L2 prefetch of
    # the element one wave of resident CTAs later (304 CTAs at Nq = 12, 152 at
    # Nq = 16); its result equals the device entry point's bit for bit.  The
    # two large meshes make every chunk longer than a wave (320 and 160
    # elements), so the prefetch runs inside each chunk; the small one has
    # tracers and chunks of one or two elements.
    w = wl.make_workload(N, shape, seed=700 + N, tracers=T)
    q32 = np.ascontiguousarray(w.q_mixed())
    with VolumeTerm.from_problem(w.problem(), precision="mixed") as vt:
        dev = vt.rhs(torch.from_numpy(q32).cuda()).cpu().numpy()
        host = np.empty_like(q32)
        vt.rhs_host(q32, host)
    assert np.array_equal(host, dev)
    assert np.all(np.isfinite(dev))
