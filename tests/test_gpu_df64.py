"""GPU tests of the double-float mode (NUMA_DF64, N = 1..7) against the oracle,
the native FP64 kernel and its own fallbacks.

The double-float kernel carries about 48 significant bits, so its error against
the FP64 oracle scales with the condition number kappa_b of each field's
sweeps: max|Jinv sum |D||F|| / max|rhs_b|, from the oracle's running error
bound.  The bar per field is max(1e-12, 16 * 2^-48 * kappa_b).  On the
benchmark workloads (per-point random velocities, kappa of order 10-100) that
is the 1e-12 of the FP64 path.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm
from conftest import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def df_tol(prob, q, ref):
    kappa = oracle.condition_numbers(prob, q, ref)
    return np.maximum(1e-12, 16 * 2.0 ** -48 * kappa), kappa


def run(prob, q, precision="df64"):
    with VolumeTerm.from_problem(prob, precision=precision) as vt:
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q)).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def check(out, ref, tol=TOL, label=""):
    errs = rel_err(out, ref)
    tol = np.broadcast_to(tol, (5,))
    for b, (mx, _) in enumerate(errs):
        assert mx <= tol[b], f"{label} {wl.FIELD_NAMES[b]}: {mx:.3e} > {tol[b]:.3e}"
    return errs


def kernel_of(prob, precision="df64"):
    with VolumeTerm.from_problem(prob, precision=precision) as vt:
        return vt.kernel_name


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (5, 4, 3)])
def test_df_matches_oracle_and_native(shape):
    w = wl.make_workload(7, shape, seed=31)
    prob = w.problem()
    ref = oracle.vol_rhs_o2(prob, w.q)
    assert kernel_of(prob) == "vol_rhs_df64_kernel<8>"
    df = run(prob, w.q, "df64")
    nat = run(prob, w.q, "fp64")
    tol, kappa = df_tol(prob, w.q, ref)
    assert np.all(tol == 1e-12), kappa       # well-conditioned: the FP64 bar applies
    e1 = check(df, ref, label="df vs oracle")
    check(nat, ref, label="native vs oracle")
    print("kappa", kappa, "df vs oracle", e1, "df vs native", rel_err(df, nat))


def test_df_full_size_workload():
    # The timed workload (N = 7, 32^3 elements, seed 1) at 1e-12.
    w = wl.bench_full()
    prob = w.problem()
    assert kernel_of(prob) == "vol_rhs_df64_kernel<8>"
    ref = oracle.vol_rhs_o2(prob, w.q)
    print("df full size", check(run(prob, w.q), ref, label="df full size"))


def test_df_ill_conditioned_manufactured_case():
    # Smooth linear velocity with a large mean on an affine mesh: kappa ~ 1e2-1e3.
    # The closed form holds; the error follows the conditioning-scaled bound.
    import test_oracle_pins as pins
    prob, q, want = pins._manufactured_linear_velocity(7)
    ref = oracle.vol_rhs_o2(prob, q)
    tol, kappa = df_tol(prob, q, ref)
    errs = check(run(prob, q), ref, tol=tol, label="df manufactured")
    print("kappa", kappa, "errors", errs)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_df_every_order_matches_oracle(N):
    # Every order with ragged element counts, against the oracle, at the
    # conditioning-scaled bar (the FP64 bar where the sweeps are well conditioned).
    for shape, seed in (((1, 1, 1), 40 + N), ((3, 2, 1), 50 + N)):
        w = wl.make_workload(N, shape, seed=seed)
        prob = w.problem()
        assert kernel_of(prob) == f"vol_rhs_df64_kernel<{N + 1}>"
        ref = oracle.vol_rhs_o2(prob, w.q)
        tol, kappa = df_tol(prob, w.q, ref)
        errs = check(run(prob, w.q), ref, tol=tol, label=f"df N={N} {shape}")
        print(N, shape, "kappa", kappa, "errors", errs)


def test_df_order_6_point_fallback_and_zero_state():
    # odd Nq: the centre row and column of the even-odd sweep; large Theta
    # perturbations take p' from pow; the unperturbed state gives exact zeros
    w = wl.make_workload(6, (2, 1, 1), seed=61)
    q = w.q.copy()
    q[4, 50:90] *= 1.05
    prob = w.problem()
    tol, _ = df_tol(prob, q, oracle.vol_rhs_o2(prob, q))
    check(run(prob, q), oracle.vol_rhs_o2(prob, q), tol=tol, label="df N=6 pow fallback")
    q0 = np.zeros_like(w.q)
    q0[0], q0[4] = w.rho_ref, w.rhotheta_ref
    assert np.all(run(prob, q0) == 0.0)


def test_df64_refuses_orders_above_7():
    from paper_1604_08501_gb300.numa_vol import NumaError
    w = wl.make_workload(8, 1, seed=1)
    with pytest.raises(NumaError, match="UNSUPPORTED"):
        VolumeTerm.from_problem(w.problem(), precision="df64")


def test_df_element_fallback_for_out_of_range_state():
    # One element holds a momentum value of 1e15 (outside [2^-40, 2^41)): that
    # element is evaluated in native FP64, the others in double-float.
    w = wl.make_workload(7, (3, 1, 1), seed=5)
    q = w.q.copy()
    q[2, 512 + 17] = 1.0e15
    prob = w.problem()
    check(run(prob, q), oracle.vol_rhs_o2(prob, q), label="element fallback")


def test_df_point_fallback_for_large_theta_perturbation():
    # |Theta - Theta_ref| / Theta_ref > 1/64 at some points: p' from the FP64 pow.
    w = wl.make_workload(7, (2, 2, 1), seed=6)
    q = w.q.copy()
    q[4, 100:140] *= 1.05
    q[4, 700:720] *= 0.97
    prob = w.problem()
    check(run(prob, q), oracle.vol_rhs_o2(prob, q), label="pow fallback")


def test_df_out_of_range_geometry_uses_native_kernel():
    w = wl.make_workload(7, (2, 1, 1), seed=8)
    prob = w.problem()
    # metric terms of ~2e13 > 2^41 cannot be split into float pairs
    prob["g"] = prob["g"] * 1e9
    prob["Jinv"] = prob["Jinv"] * 1e-18
    assert kernel_of(prob) == "vol_rhs_fp64_kernel<8>"
    check(run(prob, w.q), oracle.vol_rhs_o2(prob, w.q), label="geometry fallback")


def test_df_zero_perturbation_and_signed_values():
    mesh = wl.warped_box(7, (2, 2, 2))
    rho0, rt0 = wl.hydrostatic_reference(mesh.x[2])
    q = np.zeros((5, mesh.M))
    q[0], q[4] = rho0, rt0
    prob = {"N": 7, "Ne": mesh.Ne, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": rho0,
            "rhotheta_ref": rt0, **wl.DRY_AIR.as_dict()}
    assert np.all(run(prob, q) == 0.0)
    # exact zeros in the momentum and negative momenta
    w = wl.make_workload(7, (2, 1, 1), seed=12)
    q = w.q.copy()
    q[1, ::3] = 0.0
    q[3] = -np.abs(q[3])
    check(run(w.problem(), q), oracle.vol_rhs_o2(w.problem(), q), label="signs/zeros")
