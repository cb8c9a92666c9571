"""GPU tests of the mixed-precision mode (NUMA_MIXED): FP32 perturbation state,
FP32 geometry and arithmetic, against the FP64 oracle of the full state.

Target: per-field normwise max relative error <= 1e-5.  The FP32 error is
about 1e-7 times the sweep condition number, which is small (~3) on these
workloads; the test prints max and RMS errors per field.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import NumaError, VolumeTerm
from conftest import eos_banded_theta_ratio, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_MIXED = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def run_mixed(prob, q32):
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        assert vt.kernel_name.startswith("vol_rhs_mixed")
        out = vt.rhs(torch.from_numpy(np.ascontiguousarray(q32)).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)


def check(out, ref, label=""):
    errs = rel_err(out, ref)
    for b, (mx, _) in enumerate(errs):
        assert mx <= TOL_MIXED, f"{label} {wl.FIELD_NAMES[b]}: {mx:.3e}"
    return errs


@pytest.mark.parametrize("N", range(1, 8))
def test_mixed_every_order(N):
    w = wl.make_workload(N, (3, 2, 1), seed=40 + N)
    prob = w.problem()
    errs = check(run_mixed(prob, w.q_mixed()), oracle.vol_rhs_o2(prob, w.q), f"N={N}")
    print(N, errs)


def test_mixed_small_workload():
    w = wl.parity_small()
    prob = w.problem()
    print("small", check(run_mixed(prob, w.q_mixed()), oracle.vol_rhs_o2(prob, w.q), "small"))


def test_mixed_full_size_workload():
    w = wl.bench_full()
    prob = w.problem()
    errs = check(run_mixed(prob, w.q_mixed()), oracle.vol_rhs_o2(prob, w.q), "full size")
    print("mixed full size max/rms per field", errs)


def test_mixed_zero_perturbation_is_exactly_zero():
    mesh = wl.warped_box(7, (2, 2, 1))
    rho0, rt0 = wl.hydrostatic_reference(mesh.x[2])
    prob = {"N": 7, "Ne": mesh.Ne, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": rho0,
            "rhotheta_ref": rt0, **wl.DRY_AIR.as_dict()}
    assert np.all(run_mixed(prob, np.zeros((5, mesh.M), np.float32)) == 0.0)


def test_mixed_paper_units_full_pressure():
    # Theta_ref = 0: the perturbation is the full Theta and p' = p(Theta).
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_units_n1_by_hand.json")))
    mesh = wl.affine_box(1, (1, 1, 1), L=2.0, B=np.eye(3))
    q = np.zeros((5, 8), np.float32)
    want = np.zeros((5, 8))
    names = ("rho", "U1", "U2", "U3", "Theta")
    for node in range(8):
        env = {"i": node % 2, "j": (node // 2) % 2, "k": node // 4}
        q[:, node] = [eval(gold["state"][f], env) for f in names]
        want[:, node] = [eval(gold["rhs"][f], env) for f in names]
    prob = {"N": 1, "Ne": 1, "g": mesh.g, "Jinv": mesh.Jinv, "rho_ref": np.zeros(8),
            "rhotheta_ref": np.zeros(8), **wl.PAPER_UNITS.as_dict()}
    assert np.max(np.abs(run_mixed(prob, q) - want)) < 1e-6


def test_mixed_host_entry_point_and_large_perturbation():
    w = wl.make_workload(5, (2, 2, 2), seed=77)
    q = w.q.copy()
    q[4, :200] *= 1.04          # |Theta'/Theta_ref| > 1/64: expm1/log1p branch
    prob = w.problem()
    q32 = wl.perturbation_state(q, w.rho_ref, w.rhotheta_ref)
    dev = run_mixed(prob, q32)
    check(dev, oracle.vol_rhs_o2(prob, q), "large perturbation")
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        host = vt.rhs_host(q32)
        vt.status()                       # no bounded wait ran out
    assert np.array_equal(host.astype(np.float64), dev)


def test_mixed_n7_ranges_prefetch_and_status():
    # N = 7 runs one CTA per element with an L2 prefetch of the element one
    # wave of resident CTAs ahead: element counts below, at and above that
    # wave (a small multiple of the SM count) and the chunked host path agree.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for shape in [(1, 1, 1), (7, 5, 3), (sms, 2, 1), (sms, 3, 1), (sms, 7, 1)]:
        w = wl.make_workload(7, shape, seed=90)
        prob = w.problem()
        with VolumeTerm.from_problem(prob, precision="mixed") as vt:
            q32 = w.q_mixed()
            dev = vt.rhs(torch.from_numpy(q32).cuda())
            vt.status()
            host = vt.rhs_host(q32)
        assert np.array_equal(host, dev.cpu().numpy())
        check(host.astype(np.float64), oracle.vol_rhs_o2(prob, w.q), f"N=7 {shape}")


def test_bounded_wait_runs_out_and_reports_a_status():
    # The library's bounded mbarrier wait, made to run out on a barrier nothing
    # completes (no fault): numa_vol_status reports NUMA_ETIMEOUT, the status
    # word is cleared, and the handle still computes correct results.
    import time
    w = wl.make_workload(7, (2, 1, 1), seed=91)
    prob = w.problem()
    q32 = wl.perturbation_state(w.q, w.rho_ref, w.rhotheta_ref)
    with VolumeTerm.from_problem(prob, precision="mixed") as vt:
        vt.status()                                   # clean to begin with
        t0 = time.perf_counter()
        vt.selftest_wait(20000)                       # 20 ms limit
        with pytest.raises(NumaError, match="ETIMEOUT"):
            vt.status()
        waited = time.perf_counter() - t0
        assert 0.015 <= waited < 5.0, waited          # it waited about its limit, then gave up
        vt.status()                                   # cleared
        qd = torch.from_numpy(q32).cuda()
        out = vt.rhs(qd)
        vt.status()
        check(out.cpu().numpy().astype(np.float64), oracle.vol_rhs_o2(prob, w.q), "after a timeout")
    with pytest.raises(NumaError, match="EINVAL"):
        with VolumeTerm.from_problem(prob, precision="mixed") as vt:
            vt.selftest_wait(0)


@pytest.mark.parametrize("N", [3, 7])
def test_mixed_across_the_eos_forms(N):
    # Theta'/Theta_ref by warp in each range of the FP32 pressure perturbation
    # (5-term series, 16-term series, expm1f/log1pf) and mixed within warps.
    w = wl.make_workload(N, (3, 2, 1), seed=60 + N)
    q = w.q.copy()
    q[4] = w.rhotheta_ref * (1.0 + eos_banded_theta_ratio(w.M, seed=N))
    prob = w.problem()
    q32 = wl.perturbation_state(q, w.rho_ref, w.rhotheta_ref)
    check(run_mixed(prob, q32), oracle.vol_rhs_o2(prob, q), f"N={N} EOS forms")
