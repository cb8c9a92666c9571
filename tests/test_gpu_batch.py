"""GPU tests of batched low-storage Runge-Kutta integration (numa_batch_*).

Reference: the oracle's integrator (same scheme, its own coefficients, O2 for
the volume term), per instance.  The bar is on the state increment
dq_total = q(T) - q(0), per field, normwise:
  FP64:  max|dq - dq*| / max|dq*| <= 3e-12.  An increment is dt times a positive
         combination of 5 volume-term evaluations per step (the scheme's Butcher
         weights are positive and sum to 1).  Each evaluation meets the 1e-12
         single-evaluation bar, and its ~5e-13 difference from the oracle (the
         oracle's cancellation in p(Theta) - p(Theta_ref)) enters every stage's
         state.  So the increment's bar is three times the evaluation's.
         Separately, the batch must agree to 1e-13 with a host-driven
         integration that calls the (parity-tested) single-evaluation kernel
         once per stage: the batch adds no error of its own.
  mixed: the final state in the mode's own representation (rho', U, Theta'),
         per field normwise against the oracle's state converted to it: <= 1e-5.
         (The increment is not the right measure for FP32 storage: U ~ 10 has
         an ulp of ~1e-6, while a 0.02 s increment of U on a coarse element can
         be ~2e-4.)
Instances of a batch do not interact, so each result must be bitwise the same
alone and in company.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, NumaError, VolumeTerm
from conftest import eos_banded_theta_ratio, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DT, NSTEPS = 0.01, 2
SPECS = [(1, (2, 1, 1), 11), (3, (3, 2, 1), 12), (4, (2, 2, 2), 13), (5, (1, 2, 3), 14),
         (7, (2, 2, 1), 15), (7, (1, 1, 1), 16)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def make(spec, precision):
    N, shape, seed = spec
    w = wl.make_workload(N, shape, seed=seed)
    vt = VolumeTerm.from_problem(w.problem(), precision=precision)
    q0 = w.q_mixed() if precision == "mixed" else w.q
    return w, vt, torch.from_numpy(np.ascontiguousarray(q0)).cuda()


def increment_errors(w, q_final, nsteps=NSTEPS, mixed=False):
    ref = oracle.lsrk(w.problem(), w.q, DT, nsteps)
    got = np.asarray(q_final, dtype=np.float64)
    if mixed:   # state errors in the perturbation representation
        ref_pert = np.concatenate([(ref[0] - w.rho_ref)[None], ref[1:4],
                                   (ref[4] - w.rhotheta_ref)[None]])
        return rel_err(got, ref_pert)
    return rel_err(got - w.q, ref - w.q)


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-12), ("mixed", 1e-5)])
def test_batch_with_tracers_matches_oracle_integrator(precision, tol):
    # A batch holding instances with tracers runs the tiles' tracer forms:
    # instances of 5, 6 and 8 fields at three orders, every field against the
    # oracle's integrator (tracers as they are in the mixed mode); an instance's
    # five base fields bit for bit as the same instance without tracers in the
    # same batch; in FP64 a tracer that starts equal to Theta stays equal.
    specs = [(3, (3, 2, 1), 61, 3), (5, (2, 1, 2), 62, 1), (7, (2, 2, 1), 63, 3),
             (4, (2, 2, 1), 64, 0)]
    runs = []
    for N, shape, seed, T in specs:
        w = wl.make_workload(N, shape, seed=seed, tracers=T)
        if T == 3 and precision == "fp64" and N == 7:
            w.q[5] = w.q[4]   # Q1 = Theta
        runs.append(w)
    twin = wl.make_workload(3, (3, 2, 1), seed=61)   # the first instance without tracers
    with Batch(precision) as b:
        keep = []
        for w in runs + [twin]:
            vt = VolumeTerm.from_problem(w.problem(), precision=precision)
            q0 = w.q_mixed() if precision == "mixed" else w.q
            q = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
            b.add(vt, q)
            keep.append((vt, q))
        b.advance(NSTEPS, DT)
        torch.cuda.synchronize()
        outs = [q.cpu().numpy() for _, q in keep]
        for w, got, sp in zip(runs, outs, specs):
            ref = oracle.lsrk(w.problem(), w.q, DT, NSTEPS)
            got = got.astype(np.float64)
            if precision == "mixed":
                ref_pert = np.concatenate([(ref[0] - w.rho_ref)[None], ref[1:4],
                                           (ref[4] - w.rhotheta_ref)[None], ref[5:]])
                errs = rel_err(got, ref_pert)
            else:
                errs = rel_err(got - w.q, ref - w.q)
            assert len(errs) == w.q.shape[0]
            for f, (mx, _) in enumerate(errs):
                assert mx <= tol, (precision, sp, f, mx)
        assert np.array_equal(outs[0][:5], outs[-1])
        if precision == "fp64":
            assert np.array_equal(outs[2][5], outs[2][4])
        for vt, _ in keep:
            vt.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-12), ("mixed", 1e-5)])
def test_batch_matches_oracle_integrator(precision, tol):
    runs = [make(sp, precision) for sp in SPECS]
    with Batch(precision) as b:
        for w, vt, q in runs:
            b.add(vt, q)
        assert len(b) == len(SPECS)
        b.advance(NSTEPS, DT)
        torch.cuda.synchronize()
        for (w, vt, q), sp in zip(runs, SPECS):
            errs = increment_errors(w, q.cpu().numpy(), mixed=precision == "mixed")
            print(precision, sp, errs)
            for f, (mx, _) in enumerate(errs):
                assert mx <= tol, (sp, wl.FIELD_NAMES[f], mx)
    for _, vt, _ in runs:
        vt.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_instance_result_is_bitwise_the_same_alone_and_in_company(precision):
    alone = make(SPECS[4], precision)
    with Batch(precision) as b:
        b.add(alone[1], alone[2])
        b.advance(NSTEPS, DT)
    torch.cuda.synchronize()
    runs = [make(sp, precision) for sp in SPECS]
    with Batch(precision) as b:
        for w, vt, q in runs[::-1]:
            b.add(vt, q)
        b.advance(NSTEPS, DT)
    torch.cuda.synchronize()
    assert torch.equal(alone[2], runs[4][2])


def test_graph_replay_and_split_steps():
    # A[0] = 0, so each step starts afresh: 1 + 1 steps equal 2 steps bitwise,
    # through the captured graph (replayed for the second call).
    a = make(SPECS[2], "fp64")
    c = make(SPECS[2], "fp64")
    with Batch("fp64") as b1, Batch("fp64") as b2:
        b1.add(a[1], a[2])
        b1.advance(1, DT)
        b1.advance(1, DT)
        b2.add(c[1], c[2])
        b2.advance(2, DT)
        torch.cuda.synchronize()
    assert torch.equal(a[2], c[2])


def test_autotune_leaves_states_and_picks_tiles():
    runs = [make(sp, "fp64") for sp in SPECS]
    with Batch("fp64") as b:
        for w, vt, q in runs:
            b.add(vt, q)
        before = [q.clone() for _, _, q in runs]
        b.autotune()
        torch.cuda.synchronize()
        for q0, (_, _, q) in zip(before, runs):
            assert torch.equal(q0, q)
        for N in (1, 3, 4, 5, 7):
            assert b.tile(N + 1) >= 512 // (N + 1) ** 3
        b.advance(NSTEPS, DT)
        torch.cuda.synchronize()
        w, _, q = runs[3]
        for mx, _ in increment_errors(w, q.cpu().numpy()):
            assert mx <= 3e-12


def test_batch_equals_host_driven_integration_with_the_single_kernel():
    import oracle as _o
    A, B, _ = _o.lsrk_coefficients()
    for sp in SPECS:
        w, vt, q = make(sp, "fp64")
        with Batch("fp64") as b:
            b.add(vt, q)
            b.advance(NSTEPS, DT)
        qh = torch.from_numpy(w.q).cuda()
        dq = torch.zeros_like(qh)
        for _ in range(NSTEPS):
            for s in range(5):
                dq = A[s] * dq + DT * vt.rhs(qh)
                qh = qh + B[s] * dq
        torch.cuda.synchronize()
        for mx, _ in rel_err(q.cpu().numpy() - w.q, qh.cpu().numpy() - w.q):
            assert mx <= 1e-13, (sp, mx)
        vt.close()


def test_batch_rejects_handles_of_another_precision():
    w, vt, q = make(SPECS[1], "mixed")
    # a mixed handle with its own (float32) state, offered to an FP64 batch:
    # the C ABI rejects the precision mismatch
    with Batch("fp64") as b, pytest.raises(NumaError, match="precision"):
        b.add(vt, q)
    vt.close()


def test_batch_of_the_mixed_size_plan_on_a_sample():
    # The 64-instance plan's first 6 instances (orders 3..7, 512..32768
    # elements): the GPU batch, checked on the first 6 elements of each
    # instance against the oracle (elements evolve independently).
    plan = wl.batch_plan()[:6]
    runs = []
    for N, n, seed in plan:
        w = wl.make_workload(N, n, seed=seed)
        vt = VolumeTerm.from_problem(w.problem(), precision="fp64")
        runs.append((w, vt, torch.from_numpy(w.q).cuda()))
    with Batch("fp64") as b:
        for w, vt, q in runs:
            b.add(vt, q)
        b.advance(NSTEPS, DT)
        torch.cuda.synchronize()
    for w, vt, q in runs:
        n3 = (w.N + 1) ** 3
        m = 6 * n3
        sub = dict(w.problem(), Ne=6, g=np.ascontiguousarray(w.mesh.g[:, :m]),
                   Jinv=w.mesh.Jinv[:m], rho_ref=w.rho_ref[:m], rhotheta_ref=w.rhotheta_ref[:m])
        q0 = np.ascontiguousarray(w.q[:, :m])
        ref = oracle.lsrk(sub, q0, DT, NSTEPS)
        got = q.cpu().numpy()[:, :m]
        for f, (mx, _) in enumerate(rel_err(got - q0, ref - q0)):
            assert mx <= 3e-12, (w.N, w.Ne, f, mx)
        vt.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 3e-12), ("mixed", 1e-5)])
def test_batch_across_the_eos_branches(precision, tol):
    # Theta'/Theta_ref spread over all ranges of the pressure perturbation
    # (series of 9 and 15 terms, expm1/log1p beyond 1/8), by warp and mixed
    # within warps, as states reach after many steps on fine meshes.
    w = wl.make_workload(7, (3, 2, 1), seed=21)
    w.q[4] = w.rhotheta_ref * (1.0 + eos_banded_theta_ratio(w.M, seed=3))
    vt = VolumeTerm.from_problem(w.problem(), precision=precision)
    q0 = w.q_mixed() if precision == "mixed" else w.q
    q = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    with Batch(precision) as b:
        b.add(vt, q)
        b.advance(NSTEPS, DT)
    torch.cuda.synchronize()
    errs = increment_errors(w, q.cpu().numpy(), mixed=precision == "mixed")
    for f, (mx, _) in enumerate(errs):
        assert mx <= tol, (precision, wl.FIELD_NAMES[f], mx)
    vt.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_candidate_configuration_keeps_parity(precision):
    """Every configuration the autotuner can choose (tiles of 1..32 passes,
    CTAs per SM, item order and, in the mixed mode, either sweep per order)
    gives a result within the bar."""
    runs = [make(sp, precision) for sp in SPECS]
    refs = []
    for w, _, _ in runs:
        refs.append(oracle.lsrk(w.problem(), w.q, DT, NSTEPS))
    saved = [q.clone() for _, _, q in runs]
    sweeps = ["cuda_cores", "tensor_tf32"] if precision == "mixed" else ["cuda_cores"]
    ctas = [1, 2] if precision == "mixed" else [1]
    tol = 1e-5 if precision == "mixed" else 3e-12
    with Batch(precision) as b:
        for w, vt, q in runs:
            b.add(vt, q)
        tmems = [False, True] if precision == "mixed" else [False]
        for passes in (1, 2, 4, 8, 16, 32):
            for sweep in sweeps:
                for k in ctas:
                    for costliest, tmem in ((False, False), (True, tmems[-1])):
                        for (_, _, q), q0 in zip(runs, saved):
                            q.copy_(q0)
                        b.set_config(tile={nq: passes * (512 // nq ** 3) for nq in range(2, 9)},
                                     sweep={nq: sweep for nq in range(2, 9)}, ctas_per_sm=k,
                                     costliest_first=costliest, state_in_tmem=tmem)
                        b.advance(NSTEPS, DT)
                        b.status()
                        torch.cuda.synchronize()
                        for (w, _, q), ref, sp in zip(runs, refs, SPECS):
                            got = q.cpu().numpy().astype(np.float64)
                            if precision == "mixed":
                                ref_s = np.concatenate([(ref[0] - w.rho_ref)[None], ref[1:4],
                                                        (ref[4] - w.rhotheta_ref)[None]])
                                errs = rel_err(got, ref_s)
                            else:
                                errs = rel_err(got - w.q, ref - w.q)
                            for f, (mx, _) in enumerate(errs):
                                assert mx <= tol, (passes, sweep, k, costliest, tmem, sp, f, mx)


def test_autotune_reports_configuration():
    runs = [make(sp, "mixed") for sp in SPECS]
    with Batch("mixed", sweep="auto") as b:
        for w, vt, q in runs:
            b.add(vt, q)
        b.autotune()
        c = b.config()
        assert c["tuned_ms_per_step"] > 0 and c["tuned_candidates"] > 0
        for nq in (2, 4, 5, 6, 8):
            assert c["tile"][nq] % (512 // nq ** 3) == 0
        with pytest.raises(NumaError):
            b.set_config(tile={4: 12})   # not a multiple of the 8 elements per pass at Nq = 4
        with pytest.raises(NumaError):
            b.set_config(ctas_per_sm=3)
