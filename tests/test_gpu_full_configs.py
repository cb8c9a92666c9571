"""The batched and serving workloads at their full sizes, in the launch
configurations bench.py times, checked by properties that hold at any size.

* Batched: the 64-instance plan (N in {3, 4, 5, 7}, 512..32768 elements,
  106.8M points), autotuned tiles, 10 LSRK steps at dt = 0.01 in one launch.
  Elements evolve independently, so sampled elements of every instance (first,
  last and one more) are checked against the oracle's integrator run on those
  elements alone, per field f and in the stored representation ((rho', U,
  Theta') in the mixed mode):
      max|q_f - q*_f| <= 32 (S_f + 100 u max|q*_f|).
  u is the unit roundoff of the stored state (2^-53 FP64, 2^-24 mixed) and
  100 u max|q*_f| covers the 50 stage updates q <- q + B dq rounding q one
  ulp apart.  S_f is the oracle's own response to perturbing its inputs by
  one rounding: in the mixed mode the FP32 rounding of the state, metric,
  Jinv and reference arrays that the mixed handle actually holds; in FP64 a
  relative 2^-53 with seeded random signs on each of those inputs.  With this
  workload's smooth velocities the 10-step increments are ~1e-6 of the state,
  and the difference is set by how rounding-level perturbations propagate,
  not by the increment: the hydrostatic Theta flux (Theta ~ 300 times u_d)
  and the metric feed rounding noise into Theta', hence into p', the
  momentum and rho' over the 0.1 s, at rates no a-priori norm bound tracks
  (the coupling is the acoustic one).  A computed evaluation is an exact one
  on inputs perturbed by ~17 roundings (state and geometry 3, flux 4,
  even-odd sweep Nq/2 + 2, three directions 2, Jinv and gravity 2); by
  linear response its effect is of the order of 17 S_f, and 32 doubles that.
  An FP32 emulation of the integrator on these elements gives at most 5 (S_f
  + floor) and the FP64 differences sit near 0.6 of it.  An indexing or
  formula error moves the increment by a fair fraction of itself, far above
  the bound.
* Serving: a seeded Poisson stream (200 requests/s) of requests drawn from the
  16-instance pool, through an engine with the bench's settings (120 GB budget,
  256 members, rounds of up to 4 steps, per-member rounds; lockstep too).  Each
  sampled request's result is bit for bit the batched integrator's on the same
  instance and step count.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, Engine, VolumeTerm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DT, NSTEPS = 0.01, 10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


@pytest.fixture(scope="module")
def plan_works():
    return [wl.integration_workload(N, n, seed) for N, n, seed in wl.batch_plan()]


def oracle_sensitivity(prob, q0, mixed):
    """S_f (module docstring): max over the element of the change in the
    oracle's 10-step result, per field and in the stored representation, when
    its inputs are perturbed by one rounding; and the unperturbed result in
    that representation."""
    if mixed:
        r = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
        rr, tr = r(prob["rho_ref"]), r(prob["rhotheta_ref"])
        pp = dict(prob, g=r(prob["g"]), Jinv=r(prob["Jinv"]), rho_ref=rr, rhotheta_ref=tr)
        qp = np.stack([rr + r(q0[0] - prob["rho_ref"]), r(q0[1]), r(q0[2]), r(q0[3]),
                       tr + r(q0[4] - prob["rhotheta_ref"])])
    else:
        rng = np.random.default_rng(0)
        r = lambda a: np.asarray(a) * (1 + 2.0 ** -53 * rng.choice([-1.0, 1.0], size=np.shape(a)))
        pp = dict(prob, g=r(prob["g"]), Jinv=r(prob["Jinv"]), rho_ref=r(prob["rho_ref"]),
                  rhotheta_ref=r(prob["rhotheta_ref"]))
        qp = r(q0)

    def stored(q, p):
        if not mixed:
            return q
        return np.concatenate([(q[0] - p["rho_ref"])[None], q[1:4], (q[4] - p["rhotheta_ref"])[None]])

    ref = stored(oracle.lsrk(prob, q0, DT, NSTEPS), prob)
    per = stored(oracle.lsrk(pp, qp, DT, NSTEPS), pp)
    return np.max(np.abs(per - ref), axis=1), ref


def element_problem(w, e):
    n3 = (w.N + 1) ** 3
    sl = slice(e * n3, (e + 1) * n3)
    prob = dict(w.problem(), Ne=1, g=np.ascontiguousarray(w.mesh.g[:, sl]),
                Jinv=w.mesh.Jinv[sl], rho_ref=w.rho_ref[sl], rhotheta_ref=w.rhotheta_ref[sl])
    return prob, np.ascontiguousarray(w.q[:, sl]), sl


@pytest.mark.parametrize("precision,sweep", [("fp64", "cuda_cores"), ("mixed", "cuda_cores"),
                                             ("mixed", "tensor_tf32")])
def test_batched_full_plan_on_sampled_elements(plan_works, precision, sweep):
    vts, states = [], []
    for w in plan_works:
        vts.append(VolumeTerm.from_problem(w.problem(), precision=precision))
        q0 = w.q_mixed() if precision == "mixed" else w.q
        states.append(torch.from_numpy(np.ascontiguousarray(q0)).cuda())
    assert sum(w.M for w in plan_works) == 106_757_616
    with Batch(precision, sweep=sweep) as b:
        for vt, q in zip(vts, states):
            b.add(vt, q)
        b.autotune()
        b.advance(NSTEPS, DT)
        b.status()
        torch.cuda.synchronize()
    mixed = precision == "mixed"
    u = 2.0 ** -24 if mixed else 2.0 ** -53
    rng = np.random.default_rng(7)
    ratios = []
    for w, q in zip(plan_works, states):
        got_all = q.cpu().numpy()
        for e in (0, w.Ne - 1, int(rng.integers(w.Ne))):
            prob, q0, sl = element_problem(w, e)
            S, ref = oracle_sensitivity(prob, q0, mixed)
            got = got_all[:, sl].astype(np.float64)
            bound = 32 * (S + 100 * u * np.max(np.abs(ref), axis=1))
            for f in range(5):
                err = np.max(np.abs(got[f] - ref[f]))
                assert err <= bound[f], (precision, w.N, w.Ne, e, wl.FIELD_NAMES[f], err, bound[f])
            if not mixed:
                # The FP64 increment q(T) - q(0) against the oracle's: the
                # small-batch bar 3e-12 of the increment, plus the oracle's own
                # response to one rounding of its inputs (S_f: it holds the
                # oracle's cancellation in p(Theta) - p(Theta_ref), about
                # ulp(p) ~ 1.5e-11 Pa per evaluation, which reaches the
                # momentum increments of these smooth states, ~1e-4 over the
                # 10 steps, at ~1e-13), plus one rounding of the stored state
                # per stage.  The 3e-12 alone holds for the rough states of the
                # small-batch tests, whose increments are far larger.
                inc, inc_ref = got - q0, ref - q0
                for f in range(5):
                    err = np.max(np.abs(inc[f] - inc_ref[f]))
                    ibound = (3e-12 * np.max(np.abs(inc_ref[f])) + 4 * S[f]
                              + 50 * u * np.max(np.abs(ref[f])))
                    ratios.append(err / ibound)
                    assert err <= ibound, (w.N, w.Ne, e, wl.FIELD_NAMES[f], err, ibound)
    if ratios:
        print("FP64 increment: largest error / bound", max(ratios))
    for vt in vts:
        vt.close()


@pytest.mark.parametrize("precision,policy", [("mixed", "per_member"), ("mixed", "lockstep"),
                                              ("fp64", "per_member")])
def test_serving_stream_results_equal_the_batch(precision, policy):
    plan = wl.batch_plan(count=16)
    works = [wl.integration_workload(N, n, seed) for N, n, seed in plan]
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in works]
    q0s = [np.ascontiguousarray(w.q_mixed() if precision == "mixed" else w.q) for w in works]
    rng = np.random.Generator(np.random.PCG64(2024))
    count = 24 if precision == "mixed" else 8
    picks = rng.integers(0, len(works), size=count)
    ks = rng.choice(np.array([1, 5, 20]), size=count)
    outs = [np.empty_like(q0s[j]) for j in picks]
    with Engine(precision, budget_bytes=120 << 30, max_members=256, round_steps=4,
                round_policy=policy) as eng:
        ids = []
        for n, (j, k) in enumerate(zip(picks, ks)):   # arrivals between rounds
            ids.append(eng.submit(vts[j], q0s[j], outs[n], int(k), DT))
            if n % 3 == 2:
                eng.progress()
        eng.run_until_idle()
        assert all(eng.query(r)["status"] == "done" for r in ids)
    for n in range(0, count, 4):   # a sample, against a direct batch integration
        j, k = picks[n], int(ks[n])
        q = torch.from_numpy(q0s[j].copy()).cuda()
        with Batch(precision) as b:
            b.add(vts[j], q)
            b.advance(k, DT)
        torch.cuda.synchronize()
        assert np.array_equal(outs[n], q.cpu().numpy()), (n, j, k)
    for vt in vts:
        vt.close()
