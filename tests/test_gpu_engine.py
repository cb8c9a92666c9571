"""GPU tests of the serving engine (numa_engine_*): continuous batching of
ensemble-member requests.

* Each request's result equals the batched integrator's on the same member,
  bitwise.  It is within the batch tests' 3e-12 (FP64 increments) of the
  oracle's integrator.
* A request's result is bitwise the same alone and in a mix where other
  requests arrive while it runs.
* Admission by the HBM budget: a request that does not fit waits, then runs.
* Host-side failures return status codes and leave the engine usable:
  malformed requests, a state larger than the budget, cancellation of a queued
  and of a running request.
* Rounds of several steps, lockstep and per member: the same bits as single
  steps, in fewer rounds.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, Engine, NumaError, VolumeTerm
from conftest import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DT = 0.01
MESHES = [(3, (3, 2, 1), 31), (7, (2, 1, 1), 32), (5, (2, 2, 1), 33), (4, (2, 2, 2), 34)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


@pytest.fixture(scope="module")
def pool():
    works = [wl.make_workload(N, shape, seed=seed) for N, shape, seed in MESHES]
    vts = [VolumeTerm.from_problem(w.problem()) for w in works]
    yield works, vts
    for vt in vts:
        vt.close()


def batch_reference(vt, q0, nsteps, precision="fp64"):
    q = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    with Batch(precision) as b:
        b.add(vt, q)
        b.advance(nsteps, DT)
    torch.cuda.synchronize()
    return q.cpu().numpy()


def test_results_equal_the_batch_and_the_oracle(pool):
    works, vts = pool
    ks = [3, 1, 5, 2]
    outs = [np.empty_like(w.q) for w in works]
    with Engine("fp64", budget_bytes=1 << 30) as eng:
        ids = [eng.submit(vt, w.q, o, k, DT) for vt, w, o, k in zip(vts, works, outs, ks)]
        done = eng.run_until_idle()
        assert sorted(done) == sorted(ids)
        for rid in ids:
            assert eng.query(rid)["status"] == "done"
    for w, vt, o, k in zip(works, vts, outs, ks):
        assert np.array_equal(o, batch_reference(vt, w.q, k))
        ref = oracle.lsrk(w.problem(), w.q, DT, k)
        for f, (mx, _) in enumerate(rel_err(o - w.q, ref - w.q)):
            assert mx <= 3e-12, (w.N, k, f, mx)


def test_result_is_the_same_alone_and_in_the_mix(pool):
    works, vts = pool
    w, vt = works[1], vts[1]
    alone = np.empty_like(w.q)
    with Engine("fp64", budget_bytes=1 << 30) as eng:
        eng.submit(vt, w.q, alone, 4, DT)
        eng.run_until_idle()
    mixed = np.empty_like(w.q)
    others = [np.empty_like(x.q) for x in works]
    with Engine("fp64", budget_bytes=1 << 30) as eng:
        eng.submit(vts[0], works[0].q, others[0], 6, DT)
        eng.progress()                                    # first engine round: member 0 alone
        rid = eng.submit(vt, w.q, mixed, 4, DT)           # arrives while 0 runs
        eng.progress()
        eng.submit(vts[2], works[2].q, others[2], 2, DT)  # arrives while both run
        eng.submit(vts[3], works[3].q, others[3], 1, DT)
        eng.progress()
        assert eng.stats()["resident"] >= 2              # work overlaps in one launch
        eng.run_until_idle()
        assert eng.query(rid)["status"] == "done"
    assert np.array_equal(alone, mixed)


def test_admission_waits_for_budget(pool):
    works, vts = pool
    w = works[3]
    need = w.q.nbytes
    outs = [np.empty_like(w.q) for _ in range(3)]
    with Engine("fp64", budget_bytes=need + 4096, max_members=8) as eng:
        ids = [eng.submit(vts[3], w.q, o, 2, DT) for o in outs]
        seen = []
        while True:
            st = eng.stats()
            if st["queued"] == 0 and st["resident"] == 0:
                break
            eng.progress()
            seen.append(eng.stats()["resident"])
        assert max(seen) <= 1                             # one member fits at a time
        for rid in ids:
            assert eng.query(rid)["status"] == "done"
        assert eng.stats()["bytes_used"] == 0
    ref = batch_reference(vts[3], w.q, 2)
    for o in outs:
        assert np.array_equal(o, ref)


def test_host_side_failures_return_codes_and_leave_the_engine_usable(pool):
    works, vts = pool
    w, vt = works[0], vts[0]
    out = np.empty_like(w.q)
    with Engine("fp64", budget_bytes=w.q.nbytes + 4096) as eng:
        with pytest.raises(NumaError, match="EINVAL"):
            eng.submit(vt, w.q, out, 0, DT)                  # malformed: no steps
        with pytest.raises(NumaError, match="EINVAL"):
            eng.submit(vt, w.q, out, 2, -1.0)                # malformed: dt <= 0
        big = works[3]
        with pytest.raises(NumaError, match="ELIMIT"):
            eng.submit(vts[3], big.q, np.empty_like(big.q), 1, DT)   # exceeds the whole budget
        mixed_vt = VolumeTerm.from_problem(w.problem(), precision="mixed")
        with pytest.raises(NumaError, match="precision"):
            eng.submit(mixed_vt, w.q_mixed(), np.empty_like(w.q_mixed()), 1, DT)
        mixed_vt.close()
        # cancellation: a queued request never runs, a running one is retired
        a = eng.submit(vt, w.q, out, 5, DT)
        b = eng.submit(vt, w.q, np.empty_like(w.q), 5, DT)   # queued behind a (budget)
        eng.progress()
        assert eng.query(a)["status"] == "running" and eng.query(b)["status"] == "queued"
        eng.cancel(b)
        eng.cancel(a)
        assert eng.query(b)["status"] == "cancelled"
        eng.progress()
        assert eng.query(a)["status"] == "cancelled"
        assert eng.stats()["bytes_used"] == 0 and eng.stats()["resident"] == 0
        with pytest.raises(NumaError):
            eng.cancel(a)                                    # already finished
        # still serves
        c = eng.submit(vt, w.q, out, 1, DT)
        eng.run_until_idle()
        assert eng.query(c)["status"] == "done"
    assert np.array_equal(out, batch_reference(vt, w.q, 1))


def test_mixed_precision_engine_matches_its_batch(pool):
    works, _ = pool
    w = works[2]
    vt = VolumeTerm.from_problem(w.problem(), precision="mixed")
    q0 = w.q_mixed()
    out = np.empty_like(q0)
    with Engine("mixed", budget_bytes=1 << 28) as eng:
        eng.submit(vt, q0, out, 3, DT)
        eng.run_until_idle()
    assert np.array_equal(out, batch_reference(vt, q0, 3, "mixed"))
    vt.close()


def test_allocation_refusal_is_a_status_code(pool):
    # A budget no GPU holds: the arena's reservation is refused, create
    # returns NUMA_ENOMEM, and the device stays usable (also for torch).
    with pytest.raises(NumaError, match="ENOMEM"):
        Engine("fp64", budget_bytes=1 << 50)
    x = torch.ones(1000, device="cuda") * 2
    torch.cuda.synchronize()
    assert float(x.sum()) == 2000.0
    works, vts = pool
    out = np.empty_like(works[0].q)
    with Engine("fp64", budget_bytes=1 << 26) as eng:
        eng.submit(vts[0], works[0].q, out, 1, DT)
        eng.run_until_idle()
    assert np.array_equal(out, batch_reference(vts[0], works[0].q, 1))


def test_checkpoint_and_resume_is_bitwise(pool):
    # A request checkpointed after some rounds and resumed (remaining steps) in a
    # fresh engine ends in the same bits as the uninterrupted request.
    works, vts = pool
    w, vt = works[2], vts[2]
    full = np.empty_like(w.q)
    with Engine("fp64", budget_bytes=1 << 28) as eng:
        eng.submit(vt, w.q, full, 6, DT)
        eng.run_until_idle()
    part = np.empty_like(w.q)
    with Engine("fp64", budget_bytes=1 << 28) as eng:
        queued = eng.submit(vt, w.q, np.empty_like(w.q), 2, DT)
        snap0, d0 = eng.checkpoint(queued)                  # not admitted: the initial state
        assert d0 == 0 and np.array_equal(snap0, w.q)
        rid = eng.submit(vt, w.q, np.empty_like(w.q), 6, DT)
        eng.progress()
        eng.progress()
        snap, done = eng.checkpoint(rid)
        assert done == 2 and not np.array_equal(snap, w.q)
        eng.cancel(rid)
        eng.run_until_idle()
    with Engine("fp64", budget_bytes=1 << 28) as eng:
        eng.submit(vt, snap, part, 6 - done, DT)
        eng.run_until_idle()
    assert np.array_equal(part, full)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_step_rounds_give_the_same_bits(pool, precision):
    # Rounds of up to 4 steps (never past a completion) against single-step
    # rounds: the same final states bit for bit, in fewer rounds.
    works, _ = pool
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in works]
    q0s = [w.q_mixed() if precision == "mixed" else w.q for w in works]
    ks = [7, 3, 5, 1]
    results = {}
    for rs in (1, 4):
        outs = [np.empty_like(q) for q in q0s]
        with Engine(precision, budget_bytes=1 << 28, round_steps=rs) as eng:
            for vt, q, o, k in zip(vts, q0s, outs, ks):
                eng.submit(vt, q, o, k, DT)
            eng.run_until_idle()
            results[rs] = (outs, eng.stats()["rounds"])
    for a, b in zip(results[1][0], results[4][0]):
        assert np.array_equal(a, b)
    assert results[4][1] < results[1][1]
    for vt in vts:
        vt.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_per_member_rounds_give_the_same_bits_in_fewer_rounds(pool, precision):
    # Rounds of up to 4 steps, a 13-step request beside a stream of 1-step
    # requests (one arrives before every round).  Lockstep rounds then advance
    # everyone one step at a time; per-member rounds advance the long request
    # 4 + 4 + 4 + 1 steps, done in round 4.  Every final state is bitwise the
    # same under both policies.
    works, _ = pool
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in works]
    q0s = [w.q_mixed() if precision == "mixed" else w.q for w in works]
    outs, done_in = {}, {}
    for policy in ("lockstep", "per_member"):
        o = [np.empty_like(q0s[0])] + [np.empty_like(q0s[1 + n % 3]) for n in range(12)]
        with Engine(precision, budget_bytes=1 << 28, round_steps=4, round_policy=policy) as eng:
            long_id = eng.submit(vts[0], q0s[0], o[0], 13, DT)
            done_in[policy] = None
            for n in range(12):
                eng.submit(vts[1 + n % 3], q0s[1 + n % 3], o[1 + n], 1, DT)
                eng.progress()
                eng.drain()   # the round has run and its results are in host memory
                if done_in[policy] is None and eng.query(long_id)["status"] == "done":
                    done_in[policy] = n + 1
            eng.run_until_idle()
        outs[policy] = o
    for a, b in zip(outs["lockstep"], outs["per_member"]):
        assert np.array_equal(a, b)
    assert done_in["per_member"] == 4
    assert done_in["lockstep"] is None   # still running after 12 one-step rounds
    for vt in vts:
        vt.close()


@pytest.mark.parametrize("policy", ["lockstep", "per_member"])
def test_rounds_allocate_no_device_memory(pool, policy):
    """After the first round (the kernel's one-time set-up), rounds with
    admissions, launches and result copies leave the device's free memory and
    the PyTorch allocator's reserve unchanged: the arena and the work tables
    are reserved at create time."""
    works, vts = pool
    outs = [np.empty_like(works[n % len(works)].q) for n in range(12)]
    with Engine("fp64", budget_bytes=1 << 28, max_members=8, round_steps=2,
                round_policy=policy) as eng:
        eng.submit(vts[0], works[0].q, np.empty_like(works[0].q), 1, DT)
        eng.run_until_idle()
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        ids = []
        for n, o in enumerate(outs):
            j = n % len(works)
            ids.append(eng.submit(vts[j], works[j].q, o, 1 + n % 5, DT))
            eng.progress()
            assert torch.cuda.mem_get_info()[0] == free0
        eng.run_until_idle()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
        assert all(eng.query(r)["status"] == "done" for r in ids)
    for n, o in enumerate(outs):
        j = n % len(works)
        assert np.array_equal(o, batch_reference(vts[j], works[j].q, 1 + n % 5))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_members_with_tracers(precision):
    # A member with three tracers beside one without: the rounds run the batch's
    # tracer tiles.  Each result equals its own batch integration bit for bit
    # and the oracle's integrator within the batch's bars.
    w8 = wl.make_workload(3, (2, 2, 1), seed=470, tracers=3)
    w5 = wl.make_workload(5, (2, 1, 1), seed=471)
    ws = [w8, w5]
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in ws]
    q0s = [w.q_mixed() if precision == "mixed" else w.q for w in ws]
    outs = [np.empty_like(q) for q in q0s]
    ks = [3, 2]
    with Engine(precision, budget_bytes=1 << 30) as eng:
        ids = [eng.submit(vt, q, o, k, DT) for vt, q, o, k in zip(vts, q0s, outs, ks)]
        assert sorted(eng.run_until_idle()) == sorted(ids)
    assert np.array_equal(outs[0], batch_reference(vts[0], q0s[0], ks[0], precision))
    if precision == "fp64":
        assert np.array_equal(outs[1], batch_reference(vts[1], q0s[1], ks[1], precision))
    for w, o, k in zip(ws, outs, ks):
        ref = oracle.lsrk(w.problem(), w.q, DT, k)
        got = o.astype(np.float64)
        if precision == "mixed":
            ref = np.concatenate([(ref[0] - w.rho_ref)[None], ref[1:4],
                                  (ref[4] - w.rhotheta_ref)[None], ref[5:]])
            errs, tol = rel_err(got, ref), 1e-5
        else:
            errs, tol = rel_err(got - w.q, ref - w.q), 3e-12
        assert len(errs) == w.q.shape[0]
        for f, (mx, _) in enumerate(errs):
            assert mx <= tol, (precision, w.N, f, mx)
    for vt in vts:
        vt.close()
