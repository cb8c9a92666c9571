"""GPU tests of the tensor-core sweep of NUMA_MIXED batches
(numa_batch_set_sweep(b, NUMA_SWEEP_TENSOR_TF32)).

The D sums of Sec. 2, Eq. (2) run as TF32 split products on tcgen05 with
FP32 accumulation.  Reference: the oracle's integrator (the same five-stage
scheme over its FP64 volume term).  Bar, as for the CUDA-core mixed batch: the
final state in the mode's own representation (rho', U, Theta'), per field
normwise against the oracle's state converted to it, <= 1e-5.  The split
products carry about 2^-21 relative error per sum (against 2^-24 for FP32
FMAs), far inside that bar; the test also bounds the distance to the
CUDA-core sweep by the same 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, NumaError, VolumeTerm
from conftest import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DT, NSTEPS = 0.01, 2
# every order the batch takes; ragged element counts (partial passes) included
SPECS = [(1, (2, 1, 1), 21), (2, (3, 1, 1), 22), (3, (3, 2, 1), 23), (4, (2, 2, 2), 24),
         (5, (1, 2, 3), 25), (6, (1, 1, 2), 26), (7, (2, 2, 1), 27), (7, (1, 1, 1), 28)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def make(spec, integration=False):
    N, shape, seed = spec
    w = (wl.integration_workload(N, shape, seed=seed) if integration
         else wl.make_workload(N, shape, seed=seed))
    vt = VolumeTerm.from_problem(w.problem(), precision="mixed")
    return w, vt, torch.from_numpy(np.ascontiguousarray(w.q_mixed())).cuda()


def state_errors(w, q_final, nsteps=NSTEPS):
    ref = oracle.lsrk(w.problem(), w.q, DT, nsteps)
    ref_pert = np.concatenate([(ref[0] - w.rho_ref)[None], ref[1:4],
                               (ref[4] - w.rhotheta_ref)[None]])
    return rel_err(np.asarray(q_final, dtype=np.float64), ref_pert)


@pytest.mark.parametrize("integration", [False, True], ids=["rough", "smooth"])
def test_tensor_sweep_matches_oracle_integrator(integration):
    runs = [make(sp, integration) for sp in SPECS]
    with Batch("mixed", sweep="tensor_tf32") as b:
        assert b.sweep == "tensor_tf32"
        for w, vt, q in runs:
            b.add(vt, q)
        b.advance(NSTEPS, DT)
        b.status()
        torch.cuda.synchronize()
        for (w, vt, q), sp in zip(runs, SPECS):
            errs = state_errors(w, q.cpu().numpy())
            print(sp, errs)
            for f, (mx, _) in enumerate(errs):
                assert mx <= 1e-5, (sp, wl.FIELD_NAMES[f], mx)
    for _, vt, _ in runs:
        vt.close()


def test_tensor_sweep_close_to_cuda_core_sweep():
    a = [make(sp) for sp in SPECS]
    c = [make(sp) for sp in SPECS]
    with Batch("mixed", sweep="tensor_tf32") as bt, Batch("mixed") as bc:
        for (_, vt, q) in a:
            bt.add(vt, q)
        for (_, vt, q) in c:
            bc.add(vt, q)
        bt.advance(NSTEPS, DT)
        bc.advance(NSTEPS, DT)
        torch.cuda.synchronize()
    for (w, _, qa), (_, _, qc), sp in zip(a, c, SPECS):
        errs = rel_err(qa.double().cpu().numpy(), qc.double().cpu().numpy())
        for f, (mx, _) in enumerate(errs):
            assert mx <= 1e-5, (sp, f, mx)


def test_tensor_sweep_alone_equals_in_company():
    alone = make(SPECS[6])
    with Batch("mixed", sweep="tensor_tf32") as b:
        b.add(alone[1], alone[2])
        b.advance(NSTEPS, DT)
    torch.cuda.synchronize()
    runs = [make(sp) for sp in SPECS]
    with Batch("mixed", sweep="tensor_tf32") as b:
        for w, vt, q in runs[::-1]:
            b.add(vt, q)
        b.advance(NSTEPS, DT)
    torch.cuda.synchronize()
    assert torch.equal(alone[2], runs[6][2])


def test_sweep_switch_and_graph_replay():
    # switching sweeps recaptures; replays of the captured graph continue
    x = make(SPECS[3])
    y = make(SPECS[3])
    with Batch("mixed") as b1, Batch("mixed") as b2:
        b1.sweep = "tensor_tf32"
        b1.add(x[1], x[2])
        b1.advance(1, DT)
        b1.advance(1, DT)
        b2.add(y[1], y[2])
        b2.sweep = "tensor_tf32"
        b2.advance(2, DT)
        b2.sweep = "cuda_cores"
        assert b2.sweep == "cuda_cores"
        torch.cuda.synchronize()
    assert torch.equal(x[2], y[2])


def test_tensor_sweep_refused_for_fp64():
    with Batch("fp64") as b:
        with pytest.raises(NumaError):
            b.sweep = "tensor_tf32"
        assert b.sweep == "cuda_cores"


def test_tensor_sweep_autotune_leaves_states():
    # three instances of the batched plan's orders; the autotuner times the
    # tensor-core kernel on copies of the states
    runs = [make(sp) for sp in (SPECS[2], SPECS[4], SPECS[6])]
    with Batch("mixed", sweep="tensor_tf32") as b:
        for w, vt, q in runs:
            b.add(vt, q)
        before = [q.clone() for _, _, q in runs]
        b.autotune()
        torch.cuda.synchronize()
        for (_, _, q), q0 in zip(runs, before):
            assert torch.equal(q, q0)
        for nq in (4, 6, 8):
            assert b.tile(nq) >= 512 // nq ** 3
        b.advance(NSTEPS, DT)
        b.status()
        torch.cuda.synchronize()
    for (w, vt, q), sp in zip(runs, (SPECS[2], SPECS[4], SPECS[6])):
        for f, (mx, _) in enumerate(state_errors(w, q.cpu().numpy())):
            assert mx <= 1e-5, (sp, f, mx)
        vt.close()


def test_auto_sweep_picks_per_order_and_keeps_parity():
    runs = [make(sp) for sp in SPECS]
    with Batch("mixed", sweep="auto") as b:
        assert b.sweep == "auto"
        for w, vt, q in runs:
            b.add(vt, q)
        b.autotune()
        chosen = {nq: b.sweep_of(nq) for nq in range(2, 9)}
        assert set(chosen.values()) <= {"cuda_cores", "tensor_tf32"}
        print(chosen)
        b.advance(NSTEPS, DT)
        b.status()
        torch.cuda.synchronize()
        for (w, vt, q), sp in zip(runs, SPECS):
            for f, (mx, _) in enumerate(state_errors(w, q.cpu().numpy())):
                assert mx <= 1e-5, (sp, chosen, f, mx)
    for _, vt, _ in runs:
        vt.close()
