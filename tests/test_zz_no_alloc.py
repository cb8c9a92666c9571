"""numa_batch_advance_noalloc: the batch advance for callers that cannot
allocate device memory once running.  An example is a serving process whose
HBM budget is already committed to resident ensemble states.  Its scratch lives
in a fixed device array of the library, so the call itself allocates nothing.

Checked through the C ABI against the allocating entry point
(numa_batch_advance) on the same states, after each of two calls in a row,
with one and with three steps per call (the several-step loop inside one
persistent launch), within the tolerances the batch tests use: 1e-13 relative
on the FP64 state increments, 1e-5 on the mixed-precision states.  Across the
second call neither the device's free memory nor the PyTorch allocator's
reserved bytes change (the first call does the one-time set-up).  A stream
under capture is refused.  This file is collected last, and it also passes
alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1604_08501_gb300 import _lib, build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import Batch, VolumeTerm
from conftest import rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DT = 0.01
SPECS = [(3, (3, 2, 1), 21), (7, (2, 1, 1), 22), (5, (2, 2, 1), 23), (1, (4, 1, 1), 24)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def _arrays(vts, states):
    n = len(vts)
    handles = (C.c_void_p * n)(*[vt.handle for vt in vts])
    ptrs = (C.c_void_p * n)(*[q.data_ptr() for q in states])
    return handles, ptrs


@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-5)])
def test_noalloc_advance_matches_batch_advance_on_two_calls(precision, tol, nsteps):
    lib = _lib.load()
    works = [wl.make_workload(N, shape, seed=seed) for N, shape, seed in SPECS]
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in works]
    q0 = [w.q_mixed() if precision == "mixed" else w.q for w in works]
    qa = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in q0]   # allocating path
    qb = [t.clone() for t in qa]                                           # no-alloc path
    handles, ptrs = _arrays(vts, qb)
    stream = torch.cuda.current_stream().cuda_stream
    with Batch(precision) as b:
        for vt, q in zip(vts, qa):
            b.add(vt, q)
        for call in range(2):
            b.advance(nsteps, DT)
            torch.cuda.synchronize()
            free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
            rc = lib.numa_batch_advance_noalloc(handles, ptrs, len(vts), nsteps, DT,
                                                C.c_void_p(stream))
            assert rc == _lib.NUMA_OK
            torch.cuda.synchronize()
            if call == 1:   # after the first call's one-time set-up: nothing allocated
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_reserved() == reserved0
            for k, (a, bq) in enumerate(zip(qa, qb)):
                a_np, b_np = a.cpu().numpy().astype(np.float64), bq.cpu().numpy().astype(np.float64)
                if precision == "fp64":
                    errs = rel_err(b_np - q0[k], a_np - q0[k])
                else:
                    errs = rel_err(b_np, a_np)
                for f, (mx, _) in enumerate(errs):
                    assert mx <= tol, (precision, call, SPECS[k], f, mx)
    for vt in vts:
        vt.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-5)])
def test_noalloc_advance_with_tracers_matches_batch_advance(precision, tol):
    # Instances of 8, 6 and 5 fields: the call runs the tiles' tracer forms,
    # as numa_batch_advance does for the same instances.
    lib = _lib.load()
    specs = [(3, (3, 2, 1), 31, 3), (7, (2, 1, 1), 32, 1), (5, (2, 2, 1), 33, 0)]
    works = [wl.make_workload(N, shape, seed=seed, tracers=T) for N, shape, seed, T in specs]
    vts = [VolumeTerm.from_problem(w.problem(), precision=precision) for w in works]
    q0 = [w.q_mixed() if precision == "mixed" else w.q for w in works]
    qa = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for q in q0]
    qb = [t.clone() for t in qa]
    handles, ptrs = _arrays(vts, qb)
    with Batch(precision) as b:
        for vt, q in zip(vts, qa):
            b.add(vt, q)
        b.advance(3, DT)
        assert lib.numa_batch_advance_noalloc(handles, ptrs, len(vts), 3, DT, None) == _lib.NUMA_OK
        torch.cuda.synchronize()
        for k, (a, bq) in enumerate(zip(qa, qb)):
            a_np, b_np = a.cpu().numpy().astype(np.float64), bq.cpu().numpy().astype(np.float64)
            errs = rel_err(b_np - q0[k], a_np - q0[k]) if precision == "fp64" else rel_err(b_np, a_np)
            assert len(errs) == works[k].q.shape[0]
            for f, (mx, _) in enumerate(errs):
                assert mx <= tol, (precision, specs[k], f, mx)
    for vt in vts:
        vt.close()


def test_noalloc_rejects_counts_beyond_its_maximum_and_bad_arguments():
    lib = _lib.load()
    w = wl.make_workload(2, 1, seed=3)
    vt = VolumeTerm.from_problem(w.problem())
    q = torch.from_numpy(w.q).cuda()
    n = _lib.NUMA_NOALLOC_MAX_INSTANCES + 1
    handles = (C.c_void_p * n)(*([vt.handle] * n))
    ptrs = (C.c_void_p * n)(*([q.data_ptr()] * n))
    assert lib.numa_batch_advance_noalloc(handles, ptrs, n, 1, DT, None) == _lib.NUMA_ELIMIT
    assert lib.numa_batch_advance_noalloc(handles, ptrs, 0, 1, DT, None) == _lib.NUMA_EINVAL
    assert lib.numa_batch_advance_noalloc(None, ptrs, 1, 1, DT, None) == _lib.NUMA_EINVAL
    mis = (C.c_void_p * 1)(q.data_ptr() + 8)
    assert lib.numa_batch_advance_noalloc(handles, mis, 1, 1, DT, None) == _lib.NUMA_EINVAL
    wm = wl.make_workload(2, 1, seed=3)
    vm = VolumeTerm.from_problem(wm.problem(), precision="mixed")
    qm = torch.from_numpy(wm.q_mixed()).cuda()
    two_h = (C.c_void_p * 2)(vt.handle, vm.handle)
    two_q = (C.c_void_p * 2)(q.data_ptr(), qm.data_ptr())
    assert lib.numa_batch_advance_noalloc(two_h, two_q, 2, 1, DT, None) == _lib.NUMA_EINVAL
    # nothing was launched by the rejected calls: the states are unchanged
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), w.q)
    vt.close()
    vm.close()


def test_noalloc_refuses_a_stream_under_capture():
    lib = _lib.load()
    w = wl.make_workload(3, (2, 1, 1), seed=5)
    vt = VolumeTerm.from_problem(w.problem())
    q = torch.from_numpy(w.q).cuda()
    handles, ptrs = _arrays([vt], [q])
    side = torch.cuda.Stream()
    # the one-time set-up happens outside any capture
    assert lib.numa_batch_advance_noalloc(handles, ptrs, 1, 1, DT,
                                          C.c_void_p(side.cuda_stream)) == _lib.NUMA_OK
    torch.cuda.synchronize()
    before = q.clone()
    scratch = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        scratch.add_(1.0)   # the graph captures something of its own
        rc = lib.numa_batch_advance_noalloc(handles, ptrs, 1, 1, DT, C.c_void_p(side.cuda_stream))
    assert rc == _lib.NUMA_EINVAL
    # the graph is never replayed; nothing of the refused call ran
    torch.cuda.synchronize()
    assert torch.equal(q, before)
    del g
    vt.close()
