"""numa_vol_rhs inside a CUDA graph: a time loop can capture an evaluation (with
its surrounding PyTorch ops) once and replay it.  The replayed result must be
bitwise the eager one, in every mode and at a low and a high order."""
import numpy as np
import pytest

from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


@pytest.mark.parametrize("N,precision", [(4, "fp64"), (7, "fp64"), (7, "mixed"), (7, "df64"),
                                         (11, "fp64"), (11, "mixed")])
def test_rhs_replays_in_a_cuda_graph(N, precision):
    w = wl.make_workload(N, (3, 2, 1), seed=700 + N)
    with VolumeTerm.from_problem(w.problem(), precision=precision) as vt:
        q0 = w.q_mixed() if precision == "mixed" else w.q
        q = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
        out = torch.empty_like(q)
        eager = vt.rhs(q, torch.empty_like(q)).clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):                 # warm the launch path outside capture
            vt.rhs(q, out, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        out.zero_()
        with torch.cuda.graph(g):
            vt.rhs(q, out)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
        q.mul_(1.0)                                # replay again on the same buffers
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
