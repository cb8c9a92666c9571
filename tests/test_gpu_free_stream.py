"""Free stream on the warped benchmark box through the C ABI.

With metrics in Kopriva's conservative curl form (tests/curl_metrics.py) the
discrete metric identities hold to rounding, so a uniform flow has zero flux
divergence on curved elements: the library must give rhs = 0 to rounding in
every direction, field and order, which exercises the metric slots, the
contravariant velocity and all three sweeps on curved geometry with exact
cancellation.  Bounds, with s the largest row sum of |D| and B the oracle's
running bound J^-1 sum |D| |F|: FP64 s^2 2^-53 B (the rounding of the computed
metrics, differentiated twice; the oracle meets it, tests/test_oracle_pins.py);
mixed s^2 2^-24 B (the metrics rounded to FP32 once, then the same).
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import build
from paper_1604_08501_gb300 import workload as wl
from paper_1604_08501_gb300.numa_vol import VolumeTerm
from curl_metrics import curl_form_metrics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def free_stream_problem(N, shape):
    mesh = wl.warped_box(N, shape)
    c = wl.Constants(p0=1.0e5, R=287.0, cp=1004.0, grav=0.0)
    rho, vel, Th = 1.2, np.array([3.0, -2.0, 5.0]), 350.0
    q = np.empty((5, mesh.M))
    q[0], q[1:4], q[4] = rho, (rho * vel)[:, None], Th
    prob = {"N": N, "Ne": mesh.Ne, "g": curl_form_metrics(mesh.x, N, mesh.Ne), "Jinv": mesh.Jinv,
            "rho_ref": np.full(mesh.M, 1.1), "rhotheta_ref": np.full(mesh.M, 340.0)}
    prob.update(c.as_dict())
    return prob, q


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N,shape", [(2, (3, 2, 2)), (4, (3, 2, 1)), (7, (4, 3, 2)), (11, (2, 2, 1))])
def test_free_stream_on_warped_elements(precision, N, shape):
    prob, q = free_stream_problem(N, shape)
    B = np.max(oracle.vol_rhs_abs(prob, q), axis=1)
    s = np.max(np.sum(np.abs(oracle.diff_matrix(N)), axis=1))
    u = 2.0 ** -24 if precision == "mixed" else 2.0 ** -53
    if precision == "mixed":
        state = np.stack([q[0] - prob["rho_ref"], q[1], q[2], q[3], q[4] - prob["rhotheta_ref"]])
        state = state.astype(np.float32)
    else:
        state = q
    with VolumeTerm.from_problem(prob, precision=precision) as vt:
        rhs = vt.rhs(torch.from_numpy(np.ascontiguousarray(state)).cuda()).cpu().numpy()
    worst = np.max(np.abs(rhs.astype(np.float64)), axis=1)
    assert np.all(worst <= s * s * u * B), (worst / B, s * s * u)
