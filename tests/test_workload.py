"""The seeded input generator (no GPU): the time-integration workloads' smooth
velocity field, against the rough per-point field of the single-evaluation
workloads."""
import numpy as np

import oracle
from paper_1604_08501_gb300 import workload as wl


def test_smooth_velocities_leave_rho_and_theta_and_peak_at_vmax():
    rough = wl.make_workload(3, 3, seed=5)
    smooth = wl.integration_workload(3, 3, 5)
    assert np.array_equal(rough.q[0], smooth.q[0])          # same rho and Theta draws
    assert np.array_equal(rough.q[4], smooth.q[4])
    u = smooth.q[1:4] / smooth.q[0]
    assert np.allclose(np.max(np.abs(u), axis=1), 10.0, rtol=1e-12)   # peak |u_a| = vmax
    # smooth: neighbouring points differ by far less than the rough field's
    assert np.median(np.abs(np.diff(u, axis=1))) < 0.1 * np.median(np.abs(np.diff(rough.q[1:4] / rough.q[0], axis=1)))


def test_integration_states_stay_physical_where_rough_ones_do_not():
    # One element of the finest batch mesh (N = 7, 31^3 elements of 323 m),
    # 20 steps at dt = 0.01 s with the oracle's integrator: the smooth state
    # stays near the reference, the rough one loses positive density.
    n3 = 512
    for make, physical in ((wl.integration_workload, True),
                           (lambda N, n, s: wl.make_workload(N, n, seed=s), False)):
        w = make(7, 31, 107)
        sl = slice(6709 * n3, 6710 * n3)
        prob = dict(w.problem(), Ne=1, g=np.ascontiguousarray(w.mesh.g[:, sl]),
                    Jinv=w.mesh.Jinv[sl], rho_ref=w.rho_ref[sl], rhotheta_ref=w.rhotheta_ref[sl])
        q = oracle.lsrk(prob, np.ascontiguousarray(w.q[:, sl]), 0.01, 20)
        ok = bool(np.all(np.isfinite(q)) and np.all(q[0] > 0.5 * prob["rho_ref"]))
        assert ok == physical
