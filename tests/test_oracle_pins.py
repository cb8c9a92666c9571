"""Pins for the FP64 CPU oracle: each compares it against something the paper
or the mathematics fixes, never against a retyped copy of its own formula.

* GLL points and D: textbook closed forms for N = 1..4, three independent
  root finders, exact differentiation of polynomials of degree <= N.
* Zero perturbation: the state equals the hydrostatic reference and U = 0,
  so the rhs is exactly zero.
* Free stream on affine meshes: a uniform state gives zero flux divergence;
  on warped meshes the same holds with metrics in Kopriva's conservative
  curl form (tests/curl_metrics.py), and fails with the analytic metrics,
  which do not satisfy the discrete metric identities.
* Manufactured closed forms on a non-orthogonal affine mesh: (i) a linear
  velocity field, (ii) a linear pressure perturbation with gravity.
* The paper's nondimensional constants on one N = 1 element, derived by hand
  (tests/golden/paper_units_n1_by_hand.json).
* Structure: element independence, invariance under a cyclic permutation of
  the axes, and agreement of the three oracle forms (brute force O1, flux
  once per node O2, pointwise).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import workload as wl
from conftest import rel_err

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# GLL points and the differentiation matrix
# --------------------------------------------------------------------------

def test_gll_closed_forms():
    g = load_golden("gll_closed_forms.json")
    for key, pts in g["nodes"].items():
        N = int(key)
        want = np.array([eval(p, {"sqrt": math.sqrt}) for p in pts])
        np.testing.assert_allclose(oracle.gll_nodes(N), want, rtol=0, atol=2e-16)
        np.testing.assert_allclose(wl.gll_points(N), want, rtol=0, atol=4e-16)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_root_finders_agree(N):
    # Newton on x P_N - P_{N-1} (oracle) vs Gauss-Jacobi(1,1) roots (scipy).
    np.testing.assert_allclose(oracle.gll_nodes(N), wl.gll_points(N), rtol=0, atol=3e-16)
    # Interior nodes are roots of P_N' (numpy's Legendre series).
    if N > 1:
        dP = np.polynomial.legendre.Legendre.basis(N).deriv()
        assert np.max(np.abs(dP(oracle.gll_nodes(N)[1:-1]))) < 1e-12


def test_diff_matrix_closed_forms():
    g = load_golden("diff_matrix_closed_forms.json")
    for key, rows in g["D"].items():
        want = np.array([[float(eval(v)) for v in r] for r in rows])
        np.testing.assert_allclose(oracle.diff_matrix(int(key)), want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_diff_matrix_exact_on_polynomials(N):
    # D applied to x^m at the nodes is m x^(m-1), exactly for every m <= N.
    xi = oracle.gll_nodes(N)
    D = oracle.diff_matrix(N)
    for m in range(N + 1):
        f = xi ** m
        df = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        assert np.max(np.abs(D @ f - df)) <= 1e-13 * max(1, m), (N, m)
    # Degree N+1 is not exact.  This rules out a D that is exact only by accident.
    f = xi ** (N + 1)
    assert np.max(np.abs(D @ f - (N + 1) * xi ** N)) > 1e-6
    # Corner entries: D_00 = -N(N+1)/4 = -D_NN.
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-13
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-13


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def problem(mesh, consts, rho_ref, rt_ref):
    d = {"N": mesh.N, "Ne": mesh.Ne, "g": mesh.g, "Jinv": mesh.Jinv,
         "rho_ref": np.ascontiguousarray(np.broadcast_to(rho_ref, (mesh.M,)), dtype=np.float64),
         "rhotheta_ref": np.ascontiguousarray(np.broadcast_to(rt_ref, (mesh.M,)), dtype=np.float64)}
    d.update(consts.as_dict())
    return d


def all_forms(prob, q):
    o1 = oracle.vol_rhs_o1(prob, q)
    o2 = oracle.vol_rhs_o2(prob, q)
    return o1, o2


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 4, 7])
def test_zero_perturbation_is_exactly_zero(N):
    mesh = wl.warped_box(N, (2, 2, 2))
    rho0, rt0 = wl.hydrostatic_reference(mesh.x[2])
    q = np.zeros((5, mesh.M))
    q[0], q[4] = rho0, rt0
    prob = problem(mesh, wl.DRY_AIR, rho0, rt0)
    for out in all_forms(prob, q):
        assert np.all(out == 0.0)


@pytest.mark.parametrize("N", [1, 2, 5, 7])
def test_free_stream_affine(N):
    mesh = wl.affine_box(N, (2, 1, 2), L=3.0)
    c = wl.Constants(p0=1.0e5, R=287.0, cp=1004.0, grav=0.0)
    rho, vel, Th = 1.2, np.array([3.0, -2.0, 5.0]), 350.0
    q = np.empty((5, mesh.M))
    q[0], q[1:4], q[4] = rho, (rho * vel)[:, None], Th
    # reference differs from the state, so p' is a nonzero constant
    prob = problem(mesh, c, 1.1, 340.0)
    pp = oracle.pressure(Th, c.p0, c.R, c.cp) - oracle.pressure(340.0, c.p0, c.R, c.cp)
    # scale: largest single term J^-1 |D| |F|
    F = np.abs(mesh.g).max() * (np.abs(vel).max() * max(rho, Th, rho * np.abs(vel).max()) + abs(pp))
    scale = mesh.Jinv.max() * np.abs(oracle.diff_matrix(N)).sum(axis=1).max() * F
    for out in all_forms(prob, q):
        assert np.max(np.abs(out)) <= 1e-13 * scale


def test_curl_form_metrics_equal_the_analytic_ones_on_affine_meshes():
    from curl_metrics import curl_form_metrics
    for N in (1, 2, 4, 7):
        mesh = wl.warped_box(N, (2, 2, 2), warp=0.0)
        g = curl_form_metrics(mesh.x, N, mesh.Ne)
        assert np.max(np.abs(g - mesh.g)) <= 2e-12 * np.max(np.abs(mesh.g))


@pytest.mark.parametrize("N", [2, 3, 4, 7, 11])
def test_free_stream_warped_with_curl_form_metrics(N):
    # Uniform flow on the warped box: with curl-form metrics the flux
    # divergence vanishes to rounding.  The computed metrics carry rounding of
    # order eps s |g| (one D, s = max row sum of |D|) and the divergence
    # applies D again, so |rhs| <= s^2 eps B with B the running bound
    # J^-1 sum |D| |F|.  The analytic metrics break the discrete metric
    # identities and miss that bound by orders of magnitude (up to N = 11).
    from curl_metrics import curl_form_metrics
    mesh = wl.warped_box(N, (2, 2, 1))
    c = wl.Constants(p0=1.0e5, R=287.0, cp=1004.0, grav=0.0)
    rho, vel, Th = 1.2, np.array([3.0, -2.0, 5.0]), 350.0
    q = np.empty((5, mesh.M))
    q[0], q[1:4], q[4] = rho, (rho * vel)[:, None], Th
    s = np.max(np.sum(np.abs(oracle.diff_matrix(N)), axis=1))
    prob = problem(mesh, c, 1.1, 340.0)
    prob["g"] = curl_form_metrics(mesh.x, N, mesh.Ne)
    B = np.max(oracle.vol_rhs_abs(prob, q), axis=1)
    for out in all_forms(prob, q):
        assert np.all(np.max(np.abs(out), axis=1) <= s * s * 2.0 ** -53 * B)
    analytic = problem(mesh, c, 1.1, 340.0)
    out = oracle.vol_rhs_o2(analytic, q)
    Ba = np.max(oracle.vol_rhs_abs(analytic, q), axis=1)
    assert np.max(np.abs(out)[0]) > 100 * s * s * 2.0 ** -53 * Ba[0]


def _manufactured_linear_velocity(N):
    mesh = wl.affine_box(N, (2, 2, 2), L=2.0)
    c = wl.Constants(p0=1.0e5, R=287.17, cp=1004.67, grav=9.81)
    rho_c, Th_c = 1.3, 300.0
    alpha = np.array([1.0, -2.0, 0.5])
    beta = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.6, 0.8, 0.25]])
    u = alpha[:, None] + beta @ mesh.x
    q = np.empty((5, mesh.M))
    q[0], q[1:4], q[4] = rho_c, rho_c * u, Th_c
    prob = problem(mesh, c, rho_c, Th_c)
    trb = np.trace(beta)
    want = np.empty_like(q)
    want[0] = -rho_c * trb
    want[1:4] = -rho_c * (trb * u + beta @ u)
    want[4] = -Th_c * trb
    return prob, q, want


@pytest.mark.parametrize("N", range(2, 8))
def test_manufactured_linear_velocity(N):
    # rho, Theta constant, U = rho (alpha + beta x), Theta = Theta_ref: every flux
    # is a polynomial of degree <= 2 in xi on an affine element, so the discrete
    # volume term equals -div(u q_b) exactly (up to rounding).
    prob, q, want = _manufactured_linear_velocity(N)
    for out in all_forms(prob, q):
        for b, (mx, rms) in enumerate(rel_err(out, want)):
            assert mx < 1e-12, (N, b, mx)


def _manufactured_linear_pressure(N, consts):
    mesh = wl.affine_box(N, (2, 2, 1), L=1.5)
    Th_r, delta = 2.0, 0.05
    pi0, pi = 0.3, np.array([0.2, -0.15, 0.35])
    # Theta with p(Theta) - p(Theta_r) = pi0 + pi . x, from the equation of state
    # p = p0 (R Theta / p0)^gamma with gamma = cp / (cp - R) (Sec. 2).
    gamma = consts.cp / (consts.cp - consts.R)
    p_r = consts.p0 * (consts.R * Th_r / consts.p0) ** gamma
    pL = pi0 + pi @ mesh.x
    Th = consts.p0 / consts.R * ((p_r + pL) / consts.p0) ** (1.0 / gamma)
    rho = 1.0 + 0.1 * mesh.x[0]           # any density: U = 0 makes it flux-free
    q = np.zeros((5, mesh.M))
    q[0], q[4] = rho, Th
    prob = problem(mesh, consts, rho - delta, Th_r)
    want = np.zeros_like(q)
    want[1:4] = -pi[:, None]
    want[3] -= delta * consts.grav        # gravity: -(rho - rho_ref) g on U3 only
    return prob, q, want


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_manufactured_linear_pressure_and_gravity(N):
    c = wl.Constants(p0=1.0, R=1.0, cp=3.5, grav=2.5)   # the paper's p0, R, gamma=1.4
    prob, q, want = _manufactured_linear_pressure(N, c)
    for out in all_forms(prob, q):
        assert np.all(out[0] == 0) and np.all(out[4] == 0)
        for b in (1, 2, 3):
            err = np.max(np.abs(out[b] - want[b])) / np.max(np.abs(want[b]))
            assert err < 1e-12, (N, b, err)


def test_paper_units_by_hand_n1():
    # One N=1 element equal to the reference cube (g = I, J = 1), the paper's
    # constants p0 = 1, R = 1, gamma = 1.4, its full pressure (Theta_ref = 0)
    # and no gravity.  Expected values derived by hand in the fixture.
    gold = load_golden("paper_units_n1_by_hand.json")
    mesh = wl.affine_box(1, (1, 1, 1), L=2.0, B=np.eye(3))
    assert np.allclose(mesh.Jinv, 1.0) and np.allclose(mesh.g, np.repeat(np.eye(3).reshape(9, 1), 8, 1))
    q = np.zeros((5, 8))
    for node in range(8):
        i, j, k = node % 2, (node // 2) % 2, node // 4
        s = gold["state"]
        env = {"i": i, "j": j, "k": k}
        q[:, node] = [eval(s[f], env) for f in ("rho", "U1", "U2", "U3", "Theta")]
    prob = problem(mesh, wl.PAPER_UNITS, 0.0, 0.0)
    for out in all_forms(prob, q):
        for node in range(8):
            i, j, k = node % 2, (node // 2) % 2, node // 4
            env = {"i": i, "j": j, "k": k}
            for b, f in enumerate(("rho", "U1", "U2", "U3", "Theta")):
                want = eval(gold["rhs"][f], env)
                assert abs(out[b, node] - want) < 1e-15, (f, node, out[b, node], want)


def test_error_bound_by_hand_and_triangle_inequality():
    # By hand (the N=1 paper-units case): only the r-direction carries rho and
    # Theta fluxes, so the bound is (|F(0)| + |F(1)|)/2 = |rhs| there; U2 has
    # F_s[U2] = p on both points of each s-line, bound (p + p)/2 = p(k).
    gold = load_golden("paper_units_n1_by_hand.json")
    mesh = wl.affine_box(1, (1, 1, 1), L=2.0, B=np.eye(3))
    q = np.zeros((5, 8))
    for node in range(8):
        env = {"i": node % 2, "j": (node // 2) % 2, "k": node // 4}
        q[:, node] = [eval(gold["state"][f], env) for f in ("rho", "U1", "U2", "U3", "Theta")]
    prob = problem(mesh, wl.PAPER_UNITS, 0.0, 0.0)
    ab = oracle.vol_rhs_abs(prob, q)
    rhs = oracle.vol_rhs_o2(prob, q)
    np.testing.assert_allclose(ab[0], np.abs(rhs[0]), rtol=1e-15)
    np.testing.assert_allclose(ab[4], np.abs(rhs[4]), rtol=1e-15)
    p = np.where(np.arange(8) // 4 == 0, 1.0, 2.0 ** 1.4)
    np.testing.assert_allclose(ab[2], p, rtol=1e-15)
    # triangle inequality on a warped workload
    w = wl.make_workload(4, 2, seed=2)
    ab = oracle.vol_rhs_abs(w.problem(), w.q)
    rhs = oracle.vol_rhs_o2(w.problem(), w.q)
    assert np.all(ab >= np.abs(rhs) * (1 - 1e-14))


# --------------------------------------------------------------------------
# Structure
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", list(range(1, 8)) + [11, 15])
@pytest.mark.parametrize("n", [1, 2])
def test_forms_agree_on_warped_mesh(N, n):
    w = wl.make_workload(N, n, seed=7 + N)
    prob = w.problem()
    o1, o2 = all_forms(prob, w.q)
    for b, (mx, rms) in enumerate(rel_err(o1, o2)):
        assert mx < 1e-14, (N, b, mx)
    rng = np.random.default_rng(N)
    ids = rng.choice(w.M, size=min(w.M, 50), replace=False)
    pts = oracle.vol_rhs_points(prob, w.q, ids)
    assert np.max(np.abs(pts - o2[:, ids])) <= 1e-14 * np.max(np.abs(o2), axis=1).max()


def test_element_independence():
    w = wl.make_workload(3, 2, seed=3)
    prob = w.problem()
    base = oracle.vol_rhs_o2(prob, w.q)
    n3 = 4 ** 3
    e = 5
    q2 = w.q.copy()
    q2[:, e * n3:(e + 1) * n3] *= 1.0 + 1e-3 * np.arange(1, 6)[:, None]
    out = oracle.vol_rhs_o2(prob, q2)
    changed = np.any(out != base, axis=0).reshape(w.Ne, n3)
    assert changed[e].all()
    assert not np.delete(changed, e, axis=0).any()


def _cyclic_permutation(N, mesh, prob, q):
    """New point (i', j', k') = (k, i, j) and new axis sigma(a) = a + 1 mod 3."""
    Nq = N + 1

    def perm_scalar(a):
        a = a.reshape(mesh.Ne, Nq, Nq, Nq)          # [e][k][j][i]
        # new[e][k'][j'][i'] = old[e][k=i'][j=k'][i=j']
        return np.ascontiguousarray(np.transpose(a, (0, 2, 3, 1))).reshape(-1)

    sig = [1, 2, 0]
    g2 = np.empty_like(prob["g"])
    for d in range(3):
        for a in range(3):
            g2[3 * sig[d] + sig[a]] = perm_scalar(prob["g"][3 * d + a])
    q2 = np.empty_like(q)
    q2[0], q2[4] = perm_scalar(q[0]), perm_scalar(q[4])
    for a in range(3):
        q2[1 + sig[a]] = perm_scalar(q[1 + a])
    p2 = dict(prob, g=g2, Jinv=perm_scalar(prob["Jinv"]),
              rho_ref=perm_scalar(prob["rho_ref"]), rhotheta_ref=perm_scalar(prob["rhotheta_ref"]))
    return p2, q2, perm_scalar, sig


@pytest.mark.parametrize("N", [2, 5])
def test_axis_permutation_symmetry(N):
    w = wl.make_workload(N, 2, seed=11)
    prob = dict(w.problem(), grav=0.0)
    base = oracle.vol_rhs_o2(prob, w.q)
    p2, q2, perm, sig = _cyclic_permutation(N, w.mesh, prob, w.q)
    out = oracle.vol_rhs_o2(p2, q2)
    want = np.empty_like(base)
    want[0], want[4] = perm(base[0]), perm(base[4])
    for a in range(3):
        want[1 + sig[a]] = perm(base[1 + a])
    for b, (mx, rms) in enumerate(rel_err(out, want)):
        assert mx < 1e-13, (b, mx)


def test_workload_statistics():
    # The seeded workload has the stated structure: perturbations of order 1e-3
    # about the hydrostatic reference, velocities within (-10, 10) m/s.
    w = wl.make_workload(4, 3, seed=0)
    rel_rho = w.q[0] / w.rho_ref - 1
    assert 1e-5 < np.max(np.abs(rel_rho)) < 4e-3
    u = w.q[1:4] / w.q[0]
    assert np.max(np.abs(u)) < 10 and np.max(np.abs(u)) > 9
    assert np.all(w.mesh.Jinv > 0)
    # Same seed, same inputs; another seed, other inputs.
    assert np.array_equal(wl.make_workload(4, 3, seed=0).q, w.q)
    assert not np.array_equal(wl.make_workload(4, 3, seed=1).q, w.q)


# --------------------------------------------------------------------------
# Passive tracers (the paper's 8-field form: Q1..Q3 after Theta, Sec. 2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 4])
def test_tracers_leave_the_five_fields_unchanged(N):
    # Tracers are passive: adding them changes no bit of the other fields.
    w5 = wl.make_workload(N, 2, seed=31)
    w8 = wl.make_workload(N, 2, seed=31, tracers=3)
    r5 = oracle.vol_rhs_o2(w5.problem(), w5.q)
    r8 = oracle.vol_rhs_o2(w8.problem(), w8.q)
    assert r8.shape == (8, w8.M)
    assert np.array_equal(r8[:5], r5)


def test_tracer_copies_of_theta_and_of_a_mixing_ratio_times_rho():
    # A tracer equal to Theta is advected exactly like Theta: identical flux,
    # identical rhs bits.  A tracer c * rho (constant mixing ratio) has rhs
    # c * rhs_rho, the mass equation scaled (to rounding).
    w = wl.make_workload(3, (3, 2, 1), seed=32, tracers=3)
    q = w.q.copy()
    q[5] = q[4]
    q[6] = 0.25 * q[0]
    q[7] = 0.0
    prob = w.problem()
    for rhs in (oracle.vol_rhs_o2(prob, q), oracle.vol_rhs_o1(prob, q)):
        assert np.array_equal(rhs[5], rhs[4])
        np.testing.assert_allclose(rhs[6], 0.25 * rhs[0], rtol=0,
                                   atol=1e-14 * np.max(np.abs(rhs[0])))
        assert not np.any(rhs[7])


def test_tracer_forms_agree_and_pointwise():
    w = wl.make_workload(4, 2, seed=33, tracers=2)
    prob = w.problem()
    o1, o2 = oracle.vol_rhs_o1(prob, w.q), oracle.vol_rhs_o2(prob, w.q)
    assert o1.shape == (7, w.M)
    for f in range(7):
        assert np.max(np.abs(o1[f] - o2[f])) < 1e-14 * np.max(np.abs(o2[f])), f
    ids = np.random.default_rng(3).choice(w.M, size=60, replace=False)
    pts = oracle.vol_rhs_points(prob, w.q, ids)
    assert np.max(np.abs(pts - o2[:, ids])) <= 1e-14 * np.max(np.abs(o2))
