"""Pins for the oracle's low-storage Runge-Kutta integrator.

The coefficients are checked against the order conditions of Runge-Kutta
methods up to order 4 through their Butcher tableau.  The integrator is checked
by its observed order of convergence on y' = lam y.  Neither test re-types the
oracle's update formula.
"""
import numpy as np
import pytest

import oracle
from paper_1604_08501_gb300 import workload as wl


def butcher_from_2n(A, B):
    """Butcher tableau (a, b, c) of a 2N-storage scheme:
    dq_s = A_s dq_{s-1} + dt f(y_{s-1}),  y_s = y_{s-1} + B_s dq_s."""
    s = len(A)
    # Express dq_j and y_j as combinations of the stage derivatives k_0..k_{s-1}
    # (k_i = f at the argument of stage i), in units of dt.
    dq = np.zeros((s, s))
    y = np.zeros((s + 1, s))
    for j in range(s):
        prev = dq[j - 1] if j > 0 else np.zeros(s)
        dq[j] = A[j] * prev
        dq[j, j] += 1.0
        y[j + 1] = y[j] + B[j] * dq[j]
    a = y[:s]          # stage j is evaluated at y_j = y0 + dt sum_i a[j, i] k_i
    b = y[s]
    c = a.sum(axis=1)
    return a, b, c


def test_coefficients_satisfy_fourth_order_conditions():
    A, B, C = oracle.lsrk_coefficients()
    assert A[0] == 0.0
    a, b, c = butcher_from_2n(A, B)
    assert np.allclose(np.triu(a), 0.0)                   # explicit
    np.testing.assert_allclose(c, C, atol=1e-15)          # published stage times
    conds = {
        "b.1 = 1": (b.sum(), 1.0),
        "b.c = 1/2": (b @ c, 1 / 2),
        "b.c^2 = 1/3": (b @ c ** 2, 1 / 3),
        "b.a.c = 1/6": (b @ a @ c, 1 / 6),
        "b.c^3 = 1/4": (b @ c ** 3, 1 / 4),
        "b.(c*a.c) = 1/8": (b @ (c * (a @ c)), 1 / 8),
        "b.a.c^2 = 1/12": (b @ a @ c ** 2, 1 / 12),
        "b.a.a.c = 1/24": (b @ a @ a @ c, 1 / 24),
    }
    for name, (got, want) in conds.items():
        assert abs(got - want) < 1e-14, (name, got, want)


def test_scalar_convergence_is_fourth_order():
    lam, T = -1.3, 1.0
    errs = []
    for n in (10, 20, 40, 80):
        y = oracle.lsrk_scalar(lam, 1.0, T / n, n)
        errs.append(abs(y - np.exp(lam * T)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8) and np.all(rates < 4.4), rates


def test_lsrk_zero_steps_and_steady_state():
    w = wl.make_workload(3, 2, seed=4)
    prob = w.problem()
    assert np.array_equal(oracle.lsrk(prob, w.q, 0.01, 0), w.q)
    # the unperturbed hydrostatic state is a steady state of the volume term
    q = np.zeros_like(w.q)
    q[0], q[4] = w.rho_ref, w.rhotheta_ref
    assert np.array_equal(oracle.lsrk(prob, q, 0.01, 3), q)


def test_lsrk_one_step_matches_explicit_stages():
    # A single step from the stage definitions, with the oracle's volume term.
    w = wl.make_workload(2, 1, seed=6)
    prob = w.problem()
    A, B, _ = oracle.lsrk_coefficients()
    dt = 1e-3
    q = w.q.copy()
    dq = np.zeros_like(q)
    for s in range(5):
        dq = A[s] * dq + dt * oracle.vol_rhs_o2(prob, q)
        q = q + B[s] * dq
    np.testing.assert_allclose(oracle.lsrk(prob, w.q, dt, 1), q, rtol=1e-14, atol=0)


@pytest.mark.parametrize("N,T", [(2, 2.0), (4, 0.4)])
def test_lsrk_converges_at_fourth_order_on_the_volume_term(N, T):
    # Self-convergence of the integrator on the (nonlinear) semi-discrete
    # system of one 10 km element, against a 64-step reference.
    w = wl.make_workload(N, 1, seed=8)
    prob = w.problem()
    sols = {n: oracle.lsrk(prob, w.q, T / n, n) for n in (4, 8, 16, 64)}
    scale = np.abs(sols[64]).max(axis=1, keepdims=True)
    errs = [np.max(np.abs(sols[n] - sols[64]) / scale) for n in (4, 8, 16)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7) and np.all(rates < 4.4), (errs, rates)
