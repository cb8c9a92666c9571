"""Planted mistakes in the oracle, on the CPU: each mutation of
``oracle/numa_oracle.c`` is compiled to a temporary library, and the pins of
``test_oracle_pins.py`` must fail for it.  This shows that the pins constrain
every part of the oracle's arithmetic (signs, indices, operands, terms)."""
import os
import subprocess

import pytest

import oracle
import test_oracle_lsrk as lsrk_pins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "numa_oracle.c")

# (name, text in the oracle source, replacement, occurrence to change: None = all)
MUTATIONS = [
    ("O2 sign of the volume term", "double v = -P->Jinv[node] * s;", "double v = P->Jinv[node] * s;", 0),
    ("O1 sign of the increment", "rhs[b * M + node] - JiD * F[b]", "rhs[b * M + node] + JiD * F[b]", None),
    ("O2 D transposed in the r sweep", "P->D[i * Nq + n] * Fr", "P->D[n * Nq + i] * Fr", None),
    ("O2 D transposed in the t sweep", "P->D[k * Nq + n] * Ft", "P->D[n * Nq + k] * Ft", None),
    ("metric slots transposed",
     "double g1 = P->g[3 * d + 0][m], g2 = P->g[3 * d + 1][m], g3 = P->g[3 * d + 2][m];",
     "double g1 = P->g[d][m], g2 = P->g[3 + d][m], g3 = P->g[6 + d][m];", None),
    ("pressure term dropped from U1 flux", "F[1] = U1 * u + g1 * pp;", "F[1] = U1 * u;", None),
    ("pressure term on the wrong metric", "F[3] = U3 * u + g3 * pp;", "F[3] = U3 * u + g2 * pp;", None),
    ("reference pressure not subtracted",
     "- oracle_pressure(P->rhotheta_ref[m], P->p0, P->R, P->cp);", ";", None),
    ("gamma = cp / R", "double gamma = cp / (cp - R);", "double gamma = cp / R;", None),
    ("mass flux U instead of rho u", "F[0] = rho * u;", "F[0] = u;", None),
    ("Theta flux with rho", "F[4] = Th * u;", "F[4] = rho * u;", None),
    ("velocity divided by Theta", "+ g3 * U3) / rho;", "+ g3 * U3) / Th;", None),
    ("O2 gravity on the wrong field", "if (b == 3)\n                                    v = v -",
     "if (b == 2)\n                                    v = v -", None),
    ("O2 gravity sign", "v = v - (q[0 * M + node] - P->rho_ref[node]) * P->grav;",
     "v = v + (q[0 * M + node] - P->rho_ref[node]) * P->grav;", None),
    ("O2 s sweep dropped", "s += P->D[j * Nq + n] * Fs[(k * Nq + n) * Nq + i];", ";", None),
    ("O2 t sweep along the wrong index", "Ft[(n * Nq + j) * Nq + i]", "Ft[(n * Nq + i) * Nq + j]", None),
    ("O1 Jinv taken at the line point", "double JiD = P->Jinv[node] * P->D[iota * Nq + n];",
     "double JiD = P->Jinv[m] * P->D[iota * Nq + n];", None),
    ("O1 s line runs along i", "else if (d == 1) { m = ((e * Nq + k) * Nq + n) * Nq + i; iota = j; }",
     "else if (d == 1) { m = ((e * Nq + k) * Nq + j) * Nq + n; iota = j; }", None),
    ("D diagonal sign", "if (m != n) v += 1.0L /", "if (m != n) v -= 1.0L /", None),
    ("GLL Newton step sign", "x -= dx;", "x += dx;", None),
    ("pointwise evaluator drops Jinv", "double v = -P->Jinv[node] * s[b];", "double v = -s[b];", None),
    ("LSRK A coefficient digit", "-2404267990393.0 / 2016746695238.0", "-2404267990393.0 / 2016746695239.0", None),
    ("LSRK B coefficient sign", "    5161836677717.0 / 13612068292357.0", "    -5161836677717.0 / 13612068292357.0", None),
    ("LSRK stage update order", "q[m] = q[m] + LSRK_B[s] * dq[m];", "q[m] = q[m] + LSRK_A[s] * dq[m];", None),
    ("LSRK register not carried", "dq[m] = LSRK_A[s] * dq[m] + dt * rhs[m];", "dq[m] = dt * rhs[m];", None),
]

PIN_CHECKS = [
    lambda: pins.test_gll_closed_forms(),
    lambda: pins.test_diff_matrix_closed_forms(),
    lambda: [pins.test_diff_matrix_exact_on_polynomials(N) for N in (1, 4, 7)],
    lambda: [pins.test_zero_perturbation_is_exactly_zero(N) for N in (1, 4)],
    lambda: [pins.test_free_stream_affine(N) for N in (1, 5)],
    lambda: [pins.test_free_stream_warped_with_curl_form_metrics(N) for N in (2, 4)],
    lambda: [pins.test_manufactured_linear_velocity(N) for N in (2, 4)],
    lambda: [pins.test_manufactured_linear_pressure_and_gravity(N) for N in (1, 4)],
    lambda: pins.test_paper_units_by_hand_n1(),
    lambda: [pins.test_forms_agree_on_warped_mesh(N, 2) for N in (2, 4)],
    lambda: pins.test_element_independence(),
    lambda: pins.test_axis_permutation_symmetry(2),
    lambda: lsrk_pins.test_coefficients_satisfy_fourth_order_conditions(),
    lambda: lsrk_pins.test_scalar_convergence_is_fourth_order(),
    lambda: lsrk_pins.test_lsrk_one_step_matches_explicit_stages(),
    lambda: lsrk_pins.test_lsrk_converges_at_fourth_order_on_the_volume_term(2, 2.0),
]


def _build_variant(tmp_path, old, new, which):
    src = open(SRC).read()
    assert old in src, f"mutation anchor not found: {old!r}"
    if which is None:
        src = src.replace(old, new)
    else:
        parts = src.split(old)
        src = old.join(parts[:which + 1]) + new + old.join(parts[which + 1:])
    c = tmp_path / "mut.c"
    c.write_text(src)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    str(c), "-o", str(so), "-lm"], check=True, capture_output=True)
    return str(so)


def test_unmutated_source_passes_every_check(tmp_path):
    so = _build_variant(tmp_path, "int oracle_max_threads(void)", "int oracle_max_threads(void)", None)
    with oracle.variant(so):
        for check in PIN_CHECKS:
            check()


@pytest.mark.parametrize("name,old,new,which", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, which):
    so = _build_variant(tmp_path, old, new, which)
    caught = []
    with oracle.variant(so):
        for idx, check in enumerate(PIN_CHECKS):
            try:
                check()
            except (AssertionError, ValueError, RuntimeError, FloatingPointError):
                caught.append(idx)
    assert caught, f"no pin caught the planted mistake: {name}"
