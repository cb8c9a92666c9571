"""Metric terms in Kopriva's conservative curl form, for the free-stream tests.

Kopriva (J. Sci. Comput. 26, 2006) writes the contravariant metric terms of a
curvilinear hexahedron as a curl in reference space,

    J a^d_n = -x_d . curl_xi( X_l grad_xi X_m ),   (n, m, l) cyclic,

with every derivative taken by the GLL differentiation matrix applied to the
degree-N interpolant of the coordinates.  Because those derivatives commute
(tensor products of one D along different axes), the discrete metric
identities sum_d D_d (J a^d_n) = 0 then hold to rounding, and a uniform flow
gives a zero flux divergence on curved elements too.  In the library's slot
convention g[3 d + a] = J d(xi_d)/d(x_a) = J a^d_a.

This is test code: it uses the oracle's D and feeds the oracle and the library
the same metric arrays.
"""
import numpy as np

import oracle


def reference_derivative(f, D, axis):
    """Apply D along reference direction `axis` (0: i, 1: j, 2: k) of per-point
    data f shaped (Ne, Nq, Nq, Nq) in [e][k][j][i] order."""
    if axis == 0:
        return np.einsum("in,ekjn->ekji", D, f)
    if axis == 1:
        return np.einsum("jn,ekni->ekji", D, f)
    return np.einsum("kn,enji->ekji", D, f)


def curl_form_metrics(x, N, Ne):
    """(9, M) metric terms g[3 d + a] from the coordinates x (3, M)."""
    Nq = N + 1
    D = oracle.diff_matrix(N)
    X = np.asarray(x, dtype=np.float64).reshape(3, Ne, Nq, Nq, Nq)
    g = np.empty((9, Ne, Nq, Nq, Nq))
    for a in range(3):
        m, l = (a + 1) % 3, (a + 2) % 3
        # F_c = X_l d(X_m)/d(xi_c), c = 0, 1, 2
        F = [X[l] * reference_derivative(X[m], D, c) for c in range(3)]
        curl = (reference_derivative(F[2], D, 1) - reference_derivative(F[1], D, 2),
                reference_derivative(F[0], D, 2) - reference_derivative(F[2], D, 0),
                reference_derivative(F[1], D, 0) - reference_derivative(F[0], D, 1))
        for d in range(3):
            g[3 * d + a] = -curl[d]
    return g.reshape(9, -1)
