// GLL points and the GLL differentiation matrix, on the host.
//
// D is "the element differentiation matrix" of Sec. 2, Eq. (2): D[i][n] is the
// derivative of the n-th Lagrange polynomial through the Gauss-Lobatto-Legendre
// points, evaluated at point i.
//
// Points: -1, +1 and the roots of P_N', found by Newton's method on P_N' with
// P_N'' taken from Legendre's equation (1 - x^2) P'' = 2x P' - N(N+1) P.
// Off-diagonal entries use the closed form for GLL points,
//   D[i][n] = P_N(x_i) / (P_N(x_n) (x_i - x_n)),
// and the diagonal is set to minus the off-diagonal row sum, so that D maps
// constants to zero as exactly as rounding allows.
#include <cmath>

#include "numa_internal.h"

namespace numa {

namespace {

// P_N(x) and P_N'(x) by the three-term recurrence and the derivative identity.
void legendre(int N, long double x, long double *P, long double *dP) {
    long double p0 = 1.0L, p1 = x;
    if (N == 0) {
        *P = 1.0L;
        *dP = 0.0L;
        return;
    }
    for (int m = 2; m <= N; ++m) {
        long double p2 = ((2 * m - 1) * x * p1 - (m - 1) * p0) / m;
        p0 = p1;
        p1 = p2;
    }
    *P = p1;
    // P_N' = N (P_{N-1} - x P_N) / (1 - x^2), valid in the interior.
    *dP = N * (p0 - x * p1) / (1.0L - x * x);
}

}  // namespace

int gll_diff_matrix(int N, double *D) {
    if (N < 1 || N > NUMA_MAX_N_FP64 || !D) return NUMA_EINVAL;
    const int Nq = N + 1;
    long double x[NUMA_MAX_N_FP64 + 1], PN[NUMA_MAX_N_FP64 + 1];
    const long double pi = 3.141592653589793238462643383279502884L;
    x[0] = -1.0L;
    x[N] = 1.0L;
    for (int i = 1; i < N; ++i) {
        long double xi = -std::cos(pi * i / N);
        for (int it = 0; it < 60; ++it) {
            long double P, dP;
            legendre(N, xi, &P, &dP);
            long double d2P = (2.0L * xi * dP - N * (N + 1.0L) * P) / (1.0L - xi * xi);
            long double step = dP / d2P;
            xi -= step;
            if (std::fabs(step) < 1e-19L) break;
        }
        x[i] = xi;
    }
    for (int i = 0; i < Nq; ++i) {
        long double dP;
        legendre(N, x[i], &PN[i], &dP);
    }
    for (int i = 0; i < Nq; ++i) {
        long double diag = 0.0L;
        for (int n = 0; n < Nq; ++n) {
            if (n == i) continue;
            D[i * Nq + n] = static_cast<double>(PN[i] / (PN[n] * (x[i] - x[n])));
            diag -= D[i * Nq + n];   // minus the sum of the rounded entries
        }
        D[i * Nq + i] = static_cast<double>(diag);
    }
    return NUMA_OK;
}

void sweep_tables(int N, const double *D, double De[16], double Do[16], double Dc[4],
                  double Dcr[4]) {
    for (int t = 0; t < 16; ++t) De[t] = Do[t] = 0.0;
    for (int t = 0; t < 4; ++t) Dc[t] = Dcr[t] = 0.0;
    const int Nq = N + 1, half = Nq / 2, ctr = Nq / 2;
    for (int r = 0; r < half; ++r) {
        for (int m = 0; m < half; ++m) {
            const long double a = D[r * Nq + m], b = D[r * Nq + (Nq - 1 - m)];
            De[r * half + m] = static_cast<double>((a + b) / 2);
            Do[r * half + m] = static_cast<double>((a - b) / 2);
        }
        if (Nq & 1) {
            Dc[r] = D[r * Nq + ctr];
            Dcr[r] = D[ctr * Nq + r];
        }
    }
}

}  // namespace numa
