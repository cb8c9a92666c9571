/*
 * Oracle for the strong-form element volume term of a NUMA-style dry
 * compressible Euler model on hexahedral GLL spectral elements
 * (Kloeckner, Wilcox, Warburton, "Array Program Transformation with Loo.py by
 * Example: High-Order Finite Elements", ARRAY'16).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 CPU statement
 * of what the GPU path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant table with the CUDA library, and it includes nothing from it.
 *
 * Compiled with -ffp-contract=off so that every operation rounds as written.
 *
 * What it computes (Sec. 2, Eq. (2) "volterm", with the sign of the r- and
 * s-flux subroutines refFluxR / refFluxS of Sec. 3, which subtract
 * Jinv * D * flux from rhsq):
 *
 *   v_b(e,i,j,k) = - Jinv(e,i,j,k) * sum_{d in r,s,t} sum_n D[iota_d][n]
 *                    * F_d[b] at the node whose d-th index is replaced by n
 *                  - delta_{b,U3} * (rho - rho_ref) * grav
 *
 * with the contravariant flux of Sec. 2, Eq. (1) (flux column f_a) contracted
 * with the metric terms g_{a,d} exactly as refFluxR / refFluxS do:
 *
 *   u_d      = (g_{1d} U1 + g_{2d} U2 + g_{3d} U3) / rho
 *   F_d[rho] = rho * u_d
 *   F_d[U_a] = U_a * u_d + g_{ad} * p'
 *   F_d[Th]  = Th * u_d
 *
 * and the equation of state of Sec. 2, p(Th) = p0 (R Th / p0)^gamma with
 * gamma = cp / cv, cv = cp - R, applied as a perturbation
 * p' = p(Th) - p(Th_ref).  The reference-state pressure subtraction and the
 * gravity source are additions to the paper's gravity-free form; setting
 * rhotheta_ref = 0, rho_ref = 0 and grav = 0 recovers the paper's form
 * exactly (p(0) = 0).
 *
 * Layouts: every per-node array is [e][k][j][i] with i fastest (the paper's
 * Fortran q(i,j,k,field,e) order); the five fields are planes of length
 * Ne*Nq^3 in the order (rho, U1, U2, U3, Theta); D is row-major, D[i*Nq+n]
 * (the paper's D(i,n)); metric slot g[3*d+a] holds g_{a+1,d+1} (the paper's
 * geo slots 1-3 for r and 4-6 for s, a fastest; slots 7-9 for t).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXFIELDS 8   /* rho, U1, U2, U3, Theta and up to three tracers */
#define ORACLE_MAXNQ 16

typedef struct {
    int N;                     /* polynomial order; Nq = N + 1 points per axis */
    int64_t Ne;                /* number of elements                           */
    const double *D;           /* Nq x Nq differentiation matrix, D[i*Nq+n]    */
    const double *g[9];        /* metric terms, g[3*d+a] = g_{a+1,d+1}          */
    const double *Jinv;        /* 1 / J per node                                */
    const double *rho_ref;     /* reference density per node                    */
    const double *rhotheta_ref;/* reference Theta = rho*theta per node          */
    double p0, R, cp, grav;    /* EOS constants and gravitational acceleration  */
    int ntracers;              /* passive tracers Q1..Q3 after Theta (0..3)     */
} oracle_problem;

#define NF(P) (5 + (P)->ntracers)   /* fields of the state */

/* ------------------------------------------------------------------------- */
/* GLL nodes and the differentiation matrix (inputs of Eq. (2): "D is the    */
/* element differentiation matrix").                                          */
/* ------------------------------------------------------------------------- */

/* Legendre P_N and P_{N-1} at x by the three-term recurrence. */
static void legendre_pair(int N, long double x, long double *pN, long double *pNm1)
{
    long double pm1 = 1.0L, p = x;
    if (N == 0) { *pN = 1.0L; *pNm1 = 0.0L; return; }
    for (int m = 1; m < N; ++m) {
        long double pn = ((2.0L * m + 1.0L) * x * p - m * pm1) / (m + 1.0L);
        pm1 = p;
        p = pn;
    }
    *pN = p;
    *pNm1 = pm1;
}

/*
 * Gauss-Lobatto-Legendre nodes: -1, +1 and the N-1 roots of P_N'.  Interior
 * roots are the zeros of x P_N(x) - P_{N-1}(x) (which is proportional to
 * (1 - x^2) P_N'(x) / N); each is found by Newton's method from the
 * Chebyshev-Gauss-Lobatto guess, using d/dx [x P_N - P_{N-1}] = (N+1) P_N.
 * Output in increasing order.  Returns 0, or -1 for N outside [1, 15].
 */
int oracle_gll_nodes(int N, double *xi)
{
    if (N < 1 || N >= ORACLE_MAXNQ) return -1;
    for (int i = 0; i <= N; ++i) {
        long double x = -cosl(3.14159265358979323846264338327950288L * i / N);
        if (i == 0) { xi[i] = -1.0; continue; }
        if (i == N) { xi[i] = 1.0; continue; }
        for (int it = 0; it < 100; ++it) {
            long double pN, pNm1;
            legendre_pair(N, x, &pN, &pNm1);
            long double f = x * pN - pNm1;
            long double dx = f / ((N + 1.0L) * pN);
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        xi[i] = (double)x;
    }
    return 0;
}

/*
 * Differentiation matrix from its definition, D[i][n] = l_n'(xi_i), where
 * l_n is the Lagrange polynomial through the nodes with l_n(xi_m) = delta_nm:
 *   l_n'(xi_i) = prod_{m != n,i} (xi_i - xi_m) / prod_{m != n} (xi_n - xi_m),  i != n
 *   l_n'(xi_n) = sum_{m != n} 1 / (xi_n - xi_m)
 * evaluated in long double.  Returns 0, or -1 for N outside [1, 15].
 */
int oracle_diff_matrix(int N, const double *xi, double *D)
{
    if (N < 1 || N >= ORACLE_MAXNQ) return -1;
    const int Nq = N + 1;
    for (int i = 0; i < Nq; ++i) {
        for (int n = 0; n < Nq; ++n) {
            long double v;
            if (i == n) {
                v = 0.0L;
                for (int m = 0; m < Nq; ++m)
                    if (m != n) v += 1.0L / ((long double)xi[n] - xi[m]);
            } else {
                long double num = 1.0L, den = 1.0L;
                for (int m = 0; m < Nq; ++m) {
                    if (m != n) den *= ((long double)xi[n] - xi[m]);
                    if (m != n && m != i) num *= ((long double)xi[i] - xi[m]);
                }
                v = num / den;
            }
            D[i * Nq + n] = (double)v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Pointwise physics                                                          */
/* ------------------------------------------------------------------------- */

/* Equation of state of Sec. 2: p = p0 (R Theta / p0)^gamma, gamma = cp/(cp-R). */
double oracle_pressure(double Theta, double p0, double R, double cp)
{
    double gamma = cp / (cp - R);
    return p0 * pow(R * Theta / p0, gamma);
}

/* State and contravariant flux of direction d at one node (Eq. (1) flux
 * column f_a contracted with g_{a,d}, as in refFluxR / refFluxS). */
static void node_flux(const oracle_problem *P, const double *q, int64_t M,
                      int64_t m, int d, double F[ORACLE_MAXFIELDS])
{
    double rho = q[0 * M + m];
    double U1 = q[1 * M + m], U2 = q[2 * M + m], U3 = q[3 * M + m];
    double Th = q[4 * M + m];
    double g1 = P->g[3 * d + 0][m], g2 = P->g[3 * d + 1][m], g3 = P->g[3 * d + 2][m];
    double pp = oracle_pressure(Th, P->p0, P->R, P->cp)
              - oracle_pressure(P->rhotheta_ref[m], P->p0, P->R, P->cp);
    double u = (g1 * U1 + g2 * U2 + g3 * U3) / rho;
    F[0] = rho * u;
    F[1] = U1 * u + g1 * pp;
    F[2] = U2 * u + g2 * pp;
    F[3] = U3 * u + g3 * pp;
    F[4] = Th * u;
    /* tracers are advected like Theta: flux Q u, no pressure term (Sec. 2) */
    for (int t = 0; t < P->ntracers; ++t) F[5 + t] = q[(5 + t) * M + m] * u;
}

static int check_problem(const oracle_problem *P)
{
    if (!P || P->N < 1 || P->N >= ORACLE_MAXNQ || P->Ne < 0 || !P->D || !P->Jinv ||
        !P->rho_ref || !P->rhotheta_ref || P->ntracers < 0 || P->ntracers > 3)
        return -1;
    for (int s = 0; s < 9; ++s)
        if (!P->g[s]) return -1;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O1: brute force, one routine per reference direction, shaped like the     */
/* paper's refFluxR / refFluxS: loops e, k, j, i, n; the state, pressure and  */
/* flux at the line node n are recomputed inside the n loop, and each term   */
/* is subtracted as Jinv(i,j,k) * D(iota,n) * flux from rhs.  The t-direction */
/* is the third line of Eq. (2), written the same way.                        */
/* ------------------------------------------------------------------------- */

static void o1_direction(const oracle_problem *P, const double *q, double *rhs, int d)
{
    const int Nq = P->N + 1;
    const int64_t M = P->Ne * Nq * Nq * Nq;
    for (int64_t e = 0; e < P->Ne; ++e)
        for (int k = 0; k < Nq; ++k)
            for (int j = 0; j < Nq; ++j)
                for (int i = 0; i < Nq; ++i)
                    for (int n = 0; n < Nq; ++n) {
                        int64_t node = ((e * Nq + k) * Nq + j) * Nq + i;
                        int64_t m;
                        int iota;
                        if (d == 0) { m = ((e * Nq + k) * Nq + j) * Nq + n; iota = i; }
                        else if (d == 1) { m = ((e * Nq + k) * Nq + n) * Nq + i; iota = j; }
                        else { m = ((e * Nq + n) * Nq + j) * Nq + i; iota = k; }
                        double F[ORACLE_MAXFIELDS];
                        node_flux(P, q, M, m, d, F);
                        double JiD = P->Jinv[node] * P->D[iota * Nq + n];
                        for (int b = 0; b < NF(P); ++b)
                            rhs[b * M + node] = rhs[b * M + node] - JiD * F[b];
                    }
}

int oracle_vol_rhs_o1(const oracle_problem *P, const double *q, double *rhs)
{
    if (check_problem(P) || !q || !rhs) return -1;
    const int Nq = P->N + 1;
    const int64_t M = P->Ne * Nq * Nq * Nq;
    memset(rhs, 0, sizeof(double) * NF(P) * (size_t)M);
    for (int d = 0; d < 3; ++d) o1_direction(P, q, rhs, d);
    for (int64_t m = 0; m < M; ++m)
        rhs[3 * M + m] = rhs[3 * M + m] - (q[0 * M + m] - P->rho_ref[m]) * P->grav;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O2: fluxes once per node, then the three D contractions; Jinv applied     */
/* once to the sum.  Elements are independent (Eq. (2) couples only nodes of */
/* one element), so they are distributed over threads.                        */
/* ------------------------------------------------------------------------- */

int oracle_vol_rhs_o2(const oracle_problem *P, const double *q, double *rhs, int nthreads)
{
    if (check_problem(P) || !q || !rhs) return -1;
    const int Nq = P->N + 1;
    const int n3 = Nq * Nq * Nq;
    const int64_t M = P->Ne * n3;
    int err = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : err)
#endif
    {
        /* F[d][b][node-in-element] */
        double *F = (double *)malloc(sizeof(double) * 3 * NF(P) * (size_t)n3);
        if (!F) {
            err = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int64_t e = 0; e < P->Ne; ++e) {
                for (int l = 0; l < n3; ++l)
                    for (int d = 0; d < 3; ++d) {
                        double Fn[ORACLE_MAXFIELDS];
                        node_flux(P, q, M, e * n3 + l, d, Fn);
                        for (int b = 0; b < NF(P); ++b)
                            F[(d * NF(P) + b) * n3 + l] = Fn[b];
                    }
                for (int k = 0; k < Nq; ++k)
                    for (int j = 0; j < Nq; ++j)
                        for (int i = 0; i < Nq; ++i) {
                            int64_t node = e * n3 + (k * Nq + j) * Nq + i;
                            for (int b = 0; b < NF(P); ++b) {
                                const double *Fr = F + (0 * NF(P) + b) * n3;
                                const double *Fs = F + (1 * NF(P) + b) * n3;
                                const double *Ft = F + (2 * NF(P) + b) * n3;
                                double s = 0.0;
                                for (int n = 0; n < Nq; ++n)
                                    s += P->D[i * Nq + n] * Fr[(k * Nq + j) * Nq + n];
                                for (int n = 0; n < Nq; ++n)
                                    s += P->D[j * Nq + n] * Fs[(k * Nq + n) * Nq + i];
                                for (int n = 0; n < Nq; ++n)
                                    s += P->D[k * Nq + n] * Ft[(n * Nq + j) * Nq + i];
                                double v = -P->Jinv[node] * s;
                                if (b == 3)
                                    v = v - (q[0 * M + node] - P->rho_ref[node]) * P->grav;
                                rhs[b * M + node] = v;
                            }
                        }
            }
            free(F);
        }
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Pointwise: Eq. (2) at selected nodes only, recomputing every flux it      */
/* needs.  Used to check full-size results on a sample of nodes.             */
/* out[b*npts + p] receives field b at node_ids[p].                          */
/* ------------------------------------------------------------------------- */

int oracle_vol_rhs_points(const oracle_problem *P, const double *q, int64_t npts,
                          const int64_t *node_ids, double *out)
{
    if (check_problem(P) || !q || !out || (npts > 0 && !node_ids)) return -1;
    const int Nq = P->N + 1;
    const int64_t n3 = (int64_t)Nq * Nq * Nq;
    const int64_t M = P->Ne * n3;
    for (int64_t p = 0; p < npts; ++p) {
        int64_t node = node_ids[p];
        if (node < 0 || node >= M) return -1;
        int64_t e = node / n3;
        int64_t l = node % n3;
        int i = (int)(l % Nq), j = (int)((l / Nq) % Nq), k = (int)(l / (Nq * Nq));
        double s[ORACLE_MAXFIELDS] = {0};
        for (int d = 0; d < 3; ++d) {
            int iota = d == 0 ? i : (d == 1 ? j : k);
            for (int n = 0; n < Nq; ++n) {
                int64_t m;
                if (d == 0) m = ((e * Nq + k) * Nq + j) * Nq + n;
                else if (d == 1) m = ((e * Nq + k) * Nq + n) * Nq + i;
                else m = ((e * Nq + n) * Nq + j) * Nq + i;
                double F[ORACLE_MAXFIELDS];
                node_flux(P, q, M, m, d, F);
                for (int b = 0; b < NF(P); ++b)
                    s[b] += P->D[iota * Nq + n] * F[b];
            }
        }
        for (int b = 0; b < NF(P); ++b) {
            double v = -P->Jinv[node] * s[b];
            if (b == 3) v = v - (q[0 * M + node] - P->rho_ref[node]) * P->grav;
            out[b * npts + p] = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Running error bound of Eq. (2): the same sums with every term replaced by  */
/* its magnitude, |Jinv| * sum_d sum_n |D| |F_d[b]| (plus |(rho - rho_ref)    */
/* grav| on U3).  The ratio of its maximum to the maximum |rhs_b| is the       */
/* condition number of field b; rounding errors of any evaluation of Eq. (2)   */
/* scale with it.                                                              */
/* ------------------------------------------------------------------------- */

int oracle_vol_rhs_abs(const oracle_problem *P, const double *q, double *out)
{
    if (check_problem(P) || !q || !out) return -1;
    const int Nq = P->N + 1;
    const int64_t n3 = (int64_t)Nq * Nq * Nq;
    const int64_t M = P->Ne * n3;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t node = 0; node < M; ++node) {
        int64_t e = node / n3, l = node % n3;
        int i = (int)(l % Nq), j = (int)((l / Nq) % Nq), k = (int)(l / (Nq * Nq));
        double s[ORACLE_MAXFIELDS] = {0};
        for (int d = 0; d < 3; ++d) {
            int iota = d == 0 ? i : (d == 1 ? j : k);
            for (int n = 0; n < Nq; ++n) {
                int64_t m;
                if (d == 0) m = ((e * Nq + k) * Nq + j) * Nq + n;
                else if (d == 1) m = ((e * Nq + k) * Nq + n) * Nq + i;
                else m = ((e * Nq + n) * Nq + j) * Nq + i;
                double F[ORACLE_MAXFIELDS];
                node_flux(P, q, M, m, d, F);
                for (int b = 0; b < NF(P); ++b)
                    s[b] += fabs(P->D[iota * Nq + n]) * fabs(F[b]);
            }
        }
        for (int b = 0; b < NF(P); ++b) {
            double v = fabs(P->Jinv[node]) * s[b];
            if (b == 3) v = v + fabs((q[0 * M + node] - P->rho_ref[node]) * P->grav);
            out[b * M + node] = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Explicit time integration of dq/dt = v(q) (the volume term alone) by the  */
/* five-stage fourth-order low-storage ("2N-storage") Runge-Kutta scheme of  */
/* Carpenter and Kennedy (NASA TM-109112, 1994).  The paper's Sec. 2 frames  */
/* the volume term as the rate function of an explicit ODE solver; this      */
/* scheme is the benchmark's choice.  Per stage s = 0..4:                    */
/*     dq <- A[s] dq + dt v(q),   q <- q + B[s] dq,                          */
/* with dq = 0 before the first stage of a step.  (C[s], the stage times,    */
/* do not enter an autonomous rate function.)                                */
/* ------------------------------------------------------------------------- */

static const double LSRK_A[5] = {
    0.0,
    -567301805773.0 / 1357537059087.0,
    -2404267990393.0 / 2016746695238.0,
    -3550918686646.0 / 2091501179385.0,
    -1275806237668.0 / 842570457699.0};
static const double LSRK_B[5] = {
    1432997174477.0 / 9575080441755.0,
    5161836677717.0 / 13612068292357.0,
    1720146321549.0 / 2090206949498.0,
    3134564353537.0 / 4481467310338.0,
    2277821191437.0 / 14882151754819.0};
static const double LSRK_C[5] = {
    0.0,
    1432997174477.0 / 9575080441755.0,
    2526269341429.0 / 6820363962896.0,
    2006345519317.0 / 3224310063776.0,
    2802321613138.0 / 2924317926251.0};

/* The scheme's coefficients, for the tests that check its order conditions. */
void oracle_lsrk_coefficients(double *A, double *B, double *C)
{
    for (int s = 0; s < 5; ++s) {
        A[s] = LSRK_A[s];
        B[s] = LSRK_B[s];
        C[s] = LSRK_C[s];
    }
}

/* Advance q by nsteps steps of size dt in place.  Each stage evaluates the
 * volume term with O2. */
int oracle_lsrk(const oracle_problem *P, double *q, double dt, int nsteps, int nthreads)
{
    if (check_problem(P) || !q || nsteps < 0) return -1;
    const int Nq = P->N + 1;
    const size_t n = (size_t)NF(P) * (size_t)(P->Ne * Nq * Nq * Nq);
    double *dq = (double *)calloc(n ? n : 1, sizeof(double));
    double *rhs = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!dq || !rhs) {
        free(dq);
        free(rhs);
        return -2;
    }
    int err = 0;
    for (int step = 0; step < nsteps && !err; ++step) {
        for (int s = 0; s < 5 && !err; ++s) {
            err = oracle_vol_rhs_o2(P, q, rhs, nthreads);
            for (size_t m = 0; m < n; ++m) {
                dq[m] = LSRK_A[s] * dq[m] + dt * rhs[m];
                q[m] = q[m] + LSRK_B[s] * dq[m];
            }
        }
    }
    free(dq);
    free(rhs);
    return err;
}

/* The same scheme on the scalar test equation y' = lam y (order checks). */
double oracle_lsrk_scalar(double lam, double y0, double dt, int nsteps)
{
    double y = y0, dy = 0.0;
    for (int step = 0; step < nsteps; ++step)
        for (int s = 0; s < 5; ++s) {
            dy = LSRK_A[s] * dy + dt * lam * y;
            y = y + LSRK_B[s] * dy;
        }
    return y;
}

/* Number of threads O2 will use for nthreads <= 0 (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
