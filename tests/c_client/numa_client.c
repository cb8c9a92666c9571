/*
 * A plain C client of the volume-term library, built with a C compiler against
 * include/numa_vol.h and libnumavol.so.  The tests use it to show that the
 * boundary is C: no C++ in the header, no torch types, host buffers in and
 * out.
 *
 *   numa_client check
 *       Host-only calls, no GPU needed: the GLL differentiation matrix for
 *       N = 1 and N = 2 against their closed forms, and argument validation
 *       (NUMA_EINVAL with a message, NULL-safe destroy and kernel name).
 *
 *   numa_client rhs <problem> <out> fp64|mixed
 *       Reads a problem, evaluates the volume term through numa_vol_rhs_host
 *       and writes the rhs.
 *
 * Problem file, little-endian: int32 N, int32 num_tracers, int64 Ne, four
 * doubles (p0, R, cp, grav); then FP64 arrays of M = Ne (N+1)^3 values:
 * g[0] .. g[8], Jinv, rho_ref, rhotheta_ref; then the state, 5 + num_tracers
 * planes of M values, doubles for fp64 and floats (perturbation form) for
 * mixed.  The output file holds the rhs planes in the state's type.
 *
 * Exit status: 0 on success, 1 for a bad command line or file, 2 when a check
 * fails or the library returns an error (its message is printed).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "numa_vol.h"

static int fail(const char *what, int code) {
    fprintf(stderr, "numa_client: %s (code %d): %s\n", what, code, numa_vol_last_error());
    return 2;
}

static int close_to(const double *a, const double *b, int n, double tol) {
    for (int i = 0; i < n; ++i)
        if (fabs(a[i] - b[i]) > tol) return 0;
    return 1;
}

static int run_check(void) {
    double D[9];
    /* N = 1: nodes -1, 1; N = 2: nodes -1, 0, 1 (closed forms) */
    static const double D1[4] = {-0.5, 0.5, -0.5, 0.5};
    static const double D2[9] = {-1.5, 2.0, -0.5, -0.5, 0.0, 0.5, 0.5, -2.0, 1.5};
    int rc = numa_vol_diff_matrix(1, D);
    if (rc != NUMA_OK) return fail("numa_vol_diff_matrix(1)", rc);
    if (!close_to(D, D1, 4, 1e-15)) return fail("D for N = 1 differs from its closed form", 0);
    rc = numa_vol_diff_matrix(2, D);
    if (rc != NUMA_OK) return fail("numa_vol_diff_matrix(2)", rc);
    if (!close_to(D, D2, 9, 1e-14)) return fail("D for N = 2 differs from its closed form", 0);

    if (numa_vol_diff_matrix(0, D) != NUMA_EINVAL || numa_vol_last_error()[0] == '\0')
        return fail("N = 0 was not rejected with a message", 0);

    numa_vol *h = NULL;
    numa_constants c = {1e5, 287.17, 1004.67, 9.80616};
    numa_mesh mesh;
    memset(&mesh, 0, sizeof mesh);
    mesh.num_elements = 1;
    mesh.N = 3;
    numa_geometry geo;
    memset(&geo, 0, sizeof geo);   /* null arrays: rejected before any CUDA call */
    if (numa_vol_create(&mesh, &geo, &c, NUMA_FP64, &h) != NUMA_EINVAL || h != NULL)
        return fail("null geometry was not rejected", 0);
    if (numa_vol_create(NULL, &geo, &c, NUMA_FP64, &h) != NUMA_EINVAL)
        return fail("null mesh was not rejected", 0);
    if (numa_vol_rhs(NULL, NULL, NULL, NULL) != NUMA_EINVAL)
        return fail("null handle was not rejected", 0);
    numa_vol_destroy(NULL);
    if (strcmp(numa_vol_kernel_name(NULL), "") != 0)
        return fail("kernel name of a null handle is not empty", 0);
    printf("ok\n");
    return 0;
}

static int read_all(FILE *f, void *dst, size_t bytes) {
    return fread(dst, 1, bytes, f) == bytes;
}

static int run_rhs(const char *in_path, const char *out_path, const char *prec_name) {
    numa_precision prec;
    size_t elem;
    if (strcmp(prec_name, "fp64") == 0) {
        prec = NUMA_FP64;
        elem = sizeof(double);
    } else if (strcmp(prec_name, "mixed") == 0) {
        prec = NUMA_MIXED;
        elem = sizeof(float);
    } else {
        fprintf(stderr, "numa_client: precision must be fp64 or mixed\n");
        return 1;
    }
    FILE *f = fopen(in_path, "rb");
    if (!f) {
        fprintf(stderr, "numa_client: cannot open %s\n", in_path);
        return 1;
    }
    int32_t N, ntr;
    int64_t ne;
    double k[4];
    if (!read_all(f, &N, 4) || !read_all(f, &ntr, 4) || !read_all(f, &ne, 8) ||
        !read_all(f, k, sizeof k) || N < 1 || N > NUMA_MAX_N_FP64 || ntr < 0 ||
        ntr > NUMA_MAX_TRACERS || ne < 0) {
        fprintf(stderr, "numa_client: bad problem header\n");
        fclose(f);
        return 1;
    }
    const int64_t nq = N + 1;
    const size_t M = (size_t)ne * (size_t)(nq * nq * nq);
    const size_t planes = 5 + (size_t)ntr;
    double *arrays = malloc(12 * M * sizeof(double) + 1);
    void *q = malloc(planes * M * elem + 1);
    void *rhs = malloc(planes * M * elem + 1);
    int status = 1;
    if (!arrays || !q || !rhs) {
        fprintf(stderr, "numa_client: out of host memory\n");
        goto done;
    }
    if (!read_all(f, arrays, 12 * M * sizeof(double)) || !read_all(f, q, planes * M * elem)) {
        fprintf(stderr, "numa_client: problem file too short\n");
        goto done;
    }
    numa_mesh mesh;
    memset(&mesh, 0, sizeof mesh);
    mesh.num_elements = ne;
    mesh.N = N;
    mesh.num_tracers = ntr;
    numa_geometry geo;
    for (int a = 0; a < 9; ++a) geo.g[a] = arrays + (size_t)a * M;
    geo.Jinv = arrays + 9 * M;
    geo.rho_ref = arrays + 10 * M;
    geo.rhotheta_ref = arrays + 11 * M;
    numa_constants c = {k[0], k[1], k[2], k[3]};
    numa_vol *h = NULL;
    int rc = numa_vol_create(&mesh, &geo, &c, prec, &h);
    if (rc != NUMA_OK) {
        status = fail("numa_vol_create", rc);
        goto done;
    }
    rc = numa_vol_rhs_host(h, q, rhs);
    if (rc != NUMA_OK) {
        status = fail("numa_vol_rhs_host", rc);
        numa_vol_destroy(h);
        goto done;
    }
    fprintf(stderr, "numa_client: %s\n", numa_vol_kernel_name(h));
    numa_vol_destroy(h);
    FILE *o = fopen(out_path, "wb");
    if (!o || fwrite(rhs, 1, planes * M * elem, o) != planes * M * elem) {
        fprintf(stderr, "numa_client: cannot write %s\n", out_path);
        if (o) fclose(o);
        goto done;
    }
    fclose(o);
    status = 0;
done:
    fclose(f);
    free(arrays);
    free(q);
    free(rhs);
    return status;
}

int main(int argc, char **argv) {
    if (argc == 2 && strcmp(argv[1], "check") == 0) return run_check();
    if (argc == 5 && strcmp(argv[1], "rhs") == 0) return run_rhs(argv[2], argv[3], argv[4]);
    fprintf(stderr, "usage: numa_client check | numa_client rhs <problem> <out> fp64|mixed\n");
    return 1;
}
