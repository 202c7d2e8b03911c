/*
 * A solve through the C ABI alone (include/bcs.h; no Python, no PyTorch):
 * reads a CSR system from a binary file, uploads it from host memory, runs
 * one method of the paper (Algorithm 3, 4 or 5) with bcs_solve_host and
 * writes x.  Used by tests/test_c_abi.py.
 *
 *   c_abi_solve IN OUT KIND      solve; KIND = 0 ssBiCGSafe2, 1 p-BiCGSafe,
 *                                2 p-BiCGSafe-rr
 *   c_abi_solve --no-gpu         only the calls that need no device
 *
 * IN: int64 n, int64 nnz, int64 rowptr[n+1], int32 col[nnz],
 *     double val[nnz], double b[n] (native byte order).
 * OUT: double x[n].  stdout: one line "status iterations outer_steps
 * rr_steps rel_res_true" (the last as a C99 hex float).
 * Exit code: 0 when every call returned what was expected, else 1.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "bcs.h"

static int read_all(FILE* f, void* p, size_t size, size_t count) {
    return count == 0 || fread(p, size, count, f) == count;
}

static int no_gpu_checks(void) {
    bcs_options o;
    bcs_matrix A = NULL;
    bcs_solver S = NULL;
    const int64_t rowptr[2] = {0, 1};
    const int32_t col[1] = {0};
    const double val[1] = {1.0};
    bcs_options_default(&o);
    if (o.rr_m != 100 || o.max_outer != 30) return 1;
    if (bcs_status_string(BCS_OK) == NULL) return 1;
    /* no layout requested, and no output handle: both refused before any device work */
    if (bcs_csr_upload(1, 1, rowptr, col, val, 0, 32, 256, BCS_STORE_F64, NULL, &A) != BCS_ERR_ARG) return 1;
    if (bcs_csr_upload(1, 1, rowptr, col, val, BCS_LAYOUT_CSR, 32, 256, BCS_STORE_F64, NULL, NULL) != BCS_ERR_ARG)
        return 1;
    if (bcs_solver_create(NULL, BCS_P_BICGSAFE, 1e-10, 100, &o, &S) != BCS_ERR_ARG) return 1;
    if (bcs_solve_host(NULL, NULL, NULL, NULL, NULL) != BCS_ERR_ARG) return 1;
    printf("no-gpu checks ok\n");
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 2) return no_gpu_checks();
    if (argc != 4) {
        fprintf(stderr, "usage: %s IN OUT KIND | --no-gpu\n", argv[0]);
        return 1;
    }
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 1;
    int64_t n = 0, nnz = 0;
    if (!read_all(f, &n, sizeof n, 1) || !read_all(f, &nnz, sizeof nnz, 1) || n < 0 || nnz < 0) return 1;
    int64_t* rowptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* col = malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    double* val = malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    double* b = malloc(sizeof(double) * (size_t)(n ? n : 1));
    double* x = calloc((size_t)(n ? n : 1), sizeof(double));   /* x_0 = 0 */
    if (!rowptr || !col || !val || !b || !x) return 1;
    if (!read_all(f, rowptr, sizeof(int64_t), (size_t)(n + 1)) || !read_all(f, col, sizeof(int32_t), (size_t)nnz) ||
        !read_all(f, val, sizeof(double), (size_t)nnz) || !read_all(f, b, sizeof(double), (size_t)n))
        return 1;
    fclose(f);

    bcs_matrix A = NULL;
    bcs_solver S = NULL;
    bcs_options o;
    bcs_result r;
    int rc = bcs_csr_upload(n, nnz, rowptr, col, val, BCS_LAYOUT_CSR, 32, 256, BCS_STORE_F64, NULL, &A);
    if (rc != BCS_OK) {
        fprintf(stderr, "bcs_csr_upload: %s\n", bcs_status_string(rc));
        return 1;
    }
    bcs_options_default(&o);
    o.threads_per_row = 1;
    rc = bcs_solver_create(A, atoi(argv[3]), 1e-10, 10000, &o, &S);
    if (rc != BCS_OK) {
        fprintf(stderr, "bcs_solver_create: %s\n", bcs_status_string(rc));
        return 1;
    }
    rc = bcs_solve_host(S, b, x, &r, NULL);
    printf("%d %d %d %d %a\n", r.status, r.iterations, r.outer_steps, r.rr_steps, r.rel_res_true);
    f = fopen(argv[2], "wb");
    if (!f || fwrite(x, sizeof(double), (size_t)n, f) != (size_t)n) return 1;
    fclose(f);
    bcs_solver_destroy(S);
    bcs_matrix_free(A);
    free(rowptr);
    free(col);
    free(val);
    free(b);
    free(x);
    return rc == BCS_OK ? 0 : 1;
}
