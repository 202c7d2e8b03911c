// SELL-C-sigma sorting-window autotuner.  Host code only: every candidate is
// built and timed through the library's own entry points (upload, solver,
// solve), on copies of the matrix, so the caller's matrix and solvers are
// never touched.
#include <stdint.h>

#include <vector>

#include <cuda_runtime.h>

#include "bcs.h"
#include "bcs_tune.h"

extern "C" int bcs_autotune_sell_sigma(bcs_matrix A, int kind, int precision, int iters, const int* sigmas,
                                       int nsig, double* us_per_iter, int* best_sigma, bcs_matrix* tuned,
                                       void* stream) {
    if (tuned) *tuned = nullptr;
    if (!A || !sigmas || nsig <= 0 || !best_sigma) return BCS_ERR_ARG;
    if (kind < BCS_SSBICGSAFE2 || kind > BCS_P_BICGSAFE_RR) return BCS_ERR_ARG;
    if (precision < BCS_FP64 || precision > BCS_BF16MAT_REFINE) return BCS_ERR_ARG;
    for (int k = 0; k < nsig; ++k)
        if (sigmas[k] <= 0 || sigmas[k] % 32 != 0 || sigmas[k] > 4096) return BCS_ERR_ARG;
    int64_t n = 0, nnz = 0;
    int layouts = 0, stores = 0;
    int rc = bcs_matrix_info(A, &n, &nnz, nullptr, &layouts, &stores);
    if (rc) return rc;
    const int need = precision == BCS_FP32_REFINE ? BCS_STORE_F32 : precision == BCS_BF16MAT_REFINE ? BCS_STORE_BF16 : 0;
    if (need && !(stores & need)) return BCS_ERR_ARG;
    if (iters <= 0) iters = 20;

    // the CSR arrays back on the host: the source of every candidate's upload
    std::vector<int32_t> rp32((size_t)n + 1), col((size_t)(nnz > 0 ? nnz : 1));
    std::vector<double> val((size_t)(nnz > 0 ? nnz : 1));
    rc = bcs_matrix_export(A, rp32.data(), col.data(), val.data(), nullptr, nullptr, nullptr, nullptr, nullptr,
                           nullptr);
    if (rc) return rc;
    const std::vector<int64_t> rp(rp32.begin(), rp32.end());

    double* b = nullptr;
    double* x = nullptr;
    const size_t vb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    if (cudaMalloc(&b, vb) != cudaSuccess || cudaMalloc(&x, vb) != cudaSuccess) {
        if (b) cudaFree(b);
        return BCS_ERR_OOM;
    }
    {
        const std::vector<double> ones((size_t)(n > 0 ? n : 1), 1.0);
        if (cudaMemcpy(b, ones.data(), vb, cudaMemcpyHostToDevice) != cudaSuccess) rc = BCS_ERR_CUDA;
    }
    bcs_options o;
    bcs_options_default(&o);
    o.precision = precision;
    o.layout = BCS_LAYOUT_SELL;
    o.max_outer = 1;
    o.inner_tol = 1e-300;  // fixed iteration count: the inner runs never stop on the tolerance
    o.inner_stall = 0;
    o.history_len = 1;
    const cudaStream_t st = (cudaStream_t)stream;
    int bi = -1;
    double bt = 0.0;
    for (int k = 0; k < nsig && !rc; ++k) {
        bcs_matrix M = nullptr;
        rc = bcs_csr_upload(n, nnz, rp.data(), col.data(), val.data(), BCS_LAYOUT_SELL, 32, sigmas[k], stores,
                            stream, &M);
        if (rc) break;
        bcs_solver s = nullptr;
        rc = bcs_solver_create(M, kind, 0.0, iters, &o, &s);
        double t = 0.0;
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            if (cudaMemsetAsync(x, 0, vb, st) != cudaSuccess) {
                rc = BCS_ERR_CUDA;
                break;
            }
            bcs_result r;
            const int e = bcs_solve(s, b, x, &r, stream);
            if (e == BCS_ERR_CUDA || e == BCS_ERR_TIMEOUT || e == BCS_ERR_OOM || e == BCS_ERR_ARG) {
                rc = e;
                break;
            }
            t = r.seconds / (r.iterations > 0 ? r.iterations : 1);
        }
        bcs_solver_destroy(s);
        bcs_matrix_free(M);
        if (rc) break;
        if (us_per_iter) us_per_iter[k] = t * 1e6;
        if (bi < 0 || t < bt) {
            bi = k;
            bt = t;
        }
    }
    cudaFree(b);
    cudaFree(x);
    if (rc) return rc;
    *best_sigma = sigmas[bi];
    if (tuned)
        rc = bcs_csr_upload(n, nnz, rp.data(), col.data(), val.data(), layouts | BCS_LAYOUT_SELL, 32, sigmas[bi],
                            stores, stream, tuned);
    return rc;
}
