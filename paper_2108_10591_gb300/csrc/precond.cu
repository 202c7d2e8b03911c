// Jacobi (diagonal) preconditioning, applied on the right: the persistent
// solver runs unchanged on  A D^-1 y = b  and the solution is x = D^-1 y,
// D = diag(A).  The paper uses no preconditioner (Section 5); this is a build
// addition.  The residual b - (A D^-1) y of the solved system equals b - A x,
// so the tolerance keeps its meaning.
#include "internal.h"

namespace bcs {

int convert_values(const double* in, int valtype, void* out, int64_t m, cudaStream_t st);

namespace {

int grid_of(int64_t m) {
    const int64_t g = (m + 255) / 256;
    return (int)(g < 1 ? 1 : g > 4096 ? 4096 : g);
}

// d[i] = a_ii; flags[0] |= 1 if a diagonal entry is missing, zero or not finite
__global__ void k_diag(const int32_t* rp, const int32_t* col, const double* val, int64_t n, double* d, int* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == i) v = val[k];
        d[i] = v;
        if (!(v != 0.0) || !isfinite(v)) atomicOr(flags, 1);
    }
}

// out[k] = val[k] / d[col[k]] (column scaling; padding entries keep value 0)
__global__ void k_colscale(const int32_t* col, const double* val, const double* d, double* out, int64_t m) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = val[k] / d[col[k]];
}

__global__ void k_gather_d(const int32_t* perm, const double* d, double* dp, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dp[i] = d[perm[i]];
}

// x <- D x (into the solved system) or x <- D^-1 x (back)
__global__ void k_scale(double* x, const double* d, int64_t n, int into) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = into ? x[i] * d[i] : x[i] / d[i];
}

}  // namespace

// Build the solver's scaled value copies for its layout and value type.
int precond_setup(bcs_solver s) {
    bcs_matrix A = s->A;
    const int64_t n = A->n;
    const bool sell = s->layout == LAY_SELL;
    const int64_t m = sell ? A->padded : A->nnz;
    int rc = 0;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) rc = BCS_ERR_OOM;
    };
    int* flags = nullptr;
    alloc((void**)&s->pdiag, sizeof(double) * (size_t)(n > 0 ? n : 1));
    alloc((void**)&s->pval64, sizeof(double) * (size_t)(m > 0 ? m : 1));
    alloc((void**)&flags, sizeof(int));
    double* dp = nullptr;
    if (sell) alloc((void**)&dp, sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (s->valtype != VAL_F64) alloc(&s->pvalin, (s->valtype == VAL_F32 ? 4 : 2) * (size_t)(m > 0 ? m : 1));
    if (!rc && cudaMemset(flags, 0, sizeof(int)) != cudaSuccess) rc = BCS_ERR_CUDA;
    if (!rc && n > 0) {
        k_diag<<<grid_of(n), 256>>>(A->rowptr, A->col, A->val64, n, s->pdiag, flags);
        int hf = 0;
        if (cudaMemcpy(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = BCS_ERR_CUDA;
        else if (hf) rc = BCS_ERR_ARG;  // Jacobi needs a nonzero finite diagonal
    }
    if (!rc && m > 0) {
        if (sell) {
            k_gather_d<<<grid_of(n), 256>>>(A->perm, s->pdiag, dp, n);
            k_colscale<<<grid_of(m), 256>>>(A->scol, A->sval64, dp, s->pval64, m);
        } else {
            k_colscale<<<grid_of(m), 256>>>(A->col, A->val64, s->pdiag, s->pval64, m);
        }
        if (s->valtype != VAL_F64 && convert_values(s->pval64, s->valtype, s->pvalin, m, 0) != 0) rc = BCS_ERR_CUDA;
        if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = BCS_ERR_CUDA;
    }
    if (flags) cudaFree(flags);
    if (dp) cudaFree(dp);
    return rc;
}

int precond_scale(bcs_solver s, double* x, int into, cudaStream_t st) {
    const int64_t n = s->A->n;
    if (n <= 0) return 0;
    k_scale<<<grid_of(n), 256, 0, st>>>(x, s->pdiag, n, into);
    return cudaGetLastError() == cudaSuccess ? 0 : BCS_ERR_CUDA;
}

}  // namespace bcs
