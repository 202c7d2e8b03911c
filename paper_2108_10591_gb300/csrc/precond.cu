// Jacobi (diagonal) preconditioning, applied on the right: the persistent
// solver runs unchanged on  A D^-1 y = b  and the solution is x = D^-1 y,
// D = diag(A).  The paper uses no preconditioner (Section 5); this is a build
// addition.  The residual b - (A D^-1) y of the solved system equals b - A x,
// so the tolerance keeps its meaning.
//
// Block-Jacobi (also on the right): M = the diagonal blocks of A, bs
// consecutive rows each.  Set-up here: the blocks and their inverses, [npad][bs]
// in block columns; the solver kernel applies M^-1 itself (solver.cuh, BJ).
#include <algorithm>

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

// One warp per diagonal block (rows b0 .. b0+m-1, m <= bs <= 32): the block
// D_k from the CSR rows (a repeated entry keeps its last value), then
// Gauss-Jordan elimination on [D_k | I] in shared memory.  Pivot: the first row
// r >= p with the largest |a[r][p]| (lane 0 scans the column in order); the
// pivot row is swapped in, divided by the saved pivot, and every other row r
// (lane r) subtracts f * row p with f = a[r][p] as a[r][c] - f * a[p][c],
// product and difference rounded separately (-fmad=false): per element the
// same operations as the sequential elimination.  D and E rows beyond a ragged
// block's m columns are zero.  flags[0] |= 1 for a singular block (zero,
// NaN or infinite pivot).
__global__ void k_bj_blocks(const int32_t* rp, const int32_t* col, const double* val, int64_t n, int bs, double* D,
                            double* E, int* flags) {
    extern __shared__ double sh[];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* a = sh + (size_t)w * 2 * bs * bs;
    double* inv = a + bs * bs;
    const int64_t nb = (n + bs - 1) / bs;
    for (int64_t blk = (int64_t)blockIdx.x * nw + w; blk < nb; blk += (int64_t)gridDim.x * nw) {
        const int64_t b0 = blk * bs;
        const int m = (int)((n - b0) < bs ? (n - b0) : bs);
        for (int k = lane; k < m * m; k += 32) {
            a[k] = 0.0;
            inv[k] = 0.0;
        }
        __syncwarp();
        if (lane < m) {
            for (int k = rp[b0 + lane]; k < rp[b0 + lane + 1]; ++k) {
                const int64_t c = (int64_t)col[k] - b0;
                if (c >= 0 && c < m) a[lane * m + c] = val[k];
            }
            inv[lane * m + lane] = 1.0;
        }
        __syncwarp();
        if (lane < m)
            for (int j = 0; j < bs; ++j) D[(b0 + lane) * bs + j] = j < m ? a[lane * m + j] : 0.0;
        bool ok = true;
        for (int p = 0; p < m; ++p) {
            int piv = p;
            if (lane == 0) {
                double big = fabs(a[p * m + p]);
                for (int r = p + 1; r < m; ++r)
                    if (fabs(a[r * m + p]) > big) {
                        big = fabs(a[r * m + p]);
                        piv = r;
                    }
                if (!(big > 0.0) || !isfinite(big)) piv = -1;
            }
            piv = __shfl_sync(full, piv, 0);
            if (piv < 0) {
                ok = false;
                break;
            }
            if (piv != p && lane < m) {
                double t = a[p * m + lane];
                a[p * m + lane] = a[piv * m + lane];
                a[piv * m + lane] = t;
                t = inv[p * m + lane];
                inv[p * m + lane] = inv[piv * m + lane];
                inv[piv * m + lane] = t;
            }
            __syncwarp();
            const double d = a[p * m + p];
            __syncwarp();
            if (lane < m) {
                a[p * m + lane] = a[p * m + lane] / d;
                inv[p * m + lane] = inv[p * m + lane] / d;
            }
            __syncwarp();
            if (lane < m && lane != p) {
                const double f = a[lane * m + p];
                for (int c = 0; c < m; ++c) {
                    a[lane * m + c] = a[lane * m + c] - f * a[p * m + c];
                    inv[lane * m + c] = inv[lane * m + c] - f * inv[p * m + c];
                }
            }
            __syncwarp();
        }
        if (!ok) {
            if (lane == 0) atomicOr(flags, 1);
            continue;
        }
        if (lane < m)
            for (int j = 0; j < bs; ++j) E[(b0 + lane) * bs + j] = j < m ? inv[lane * m + j] : 0.0;
        __syncwarp();
    }
}

// x <- M x in place, M = [rows][bs] block columns (D: into the solved system,
// E: back), one warp per 32-row tile: every lane's value is loaded before the
// first shuffle, so no lane overwrites a value another still needs.  The sum
// runs over the block's columns in order with fma from zero (rows >= n take
// part with 0 and their entries of M are zero).
__global__ void k_bj_apply(const double* M, double* x, int64_t n, int bs) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (n + 31) / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = wid; t < ntiles; t += nwarps) {
        const int64_t row = t * 32 + lane;
        const double v = row < n ? x[row] : 0.0;
        const int base = lane & ~(bs - 1);
        double acc = 0.0;
        for (int j = 0; j < bs; ++j) acc = fma(M[row * bs + j], __shfl_sync(full, v, base + j), acc);
        if (row < n) x[row] = acc;
    }
}

__global__ void k_to_f32(const double* in, float* out, int64_t m) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = __double2float_rn(in[k]);
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

// Block-Jacobi set-up: D and E = D^-1 ([npad][bs], FP64; rows >= n zero), E in
// FP32 for the refinement modes, and the solver's M^-1 copies (eight inner-type
// vectors and one FP64 vector).  BCS_ERR_ARG for a singular block.
int bjacobi_setup(bcs_solver s) {
    bcs_matrix A = s->A;
    const int64_t n = A->n;
    const int bs = s->bj_bs;
    const int64_t npad = std::max<int64_t>(((n + 31) / 32) * 32, 32);
    const size_t m = (size_t)npad * (size_t)bs;
    int rc = 0;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) rc = BCS_ERR_OOM;
    };
    int* flags = nullptr;
    alloc((void**)&s->bjD, sizeof(double) * m);
    alloc((void**)&s->bjE, sizeof(double) * m);
    if (s->vt_f32) alloc((void**)&s->bjE32, sizeof(float) * m);
    alloc(&s->bjhat, 8 * (size_t)npad * s->vbytes);
    alloc((void**)&s->bjxh, sizeof(double) * (size_t)npad);
    alloc((void**)&flags, sizeof(int));
    if (!rc && (cudaMemset(s->bjD, 0, sizeof(double) * m) != cudaSuccess ||
                cudaMemset(s->bjE, 0, sizeof(double) * m) != cudaSuccess ||
                cudaMemset(s->bjhat, 0, 8 * (size_t)npad * s->vbytes) != cudaSuccess ||
                cudaMemset(s->bjxh, 0, sizeof(double) * (size_t)npad) != cudaSuccess ||
                cudaMemset(flags, 0, sizeof(int)) != cudaSuccess))
        rc = BCS_ERR_CUDA;
    if (!rc && n > 0) {
        const int warps = 2;
        const size_t smem = (size_t)warps * 2 * bs * bs * sizeof(double);
        const int64_t nb = (n + bs - 1) / bs;
        const int grid = (int)std::min<int64_t>((nb + warps - 1) / warps, 65535);
        k_bj_blocks<<<grid, warps * 32, smem>>>(A->rowptr, A->col, A->val64, n, bs, s->bjD, s->bjE, flags);
        int hf = 0;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = BCS_ERR_CUDA;
        else if (hf)
            rc = BCS_ERR_ARG;   // a singular diagonal block
    }
    if (!rc && s->vt_f32) {
        k_to_f32<<<grid_of((int64_t)m), 256>>>(s->bjE, s->bjE32, (int64_t)m);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = BCS_ERR_CUDA;
    }
    if (flags) cudaFree(flags);
    return rc;
}

// x <- D x (inverse = 0: a start vector into the solved system) or x <- E x
// (inverse = 1: the solved system's iterate back to x), in place
int bjacobi_apply(bcs_solver s, double* x, int inverse, cudaStream_t st) {
    const int64_t n = s->A->n;
    if (n <= 0) return 0;
    const int64_t ntiles = (n + 31) / 32;
    const int grid = (int)std::min<int64_t>((ntiles + 7) / 8, 65535);
    k_bj_apply<<<grid, 256, 0, st>>>(inverse ? s->bjE : s->bjD, x, n, s->bj_bs);
    return cudaGetLastError() == cudaSuccess ? 0 : BCS_ERR_CUDA;
}

}  // namespace bcs
