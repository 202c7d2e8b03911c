// Matrix upload and format build (all on the device): CSR validation, FP32 /
// BF16 value copies, SELL-C-sigma construction, export, and the standalone
// y = A x entry point.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "device.cuh"

using namespace bcs;

namespace {

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) { rc = BCS_ERR_CUDA; goto done; } \
    } while (0)

// ---- validation: rowptr[0]=0, non-decreasing, rowptr[n]=nnz; columns in
// range and strictly ascending in each row.  Writes the int32 row pointer.
__global__ void k_check_rowptr(const int64_t* rp64, int64_t n, int64_t nnz, int32_t* rp32, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = rp64[i];
        if (v < 0 || v > nnz) atomicOr(bad, 1);
        if (i == 0 && v != 0) atomicOr(bad, 1);
        if (i == n && v != nnz) atomicOr(bad, 1);
        if (i < n && rp64[i + 1] < v) atomicOr(bad, 1);
        rp32[i] = (int32_t)v;
    }
}

__global__ void k_check_cols(const int32_t* rp, const int32_t* col, int64_t n, int* bad, int* maxlen) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = rp[i], e = rp[i + 1];
        int prev = -1;
        for (int k = b; k < e; ++k) {
            const int c = col[k];
            if (c < 0 || c >= n || c <= prev) { atomicOr(bad, 2); break; }
            prev = c;
        }
        atomicMax(maxlen, e - b);
    }
}

// FP64 -> FP32, round to nearest.
__global__ void k_to_f32(const double* in, float* out, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

// FP64 -> BF16, round to nearest even, one rounding: first to FP32 with
// round-to-odd (truncate, then set the last bit if anything was dropped),
// which keeps enough information for the final FP32 -> BF16 nearest-even
// rounding to equal the direct rounding of the FP64 value.
__device__ __forceinline__ uint16_t f64_to_bf16(double d) {
    if (isnan(d)) return (uint16_t)(((__double_as_longlong(d) >> 48) & 0x8000) | 0x7FC0);
    float f = __double2float_rz(d);
    unsigned u = __float_as_uint(f);
    if ((double)f != d && (u & 0x7F800000u) != 0x7F800000u) u |= 1u;
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // +-inf
    const unsigned lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}
__global__ void k_to_bf16(const double* in, uint16_t* out, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = f64_to_bf16(in[i]);
}

// ---- SELL-C-sigma ---------------------------------------------------------------
// One CTA per sigma-window: the position of row i inside its window is the
// number of rows that are longer, or as long and earlier (a stable sort by
// length, descending).
__global__ void k_sell_sort(const int32_t* rp, int64_t n, int sigma, int32_t* perm) {
    extern __shared__ int s_len[];
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int cnt = (int)((n - w0) < sigma ? (n - w0) : sigma);
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) s_len[j] = rp[w0 + j + 1] - rp[w0 + j];
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int lj = s_len[j];
        int rank = 0;
        for (int k = 0; k < cnt; ++k) {
            const int lk = s_len[k];
            rank += (lk > lj) || (lk == lj && k < j);
        }
        perm[w0 + rank] = (int32_t)(w0 + j);
    }
}
__global__ void k_invert(const int32_t* perm, int32_t* inv, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        inv[perm[p]] = (int32_t)p;
}
// slice widths (one warp per slice): longest row of the slice
__global__ void k_sell_width(const int32_t* rp, const int32_t* perm, int64_t n, int64_t nslices, int64_t* width) {
    const int lane = threadIdx.x & 31;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; s < nslices;
         s += (int64_t)gridDim.x * blockDim.x / 32) {
        const int64_t p = s * 32 + lane;
        int len = 0;
        if (p < n) {
            const int r = perm[p];
            len = rp[r + 1] - rp[r];
        }
        for (int off = 16; off > 0; off >>= 1) len = max(len, __shfl_xor_sync(kFull, len, off));
        if (lane == 0) width[s] = (int64_t)len * 32;
    }
}
// exclusive scan of m values into out[0..m] (single CTA; a one-off set-up step)
__global__ void k_scan(const int64_t* in, int64_t m, int64_t* out) {
    __shared__ int64_t s_part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t chunk = (m + T - 1) / T;
    const int64_t b0 = (int64_t)t * chunk, b = b0 < m ? b0 : m;
    const int64_t e = (b + chunk) < m ? (b + chunk) : m;
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += in[i];
    s_part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int k = 0; k < T; ++k) { const int64_t v = s_part[k]; s_part[k] = run; run += v; }
        out[m] = run;
    }
    __syncthreads();
    int64_t run = s_part[t];
    for (int64_t i = b; i < e; ++i) { out[i] = run; run += in[i]; }
}
template <class V>
__global__ void k_sell_fill(const int32_t* rp, const int32_t* col, const V* val, const int32_t* perm, const int32_t* inv,
                            const int64_t* sptr, int64_t n, int64_t nslices, int32_t* scol, V* sval) {
    const int lane = threadIdx.x & 31;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; s < nslices;
         s += (int64_t)gridDim.x * blockDim.x / 32) {
        const int64_t p = s * 32 + lane;
        const int64_t base = sptr[s], width = (sptr[s + 1] - base) / 32;
        int b = 0, len = 0;
        if (p < n) {
            const int r = perm[p];
            b = rp[r];
            len = rp[r + 1] - b;
        }
        const int32_t pad = (int32_t)(p < n ? p : n - 1);
        for (int64_t k = 0; k < width; ++k) {
            const int64_t dst = base + k * 32 + lane;
            if (k < len) {
                if (scol) scol[dst] = inv[col[b + k]];
                sval[dst] = val[b + k];
            } else {
                if (scol) scol[dst] = pad;
                sval[dst] = V(0);
            }
        }
    }
}

int grid_for(int64_t m, int block) {
    int64_t g = (m + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 65535 * 8));
}

// ---- standalone SpMV ---------------------------------------------------------------
template <class VT, class MT, int LAYOUT, int T>
__global__ void __launch_bounds__(256) k_spmv(KParams P, const MT* val, const VT* x, VT* y) {
    __shared__ VT s_buf[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t tile = (int64_t)blockIdx.x * 8 + warp; tile < P.ntiles; tile += nw) {
        const VT v = tile_spmv<VT, MT, LAYOUT, T>(P, val, x, tile, s_buf[warp]);
        const int64_t row = tile * 32 + lane;
        if (row < P.n) y[row] = v;
    }
}
template <class VT>
__global__ void k_gather(const int32_t* perm, const VT* src, VT* dst, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = src[perm[p]];
}
template <class VT>
__global__ void k_scatter(const int32_t* perm, const VT* src, VT* dst, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        dst[perm[p]] = src[p];
}

template <class VT, class MT>
int spmv_launch(bcs_matrix A, int layout, const MT* val, const VT* x, VT* y, int tpr, cudaStream_t st) {
    KParams P;
    memset(&P, 0, sizeof(P));
    P.n = A->n;
    P.ntiles = (A->n + 31) / 32;
    int sms = 148;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((P.ntiles + 7) / 8, (int64_t)sms * 8));
    if (layout == BCS_LAYOUT_SELL) {
        P.slice_ptr = A->slice_ptr;
        P.col = A->scol;
        VT* xp = (VT*)A->scratch;
        VT* yp = xp + A->n;
        const int g = grid_for(A->n, 256);
        k_gather<VT><<<g, 256, 0, st>>>(A->perm, x, xp, A->n);
        k_spmv<VT, MT, LAY_SELL, 1><<<grid, 256, 0, st>>>(P, val, xp, yp);
        k_scatter<VT><<<g, 256, 0, st>>>(A->perm, yp, y, A->n);
    } else {
        P.rowptr = A->rowptr;
        P.col = A->col;
        switch (tpr) {
            case -1: k_spmv<VT, MT, LAY_CSR, 0><<<grid, 256, 0, st>>>(P, val, x, y); break;
            case 1: k_spmv<VT, MT, LAY_CSR, 1><<<grid, 256, 0, st>>>(P, val, x, y); break;
            case 4: k_spmv<VT, MT, LAY_CSR, 4><<<grid, 256, 0, st>>>(P, val, x, y); break;
            case 8: k_spmv<VT, MT, LAY_CSR, 8><<<grid, 256, 0, st>>>(P, val, x, y); break;
            default: k_spmv<VT, MT, LAY_CSR, 32><<<grid, 256, 0, st>>>(P, val, x, y); break;
        }
    }
    return cudaGetLastError() == cudaSuccess ? BCS_OK : BCS_ERR_CUDA;
}

}  // namespace

namespace bcs {
// value copies with the upload's roundings (used by the preconditioner's scaled copies)
int convert_values(const double* in, int valtype, void* out, int64_t m, cudaStream_t st) {
    if (m <= 0) return 0;
    if (valtype == VAL_F32) k_to_f32<<<grid_for(m, 256), 256, 0, st>>>(in, (float*)out, m);
    else if (valtype == VAL_BF16) k_to_bf16<<<grid_for(m, 256), 256, 0, st>>>(in, (uint16_t*)out, m);
    else return (int)cudaMemcpyAsync(out, in, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    return (int)cudaGetLastError();
}
// Lanes per CSR row when the caller does not choose: the autotuned value for
// the precision if there is one, else adaptive for heavy-tailed row lengths in
// the refinement modes, else one lane per row (no cross-lane reduction: on
// GB300 an FP64 shuffle-add costs an FP64-pipe slot like an FMA).
int default_tpr(const bcs_matrix_s* A, int precision) {
    if (precision >= 0 && precision < 3 && A->tuned_tpr[precision]) return A->tuned_tpr[precision];
    // heavy-tailed row lengths in the refinement modes: adaptive (the warp takes
    // the long rows together).  FP64 keeps one lane per row, whose sums follow
    // the plain row order (bit-identical to a sequential FP64 solve).
    if (precision != BCS_FP64 && (double)A->max_row > 4.0 * A->avg_row + 4.0 && A->max_row > kLongRow) return -1;
    return 1;
}
}  // namespace bcs

extern "C" {

int bcs_csr_upload(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                   int layouts, int sell_C, int sell_sigma, int stores, void* stream, bcs_matrix* out) {
    NvtxRange nv("bcs_csr_upload");
    if (!out) return BCS_ERR_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || n >= (1ll << 31) || nnz >= (1ll << 31)) return BCS_ERR_ARG;
    if (!rowptr || (nnz > 0 && (!col || !val))) return BCS_ERR_ARG;
    if ((layouts & (BCS_LAYOUT_CSR | BCS_LAYOUT_SELL)) == 0 || (layouts & ~3)) return BCS_ERR_ARG;
    if (layouts & BCS_LAYOUT_SELL) {
        if (sell_C != 32 || sell_sigma <= 0 || sell_sigma % 32 != 0 || sell_sigma > 4096) return BCS_ERR_ARG;
    }
    if (stores & ~7) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = BCS_OK;
    bcs_matrix A = new bcs_matrix_s();
    int64_t* rp64 = nullptr;
    int* flags = nullptr;  // [0] bad, [1] max row length
    int32_t* inv = nullptr;    // SELL build: inverse permutation
    int64_t* width = nullptr;  // SELL build: padded entries per slice
    int hflags[2] = {0, 0};
    const int64_t m = std::max<int64_t>(nnz, 1);
    A->n = n;
    A->nnz = nnz;
    A->layouts = layouts;
    A->stores = stores | BCS_STORE_F64;
    cudaGetDevice(&A->device);
    CK(cudaMalloc(&rp64, sizeof(int64_t) * (n + 1)));
    CK(cudaMalloc(&flags, sizeof(int) * 2));
    CK(cudaMalloc(&A->rowptr, sizeof(int32_t) * (n + 1)));
    CK(cudaMalloc(&A->col, sizeof(int32_t) * m));
    CK(cudaMalloc(&A->val64, sizeof(double) * m));
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * 2, st));
    CK(cudaMemcpyAsync(rp64, rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (nnz > 0) {
        CK(cudaMemcpyAsync(A->col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(A->val64, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
    }
    k_check_rowptr<<<grid_for(n + 1, 256), 256, 0, st>>>(rp64, n, nnz, A->rowptr, flags);
    CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflags[0]) { rc = BCS_ERR_ARG; goto done; }
    if (n > 0) k_check_cols<<<grid_for(n, 256), 256, 0, st>>>(A->rowptr, A->col, n, flags, flags + 1);
    CK(cudaMemcpyAsync(hflags, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hflags[0]) { rc = BCS_ERR_ARG; goto done; }
    A->max_row = hflags[1];
    A->avg_row = n > 0 ? (double)nnz / (double)n : 0.0;
    if (stores & BCS_STORE_F32) {
        CK(cudaMalloc(&A->val32, sizeof(float) * m));
        k_to_f32<<<grid_for(m, 256), 256, 0, st>>>(A->val64, A->val32, nnz);
    }
    if (stores & BCS_STORE_BF16) {
        CK(cudaMalloc(&A->valbf16, sizeof(uint16_t) * m));
        k_to_bf16<<<grid_for(m, 256), 256, 0, st>>>(A->val64, A->valbf16, nnz);
    }
    if (layouts & BCS_LAYOUT_SELL) {
        const int64_t ns = (n + 31) / 32;
        A->sell_C = 32;
        A->sell_sigma = sell_sigma;
        A->nslices = ns;
        CK(cudaMalloc(&A->perm, sizeof(int32_t) * std::max<int64_t>(n, 1)));
        CK(cudaMalloc(&inv, sizeof(int32_t) * std::max<int64_t>(n, 1)));
        CK(cudaMalloc(&width, sizeof(int64_t) * std::max<int64_t>(ns, 1)));
        CK(cudaMalloc(&A->slice_ptr, sizeof(int64_t) * (ns + 1)));
        CK(cudaMalloc(&A->scratch, sizeof(double) * 2 * std::max<int64_t>(n, 1)));
        if (n > 0) {
            const int nwin = (int)((n + sell_sigma - 1) / sell_sigma);
            k_sell_sort<<<nwin, std::min(sell_sigma, 1024), sizeof(int) * sell_sigma, st>>>(A->rowptr, n, sell_sigma, A->perm);
            k_invert<<<grid_for(n, 256), 256, 0, st>>>(A->perm, inv, n);
            k_sell_width<<<grid_for(ns * 32, 256), 256, 0, st>>>(A->rowptr, A->perm, n, ns, width);
            k_scan<<<1, 1024, 0, st>>>(width, ns, A->slice_ptr);
        } else {
            CK(cudaMemsetAsync(A->slice_ptr, 0, sizeof(int64_t), st));
        }
        CK(cudaMemcpyAsync(&A->padded, A->slice_ptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        {
            const int64_t pm = std::max<int64_t>(A->padded, 1);
            CK(cudaMalloc(&A->scol, sizeof(int32_t) * pm));
            CK(cudaMalloc(&A->sval64, sizeof(double) * pm));
            if (A->val32) CK(cudaMalloc(&A->sval32, sizeof(float) * pm));
            if (A->valbf16) CK(cudaMalloc(&A->svalbf16, sizeof(uint16_t) * pm));
            if (n > 0) {
                const int g = grid_for(ns * 32, 256);
                k_sell_fill<double><<<g, 256, 0, st>>>(A->rowptr, A->col, A->val64, A->perm, inv, A->slice_ptr, n, ns,
                                                      A->scol, A->sval64);
                if (A->val32)
                    k_sell_fill<float><<<g, 256, 0, st>>>(A->rowptr, A->col, A->val32, A->perm, inv, A->slice_ptr, n,
                                                         ns, nullptr, A->sval32);
                if (A->valbf16)
                    k_sell_fill<uint16_t><<<g, 256, 0, st>>>(A->rowptr, A->col, A->valbf16, A->perm, inv, A->slice_ptr,
                                                            n, ns, nullptr, A->svalbf16);
            }
        }
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
done:
    if (rp64) cudaFree(rp64);
    if (flags) cudaFree(flags);
    if (inv) cudaFree(inv);
    if (width) cudaFree(width);
    if (rc != BCS_OK) {
        bcs_matrix_free(A);
        return rc;
    }
    *out = A;
    return BCS_OK;
}

int bcs_matrix_info(bcs_matrix A, int64_t* n, int64_t* nnz, int64_t* sell_padded, int* layouts, int* stores) {
    if (!A) return BCS_ERR_ARG;
    if (n) *n = A->n;
    if (nnz) *nnz = A->nnz;
    if (sell_padded) *sell_padded = A->padded;
    if (layouts) *layouts = A->layouts;
    if (stores) *stores = A->stores;
    return BCS_OK;
}

int bcs_matrix_export(bcs_matrix A, int32_t* rowptr, int32_t* col, double* val64, float* val32, uint16_t* valbf16,
                      int32_t* perm, int64_t* slice_ptr, int32_t* scol, double* sval64) {
    if (!A) return BCS_ERR_ARG;
    const bool sell = (A->layouts & BCS_LAYOUT_SELL) != 0;
    if ((val32 && !A->val32) || (valbf16 && !A->valbf16)) return BCS_ERR_ARG;
    if ((perm || slice_ptr || scol || sval64) && !sell) return BCS_ERR_ARG;
    int rc = BCS_OK;
    CK(cudaDeviceSynchronize());
    if (rowptr) CK(cudaMemcpy(rowptr, A->rowptr, sizeof(int32_t) * (A->n + 1), cudaMemcpyDeviceToHost));
    if (col && A->nnz) CK(cudaMemcpy(col, A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost));
    if (val64 && A->nnz) CK(cudaMemcpy(val64, A->val64, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost));
    if (val32 && A->nnz) CK(cudaMemcpy(val32, A->val32, sizeof(float) * A->nnz, cudaMemcpyDeviceToHost));
    if (valbf16 && A->nnz) CK(cudaMemcpy(valbf16, A->valbf16, sizeof(uint16_t) * A->nnz, cudaMemcpyDeviceToHost));
    if (perm && A->n) CK(cudaMemcpy(perm, A->perm, sizeof(int32_t) * A->n, cudaMemcpyDeviceToHost));
    if (slice_ptr) CK(cudaMemcpy(slice_ptr, A->slice_ptr, sizeof(int64_t) * (A->nslices + 1), cudaMemcpyDeviceToHost));
    if (scol && A->padded) CK(cudaMemcpy(scol, A->scol, sizeof(int32_t) * A->padded, cudaMemcpyDeviceToHost));
    if (sval64 && A->padded) CK(cudaMemcpy(sval64, A->sval64, sizeof(double) * A->padded, cudaMemcpyDeviceToHost));
done:
    return rc;
}

int bcs_spmv(bcs_matrix A, int layout, int store, const void* x, void* y, int vec_f32, int threads_per_row,
             void* stream) {
    if (!A || !x || !y) return BCS_ERR_ARG;
    if (A->n > 0 && (!device_reachable(x) || !device_reachable(y))) return BCS_ERR_ARG;
    if (layout != BCS_LAYOUT_CSR && layout != BCS_LAYOUT_SELL) return BCS_ERR_ARG;
    if (!(A->layouts & layout)) return BCS_ERR_ARG;
    if (store != BCS_STORE_F64 && store != BCS_STORE_F32 && store != BCS_STORE_BF16) return BCS_ERR_ARG;
    if (!vec_f32 && store != BCS_STORE_F64) return BCS_ERR_ARG;  // FP64 vectors use the FP64 values
    int tpr = threads_per_row ? threads_per_row
                              : default_tpr(A, !vec_f32 ? BCS_FP64 : store == BCS_STORE_BF16 ? BCS_BF16MAT_REFINE
                                                                                              : BCS_FP32_REFINE);
    if (tpr != 1 && tpr != 4 && tpr != 8 && tpr != 32 && tpr != -1) return BCS_ERR_ARG;
    if (A->n == 0) return BCS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const bool sell = layout == BCS_LAYOUT_SELL;
    if (!vec_f32) {
        return spmv_launch<double, double>(A, layout, sell ? A->sval64 : A->val64, (const double*)x, (double*)y, tpr, st);
    }
    if (store == BCS_STORE_F64) {
        return BCS_ERR_ARG;
    } else if (store == BCS_STORE_F32) {
        if (!A->val32) return BCS_ERR_ARG;
        return spmv_launch<float, float>(A, layout, sell ? A->sval32 : A->val32, (const float*)x, (float*)y, tpr, st);
    } else {
        if (!A->valbf16) return BCS_ERR_ARG;
        return spmv_launch<float, uint16_t>(A, layout, sell ? A->svalbf16 : A->valbf16, (const float*)x, (float*)y, tpr,
                                           st);
    }
}

void bcs_matrix_free(bcs_matrix A) {
    if (!A) return;
    cudaDeviceSynchronize();
    void* ptrs[] = {A->rowptr, A->col, A->val64, A->val32, A->valbf16, A->perm, A->slice_ptr,
                    A->scol, A->sval64, A->sval32, A->svalbf16, A->scratch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete A;
}

}  // extern "C"
