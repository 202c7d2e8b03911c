// C ABI: solver objects, single and batched solves, status strings.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "solver.cuh"

using namespace bcs;

namespace bcs {
#define BCS_DECL(tag)                                                                                  \
    int dispatch_##tag##_0(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid); \
    int dispatch_##tag##_1(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid);
BCS_DECL(f64)
BCS_DECL(f32)
BCS_DECL(bf16)
#undef BCS_DECL
int dispatch_batched_f64(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters);
int dispatch_batched_f32(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters);
int dispatch_batched_bf16(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters);
int default_tpr(const bcs_matrix_s* A);
}  // namespace bcs

namespace {

int dispatch(const KParams* P, int vt_f32, int valtype, int layout, int tpr, int grid, cudaStream_t st, int* mg) {
    const bool sub0 = layout == LAY_SELL || tpr == 1;
    if (!vt_f32) return sub0 ? dispatch_f64_0(P, layout, tpr, grid, st, mg) : dispatch_f64_1(P, layout, tpr, grid, st, mg);
    if (valtype == VAL_F32)
        return sub0 ? dispatch_f32_0(P, layout, tpr, grid, st, mg) : dispatch_f32_1(P, layout, tpr, grid, st, mg);
    return sub0 ? dispatch_bf16_0(P, layout, tpr, grid, st, mg) : dispatch_bf16_1(P, layout, tpr, grid, st, mg);
}

int dispatch_b(const BatchArgs* B, int vt_f32, int valtype, int tpr, int nc, cudaStream_t st, int* mc) {
    if (!vt_f32) return dispatch_batched_f64(B, tpr, nc, st, mc);
    if (valtype == VAL_F32) return dispatch_batched_f32(B, tpr, nc, st, mc);
    return dispatch_batched_bf16(B, tpr, nc, st, mc);
}

bool valid_tpr(int t) { return t == 1 || t == 4 || t == 8 || t == 32; }

long long budget_cycles(double ms) {
    // SM cycles per millisecond at the GB300's maximum SM clock (2070 MHz);
    // at lower clocks the wait lasts proportionally longer in wall time.
    double c = ms * 2.07e6;
    if (!(c > 0)) c = 2.07e6;
    if (c > 4.0e12) c = 4.0e12;
    return (long long)c;
}

int precision_types(bcs_matrix A, int precision, int* vt_f32, int* valtype) {
    switch (precision) {
        case BCS_FP64: *vt_f32 = 0; *valtype = VAL_F64; return BCS_OK;
        case BCS_FP32_REFINE:
            if (!A->val32) return BCS_ERR_ARG;
            *vt_f32 = 1; *valtype = VAL_F32; return BCS_OK;
        case BCS_BF16MAT_REFINE:
            if (!A->valbf16) return BCS_ERR_ARG;
            *vt_f32 = 1; *valtype = VAL_BF16; return BCS_OK;
        default: return BCS_ERR_ARG;
    }
}

const void* inner_values(bcs_matrix A, int layout, int valtype) {
    const bool sell = layout == LAY_SELL;
    if (valtype == VAL_F64) return sell ? (const void*)A->sval64 : (const void*)A->val64;
    if (valtype == VAL_F32) return sell ? (const void*)A->sval32 : (const void*)A->val32;
    return sell ? (const void*)A->svalbf16 : (const void*)A->valbf16;
}

int check_options(const bcs_options& o) {
    if (o.rr_m <= 0 || o.rr_M < 0 || o.max_outer <= 0 || o.history_len < 0) return BCS_ERR_ARG;
    if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return BCS_ERR_ARG;
    if (o.layout != BCS_LAYOUT_CSR && o.layout != BCS_LAYOUT_SELL) return BCS_ERR_ARG;
    if (o.threads_per_row != 0 && !valid_tpr(o.threads_per_row)) return BCS_ERR_ARG;
    if (o.ctas_per_sm < 0 || o.ctas_per_sm > 8 || o.max_ctas < 0) return BCS_ERR_ARG;
    if (!(o.spin_budget_ms > 0.0)) return BCS_ERR_ARG;
    if (o.inner_maxit < 0 || o.inner_stall < 0) return BCS_ERR_ARG;
    return BCS_OK;
}

}  // namespace

extern "C" {

void bcs_options_default(bcs_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->rr_m = 100;
    o->rr_M = 0;  // 0 = maxit
    o->precision = BCS_FP64;
    o->inner_tol = 1e-3;
    o->max_outer = 30;
    o->history_len = 4096;
    o->layout = BCS_LAYOUT_CSR;
    o->threads_per_row = 0;
    o->ctas_per_sm = 0;
    o->max_ctas = 0;
    o->spin_budget_ms = 2000.0;
    o->inner_maxit = 0;
    o->inner_stall = 50;
}

const char* bcs_status_string(int s) {
    switch (s) {
        case BCS_OK: return "ok";
        case BCS_NOT_CONVERGED: return "not converged (iteration or outer-step limit reached)";
        case BCS_ERR_ARG: return "invalid argument";
        case BCS_ERR_CUDA: return "CUDA error";
        case BCS_ERR_BREAKDOWN: return "breakdown (zero denominator in the scalar recurrence)";
        case BCS_ERR_TIMEOUT: return "grid barrier timed out";
        case BCS_ERR_NONFINITE: return "non-finite value in the scalar recurrence";
        case BCS_ERR_OOM: return "device allocation failed";
        default: return "unknown status";
    }
}

void bcs_solver_destroy(bcs_solver s) {
    if (!s) return;
    cudaDeviceSynchronize();
    void* ptrs[] = {s->vecmem, s->x64w, s->b64w, s->partials, s->bar, s->hist, s->scal, s->out, s->xb_dev};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (s->host_out) cudaFreeHost(s->host_out);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    delete s;
}

int bcs_solver_create(bcs_matrix A, int kind, double tol, int maxit, const bcs_options* opt, bcs_solver* out) {
    if (!out) return BCS_ERR_ARG;
    *out = nullptr;
    if (!A || kind < BCS_SSBICGSAFE2 || kind > BCS_P_BICGSAFE_RR || !(tol >= 0.0) || maxit < 0) return BCS_ERR_ARG;
    bcs_options o;
    if (opt) o = *opt; else bcs_options_default(&o);
    if (o.rr_M == 0) o.rr_M = maxit + 1;
    int rc = check_options(o);
    if (rc) return rc;
    if (!(A->layouts & o.layout)) return BCS_ERR_ARG;
    bcs_solver s = new bcs_solver_s();
    s->A = A;
    s->kind = kind;
    s->tol = tol;
    s->maxit = maxit;
    s->opt = o;
    rc = precision_types(A, o.precision, &s->vt_f32, &s->valtype);
    if (rc) { delete s; return rc; }
    s->layout = o.layout == BCS_LAYOUT_SELL ? LAY_SELL : LAY_CSR;
    s->tpr = s->layout == LAY_SELL ? 1 : (o.threads_per_row ? o.threads_per_row : default_tpr(A));
    s->vbytes = s->vt_f32 ? sizeof(float) : sizeof(double);
    const int64_t n = A->n, nn = std::max<int64_t>(n, 1);
    const int64_t ntiles = (n + 31) / 32;
    int maxg = 0;
    if (dispatch(nullptr, s->vt_f32, s->valtype, s->layout, s->tpr, 0, 0, &maxg) != 0 || maxg <= 0) {
        delete s;
        return BCS_ERR_CUDA;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = maxg;
    if (o.ctas_per_sm > 0) grid = std::min(grid, o.ctas_per_sm * sms);
    if (o.max_ctas > 0) grid = std::min(grid, o.max_ctas);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (ntiles + kSolveWarps - 1) / kSolveWarps));
    // each lane's exact inner-product partial holds one product per tile: keep
    // the tiles per warp below 2^16 so that it cannot overflow its 128 bits
    if ((ntiles + (int64_t)grid * kSolveWarps - 1) / ((int64_t)grid * kSolveWarps) >= (1 << 16)) {
        delete s;
        return BCS_ERR_ARG;
    }
    s->grid = grid;
    auto alloc = [&](void** p, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = BCS_ERR_OOM;
    };
    // vectors padded to whole 32-row tiles: the staging copies move full tiles
    const int64_t npad = ((n + 31) / 32) * 32 > 0 ? ((n + 31) / 32) * 32 : 32;
    alloc(&s->vecmem, (size_t)NVEC * npad * s->vbytes);
    if (s->layout == LAY_SELL) {
        alloc((void**)&s->x64w, sizeof(double) * nn);
        alloc((void**)&s->b64w, sizeof(double) * nn);
    }
    alloc((void**)&s->partials, sizeof(double) * 2 * (size_t)grid * NSLOT * kRec);
    alloc((void**)&s->bar, 64);
    alloc((void**)&s->hist, sizeof(double) * std::max(o.history_len, 1));
    alloc((void**)&s->scal, sizeof(double) * 4 * std::max(o.history_len, 1));
    alloc((void**)&s->out, sizeof(double) * NOUT);
    if (!rc && cudaMallocHost((void**)&s->host_out, sizeof(double) * NOUT + 64) != cudaSuccess) rc = BCS_ERR_OOM;
    if (!rc && (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess)) rc = BCS_ERR_CUDA;
    if (!rc && cudaMemset(s->partials, 0, sizeof(double) * 2 * (size_t)grid * NSLOT * kRec) != cudaSuccess) rc = BCS_ERR_CUDA;
    if (rc) {
        bcs_solver_destroy(s);
        return rc;
    }
    *out = s;
    return BCS_OK;
}

static void fill_params(bcs_solver s, const double* b, double* x, KParams* P) {
    bcs_matrix A = s->A;
    memset(P, 0, sizeof(*P));
    P->n = A->n;
    P->ntiles = (A->n + 31) / 32;
    P->kind = s->kind;
    P->maxit = s->maxit;
    P->rr_m = s->opt.rr_m;
    P->rr_M = s->opt.rr_M;
    P->max_outer = s->opt.max_outer;
    P->mixed = s->vt_f32;
    P->hist_cap = s->opt.history_len;
    P->inner_maxit = s->opt.inner_maxit;
    P->inner_stall = s->opt.inner_stall;
    P->tol = s->tol;
    P->inner_tol = s->opt.inner_tol;
    P->spin_budget = budget_cycles(s->opt.spin_budget_ms);
    if (s->layout == LAY_SELL) {
        P->slice_ptr = A->slice_ptr;
        P->col = A->scol;
        P->perm = A->perm;
        P->val64 = A->sval64;
        P->x64 = s->x64w;
        P->b64 = s->b64w;
        P->b64w = s->b64w;
    } else {
        P->rowptr = A->rowptr;
        P->col = A->col;
        P->val64 = A->val64;
        P->x64 = x;
        P->b64 = b;
    }
    P->val = inner_values(A, s->layout, s->valtype);
    P->b = b;
    P->x = x;
    const size_t npad = (size_t)std::max<int64_t>(((A->n + 31) / 32) * 32, 32);
    for (int v = 0; v < NVEC; ++v) P->vec[v] = (char*)s->vecmem + (size_t)v * npad * s->vbytes;
    P->partials = s->partials;
    P->bar = s->bar;
    P->err = (int*)(s->bar + 4);
    P->hist = s->hist;
    P->scal = s->scal;
    P->out = s->out;
}

static int finish(bcs_solver s, cudaStream_t st, bcs_result* res) {
    int herr = 0;
    if (cudaMemcpyAsync(s->host_out, s->out, sizeof(double) * NOUT, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return BCS_ERR_CUDA;
    if (cudaMemcpyAsync(s->host_out + NOUT, s->bar + 4, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return BCS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BCS_ERR_CUDA;
    memcpy(&herr, s->host_out + NOUT, sizeof(int));
    const double* o = s->host_out;
    int status = herr ? herr : (int)o[O_STATUS];
    s->hist_len = (int)o[O_HISTLEN];
    s->last_iters = (int)o[O_ITERS];
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = status;
        res->iterations = (int)o[O_ITERS];
        res->outer_steps = (int)o[O_OUTER];
        res->rr_steps = (int)o[O_RR];
        res->fallbacks = (int)o[O_FALLBACK];
        res->rel_res_recursive = o[O_RECREL];
        res->rel_res_true = o[O_TRUEREL];
        res->r0_norm = o[O_R0];
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev0, s->ev1) == cudaSuccess) res->seconds = ms * 1e-3;
    }
    return status;
}

static int launch(bcs_solver s, const double* b, double* x, cudaStream_t st) {
    KParams P;
    fill_params(s, b, x, &P);
    if (cudaMemsetAsync(s->bar, 0, 64, st) != cudaSuccess) return BCS_ERR_CUDA;
    if (cudaMemsetAsync(s->out, 0, sizeof(double) * NOUT, st) != cudaSuccess) return BCS_ERR_CUDA;
    cudaEventRecord(s->ev0, st);
    const int e = dispatch(&P, s->vt_f32, s->valtype, s->layout, s->tpr, s->grid, st, nullptr);
    cudaEventRecord(s->ev1, st);
    return e == 0 ? BCS_OK : BCS_ERR_CUDA;
}

int bcs_solve(bcs_solver s, const double* b_dev, double* x_dev, bcs_result* res, void* stream) {
    if (!s || (s->A->n > 0 && (!b_dev || !x_dev))) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->A->n == 0) {
        if (res) { memset(res, 0, sizeof(*res)); }
        return BCS_OK;
    }
    int rc = launch(s, b_dev, x_dev, st);
    if (rc) return rc;
    return finish(s, st, res);
}

int bcs_solve_host(bcs_solver s, const double* b_host, double* x_host, bcs_result* res, void* stream) {
    if (!s || (s->A->n > 0 && (!b_host || !x_host))) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = s->A->n;
    if (n == 0) {
        if (res) memset(res, 0, sizeof(*res));
        return BCS_OK;
    }
    if (!s->xb_dev && cudaMalloc(&s->xb_dev, sizeof(double) * 2 * n) != cudaSuccess) return BCS_ERR_OOM;
    double* bd = s->xb_dev;
    double* xd = s->xb_dev + n;
    if (cudaMemcpyAsync(bd, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) return BCS_ERR_CUDA;
    if (cudaMemcpyAsync(xd, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) return BCS_ERR_CUDA;
    int rc = launch(s, bd, xd, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(x_host, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess) return BCS_ERR_CUDA;
    return finish(s, st, res);
}

int bcs_get_history(bcs_solver s, double* out, int cap, int* len) {
    if (!s || cap < 0) return BCS_ERR_ARG;
    const int avail = std::min(s->hist_len, s->opt.history_len);
    if (len) *len = avail;
    const int m = std::min(avail, cap);
    if (out && m > 0 && cudaMemcpy(out, s->hist, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BCS_ERR_CUDA;
    return BCS_OK;
}

int bcs_get_scalars(bcs_solver s, double* out, int cap, int* len) {
    if (!s || cap < 0) return BCS_ERR_ARG;
    const int avail = std::min(s->hist_len, s->opt.history_len);
    if (len) *len = avail;
    const int m = std::min(avail, cap);
    if (out && m > 0 && cudaMemcpy(out, s->scal, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return BCS_ERR_CUDA;
    return BCS_OK;
}

int bcs_solve_batched(int nsys, const bcs_matrix* A, int kind, double tol, int maxit, const bcs_options* opt,
                      const double* const* b, double* const* x, bcs_result* res, void* stream) {
    if (nsys < 0 || (nsys > 0 && (!A || !b || !x))) return BCS_ERR_ARG;
    if (kind < BCS_SSBICGSAFE2 || kind > BCS_P_BICGSAFE_RR || !(tol >= 0.0) || maxit < 0) return BCS_ERR_ARG;
    if (nsys == 0) return BCS_OK;
    bcs_options o;
    if (opt) o = *opt; else bcs_options_default(&o);
    if (o.rr_M == 0) o.rr_M = maxit + 1;
    o.layout = BCS_LAYOUT_CSR;
    int rc = check_options(o);
    if (rc) return rc;
    int vt_f32 = 0, valtype = 0;
    int64_t maxn = 1;
    double sum_avg = 0.0;
    for (int k = 0; k < nsys; ++k) {
        if (!A[k] || !(A[k]->layouts & BCS_LAYOUT_CSR)) return BCS_ERR_ARG;
        if ((A[k]->n + 31) / 32 >= (int64_t)(1 << 16) * kWarps) return BCS_ERR_ARG;  // see bcs_solver_create
        if (A[k]->n > 0 && (!b[k] || !x[k])) return BCS_ERR_ARG;
        rc = precision_types(A[k], o.precision, &vt_f32, &valtype);
        if (rc) return rc;
        maxn = std::max(maxn, A[k]->n);
        sum_avg += A[k]->avg_row;
    }
    int tpr = o.threads_per_row;
    if (!tpr) {
        const double avg = sum_avg / nsys;
        tpr = vt_f32 ? 8 : 1;  // FP64: one lane per row keeps shuffle-adds off the FP64 units
        (void)avg;
    }
    if (tpr != 1 && tpr != 8) return BCS_ERR_ARG;
    const int csize = o.ctas_per_sm > 0 ? o.ctas_per_sm : 4;  // CTAs per cluster
    if (csize != 1 && csize != 2 && csize != 4 && csize != 8 && csize != 16) return BCS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vbytes = vt_f32 ? sizeof(float) : sizeof(double);
    // largest systems first
    std::vector<int> order(nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return A[a]->nnz + A[a]->n > A[c]->nnz + A[c]->n; });
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.nsys = nsys;
    B.csize = csize;
    int maxc = 0;
    if (dispatch_b(&B, vt_f32, valtype, tpr, 0, st, &maxc) != 0 || maxc <= 0) return BCS_ERR_CUDA;
    int nclusters = maxc;
    if (o.max_ctas > 0) nclusters = std::max(1, std::min(nclusters, o.max_ctas / csize));
    nclusters = std::min(nclusters, nsys);
    B.vec_bytes = ((size_t)maxn * vbytes + 255) / 256 * 256;
    B.ws_group_bytes = B.vec_bytes * NVEC;
    std::vector<KParams> hp(nsys);
    KParams* dsys = nullptr;
    int* dorder = nullptr;
    int* dctl = nullptr;
    char* ws = nullptr;
    double* parts = nullptr;
    double* outs = nullptr;
    std::vector<double> hout((size_t)nsys * NOUT);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    int herr = 0;
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && !rc) rc = BCS_ERR_CUDA; };
    ck(cudaMalloc(&dsys, sizeof(KParams) * nsys));
    ck(cudaMalloc(&dorder, sizeof(int) * nsys));
    ck(cudaMalloc(&dctl, sizeof(int) * (2 + nclusters)));  // counter, slots[nclusters], error word
    if (!rc && cudaMalloc(&ws, B.ws_group_bytes * nclusters) != cudaSuccess) rc = BCS_ERR_OOM;
    ck(cudaMalloc(&parts, sizeof(double) * 2 * NSLOT * kRec * csize * nclusters));
    ck(cudaMalloc(&outs, sizeof(double) * NOUT * nsys));
    if (!rc) {
        for (int k = 0; k < nsys; ++k) {
            KParams& P = hp[k];
            memset(&P, 0, sizeof(P));
            bcs_matrix M = A[k];
            P.n = M->n;
            P.ntiles = (M->n + 31) / 32;
            P.kind = kind;
            P.maxit = maxit;
            P.rr_m = o.rr_m;
            P.rr_M = o.rr_M;
            P.max_outer = o.max_outer;
            P.mixed = vt_f32;
            P.hist_cap = 0;
            P.inner_maxit = o.inner_maxit;
            P.inner_stall = o.inner_stall;
            P.tol = tol;
            P.inner_tol = o.inner_tol;
            P.rowptr = M->rowptr;
            P.col = M->col;
            P.val64 = M->val64;
            P.val = inner_values(M, LAY_CSR, valtype);
            P.b = b[k];
            P.x = x[k];
            P.x64 = x[k];
            P.b64 = b[k];
            P.out = outs + (size_t)k * NOUT;
            P.err = dctl + 1 + nclusters;
        }
        ck(cudaMemcpyAsync(dsys, hp.data(), sizeof(KParams) * nsys, cudaMemcpyHostToDevice, st));
        ck(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        ck(cudaMemsetAsync(dctl, 0, sizeof(int) * (2 + nclusters), st));
        ck(cudaMemsetAsync(outs, 0, sizeof(double) * NOUT * nsys, st));
        ck(cudaMemsetAsync(parts, 0, sizeof(double) * 2 * NSLOT * kRec * csize * nclusters, st));
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
    }
    if (!rc) {
        B.sys = dsys;
        B.order = dorder;
        B.counter = dctl;
        B.slots = dctl + 1;
        B.ws = ws;
        B.partials = parts;
        cudaEventRecord(e0, st);
        if (dispatch_b(&B, vt_f32, valtype, tpr, nclusters, st, nullptr) != 0) rc = BCS_ERR_CUDA;
        cudaEventRecord(e1, st);
        ck(cudaMemcpyAsync(hout.data(), outs, sizeof(double) * NOUT * nsys, cudaMemcpyDeviceToHost, st));
        ck(cudaMemcpyAsync(&herr, dctl + 1 + nclusters, sizeof(int), cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
        cudaEventElapsedTime(&ms, e0, e1);
    }
    int worst = herr ? herr : BCS_OK;
    if (!rc) {
        for (int k = 0; k < nsys; ++k) {
            const double* ob = hout.data() + (size_t)k * NOUT;
            const int stt = (int)ob[O_STATUS];
            if (stt < 0 && (worst >= 0 || stt < worst)) worst = stt;
            else if (stt > 0 && worst == BCS_OK) worst = stt;
            if (res) {
                bcs_result& r = res[k];
                memset(&r, 0, sizeof(r));
                r.status = stt;
                r.iterations = (int)ob[O_ITERS];
                r.outer_steps = (int)ob[O_OUTER];
                r.rr_steps = (int)ob[O_RR];
                r.fallbacks = (int)ob[O_FALLBACK];
                r.rel_res_recursive = ob[O_RECREL];
                r.rel_res_true = ob[O_TRUEREL];
                r.r0_norm = ob[O_R0];
                r.seconds = ms * 1e-3;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    void* ptrs[] = {dsys, dorder, dctl, ws, parts, outs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    return rc ? rc : worst;
}

}  // extern "C"
