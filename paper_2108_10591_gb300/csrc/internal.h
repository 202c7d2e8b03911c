// Internal declarations shared by the translation units of libbcs.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bcs.h"

namespace bcs {

// Named range on the profiler timeline (NVTX) for the duration of a scope;
// costs a branch when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Slots of the per-CTA inner-product partials (Alg. 3/4: a..h and r; plus the
// FP64 true-residual norm of the outer step).
enum Slot { SA = 0, SB, SC, SD, SE, SF, SG, SH, SR, ST, NSLOT_USED, NSLOT = 16 };

// Krylov vectors of one solve (VT = double in FP64 mode, float in the
// refinement modes).  s and s2 alternate between iterations.
enum Vec { V_R = 0, V_RS, V_S, V_S2, V_Y, V_T, V_P, V_U, V_Z, V_W, V_L, V_G, V_O, V_BIN, V_D, NVEC };

// Result block written by CTA 0 at the end of a solve (device memory).
enum Out { O_STATUS = 0, O_ITERS, O_OUTER, O_RR, O_FALLBACK, O_RECREL, O_TRUEREL, O_R0, O_HISTLEN, O_SYNCS, O_REDUCTIONS,
           O_SPMV, O_T0, O_T1, NOUT = 16 };

enum Layout { LAY_CSR = 0, LAY_SELL = 1 };
enum ValType { VAL_F64 = 0, VAL_F32 = 1, VAL_BF16 = 2 };

constexpr int kBlock = 256;            // threads per CTA of the batched solver and the dot kernels
constexpr int kWarps = kBlock / 32;
// The single-system persistent solver runs one CTA of 24 warps per SM: one
// exact partial record per SM keeps the grid-wide reduction short.
constexpr int kSolveWarps = 24;
constexpr int kSolveBlock = kSolveWarps * 32;

struct KParams {
    int64_t n;
    int64_t ntiles;         // 32-row tiles
    int kind, maxit, rr_m, rr_M, max_outer, mixed, hist_cap;
    int inner_maxit, inner_stall;  // refinement modes: inner-run cap and stall window (0 = off)
    double tol, inner_tol;
    long long spin_budget;  // clock64 cycles per barrier wait
    // matrix: CSR (rowptr, col, val) or SELL (slice_ptr, col=scol, val=sval, perm)
    const int32_t* rowptr;
    const int32_t* col;
    const void* val;        // inner-solve value type (MT)
    const double* val64;    // FP64 values (outer residual)
    const int32_t* perm;    // SELL: original row of permuted position; nullptr for CSR
    const int64_t* slice_ptr;
    // caller vectors (original order)
    const double* b;
    double* x;
    // FP64 working vectors in the solve's row order (== b, x for CSR)
    double* x64;
    const double* b64;
    double* b64w;           // SELL: writable permuted copy of b
    void* vec[NVEC];
    double* partials;       // exact partial records: [2][CTAs][NSLOT][kRec = 4] 64-bit words
    unsigned* bar;          // barrier counter, zero at launch
    unsigned* tilectr;      // two tile counters (dynamic tile order), zero at launch; nullptr: static order
    int* err;               // error flag, zero at launch
    double* hist;           // [hist_cap]
    double* scal;           // [4*hist_cap]
    double* out;            // [NOUT]
    int l2hint;             // launch the L2-hinted kernel (FP32 vectors, CSR, one lane per row; see l2_hint_pays)
    int wa_hi;              // FP64, static order: the kernel whose inner-product terms sit 12 bits higher
                            // (wa_acc shift 14; at most 64 products per lane)
    // block-Jacobi right preconditioning (bs = 0: none): M^-1 in the inner
    // value type and in FP64, [rows][bs] in block columns (rows padded to
    // whole tiles, zero there); the M^-1 copies of r, s, s2, w, u, t, y and the
    // inner iterate (inner type) and of the FP64 iterate
    int bs;
    const void* bj;
    const double* bj64;
    void* hat[8];
    double* xhat64;
    // row-partitioned solve (include/bcs_dist.h): this rank's first global
    // row, which of its rows other ranks need (per local row: entries
    // send_ptr[row] .. send_ptr[row+1] of send_dst = (rank, offset in that
    // rank's vectors)), whether a tile has such rows, and every rank's vectors
    // ([rank][NVEC + 1], the FP64 x last); the caller's b and x in global rows.
    int64_t row0;
    const int32_t* send_ptr;
    const int2* send_dst;
    const unsigned char* tile_send;
    void* const* peer_vec;
    const double* bg;
    double* xg;
};

constexpr int kDistMaxRanks = 16;   // BCS_DIST_MAX_RANKS

// True when the current device can dereference p: device or managed memory, or
// page-locked host memory mapped into the device's address space.  The entry
// points that take device vectors refuse anything else (plain pageable host
// memory would be read by a kernel as a device address).
bool device_reachable(const void* p);
// Whether a solve with FP32 vectors of `rows` padded rows (all ranks together)
// should mark its single-use streams evict_first (KParams::l2hint).
bool l2_hint_pays(int vt_f32, int64_t rows);
// A partitioned solve: CTAs [cta0[r], cta0[r+1]) of the cooperative grid form
// rank r, whose parameters are params[r].
struct DistArgs {
    const KParams* params;
    int cta0[kDistMaxRanks + 1];
    int nranks;
    // records and barrier: this launch's CTAs are rec_offset .. rec_offset +
    // gridDim - 1 of rec_total (one launch per GPU: rank * CTAs per rank, of
    // ranks * CTAs per rank); the barrier counter has passed bar_base barriers
    int rec_offset, rec_total;
    unsigned bar_base;
    int sys;   // the ranks are on several GPUs: system-scope barrier
};

// Batched solves: the systems' parameter blocks (without workspace), their
// order, the work-list counter and each cluster's current system, and the
// clusters' workspace (NVEC vectors of vec_bytes each) and partials.
struct BatchArgs {
    const KParams* sys;
    const int* order;
    int nsys;
    int* counter;
    int* slots;
    char* ws;
    size_t ws_group_bytes, vec_bytes;
    double* partials;
    int csize;
};

}  // namespace bcs

struct bcs_matrix_s {
    int64_t n = 0, nnz = 0;
    int layouts = 0, stores = 0;
    int device = 0;
    // CSR
    int32_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val64 = nullptr;
    float* val32 = nullptr;
    uint16_t* valbf16 = nullptr;
    // SELL-C-sigma
    int sell_C = 32, sell_sigma = 0;
    int64_t nslices = 0, padded = 0;
    int32_t* perm = nullptr;
    int64_t* slice_ptr = nullptr;
    int32_t* scol = nullptr;
    double* sval64 = nullptr;
    float* sval32 = nullptr;
    uint16_t* svalbf16 = nullptr;
    double* scratch = nullptr;   // 2n doubles: permuted x and y of bcs_spmv on SELL
    // row-length statistics (threads-per-row choice)
    double avg_row = 0;
    int max_row = 0;
    int tuned_tpr[3] = {0, 0, 0};     // per precision (BCS_FP64, BCS_FP32_REFINE, BCS_BF16MAT_REFINE)
    int tuned_layout[3] = {0, 0, 0};  // BCS_LAYOUT_CSR / BCS_LAYOUT_SELL, 0 = not tuned
};

struct bcs_solver_s {
    bcs_matrix A = nullptr;
    int kind = 0, maxit = 0;
    double tol = 0;
    bcs_options opt;
    int vt_f32 = 0, valtype = 0, layout = 0, tpr = 1, dyn = 0;
    int l2hint = 0;               // KParams::l2hint
    int grid = 0;
    size_t vbytes = 0;
    void* vecmem = nullptr;       // NVEC vectors
    double* x64w = nullptr;       // SELL: permuted x (FP64)
    double* b64w = nullptr;       // SELL: permuted b (FP64)
    double* partials = nullptr;
    unsigned* bar = nullptr;      // [1] counter, [2] error flag as int (same allocation)
    double* hist = nullptr;
    double* scal = nullptr;
    double* out = nullptr;
    double* host_out = nullptr;   // pinned copy of out
    double* xb_dev = nullptr;     // bcs_solve_host staging (2n doubles), allocated on first use
    int precond = 0;              // BCS_PRECOND_*
    double* pdiag = nullptr;      // Jacobi: diag(A) in the caller's row order
    double* pval64 = nullptr;     // Jacobi: A D^-1 in the solver's layout, FP64
    void* pvalin = nullptr;       // Jacobi: A D^-1 in the inner value type (refinement modes)
    int bj_bs = 0;                // block-Jacobi: rows per block (0: not block-Jacobi)
    double* bjD = nullptr;        // block-Jacobi: the diagonal blocks, [npad][bs] FP64
    double* bjE = nullptr;        // block-Jacobi: their inverses, [npad][bs] FP64
    float* bjE32 = nullptr;       // block-Jacobi: the inverses in FP32 (refinement modes)
    void* bjhat = nullptr;        // block-Jacobi: eight M^-1 copies in the inner vector type
    double* bjxh = nullptr;       // block-Jacobi: M^-1 y (FP64)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int hist_len = 0;
    int last_iters = 0;
};

// A reusable batched solve (bcs_batch_create): workspace, parameter blocks and
// the captured launch sequence live as long as the handle.
struct bcs_batch_s {
    int nsys = 0, vt_f32 = 0, valtype = 0, tpr = 1, nclusters = 0;
    std::vector<int64_t> n;
    bcs::BatchArgs B;
    // the second lane (bcs_options::big_ctas): the largest systems, bigger clusters,
    // launched on a side stream concurrently with the first lane
    int nbig = 0, nclusters2 = 0;
    bcs::BatchArgs B2;
    int* dctl2 = nullptr;
    char* ws2 = nullptr;
    double* parts2 = nullptr;
    int* herr2 = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    bcs::KParams* hp = nullptr;   // pinned [nsys]
    bcs::KParams* dsys = nullptr;
    int* dorder = nullptr;
    int* dctl = nullptr;
    char* ws = nullptr;
    double* parts = nullptr;
    double* outs = nullptr;
    double* hout = nullptr;       // pinned [nsys * NOUT] + error word
    int* herr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_failed = 0;
};
