/*
 * bcs.h -- C ABI of the GB300 (sm_103a) pipelined BiCGSafe solver library.
 *
 * Solves nonsymmetric sparse A x = b with the single-reduction ssBiCGSafe2
 * method and its pipelined variants, after Huynh & Suito, "Communication-
 * hiding pipelined BiCGSafe methods for solving large linear systems"
 * (arXiv 2108.10591):
 *   BCS_SSBICGSAFE2    Section 2, Algorithm 3 (one phase of nine inner products)
 *   BCS_P_BICGSAFE     Section 3, Algorithm 4 (the inner-product phase of
 *                      iteration i overlaps the product A s_i; Eqs. (s)-(g))
 *   BCS_P_BICGSAFE_RR  Section 4, Algorithm 5 (residual replacement every m
 *                      iterations while i < M)
 * Every solve runs as one persistent CUDA kernel; the scalar recurrence
 * (alpha, beta, zeta, eta and the stop test) stays on the device.
 *
 * Conventions for every entry point:
 *  - Return value: BCS_OK (0) or a BCS_* status below; no exceptions, no
 *    process exit.  BCS_NOT_CONVERGED (positive) still leaves a valid best
 *    iterate in x.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device (for example a PyTorch tensor's
 *    data_ptr()).  The caller owns every buffer it passes; the library owns
 *    the matrix and solver objects and frees them in bcs_matrix_free /
 *    bcs_solver_destroy.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Objects are not thread-safe; a matrix may be shared by several solvers
 *    as long as it outlives them.
 *  - Vectors are FP64, length n, in the original row order, contiguous.
 */
#ifndef BCS_H
#define BCS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcs_matrix_s* bcs_matrix;
typedef struct bcs_solver_s* bcs_solver;
typedef struct bcs_batch_s* bcs_batch;

/* Methods (the paper's Algorithms 3, 4 and 5). */
enum { BCS_SSBICGSAFE2 = 0, BCS_P_BICGSAFE = 1, BCS_P_BICGSAFE_RR = 2 };

/* Precision of a solve.  BCS_FP64: vectors, matrix and arithmetic in FP64
 * (the paper's setting, Section 5).  BCS_FP32_REFINE / BCS_BF16MAT_REFINE:
 * inner solves with FP32 vectors and an FP32 / BF16 copy of the matrix
 * values, FP64 inner-product accumulation and FP64 scalars, wrapped in FP64
 * iterative refinement (r = b - A x with the FP64 matrix, x += d in FP64).
 * The paper has no counterpart of the two refinement modes. */
enum { BCS_FP64 = 0, BCS_FP32_REFINE = 1, BCS_BF16MAT_REFINE = 2 };

/* Matrix layouts held on the device (bit mask for bcs_csr_upload).
 * BCS_LAYOUT_AUTO (solver option only): the layout bcs_autotune chose for the
 * matrix and precision, CSR if it was not tuned. */
enum { BCS_LAYOUT_AUTO = 0, BCS_LAYOUT_CSR = 1, BCS_LAYOUT_SELL = 2 };
/* Preconditioning (no counterpart in the paper, which uses none: Section 5).
 * BCS_PRECOND_JACOBI: right preconditioning with D = diag(A): the solver runs
 * on A D^-1 y = b (scaled copies of the matrix values, built at
 * bcs_solver_create) and returns x = D^-1 y; x0 enters as y0 = D x0.  The
 * residual of the solved system equals b - A x, so tol keeps its meaning.
 * Requires every diagonal entry stored, nonzero and finite (else
 * BCS_ERR_ARG at bcs_solver_create).
 * BCS_PRECOND_BLOCK_JACOBI: right preconditioning with M = the diagonal blocks
 * of A, bcs_options.block_size consecutive rows each (the last block holds the
 * remaining rows): the solver runs on (A M^-1) y = b from y0 = M x0 and returns
 * x = M^-1 y.  The inverse blocks are formed at bcs_solver_create by
 * Gauss-Jordan elimination with partial pivoting (BCS_ERR_ARG for a singular
 * block).  M^-1 is not folded into the matrix: every vector that the solver
 * multiplies by A is also written as M^-1 v by the same pass that writes v
 * (the blocks lie inside the solver's 32-row tiles, so this needs no extra
 * barrier), and the products gather that copy.  Single-system solves with
 * CSR, one lane per row and the static tile order (the defaults, including
 * BCS_LAYOUT_AUTO on a matrix tuned to SELL, are adjusted; an explicit other
 * choice is BCS_ERR_ARG), all three kinds (the replacement
 * steps of BCS_P_BICGSAFE_RR form the copies of u, t, y, x and r they
 * multiply). */
enum { BCS_PRECOND_NONE = 0, BCS_PRECOND_JACOBI = 1, BCS_PRECOND_BLOCK_JACOBI = 2 };

/* Value copies held on the device (bit mask; FP64 is always kept). */
enum { BCS_STORE_F64 = 1, BCS_STORE_F32 = 2, BCS_STORE_BF16 = 4 };

/* Status codes. */
enum {
    BCS_OK = 0,
    BCS_NOT_CONVERGED = 1,  /* maxit (or max_outer) reached; x holds the last iterate */
    BCS_ERR_ARG = -1,       /* invalid argument or invalid CSR (see bcs_csr_upload) */
    BCS_ERR_CUDA = -2,      /* a CUDA call failed (includes no device) */
    BCS_ERR_BREAKDOWN = -3, /* zero denominator g+beta*h, zeta*f or (s,s) before convergence */
    BCS_ERR_TIMEOUT = -4,   /* a grid barrier waited past the spin budget */
    BCS_ERR_NONFINITE = -5, /* NaN or Inf in the scalar recurrence */
    BCS_ERR_OOM = -6        /* device allocation failed */
};

typedef struct {
    int rr_m;             /* Alg. 5 replacement epoch m (default 100; Section 5.2 uses 100 and 96) */
    int rr_M;             /* Alg. 5 replacement limit M: replace only while i < M (0, the default:
                             M = maxit + 1, no limit within the iteration budget) */
    int precision;        /* BCS_FP64 (default) | BCS_FP32_REFINE | BCS_BF16MAT_REFINE */
    double inner_tol;     /* refinement modes: inner stop at ||r_inner|| <= inner_tol*||r_outer|| (default 1e-2) */
    int max_outer;        /* outer steps: true-residual checks / restarts / refinement steps (default 30) */
    int history_len;      /* capacity of the residual history (default 4096 entries) */
    int layout;           /* BCS_LAYOUT_AUTO (default: tuned, else CSR), BCS_LAYOUT_CSR or BCS_LAYOUT_SELL
                             (must have been uploaded) */
    int threads_per_row;  /* CSR only: 1, 4, 8 or 32 lanes per row, or -1 = adaptive (one lane per row,
                             the whole warp for rows of more than 32 entries); 0 = the library's choice
                             (the tuned value, else -1 for heavy-tailed row lengths in the refinement
                             modes, else 1: one lane per row keeps FP64 sums in plain row order) */
    int ctas_per_sm;      /* single system: CTAs per SM, 0 = by occupancy (one 24-warp CTA); batched
                             solves: CTAs per cluster (one cluster per system), 0 = 2; 1..8 */
    int max_ctas;         /* 0 = no cap; otherwise an upper bound on the grid size */
    double spin_budget_ms;/* per grid-barrier wait before BCS_ERR_TIMEOUT (default 2000 ms) */
    int inner_maxit;      /* refinement modes: at most this many iterations per inner run (0 = no cap) */
    int inner_stall;      /* refinement modes: end an inner run after this many iterations without a new
                             smallest recursive residual (default 20; 0 = off); the FP64 outer step
                             then recomputes the true residual and starts a fresh Krylov space */
    int tile_order;       /* single system: 0 = library choice, 1 = static (tile t to warp t mod warps),
                             2 = dynamic (warps claim tiles from a counter); FP64 results do not depend on
                             it, refinement-mode results may in the last bits */
    int precond;          /* BCS_PRECOND_NONE (default), BCS_PRECOND_JACOBI or BCS_PRECOND_BLOCK_JACOBI
                             (single-system solves) */
    int big_ctas;         /* batched solves: 0 (default) = one lane; 2, 4, 8 or 16 = the largest systems
                             are solved concurrently by a second persistent launch whose clusters have
                             this many CTAs (larger than ctas_per_sm), so that the longest solves do not
                             run alone on two CTAs at the end of the batch */
    int big_systems;      /* batched solves with big_ctas: how many of the largest systems (by nnz + n)
                             take the second lane, one cluster each; 0 = as many clusters of big_ctas as
                             fit in a quarter of the device */
    int block_size;       /* BCS_PRECOND_BLOCK_JACOBI: rows per diagonal block, 1, 2, 4, 8, 16 or 32
                             (0 = the default, 8) */
} bcs_options;

typedef struct {
    int status;               /* BCS_* */
    int iterations;           /* total iterations over all inner runs (the paper's i at the stop) */
    int outer_steps;          /* true-residual evaluations (1 = converged on the first check) */
    int rr_steps;             /* residual replacements performed (Alg. 5) */
    int fallbacks;            /* iterations whose zeta, eta fell back to the i = 0 formulas */
    double rel_res_recursive; /* sqrt(r_i)/||r_0|| at the last stop test */
    double rel_res_true;      /* ||b - A x||_2 / ||b - A x_0||_2 in FP64 at exit */
    double r0_norm;           /* ||b - A x_0||_2 */
    double seconds;           /* device time of the solve (CUDA events) */
    int grid_syncs;           /* grid-wide (or cluster) barriers the solve passed */
    int reductions;           /* grid-wide reductions of inner-product partials (one per iteration,
                                 plus one per true-residual check) */
    int spmv_passes;          /* passes over the matrix (two per iteration, Table 1; plus set-up,
                                 true-residual checks and five per residual replacement) */
    double t_start, t_end;    /* device clock (ns, %globaltimer) when the solve of this system started and
                                 ended inside the kernel (batched solves: per system) */
} bcs_result;

/* Fill *opt with the defaults listed above. */
void bcs_options_default(bcs_options* opt);

/*
 * Copy a CSR matrix (host arrays) to the device and build the requested
 * layouts and value copies there.  Defines A of "Ax = b" (Section 2).
 *   n, nnz      rows (= columns) and nonzeros; 0 <= n, nnz < 2^31.
 *   rowptr      host int64[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = nnz.
 *   col         host int32[nnz], 0 <= col < n, strictly ascending within a row.
 *   val         host double[nnz].
 *   layouts     BCS_LAYOUT_CSR and/or BCS_LAYOUT_SELL.
 *   sell_C      SELL slice height; must be 32 (one warp per slice).
 *   sell_sigma  SELL sorting window, a positive multiple of sell_C (<= 4096).
 *               SELL-C-sigma: rows sorted by length, descending and stable,
 *               inside windows of sigma rows; slices stored column-major and
 *               padded with value 0 and the padded row's own index.
 *   stores      extra value copies (BCS_STORE_F32 rounds to nearest,
 *               BCS_STORE_BF16 rounds to nearest even); FP64 is always kept.
 * The CSR is validated on the device; any violation returns BCS_ERR_ARG
 * without fixing the input.  The library owns the returned matrix.
 */
int bcs_csr_upload(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                   const double* val, int layouts, int sell_C, int sell_sigma, int stores,
                   void* stream, bcs_matrix* out);

/* Sizes of an uploaded matrix (any pointer may be NULL). */
int bcs_matrix_info(bcs_matrix A, int64_t* n, int64_t* nnz, int64_t* sell_padded, int* layouts, int* stores);

/*
 * Copy the device-side format arrays back to host buffers (for bit-exact
 * checks of the format build).  Any pointer may be NULL.
 *   CSR : rowptr int32[n+1], col int32[nnz], val64 double[nnz], val32 float[nnz],
 *         valbf16 uint16[nnz] (BF16 bit patterns).
 *   SELL: perm int32[n] (original row at permuted position p), slice_ptr
 *         int64[n/32+1] (element offsets), scol int32[padded] (permuted
 *         column indices), sval64 double[padded].
 * Returns BCS_ERR_ARG if a requested layout or store is absent.
 */
int bcs_matrix_export(bcs_matrix A, int32_t* rowptr, int32_t* col, double* val64, float* val32,
                      uint16_t* valbf16, int32_t* perm, int64_t* slice_ptr, int32_t* scol,
                      double* sval64);

/*
 * y = A x on the device (the "MV" of Section 3 and Table 1).
 *   layout  BCS_LAYOUT_CSR or BCS_LAYOUT_SELL (must be uploaded).
 *   store   BCS_STORE_F64 / F32 / BF16: which value copy to use.
 *   x, y    device vectors of n elements in original row order, FP64 when
 *           vec_f32 == 0, FP32 otherwise; x and y must not overlap.
 *   threads_per_row  CSR lanes per row (1, 4, 8, 32, or -1 = adaptive; 0 = automatic).
 * Rows are summed with fused multiply-adds; with one lane per row (and for
 * SELL) in storage order.  Asynchronous on stream.  The SELL path permutes x
 * and y through a scratch buffer owned by A, so SELL calls on one matrix
 * must not run concurrently on different streams.  BCS_ERR_ARG when x or y
 * is not memory the device can read (see bcs_solve).
 */
int bcs_spmv(bcs_matrix A, int layout, int store, const void* x, void* y, int vec_f32,
             int threads_per_row, void* stream);

/*
 * Correctly rounded inner product (x, y) = sum_i x_i y_i of two device
 * vectors: the a_i ... r_i of Algorithms 3-5, computed the way the solver
 * computes them.  Each product is formed exactly as an integer and
 * accumulated in 128-bit fixed point on the integer units; the sum is rounded
 * once to nearest even, so the result does not depend on the order of the
 * terms or the launch configuration.  Bits more than about 2^-107 below the
 * largest product are dropped; they add up to at most n 2^-107 of it, so the
 * result is the correctly rounded one unless |(x, y)| falls below about
 * n 2^-54 times the largest |x_i y_i| (a cancellation of 2^34 for n = 10^6).
 *   n        number of elements (>= 0).
 *   x, y     device vectors, FP64 when vec_f32 == 0, FP32 otherwise.
 *   result   host double receiving the value (a NaN or Inf operand gives NaN).
 * Synchronises the stream; allocates and frees a small device buffer.
 * BCS_ERR_ARG when x or y is not memory the device can read (see bcs_solve).
 */
int bcs_dot(int64_t n, const void* x, const void* y, int vec_f32, double* result, void* stream);

/*
 * bcs_dot without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * whose device memory is all owned by another allocator (for example a
 * framework's caching allocator), or latency-sensitive loops in which a
 * cudaMalloc/cudaFree (which synchronise the device) would stall.  It runs
 * bcs_dot's kernels, but the per-CTA partial sums go to a fixed 128 KiB array
 * that the library holds on every GPU that loads it until the process exits
 * (at most 256 CTAs).  The value is the correctly rounded (x, y), as bcs_dot's
 * is, unless the sum cancels below about n 2^-54 of its largest product (see
 * bcs_dot): the dropped bits depend on how the terms are split over CTAs, and
 * the two calls split them differently, so under such cancellation their last
 * bits may differ.
 *   n           number of elements, 0 <= n <= 2^33 (BCS_ERR_ARG beyond that).
 *   x, y        device vectors, FP64 when vec_f32 == 0, FP32 otherwise.
 *   result_dev  device double receiving the value; written asynchronously on
 *               stream (synchronise before reading it).
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the process; make that first call before
 * any stream capture.  cudaDeviceReset unloads the library's device code, so
 * the kept address is no longer valid: do not call this entry point on a
 * device after resetting it in the same process.  All calls
 * share the one array, so calls that overlap on the GPU (different streams,
 * or different host threads on one device) race: serialise them.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.
 */
int bcs_dot_noalloc(int64_t n, const void* x, const void* y, int vec_f32, double* result_dev, void* stream);

/* Free a matrix (NULL is ignored).  Waits for the device first. */
void bcs_matrix_free(bcs_matrix A);

/*
 * Create a solver for A (Algorithm 3, 4 or 5 by kind).
 *   tol    epsilon of the stop test ||r_i|| <= eps ||r_0|| (Section 5; the
 *          paper uses 1e-8).  At recursive convergence the FP64 true residual
 *          is checked against the same bound and the method restarts from x
 *          while it is above (at most max_outer - 1 restarts).
 *   maxit  iteration limit over all inner runs (the paper uses 1e4).
 *   opt    NULL for defaults.
 * Allocates the Krylov workspace on the device (about 16 n-vectors).
 */
int bcs_solver_create(bcs_matrix A, int kind, double tol, int maxit, const bcs_options* opt,
                      bcs_solver* out);

/*
 * Solve A x = b.  b_dev: device double[n]; x_dev: device double[n], x_0 on
 * entry (the paper's experiments use x_0 = 0), the solution on exit.  Fills
 * *res (may be NULL).  Synchronises the stream before returning.
 * Before any launch, b_dev and x_dev are checked with cudaPointerGetAttributes:
 * device or managed memory, or page-locked host memory mapped for the
 * device, is accepted; anything else (for example pageable host memory,
 * which a kernel would read as a device address) gives BCS_ERR_ARG.
 */
int bcs_solve(bcs_solver s, const double* b_dev, double* x_dev, bcs_result* res, void* stream);

/*
 * Same as bcs_solve with host buffers: copies b and x_0 to the device, solves
 * and copies x back, all on stream (end-to-end entry point).
 */
int bcs_solve_host(bcs_solver s, const double* b_host, double* x_host, bcs_result* res, void* stream);

/*
 * Relative recursive residuals sqrt(r_i)/||r_0|| of the last solve, one per
 * evaluated stop test (all inner runs), and the scalars alpha, beta, zeta,
 * eta of the first inner run (4 per iteration).  out/scal may be NULL;
 * *len receives the number of entries available (capped by history_len).
 */
int bcs_get_history(bcs_solver s, double* out, int cap, int* len);
int bcs_get_scalars(bcs_solver s, double* out, int cap, int* len);

/*
 * Block-Jacobi solvers (BCS_PRECOND_BLOCK_JACOBI): copy the diagonal blocks D
 * and their inverses E to host buffers of n * block_size doubles each (either
 * may be NULL).  Row i of the block that starts at row b0 and holds m rows
 * stores its m entries in the block's columns b0 .. b0+m-1 at
 * i * block_size + j, j < m, and zero for j >= m.  *bs receives block_size
 * (may be NULL).  BCS_ERR_ARG for a solver without block-Jacobi
 * preconditioning.  Synchronous (waits for the device).  No counterpart in the
 * paper (a build addition, like the preconditioner itself).
 */
int bcs_solver_precond_blocks(bcs_solver s, double* D, double* E, int* bs);

/* Free a solver (NULL is ignored).  Waits for the device first (a solve still
 * in flight on any stream finishes before its workspace is released). */
void bcs_solver_destroy(bcs_solver s);

/*
 * Solve nsys independent systems A[k] x[k] = b[k] in one persistent launch
 * (no counterpart in the paper: it solves one system at a time).  Each
 * system is handled by one thread-block cluster, taken from a work list in
 * decreasing size; a system retires as soon as it converges.
 *   A      host array of nsys matrix handles (CSR layout).
 *   b, x   host arrays of nsys device pointers (double[n_k] each).
 *   res    host array of nsys results (may be NULL).
 *   kind, tol, maxit, opt as for bcs_solver_create (opt->precision selects
 *   FP64 or FP32 + FP64 refinement; history is not recorded).
 * Synchronises the stream before returning.  Returns the worst status.
 */
int bcs_solve_batched(int nsys, const bcs_matrix* A, int kind, double tol, int maxit,
                      const bcs_options* opt, const double* const* b, double* const* x,
                      bcs_result* res, void* stream);

/*
 * Reusable batched solve (no counterpart in the paper).  bcs_batch_create
 * validates the nsys matrices and options exactly as bcs_solve_batched,
 * allocates the workspace once and fixes the work order (largest systems
 * first); bcs_batch_solve then solves the same systems for new right-hand
 * sides: b[k], x[k] as for bcs_solve_batched (x[k] in: x0, out: solution).
 * The first solve captures the launch sequence (parameter upload, counter
 * resets, the persistent kernel, result download) in a CUDA graph that later
 * solves replay; if capture is not possible the sequence is issued directly.
 * bcs_batch_solve synchronises the stream and returns the worst status; a
 * handle is not thread-safe and runs one solve at a time.  Every b[k], x[k]
 * is checked as in bcs_solve (BCS_ERR_ARG before any launch).  The matrices must
 * outlive the handle.  bcs_batch_destroy(NULL) is ignored.
 * Errors: BCS_ERR_ARG (invalid arguments), BCS_ERR_OOM, BCS_ERR_CUDA.
 */
int bcs_batch_create(int nsys, const bcs_matrix* A, int kind, double tol, int maxit,
                     const bcs_options* opt, bcs_batch* out);
int bcs_batch_solve(bcs_batch bt, const double* const* b, double* const* x, bcs_result* res, void* stream);
void bcs_batch_destroy(bcs_batch bt);

/* One measured candidate of the autotuner. */
typedef struct {
    int layout;            /* BCS_LAYOUT_CSR or BCS_LAYOUT_SELL */
    int threads_per_row;   /* CSR lanes per row (1 for SELL) */
    int cluster_ctas;      /* batched: CTAs per cluster; 0 for single-system candidates */
    double us_per_iter;    /* device time per iteration (single system) or per batch iteration */
} bcs_tune_entry;

/*
 * Autotuner (no counterpart in the paper).  Times `iters` iterations (0 = 20)
 * of the persistent solver of method `kind` in `precision` (tolerance 0, one
 * run, b = ones, x0 = 0) for every candidate the matrix supports: CSR with 1,
 * 4, 8 or 32 lanes per row or adaptive lanes (-1), and SELL-C-sigma if
 * uploaded; each candidate
 * is run twice and the second run timed.  The fastest is recorded in A for
 * that precision: solvers created later with layout BCS_LAYOUT_AUTO and
 * threads_per_row 0 use it, and bcs_spmv uses its lanes per row.
 *   entries   host array of cap entries (may be NULL): the measurements,
 *             in candidate order; *count (may be NULL) the number of candidates.
 *   best      (may be NULL) the chosen candidate.
 * Synchronises the stream.  Errors: BCS_ERR_ARG, BCS_ERR_OOM, BCS_ERR_CUDA.
 */
int bcs_autotune(bcs_matrix A, int kind, int precision, int iters, bcs_tune_entry* entries, int cap,
                 int* count, bcs_tune_entry* best, void* stream);

/*
 * Batched autotuner: times `iters` iterations (0 = 20) per system of the
 * batched solve of the nsys systems for CSR lanes per row 1 and 8 and
 * clusters of 1, 2, 4 and 8 CTAs, with the other settings taken from opt
 * (may be NULL).  *best_opt (required) receives opt with the fastest
 * threads_per_row and ctas_per_sm (CTAs per cluster) filled in, ready for
 * bcs_batch_create.  entries, cap, count as for bcs_autotune.
 */
int bcs_batch_autotune(int nsys, const bcs_matrix* A, int kind, const bcs_options* opt, int iters,
                       bcs_tune_entry* entries, int cap, int* count, bcs_options* best_opt, void* stream);

/* Static English name of a status code. */
const char* bcs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BCS_H */
