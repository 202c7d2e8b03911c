/*
 * bcs_dist.h -- the row-partitioned solve (Section 3 and Section 5.3 of
 * Huynh & Suito, arXiv 2108.10591: every process owns a contiguous block of
 * rows and its slice of every Krylov vector; each iteration needs a halo
 * exchange before each matrix-vector product and one global reduction of the
 * nine inner products, which the pipelined methods overlap with A s_i).
 *
 * Ranks here are groups of CTAs of one cooperative launch on one GPU: every
 * rank has its own row block (local CSR with renumbered columns), its own
 * Krylov vectors with halo space, and pushes the boundary values that other
 * ranks need directly into their halo buffers as it computes them; the exact
 * per-CTA inner-product records of all ranks are summed in one fixed order,
 * so every rank obtains bitwise the same scalars.  The inner products are
 * exact sums rounded once, and every row is summed in its CSR order, so a
 * partitioned FP64 solve is bit-identical to the unpartitioned one (and to
 * the CPU oracle) for any number of ranks.
 *
 * Error codes, options and results are those of bcs.h.
 */
#ifndef BCS_DIST_H
#define BCS_DIST_H

#include <stdint.h>

#include "bcs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest number of ranks of a partitioned solve. */
#define BCS_DIST_MAX_RANKS 16

/*
 * Contiguous row blocks balanced by work: rank k owns rows
 * [bounds[k], bounds[k+1]), bounds[0] = 0, bounds[nparts] = n, and the blocks
 * split the weight nnz + n (every nonzero and every row of Krylov vector
 * work) as evenly as whole rows allow.
 *   rowptr  host int64[n+1], monotone, rowptr[0] = 0.
 *   bounds  host int64[nparts+1] (output).
 * BCS_ERR_ARG for n < 0, nparts outside 1..BCS_DIST_MAX_RANKS or a
 * non-monotone rowptr.  Host code only; no device is needed.
 */
int bcs_partition_rows(int64_t n, const int64_t* rowptr, int nparts, int64_t* bounds);

/*
 * The halo plan of one rank (host code only; no device is needed).  Rank r
 * owns rows [bounds[r], bounds[r+1]); nloc = bounds[r+1] - bounds[r] and
 * npad = nloc rounded up to a multiple of 32.  Its vectors are extended by a
 * left halo at offsets [-nleft, 0) and a right halo at [npad, npad + nright),
 * offsets counted from its first owned row: the left halo holds, in
 * ascending order, the columns below bounds[r] that its rows reference, the
 * right halo those at or above bounds[r+1].
 *   local_col   int32[nnz of the block] (or NULL): the block's column indices
 *               in that offset space, in CSR order (ascending within a row,
 *               like the input).
 *   left_cols, right_cols  int64[nleft], int64[nright] (or NULL): the global
 *               columns of the halo entries.
 *   send_row, send_rank, send_off  [nsend] each (or NULL): the values this
 *               rank sends before each matrix-vector product, one entry per
 *               (owned row, receiving rank) pair, sorted by row then rank:
 *               local row, receiving rank, and the offset in the receiver's
 *               offset space at which the value lands.
 * Call with NULL arrays first to obtain nleft, nright and nsend.
 * rowptr int64[n+1], col int32[nnz] (0 <= col < n, ascending within rows).
 * BCS_ERR_ARG on invalid arguments.
 */
int bcs_halo_plan(int64_t n, const int64_t* rowptr, const int32_t* col, int nparts, const int64_t* bounds,
                  int rank, int64_t* nleft, int64_t* nright, int64_t* nsend, int32_t* local_col, int64_t* left_cols,
                  int64_t* right_cols, int32_t* send_row, int32_t* send_rank, int64_t* send_off);

typedef struct bcs_dist_s* bcs_dist;

/*
 * A partitioned solver for A (host CSR, validated like bcs_csr_upload) over
 * nparts ranks on the current device.  bounds: host int64[nparts+1] as from
 * bcs_partition_rows, or NULL to use bcs_partition_rows.  kind, tol, maxit
 * and opt as for bcs_solver_create; the layout is CSR with one lane per row
 * and the tile order static (other values of those options are refused);
 * opt->precision selects FP64 or the FP32 / BF16 refinement modes.  The
 * device's co-resident CTAs are shared among the ranks in proportion to
 * their rows (at least one each).  Copies the matrix; the caller keeps its
 * arrays.  BCS_ERR_OOM when the device memory runs out.
 */
int bcs_dist_create(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                    int nparts, const int64_t* bounds, int kind, double tol, int maxit, const bcs_options* opt,
                    bcs_dist* out);

/*
 * Solve A x = b with the partitioned solver: b_dev, x_dev device double[n]
 * in the original row order (x_dev holds x_0 on entry, x on exit); every
 * rank copies its rows in and out.  One cooperative launch on stream; fills
 * *res like bcs_solve (the counters are those of every rank, which agree).
 * Synchronises the stream.  b_dev and x_dev are checked as in bcs_solve.
 */
int bcs_dist_solve(bcs_dist d, const double* b_dev, double* x_dev, bcs_result* res, void* stream);

/* Relative recursive residual history and (alpha, beta, zeta, eta) of the
 * last solve, as bcs_get_history / bcs_get_scalars. */
int bcs_dist_get_history(bcs_dist d, double* out, int cap, int* len);
int bcs_dist_get_scalars(bcs_dist d, double* out, int cap, int* len);

/*
 * One rank per process and GPU (the multi-GPU form of the same solve).  Every
 * process calls bcs_dist_rank_create with the same matrix, nparts and bounds
 * and its own rank, on its own device (the devices are taken to be alike: each
 * rank uses all co-resident CTAs of its GPU).  Each rank's vectors, FP64 x,
 * inner-product records and barrier word live in one device arena; the ranks
 * exchange its CUDA IPC handle (bcs_dist_rank_export, BCS_DIST_HANDLE_BYTES
 * bytes, e.g. through torch.distributed.all_gather_object) and every rank
 * opens the others' (bcs_dist_rank_connect, handles in rank order; needs peer
 * access between the GPUs, e.g. NVLink).  The halo values are then stored
 * straight into the other GPUs' memory and all ranks meet at rank 0's barrier
 * counter with system-scope release/acquire; every rank sums all ranks'
 * records (in rank 0's arena) in the same order.  bcs_dist_solve then runs on
 * every process at about the same time (a rank that starts more than
 * spin_budget_ms after the others makes them return BCS_ERR_TIMEOUT; after
 * any error, destroy and re-create the solvers on every rank); b_dev and
 * x_dev are full-length on every process's device, and each rank writes its
 * own rows of x.  Not measured: the machines this library was built on give
 * every run one GPU, so only the one-rank form of this path has run.
 */
#define BCS_DIST_HANDLE_BYTES 64
int bcs_dist_rank_create(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                         int nparts, const int64_t* bounds, int rank, int kind, double tol, int maxit,
                         const bcs_options* opt, bcs_dist* out);
int bcs_dist_rank_export(bcs_dist d, void* handle);
int bcs_dist_rank_connect(bcs_dist d, const void* handles);

/* Rank r's block and halo sizes and its number of CTAs (any pointer may be NULL;
 * a process of the multi-GPU form knows its own rank only). */
int bcs_dist_info(bcs_dist d, int rank, int64_t* row0, int64_t* nloc, int64_t* nleft, int64_t* nright,
                  int64_t* nsend, int* ctas);

/* Free the solver (NULL is ignored).  Waits for the device first. */
void bcs_dist_destroy(bcs_dist d);

#ifdef __cplusplus
}
#endif

#endif /* BCS_DIST_H */
