/*
 * bcs_tune.h -- SELL-C-sigma sorting-window autotuner (a build addition: the
 * paper's experiments use CSR, Section 5).  Same conventions as bcs.h:
 * status codes, caller-owned host buffers, library-owned matrix objects.
 */
#ifndef BCS_TUNE_H
#define BCS_TUNE_H

#include "bcs.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * SELL-C-sigma keeps C = 32 (one warp per slice, one lane per row); sigma,
 * the window within which rows are sorted by length, trades padding against
 * locality.  For each sigma in sigmas[0..nsig) (multiples of 32, at most
 * 4096) a temporary copy of A with that SELL layout is uploaded and `iters`
 * iterations (0 = 20) of the persistent solver (method `kind`, `precision`,
 * layout SELL, tolerance 0, b = ones, x0 = 0) are timed; each candidate runs
 * twice and the second run is timed.  A is not modified (solvers that use it
 * stay valid).
 *   us_per_iter  host array of nsig doubles (may be NULL): device time per
 *                iteration of each candidate, in candidate order.
 *   best_sigma   receives the fastest sigma.
 *   tuned        (may be NULL) receives a new matrix with A's layouts and
 *                value stores and the SELL layout built at the fastest
 *                sigma; the caller frees it with bcs_matrix_free.
 * Synchronises the stream.  Errors: BCS_ERR_ARG (A or best_sigma NULL,
 * nsig <= 0, a sigma out of range, kind or precision invalid, A without the
 * value copy the precision needs), BCS_ERR_OOM, BCS_ERR_CUDA.
 */
int bcs_autotune_sell_sigma(bcs_matrix A, int kind, int precision, int iters, const int* sigmas, int nsig,
                            double* us_per_iter, int* best_sigma, bcs_matrix* tuned, void* stream);

#ifdef __cplusplus
}
#endif

#endif
