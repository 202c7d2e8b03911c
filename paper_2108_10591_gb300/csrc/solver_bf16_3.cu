// Persistent solver kernels, float vectors and uint16_t matrix values, block-Jacobi
// right preconditioning (instantiation subset 3).
#include "solver.cuh"

namespace bcs {
int dispatch_bf16_3(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<float, uint16_t, 3>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
