// Persistent solver kernels, float vectors and uint16_t matrix values (instantiation subset 2: dynamic tile order).
#include "solver.cuh"

namespace bcs {
int dispatch_bf16_2(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<float, uint16_t, 2>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
