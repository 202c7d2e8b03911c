// Persistent solver kernels, float vectors and float matrix values (instantiation subset 1).
#include "solver.cuh"

namespace bcs {
int dispatch_f32_1(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<float, float, 1>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
