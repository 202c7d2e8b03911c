// Persistent solver kernels with float vectors and float matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_f32(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<float, float>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
