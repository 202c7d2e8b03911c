// Persistent solver kernels with float vectors and uint16_t matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_bf16(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<float, uint16_t>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
