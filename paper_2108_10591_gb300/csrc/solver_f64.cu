// Persistent solver kernels with double vectors and double matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_f64(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<double, double>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
