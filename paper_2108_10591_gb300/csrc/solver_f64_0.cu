// Persistent solver kernels, double vectors and double matrix values (instantiation subset 0).
#include "solver.cuh"

namespace bcs {
int dispatch_f64_0(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<double, double, 0>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
