// Persistent solver kernels, double vectors and double matrix values (instantiation subset 1).
#include "solver.cuh"

namespace bcs {
int dispatch_f64_1(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<double, double, 1>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
