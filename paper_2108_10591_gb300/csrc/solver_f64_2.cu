// Persistent solver kernels, double vectors and double matrix values (instantiation subset 2: dynamic tile order).
#include "solver.cuh"

namespace bcs {
int dispatch_f64_2(const KParams* P, int layout, int tpr, int grid, cudaStream_t st, int* max_grid) {
    return dispatch<double, double, 2>(P, layout, tpr, grid, st, max_grid);
}
}  // namespace bcs
