// Partitioned-solve kernel, double vectors and FP64 matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_dist_f64(const DistArgs* D, int grid, cudaStream_t st, int* max_grid) {
    return dispatch_dist<double, double>(D, grid, st, max_grid);
}
}  // namespace bcs
