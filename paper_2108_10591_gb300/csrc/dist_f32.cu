// Partitioned-solve kernel, float vectors and FP32 matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_dist_f32(const DistArgs* D, int grid, cudaStream_t st, int* max_grid) {
    return dispatch_dist<float, float>(D, grid, st, max_grid);
}
}  // namespace bcs
