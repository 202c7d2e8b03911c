// Partitioned-solve kernel, float vectors and BF16 matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_dist_bf16(const DistArgs* D, int grid, cudaStream_t st, int* max_grid) {
    return dispatch_dist<float, uint16_t>(D, grid, st, max_grid);
}
}  // namespace bcs
