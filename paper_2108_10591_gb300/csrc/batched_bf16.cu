// Batched (one cluster per system) solver kernels with float vectors and uint16_t matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_batched_bf16(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters) {
    return dispatch_batched<float, uint16_t>(B, tpr, nclusters, st, max_clusters);
}
}  // namespace bcs
