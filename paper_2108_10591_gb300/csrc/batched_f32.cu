// Batched (one cluster per system) solver kernels with float vectors and float matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_batched_f32(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters) {
    return dispatch_batched<float, float>(B, tpr, nclusters, st, max_clusters);
}
}  // namespace bcs
