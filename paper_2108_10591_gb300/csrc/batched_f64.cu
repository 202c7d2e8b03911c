// Batched (one cluster per system) solver kernels with double vectors and double matrix values.
#include "solver.cuh"

namespace bcs {
int dispatch_batched_f64(const BatchArgs* B, int tpr, int nclusters, cudaStream_t st, int* max_clusters) {
    return dispatch_batched<double, double>(B, tpr, nclusters, st, max_clusters);
}
}  // namespace bcs
