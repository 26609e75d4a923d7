// Persistent batched K1 for float storage.
#include "batch_k1.cuh"

namespace dgf {
template cudaError_t k1_batched_kernel_t<float>(int, int, size_t, void**, int, int*);
}  // namespace dgf
