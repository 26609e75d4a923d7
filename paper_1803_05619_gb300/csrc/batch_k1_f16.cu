// Persistent batched K1 for __half storage.
#include "batch_k1.cuh"

namespace dgf {
template cudaError_t k1_batched_kernel_t<__half>(int, int, size_t, void**, int, int*);
}  // namespace dgf
