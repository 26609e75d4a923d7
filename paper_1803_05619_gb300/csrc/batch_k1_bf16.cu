// Persistent batched K1 for __nv_bfloat16 storage.
#include "batch_k1.cuh"

namespace dgf {
template cudaError_t k1_batched_kernel_t<__nv_bfloat16>(int, int, size_t, void**, int, int*);
}  // namespace dgf
