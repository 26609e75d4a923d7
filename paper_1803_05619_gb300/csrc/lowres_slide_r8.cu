// Sliding-sum K1 and K4 for radius 8 (explicit instantiation).
#include "lowres_slide_launch.cuh"

namespace dgf {
template cudaError_t launch_k1_slide_r<8>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int, float,
                                           int, int, cudaStream_t);
template cudaError_t launch_k4_slide_r<8>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*,
                                           int, int, int, float, int, int, cudaStream_t);
}  // namespace dgf
