// K4 (low-resolution backward), column-walking form, radius 4.
#include "lowres_fast_launch.cuh"

namespace dgf {
template cudaError_t launch_k4_fast<4>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*, int,
                                       int, int, float, const LowCfg&, const TmaTriple*, uint32_t*, const float4*,
                                       cudaStream_t);
}  // namespace dgf
