// K1 (low-resolution coefficients), column-walking form, radius 8.
#include "lowres_fast_launch.cuh"

namespace dgf {
template cudaError_t launch_k1_fast<8>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int, float,
                                       const LowCfg&, const TmaPair&, size_t, uint32_t*, float4*, cudaStream_t);
}  // namespace dgf
