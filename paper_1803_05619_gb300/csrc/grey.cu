// Grey guide of Sec. 4.2 (DGF_b): when the guide has n_I channels and the
// output C != n_I, the transformation F is the mean over the guide's
// channels, and that one grey plane guides every output channel.
//   KG   G[n, c] = (sum over k of I[n, k]) / n_I for every c < C, held in
//        FP32 (no rounding to the storage type: the layer reads this guide
//        as FP32 whatever the storage type of its other tensors)
//   KGT  the adjoint: d I[n, k] = (sum over c of d G[n, c]) / n_I for every
//        k < n_I (the channel mean hands 1 / n_I of the summed gradient to
//        each guide channel), stored in the storage type (the low-res
//        guide gradients it sums are FP32, as K4 writes them for an FP32 guide)
// Both are streaming passes over whole planes: each thread moves VEC
// consecutive pixels of one image (16-byte vectors of the source when every
// plane start is aligned), the channels summed in order in FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace dgf {

// KG and KGT: dst[n, j] = (sum over i < n_src of src[n, i]) / n_I for every
// j < n_dst (KG: TD = float).
template <typename TS, typename TD, int VEC>
__global__ void __launch_bounds__(kThreads) k_grey(const TS* __restrict__ src, TD* __restrict__ dst, int N,
                                                   int n_src, int n_dst, int n_in, size_t plane) {
    const size_t nv = plane / VEC, total = (size_t)N * nv;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const size_t n = v / nv, px = (v - n * nv) * VEC;
        float s[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) s[k] = 0.f;
        for (int i = 0; i < n_src; ++i) {
            float x[VEC];
            load_vec<TS, VEC>(src + (n * n_src + i) * plane + px, x);
#pragma unroll
            for (int k = 0; k < VEC; ++k) s[k] = __fadd_rn(s[k], x[k]);
        }
        float g[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[k] = n_in == 1 ? s[k] : __fdiv_rn(s[k], (float)n_in);
        for (int j = 0; j < n_dst; ++j) store_vec<TD, VEC>(dst + (n * n_dst + j) * plane + px, g);
    }
}

template <typename TS, typename TD>
static cudaError_t grey_go(const void* src, void* dst, int N, int n_src, int n_dst, int n_in, size_t plane,
                           cudaStream_t s) {
    constexpr int V16 = 16 / (int)sizeof(TS);
    constexpr size_t kAlign = V16 * sizeof(TD) > V16 * sizeof(TS) ? V16 * sizeof(TD) : V16 * sizeof(TS);
    const bool wide = plane % V16 == 0 && reinterpret_cast<uintptr_t>(src) % kAlign == 0 &&
                      reinterpret_cast<uintptr_t>(dst) % kAlign == 0;
    const size_t vecs = (size_t)N * (wide ? plane / V16 : plane);
    const int blocks = (int)std::min<size_t>((vecs + kThreads - 1) / kThreads, (size_t)152 * 16);
    if (blocks == 0) return cudaSuccess;
    if (wide)
        k_grey<TS, TD, V16><<<blocks, kThreads, 0, s>>>(static_cast<const TS*>(src), static_cast<TD*>(dst), N, n_src,
                                                        n_dst, n_in, plane);
    else
        k_grey<TS, TD, 1><<<blocks, kThreads, 0, s>>>(static_cast<const TS*>(src), static_cast<TD*>(dst), N, n_src,
                                                      n_dst, n_in, plane);
    return cudaGetLastError();
}

cudaError_t launch_grey_mean(dgf_dtype dt, const void* I, float* G, int N, int n_in, int C, size_t plane,
                             cudaStream_t s) {
    if (N == 0 || plane == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return grey_go<float, float>(I, G, N, n_in, C, n_in, plane, s);
        case DGF_BF16: return grey_go<__nv_bfloat16, float>(I, G, N, n_in, C, n_in, plane, s);
        case DGF_F16: return grey_go<__half, float>(I, G, N, n_in, C, n_in, plane, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_grey_adjoint(dgf_dtype dt, bool src_f32, const void* dG, void* dI, int N, int n_in, int C,
                                size_t plane, cudaStream_t s) {
    if (N == 0 || plane == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return grey_go<float, float>(dG, dI, N, C, n_in, n_in, plane, s);
        case DGF_BF16:
            return src_f32 ? grey_go<float, __nv_bfloat16>(dG, dI, N, C, n_in, n_in, plane, s)
                           : grey_go<__nv_bfloat16, __nv_bfloat16>(dG, dI, N, C, n_in, n_in, plane, s);
        case DGF_F16:
            return src_f32 ? grey_go<float, __half>(dG, dI, N, C, n_in, n_in, plane, s)
                           : grey_go<__half, __half>(dG, dI, N, C, n_in, n_in, plane, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
