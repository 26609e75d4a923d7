// Grey guide of Sec. 6.3 (DGF_b): when the guide has n_I channels and the
// output C != n_I, the transformation F is the mean over the guide's
// channels, and that one grey plane guides every output channel.
//   KG   G[n, c] = (sum over k of I[n, k]) / n_I for every c < C, rounded to
//        the storage type (the layer reads its guides in that type)
//   KGT  the adjoint: d I[n, k] = (sum over c of d G[n, c]) / n_I for every
//        k < n_I (the channel mean hands 1 / n_I of the summed gradient to
//        each guide channel)
// Both are streaming passes over whole planes: each thread moves VEC
// consecutive pixels of one image (16-byte vectors when every plane start is
// 16-byte aligned), the channels summed in order in FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace dgf {

// KG (MODE 0) and KGT (MODE 1): out[n, j] = (sum over i < n_src of src[n, i]) / n_I
// for every j < n_dst.
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_grey(const T* __restrict__ src, T* __restrict__ dst, int N,
                                                   int n_src, int n_dst, int n_in, size_t plane) {
    const size_t nv = plane / VEC, total = (size_t)N * nv;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const size_t n = v / nv, px = (v - n * nv) * VEC;
        float s[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) s[k] = 0.f;
        for (int i = 0; i < n_src; ++i) {
            float x[VEC];
            load_vec<T, VEC>(src + (n * n_src + i) * plane + px, x);
#pragma unroll
            for (int k = 0; k < VEC; ++k) s[k] = __fadd_rn(s[k], x[k]);
        }
        float g[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[k] = n_in == 1 ? s[k] : __fdiv_rn(s[k], (float)n_in);
        for (int j = 0; j < n_dst; ++j) store_vec<T, VEC>(dst + (n * n_dst + j) * plane + px, g);
    }
}

template <typename T>
static cudaError_t grey_go(const void* src, void* dst, int N, int n_src, int n_dst, int n_in, size_t plane,
                           cudaStream_t s) {
    constexpr int V16 = 16 / (int)sizeof(T);
    const bool wide = plane % V16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(dst) % 16 == 0;
    const size_t vecs = (size_t)N * (wide ? plane / V16 : plane);
    const int blocks = (int)std::min<size_t>((vecs + kThreads - 1) / kThreads, (size_t)152 * 16);
    if (blocks == 0) return cudaSuccess;
    if (wide)
        k_grey<T, V16><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(src), static_cast<T*>(dst), N, n_src,
                                                   n_dst, n_in, plane);
    else
        k_grey<T, 1><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(src), static_cast<T*>(dst), N, n_src, n_dst,
                                                 n_in, plane);
    return cudaGetLastError();
}

static cudaError_t grey_d(dgf_dtype dt, const void* src, void* dst, int N, int n_src, int n_dst, int n_in,
                          size_t plane, cudaStream_t s) {
    switch (dt) {
        case DGF_F32: return grey_go<float>(src, dst, N, n_src, n_dst, n_in, plane, s);
        case DGF_BF16: return grey_go<__nv_bfloat16>(src, dst, N, n_src, n_dst, n_in, plane, s);
        case DGF_F16: return grey_go<__half>(src, dst, N, n_src, n_dst, n_in, plane, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_grey_mean(dgf_dtype dt, const void* I, void* G, int N, int n_in, int C, size_t plane,
                             cudaStream_t s) {
    if (N == 0 || plane == 0) return cudaSuccess;
    return grey_d(dt, I, G, N, n_in, C, n_in, plane, s);
}

cudaError_t launch_grey_adjoint(dgf_dtype dt, const void* dG, void* dI, int N, int n_in, int C, size_t plane,
                                cudaStream_t s) {
    if (N == 0 || plane == 0) return cudaSuccess;
    return grey_d(dt, dG, dI, N, C, n_in, n_in, plane, s);
}

}  // namespace dgf
