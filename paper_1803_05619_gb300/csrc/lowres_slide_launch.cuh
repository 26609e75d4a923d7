// Kernels and launchers of the sliding-sum low-resolution stage
// (lowres_slide.cuh); one translation unit per radius instantiates them.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"
#include "lowres_slide.cuh"

namespace dgf {

// CTA b of plane b / nx owns WPC consecutive strip segments of that plane
// (segment item k: strip k % nstrip, S output rows from (k / nstrip) S), one
// per warp; the warps of a CTA are independent (no barrier), each with its
// own shared-memory ring.
template <typename TG, typename TP, int R, int V>
__global__ void __launch_bounds__(slide_wpc<k1_slide_warp_bytes<TG, TP, R, V>()>() * 32)
    k1_slide(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef, int h, int w, float eps,
             int S, int nx, int aligned) {
    extern __shared__ __align__(16) float4 k1slring[];
    using Gm = SlideGeom<R, V>;
    constexpr int WPC = slide_wpc<k1_slide_warp_bytes<TG, TP, R, V>()>();
    const int warp = threadIdx.x >> 5;
    const int plane = blockIdx.x / nx;
    const int item = (blockIdx.x - plane * nx) * WPC + warp;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    if (item >= nstrip * nseg) return;  // whole warp leaves together
    const size_t hw = (size_t)h * w;
    float4* ring = k1slring + (size_t)warp * (k1_slide_warp_bytes<TG, TP, R, V>() / 16);
    k1_slide_segment<TG, TP, R, V>(G + plane * hw, P + plane * hw, coef + plane * hw, h, w, eps,
                                   (item % nstrip) * Gm::OUTC - Gm::HB, (item / nstrip) * S, S, aligned != 0, ring);
}

// K4: the same decomposition as K1.
template <typename TG, typename TP, typename TD, int R, int V>
__global__ void __launch_bounds__(slide_wpc<k4_slide_warp_bytes<TG, TP, R, V>()>() * 32)
    k4_slide(const TG* __restrict__ G, const TP* __restrict__ P, const float2* __restrict__ dcoef,
             TP* __restrict__ dP, TD* __restrict__ dG, int h, int w, float eps, int S, int nx, int aligned,
             int aligned_pairs) {
    extern __shared__ __align__(16) float4 k4slring[];
    using Gm = SlideGeom<R, V>;
    constexpr int WPC = slide_wpc<k4_slide_warp_bytes<TG, TP, R, V>()>();
    const int warp = threadIdx.x >> 5;
    const int plane = blockIdx.x / nx;
    const int item = (blockIdx.x - plane * nx) * WPC + warp;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    if (item >= nstrip * nseg) return;  // whole warp leaves together
    const size_t hw = (size_t)h * w;
    float4* ring = k4slring + (size_t)warp * (k4_slide_warp_bytes<TG, TP, R, V>() / 16);
    k4_slide_segment<TG, TP, TD, R, V>(G + plane * hw, P + plane * hw, dcoef + plane * hw,
                                       dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr, h, w, eps,
                                       (item % nstrip) * Gm::OUTC - Gm::HB, (item / nstrip) * S, S, aligned != 0,
                                       aligned_pairs != 0, ring);
}

template <typename TG, typename TP, int R, int V>
constexpr int k1_slide_wpc() {
    return slide_wpc<k1_slide_warp_bytes<TG, TP, R, V>()>();
}
template <typename TG, typename TP, int R, int V>
constexpr int k4_slide_wpc() {
    return slide_wpc<k4_slide_warp_bytes<TG, TP, R, V>()>();
}
template <typename TG, typename TP, int R, int V>
constexpr size_t k1_slide_smem() {
    return (size_t)k1_slide_wpc<TG, TP, R, V>() * k1_slide_warp_bytes<TG, TP, R, V>();
}
template <typename TG, typename TP, int R, int V>
constexpr size_t k4_slide_smem() {
    return (size_t)k4_slide_wpc<TG, TP, R, V>() * k4_slide_warp_bytes<TG, TP, R, V>();
}

template <typename K>
static cudaError_t slide_prep(K kernel, size_t smem) {
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) cudaGetLastError();  // reported once, here
        return e;
    }
    return cudaSuccess;
}

static inline bool slide_ptr_aligned(const void* p, size_t bytes) {
    return p == nullptr || reinterpret_cast<uintptr_t>(p) % bytes == 0;
}

template <typename TG, typename TP, int R, int V>
static cudaError_t k1_slide_go(const void* G, const void* P, float2* coef, int planes, int h, int w, float eps,
                               int S, cudaStream_t s) {
    using Gm = SlideGeom<R, V>;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    constexpr int WPC = k1_slide_wpc<TG, TP, R, V>();
    const int nx = (nstrip * nseg + WPC - 1) / WPC;  // CTAs per plane
    const long long ctas = (long long)nx * planes;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    constexpr size_t smem = k1_slide_smem<TG, TP, R, V>();
    auto kern = k1_slide<TG, TP, R, V>;
    cudaError_t e = slide_prep(kern, smem);
    if (e != cudaSuccess) return e;
    const int aligned = w % V == 0 && slide_ptr_aligned(G, V * sizeof(TG)) && slide_ptr_aligned(P, V * sizeof(TP));
    kern<<<(unsigned)ctas, WPC * 32, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P), coef, h, w,
                                                 eps, S, nx, aligned);
    return cudaGetLastError();
}

template <typename TG, typename TP, typename TD, int R, int V>
static cudaError_t k4_slide_go(const void* G, const void* P, const float2* dcoef, void* dP, void* dG, int planes,
                               int h, int w, float eps, int S, cudaStream_t s) {
    using Gm = SlideGeom<R, V>;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    constexpr int WPC = k4_slide_wpc<TG, TP, R, V>();
    const int nx = (nstrip * nseg + WPC - 1) / WPC;  // CTAs per plane
    const long long ctas = (long long)nx * planes;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    constexpr size_t smem = k4_slide_smem<TG, TP, R, V>();
    auto kern = k4_slide<TG, TP, TD, R, V>;
    cudaError_t e = slide_prep(kern, smem);
    if (e != cudaSuccess) return e;
    const int aligned = w % V == 0 && slide_ptr_aligned(G, V * sizeof(TG)) && slide_ptr_aligned(P, V * sizeof(TP)) &&
                        slide_ptr_aligned(dP, V * sizeof(TP)) && slide_ptr_aligned(dG, V * sizeof(TD));
    const int aligned_pairs = w % 2 == 0 && slide_ptr_aligned(dcoef, 16);
    kern<<<(unsigned)ctas, WPC * 32, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P), dcoef,
                                                 static_cast<TP*>(dP), static_cast<TD*>(dG), h, w, eps, S, nx,
                                                 aligned, aligned_pairs);
    return cudaGetLastError();
}

// The columns per lane (V) built for each radius: 2 and 8 for R <= 2, 4 for
// every R (wider lanes at larger radii would not fit the rings of the
// batched K1's eight warps).
template <int R, int V>
constexpr bool k1_slide_built() {
    return (V == 2 && R <= 2) || V == 4 || (V == 8 && R <= 2);
}
template <int R, int V>
constexpr bool k4_slide_built() {
    return (V == 2 && R <= 2) || V == 4 || (V == 8 && R <= 2);
}

template <int R>
cudaError_t launch_k1_slide_r(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes, int h,
                              int w, float eps, int S, int V, cudaStream_t s) {
#define DGF_K1S(VV)                                                                                          \
    if (V == VV) {                                                                                           \
        if constexpr (k1_slide_built<R, VV>()) {                                                             \
            switch (dt) {                                                                                    \
                case DGF_BF16:                                                                               \
                    return gf32 ? k1_slide_go<float, __nv_bfloat16, R, VV>(G, P, coef, planes, h, w, eps, S, s) \
                                : k1_slide_go<__nv_bfloat16, __nv_bfloat16, R, VV>(G, P, coef, planes, h, w, eps, S, s); \
                case DGF_F16:                                                                                \
                    return gf32 ? k1_slide_go<float, __half, R, VV>(G, P, coef, planes, h, w, eps, S, s)     \
                                : k1_slide_go<__half, __half, R, VV>(G, P, coef, planes, h, w, eps, S, s);   \
                default: return cudaErrorInvalidValue;                                                       \
            }                                                                                                \
        }                                                                                                    \
    }
    DGF_K1S(2)
    DGF_K1S(4)
    DGF_K1S(8)
#undef DGF_K1S
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t launch_k4_slide_r(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP,
                              void* dG, int planes, int h, int w, float eps, int S, int V, cudaStream_t s) {
#define DGF_K4S(VV)                                                                                               \
    if (V == VV) {                                                                                                \
        if constexpr (k4_slide_built<R, VV>()) {                                                                  \
            switch (dt) {                                                                                         \
                case DGF_BF16:                                                                                    \
                    return gf32 ? k4_slide_go<float, __nv_bfloat16, float, R, VV>(G, P, dcoef, dP, dG, planes, h, w, \
                                                                                  eps, S, s)                     \
                                : k4_slide_go<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, R, VV>(               \
                                      G, P, dcoef, dP, dG, planes, h, w, eps, S, s);                              \
                case DGF_F16:                                                                                     \
                    return gf32 ? k4_slide_go<float, __half, float, R, VV>(G, P, dcoef, dP, dG, planes, h, w, eps, S, \
                                                                           s)                                     \
                                : k4_slide_go<__half, __half, __half, R, VV>(G, P, dcoef, dP, dG, planes, h, w, eps, \
                                                                             S, s);                               \
                default: return cudaErrorInvalidValue;                                                            \
            }                                                                                                     \
        }                                                                                                         \
    }
    DGF_K4S(2)
    DGF_K4S(4)
    DGF_K4S(8)
#undef DGF_K4S
    return cudaErrorInvalidValue;
}

}  // namespace dgf
