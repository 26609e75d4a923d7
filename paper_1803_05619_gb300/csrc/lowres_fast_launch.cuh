// Column-walking low-resolution kernels (see lowres_fast.cuh) and their
// launchers, templated on the radius.  Each radius is instantiated in its
// own translation unit (lowres_k1_r*.cu, lowres_k4_r*.cu) so the build
// compiles them in parallel.
#pragma once

#include "kernels.h"
#include "lowres_fast.cuh"
#include "lowres_strip.cuh"
#include "lowres_strip2.cuh"

namespace dgf {

template <typename TG, typename TP, int R>
__global__ void __launch_bounds__(kLowThreads) k1_coef_fast(const TG* __restrict__ G, const TP* __restrict__ P,
                                                            float2* __restrict__ coef, int h, int w, float eps,
                                                            int CW, int EY1, const __grid_constant__ TmaPair tma,
                                                            uint32_t* status) {
    extern __shared__ __align__(128) float smem[];
    FastTile t;
    t.h = h; t.w = w; t.CW = CW; t.EY1 = EY1; t.log2cw = ilog2(CW); t.eps = eps;
    t.TX = CW - 2 * R; t.TY = EY1 - 2 * R;
    t.tx0 = blockIdx.x * t.TX; t.ty0 = blockIdx.y * t.TY;
    const size_t plane = blockIdx.z, hw = (size_t)h * w;
    coef_tile_fast<TG, TP, R>(G + plane * hw, P + plane * hw, coef + plane * hw, t, smem,
                              tma.enabled ? &tma.a : nullptr, tma.enabled ? &tma.b : nullptr, (int)plane, status);
}

template <typename TG, typename TP, typename TD, int R>
__global__ void __launch_bounds__(kLowThreads) k4_lowres_bwd_fast(const TG* __restrict__ G, const TP* __restrict__ P,
                                                                  const float2* __restrict__ dcoef,
                                                                  TP* __restrict__ dP, TD* __restrict__ dG, int h,
                                                                  int w, float eps, int CW, int EY1) {
    extern __shared__ __align__(128) float smem[];
    FastTile t;
    t.h = h; t.w = w; t.CW = CW; t.EY1 = EY1; t.log2cw = ilog2(CW); t.eps = eps;
    t.TX = CW - 2 * R; t.TY = EY1 - 2 * R;
    t.tx0 = blockIdx.x * t.TX; t.ty0 = blockIdx.y * t.TY;
    const size_t plane = blockIdx.z, hw = (size_t)h * w;
    lowres_bwd_tile_fast<TG, TP, TD, R>(G + plane * hw, P + plane * hw, dcoef + plane * hw,
                                        dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr, t, smem);
}


// Warp-strip K1 (R = 1, 2; two columns per lane): warp w of the grid owns
// strip (w % nstrip) of row segment (w / nstrip) % nseg of plane w / (nstrip nseg).
template <typename TG, typename TP, int R>
__global__ void __launch_bounds__(kStripWarps * 32) k1_coef_strip(const TG* __restrict__ G, const TP* __restrict__ P,
                                                                   float2* __restrict__ coef, int h, int w, float eps,
                                                                   int seg, int nstrip, int nseg, int planes,
                                                                   float4* __restrict__ stats, int mean) {
    const int gw = blockIdx.x * kStripWarps + (threadIdx.x >> 5);
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    StripGeom s;
    s.h = h;
    s.w = w;
    s.x0 = strip * strip2_out_cols(R) - 2 * R;
    s.y0 = sg * seg;
    s.seg = seg;
    s.mean = mean;
    const size_t hw = (size_t)h * w;
    coef_strip2<TG, TP, R>(G + plane * hw, P + plane * hw, coef + plane * hw, s, eps,
                           stats ? stats + plane * hw : nullptr);
}

// Warp-strip K1 with TMA staging: same decomposition; each warp's rows
// come through its own slot ring in dynamic shared memory.
template <typename TG, typename TP, int R>
__global__ void __launch_bounds__(kStripWarps * 32)
    k1_coef_strip_tma(const __grid_constant__ TmaPair maps, float2* __restrict__ coef, float4* __restrict__ stats,
                      int h, int w, float eps, int seg, int nstrip, int nseg, int planes, uint32_t* status, int mean) {
    extern __shared__ __align__(1024) unsigned char k1ring[];
    constexpr int NS = StripTmaCfg<R>::NS, RB = StripTmaCfg<R>::RB;
    constexpr int SLOT = strip2_box_bytes((int)sizeof(TG), RB) + strip2_box_bytes((int)sizeof(TP), RB);
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kStripWarps + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    StripGeom s;
    s.h = h;
    s.w = w;
    s.x0 = strip * strip2_out_cols(R) - 2 * R;
    s.y0 = sg * seg;
    s.seg = seg;
    s.mean = mean;
    unsigned char* ring = k1ring + (size_t)warp * NS * SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k1ring + (size_t)kStripWarps * NS * SLOT) + warp * NS;
    const size_t hw = (size_t)h * w;
    coef_strip2_tma<TG, TP, R>(&maps, plane, coef + plane * hw, stats ? stats + plane * hw : nullptr, s, eps, ring,
                               bars, status);
}

// Warp-strip K4 (R = 1, 2), same work decomposition as k1_coef_strip, in
// CTAs of 4 warps (its register footprint is large, and small CTAs let the
// SM keep more of them resident).
template <typename TG, typename TP, typename TD, int R>
__global__ void __launch_bounds__(kK4StripWarps * 32)
    k4_lowres_bwd_strip(const TG* __restrict__ G, const TP* __restrict__ P, const float2* __restrict__ dcoef,
                        TP* __restrict__ dP, TD* __restrict__ dG, int h, int w, float eps, int seg, int nstrip,
                        int nseg, int planes, int mean) {
    const int gw = blockIdx.x * kK4StripWarps + (threadIdx.x >> 5);
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    StripGeom s;
    s.h = h;
    s.w = w;
    s.x0 = strip * (32 - 4 * R) - 2 * R;
    s.y0 = sg * seg;
    s.seg = seg;
    s.mean = mean;
    const size_t hw = (size_t)h * w;
    lowres_bwd_strip<TG, TP, TD, R>(G + plane * hw, P + plane * hw, dcoef + plane * hw,
                                    dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr, s, eps);
}

template <typename TG, typename TP, typename TD, int R>
__global__ void __launch_bounds__(kK4StripWarps * 32)
    k4_lowres_bwd_strip_tma(const __grid_constant__ TmaTriple maps, TP* __restrict__ dP, TD* __restrict__ dG, int h,
                            int w, float eps, int seg, int nstrip, int nseg, int planes, uint32_t* status, int mean) {
    extern __shared__ __align__(1024) unsigned char k4ring[];
    constexpr int NS = StripTmaCfg<R>::NS4, RB = StripTmaCfg<R>::RB;
    constexpr int SLOT = strip_box_bytes(R, (int)sizeof(TG), RB) + strip_box_bytes(R, (int)sizeof(TP), RB) +
                         align128i(RB * 2 * (32 + 2) * 4);
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kK4StripWarps + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    StripGeom s;
    s.h = h;
    s.w = w;
    s.x0 = strip * (32 - 4 * R) - 2 * R;
    s.y0 = sg * seg;
    s.seg = seg;
    s.mean = mean;
    const size_t hw = (size_t)h * w;
    unsigned char* ring = k4ring + (size_t)warp * NS * SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k4ring + (size_t)kK4StripWarps * NS * SLOT) + warp * NS;
    lowres_bwd_strip_tma<TG, TP, TD, R>(&maps, plane, dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr,
                                        s, eps, ring, bars, status);
}

// Two-column K4 from saved statistics: warp w owns strip (w % nstrip) of the
// two-column geometry (64 - 4R outputs) of segment (w / nstrip) % nseg.
template <typename TG, typename TP, typename TD, int R>
__global__ void __launch_bounds__(kK4StripWarps * 32)
    k4_lowres_bwd_strip2_stats(const TG* __restrict__ G, const TP* __restrict__ P, const float2* __restrict__ dcoef,
                               const float4* __restrict__ stats, TP* __restrict__ dP, TD* __restrict__ dG, int h,
                               int w, int seg, int nstrip, int nseg, int planes, int mean) {
    const int gw = blockIdx.x * kK4StripWarps + (threadIdx.x >> 5);
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    StripGeom s;
    s.h = h;
    s.w = w;
    s.x0 = strip * strip2_out_cols(R) - 2 * R;
    s.y0 = sg * seg;
    s.seg = seg;
    s.mean = mean;
    const size_t hw = (size_t)h * w;
    lowres_bwd_strip2_stats<TG, TP, TD, R>(G + plane * hw, P + plane * hw, dcoef + plane * hw, stats + plane * hw,
                                           dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr, s);
}

template <typename K>
static inline cudaError_t fast_prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename TG, typename TP, int R>
static cudaError_t k1f_go(const void* G, const void* P, float2* coef, int planes, int h, int w, float eps,
                          const LowCfg& c, const TmaPair& tma, size_t smem, uint32_t* status, float4* stats, cudaStream_t s) {
    if constexpr (R <= 2) {
        if (c.fast == 2) {
            const int seg = c.a, nstrip = (w + strip2_out_cols(R) - 1) / strip2_out_cols(R), nseg = (h + seg - 1) / seg;
            const long long warps = (long long)nstrip * nseg * planes;
            const int ctas = (int)((warps + kStripWarps - 1) / kStripWarps);
            if (tma.enabled) {
                constexpr int smem_t = k1_strip2_tma_smem<TG, TP, R>();
                auto kern = k1_coef_strip_tma<TG, TP, R>;
                cudaError_t e = fast_prep(kern, smem_t);
                if (e != cudaSuccess) return e;
                kern<<<ctas, kStripWarps * 32, smem_t, s>>>(tma, coef, stats, h, w, eps, seg, nstrip, nseg, planes,
                                                             status, c.mean);
                return cudaGetLastError();
            }
            k1_coef_strip<TG, TP, R><<<ctas, kStripWarps * 32, 0, s>>>(
                static_cast<const TG*>(G), static_cast<const TP*>(P), coef, h, w, eps, seg, nstrip, nseg, planes, stats, c.mean);
            return cudaGetLastError();
        }
    }
    auto kern = k1_coef_fast<TG, TP, R>;
    cudaError_t e = fast_prep(kern, smem);
    if (e != cudaSuccess) return e;
    int gx, gy;
    low_grid(c, R, h, w, gx, gy);
    kern<<<dim3(gx, gy, planes), kLowThreads, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P),
                                                         coef, h, w, eps, c.a, c.b, tma, status);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_k1_fast(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes,
                           int h, int w, float eps, const LowCfg& c, const TmaPair& tma, size_t smem,
                           uint32_t* status, float4* stats, cudaStream_t s) {
    switch (dt) {
        case DGF_F32: return k1f_go<float, float, R>(G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
        case DGF_BF16:
            return gf32 ? k1f_go<float, __nv_bfloat16, R>(G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s)
                        : k1f_go<__nv_bfloat16, __nv_bfloat16, R>(G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
        case DGF_F16:
            return gf32 ? k1f_go<float, __half, R>(G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s)
                        : k1f_go<__half, __half, R>(G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
    }
    return cudaErrorInvalidValue;
}

template <typename TG, typename TP, typename TD, int R>
static cudaError_t k4f_go(const void* G, const void* P, const float2* dcoef, void* dP, void* dG, int planes,
                          int h, int w, float eps, const LowCfg& c, const TmaTriple* tma, uint32_t* status,
                          const float4* stats, cudaStream_t s) {
    if constexpr (R <= 2) {
        if (c.fast == 2) {
            const int seg = c.a, nstrip = (w + (32 - 4 * R) - 1) / (32 - 4 * R), nseg = (h + seg - 1) / seg;
            const long long warps = (long long)nstrip * nseg * planes;
            const int ctas = (int)((warps + kK4StripWarps - 1) / kK4StripWarps);
            if (stats != nullptr) {
                const int nstrip2 = (w + strip2_out_cols(R) - 1) / strip2_out_cols(R);
                const long long warps2 = (long long)nstrip2 * nseg * planes;
                const int ctas2 = (int)((warps2 + kK4StripWarps - 1) / kK4StripWarps);
                k4_lowres_bwd_strip2_stats<TG, TP, TD, R><<<ctas2, kK4StripWarps * 32, 0, s>>>(
                    static_cast<const TG*>(G), static_cast<const TP*>(P), dcoef, stats, static_cast<TP*>(dP),
                    static_cast<TD*>(dG), h, w, seg, nstrip2, nseg, planes, c.mean);
                return cudaGetLastError();
            }
            if (tma != nullptr && tma->enabled) {
                constexpr int smem_t = k4_strip_tma_smem<TG, TP, R>();
                auto kern = k4_lowres_bwd_strip_tma<TG, TP, TD, R>;
                cudaError_t e = fast_prep(kern, smem_t);
                if (e != cudaSuccess) return e;
                kern<<<ctas, kK4StripWarps * 32, smem_t, s>>>(*tma, static_cast<TP*>(dP), static_cast<TD*>(dG), h, w,
                                                               eps, seg, nstrip, nseg, planes, status, c.mean);
                return cudaGetLastError();
            }
            k4_lowres_bwd_strip<TG, TP, TD, R><<<ctas, kK4StripWarps * 32, 0, s>>>(
                static_cast<const TG*>(G), static_cast<const TP*>(P), dcoef, static_cast<TP*>(dP),
                static_cast<TD*>(dG), h, w, eps, seg, nstrip, nseg, planes, c.mean);
            return cudaGetLastError();
        }
    }
    const size_t smem = k4_fast_smem_bytes(R, c.a, c.b);
    auto kern = k4_lowres_bwd_fast<TG, TP, TD, R>;
    cudaError_t e = fast_prep(kern, smem);
    if (e != cudaSuccess) return e;
    int gx, gy;
    low_grid(c, R, h, w, gx, gy);
    kern<<<dim3(gx, gy, planes), kLowThreads, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P),
                                                         dcoef, static_cast<TP*>(dP), static_cast<TD*>(dG), h, w,
                                                         eps, c.a, c.b);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_k4_fast(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP,
                           void* dG, int planes, int h, int w, float eps, const LowCfg& c, const TmaTriple* tma, uint32_t* status,
                           const float4* stats, cudaStream_t s) {
    switch (dt) {
        case DGF_F32: return k4f_go<float, float, float, R>(G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
        case DGF_BF16:
            return gf32 ? k4f_go<float, __nv_bfloat16, float, R>(G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s)
                        : k4f_go<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, R>(G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
        case DGF_F16:
            return gf32 ? k4f_go<float, __half, float, R>(G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s)
                        : k4f_go<__half, __half, __half, R>(G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
