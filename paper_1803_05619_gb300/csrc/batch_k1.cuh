// Persistent K1 of the batched forward: one CTA loop over the flat list of
// low-resolution tiles of every image (descriptor table in the kernel
// parameters).  Instantiated per storage type in batch_k1_*.cu.
#pragma once

#include "batch.cuh"
#include "kernels.h"
#include "lowres_fast.cuh"
#include "lowres_generic.cuh"
#include "lowres_strip.cuh"
#include "lowres_strip2.cuh"
#include "lowres_slide.cuh"

namespace dgf {

// Sliding-sum strips of radius R with V columns per lane (16-bit storage):
// CTA t takes work item t (one per CTA, as the single call's kernel: the
// grid is the whole item list), WPC strip segments (the single call's warps
// per CTA), one per warp, each with its own shared-memory ring.
template <typename T, int R, int V>
__global__ void __launch_bounds__(slide_wpc<k1_slide_warp_bytes<T, T, R, V>()>() * 32)
    k1_slide_batched(const __grid_constant__ BatchParams bp, uint32_t*) {
    extern __shared__ __align__(16) float4 k1sbring[];
    using Gm = SlideGeom<R, V>;
    constexpr int WPC = slide_wpc<k1_slide_warp_bytes<T, T, R, V>()>();
    const int tile = blockIdx.x;
    if (tile >= bp.k1_total) return;
    const int warp = threadIdx.x >> 5;
    const int i = batch_find(bp.k1_start, bp.n, tile);
    const BatchImage& im = bp.img[i];
    const int local = tile - bp.k1_start[i];
    const int h = im.h_l, w = im.w_l, S = im.k1_tx;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    const int plane = local / im.k1_nx;
    const int item = (local - plane * im.k1_nx) * WPC + warp;
    if (item >= nstrip * nseg) return;  // whole warp leaves together
    const size_t hw = (size_t)h * w;
    const T* G = static_cast<const T*>(im.I_l) + plane * hw;
    const T* P = static_cast<const T*>(im.p_l) + plane * hw;
    const bool aligned = w % V == 0 && reinterpret_cast<uintptr_t>(G) % (V * sizeof(T)) == 0 &&
                         reinterpret_cast<uintptr_t>(P) % (V * sizeof(T)) == 0;
    float4* ring = k1sbring + (size_t)warp * (k1_slide_warp_bytes<T, T, R, V>() / 16);
    k1_slide_segment<T, T, R, V>(G, P, im.coef + plane * hw, h, w, im.eps, (item % nstrip) * Gm::OUTC - Gm::HB,
                                 (item / nstrip) * S, S, aligned, ring);
}

// MODE 2: warp strips of radius R (a work item is 8 strip segments, one per
// warp); MODE 1: column-walking tiles of radius R; MODE 0: generic tiles.
template <typename T, int R, int MODE>
__global__ void __launch_bounds__(kThreads) k1_coef_batched(const __grid_constant__ BatchParams bp,
                                                            uint32_t* status) {
    extern __shared__ __align__(128) float smem[];
    for (int tile = blockIdx.x; tile < bp.k1_total; tile += gridDim.x) {
        const int i = batch_find(bp.k1_start, bp.n, tile);
        const BatchImage& im = bp.img[i];
        const int local = tile - bp.k1_start[i];
        if constexpr (MODE == 2) {
            const int nstrip = (im.w_l + strip2_out_cols(R) - 1) / strip2_out_cols(R);
            const int nseg = (im.h_l + im.k1_tx - 1) / im.k1_tx;
            const int plane = local / im.k1_nx;
            const int item = (local - plane * im.k1_nx) * kWarps + (threadIdx.x >> 5);
            if (item < nstrip * nseg) {  // warp-uniform; no barrier follows
                StripGeom sg;
                sg.h = im.h_l;
                sg.w = im.w_l;
                sg.x0 = (item % nstrip) * strip2_out_cols(R) - 2 * R;
                sg.y0 = (item / nstrip) * im.k1_tx;
                sg.seg = im.k1_tx;
                const size_t hw = (size_t)im.h_l * im.w_l;
                coef_strip2<T, T, R>(static_cast<const T*>(im.I_l) + plane * hw,
                                    static_cast<const T*>(im.p_l) + plane * hw, im.coef + plane * hw, sg, im.eps);
            }
            continue;
        }
        const int per_plane = im.k1_nx * im.k1_ny;
        const int plane = local / per_plane;
        const int tp = local - plane * per_plane;
        const int ty = tp / im.k1_nx, tx = tp - ty * im.k1_nx;
        const size_t hw = (size_t)im.h_l * im.w_l;
        const T* G = static_cast<const T*>(im.I_l) + plane * hw;
        const T* P = static_cast<const T*>(im.p_l) + plane * hw;
        if constexpr (MODE == 1) {
            FastTile f;
            f.h = im.h_l; f.w = im.w_l; f.CW = im.k1_tx; f.EY1 = im.k1_ty; f.log2cw = ilog2(im.k1_tx);
            f.eps = im.eps; f.TX = im.k1_tx - 2 * R; f.TY = im.k1_ty - 2 * R;
            f.tx0 = tx * f.TX; f.ty0 = ty * f.TY;
            coef_tile_fast<T, T, R>(G, P, im.coef + plane * hw, f, smem, nullptr, nullptr, plane, status);
        } else {
            LowresTile t;
            t.init(im.h_l, im.w_l, im.r, im.eps, ty * im.k1_ty, tx * im.k1_tx, im.k1_ty, im.k1_tx);
            coef_tile<T, T>(G, P, im.coef + plane * hw, t, smem, nullptr, nullptr, plane, status);
        }
    }
}

template <typename K>
static cudaError_t k1b_attr(K kern, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename T, int R, int MODE>
static cudaError_t k1b_get(size_t smem, void** fn, int* threads) {
    *fn = (void*)k1_coef_batched<T, R, MODE>;
    if (threads) *threads = kThreads;
    return k1b_attr(k1_coef_batched<T, R, MODE>, smem);
}

template <typename T, int R, int V>
static cudaError_t k1b_slide(size_t smem, void** fn, int* threads) {
    *fn = (void*)k1_slide_batched<T, R, V>;
    if (threads) *threads = slide_wpc<k1_slide_warp_bytes<T, T, R, V>()>() * 32;
    return k1b_attr(k1_slide_batched<T, R, V>, smem);
}

template <typename T>
cudaError_t k1_batched_kernel_t(int r, int mode, size_t smem, void** fn, int V, int* threads) {
    if constexpr (sizeof(T) == 2) {
        if (mode == 3) {  // the column widths the single-call sliding K1 is built for
            if (V == 2 && r == 1) return k1b_slide<T, 1, 2>(smem, fn, threads);
            if (V == 2 && r == 2) return k1b_slide<T, 2, 2>(smem, fn, threads);
            if (V == 4 && r == 1) return k1b_slide<T, 1, 4>(smem, fn, threads);
            if (V == 4 && r == 2) return k1b_slide<T, 2, 4>(smem, fn, threads);
            if (V == 4 && r == 4) return k1b_slide<T, 4, 4>(smem, fn, threads);
            if (V == 4 && r == 8) return k1b_slide<T, 8, 4>(smem, fn, threads);
            if (V == 8 && r == 1) return k1b_slide<T, 1, 8>(smem, fn, threads);
            if (V == 8 && r == 2) return k1b_slide<T, 2, 8>(smem, fn, threads);
            return cudaErrorInvalidValue;
        }
    }
    if (mode == 2) {
        if (r == 1) return k1b_get<T, 1, 2>(smem, fn, threads);
        if (r == 2) return k1b_get<T, 2, 2>(smem, fn, threads);
    }
    if (mode == 1) {
        switch (r) {
            case 1: return k1b_get<T, 1, 1>(smem, fn, threads);
            case 2: return k1b_get<T, 2, 1>(smem, fn, threads);
            case 4: return k1b_get<T, 4, 1>(smem, fn, threads);
            case 8: return k1b_get<T, 8, 1>(smem, fn, threads);
        }
    }
    return k1b_get<T, 0, 0>(smem, fn, threads);
}

}  // namespace dgf
