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

// MODE 3: sliding-sum strips of radius R with V columns per lane (16-bit
// storage; a work item is 8 strip segments, one per warp, each with its own
// shared-memory ring); MODE 2: warp strips of radius R (a work item is 8
// strip segments, one per warp); MODE 1: column-walking tiles of radius R;
// MODE 0: generic tiles.
template <typename T, int R, int MODE, int VS = 4>
__global__ void __launch_bounds__(kThreads) k1_coef_batched(const __grid_constant__ BatchParams bp,
                                                            uint32_t* status) {
    extern __shared__ __align__(128) float smem[];
    for (int tile = blockIdx.x; tile < bp.k1_total; tile += gridDim.x) {
        const int i = batch_find(bp.k1_start, bp.n, tile);
        const BatchImage& im = bp.img[i];
        const int local = tile - bp.k1_start[i];
        if constexpr (MODE == 3) {
            constexpr int V = VS;  // the class's columns per lane (the single call's)
            using Gm = SlideGeom<R, V>;
            const int nstrip = (im.w_l + Gm::OUTC - 1) / Gm::OUTC;
            const int nseg = (im.h_l + im.k1_tx - 1) / im.k1_tx;
            const int plane = local / im.k1_nx;
            const int warp = threadIdx.x >> 5;
            const int item = (local - plane * im.k1_nx) * kWarps + warp;
            if (item < nstrip * nseg) {  // warp-uniform; no barrier follows
                const size_t hw = (size_t)im.h_l * im.w_l;
                const T* G = static_cast<const T*>(im.I_l) + plane * hw;
                const T* P = static_cast<const T*>(im.p_l) + plane * hw;
                const bool aligned = im.w_l % V == 0 && reinterpret_cast<uintptr_t>(G) % (V * sizeof(T)) == 0 &&
                                     reinterpret_cast<uintptr_t>(P) % (V * sizeof(T)) == 0;
                float4* ring = reinterpret_cast<float4*>(smem) + (size_t)warp * (k1_slide_warp_bytes<T, T, R, V>() / 16);
                k1_slide_segment<T, T, R, V>(G, P, im.coef + plane * hw, im.h_l, im.w_l, im.eps,
                                             (item % nstrip) * Gm::OUTC - Gm::HB, (item / nstrip) * im.k1_tx,
                                             im.k1_tx, aligned, ring);
            }
            continue;
        } else if constexpr (MODE == 2) {
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

template <typename T, int R, int MODE, int VS = 4>
static cudaError_t k1b_get(size_t smem, void** fn) {
    *fn = (void*)k1_coef_batched<T, R, MODE, VS>;
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(k1_coef_batched<T, R, MODE, VS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    return cudaSuccess;
}

template <typename T>
cudaError_t k1_batched_kernel_t(int r, int mode, size_t smem, void** fn, int V) {
    if constexpr (sizeof(T) == 2) {
        if (mode == 3) {  // the column widths the single-call sliding K1 is built for
            if (V == 2 && r == 1) return k1b_get<T, 1, 3, 2>(smem, fn);
            if (V == 2 && r == 2) return k1b_get<T, 2, 3, 2>(smem, fn);
            if (V == 4 && r == 1) return k1b_get<T, 1, 3, 4>(smem, fn);
            if (V == 4 && r == 2) return k1b_get<T, 2, 3, 4>(smem, fn);
            if (V == 4 && r == 4) return k1b_get<T, 4, 3, 4>(smem, fn);
            if (V == 4 && r == 8) return k1b_get<T, 8, 3, 4>(smem, fn);
            if (V == 8 && r == 1) return k1b_get<T, 1, 3, 8>(smem, fn);
            if (V == 8 && r == 2) return k1b_get<T, 2, 3, 8>(smem, fn);
            return cudaErrorInvalidValue;
        }
    }
    if (mode == 2) {
        if (r == 1) return k1b_get<T, 1, 2>(smem, fn);
        if (r == 2) return k1b_get<T, 2, 2>(smem, fn);
    }
    if (mode == 1) {
        switch (r) {
            case 1: return k1b_get<T, 1, 1>(smem, fn);
            case 2: return k1b_get<T, 2, 1>(smem, fn);
            case 4: return k1b_get<T, 4, 1>(smem, fn);
            case 8: return k1b_get<T, 8, 1>(smem, fn);
        }
    }
    return k1b_get<T, 0, 0>(smem, fn);
}

}  // namespace dgf
