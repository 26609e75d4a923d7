// Persistent K1 of the batched forward: one CTA loop over the flat list of
// low-resolution tiles of every image (descriptor table in the kernel
// parameters).  Instantiated per storage type in batch_k1_*.cu.
#pragma once

#include "batch.cuh"
#include "kernels.h"
#include "lowres_fast.cuh"
#include "lowres_generic.cuh"

namespace dgf {

template <typename T>
__global__ void __launch_bounds__(kThreads) k1_coef_batched(const __grid_constant__ BatchParams bp,
                                                            uint32_t* status) {
    extern __shared__ __align__(128) float smem[];
    for (int tile = blockIdx.x; tile < bp.k1_total; tile += gridDim.x) {
        const int i = batch_find(bp.k1_start, bp.n, tile);
        const BatchImage& im = bp.img[i];
        const int local = tile - bp.k1_start[i];
        const int per_plane = im.k1_nx * im.k1_ny;
        const int plane = local / per_plane;
        const int tp = local - plane * per_plane;
        const int ty = tp / im.k1_nx, tx = tp - ty * im.k1_nx;
        const size_t hw = (size_t)im.h_l * im.w_l;
        const T* G = static_cast<const T*>(im.I_l) + plane * hw;
        const T* P = static_cast<const T*>(im.p_l) + plane * hw;
        if (im.k1_fast) {
            FastTile f;
            f.h = im.h_l; f.w = im.w_l; f.CW = im.k1_tx; f.EY1 = im.k1_ty; f.log2cw = ilog2(im.k1_tx);
            f.eps = im.eps; f.TX = im.k1_tx - 2 * im.r; f.TY = im.k1_ty - 2 * im.r;
            f.tx0 = tx * f.TX; f.ty0 = ty * f.TY;
            switch (im.r) {
                case 1: coef_tile_fast<T, T, 1>(G, P, im.coef + plane * hw, f, smem, nullptr, nullptr, plane, status); break;
                case 2: coef_tile_fast<T, T, 2>(G, P, im.coef + plane * hw, f, smem, nullptr, nullptr, plane, status); break;
                case 4: coef_tile_fast<T, T, 4>(G, P, im.coef + plane * hw, f, smem, nullptr, nullptr, plane, status); break;
                default: coef_tile_fast<T, T, 8>(G, P, im.coef + plane * hw, f, smem, nullptr, nullptr, plane, status); break;
            }
        } else {
            LowresTile t;
            t.init(im.h_l, im.w_l, im.r, im.eps, ty * im.k1_ty, tx * im.k1_tx, im.k1_ty, im.k1_tx);
            coef_tile<T, T>(G, P, im.coef + plane * hw, t, smem, nullptr, nullptr, plane, status);
        }
    }
}


template <typename T>
cudaError_t k1_batched_kernel_t(size_t smem, void** fn) {
    *fn = (void*)k1_coef_batched<T>;
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(k1_coef_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

}  // namespace dgf
