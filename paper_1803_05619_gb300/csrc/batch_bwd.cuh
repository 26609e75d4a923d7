// Persistent kernels of the batched backward (16-bit storage): the K3 strip
// walk and the sliding K4 over a flat work list of every image's strip
// segments, one kernel per node class, with the descriptor table in the
// kernel parameters (a CUDA-graph replay updates it in place).  Each image
// runs exactly the arithmetic of its single call: the plain-load K3 walk
// (the same bits as the TMA-staged one, at any segment length) and the
// sliding K4 with the single call's segment length and columns per lane.
#pragma once

#include "batch.cuh"
#include "hires_strip.cuh"
#include "lowres_slide.cuh"
#include "tma.cuh"

namespace dgf {

// Warps per CTA and shared memory of a K3 class: the TMA-staged walk's
// (16-byte vectors and tensor maps), else plain loads with kWarps warps and
// no ring.
template <typename T, int VEC, int F, bool TMA>
struct K3BatchShape {
    static_assert(!TMA || VEC * sizeof(T) == 16, "TMA staging needs 16-byte vectors");
    static constexpr int WPC = TMA ? K3Tma<T, VEC, F>::WPC : kWarps;
    static constexpr size_t SMEM = TMA ? K3Tma<T, VEC, F>::CTA_BYTES : 0;
};

// K3 class (vector width VEC, factor F, staging): CTA t takes work item t
// (the grid is the whole item list), WPC strip segments of one plane, one
// per warp.  TMA: every image of the class has tensor maps and is staged
// through the warp's slot ring; else plain loads (the same bits).
template <typename T, int VEC, int F, bool TMA>
__global__ void __launch_bounds__(K3BatchShape<T, VEC, F, TMA>::WPC * 32)
    k3_batched(const __grid_constant__ BwdParams bp, uint32_t* status) {
    using Sh = K3BatchShape<T, VEC, F, TMA>;
    constexpr int OUT = K3Strip<VEC, F>::OUT;
    extern __shared__ __align__(1024) unsigned char k3bring[];
    const int tile = blockIdx.x;
    if (tile >= bp.total) return;
    const int warp = threadIdx.x >> 5;
    const int i = batch_find(bp.start, bp.n, tile);
    const BwdImage& im = bp.img[i];
    const int local = tile - bp.start[i];
    const int h_l = im.h_l, w_l = im.w_l, h = im.h, w = im.w, ls = im.k3_ls;
    const int plane = local / im.k3_nx;
    const int seg_item = (local - plane * im.k3_nx) * Sh::WPC + warp;
    const int nstrip = (w_l + OUT - 1) / OUT, nseg = (h_l + ls - 1) / ls;
    if (seg_item >= nstrip * nseg) return;  // whole warp leaves together
    const int strip = seg_item % nstrip, sg = seg_item / nstrip;
    const int ia = sg * ls, ib = min(ia + ls, h_l);
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    T* dG = im.dIh ? static_cast<T*>(im.dIh) + plane * hw : nullptr;
    if constexpr (TMA) {
        using B = K3Tma<T, VEC, F>;
        const K3Maps* maps = static_cast<const K3Maps*>(im.k3_maps);
        if ((threadIdx.x & 31) == 0) {
            tensormap_acquire(&maps->r);
            tensormap_acquire(&maps->g);
        }
        __syncwarp();
        unsigned char* ring = k3bring + (size_t)warp * B::NSB * B::SLOT;
        uint64_t* bars = reinterpret_cast<uint64_t*>(k3bring + (size_t)B::WPC * B::NSB * B::SLOT) + warp * B::NSB;
        k3_strip_tma<T, VEC, F>(im.coef + plane * lw, maps, dG, im.dcoef + plane * lw, h_l, w_l, h, w, strip, ia, ib,
                                plane, ring, bars, status);
    } else {
        k3_strip<T, VEC, F>(im.coef + plane * lw, static_cast<const T*>(im.dO) + plane * hw,
                            static_cast<const T*>(im.I_h) + plane * hw, dG, im.dcoef + plane * lw, h_l, w_l, h, w,
                            strip, ia, ib);
    }
}

// K4 class (radius R, columns per lane V): CTA t takes work item t (the
// grid is the whole item list), WPC sliding strip segments of one plane, one
// per warp, each with its own shared-memory ring.
template <typename T, int R, int V>
__global__ void __launch_bounds__(slide_wpc<k4_slide_warp_bytes<T, T, R, V>()>() * 32)
    k4_batched(const __grid_constant__ BwdParams bp) {
    extern __shared__ __align__(16) float4 k4bring[];
    using Gm = SlideGeom<R, V>;
    constexpr int WPC = slide_wpc<k4_slide_warp_bytes<T, T, R, V>()>();
    const int tile = blockIdx.x;
    if (tile >= bp.total) return;
    const int warp = threadIdx.x >> 5;
    const int i = batch_find(bp.start, bp.n, tile);
    const BwdImage& im = bp.img[i];
    const int local = tile - bp.start[i];
    const int h = im.h_l, w = im.w_l, S = im.k4_S;
    const int plane = local / im.k4_nx;
    const int item = (local - plane * im.k4_nx) * WPC + warp;
    const int nstrip = (w + Gm::OUTC - 1) / Gm::OUTC, nseg = (h + S - 1) / S;
    if (item >= nstrip * nseg) return;  // whole warp leaves together
    const size_t lw = (size_t)h * w;
    T* dP = im.dp ? static_cast<T*>(im.dp) + plane * lw : nullptr;
    T* dG = im.dIl ? static_cast<T*>(im.dIl) + plane * lw : nullptr;
    float4* ring = k4bring + (size_t)warp * (k4_slide_warp_bytes<T, T, R, V>() / 16);
    k4_slide_segment<T, T, T, R, V>(static_cast<const T*>(im.I_l) + plane * lw,
                                    static_cast<const T*>(im.p_l) + plane * lw, im.dcoef + plane * lw, dP, dG, h, w,
                                    im.eps, (item % nstrip) * Gm::OUTC - Gm::HB, (item / nstrip) * S, S,
                                    im.k4_aligned != 0, im.k4_pairs != 0, ring);
}

}  // namespace dgf
