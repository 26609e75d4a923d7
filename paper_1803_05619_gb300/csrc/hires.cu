// High-resolution kernels: K2 (bilinear upsampling of Abar, bbar and the
// affine step, Eq. 2) and K3 (the transposed upsampler of Algorithm 1's
// first two lines as a gather, plus d I_h = d O_h * Abar_h).
#include <cmath>
#include <map>
#include <mutex>

#include "batch.cuh"
#include "common.cuh"
#include "hires.cuh"
#include "hires_strip.cuh"
#include "tma.cuh"
#include "kernels.h"

namespace dgf {

template <typename T, int VEC, int F, int MODE, typename TI = T>
__global__ void __launch_bounds__(kThreads) k2_apply(const float2* __restrict__ coef, const TI* __restrict__ in,
                                                     T* __restrict__ out, int h_l, int w_l, int h, int w,
                                                     int TH, int pitch) {
    extern __shared__ __align__(128) float2 sAB[];
    const size_t plane = blockIdx.z;
    apply_tile<T, VEC, F, MODE, TI>(coef + plane * h_l * w_l, in + plane * h * w, out + plane * h * w, h_l,
                                w_l, h, w, blockIdx.y * TH, blockIdx.x * 32 * VEC, TH, pitch, sAB);
}

// K3 fast path: warp w of the grid owns strip (w % nstrip) of segment
// (w / nstrip) % nseg (LS low-res rows each) of plane w / (nstrip nseg).
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(kThreads) k3_hires_bwd(const float2* __restrict__ coef, const T* __restrict__ R,
                                                         const T* __restrict__ G, T* __restrict__ dG,
                                                         float2* __restrict__ dcoef, int h_l, int w_l, int h, int w,
                                                         int LS, int nstrip, int nseg, int planes) {
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    k3_strip<T, VEC, F>(coef + plane * lw, R + plane * hw, G + plane * hw, dG ? dG + plane * hw : nullptr,
                        dcoef + plane * lw, h_l, w_l, h, w, strip, sg * LS, min(sg * LS + LS, h_l));
}

// K3 fast path with TMA staging (16-byte vectors): same decomposition,
// WPC warps per CTA, each warp's blocks staged through its own slot ring.
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(K3Tma<T, VEC, F>::WPC * 32)
    k3_hires_bwd_tma(const float2* __restrict__ coef, const __grid_constant__ K3Maps maps, T* __restrict__ dG,
                     float2* __restrict__ dcoef, int h_l, int w_l, int h, int w, int LS, int nstrip, int nseg,
                     int planes, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char k3ring[];
    using B = K3Tma<T, VEC, F>;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * B::WPC + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    unsigned char* ring = k3ring + (size_t)warp * B::NSB * B::SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k3ring + (size_t)B::WPC * B::NSB * B::SLOT) + warp * B::NSB;
    k3_strip_tma<T, VEC, F>(coef + plane * lw, &maps, dG ? dG + plane * hw : nullptr, dcoef + plane * lw, h_l, w_l,
                            h, w, strip, sg * LS, min(sg * LS + LS, h_l), plane, ring, bars, status);
}

// -------------------------------------------------- K3 general (any ratio)
// One thread per low-res (i, j): sum over the high-res rows/columns whose
// (clamped) taps include it.  Slow but exact for every size; the fast tile
// above covers integer factors.
template <typename T, typename TG = T>
__global__ void __launch_bounds__(kThreads) k3_gather_general(const T* __restrict__ R, const TG* __restrict__ G,
                                                              float2* __restrict__ dcoef, int h_l, int w_l,
                                                              int h, int w) {
    const size_t plane = blockIdx.z;
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * kWarps + (threadIdx.x >> 5);
    if (i >= h_l || j >= w_l) return;
    R += plane * h * w;
    G += plane * h * w;
    const long long ylo_ll = ((long long)(i - 1) * h) / h_l - 2;
    const long long yhi_ll = ((long long)(i + 2) * h) / h_l + 2;
    const long long xlo_ll = ((long long)(j - 1) * w) / w_l - 2;
    const long long xhi_ll = ((long long)(j + 2) * w) / w_l + 2;
    const int ylo = (int)max(ylo_ll, 0LL), yhi = (int)min(yhi_ll, (long long)h - 1);
    const int xlo = (int)max(xlo_ll, 0LL), xhi = (int)min(xhi_ll, (long long)w - 1);
    float su = 0.f, sv = 0.f;
    for (int y = ylo; y <= yhi; ++y) {
        const Tap ty = tap_general(y, h_l, h);
        const int a0 = min(ty.i0, h_l - 1), a1 = min(ty.i0 + 1, h_l - 1);
        const float wy = (a0 == i ? 1.f - ty.lam : 0.f) + (a1 == i ? ty.lam : 0.f);
        if (wy == 0.f) continue;
        float ru = 0.f, rv = 0.f;
        for (int x = xlo; x <= xhi; ++x) {
            const Tap tx = tap_general(x, w_l, w);
            const int b0 = min(tx.i0, w_l - 1), b1 = min(tx.i0 + 1, w_l - 1);
            const float wx = (b0 == j ? 1.f - tx.lam : 0.f) + (b1 == j ? tx.lam : 0.f);
            if (wx == 0.f) continue;
            const float r = to_f32<T>(R[(size_t)y * w + x]);
            ru = fmaf(wx, r * to_f32<TG>(G[(size_t)y * w + x]), ru);
            rv = fmaf(wx, r, rv);
        }
        su = fmaf(wy, ru, su);
        sv = fmaf(wy, rv, sv);
    }
    dcoef[plane * h_l * w_l + (size_t)i * w_l + j] = make_float2(su, sv);
}

// K2 strips (integer F dividing VEC): warp w of the grid owns strip
// (w % nstrip) of segment (w / nstrip) % nseg (LS low-res rows) of plane
// w / (nstrip nseg).
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(kThreads) k2_apply_strip(const float2* __restrict__ coef, const T* __restrict__ in,
                                                           T* __restrict__ out, int h_l, int w_l, int h, int w, int LS,
                                                           int nstrip, int nseg, int planes) {
    extern __shared__ __align__(128) unsigned char k2slots[];
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kWarps + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    k2_strip_async<T, VEC, F>(coef + plane * lw, in + plane * hw, out + plane * hw, h_l, w_l, h, w, strip, sg * LS,
                              min(sg * LS + LS, h_l), k2slots + warp * K2Async<T, VEC, F>::WARP_BYTES);
}

template <typename T, int VEC, int F>
__global__ void __launch_bounds__(K2Tma<T, VEC, F>::WPC * 32)
    k2_apply_strip_tma(const float2* __restrict__ coef, const __grid_constant__ K2Map map, T* __restrict__ out,
                       int h_l, int w_l, int h, int w, int LS, int nstrip, int nseg, int planes, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char k2ring[];
    using B = K2Tma<T, VEC, F>;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * B::WPC + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    unsigned char* ring = k2ring + (size_t)warp * B::NSB * B::SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k2ring + (size_t)B::WPC * B::NSB * B::SLOT) + warp * B::NSB;
    k2_strip_tma<T, VEC, F>(coef + plane * lw, &map.m, out + plane * hw, h_l, w_l, h, w, strip, sg * LS,
                            min(sg * LS + LS, h_l), plane, ring, bars, status);
}

// ------------------------------------------------------- batched K2 (persistent)
template <typename T, int VEC, int F>
__device__ __forceinline__ void apply_batched_tile(const BatchImage& im, int local, float2* sAB) {
    if constexpr (F > 0 && VEC % F == 0) {
        // strips: a work item is kWarps strip segments, one per warp (k2_th = LS)
        const int nstrip = (im.w_l + 32 * (VEC / F) - 1) / (32 * (VEC / F));
        const int nseg = (im.h_l + im.k2_th - 1) / im.k2_th;
        const int plane = local / im.k2_nx;
        const int item = (local - plane * im.k2_nx) * kWarps + (threadIdx.x >> 5);
        if (item < nstrip * nseg) {  // warp-uniform; no barrier follows
            const int strip = item % nstrip, sg = item / nstrip;
            const size_t hw = (size_t)im.h * im.w, lw = (size_t)im.h_l * im.w_l;
            k2_strip_async<T, VEC, F>(im.coef + plane * lw, static_cast<const T*>(im.I_h) + plane * hw,
                                      static_cast<T*>(im.O_h) + plane * hw, im.h_l, im.w_l, im.h, im.w, strip,
                                      sg * im.k2_th, min(sg * im.k2_th + im.k2_th, im.h_l),
                                      reinterpret_cast<unsigned char*>(sAB) +
                                          (threadIdx.x >> 5) * K2Async<T, VEC, F>::WARP_BYTES);
        }
        return;
    }
    const int per_plane = im.k2_nx * im.k2_ny;
    const int plane = local / per_plane;
    const int tp = local - plane * per_plane;
    const int ty = tp / im.k2_nx, tx = tp - ty * im.k2_nx;
    const size_t hw = (size_t)im.h * im.w, lw = (size_t)im.h_l * im.w_l;
    const int pitch = k2_pitch(VEC, F, im.w_l, im.w);
    apply_tile<T, VEC, F, 0>(im.coef + plane * lw, static_cast<const T*>(im.I_h) + plane * hw,
                             static_cast<T*>(im.O_h) + plane * hw, im.h_l, im.w_l, im.h, im.w,
                             ty * im.k2_th, tx * 32 * VEC, im.k2_th, pitch, sAB);
}

// One persistent kernel per (storage type, vector width, factor) class:
// each graph node walks the flat tile list of the images of its class.
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(kThreads) k2_apply_batched(const __grid_constant__ BatchParams bp, uint32_t*) {
    extern __shared__ __align__(128) float2 sAB[];
    for (int tile = blockIdx.x; tile < bp.k2_total; tile += gridDim.x) {
        const int i = batch_find(bp.k2_start, bp.n, tile);
        apply_batched_tile<T, VEC, F>(bp.img[i], tile - bp.k2_start[i], sAB);
    }
}

// K2 strips staged by TMA (16-byte vectors; every image of the class has a
// tensor map of I_h in device memory): a work item is WPC strip segments of
// one plane, one per warp, each with its own slot ring (k2_th = LS).
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(K2Tma<T, VEC, F>::WPC * 32)
    k2_strip_batched_tma(const __grid_constant__ BatchParams bp, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char k2bring[];
    using B = K2Tma<T, VEC, F>;
    const int warp = threadIdx.x >> 5;
    unsigned char* ring = k2bring + (size_t)warp * B::NSB * B::SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k2bring + (size_t)B::WPC * B::NSB * B::SLOT) + warp * B::NSB;
    for (int tile = blockIdx.x; tile < bp.k2_total; tile += gridDim.x) {
        const int i = batch_find(bp.k2_start, bp.n, tile);
        const BatchImage& im = bp.img[i];
        const int local = tile - bp.k2_start[i];
        const int nstrip = (im.w_l + 32 * (VEC / F) - 1) / (32 * (VEC / F));
        const int nseg = (im.h_l + im.k2_th - 1) / im.k2_th;
        const int plane = local / im.k2_nx;
        const int item = (local - plane * im.k2_nx) * B::WPC + warp;
        if (item >= nstrip * nseg) continue;  // warp-uniform; no barrier follows
        const int strip = item % nstrip, sg = item / nstrip;
        const CUtensorMap* map = static_cast<const CUtensorMap*>(im.k2_map);
        if ((threadIdx.x & 31) == 0) tensormap_acquire(map);
        __syncwarp();
        const size_t hw = (size_t)im.h * im.w, lw = (size_t)im.h_l * im.w_l;
        if (!k2_strip_tma<T, VEC, F>(im.coef + plane * lw, map, static_cast<T*>(im.O_h) + plane * hw, im.h_l, im.w_l,
                                     im.h, im.w, strip, sg * im.k2_th, min(sg * im.k2_th + im.k2_th, im.h_l), plane,
                                     ring, bars, status))
            return;  // timeout recorded; this warp stops
    }
}

// ------------------------------------------------------------------ host side
// rows of the raw low-res coefficient block a K2 tile of TH rows touches
static int k2_raw_rows(int F, int h_l, int h, int TH) {
    if (F > 0) return TH / F + 3;
    return (int)(((long long)TH * h_l + h - 1) / h) + 3;
}

size_t k2_smem_bytes(int vec, int F, int h_l, int h, int w_l, int w, int TH) {
    return (size_t)(TH + k2_raw_rows(F, h_l, h, TH)) * k2_pitch(vec, F, w_l, w) * sizeof(float2);
}

bool k3_fast_ok(int vec, int F) {
    return (vec == 8 && (F == 4 || F == 8)) || (vec == 4 && (F == 4 || F == 2)) ||
           (vec == 2 && F == 2);
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

bool k2_strip_ok(int vec, int F) { return (F == 2 || F == 4 || F == 8) && vec >= F && vec % F == 0; }

size_t k2_strip_batched_smem(int esize, int vec, int F) {
    const int nsb = F == 2 ? 6 : (F == 4 ? 3 : 2);
    return (size_t)kWarps * nsb * (32 * vec) * F * esize;
}

// Segment length near `ls` whose grid fills whole waves of the kernel's
// resident CTA slots, so no SM idles through a last partial wave (the strip
// kernels give the same bits at every segment length).  `halo`: extra
// low-res rows a segment walks besides its own.
static std::mutex g_occ_mu;
static std::map<const void*, int> g_occ;  // resident CTAs per SM, per kernel
static int g_occ_sms = 0;

template <typename K>
static int wave_fit_ls(K kern, int threads, size_t smem, int ls, int nstrip, int rows, int planes, int wpc,
                       float halo) {
    int occ = 0, sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        if (g_occ_sms == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&g_occ_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                g_occ_sms = 152;
            }
        }
        sms = g_occ_sms;
        auto it = g_occ.find((const void*)kern);
        if (it == g_occ.end()) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
                cudaGetLastError();
                occ = 0;
            }
            g_occ[(const void*)kern] = occ;
        } else {
            occ = it->second;
        }
    }
    if (occ <= 0 || ls < 2) return ls;
    const double slots = (double)occ * sms;
    int best = ls;
    double best_cost = 1e30;
    for (int c = std::max(2, ls / 2); c <= ls + ls / 2; ++c) {
        const long long ctas = ((long long)nstrip * ((rows + c - 1) / c) * planes + wpc - 1) / wpc;
        const double waves = (double)ctas / slots;
        const double eff = waves / std::ceil(waves);
        const double cost = (c + halo) / (double)c / eff;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

template <typename T, int VEC, int F>
static cudaError_t k2s_go(const float2* coef, const void* in, void* out, int planes, int h_l, int w_l, int h, int w,
                          int LS, const K2Map* map, uint32_t* status, cudaStream_t s) {
    const int nstrip = (w_l + 32 * (VEC / F) - 1) / (32 * (VEC / F));
    if constexpr (VEC * sizeof(T) == 16) {
        if (map != nullptr) {
            using B = K2Tma<T, VEC, F>;
            auto kern = k2_apply_strip_tma<T, VEC, F>;
            cudaError_t e = prep(kern, B::CTA_BYTES);
            if (e != cudaSuccess) return e;
            LS = wave_fit_ls(kern, B::WPC * 32, B::CTA_BYTES, LS, nstrip, h_l, planes, B::WPC, 0.25f);
            const int nseg = (h_l + LS - 1) / LS;
            const long long warps = (long long)nstrip * nseg * planes;
            const int ctas = (int)((warps + B::WPC - 1) / B::WPC);
            kern<<<ctas, B::WPC * 32, B::CTA_BYTES, s>>>(coef, *map, static_cast<T*>(out), h_l, w_l, h, w, LS, nstrip,
                                                          nseg, planes, status);
            return cudaGetLastError();
        }
    }
    constexpr size_t smem = kWarps * K2Async<T, VEC, F>::WARP_BYTES;
    auto kern = k2_apply_strip<T, VEC, F>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    LS = wave_fit_ls(kern, kThreads, smem, LS, nstrip, h_l, planes, kWarps, 0.25f);
    const int nseg = (h_l + LS - 1) / LS;
    const long long warps = (long long)nstrip * nseg * planes;
    const int ctas = (int)((warps + kWarps - 1) / kWarps);
    kern<<<ctas, kThreads, smem, s>>>(coef, static_cast<const T*>(in), static_cast<T*>(out), h_l, w_l, h, w, LS,
                                      nstrip, nseg, planes);
    return cudaGetLastError();
}

template <typename T, int VEC, int F, int MODE, typename TI = T>
static cudaError_t k2_go(const float2* coef, const void* in, void* out, int planes, int h_l, int w_l,
                         int h, int w, int TH, cudaStream_t s) {
    const int pitch = k2_pitch(VEC, F, w_l, w);
    const size_t smem = k2_smem_bytes(VEC, F, h_l, h, w_l, w, TH);
    auto kern = k2_apply<T, VEC, F, MODE, TI>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + 32 * VEC - 1) / (32 * VEC), (h + TH - 1) / TH, planes);
    kern<<<grid, kThreads, smem, s>>>(coef, static_cast<const TI*>(in), static_cast<T*>(out), h_l, w_l, h,
                                      w, TH, pitch);
    return cudaGetLastError();
}

template <typename T, int MODE, typename TI = T>
static cudaError_t k2_dispatch(const float2* coef, const void* in, void* out, int planes, int h_l,
                               int w_l, int h, int w, int vec, int F, int TH, cudaStream_t s) {
    constexpr int VW = 16 / sizeof(T), VH = 8 / sizeof(T);
    if (vec == VW) {
        if (F == 4) return k2_go<T, VW, 4, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
        if (F == 8) return k2_go<T, VW, 8, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
        return k2_go<T, VW, 0, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
    }
    if (vec == VH) {
        if (F == 4) return k2_go<T, VH, 4, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
        if (F == 8) return k2_go<T, VH, 8, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
        return k2_go<T, VH, 0, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
    }
    return k2_go<T, 1, 0, MODE, TI>(coef, in, out, planes, h_l, w_l, h, w, TH, s);
}

template <typename T>
static cudaError_t k2s_dispatch(const float2* coef, const void* in, void* out, int planes, int h_l, int w_l, int h,
                                int w, int vec, int F, int LS, const K2Map* map, uint32_t* status, cudaStream_t s) {
    constexpr int VW = 16 / sizeof(T), VH = 8 / sizeof(T);
#define DGF_K2S(V, FF)                                                                                        \
    if (vec == V && F == FF) return k2s_go<T, V, FF>(coef, in, out, planes, h_l, w_l, h, w, LS, map, status, s);
    DGF_K2S(VW, 2)
    DGF_K2S(VW, 4)
    if constexpr (VW >= 8) { DGF_K2S(VW, 8) }
    DGF_K2S(VH, 2)
    if constexpr (VH >= 4) { DGF_K2S(VH, 4) }
#undef DGF_K2S
    return cudaErrorInvalidValue;
}

cudaError_t launch_k2_strip(dgf_dtype dt, const float2* coef, const void* in, void* out, int planes, int h_l,
                            int w_l, int h, int w, int vec, int F, int LS, const K2Map* map, uint32_t* status,
                            cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k2s_dispatch<float>(coef, in, out, planes, h_l, w_l, h, w, vec, F, LS, map, status, s);
        case DGF_BF16:
            return k2s_dispatch<__nv_bfloat16>(coef, in, out, planes, h_l, w_l, h, w, vec, F, LS, map, status, s);
        case DGF_F16: return k2s_dispatch<__half>(coef, in, out, planes, h_l, w_l, h, w, vec, F, LS, map, status, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_k2(dgf_dtype dt, int mode, const float2* coef, const void* in, void* out, int planes,
                      int h_l, int w_l, int h, int w, int vec, int F, int TH, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32:
            return mode == 0 ? k2_dispatch<float, 0>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s)
                             : k2_dispatch<float, 1>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
        case DGF_BF16:
            return mode == 0 ? k2_dispatch<__nv_bfloat16, 0>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s)
                             : k2_dispatch<__nv_bfloat16, 1>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
        case DGF_F16:
            return mode == 0 ? k2_dispatch<__half, 0>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s)
                             : k2_dispatch<__half, 1>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
    }
    return cudaErrorInvalidValue;
}

// K2 tiles (MODE 0) reading an FP32 guide while storing O_h in the 16-bit
// type dt (a grey guide held in FP32 over 16-bit data).
cudaError_t launch_k2_guide_f32(dgf_dtype dt, const float2* coef, const float* in, void* out, int planes, int h_l,
                                int w_l, int h, int w, int vec, int F, int TH, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k2_dispatch<float, 0>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
        case DGF_BF16:
            return k2_dispatch<__nv_bfloat16, 0, float>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
        case DGF_F16: return k2_dispatch<__half, 0, float>(coef, in, out, planes, h_l, w_l, h, w, vec, F, TH, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int VEC, int F>
static cudaError_t k3_go(const float2* coef, const void* R, const void* G, void* dG, float2* dcoef,
                         int planes, int h_l, int w_l, int h, int w, int LS, const K3Maps* maps, uint32_t* status,
                         cudaStream_t s) {
    constexpr int OUT = K3Strip<VEC, F>::OUT;
    const int nstrip = (w_l + OUT - 1) / OUT;
    if constexpr (VEC * sizeof(T) == 16) {
        if (maps != nullptr) {
            using B = K3Tma<T, VEC, F>;
            auto kern = k3_hires_bwd_tma<T, VEC, F>;
            cudaError_t e = prep(kern, B::CTA_BYTES);
            if (e != cudaSuccess) return e;
            LS = wave_fit_ls(kern, B::WPC * 32, B::CTA_BYTES, LS, nstrip, h_l, planes, B::WPC, 1.f);
            const int nseg = (h_l + LS - 1) / LS;
            const long long warps = (long long)nstrip * nseg * planes;
            const int ctas = (int)((warps + B::WPC - 1) / B::WPC);
            kern<<<ctas, B::WPC * 32, B::CTA_BYTES, s>>>(coef, *maps, static_cast<T*>(dG), dcoef, h_l, w_l, h, w,
                                                          LS, nstrip, nseg, planes, status);
            return cudaGetLastError();
        }
    }
    LS = wave_fit_ls(k3_hires_bwd<T, VEC, F>, kThreads, 0, LS, nstrip, h_l, planes, kWarps, 1.f);
    const int nseg = (h_l + LS - 1) / LS;
    const long long warps = (long long)nstrip * nseg * planes;
    const int ctas = (int)((warps + kWarps - 1) / kWarps);
    k3_hires_bwd<T, VEC, F><<<ctas, kThreads, 0, s>>>(coef, static_cast<const T*>(R), static_cast<const T*>(G),
                                                      static_cast<T*>(dG), dcoef, h_l, w_l, h, w, LS, nstrip, nseg,
                                                      planes);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t k3_dispatch(const float2* coef, const void* R, const void* G, void* dG, float2* dcoef,
                               int planes, int h_l, int w_l, int h, int w, int vec, int F, int LTH,
                               const K3Maps* maps, uint32_t* status, cudaStream_t s) {
    if constexpr (sizeof(T) == 2) {
        if (vec == 8 && F == 4) return k3_go<T, 8, 4>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
        if (vec == 8 && F == 8) return k3_go<T, 8, 8>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
        if (vec == 4 && F == 4) return k3_go<T, 4, 4>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
        if (vec == 4 && F == 2) return k3_go<T, 4, 2>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
    } else {
        if (vec == 4 && F == 4) return k3_go<T, 4, 4>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
        if (vec == 4 && F == 2) return k3_go<T, 4, 2>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
        if (vec == 2 && F == 2) return k3_go<T, 2, 2>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, LTH, maps, status, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_k3(dgf_dtype dt, const float2* coef, const void* R, const void* G, void* dG,
                      float2* dcoef, int planes, int h_l, int w_l, int h, int w, int vec, int F, int LTH,
                      const K3Maps* maps, uint32_t* status, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k3_dispatch<float>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, vec, F, LTH, maps, status, s);
        case DGF_BF16: return k3_dispatch<__nv_bfloat16>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, vec, F, LTH, maps, status, s);
        case DGF_F16: return k3_dispatch<__half>(coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, vec, F, LTH, maps, status, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, typename TG = T>
static cudaError_t k3g_go(const void* R, const void* G, float2* dcoef, int planes, int h_l, int w_l, int h,
                          int w, cudaStream_t s) {
    dim3 grid((w_l + 31) / 32, (h_l + kWarps - 1) / kWarps, planes);
    k3_gather_general<T, TG><<<grid, kThreads, 0, s>>>(static_cast<const T*>(R), static_cast<const TG*>(G), dcoef,
                                                       h_l, w_l, h, w);
    return cudaGetLastError();
}

cudaError_t launch_k3_general(dgf_dtype dt, const void* R, const void* G, float2* dcoef, int planes,
                              int h_l, int w_l, int h, int w, cudaStream_t s, bool guide_f32) {
    if (planes == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k3g_go<float>(R, G, dcoef, planes, h_l, w_l, h, w, s);
        case DGF_BF16:
            return guide_f32 ? k3g_go<__nv_bfloat16, float>(R, G, dcoef, planes, h_l, w_l, h, w, s)
                             : k3g_go<__nv_bfloat16>(R, G, dcoef, planes, h_l, w_l, h, w, s);
        case DGF_F16:
            return guide_f32 ? k3g_go<__half, float>(R, G, dcoef, planes, h_l, w_l, h, w, s)
                             : k3g_go<__half>(R, G, dcoef, planes, h_l, w_l, h, w, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int VEC, int F>
static cudaError_t k2b_get(size_t smem, void** fn) {
    *fn = (void*)k2_apply_batched<T, VEC, F>;
    return prep(k2_apply_batched<T, VEC, F>, smem);
}

template <typename T>
static cudaError_t k2b_dispatch(int vec, int F, size_t smem, void** fn) {
    constexpr int VW = 16 / sizeof(T), VH = 8 / sizeof(T);
    if (vec == VW) {
        if (F == 2) return k2b_get<T, VW, 2>(smem, fn);
        if (F == 4) return k2b_get<T, VW, 4>(smem, fn);
        if (F == 8) return k2b_get<T, VW, 8>(smem, fn);
        return k2b_get<T, VW, 0>(smem, fn);
    }
    if (vec == VH) {
        if (F == 2) return k2b_get<T, VH, 2>(smem, fn);
        if (F == 4) return k2b_get<T, VH, 4>(smem, fn);
        if (F == 8) return k2b_get<T, VH, 8>(smem, fn);
        return k2b_get<T, VH, 0>(smem, fn);
    }
    return k2b_get<T, 1, 0>(smem, fn);
}

template <typename T, int VEC, int F>
static cudaError_t k2bt_get(void** fn, size_t* smem, int* threads) {
    using B = K2Tma<T, VEC, F>;
    *fn = (void*)k2_strip_batched_tma<T, VEC, F>;
    *smem = B::CTA_BYTES;
    *threads = B::WPC * 32;
    return prep(k2_strip_batched_tma<T, VEC, F>, B::CTA_BYTES);
}

template <typename T>
static cudaError_t k2bt_dispatch(int vec, int F, void** fn, size_t* smem, int* threads) {
    constexpr int VW = 16 / sizeof(T);
    if (vec == VW) {
        if (F == 2) return k2bt_get<T, VW, 2>(fn, smem, threads);
        if (F == 4) return k2bt_get<T, VW, 4>(fn, smem, threads);
        if constexpr (VW >= 8)
            if (F == 8) return k2bt_get<T, VW, 8>(fn, smem, threads);
    }
    return cudaErrorInvalidValue;
}

cudaError_t k2_batched_tma_kernel(dgf_dtype dt, int vec, int F, void** fn, size_t* smem, int* threads) {
    switch (dt) {
        case DGF_F32: return k2bt_dispatch<float>(vec, F, fn, smem, threads);
        case DGF_BF16: return k2bt_dispatch<__nv_bfloat16>(vec, F, fn, smem, threads);
        case DGF_F16: return k2bt_dispatch<__half>(vec, F, fn, smem, threads);
    }
    return cudaErrorInvalidValue;
}

cudaError_t k2_batched_kernel(dgf_dtype dt, int vec, int F, size_t smem, void** fn) {
    switch (dt) {
        case DGF_F32: return k2b_dispatch<float>(vec, F, smem, fn);
        case DGF_BF16: return k2b_dispatch<__nv_bfloat16>(vec, F, smem, fn);
        case DGF_F16: return k2b_dispatch<__half>(vec, F, smem, fn);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
