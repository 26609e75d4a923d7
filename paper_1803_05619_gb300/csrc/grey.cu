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
// With an integer factor F in {2, 4, 8} the high-resolution guide is never
// materialised: the high-resolution kernels read the n_I guide channels and
// form the same FP32 mean in registers.
//   K2grey  O_h[n, c] = Abar_h[n, c] G_h[n] + bbar_h[n, c] for all C output
//           channels of a tile, the grey G_h formed once per pixel
//   K3grey  the transposed upsampler of Algorithm 1 per output channel
//           (d Abar, d bbar from d O_h G_h and d O_h), and
//           d I_h[n, k] = (sum over c of d O_h[n, c] Abar_h[n, c]) / n_I for
//           every guide channel k, written once per pixel from FP32 sums
// Only the low-resolution guide (small) still goes through KG and KGT.
#include "hires.cuh"
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


// ------------------------------------------------------------------ K2grey
// Rows of a tile are walked with the next row's guide vectors already in
// flight.  NI, NC > 0 fix the guide and output channel counts at compile time
// (the RGB guide with one output channel); 0 takes them from the arguments.
template <typename T, int VEC, int NI>
struct GreyRow {
    static constexpr int kN = NI > 0 ? NI : 1;
    Vec<T, VEC> x[kN];
};

// The grey guide of VEC pixels: the channels summed in order in FP32, one
// division by n_I.
template <typename T, int VEC, int NI>
__device__ __forceinline__ void grey_of(const GreyRow<T, VEC, NI>& row, float (&g)[VEC], float nf) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) g[k] = to_f32<T>(row.x[0].v[k]);
#pragma unroll
    for (int ci = 1; ci < NI; ++ci)
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[k] = __fadd_rn(g[k], to_f32<T>(row.x[ci].v[k]));
    if (NI != 1) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) g[k] = __fdiv_rn(g[k], nf);
    }
}

// One CTA per tile of TH high-res rows x 32 VEC columns of one image: the
// y-interpolated coefficients of all C output channels staged in shared
// memory (as the K2 tiles do: one column per low-res column of the tile plus
// a replicated border column on each side), then each warp walks its rows,
// forms the grey guide of VEC pixels from the n_I guide channels and writes
// the C output channels.
template <typename T, int VEC, int F, int NI, int NC>
__global__ void __launch_bounds__(kThreads) k2_grey_apply(const float2* __restrict__ coef, const T* __restrict__ I_h,
                                                          T* __restrict__ O_h, int C_arg, int n_in_arg, int h_l,
                                                          int w_l, int h, int w, int TH) {
    extern __shared__ __align__(16) float2 sAB[];  // [C][TH][pitch]
    constexpr int TW = 32 * VEC;
    constexpr int pitch = TW / F + 2;
    const int C = NC > 0 ? NC : C_arg, n_in = NI > 0 ? NI : n_in_arg;
    const size_t n = blockIdx.z;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    const int Y0 = blockIdx.y * TH, X0 = blockIdx.x * TW;
    const int jlo = X0 / F - 1;
    const int nst = C * TH * pitch;
    for (int idx = threadIdx.x; idx < nst; idx += kThreads) {
        const int ch = idx / (TH * pitch);
        const int rem = idx - ch * TH * pitch;
        const int i = rem / pitch, c = rem - i * pitch;
        const int y = Y0 + i;
        if (y >= h) continue;
        const int q = y % F, j = y / F, t2 = 2 * q + 1 - F;
        const int yi0 = t2 < 0 ? j - 1 : j;
        const float lam = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
        const int r0 = clampi(yi0, 0, h_l - 1), r1 = clampi(yi0 + 1, 0, h_l - 1);
        const int jj = clampi(jlo + c, 0, w_l - 1);
        const float2* cp = coef + (n * C + ch) * lw;
        const float2 a = cp[(size_t)r0 * w_l + jj], b = cp[(size_t)r1 * w_l + jj];
        sAB[idx] = make_float2(lerp(a.x, b.x, lam), lerp(a.y, b.y, lam));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = X0 + lane * VEC;
    if (xs >= w) return;  // w is a multiple of VEC: a vector is wholly inside or outside
    int cc[VEC];
    float ll[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) col_tap<F>(lane * VEC + k, cc[k], ll[k]);
    const float nf = (float)n_in;
    const int rows = min(TH, h - Y0);
    const T* src = I_h + n * n_in * hw + xs;
    auto store_row = [&](int i, const float (&g)[VEC]) {
        const size_t px = (size_t)(Y0 + i) * w + xs;
        for (int c = 0; c < C; ++c) {
            const float2* row = sAB + (c * TH + i) * pitch;
            float o[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const float2 s0 = row[cc[k]], s1 = row[cc[k] + 1];
                o[k] = fmaf(lerp(s0.x, s1.x, ll[k]), g[k], lerp(s0.y, s1.y, ll[k]));
            }
            store_vec<T, VEC>(O_h + (n * C + c) * hw + px, o);
        }
    };
    if constexpr (NI > 0) {
        GreyRow<T, VEC, NI> cur, nxt;
        auto load = [&](int i, GreyRow<T, VEC, NI>& rr) {
            const T* p = src + (size_t)(Y0 + i) * w;
#pragma unroll
            for (int ci = 0; ci < NI; ++ci) rr.x[ci] = ldg_vec<T, VEC>(p + ci * hw);
        };
        if (warp < rows) load(warp, cur);
        for (int i = warp; i < rows; i += kWarps) {
            if (i + kWarps < rows) load(i + kWarps, nxt);
            float g[VEC];
            grey_of<T, VEC, NI>(cur, g, nf);
            store_row(i, g);
            cur = nxt;
        }
    } else {
        for (int i = warp; i < rows; i += kWarps) {
            const T* p = src + (size_t)(Y0 + i) * w;
            float g[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) g[k] = 0.f;
            for (int ci = 0; ci < n_in; ++ci) {
                float x[VEC];
                load_vec<T, VEC>(p + ci * hw, x);
#pragma unroll
                for (int k = 0; k < VEC; ++k) g[k] = __fadd_rn(g[k], x[k]);
            }
            if (n_in != 1) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) g[k] = __fdiv_rn(g[k], nf);
            }
            store_row(i, g);
        }
    }
}

// ------------------------------------------------------------------ K3grey
// One CTA per tile of LTH x LTW low-res cells of one image (the K3 tile of
// the guidance-transform backward): every high-res row whose bilinear taps
// reach the tile is read once (d O_h of the C channels, the n_I guide
// channels), its row partials of d O_h G_h and d O_h land in shared memory
// per output channel, and a column pass gathers d Abar, d bbar of the owned
// cells.  The tile also owns the high-res pixels of its cells (rows
// F i0 .. F (i0 + LTH) - 1, columns F j0 .. F (j0 + LTW) - 1: whole lane
// vectors 1 .. F LTW / VEC of its rows), for which it writes d I_h from
// Abar_h (y-interpolated into shared memory before the walk).  With NI, NC
// fixed the next row's inputs are in flight while a row is processed.
template <typename T, int VEC, int F, int NI, int NC>
__global__ void __launch_bounds__(kThreads) k3_grey_bwd(const T* __restrict__ R, const T* __restrict__ I_h,
                                                        const float2* __restrict__ coef, float2* __restrict__ dcoef,
                                                        T* __restrict__ dI_h, int C_arg, int n_in_arg, int h_l,
                                                        int w_l, int h, int w, int LTH) {
    extern __shared__ __align__(16) float smem[];
    using S = K3Shape<VEC, F>;
    constexpr int H0 = S::H0, LTW = S::LTW, SXP = S::SXP;
    constexpr int kOwnLanes = F * LTW / VEC;
    const int C = NC > 0 ? NC : C_arg, n_in = NI > 0 ? NI : n_in_arg;
    const size_t n = blockIdx.z;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    const int i0 = blockIdx.y * LTH, j0 = blockIdx.x * LTW;
    const int FR = F * (LTH + 1), OR = F * LTH;
    const int yf0 = F * (i0 - 1) + H0;
    const int XS = F * j0 - VEC;
    float2* Sx = reinterpret_cast<float2*>(smem);  // [C][FR][SXP]
    float* Ay = smem + 2 * C * FR * SXP;           // [C][OR][SXP] (only with d I_h)
    if (dI_h != nullptr) {
        // Abar along y for the owned rows, low-res columns j0 - 1 .. j0 + LTW (clamped)
        const int nst = C * OR * SXP;
        for (int idx = threadIdx.x; idx < nst; idx += kThreads) {
            const int ch = idx / (OR * SXP);
            const int rem = idx - ch * OR * SXP;
            const int oy = rem / SXP, c = rem - oy * SXP;
            const int y = F * i0 + oy;
            if (y >= h) continue;
            const int q = y % F, j = y / F, t2 = 2 * q + 1 - F;
            const int yi0 = t2 < 0 ? j - 1 : j;
            const float lam = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
            const int r0 = clampi(yi0, 0, h_l - 1), r1 = clampi(yi0 + 1, 0, h_l - 1);
            const int jj = clampi(j0 - 1 + c, 0, w_l - 1);
            const float2* cp = coef + (n * C + ch) * lw;
            Ay[idx] = lerp(cp[(size_t)r0 * w_l + jj].x, cp[(size_t)r1 * w_l + jj].x, lam);
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = XS + lane * VEC;
    const bool col_ok = xs >= 0 && xs < w;
    const bool own_col = dI_h != nullptr && lane >= 1 && lane <= kOwnLanes && xs < w;
    int cc[VEC];
    float ll[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) col_tap<F>(own_col ? (lane - 1) * VEC + k : 0, cc[k], ll[k]);
    const float nf = (float)n_in;
    const T* gsrc = I_h + n * n_in * hw + (col_ok ? xs : 0);
    const T* rsrc = R + n * C * hw + (col_ok ? xs : 0);
    auto row_ok = [&](int fr) {
        const int y = yf0 + fr;
        return col_ok && y >= 0 && y < h;
    };
    // one row: g = the grey guide, rr(c) = d O_h of channel c (zeros outside the image)
    auto process = [&](int fr, const float (&g)[VEC], auto&& rr_of) {
        const int y = yf0 + fr;
        const int oy = y - F * i0;
        const bool own = own_col && oy >= 0 && oy < OR && y < h;
        float dg[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) dg[k] = 0.f;
        auto one = [&](int c) {
            float rr[VEC], u[VEC];
            rr_of(c, rr);
#pragma unroll
            for (int k = 0; k < VEC; ++k) u[k] = rr[k] * g[k];
            k3_row_to_smem<VEC, F>(u, rr, lane, Sx + (c * FR + fr) * SXP);
            if (own) {
                const float* arow = Ay + (c * OR + oy) * SXP;
#pragma unroll
                for (int k = 0; k < VEC; ++k) dg[k] = fmaf(rr[k], lerp(arow[cc[k]], arow[cc[k] + 1], ll[k]), dg[k]);
            }
        };
        if constexpr (NC > 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) one(c);
        } else {
            for (int c = 0; c < C; ++c) one(c);
        }
        if (own) {
            if (n_in != 1) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) dg[k] = __fdiv_rn(dg[k], nf);
            }
            const size_t px = (size_t)y * w + xs;
            for (int ci = 0; ci < n_in; ++ci) store_vec<T, VEC>(dI_h + (n * n_in + ci) * hw + px, dg);
        }
    };
    if constexpr (NI > 0 && NC > 0) {
        struct Row {
            GreyRow<T, VEC, NI> x;
            Vec<T, VEC> r[NC];
        };
        Vec<T, VEC> zero;
#pragma unroll
        for (int k = 0; k < VEC; ++k) zero.v[k] = from_f32<T>(0.f);
        auto load = [&](int fr, Row& rw) {
            if (row_ok(fr)) {
                const size_t off = (size_t)(yf0 + fr) * w;
#pragma unroll
                for (int ci = 0; ci < NI; ++ci) rw.x.x[ci] = ldg_vec<T, VEC>(gsrc + off + ci * hw);
#pragma unroll
                for (int c = 0; c < NC; ++c) rw.r[c] = ldg_vec<T, VEC>(rsrc + off + c * hw);
            } else {
#pragma unroll
                for (int ci = 0; ci < NI; ++ci) rw.x.x[ci] = zero;
#pragma unroll
                for (int c = 0; c < NC; ++c) rw.r[c] = zero;
            }
        };
        Row cur, nxt;
        if (warp < FR) load(warp, cur);
        for (int fr = warp; fr < FR; fr += kWarps) {
            if (fr + kWarps < FR) load(fr + kWarps, nxt);
            float g[VEC];
            grey_of<T, VEC, NI>(cur.x, g, nf);
            process(fr, g, [&](int c, float (&rr)[VEC]) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) rr[k] = to_f32<T>(cur.r[c].v[k]);
            });
            cur = nxt;
        }
    } else {
        for (int fr = warp; fr < FR; fr += kWarps) {
            const bool ok = row_ok(fr);
            const size_t off = (size_t)(yf0 + fr) * w;
            float g[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) g[k] = 0.f;
            if (ok) {
                for (int ci = 0; ci < n_in; ++ci) {
                    float x[VEC];
                    load_vec<T, VEC>(gsrc + off + ci * hw, x);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) g[k] = __fadd_rn(g[k], x[k]);
                }
                if (n_in != 1) {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) g[k] = __fdiv_rn(g[k], nf);
                }
            }
            process(fr, g, [&](int c, float (&rr)[VEC]) {
                if (ok) {
                    load_vec<T, VEC>(rsrc + off + c * hw, rr);
                } else {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) rr[k] = 0.f;
                }
            });
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < C; ++c)
        k3_gather_columns<VEC, F>(Sx + c * FR * SXP, i0, j0, LTH, h_l, w_l, dcoef + (n * C + c) * lw);
}

// (T, VEC, F) combinations of the folded kernels: those of the K3 tile
#define DGF_GREY_DISPATCH(FN, ...)                                                \
    do {                                                                          \
        if constexpr (sizeof(T) == 2) {                                           \
            if (vec == 8 && F == 4) return FN<T, 8, 4>(__VA_ARGS__);              \
            if (vec == 8 && F == 8) return FN<T, 8, 8>(__VA_ARGS__);              \
            if (vec == 4 && F == 4) return FN<T, 4, 4>(__VA_ARGS__);              \
            if (vec == 4 && F == 2) return FN<T, 4, 2>(__VA_ARGS__);              \
        } else {                                                                  \
            if (vec == 4 && F == 4) return FN<T, 4, 4>(__VA_ARGS__);              \
            if (vec == 4 && F == 2) return FN<T, 4, 2>(__VA_ARGS__);              \
            if (vec == 2 && F == 2) return FN<T, 2, 2>(__VA_ARGS__);              \
        }                                                                         \
        return cudaErrorInvalidValue;                                             \
    } while (0)

static bool grey_combo(int esz, int vec, int F) {
    if (esz == 2) return (vec == 8 && (F == 4 || F == 8)) || (vec == 4 && (F == 4 || F == 2));
    return (vec == 4 && (F == 4 || F == 2)) || (vec == 2 && F == 2);
}

constexpr size_t kGreySmemCap = 96 * 1024;  // shared memory a tile aims for (more only for large C)
constexpr size_t kGreySmemMax = 200 * 1024;

static int k2_grey_th(int C, int vec, int F) {
    const size_t row = (size_t)C * (32 * vec / F + 2) * sizeof(float2);
    int th = 32;
    while (th > 1 && th * row > kGreySmemCap) th >>= 1;
    return th;
}
static size_t k3_grey_smem(int C, int vec, int F, int LTH, bool dI) {
    const int SXP = (vec / F == 1 ? 29 : 30 * (vec / F)) + 2;
    return (size_t)C * SXP * (2 * sizeof(float) * F * (LTH + 1) + (dI ? sizeof(float) * F * LTH : 0));
}
static int k3_grey_lth(int C, int vec, int F, bool dI) {
    int lth = F >= 8 ? 8 : 16;
    while (lth > 1 && k3_grey_smem(C, vec, F, lth, dI) > kGreySmemCap) lth >>= 1;
    return lth;
}

int grey_fold_vec(dgf_dtype dt, int F, int C, int w, std::initializer_list<const void*> ptrs) {
    if (F != 2 && F != 4 && F != 8) return 0;
    const int esz = dt == DGF_F32 ? 4 : 2;
    for (int v = 16 / esz; v >= 8 / esz; v >>= 1) {
        if (w % v != 0 || !grey_combo(esz, v, F)) continue;
        bool al = true;
        for (const void* p : ptrs)
            if (p != nullptr && reinterpret_cast<uintptr_t>(p) % (size_t)(v * esz) != 0) al = false;
        if (!al) continue;
        if (k2_grey_th(C, v, F) * (size_t)C * (32 * v / F + 2) * sizeof(float2) > kGreySmemMax) return 0;
        if (k3_grey_smem(C, v, F, 1, true) > kGreySmemMax) return 0;
        return v;
    }
    return 0;
}

template <typename K>
static cudaError_t grey_prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename T, int VEC, int F>
static cudaError_t k2grey_go(const float2* coef, const void* I_h, void* O_h, int N, int C, int n_in, int h_l,
                             int w_l, int h, int w, cudaStream_t s) {
    const int TH = k2_grey_th(C, VEC, F);
    const size_t smem = (size_t)C * TH * (32 * VEC / F + 2) * sizeof(float2);
    auto kern = (n_in == 3 && C == 1) ? k2_grey_apply<T, VEC, F, 3, 1> : k2_grey_apply<T, VEC, F, 0, 0>;
    cudaError_t e = grey_prep(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + 32 * VEC - 1) / (32 * VEC), (h + TH - 1) / TH, N);
    kern<<<grid, kThreads, smem, s>>>(coef, static_cast<const T*>(I_h), static_cast<T*>(O_h), C, n_in, h_l, w_l, h, w,
                                      TH);
    return cudaGetLastError();
}

template <typename T, int VEC, int F>
static cudaError_t k3grey_go(const void* R, const void* I_h, const float2* coef, float2* dcoef, void* dI_h, int N,
                             int C, int n_in, int h_l, int w_l, int h, int w, cudaStream_t s) {
    constexpr int LTW = K3Shape<VEC, F>::LTW;
    const bool dI = dI_h != nullptr;
    const int LTH = k3_grey_lth(C, VEC, F, dI);
    const size_t smem = k3_grey_smem(C, VEC, F, LTH, dI);
    auto kern = (n_in == 3 && C == 1) ? k3_grey_bwd<T, VEC, F, 3, 1> : k3_grey_bwd<T, VEC, F, 0, 0>;
    cudaError_t e = grey_prep(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w_l + LTW - 1) / LTW, (h_l + LTH - 1) / LTH, N);
    kern<<<grid, kThreads, smem, s>>>(static_cast<const T*>(R), static_cast<const T*>(I_h), coef, dcoef,
                                      static_cast<T*>(dI_h), C, n_in, h_l, w_l, h, w, LTH);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t k2grey_d(const float2* coef, const void* I_h, void* O_h, int N, int C, int n_in, int h_l, int w_l,
                            int h, int w, int vec, int F, cudaStream_t s) {
    DGF_GREY_DISPATCH(k2grey_go, coef, I_h, O_h, N, C, n_in, h_l, w_l, h, w, s);
}

template <typename T>
static cudaError_t k3grey_d(const void* R, const void* I_h, const float2* coef, float2* dcoef, void* dI_h, int N,
                            int C, int n_in, int h_l, int w_l, int h, int w, int vec, int F, cudaStream_t s) {
    DGF_GREY_DISPATCH(k3grey_go, R, I_h, coef, dcoef, dI_h, N, C, n_in, h_l, w_l, h, w, s);
}

cudaError_t launch_k2_grey(dgf_dtype dt, const float2* coef, const void* I_h, void* O_h, int N, int C, int n_in,
                           int h_l, int w_l, int h, int w, int F, int vec, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k2grey_d<float>(coef, I_h, O_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
        case DGF_BF16: return k2grey_d<__nv_bfloat16>(coef, I_h, O_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
        case DGF_F16: return k2grey_d<__half>(coef, I_h, O_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_k3_grey(dgf_dtype dt, const void* R, const void* I_h, const float2* coef, float2* dcoef,
                           void* dI_h, int N, int C, int n_in, int h_l, int w_l, int h, int w, int F, int vec,
                           cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k3grey_d<float>(R, I_h, coef, dcoef, dI_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
        case DGF_BF16:
            return k3grey_d<__nv_bfloat16>(R, I_h, coef, dcoef, dI_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
        case DGF_F16: return k3grey_d<__half>(R, I_h, coef, dcoef, dI_h, N, C, n_in, h_l, w_l, h, w, vec, F, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
