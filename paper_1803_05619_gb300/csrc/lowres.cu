// Low-resolution kernels: K1 (statistics -> A, b -> Abar, bbar) and K4
// (recompute + Algorithm 1's low-resolution gradients).
#include <algorithm>

#include "batch.cuh"
#include "kernels.h"
#include "lowres_fast.cuh"
#include "lowres_generic.cuh"
#include "lowres_strip.cuh"
#include "lowres_strip2.cuh"
#include "lowres_slide.cuh"

namespace dgf {

bool slide_radius(int r) { return r == 1 || r == 2 || r == 4 || r == 8; }
int slide_k1_v(int) { return 4; }
int slide_k4_v(int) { return 4; }
bool slide_v_built(int r, int V, bool) {
    if (V == 2 || V == 8) return r <= 2;
    return V == 4;
}
int slide_auto_seg(int h, int r) { return h <= 128 ? std::max(8, 2 * r) : std::max(16, 4 * r); }
int slide_out_cols(int r, int V) {
    const int hb = V * ((2 * r + V - 1) / V);
    return 32 * V - 2 * hb;
}
// per-warp bytes and warps per CTA of the sliding K1 for 16-bit G and P
// (the batched kernel's types), taken from the device code's own constants
template <int R, int V>
static size_t k1_slide_warp16() {
    return (size_t)k1_slide_warp_bytes<__nv_bfloat16, __nv_bfloat16, R, V>();
}
template <int R, int V>
static int k1_slide_wpc16() {
    return slide_wpc<k1_slide_warp_bytes<__nv_bfloat16, __nv_bfloat16, R, V>()>();
}
#define DGF_SLIDE_K1_SHAPES(X) X(1, 2) X(2, 2) X(1, 4) X(2, 4) X(4, 4) X(8, 4) X(1, 8) X(2, 8)
size_t k1_slide_smem_bytes(int r, int V, int warps) {
    size_t b = 0;
#define DGF_X(RR, VV) \
    if (r == RR && V == VV) b = k1_slide_warp16<RR, VV>();
    DGF_SLIDE_K1_SHAPES(DGF_X)
#undef DGF_X
    return b * (size_t)warps;
}
int k1_slide_batched_wpc(int r, int V) {
#define DGF_X(RR, VV) \
    if (r == RR && V == VV) return k1_slide_wpc16<RR, VV>();
    DGF_SLIDE_K1_SHAPES(DGF_X)
#undef DGF_X
    return kWarps;
}
#undef DGF_SLIDE_K1_SHAPES

static cudaError_t launch_k1_slide(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes,
                                   int h, int w, int r, float eps, const LowCfg& c, cudaStream_t s) {
    const int S = c.a > 0 ? c.a : slide_auto_seg(h, r);
    const int V = c.b > 0 ? c.b : slide_k1_v(r);
    switch (r) {
        case 1: return launch_k1_slide_r<1>(dt, gf32, G, P, coef, planes, h, w, eps, S, V, s);
        case 2: return launch_k1_slide_r<2>(dt, gf32, G, P, coef, planes, h, w, eps, S, V, s);
        case 4: return launch_k1_slide_r<4>(dt, gf32, G, P, coef, planes, h, w, eps, S, V, s);
        case 8: return launch_k1_slide_r<8>(dt, gf32, G, P, coef, planes, h, w, eps, S, V, s);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t launch_k4_slide(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef,
                                   void* dP, void* dG, int planes, int h, int w, int r, float eps, const LowCfg& c,
                                   cudaStream_t s) {
    const int S = c.a > 0 ? c.a : slide_auto_seg(h, r);
    const int V = c.b > 0 ? c.b : slide_k4_v(r);
    switch (r) {
        case 1: return launch_k4_slide_r<1>(dt, gf32, G, P, dcoef, dP, dG, planes, h, w, eps, S, V, s);
        case 2: return launch_k4_slide_r<2>(dt, gf32, G, P, dcoef, dP, dG, planes, h, w, eps, S, V, s);
        case 4: return launch_k4_slide_r<4>(dt, gf32, G, P, dcoef, dP, dG, planes, h, w, eps, S, V, s);
        case 8: return launch_k4_slide_r<8>(dt, gf32, G, P, dcoef, dP, dG, planes, h, w, eps, S, V, s);
    }
    return cudaErrorInvalidValue;
}

template <typename TG, typename TP>
__global__ void __launch_bounds__(kThreads) k1_coef(const TG* __restrict__ G, const TP* __restrict__ P,
                                                    float2* __restrict__ coef, int h, int w, int r,
                                                    float eps, int TY, int TX,
                                                    const __grid_constant__ TmaPair tma,
                                                    uint32_t* status, int mean) {
    extern __shared__ __align__(128) float smem[];
    LowresTile t;
    t.init(h, w, r, eps, blockIdx.y * TY, blockIdx.x * TX, TY, TX);
    t.mean = mean;
    const size_t plane = blockIdx.z;
    const size_t hw = (size_t)h * w;
    coef_tile<TG, TP>(G + plane * hw, P + plane * hw, coef + plane * hw, t, smem,
                      tma.enabled ? &tma.a : nullptr, tma.enabled ? &tma.b : nullptr, (int)plane,
                      status);
}

// ---------------------------------------------------------------------- K4
// Algorithm 1 at low resolution.  With d Abar, d bbar from the high-res
// pass: dA = f_mu^T(d Abar), db = f_mu^T(d bbar); per window m
//   alpha = dA - db mu, gamma = alpha / (var + eps)   (d Sigma_GO),
//   beta = -gamma A                                   (d Sigma_G);
// then, summing over the windows m that contain pixel i, in centred form,
//   dP_i = sum [gamma (G_i - mu) + db] / N_m,
//   dG_i = sum [gamma (P_i - nu) + 2 beta (G_i - mu) - db A] / N_m,
// which equals Algorithm 1's d O_l and d G_l (the uncentred terms
// -d Sigma_GO Gbar etc. regroup into the differences).  Every sum is a
// separable window pass; G and P are shifted by the tile mean first.
template <typename TG, typename TP, typename TD>
__device__ void lowres_bwd_tile(const TG* __restrict__ G, const TP* __restrict__ P,
                                const float2* __restrict__ dcoef, TP* __restrict__ dP,
                                TD* __restrict__ dG, const LowresTile& t, float* smem) {
    const int n2 = t.EY2 * t.EX2, n1 = t.EY1 * t.EX1;
    const int nh = max(4 * t.EY2 * t.EX1, 7 * t.EY1 * t.TX);
    float* sG = smem;
    float* sP = sG + n2;
    float* sDA = sP + n2;
    float* sDB = sDA + n2;
    float* hbuf = sDB + n2;
    float* e1 = hbuf + nh;  // mu, nu, var+eps, A, dA, db on E1
    float* q = e1 + 6 * n1;  // the seven quantities whose window sums form dP, dG
    float* red = q + 7 * n1;

    stage_plane<TG>(G, sG, t);
    stage_plane<TP>(P, sP, t);
    for (int idx = threadIdx.x; idx < n2; idx += kThreads) {
        const int ey = idx / t.EX2, ex = idx - ey * t.EX2;
        const int gy = t.ty0 - 2 * t.r + ey, gx = t.tx0 - 2 * t.r + ex;
        float a = 0.f, b = 0.f;
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const float2 c = dcoef[(size_t)gy * t.w + gx];
            const float n = (float)(t.cnt(gy, t.h) * t.cnt(gx, t.w));
            a = c.x / n;
            b = c.y / n;
        }
        sDA[idx] = a;
        sDB[idx] = b;
    }
    __syncthreads();
    // tile shift K = mean of the in-image output pixels (conditioning only)
    {
        float sg = 0.f, sp = 0.f, c = 0.f;
        for (int idx = threadIdx.x; idx < t.TY * t.TX; idx += kThreads) {
            const int y = idx / t.TX, x = idx - y * t.TX;
            if (t.ty0 + y < t.h && t.tx0 + x < t.w) {
                const int o = (y + 2 * t.r) * t.EX2 + x + 2 * t.r;
                sg += sG[o];
                sp += sP[o];
                c += 1.f;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sg += __shfl_down_sync(0xffffffffu, sg, off);
            sp += __shfl_down_sync(0xffffffffu, sp, off);
            c += __shfl_down_sync(0xffffffffu, c, off);
        }
        if ((threadIdx.x & 31) == 0) {
            red[(threadIdx.x >> 5) * 3 + 0] = sg;
            red[(threadIdx.x >> 5) * 3 + 1] = sp;
            red[(threadIdx.x >> 5) * 3 + 2] = c;
        }
    }
    const int nhr = t.EY2 * t.EX1;
    stats_rows(sG, sP, hbuf, hbuf + nhr, hbuf + 2 * nhr, hbuf + 3 * nhr, t);
    __syncthreads();
    float KG = 0.f, KP = 0.f;
    {
        float sg = 0.f, sp = 0.f, c = 0.f;
        for (int k = 0; k < kWarps; ++k) {
            sg += red[k * 3 + 0];
            sp += red[k * 3 + 1];
            c += red[k * 3 + 2];
        }
        if (c > 0.f) {
            KG = sg / c;
            KP = sp / c;
        }
    }
    float* eMU = e1;
    float* eNU = e1 + n1;
    float* eVE = e1 + 2 * n1;
    float* eA = e1 + 3 * n1;
    float* eDA = e1 + 4 * n1;
    float* eDB = e1 + 5 * n1;
    for (int idx = threadIdx.x; idx < n1; idx += kThreads) {
        const int ey1 = idx / t.EX1, ex = idx - ey1 * t.EX1;
        const int gy = t.ty0 - t.r + ey1, gx = t.tx0 - t.r + ex;
        float mu = 0.f, nu = 0.f, ve = 1.f, A = 0.f;
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const Moments m = stats_window(hbuf, hbuf + nhr, hbuf + 2 * nhr, hbuf + 3 * nhr, ey1, ex, t);
            mu = m.mu;
            nu = m.nu;
            ve = m.var + t.eps;
            A = m.cov / ve;
        }
        eMU[idx] = mu; eNU[idx] = nu; eVE[idx] = ve; eA[idx] = A;
    }
    __syncthreads();
    // dA = f_mu^T(d Abar), db = f_mu^T(d bbar) on E1: window sums of (d/N)
    box_rows(sDA, t.EX2, t.EY2, t.tx0 - 2 * t.r, hbuf, t.EX1, t.tx0 - t.r, t.EX1, t.w, t.r);
    box_rows(sDB, t.EX2, t.EY2, t.tx0 - 2 * t.r, hbuf + nhr, t.EX1, t.tx0 - t.r, t.EX1, t.w, t.r);
    __syncthreads();
    for (int idx = threadIdx.x; idx < n1; idx += kThreads) {
        const int ey1 = idx / t.EX1, ex = idx - ey1 * t.EX1;
        const int gy = t.ty0 - t.r + ey1, gx = t.tx0 - t.r + ex;
        float da = 0.f, db = 0.f;
        if (!t.mean && gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            // no box mean of A, b: dA, db are d Abar, d bbar themselves
            const float2 c = dcoef[(size_t)gy * t.w + gx];
            da = c.x;
            db = c.y;
        } else if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const int lo = max(gy - t.r, 0), hi = min(gy + t.r, t.h - 1);
            for (int k = lo; k <= hi; ++k) {
                const int o = (k - (t.ty0 - 2 * t.r)) * t.EX1 + ex;
                da += hbuf[o];
                db += hbuf[nhr + o];
            }
        }
        eDA[idx] = da;
        eDB[idx] = db;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n1; idx += kThreads) {
        const int ey1 = idx / t.EX1, ex = idx - ey1 * t.EX1;
        const int gy = t.ty0 - t.r + ey1, gx = t.tx0 - t.r + ex;
        float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const float n = (float)(t.cnt(gy, t.h) * t.cnt(gx, t.w));
            const float db = eDB[idx], A = eA[idx];
            const float mus = eMU[idx] - KG, nus = eNU[idx] - KP;
            const float alpha = fmaf(-db, eMU[idx], eDA[idx]);
            const float gamma = alpha / eVE[idx];
            const float beta = -gamma * A;
            v[0] = gamma / n;
            v[1] = gamma * mus / n;
            v[2] = gamma * nus / n;
            v[3] = beta / n;
            v[4] = beta * mus / n;
            v[5] = db / n;
            v[6] = db * A / n;
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) q[k * n1 + idx] = v[k];
    }
    __syncthreads();
    const int nq = t.EY1 * t.TX;
#pragma unroll 1
    for (int k = 0; k < 7; ++k)
        box_rows(q + k * n1, t.EX1, t.EY1, t.tx0 - t.r, hbuf + k * nq, t.TX, t.tx0, t.TX, t.w, t.r);
    __syncthreads();
    const int n0 = t.TY * t.TX;
    for (int idx = threadIdx.x; idx < n0; idx += kThreads) {
        const int y = idx / t.TX, x = idx - y * t.TX;
        const int gy = t.ty0 + y, gx = t.tx0 + x;
        if (gy >= t.h || gx >= t.w) continue;
        const int lo = max(gy - t.r, 0), hi = min(gy + t.r, t.h - 1);
        float S[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = lo; k <= hi; ++k) {
            const int o = (k - (t.ty0 - t.r)) * t.TX + x;
#pragma unroll
            for (int m = 0; m < 7; ++m) S[m] += hbuf[m * nq + o];
        }
        const int o2 = (y + 2 * t.r) * t.EX2 + x + 2 * t.r;
        const float g = sG[o2] - KG, p = sP[o2] - KP;
        const size_t go = (size_t)gy * t.w + gx;
        if (dP != nullptr) dP[go] = from_f32<TP>(fmaf(g, S[0], S[5] - S[1]));
        if (dG != nullptr) {
            const float v = fmaf(p, S[0], -S[2]) + 2.f * fmaf(g, S[3], -S[4]) - S[6];
            dG[go] = from_f32<TD>(v);
        }
    }
    __syncthreads();
}

template <typename TG, typename TP, typename TD>
__global__ void __launch_bounds__(kThreads) k4_lowres_bwd(const TG* __restrict__ G, const TP* __restrict__ P,
                                                          const float2* __restrict__ dcoef,
                                                          TP* __restrict__ dP, TD* __restrict__ dG,
                                                          int h, int w, int r, float eps, int TY, int TX,
                                                          int mean) {
    extern __shared__ __align__(128) float smem[];
    LowresTile t;
    t.init(h, w, r, eps, blockIdx.y * TY, blockIdx.x * TX, TY, TX);
    t.mean = mean;
    const size_t plane = blockIdx.z;
    const size_t hw = (size_t)h * w;
    lowres_bwd_tile<TG, TP, TD>(G + plane * hw, P + plane * hw, dcoef + plane * hw,
                                dP ? dP + plane * hw : nullptr, dG ? dG + plane * hw : nullptr, t,
                                smem);
}

// ------------------------------------------------------------------ host side
size_t k1_smem_bytes(int r, int TY, int TX) {
    const size_t EY2 = TY + 4 * r, EX2 = TX + 4 * r, EX1 = TX + 2 * r;
    size_t floats = 2 * EY2 * EX2 + 4 * EY2 * EX1;
    // TMA staging lands inside the row-statistics region, plus alignment slack
    return floats * sizeof(float) + tma_extra_bytes(r, TY, TX);
}

size_t k4_smem_bytes(int r, int TY, int TX) {
    const size_t EY2 = TY + 4 * r, EX2 = TX + 4 * r, EY1 = TY + 2 * r, EX1 = TX + 2 * r;
    const size_t n2 = EY2 * EX2, n1 = EY1 * EX1;
    const size_t nh = std::max(4 * EY2 * EX1, 7 * EY1 * (size_t)TX);
    return (4 * n2 + nh + 13 * n1 + 3 * kWarps) * sizeof(float);
}

bool low_fast_radius(int r) { return r == 1 || r == 2 || r == 4 || r == 8; }

size_t k1_fast_smem_bytes(int r, int CW, int EY1, size_t tma_landing) {
    const size_t e2 = (size_t)(CW + 2 * r) * (EY1 + 2 * r), e1 = (size_t)CW * EY1;
    size_t floats = 2 * e2 + 2 * e1;
    if (r > 2) floats += (size_t)4 * (EY1 + 2 * r) * CW;  // row statistics of the staged walk
    const size_t base = floats * sizeof(float);
    // the TMA landing buffers overlap sA, sB (and what follows) and may extend past them
    const size_t land_end = 2 * e2 * sizeof(float) + tma_landing;
    return std::max(base, land_end);
}

size_t k4_fast_smem_bytes(int r, int CW, int EY1) {
    const size_t e2 = (size_t)(CW + 2 * r) * (EY1 + 2 * r), e1 = (size_t)CW * EY1;
    size_t floats = 4 * e2 + (r == 1 ? kNQD : kNQ) * e1 + 3 * (kLowThreads / 32);
    if (r > 2) floats += 8 + std::max((size_t)6 * (EY1 + 2 * r) * CW, (size_t)kNQ * e1);
    return floats * sizeof(float);
}

size_t k1_cfg_smem(const LowCfg& c, int r, size_t tma_landing) {
    if (c.fast == 3) {  // batched: the single call's warps per CTA
        const int V = c.b > 0 ? c.b : slide_k1_v(r);
        return k1_slide_smem_bytes(r, V, k1_slide_batched_wpc(r, V));
    }
    if (c.fast == 2) return 0;  // warp strips keep everything in registers
    return c.fast ? k1_fast_smem_bytes(r, c.a, c.b, tma_landing) : k1_smem_bytes(r, c.a, c.b);
}

size_t k4_cfg_smem(const LowCfg& c, int r) {
    if (c.fast == 2 || c.fast == 3) return 0;  // strips (the sliding form sizes its own ring at launch)
    return c.fast ? k4_fast_smem_bytes(r, c.a, c.b) : k4_smem_bytes(r, c.a, c.b);
}

void low_grid(const LowCfg& c, int r, int h, int w, int& gx, int& gy) {
    if (c.fast == 3) {
        // batched work items: one strip segment per warp of a CTA (the single
        // call's warps per CTA)
        const int V = c.b > 0 ? c.b : slide_k1_v(r), S = c.a > 0 ? c.a : slide_auto_seg(h, r);
        const int nstrip = (w + slide_out_cols(r, V) - 1) / slide_out_cols(r, V), nseg = (h + S - 1) / S;
        const int wpc = k1_slide_batched_wpc(r, V);
        gx = (nstrip * nseg + wpc - 1) / wpc;
        gy = 1;
        return;
    }
    if (c.fast == 2) {
        // work items of 8 warp strips (one CTA) per plane, in one row
        const int nstrip = (w + strip2_out_cols(r) - 1) / strip2_out_cols(r), nseg = (h + c.a - 1) / c.a;
        gx = (nstrip * nseg + kWarps - 1) / kWarps;  // batched work items: one strip segment per warp of a CTA
        gy = 1;
        return;
    }
    if (c.fast) {
        const int TX = c.a - 2 * r, TY = c.b - 2 * r;
        gx = (w + TX - 1) / TX;
        gy = (h + TY - 1) / TY;
    } else {
        gx = (w + c.b - 1) / c.b;
        gy = (h + c.a - 1) / c.a;
    }
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename TG, typename TP>
static cudaError_t k1_go(const void* G, const void* P, float2* coef, int planes, int h, int w, int r,
                         float eps, const LowCfg& c, const TmaPair& tma, size_t smem, uint32_t* status,
                         cudaStream_t s) {
    auto kern = k1_coef<TG, TP>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    int gx, gy;
    low_grid(c, r, h, w, gx, gy);
    kern<<<dim3(gx, gy, planes), kThreads, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P), coef,
                                                      h, w, r, eps, c.a, c.b, tma, status, c.mean);
    return cudaGetLastError();
}

cudaError_t launch_k1(dgf_dtype dt, bool guide_f32, const void* G, const void* P, float2* coef, int planes,
                      int h, int w, int r, float eps, const LowCfg& c, const TmaPair& tma, size_t smem,
                      uint32_t* status, float4* stats, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    if (c.fast == 3) return launch_k1_slide(dt, guide_f32, G, P, coef, planes, h, w, r, eps, c, s);
    if (c.fast) {
        switch (r) {
            case 1: return launch_k1_fast<1>(dt, guide_f32, G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
            case 2: return launch_k1_fast<2>(dt, guide_f32, G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
            case 4: return launch_k1_fast<4>(dt, guide_f32, G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
            case 8: return launch_k1_fast<8>(dt, guide_f32, G, P, coef, planes, h, w, eps, c, tma, smem, status, stats, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (dt) {
        case DGF_F32:
            return k1_go<float, float>(G, P, coef, planes, h, w, r, eps, c, tma, smem, status, s);
        case DGF_BF16:
            return guide_f32 ? k1_go<float, __nv_bfloat16>(G, P, coef, planes, h, w, r, eps, c, tma, smem, status, s)
                             : k1_go<__nv_bfloat16, __nv_bfloat16>(G, P, coef, planes, h, w, r, eps, c, tma, smem, status, s);
        case DGF_F16:
            return guide_f32 ? k1_go<float, __half>(G, P, coef, planes, h, w, r, eps, c, tma, smem, status, s)
                             : k1_go<__half, __half>(G, P, coef, planes, h, w, r, eps, c, tma, smem, status, s);
    }
    return cudaErrorInvalidValue;
}

template <typename TG, typename TP, typename TD>
static cudaError_t k4_go(const void* G, const void* P, const float2* dcoef, void* dP, void* dG,
                         int planes, int h, int w, int r, float eps, const LowCfg& c, cudaStream_t s) {
    const size_t smem = k4_smem_bytes(r, c.a, c.b);
    auto kern = k4_lowres_bwd<TG, TP, TD>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    int gx, gy;
    low_grid(c, r, h, w, gx, gy);
    kern<<<dim3(gx, gy, planes), kThreads, smem, s>>>(static_cast<const TG*>(G), static_cast<const TP*>(P), dcoef,
                                                      static_cast<TP*>(dP), static_cast<TD*>(dG), h, w, r, eps,
                                                      c.a, c.b, c.mean);
    return cudaGetLastError();
}

cudaError_t launch_k4(dgf_dtype dt, bool guide_f32, const void* G, const void* P, const float2* dcoef,
                      void* dP, void* dG, int planes, int h, int w, int r, float eps, const LowCfg& c,
                      const TmaTriple* tma, uint32_t* status, const float4* stats, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    if (c.fast == 3) return launch_k4_slide(dt, guide_f32, G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s);
    if (c.fast) {
        switch (r) {
            case 1: return launch_k4_fast<1>(dt, guide_f32, G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
            case 2: return launch_k4_fast<2>(dt, guide_f32, G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
            case 4: return launch_k4_fast<4>(dt, guide_f32, G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
            case 8: return launch_k4_fast<8>(dt, guide_f32, G, P, dcoef, dP, dG, planes, h, w, eps, c, tma, status, stats, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (dt) {
        case DGF_F32:
            return k4_go<float, float, float>(G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s);
        case DGF_BF16:
            return guide_f32
                       ? k4_go<float, __nv_bfloat16, float>(G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s)
                       : k4_go<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16>(G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s);
        case DGF_F16:
            return guide_f32
                       ? k4_go<float, __half, float>(G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s)
                       : k4_go<__half, __half, __half>(G, P, dcoef, dP, dG, planes, h, w, r, eps, c, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t k1_batched_kernel_t(int r, int mode, size_t smem, void** fn, int V, int* threads);

cudaError_t k1_batched_kernel(dgf_dtype dt, int r, int mode, size_t smem, void** fn, int V, int* threads) {
    switch (dt) {
        case DGF_F32: return k1_batched_kernel_t<float>(r, mode, smem, fn, V, threads);
        case DGF_BF16: return k1_batched_kernel_t<__nv_bfloat16>(r, mode, smem, fn, V, threads);
        case DGF_F16: return k1_batched_kernel_t<__half>(r, mode, smem, fn, V, threads);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
