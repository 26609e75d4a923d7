// Guidance transform F of Sec. 3.4 (1x1 conv 3 -> hidden, leaky ReLU,
// 1x1 conv hidden -> 3 with bias), fused into the layer's kernels as
// per-pixel register FMAs with the weights in constant memory:
//   K5  G_l = f x f block mean of F(I_h)                      (forward)
//   K2g O_h = Abar_h * F(I_h) + bbar_h, three channels at once (forward)
//   K3g d Abar, d bbar from d O_h and F(I_h)                  (backward)
//   K6  d G_h = d O_h * Abar_h + d G_l / f^2 (block mean transposed), chained
//       through F to d I_h, plus the weight gradients     (backward; Algorithm
//       1's last line, d I_h = d G_h . grad F)
// With F applied to each guide on its own (G_l = F(I_l), the literal reading
// of Sec. 3.4), K5L forms G_l per low-res pixel instead of K5, K6 takes no
// d G_l term, and K6L chains d G_l through F at low resolution to d I_l and
// adds its weight-gradient terms as further partial rows.
// The hidden width is padded to 16 with zero weights, which leaves every
// output unchanged and keeps all loops fully unrolled.
#include <algorithm>

#include "common.cuh"
#include "hires.cuh"
#include "kernels.h"

namespace dgf {

constexpr int kHid = 16;
constexpr int kWGrad = kHid * 3 + 3 * kHid + 3;  // padded [dw1 | dw2 | db2]

__constant__ float c_w1[kHid * 3];  // [k][c]
__constant__ float c_w2[3 * kHid];  // [c][k]
__constant__ float c_b2[3];

__device__ __forceinline__ float lrelu(float z, float slope) { return z > 0.f ? z : slope * z; }

// The weights again as pairs {w, w} (filled from c_w1, c_w2, c_b2 by
// guide_upload), so a paired instruction takes them straight from the
// constant bank.
constexpr int kWPairs = kHid * 3 + 3 * kHid + 3;
__constant__ f32x2 c_wx2[kWPairs];  // [w1 (k, c) | w2 (c, k) | b2]
// ... and as pairs of neighbouring hidden units {w[k], w[k + 1]} (k even),
// so K6 works on two hidden units per paired instruction
constexpr int kHP = kHid / 2;
constexpr int kHidPairs = kHP * 3 + 3 * kHP;
__constant__ f32x2 c_wh[kHidPairs];  // [w1 (k / 2, c) | w2 (c, k / 2)]
__device__ f32x2 g_wx2_stage[kWPairs + kHidPairs];

__global__ void k_splat_weights(const float* __restrict__ w1, const float* __restrict__ w2,
                                const float* __restrict__ b2, int hidden) {
    const int i = threadIdx.x;
    auto W1 = [&](int k, int c) { return k < hidden ? w1[k * 3 + c] : 0.f; };
    auto W2 = [&](int c, int k) { return k < hidden ? w2[c * hidden + k] : 0.f; };
    if (i < kWPairs) {
        float v = 0.f;
        if (i < kHid * 3) {
            const int k = i / 3, c = i - 3 * k;
            v = W1(k, c);
        } else if (i < 2 * kHid * 3) {
            const int c = (i - kHid * 3) / kHid, k = (i - kHid * 3) - c * kHid;
            v = W2(c, k);
        } else {
            v = b2[i - 2 * kHid * 3];
        }
        g_wx2_stage[i] = f2_pack(v, v);
    } else if (i < kWPairs + kHidPairs) {
        const int j = i - kWPairs;
        if (j < kHP * 3) {
            const int q = j / 3, c = j - 3 * q;
            g_wx2_stage[i] = f2_pack(W1(2 * q, c), W1(2 * q + 1, c));
        } else {
            const int c = (j - kHP * 3) / kHP, q = (j - kHP * 3) - c * kHP;
            g_wx2_stage[i] = f2_pack(W2(c, 2 * q), W2(c, 2 * q + 1));
        }
    }
}

// guide_eval for two pixels (a, b) at once; per pixel the same operations in
// the same order as guide_eval.  Used where registers are plentiful (K5):
// in the high-res kernels that hold VEC pixels per thread the register
// pairs it needs cost more occupancy than the saved issue slots gain.
__device__ __forceinline__ void guide_eval2(const float (&xa)[3], const float (&xb)[3], float slope,
                                            float (&ga)[3], float (&gb)[3]) {
    const f32x2 x0 = f2_pack(xa[0], xb[0]), x1 = f2_pack(xa[1], xb[1]), x2 = f2_pack(xa[2], xb[2]);
    const f32x2* w1 = c_wx2;
    const f32x2* w2 = c_wx2 + kHid * 3;
    const f32x2* bb = c_wx2 + 2 * kHid * 3;
    f32x2 g0 = bb[0], g1 = bb[1], g2 = bb[2];
#pragma unroll
    for (int k = 0; k < kHid; ++k) {
        const f32x2 z = f2x_fma(w1[k * 3 + 2], x2, f2x_fma(w1[k * 3 + 1], x1, f2x_mul(w1[k * 3 + 0], x0)));
        float za, zb;
        f2_unpack(z, za, zb);
        const f32x2 hk = f2_pack(lrelu(za, slope), lrelu(zb, slope));
        g0 = f2x_fma(w2[0 * kHid + k], hk, g0);
        g1 = f2x_fma(w2[1 * kHid + k], hk, g1);
        g2 = f2x_fma(w2[2 * kHid + k], hk, g2);
    }
    f2_unpack(g0, ga[0], gb[0]);
    f2_unpack(g1, ga[1], gb[1]);
    f2_unpack(g2, ga[2], gb[2]);
}

__device__ __forceinline__ void guide_eval(const float (&x)[3], float slope, float (&g)[3]) {
    g[0] = c_b2[0];
    g[1] = c_b2[1];
    g[2] = c_b2[2];
#pragma unroll
    for (int k = 0; k < kHid; ++k) {
        const float z = fmaf(c_w1[k * 3 + 2], x[2], fmaf(c_w1[k * 3 + 1], x[1], c_w1[k * 3 + 0] * x[0]));
        const float hk = lrelu(z, slope);
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] = fmaf(c_w2[c * kHid + k], hk, g[c]);
    }
}

// ------------------------------------------------------------------- K5
template <typename T>
__global__ void __launch_bounds__(kThreads) k5_guide_down(const T* __restrict__ I_h, float* __restrict__ G_l,
                                                          int h_l, int w_l, int h, int w, int f,
                                                          float slope) {
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i = blockIdx.y;
    const size_t n = blockIdx.z;
    if (j >= w_l) return;
    const size_t hw = (size_t)h * w;
    const T* base = I_h + n * 3 * hw;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int dy = 0; dy < f; ++dy) {
        const size_t row = (size_t)(f * i + dy) * w + (size_t)f * j;
        int dx = 0;
        for (; dx + 1 < f; dx += 2) {  // two pixels per paired instruction
            float xa[3], xb[3], ga[3], gb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xa[c] = to_f32<T>(base[c * hw + row + dx]);
                xb[c] = to_f32<T>(base[c * hw + row + dx + 1]);
            }
            guide_eval2(xa, xb, slope, ga, gb);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += ga[c] + gb[c];
        }
        for (; dx < f; ++dx) {
            float x[3], g[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = to_f32<T>(base[c * hw + row + dx]);
            guide_eval(x, slope, g);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += g[c];
        }
    }
    const float inv = (float)(f * f);
    const size_t lw = (size_t)h_l * w_l;
#pragma unroll
    for (int c = 0; c < 3; ++c) G_l[(n * 3 + c) * lw + (size_t)i * w_l + j] = acc[c] / inv;
}

// K5 that also keeps F(I_h) (FP32) in G_h, for an even factor FF known at
// compile time: a thread's FF pixels of a row arrive as one vector load per
// channel, are evaluated in pairs and summed in the order of k5_guide_down
// (so G_l has its bits), and each channel's FF values leave as one vector
// store (I_h 16-byte aligned and w = FF w_l keep every vector aligned).
template <typename T, int FF>
__global__ void __launch_bounds__(kThreads) k5_guide_down_keep(const T* __restrict__ I_h, float* __restrict__ G_l,
                                                               int h_l, int w_l, int h, int w, float slope,
                                                               float* __restrict__ G_h) {
    static_assert(FF % 2 == 0, "pixel pairs");
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i = blockIdx.y;
    const size_t n = blockIdx.z;
    if (j >= w_l) return;
    const size_t hw = (size_t)h * w;
    const T* base = I_h + n * 3 * hw;
    float* gbase = G_h + n * 3 * hw;
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int dy = 0; dy < FF; ++dy) {
        const size_t row = (size_t)(FF * i + dy) * w + (size_t)FF * j;
        Vec<T, FF> in[3];  // the row's FF pixels of each channel, one vector load each
#pragma unroll
        for (int c = 0; c < 3; ++c) in[c] = *reinterpret_cast<const Vec<T, FF>*>(base + c * hw + row);
        float gv[3][FF];
#pragma unroll
        for (int dx = 0; dx < FF; dx += 2) {
            float xa[3], xb[3], ga[3], gb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xa[c] = to_f32<T>(in[c].v[dx]);
                xb[c] = to_f32<T>(in[c].v[dx + 1]);
            }
            guide_eval2(xa, xb, slope, ga, gb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[c] += ga[c] + gb[c];
                gv[c][dx] = ga[c];
                gv[c][dx + 1] = gb[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Vec<float, FF> v;
#pragma unroll
            for (int k = 0; k < FF; ++k) v.v[k] = gv[c][k];
            *reinterpret_cast<Vec<float, FF>*>(gbase + c * hw + row) = v;
        }
    }
    const float inv = (float)(FF * FF);
    const size_t lw = (size_t)h_l * w_l;
#pragma unroll
    for (int c = 0; c < 3; ++c) G_l[(n * 3 + c) * lw + (size_t)i * w_l + j] = acc[c] / inv;
}

// ------------------------------------------------------------------ K2g
template <typename T, int VEC, int F>
__global__ void __launch_bounds__(kThreads) k2_apply_guided(const float2* __restrict__ coef,
                                                            const T* __restrict__ I_h, T* __restrict__ O_h,
                                                            int h_l, int w_l, int h, int w, int TH, float slope) {
    extern __shared__ __align__(128) float2 sAB[];
    constexpr int TW = 32 * VEC;
    const int pitch = TW / F + 2;
    const size_t n = blockIdx.z;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    const int Y0 = blockIdx.y * TH, X0 = blockIdx.x * TW;
    const int jlo = X0 / F - 1;
    const int nst = 3 * TH * pitch;
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
        const float2* cp = coef + (n * 3 + ch) * lw;
        const float2 a = cp[(size_t)r0 * w_l + jj], b = cp[(size_t)r1 * w_l + jj];
        sAB[idx] = make_float2(lerp(a.x, b.x, lam), lerp(a.y, b.y, lam));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = X0 + lane * VEC;
    if (xs >= w) return;
    int cc[VEC];
    float ll[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) col_tap<F>(lane * VEC + k, cc[k], ll[k]);
    for (int i = warp; i < TH; i += kWarps) {
        const int y = Y0 + i;
        if (y >= h) break;
        float x[3][VEC];
#pragma unroll
        for (int c = 0; c < 3; ++c) load_vec<T, VEC>(I_h + (n * 3 + c) * hw + (size_t)y * w + xs, x[c]);
        float o[3][VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const float xi[3] = {x[0][k], x[1][k], x[2][k]};
            float g[3];
            guide_eval(xi, slope, g);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2* row = sAB + (c * TH + i) * pitch;
                const float2 s0 = row[cc[k]], s1 = row[cc[k] + 1];
                o[c][k] = fmaf(lerp(s0.x, s1.x, ll[k]), g[c], lerp(s0.y, s1.y, ll[k]));
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) store_vec<T, VEC>(O_h + (n * 3 + c) * hw + (size_t)y * w + xs, o[c]);
    }
}

// ------------------------------------------------------------------ K3g
// GH: G_h = F(I_h) is given in FP32 (the forward's K5 kept it: the same bits
// guide_eval gives) and read instead of evaluating F per pixel.
template <typename T, int VEC, int F, bool GH>
__global__ void __launch_bounds__(kThreads) k3_hires_bwd_guided(const T* __restrict__ R, const T* __restrict__ I_h,
                                                                const float* __restrict__ G_h,
                                                                float2* __restrict__ dcoef, int h_l, int w_l,
                                                                int h, int w, int LTH, float slope) {
    extern __shared__ __align__(128) float smem[];
    using S = K3Shape<VEC, F>;
    constexpr int H0 = S::H0, LTW = S::LTW, SXP = S::SXP;
    const size_t n = blockIdx.z;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    const int i0 = blockIdx.y * LTH, j0 = blockIdx.x * LTW;
    const int FR = F * (LTH + 1);
    const int yf0 = F * (i0 - 1) + H0;
    const int XS = F * j0 - VEC;
    float2* Sx = reinterpret_cast<float2*>(smem);  // [3][FR][SXP]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = XS + lane * VEC;
    const bool col_ok = xs >= 0 && xs < w;
    for (int fr = warp; fr < FR; fr += kWarps) {
        const int y = yf0 + fr;
        const bool ok = col_ok && y >= 0 && y < h;
        float r[3][VEC], x[3][VEC];  // x: I_h, or G_h itself with GH
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                load_vec<T, VEC>(R + (n * 3 + c) * hw + (size_t)y * w + xs, r[c]);
                if constexpr (GH)
                    load_vec<float, VEC>(G_h + (n * 3 + c) * hw + (size_t)y * w + xs, x[c]);
                else
                    load_vec<T, VEC>(I_h + (n * 3 + c) * hw + (size_t)y * w + xs, x[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < VEC; ++k) r[c][k] = x[c][k] = 0.f;
        }
        float u[3][VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            float g[3];
            if constexpr (GH) {
                g[0] = x[0][k];
                g[1] = x[1][k];
                g[2] = x[2][k];
            } else {
                const float xi[3] = {x[0][k], x[1][k], x[2][k]};
                guide_eval(xi, slope, g);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c][k] = ok ? r[c][k] * g[c] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) k3_row_to_smem<VEC, F>(u[c], r[c], lane, Sx + (c * FR + fr) * SXP);
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 3; ++c)
        k3_gather_columns<VEC, F>(Sx + c * FR * SXP, i0, j0, LTH, h_l, w_l, dcoef + (n * 3 + c) * lw);
}

// ------------------------------------------------------------------- K6
// Persistent over high-res tiles (TH rows x 32*VEC columns of one image), one
// CTA per SM (the 99 weight-gradient sums live in registers); each warp
// walks its rows of a tile with the next row's packed inputs already in
// flight.  Each CTA writes one partial row of the sums; a second kernel adds
// the partials in a fixed order.
// LOW: whether d G_l / f^2 joins d G_h (the block-mean form of the low-res
// guide); without it (G_l = F(I_l)) K6L takes d G_l instead.
template <typename T, int VEC, int F, bool LOW>
__global__ void __launch_bounds__(kThreads, 1) k6_guide_bwd(const float2* __restrict__ coef,
                                                           const float* __restrict__ dG_l,
                                                           const T* __restrict__ R, const T* __restrict__ I_h,
                                                           T* __restrict__ dI_h, float* __restrict__ partials,
                                                           int N, int h_l, int w_l, int h, int w, int TH,
                                                           float slope) {
    extern __shared__ __align__(128) float sA[];  // [3][TH][pitch] Abar along y
    __shared__ float red[kWarps][kWGrad];
    constexpr int TW = 32 * VEC;
    const int pitch = TW / F + 2;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    const int tiles_x = (w + TW - 1) / TW, tiles_y = (h + TH - 1) / TH;
    const int total = tiles_x * tiles_y * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float inv_ff = 1.f / (float)(F * F);
    // weight-gradient sums, two hidden units per register pair: gw1[q * 3 + c]
    // holds units (2q, 2q + 1) of input channel c, gw2[c * kHP + q] likewise
    f32x2 gw1[kHP * 3], gw2[3 * kHP];
    float gb2[3];
#pragma unroll
    for (int k = 0; k < kHP * 3; ++k) gw1[k] = gw2[k] = f2_splat(0.f);
    gb2[0] = gb2[1] = gb2[2] = 0.f;
    const f32x2* W1p = c_wh;
    const f32x2* W2p = c_wh + kHP * 3;
    static_assert(VEC % F == 0, "a lane's pixels cover whole low-res cells");
    constexpr int KC = VEC / F;  // low-res cells per lane
    using VT = Vec<T, VEC>;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y);
        const int tl = tile - n * tiles_x * tiles_y;
        const int ty = tl / tiles_x, tx = tl - ty * tiles_x;
        const int Y0 = ty * TH, X0 = tx * TW;
        const int jlo = X0 / F - 1;
        const int nst = 3 * TH * pitch;
        __syncthreads();
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
            const float2* cp = coef + ((size_t)n * 3 + ch) * lw;
            sA[idx] = lerp(cp[(size_t)r0 * w_l + jj].x, cp[(size_t)r1 * w_l + jj].x, lam);
        }
        __syncthreads();
        const int xs = X0 + lane * VEC;
        if (xs >= w) continue;
        // rows of this warp: i = warp, warp + kWarps, ...; each row's packed
        // input vectors are loaded one row ahead
        const T* xb = I_h + (size_t)n * 3 * hw + xs;
        const T* rb = R + (size_t)n * 3 * hw + xs;
        VT xv[3], rv[3];
        if (warp < TH && Y0 + warp < h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv[c] = ldg_vec<T, VEC>(xb + c * hw + (size_t)(Y0 + warp) * w);
                rv[c] = ldg_vec<T, VEC>(rb + c * hw + (size_t)(Y0 + warp) * w);
            }
        }
        for (int i = warp; i < TH; i += kWarps) {
            const int y = Y0 + i;
            if (y >= h) break;
            const int yn = y + kWarps;
            VT xn[3], rn[3];
            if (i + kWarps < TH && yn < h) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xn[c] = ldg_vec<T, VEC>(xb + c * hw + (size_t)yn * w);
                    rn[c] = ldg_vec<T, VEC>(rb + c * hw + (size_t)yn * w);
                }
            }
            const int yl = y / F;
            float dl[3][KC];  // d G_l of the lane's low-res cells on row yl
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int kc = 0; kc < KC; ++kc)
                    dl[c][kc] = LOW ? dG_l[((size_t)n * 3 + c) * lw + (size_t)yl * w_l + xs / F + kc] : 0.f;
            VT ov[3];
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                // bilinear tap along x of pixel lane * VEC + k of the tile
                const int q = k % F, t2 = 2 * q + 1 - F;
                const int c0 = lane * KC + k / F + (t2 >= 0 ? 1 : 0);
                const float lamx = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
                float dg[3], xk[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float* row = sA + (c * TH + i) * pitch;
                    const float A = lerp(row[c0], row[c0 + 1], lamx);
                    xk[c] = to_f32<T>(xv[c].v[k]);
                    dg[c] = fmaf(to_f32<T>(rv[c].v[k]), A, dl[c][k / F] * inv_ff);
                    gb2[c] += dg[c];
                }
                // two hidden units per paired instruction: z, the leaky ReLU
                // factor m (1 or slope: h = z m and d z = d h m), d h = W2^T d G,
                // the two weight-gradient outer products and d I = W1^T d z
                const f32x2 xs0 = f2_splat(xk[0]), xs1 = f2_splat(xk[1]), xs2 = f2_splat(xk[2]);
                const f32x2 d0 = f2_splat(dg[0]), d1 = f2_splat(dg[1]), d2 = f2_splat(dg[2]);
                f32x2 dx0 = f2_splat(0.f), dx1 = f2_splat(0.f), dx2 = f2_splat(0.f);
#pragma unroll
                for (int q2 = 0; q2 < kHP; ++q2) {
                    const f32x2 z = f2x_fma(W1p[q2 * 3 + 2], xs2, f2x_fma(W1p[q2 * 3 + 1], xs1, f2x_mul(W1p[q2 * 3 + 0], xs0)));
                    float za, zb;
                    f2_unpack(z, za, zb);
                    const f32x2 m = f2_pack(za > 0.f ? 1.f : slope, zb > 0.f ? 1.f : slope);
                    const f32x2 hk = f2x_mul(z, m);
                    const f32x2 dh = f2x_fma(W2p[2 * kHP + q2], d2, f2x_fma(W2p[kHP + q2], d1, f2x_mul(W2p[q2], d0)));
                    const f32x2 dz = f2x_mul(dh, m);
                    gw2[0 * kHP + q2] = f2x_fma(d0, hk, gw2[0 * kHP + q2]);
                    gw2[1 * kHP + q2] = f2x_fma(d1, hk, gw2[1 * kHP + q2]);
                    gw2[2 * kHP + q2] = f2x_fma(d2, hk, gw2[2 * kHP + q2]);
                    gw1[q2 * 3 + 0] = f2x_fma(dz, xs0, gw1[q2 * 3 + 0]);
                    gw1[q2 * 3 + 1] = f2x_fma(dz, xs1, gw1[q2 * 3 + 1]);
                    gw1[q2 * 3 + 2] = f2x_fma(dz, xs2, gw1[q2 * 3 + 2]);
                    dx0 = f2x_fma(W1p[q2 * 3 + 0], dz, dx0);
                    dx1 = f2x_fma(W1p[q2 * 3 + 1], dz, dx1);
                    dx2 = f2x_fma(W1p[q2 * 3 + 2], dz, dx2);
                }
                ov[0].v[k] = from_f32<T>(f2_lo(dx0) + f2_hi(dx0));  // even and odd hidden units
                ov[1].v[k] = from_f32<T>(f2_lo(dx1) + f2_hi(dx1));
                ov[2].v[k] = from_f32<T>(f2_lo(dx2) + f2_hi(dx2));
            }
            if (dI_h != nullptr) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<VT*>(dI_h + ((size_t)n * 3 + c) * hw + (size_t)y * w + xs) = ov[c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv[c] = xn[c];
                rv[c] = rn[c];
            }
        }
    }
    // block reduction of the 99 sums (fixed order), one partial row per CTA
#pragma unroll
    for (int k = 0; k < kWGrad; ++k) {
        float v;
        if (k < kHid * 3) {  // w1 (unit kk, channel c)
            const int kk = k / 3, c = k - 3 * kk;
            v = (kk & 1) ? f2_hi(gw1[(kk >> 1) * 3 + c]) : f2_lo(gw1[(kk >> 1) * 3 + c]);
        } else if (k < 2 * kHid * 3) {  // w2 (channel c, unit kk)
            const int c = (k - kHid * 3) / kHid, kk = (k - kHid * 3) - c * kHid;
            v = (kk & 1) ? f2_hi(gw2[c * kHP + (kk >> 1)]) : f2_lo(gw2[c * kHP + (kk >> 1)]);
        } else {
            v = gb2[k - 2 * kHid * 3];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kWGrad; k += kThreads) {
        float s = 0.f;
        for (int wi = 0; wi < kWarps; ++wi) s += red[wi][k];
        partials[(size_t)blockIdx.x * kWGrad + k] = s;
    }
}

// ------------------------------------------------------------------ K5L
// G_l = F(I_l) per low-res pixel (the transform applied to the low-res guide).
template <typename T>
__global__ void __launch_bounds__(kThreads) k5_guide_low(const T* __restrict__ I_l, float* __restrict__ G_l,
                                                         int N, size_t lw, float slope) {
    const size_t total = (size_t)N * lw;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const size_t n = v / lw, px = v - n * lw;
        float x[3], g[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = to_f32<T>(I_l[(n * 3 + c) * lw + px]);
        guide_eval(x, slope, g);
#pragma unroll
        for (int c = 0; c < 3; ++c) G_l[(n * 3 + c) * lw + px] = g[c];
    }
}

// ------------------------------------------------------------------ K6L
// d G_l through F at low resolution: d I_l = W1^T d z and the weight-gradient
// terms of the low-res pixels, one partial row per CTA (rows after K6's).
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k6_guide_low(const float* __restrict__ dG_l,
                                                           const T* __restrict__ I_l, T* __restrict__ dI_l,
                                                           float* __restrict__ partials, int N, size_t lw,
                                                           float slope) {
    __shared__ float red[kWarps][kWGrad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float gw1[kHid * 3], gw2[3 * kHid], gb2[3];
#pragma unroll
    for (int k = 0; k < kHid * 3; ++k) gw1[k] = gw2[k] = 0.f;
    gb2[0] = gb2[1] = gb2[2] = 0.f;
    const size_t total = (size_t)N * lw;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (size_t)gridDim.x * blockDim.x) {
        const size_t n = v / lw, px = v - n * lw;
        float x[3], dg[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = to_f32<T>(I_l[(n * 3 + c) * lw + px]);
            dg[c] = dG_l[(n * 3 + c) * lw + px];
            gb2[c] += dg[c];
        }
        float dx0 = 0.f, dx1 = 0.f, dx2 = 0.f;
#pragma unroll
        for (int kk = 0; kk < kHid; ++kk) {
            const float z = fmaf(c_w1[kk * 3 + 2], x[2], fmaf(c_w1[kk * 3 + 1], x[1], c_w1[kk * 3 + 0] * x[0]));
            const float hk = lrelu(z, slope);
            const float dh = fmaf(c_w2[2 * kHid + kk], dg[2], fmaf(c_w2[1 * kHid + kk], dg[1], c_w2[kk] * dg[0]));
            const float dz = z > 0.f ? dh : slope * dh;
#pragma unroll
            for (int c = 0; c < 3; ++c) gw2[c * kHid + kk] = fmaf(dg[c], hk, gw2[c * kHid + kk]);
            gw1[kk * 3 + 0] = fmaf(dz, x[0], gw1[kk * 3 + 0]);
            gw1[kk * 3 + 1] = fmaf(dz, x[1], gw1[kk * 3 + 1]);
            gw1[kk * 3 + 2] = fmaf(dz, x[2], gw1[kk * 3 + 2]);
            dx0 = fmaf(c_w1[kk * 3 + 0], dz, dx0);
            dx1 = fmaf(c_w1[kk * 3 + 1], dz, dx1);
            dx2 = fmaf(c_w1[kk * 3 + 2], dz, dx2);
        }
        if (dI_l != nullptr) {
            dI_l[(n * 3 + 0) * lw + px] = from_f32<T>(dx0);
            dI_l[(n * 3 + 1) * lw + px] = from_f32<T>(dx1);
            dI_l[(n * 3 + 2) * lw + px] = from_f32<T>(dx2);
        }
    }
    // block reduction of the 99 sums (fixed order), one partial row per CTA
#pragma unroll
    for (int k = 0; k < kWGrad; ++k) {
        float v = k < 48 ? gw1[k] : (k < 96 ? gw2[k - 48] : gb2[k - 96]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kWGrad; k += kThreads) {
        float s = 0.f;
        for (int wi = 0; wi < kWarps; ++wi) s += red[wi][k];
        partials[(size_t)blockIdx.x * kWGrad + k] = s;
    }
}

__global__ void k6_reduce(const float* __restrict__ partials, int nblocks, float* __restrict__ dW,
                          int hidden) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kWGrad) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kWGrad + k];
    // padded [w1 16x3 | w2 3x16 | b2 3] -> caller's [w1 hidden x 3 | w2 3 x hidden | b2 3]
    if (k < kHid * 3) {
        const int kk = k / 3;
        if (kk < hidden) dW[k] = s;
    } else if (k < 2 * kHid * 3) {
        const int c = (k - kHid * 3) / kHid, kk = (k - kHid * 3) % kHid;
        if (kk < hidden) dW[hidden * 3 + c * hidden + kk] = s;
    } else {
        dW[hidden * 6 + (k - 2 * kHid * 3)] = s;
    }
}

// ------------------------------------------------------------------ host
cudaError_t guide_upload(const float* w1, const float* w2, const float* b2, int hidden, cudaStream_t s) {
    static const float zeros[kHid * 3] = {0.f};
    cudaError_t e;
    e = cudaMemcpyToSymbolAsync(c_w1, w1, sizeof(float) * hidden * 3, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (hidden < kHid) {
        e = cudaMemcpyToSymbolAsync(c_w1, zeros, sizeof(float) * (kHid - hidden) * 3,
                                    sizeof(float) * hidden * 3, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    for (int c = 0; c < 3; ++c) {
        e = cudaMemcpyToSymbolAsync(c_w2, w2 + c * hidden, sizeof(float) * hidden, sizeof(float) * c * kHid,
                                    cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        if (hidden < kHid) {
            e = cudaMemcpyToSymbolAsync(c_w2, zeros, sizeof(float) * (kHid - hidden),
                                        sizeof(float) * (c * kHid + hidden), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    e = cudaMemcpyToSymbolAsync(c_b2, b2, sizeof(float) * 3, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_splat_weights<<<1, 160, 0, s>>>(w1, w2, b2, hidden);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    void* stage = nullptr;
    if ((e = cudaGetSymbolAddress(&stage, g_wx2_stage)) != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(c_wx2, stage, sizeof(f32x2) * kWPairs, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_wh, static_cast<f32x2*>(stage) + kWPairs, sizeof(f32x2) * kHidPairs, 0,
                                   cudaMemcpyDeviceToDevice, s);
}

template <typename T>
static cudaError_t k5_go(const void* I_h, float* G_l, int N, int h_l, int w_l, int h, int w, int F,
                         float slope, float* G_h, cudaStream_t s) {
    dim3 grid((w_l + kThreads - 1) / kThreads, h_l, N);
    const T* in = static_cast<const T*>(I_h);
    if (G_h != nullptr && F == 2) k5_guide_down_keep<T, 2><<<grid, kThreads, 0, s>>>(in, G_l, h_l, w_l, h, w, slope, G_h);
    else if (G_h != nullptr && F == 4) k5_guide_down_keep<T, 4><<<grid, kThreads, 0, s>>>(in, G_l, h_l, w_l, h, w, slope, G_h);
    else if (G_h != nullptr && F == 8) k5_guide_down_keep<T, 8><<<grid, kThreads, 0, s>>>(in, G_l, h_l, w_l, h, w, slope, G_h);
    else k5_guide_down<T><<<grid, kThreads, 0, s>>>(in, G_l, h_l, w_l, h, w, F, slope);
    return cudaGetLastError();
}

cudaError_t launch_k5(dgf_dtype dt, const void* I_h, float* G_l, int N, int h_l, int w_l, int h, int w,
                      int F, float slope, cudaStream_t s, float* G_h) {
    if (N == 0) return cudaSuccess;
    // the vector writes of G_h need a factor of 2, 4 or 8 (w = F w_l keeps every
    // thread's FF floats aligned to FF floats)
    if (G_h != nullptr && F != 2 && F != 4 && F != 8) return cudaErrorInvalidValue;
    switch (dt) {
        case DGF_F32: return k5_go<float>(I_h, G_l, N, h_l, w_l, h, w, F, slope, G_h, s);
        case DGF_BF16: return k5_go<__nv_bfloat16>(I_h, G_l, N, h_l, w_l, h, w, F, slope, G_h, s);
        case DGF_F16: return k5_go<__half>(I_h, G_l, N, h_l, w_l, h, w, F, slope, G_h, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t k5l_go(const void* I_l, float* G_l, int N, size_t lw, float slope, cudaStream_t s) {
    const int blocks = (int)std::min<size_t>(((size_t)N * lw + kThreads - 1) / kThreads, (size_t)152 * 8);
    k5_guide_low<T><<<blocks, kThreads, 0, s>>>(static_cast<const T*>(I_l), G_l, N, lw, slope);
    return cudaGetLastError();
}

cudaError_t launch_k5_low(dgf_dtype dt, const void* I_l, float* G_l, int N, int h_l, int w_l, float slope,
                          cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const size_t lw = (size_t)h_l * w_l;
    switch (dt) {
        case DGF_F32: return k5l_go<float>(I_l, G_l, N, lw, slope, s);
        case DGF_BF16: return k5l_go<__nv_bfloat16>(I_l, G_l, N, lw, slope, s);
        case DGF_F16: return k5l_go<__half>(I_l, G_l, N, lw, slope, s);
    }
    return cudaErrorInvalidValue;
}

int k6_low_blocks(int N, int h_l, int w_l) {
    const size_t px = (size_t)N * h_l * w_l;
    return (int)std::max<size_t>(1, std::min<size_t>((px + kThreads - 1) / kThreads, (size_t)152));
}

template <typename T>
static cudaError_t k6l_go(const float* dG_l, const void* I_l, void* dI_l, float* partials, int N, int h_l,
                          int w_l, float slope, cudaStream_t s) {
    k6_guide_low<T><<<k6_low_blocks(N, h_l, w_l), kThreads, 0, s>>>(
        dG_l, static_cast<const T*>(I_l), static_cast<T*>(dI_l), partials, N, (size_t)h_l * w_l, slope);
    return cudaGetLastError();
}

cudaError_t launch_k6_low(dgf_dtype dt, const float* dG_l, const void* I_l, void* dI_l, float* partials, int N,
                          int h_l, int w_l, float slope, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    switch (dt) {
        case DGF_F32: return k6l_go<float>(dG_l, I_l, dI_l, partials, N, h_l, w_l, slope, s);
        case DGF_BF16: return k6l_go<__nv_bfloat16>(dG_l, I_l, dI_l, partials, N, h_l, w_l, slope, s);
        case DGF_F16: return k6l_go<__half>(dG_l, I_l, dI_l, partials, N, h_l, w_l, slope, s);
    }
    return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename T, int VEC, int F>
static cudaError_t k2g_go(const float2* coef, const void* I_h, void* O_h, int N, int h_l, int w_l, int h,
                          int w, int TH, float slope, cudaStream_t s) {
    const size_t smem = (size_t)3 * TH * (32 * VEC / F + 2) * sizeof(float2);
    auto kern = k2_apply_guided<T, VEC, F>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + 32 * VEC - 1) / (32 * VEC), (h + TH - 1) / TH, N);
    kern<<<grid, kThreads, smem, s>>>(coef, static_cast<const T*>(I_h), static_cast<T*>(O_h), h_l, w_l, h, w,
                                      TH, slope);
    return cudaGetLastError();
}

template <typename T, int VEC, int F>
static cudaError_t k3g_go(const void* R, const void* I_h, const float* G_h, float2* dcoef, int N, int h_l, int w_l,
                          int h, int w, int LTH, float slope, cudaStream_t s) {
    constexpr int LTW = K3Shape<VEC, F>::LTW, SXP = K3Shape<VEC, F>::SXP;
    const size_t smem = (size_t)3 * F * (LTH + 1) * SXP * sizeof(float2);
    auto kern = G_h != nullptr ? k3_hires_bwd_guided<T, VEC, F, true> : k3_hires_bwd_guided<T, VEC, F, false>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w_l + LTW - 1) / LTW, (h_l + LTH - 1) / LTH, N);
    kern<<<grid, kThreads, smem, s>>>(static_cast<const T*>(R), static_cast<const T*>(I_h), G_h, dcoef, h_l, w_l,
                                      h, w, LTH, slope);
    return cudaGetLastError();
}

static int g_sms = 0;
static int sm_count() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

int k6_blocks(int N, int h, int w) {
    (void)N; (void)h; (void)w;
    return std::min(sm_count(), kMaxK6Blocks);  // one CTA per SM (its registers allow no second)
}

template <typename T, int VEC, int F>
static cudaError_t k6_go(const float2* coef, const float* dG_l, const void* R, const void* I_h, void* dI_h,
                         float* partials, int N, int h_l, int w_l, int h, int w, float slope, cudaStream_t s) {
    const int TH = 32;
    const size_t smem = (size_t)3 * TH * (32 * VEC / F + 2) * sizeof(float);
    auto kern = dG_l != nullptr ? k6_guide_bwd<T, VEC, F, true> : k6_guide_bwd<T, VEC, F, false>;
    cudaError_t e = prep(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<k6_blocks(N, h, w), kThreads, smem, s>>>(coef, dG_l, static_cast<const T*>(R),
                                                    static_cast<const T*>(I_h), static_cast<T*>(dI_h),
                                                    partials, N, h_l, w_l, h, w, TH, slope);
    return cudaGetLastError();
}

// (vec, F) combinations of the guided kernels: those of the fast K3 tile.
#define DGF_GUIDED_DISPATCH(FN, ...)                                              \
    do {                                                                          \
        if (sizeof(T) == 2) {                                                     \
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

template <typename T>
static cudaError_t k2g_d(const float2* coef, const void* I_h, void* O_h, int N, int h_l, int w_l, int h,
                         int w, int vec, int F, int TH, float slope, cudaStream_t s) {
    DGF_GUIDED_DISPATCH(k2g_go, coef, I_h, O_h, N, h_l, w_l, h, w, TH, slope, s);
}

template <typename T>
static cudaError_t k3g_d(const void* R, const void* I_h, const float* G_h, float2* dcoef, int N, int h_l, int w_l,
                         int h, int w, int vec, int F, int LTH, float slope, cudaStream_t s) {
    DGF_GUIDED_DISPATCH(k3g_go, R, I_h, G_h, dcoef, N, h_l, w_l, h, w, LTH, slope, s);
}

template <typename T>
static cudaError_t k6_d(const float2* coef, const float* dG_l, const void* R, const void* I_h, void* dI_h,
                        float* partials, int N, int h_l, int w_l, int h, int w, int vec, int F,
                        float slope, cudaStream_t s) {
    DGF_GUIDED_DISPATCH(k6_go, coef, dG_l, R, I_h, dI_h, partials, N, h_l, w_l, h, w, slope, s);
}

// 16-byte vectors, else 8-byte vectors (pointers are checked 16-byte aligned)
static int guided_vec(dgf_dtype dt, int w) {
    const int esz = dt == DGF_F32 ? 4 : 2;
    for (int v = 16 / esz; v >= 8 / esz; v >>= 1)
        if (w % v == 0) return v;
    return 1;
}

cudaError_t launch_k2_guided(dgf_dtype dt, const float2* coef, const void* I_h, void* O_h, int N, int h_l,
                             int w_l, int h, int w, int F, int TH, float slope, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int vec = guided_vec(dt, w);
    switch (dt) {
        case DGF_F32: return k2g_d<float>(coef, I_h, O_h, N, h_l, w_l, h, w, vec, F, TH, slope, s);
        case DGF_BF16: return k2g_d<__nv_bfloat16>(coef, I_h, O_h, N, h_l, w_l, h, w, vec, F, TH, slope, s);
        case DGF_F16: return k2g_d<__half>(coef, I_h, O_h, N, h_l, w_l, h, w, vec, F, TH, slope, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_k3_guided(dgf_dtype dt, const void* R, const void* I_h, float2* dcoef, int N, int h_l,
                             int w_l, int h, int w, int F, float slope, cudaStream_t s, const float* G_h) {
    if (N == 0) return cudaSuccess;
    const int vec = guided_vec(dt, w);
    // the FP32 guide's vectors (VEC floats) must be aligned as the loads need
    if (G_h != nullptr && reinterpret_cast<uintptr_t>(G_h) % (vec * sizeof(float)) != 0) return cudaErrorInvalidValue;
    const int LTH = F >= 8 ? 4 : 8;
    switch (dt) {
        case DGF_F32: return k3g_d<float>(R, I_h, G_h, dcoef, N, h_l, w_l, h, w, vec, F, LTH, slope, s);
        case DGF_BF16: return k3g_d<__nv_bfloat16>(R, I_h, G_h, dcoef, N, h_l, w_l, h, w, vec, F, LTH, slope, s);
        case DGF_F16: return k3g_d<__half>(R, I_h, G_h, dcoef, N, h_l, w_l, h, w, vec, F, LTH, slope, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_k6(dgf_dtype dt, const float2* coef, const float* dG_l, const void* R, const void* I_h,
                      void* dI_h, float* partials, int N, int h_l, int w_l, int h, int w, int F, float slope,
                      cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int vec = guided_vec(dt, w);
    switch (dt) {
        case DGF_F32: return k6_d<float>(coef, dG_l, R, I_h, dI_h, partials, N, h_l, w_l, h, w, vec, F, slope, s);
        case DGF_BF16: return k6_d<__nv_bfloat16>(coef, dG_l, R, I_h, dI_h, partials, N, h_l, w_l, h, w, vec, F, slope, s);
        case DGF_F16: return k6_d<__half>(coef, dG_l, R, I_h, dI_h, partials, N, h_l, w_l, h, w, vec, F, slope, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_wreduce(const float* partials, int nblocks, float* dW, int hidden, cudaStream_t s) {
    k6_reduce<<<1, 128, 0, s>>>(partials, nblocks, dW, hidden);
    return cudaGetLastError();
}

bool guided_supported(dgf_dtype dt, int w, int F) {
    const int vec = guided_vec(dt, w);
    if (dt == DGF_F32) return (vec == 4 && (F == 4 || F == 2)) || (vec == 2 && F == 2);
    return (vec == 8 && (F == 4 || F == 8)) || (vec == 4 && (F == 4 || F == 2));
}

}  // namespace dgf
