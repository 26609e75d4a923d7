// Device tile functions of the high-resolution stage (shared by the
// identity-guide kernels and the guidance-transform kernels).
//
// Both stream the high-resolution planes with aligned vector accesses of
// VEC elements (16 or 8 bytes), one warp per row segment of 32*VEC pixels.
// The low-resolution coefficients a tile needs are first interpolated along
// y into shared memory (one row per high-res row, one column per low-res
// column plus a replicated border column on each side, which makes the
// clamp of the bilinear taps free); each pixel then needs one lerp along x.
#pragma once

#include "common.cuh"

namespace dgf {

// ----------------------------------------------------------------- K2 tile
// F > 0: integer factor (w = F w_l, h = F h_l); F = 0: any ratio.
// MODE 0: out = Abar_h * in + bbar_h (O_h);  MODE 1: out = Abar_h * in (d I_h).
template <int F>
__device__ __forceinline__ void col_tap(int pos, int& c, float& lam) {
    // pos = position of the pixel inside the tile (tile origin is a multiple of F)
    const int q = pos % F, j = pos / F;
    const int t2 = 2 * q + 1 - F;
    c = j + (t2 >= 0 ? 1 : 0);  // smem column of the first tap (column 0 = low-res jlo)
    lam = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
}

// TI: type of `in` (the guide in MODE 0, held in FP32 for a grey guide over
// 16-bit data; d O_h in MODE 1); `out` is stored in T.
template <typename T, int VEC, int F, int MODE, typename TI = T>
__device__ void apply_tile(const float2* __restrict__ coef, const TI* __restrict__ in,
                           T* __restrict__ out, int h_l, int w_l, int h, int w, int Y0, int X0, int TH,
                           int pitch, float2* sAB) {
    constexpr int TW = 32 * VEC;
    constexpr int U = 4;  // rows in flight per thread
    constexpr int FF = F > 0 ? F : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xs = X0 + lane * VEC;
    const bool col_ok = xs < w;
    // issue the first rows' loads before staging, so both latencies overlap
    Vec<TI, VEC> raw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int i = warp + u * kWarps, y = Y0 + i;
        if (col_ok && i < TH && y < h) raw[u] = ldg_vec<TI, VEC>(in + (size_t)y * w + xs);
    }
    int jlo;
    int ncol;
    if (F > 0) {
        jlo = X0 / FF - 1;
        ncol = TW / FF + 2;
    } else {
        const int xl = min(X0 + TW, w) - 1;
        jlo = tap_general(X0, w_l, w).i0;
        ncol = tap_general(xl, w_l, w).i0 - jlo + 2;
    }
    // low-res rows the tile's taps reach, clamped to the image
    const int ylast = min(Y0 + TH, h) - 1;
    const Tap tfirst = F > 0 ? tap_int<FF>(Y0) : tap_general(Y0, h_l, h);
    const Tap tlast = F > 0 ? tap_int<FF>(ylast) : tap_general(ylast, h_l, h);
    const int rlo = clampi(tfirst.i0, 0, h_l - 1);
    const int rhi = clampi(tlast.i0 + 1, 0, h_l - 1);
    const int nrows = rhi - rlo + 1;
    float2* sRaw = sAB + TH * pitch;  // nrows x ncol raw coefficients
    // phase 1: every low-res coefficient the tile needs, loaded once (8 loads in flight per thread)
    {
        const int n = nrows * ncol;
        for (int base = threadIdx.x; base < n; base += 8 * kThreads) {
            float2 v[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int idx = base + b * kThreads;
                if (idx < n) {
                    const int rr = idx / ncol, c = idx - rr * ncol;
                    v[b] = coef[(size_t)(rlo + rr) * w_l + clampi(jlo + c, 0, w_l - 1)];
                }
            }
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int idx = base + b * kThreads;
                if (idx < n) sRaw[idx] = v[b];
            }
        }
    }
    __syncthreads();
    // phase 2: interpolate along y, one row per high-res row of the tile
    const int nst = TH * ncol;
    for (int idx = threadIdx.x; idx < nst; idx += kThreads) {
        const int i = idx / ncol, c = idx - i * ncol;
        const int y = Y0 + i;
        if (y >= h) continue;
        const Tap ty = F > 0 ? tap_int<FF>(y) : tap_general(y, h_l, h);
        const int r0 = clampi(ty.i0, 0, h_l - 1) - rlo, r1 = clampi(ty.i0 + 1, 0, h_l - 1) - rlo;
        const float2 a = sRaw[r0 * ncol + c];
        const float2 b = sRaw[r1 * ncol + c];
        sAB[i * pitch + c] = make_float2(lerp(a.x, b.x, ty.lam), lerp(a.y, b.y, ty.lam));
    }
    __syncthreads();
    if (col_ok) {
        // column taps of this lane's VEC pixels (same for every row)
        int cc[VEC];
        float ll[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            if (F > 0) {
                col_tap<FF>(lane * VEC + k, cc[k], ll[k]);
            } else {
                const Tap tx = tap_general(xs + k, w_l, w);
                cc[k] = tx.i0 - jlo;
                ll[k] = tx.lam;
            }
        }
        for (int i0 = warp; i0 < TH; i0 += kWarps * U) {
            if (i0 != warp) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * kWarps, y = Y0 + i;
                    if (i < TH && y < h) raw[u] = ldg_vec<TI, VEC>(in + (size_t)y * w + xs);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * kWarps, y = Y0 + i;
                if (i < TH && y < h) {
                    float g[VEC];
                    unpack_vec<TI, VEC>(raw[u], g);
                    const float2* row = sAB + i * pitch;
                    float o[VEC];
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const float2 s0 = row[cc[k]], s1 = row[cc[k] + 1];
                        const float A = lerp(s0.x, s1.x, ll[k]);
                        if (MODE == 0) {
                            const float B = lerp(s0.y, s1.y, ll[k]);
                            o[k] = fmaf(A, g[k], B);
                        } else {
                            o[k] = A * g[k];
                        }
                    }
                    store_vec<T, VEC>(out + (size_t)y * w + xs, o);
                }
            }
        }
    }
    __syncthreads();
}

// -------------------------------------------------------- K3 tile (integer F)
// The tile owns low-res rows [i0, i0 + LTH) and columns [j0, j0 + LTW) and
// gathers, for each owned (i, j), the transposed bilinear weights of every
// high-res pixel whose taps include it:
//   d Abar(i, j) = sum_y,x wy(y, i) wx(x, j) R(y, x) G(y, x),
//   d bbar(i, j) = sum_y,x wy(y, i) wx(x, j) R(y, x),
// so every output is written once and no atomics are needed.  Pixels whose
// tap falls outside the image (virtual low-res row/column -1 or h_l / w_l)
// fold into the border row/column, as the clamp in the forward does.
// The row sums along x are formed in registers and combined across lanes
// with warp shuffles; the column sums along y read them from shared memory.
template <int VEC, int F>
struct K3Shape {
    static constexpr int K = VEC / F;                     // low-res columns per lane
    static constexpr int H0 = F / 2;                      // first q with a right-hand tap
    static constexpr int LTW = (K == 1) ? 29 : 30 * K;    // owned low-res columns
    static constexpr int SXP = LTW + 2;                   // shared-memory pitch
};

// Row partials of one warp-row: each lane's VEC pixels (values u = R G and
// v = R) weighted onto the K + 2 low-res columns they tap, then combined
// across lanes so that lane l holds the complete row sums of the K columns
// jb(l) .. jb(l) + K - 1 it owns (jb(l) = first tap of its first pixel);
// those land in shared-memory columns (l - 1) K + c.
template <int VEC, int F>
__device__ __forceinline__ void k3_row_to_smem(const float (&u)[VEC], const float (&v)[VEC], int lane,
                                               float2* sx_row) {
    using S = K3Shape<VEC, F>;
    constexpr int K = S::K, SXP = S::SXP, NC = K + 2;
    float pu[NC], pv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) pu[c] = pv[c] = 0.f;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int q = k % F, jr = k / F, t2 = 2 * q + 1 - F;
        const int cl = jr + (t2 >= 0 ? 1 : 0);
        const float lam = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
        pu[cl] = fmaf(1.f - lam, u[k], pu[cl]);
        pv[cl] = fmaf(1.f - lam, v[k], pv[cl]);
        pu[cl + 1] = fmaf(lam, u[k], pu[cl + 1]);
        pv[cl + 1] = fmaf(lam, v[k], pv[cl + 1]);
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float su = pu[c], sv = pv[c];
#pragma unroll
        for (int m = 1; m <= 2; ++m) {
            if (c + m * K <= K + 1) {
                constexpr int dummy = 0;
                (void)dummy;
                const int src = (c + m * K <= K + 1) ? c + m * K : 0;
                const float tu = __shfl_up_sync(0xffffffffu, pu[src], m);
                const float tv = __shfl_up_sync(0xffffffffu, pv[src], m);
                if (lane >= m) {
                    su += tu;
                    sv += tv;
                }
            }
        }
        const int idx = (lane - 1) * K + c;
        if (idx >= 0 && idx < SXP) sx_row[idx] = make_float2(su, sv);
    }
}

// Column pass: for each owned low-res (i, j) sum the row sums of the 2F
// high-res rows whose taps include row i, with their y weights.  Virtual
// taps outside the image fold into the border row/column.
template <int VEC, int F>
__device__ __forceinline__ void k3_gather_columns(const float2* Sx, int i0, int j0, int LTH, int h_l,
                                                  int w_l, float2* __restrict__ dcoef) {
    using S = K3Shape<VEC, F>;
    constexpr int H0 = S::H0, LTW = S::LTW, SXP = S::SXP;
    const int yf0 = F * (i0 - 1) + H0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int li = warp; li < LTH; li += kWarps) {
        const int i = i0 + li;
        if (i >= h_l) break;
        const bool top = (i == 0), bottom = (i == h_l - 1);
        for (int lj = lane; lj < LTW; lj += 32) {
            const int j = j0 + lj;
            if (j >= w_l) break;
            const int c = lj + 1;
            const bool left = (j == 0), right = (j == w_l - 1);
            float su = 0.f, sv = 0.f;
#pragma unroll
            for (int tt = 0; tt < 2 * F; ++tt) {
                // tt < F: rows whose first tap is i; tt >= F: rows whose second tap is i
                const int t = tt % F;
                const int y = (tt < F) ? F * i + H0 + t : F * (i - 1) + H0 + t;
                const int q = (H0 + t) % F;
                const int t2 = 2 * q + 1 - F;
                const float lam = (float)(t2 < 0 ? t2 + 2 * F : t2) / (float)(2 * F);
                float wgt;
                if (tt < F) wgt = bottom ? 1.f : 1.f - lam;
                else wgt = top ? 1.f : lam;
                const float2* row = Sx + (y - yf0) * SXP;
                float2 v = row[c];
                if (left) { v.x += row[0].x; v.y += row[0].y; }
                if (right) { v.x += row[c + 1].x; v.y += row[c + 1].y; }
                su = fmaf(wgt, v.x, su);
                sv = fmaf(wgt, v.y, sv);
            }
            dcoef[(size_t)i * w_l + j] = make_float2(su, sv);
        }
    }
}

}  // namespace dgf
