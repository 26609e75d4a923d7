// Low-resolution stage as warp-strip column walks (radius R = 1 or 2).
//
// One warp owns a strip of 32 consecutive low-res columns and walks down a
// segment of rows.  Each lane holds one column: horizontal window terms come
// from the neighbouring lanes by warp shuffles, vertical window terms from a
// register ring of the last 2R + 1 rows (the walk is unrolled by 2R + 1 so
// every ring slot is a fixed register).  No shared memory, no barriers: the
// row loads of a whole ring period are issued before that period is
// processed.  Lanes [2R, 32 - 2R) produce outputs; the 2R lanes on each side
// are the strip's halo (neighbouring strips overlap by 4R columns), and the
// first 4R rows of a segment only fill the rings.
//
// Statistics are exactly centred as in the tile kernels: each row segment is
// centred on its own mean and rows are combined with Chan's update.
#pragma once

#include "common.cuh"

namespace dgf {

constexpr int kStripWarps = 8;  // warps per CTA (independent strips)

__device__ __forceinline__ float shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_dn(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

// Sum of v over lanes l - R .. l + R (values of lanes outside the warp are
// don't-care: only lanes [R, 32 - R) use the result).
template <int R>
__device__ __forceinline__ float hsum(float v) {
    float s = v;
#pragma unroll
    for (int d = 1; d <= R; ++d) s += shfl_up(v, d) + shfl_dn(v, d);
    return s;
}

struct StripGeom {
    int h, w;
    int x0;       // global column of lane 0 (first input column, may be negative)
    int y0;       // first output row of the segment
    int seg;      // output rows of the segment
};

// ------------------------------------------------------------------- K1
// Eq. 1's least-squares A, b per clipped window, then their box mean, for
// one strip segment.  Writes Abar, bbar for lanes [2R, 32 - 2R).
template <typename TG, typename TP, int R>
__device__ void coef_strip(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                           const StripGeom& s, float eps) {
    constexpr int W = 2 * R + 1;
    const int lane = threadIdx.x & 31;
    const int x = s.x0 + lane;
    const bool xin = x >= 0 && x < s.w;
    // column facts of this lane's window (same for every row)
    float mk[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const int xx = x - R + k;
        mk[k] = (xx >= 0 && xx < s.w) ? 1.f : 0.f;
    }
    const float nx = xin ? (float)(min(x + R, s.w - 1) - max(x - R, 0) + 1) : 1.f;
    const float inx = __frcp_rn(nx);
    const bool out_lane = lane >= 2 * R && lane < 32 - 2 * R && xin;
    // level-1 ring: row statistics of input rows; level-2 ring: horizontal box sums of A, b
    float mg[W], mp[W], sgg[W], sgp[W], vr[W], ha[W], hb[W];
#pragma unroll
    for (int k = 0; k < W; ++k) mg[k] = mp[k] = sgg[k] = sgp[k] = vr[k] = ha[k] = hb[k] = 0.f;
    // input row e enters ring 1 in slot (e - e_first) % W; the window of row
    // c = e - R is then complete, and its A, b enter ring 2 in slot (c - c_first) % W;
    // the output row c - R is complete after that.
    const int e_first = s.y0 - 2 * R;
    const int e_last = s.y0 + s.seg + 2 * R;  // exclusive
    for (int base = e_first; base < e_last; base += W) {
        float gv[W], pv[W];
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            const bool ok = xin && e >= 0 && e < s.h && e < e_last;
            gv[u] = ok ? to_f32<TG>(G[(size_t)e * s.w + x]) : 0.f;
            pv[u] = ok ? to_f32<TP>(P[(size_t)e * s.w + x]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            if (e >= e_last) break;  // uniform across the warp
            // ---- level 1: row statistics of input row e at this lane's column
            float g[W], p[W];
            g[R] = gv[u];
            p[R] = pv[u];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                g[R - d] = shfl_up(gv[u], d);
                g[R + d] = shfl_dn(gv[u], d);
                p[R - d] = shfl_up(pv[u], d);
                p[R + d] = shfl_dn(pv[u], d);
            }
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                s1 += g[k];
                s2 += p[k];
            }
            const float m1 = s1 * inx, m2 = s2 * inx;
            float a = 0.f, c = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const float dg = mk[k] * (g[k] - m1);
                a = fmaf(dg, dg, a);
                c = fmaf(dg, p[k] - m2, c);
            }
            mg[u] = m1;
            mp[u] = m2;
            sgg[u] = a;
            sgp[u] = c;
            vr[u] = (e >= 0 && e < s.h) ? 1.f : 0.f;
            // ---- window of row ce = e - R (rows ce - R .. ce + R = ring 1)
            const int ce = e - R;
            float A = 0.f, b = 0.f;
            if (xin && ce >= 0 && ce < s.h && e - e_first >= 2 * R) {
                const float ny = (float)(min(ce + R, s.h - 1) - max(ce - R, 0) + 1);
                float t1 = 0.f, t2 = 0.f, ta = 0.f, tc = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    t1 += mg[k];
                    t2 += mp[k];
                    ta += sgg[k];
                    tc += sgp[k];
                }
                const float iny = __frcp_rn(ny);
                const float mu = t1 * iny, nu = t2 * iny;
                float dgg = 0.f, dgp = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const float dg = vr[k] * (mg[k] - mu);
                    dgg = fmaf(dg, dg, dgg);
                    dgp = fmaf(dg, mp[k] - nu, dgp);
                }
                const float inn = __frcp_rn(nx * ny);
                const float var = fmaf(nx, dgg, ta) * inn;
                const float cov = fmaf(nx, dgp, tc) * inn;
                A = cov * __frcp_rn(var + eps);
                b = fmaf(-A, mu, nu);
            }
            // ---- level 2: horizontal box sums of A, b; ring 2 over rows ce
            ha[u] = hsum<R>(A);
            hb[u] = hsum<R>(b);
            const int co = ce - R;  // output row, complete once ring 2 holds rows co - R .. co + R
            if (out_lane && co >= s.y0 && co < s.y0 + s.seg && co < s.h && e - e_first >= 4 * R) {
                float sa = 0.f, sb = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    sa += ha[k];
                    sb += hb[k];
                }
                const float n = nx * (float)(min(co + R, s.h - 1) - max(co - R, 0) + 1);
                const float inn = __frcp_rn(n);
                coef[(size_t)co * s.w + x] = make_float2(sa * inn, sb * inn);
            }
        }
    }
}

}  // namespace dgf
