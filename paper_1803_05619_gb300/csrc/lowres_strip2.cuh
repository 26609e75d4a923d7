// K1 as warp strips with two low-res columns per lane (radius R = 1 or 2).
//
// Same walk as the one-column strips of lowres_strip.cuh (a warp walks down a
// segment of rows; register rings of the last 2R + 1 rows; exactly centred
// statistics), with each lane holding columns xa = x0 + 2 lane and xa + 1.
// A row's horizontal taps for both columns come from the lane itself and R
// shuffles from each neighbouring lane, so the shuffles, loads and loop
// overhead are shared by two outputs, and the halo is R lanes per side
// (2R columns) out of 32: 64 - 4R outputs per strip instead of 32 - 4R.
// Per column the arithmetic is the one-column strip's, term for term.
#pragma once

#include "lowres_strip.cuh"

namespace dgf {

template <int R>
struct Strip2Lane {
    float mk[2][2 * R + 1];  // 1 where column xa + c - R + k is inside the image
    int nx[2];               // clipped window widths of the two columns
    bool xin[2];             // columns inside the image
    bool out[2];             // column written by this lane (lanes [R, 32 - R), inside the image)
};

template <int R>
__device__ __forceinline__ Strip2Lane<R> strip2_lane(int xa, int w) {
    Strip2Lane<R> ln;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int x = xa + c;
        ln.xin[c] = x >= 0 && x < w;
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k) {
            const int xx = x - R + k;
            ln.mk[c][k] = (xx >= 0 && xx < w) ? 1.f : 0.f;
        }
        ln.nx[c] = ln.xin[c] ? min(x + R, w - 1) - max(x - R, 0) + 1 : 1;
        ln.out[c] = lane >= R && lane < 32 - R && ln.xin[c];
    }
    return ln;
}

template <int R>
struct Strip2Ring {
    static constexpr int W = 2 * R + 1;
    float mg[2][W], mp[2][W], sgg[2][W], sgp[2][W], ha[2][W], hb[2][W];
    float vr[W];
};

// The 2R + 2 consecutive values a lane's two windows span, from its own pair
// (v0, v1) and R shuffles from each neighbour: T[c .. c + 2R] are column c's taps.
template <int R>
__device__ __forceinline__ void strip2_taps(float v0, float v1, float (&T)[2 * R + 2]) {
    if constexpr (R == 1) {
        T[0] = shfl_up(v1, 1);
        T[1] = v0;
        T[2] = v1;
        T[3] = shfl_dn(v0, 1);
    } else {
        T[0] = shfl_up(v0, 1);
        T[1] = shfl_up(v1, 1);
        T[2] = v0;
        T[3] = v1;
        T[4] = shfl_dn(v0, 1);
        T[5] = shfl_dn(v1, 1);
    }
}

// K1 for input row e entering ring slot U (both columns).  INT: interior
// ring period.  stats non-null: also write (mu, nu, 1/(var + eps), A) for the
// segment's rows.
template <int R, bool INT>
__device__ __forceinline__ void strip2_k1_row(Strip2Ring<R>& q, const Strip2Lane<R>& ln, int U, float g0, float g1,
                                              float p0, float p1, int e, int e_first, int xa,
                                              float2* __restrict__ coef, float4* __restrict__ stats,
                                              const StripGeom& s, float eps) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW = 1.f / (float)W;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    const int lane = threadIdx.x & 31;
    // ---- level 1: centred statistics of row e over each column's window
    float TG[2 * R + 2], TP[2 * R + 2];
    strip2_taps<R>(g0, g1, TG);
    strip2_taps<R>(p0, p1, TP);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            s1 += TG[c + k];
            s2 += TP[c + k];
        }
        const float inx = INT ? kInvW : inv_count(ln.nx[c]);
        const float m1 = s1 * inx, m2 = s2 * inx;
        float a = 0.f, cc = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float dg = INT ? TG[c + k] - m1 : ln.mk[c][k] * (TG[c + k] - m1);
            a = fmaf(dg, dg, a);
            cc = fmaf(dg, TP[c + k] - m2, cc);
        }
        q.mg[c][U] = m1;
        q.mp[c][U] = m2;
        q.sgg[c][U] = a;
        q.sgp[c][U] = cc;
    }
    q.vr[U] = (INT || (e >= 0 && e < s.h)) ? 1.f : 0.f;
    // ---- Eq. 1's A, b of window row ce = e - R for each column
    const int ce = e - R;
    float A[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
    const int ny = INT ? W : min(ce + R, s.h - 1) - max(ce - R, 0) + 1;
    const bool rows_ok = INT || (ce >= 0 && ce < s.h && e - e_first >= 2 * R);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (INT || (rows_ok && ln.xin[c])) {
            float t1 = 0.f, t2 = 0.f, ta = 0.f, tc = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                t1 += q.mg[c][k];
                t2 += q.mp[c][k];
                ta += q.sgg[c][k];
                tc += q.sgp[c][k];
            }
            const float iny = INT ? kInvW : inv_count(ny);
            const float mu = t1 * iny, nu = t2 * iny;
            float dgg = 0.f, dgp = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const float dg = INT ? q.mg[c][k] - mu : q.vr[k] * (q.mg[c][k] - mu);
                dgg = fmaf(dg, dg, dgg);
                dgp = fmaf(dg, q.mp[c][k] - nu, dgp);
            }
            const float nxf = INT ? (float)W : (float)ln.nx[c];
            const float inn = INT ? kInvW2 : inv_count(ln.nx[c] * ny);
            const float var = fmaf(nxf, dgg, ta) * inn;
            const float cov = fmaf(nxf, dgp, tc) * inn;
            const float ive = rcp_approx(var + eps);
            A[c] = cov * ive;
            b[c] = fmaf(-A[c], mu, nu);
            if (stats != nullptr && ln.out[c] && ce >= s.y0 && ce < s.y0 + s.seg)
                stats[(size_t)ce * s.w + xa + c] = make_float4(mu, nu, ive, A[c]);
            if (!s.mean && ln.out[c] && ce >= s.y0 && ce < s.y0 + s.seg)
                coef[(size_t)ce * s.w + xa + c] = make_float2(A[c], b[c]);  // no box mean: A_l, b_l
        }
    }
    if (!s.mean) return;
    // ---- level 2: horizontal box sums of A, b per column; vertical sum over the ring
    {
        float TA[2 * R + 2], TB[2 * R + 2];
        strip2_taps<R>(A[0], A[1], TA);
        strip2_taps<R>(b[0], b[1], TB);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                sa += TA[c + k];
                sb += TB[c + k];
            }
            q.ha[c][U] = sa;
            q.hb[c][U] = sb;
        }
    }
    const int co = ce - R;  // output row; level 2 holds window rows co - R .. co + R
    const bool row_out = INT || (co >= s.y0 && co < s.y0 + s.seg && co < s.h && e - e_first >= 4 * R);
    if (row_out) {
        const int nyo = INT ? W : min(co + R, s.h - 1) - max(co - R, 0) + 1;
        float2 o[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                sa += q.ha[c][k];
                sb += q.hb[c][k];
            }
            const float inn = INT ? kInvW2 : inv_count(ln.nx[c] * nyo);
            o[c] = make_float2(sa * inn, sb * inn);
        }
        float2* dst = coef + (size_t)co * s.w + xa;
        const bool w0 = INT ? (lane >= R && lane < 32 - R) : ln.out[0];
        const bool w1 = INT ? (lane >= R && lane < 32 - R) : ln.out[1];
        if (w0) dst[0] = o[0];
        if (w1) dst[1] = o[1];
    }
}

template <typename TG, typename TP, int R>
__device__ __forceinline__ void strip2_ring_init(Strip2Ring<R>& q) {
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) {
        q.vr[k] = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) q.mg[c][k] = q.mp[c][k] = q.sgg[c][k] = q.sgp[c][k] = q.ha[c][k] = q.hb[c][k] = 0.f;
    }
}

// Strip geometry: x0 = strip (64 - 4R) - 2R, lane columns xa = x0 + 2 lane.
__host__ __device__ constexpr int strip2_out_cols(int R) { return 64 - 4 * R; }

// K1 for one strip segment, rows loaded one ring period ahead.
template <typename TG, typename TP, int R>
__device__ void coef_strip2(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                            const StripGeom& s, float eps, float4* __restrict__ stats = nullptr) {
    constexpr int W = 2 * R + 1;
    const int xa = s.x0 + 2 * (int)(threadIdx.x & 31);
    const Strip2Lane<R> ln = strip2_lane<R>(xa, s.w);
    const bool cols_int = s.x0 >= 0 && s.x0 + 64 <= s.w;
    Strip2Ring<R> q;
    strip2_ring_init<TG, TP, R>(q);
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, s.h) + 2 * R;
    float gn[2][W], pn[2][W];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            const bool row = e >= 0 && e < s.h && e < e_last;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const bool ok = row && ln.xin[c];
                gn[c][u] = ok ? to_f32<TG>(G[(size_t)e * s.w + xa + c]) : 0.f;
                pn[c][u] = ok ? to_f32<TP>(P[(size_t)e * s.w + xa + c]) : 0.f;
            }
        }
    };
    load(e_first);
    for (int base = e_first; base < e_last; base += W) {
        float gv[2][W], pv[2][W];
#pragma unroll
        for (int u = 0; u < W; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                gv[c][u] = gn[c][u];
                pv[c][u] = pn[c][u];
            }
        if (base + W < e_last) load(base + W);  // next period in flight while this one computes
        const bool row_int = cols_int && base >= 3 * R && base - e_first >= 4 * R && base + W <= s.h &&
                             base + W <= e_last;
        if (row_int) {
#pragma unroll
            for (int u = 0; u < W; ++u)
                strip2_k1_row<R, true>(q, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], base + u, e_first, xa, coef,
                                       stats, s, eps);
        } else {
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (base + u >= e_last) break;  // uniform across the warp
                strip2_k1_row<R, false>(q, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], base + u, e_first, xa,
                                        coef, stats, s, eps);
            }
        }
    }
}

// Same walk with TMA staging: boxes of (64 + U) columns x RB rows, the
// strip's first column rounded down to the 16-byte unit U.
__host__ __device__ constexpr int strip2_box_cols(int esize) { return 64 + 16 / esize; }
__host__ __device__ constexpr int strip2_box_bytes(int esize, int rows) {
    return align128i(rows * strip2_box_cols(esize) * esize);
}

template <typename TG, typename TP, int R>
__device__ void coef_strip2_tma(const TmaPair* maps, int plane, float2* __restrict__ coef, float4* __restrict__ stats,
                                const StripGeom& s, float eps, unsigned char* ring, uint64_t* bars, uint32_t* status) {
    constexpr int W = 2 * R + 1, RB = StripTmaCfg<R>::RB, NS = StripTmaCfg<R>::NS, NP = RB / W;
    constexpr int UG = 16 / (int)sizeof(TG), UP = 16 / (int)sizeof(TP);
    constexpr int BXG = strip2_box_cols((int)sizeof(TG)), BXP = strip2_box_cols((int)sizeof(TP));
    constexpr int BG = strip2_box_bytes((int)sizeof(TG), RB), BP = strip2_box_bytes((int)sizeof(TP), RB);
    constexpr int SLOT = BG + BP;
    constexpr uint32_t TX = (uint32_t)(RB * BXG * (int)sizeof(TG) + RB * BXP * (int)sizeof(TP));
    const int lane = threadIdx.x & 31;
    const int xa = s.x0 + 2 * lane;
    const Strip2Lane<R> ln = strip2_lane<R>(xa, s.w);
    const bool cols_int = s.x0 >= 0 && s.x0 + 64 <= s.w;
    Strip2Ring<R> q;
    strip2_ring_init<TG, TP, R>(q);
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, s.h) + 2 * R;
    const int nblk = (e_last - e_first + RB - 1) / RB;
    const int xg = floor_to(s.x0, UG), xp = floor_to(s.x0, UP);
    const int og = s.x0 - xg + 2 * lane, op = s.x0 - xp + 2 * lane;
    const uint32_t ring_s = smem_u32(ring), bar_s = smem_u32(bars);
    auto issue = [&](int m) {  // lane 0: block m into slot m % NS
        const int slot = m % NS;
        const uint32_t bar = bar_s + 8u * slot, dst = ring_s + (uint32_t)(slot * SLOT);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(TX) : "memory");
        tma_load_3d(dst, &maps->a.map, xg, e_first + m * RB, plane, bar);
        tma_load_3d(dst + BG, &maps->b.map, xp, e_first + m * RB, plane, bar);
    };
    if (lane == 0) {
        for (int k = 0; k < NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * k) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int m = 0; m < min(NS, nblk); ++m) issue(m);
    }
    __syncwarp();
    int m = 0;
    bool ok = true;
    for (; m < nblk; ++m) {
        const int slot = m % NS;
        if (!__all_sync(0xffffffffu, mbar_wait(bar_s + 8u * slot, (uint32_t)((m / NS) & 1), kWaitLimit))) {
            ok = false;
            break;
        }
        const TG* sg = reinterpret_cast<const TG*>(ring + slot * SLOT) + og;
        const TP* sp = reinterpret_cast<const TP*>(ring + slot * SLOT + BG) + op;
#pragma unroll 1  // one copy of the period's code (ring slots are fixed within a period)
        for (int pp = 0; pp < NP; ++pp) {
            const int base = e_first + m * RB + pp * W;
            float gv[2][W], pv[2][W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const int o_g = (pp * W + u) * BXG, o_p = (pp * W + u) * BXP;
                // columns outside the image read as zero (the box's fill) and are masked like the plain loads
                gv[0][u] = ln.xin[0] ? to_f32<TG>(sg[o_g]) : 0.f;
                gv[1][u] = ln.xin[1] ? to_f32<TG>(sg[o_g + 1]) : 0.f;
                pv[0][u] = ln.xin[0] ? to_f32<TP>(sp[o_p]) : 0.f;
                pv[1][u] = ln.xin[1] ? to_f32<TP>(sp[o_p + 1]) : 0.f;
            }
            if (pp == NP - 1) {
                __syncwarp();  // every lane has read the slot
                if (lane == 0 && m + NS < nblk) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(m + NS);
                }
            }
            if (base >= e_last) continue;  // uniform
            const bool row_int = cols_int && base >= 3 * R && base - e_first >= 4 * R && base + W <= s.h &&
                                 base + W <= e_last;
            if (row_int) {
#pragma unroll
                for (int u = 0; u < W; ++u)
                    strip2_k1_row<R, true>(q, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], base + u, e_first, xa,
                                           coef, stats, s, eps);
            } else {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    if (base + u >= e_last) break;  // uniform across the warp
                    strip2_k1_row<R, false>(q, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], base + u, e_first,
                                            xa, coef, stats, s, eps);
                }
            }
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        for (int qb = m; qb < nblk && qb < m + NS; ++qb)
            mbar_wait(bar_s + 8u * (qb % NS), (uint32_t)((qb / NS) & 1), kWaitLimit);
    }
}

// shared memory of one CTA of two-column K1 strips staged by TMA
template <typename TG, typename TP, int R>
__host__ __device__ constexpr int k1_strip2_tma_smem() {
    return kStripWarps * StripTmaCfg<R>::NS *
               (strip2_box_bytes((int)sizeof(TG), StripTmaCfg<R>::RB) +
                strip2_box_bytes((int)sizeof(TP), StripTmaCfg<R>::RB)) +
           kStripWarps * StripTmaCfg<R>::NS * 8;
}

}  // namespace dgf
