// K1, and K4 from saved window statistics, as warp strips with two low-res
// columns per lane (radius R = 1 or 2).
//
// Same walk as the one-column strips of lowres_strip.cuh (a warp walks down a
// segment of rows; register rings of the last 2R + 1 rows; exactly centred
// statistics), with each lane holding columns xa = x0 + 2 lane and xa + 1.
// A row's horizontal taps for both columns come from the lane itself and R
// shuffles from each neighbouring lane, so the shuffles, loads and loop
// overhead are shared by two outputs, and the halo is R lanes per side
// (2R columns) out of 32: 64 - 4R outputs per strip instead of 32 - 4R.
// The two columns run in lock step as the halves of f32x2 register pairs
// (common.cuh): per column the arithmetic is the one-column walk's, term for
// term, through non-contracting round-to-nearest intrinsics, so a column's
// bits do not depend on the strip or segment that computed it.
#pragma once

#include <type_traits>

#include "lowres_strip.cuh"

namespace dgf {

template <int R>
struct Strip2Lane {
    f32x2 mk[2 * R + 1];  // per tap k: 1 where column xa + c - R + k is inside the image (halves c = 0, 1)
    f32x2 nx, inx;        // clipped window widths of the two columns, and their reciprocals
    f32x2 xin2;           // 1 for the columns inside the image
    int nx_i[2];          // the widths as integers (count-table index)
    bool xin[2];          // columns inside the image
    bool out[2];          // column written by this lane (lanes [R, 32 - R), inside the image)
};

template <int R>
__device__ __forceinline__ Strip2Lane<R> strip2_lane(int xa, int w) {
    Strip2Lane<R> ln;
    const int lane = threadIdx.x & 31;
    float mk[2][2 * R + 1];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int x = xa + c;
        ln.xin[c] = x >= 0 && x < w;
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k) {
            const int xx = x - R + k;
            mk[c][k] = (xx >= 0 && xx < w) ? 1.f : 0.f;
        }
        ln.nx_i[c] = ln.xin[c] ? min(x + R, w - 1) - max(x - R, 0) + 1 : 1;
        ln.out[c] = lane >= R && lane < 32 - R && ln.xin[c];
    }
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) ln.mk[k] = f2_pack(mk[0][k], mk[1][k]);
    ln.nx = f2_pack((float)ln.nx_i[0], (float)ln.nx_i[1]);
    ln.inx = f2_pack(inv_count(ln.nx_i[0]), inv_count(ln.nx_i[1]));
    ln.xin2 = f2_pack(ln.xin[0] ? 1.f : 0.f, ln.xin[1] ? 1.f : 0.f);
    return ln;
}

// Register rings of the last 2R + 1 rows, one pair {column xa, column xa + 1}
// per entry; vr holds {v, v} with v = 1 for rows inside the image.
template <int R>
struct Strip2Ring {
    static constexpr int W = 2 * R + 1;
    f32x2 mg[W], mp[W], sgg[W], sgp[W], ha[W], hb[W], vr[W];
};

// The lane's 2R + 1 tap pairs of one row: Q[k] = {T[k], T[k + 1]} where
// T[0 .. 2R + 1] are the 2R + 2 consecutive values its two windows span
// (its own pair (v0, v1) and R shuffles from each neighbouring lane), so
// Q[k] holds tap k of column xa and of column xa + 1.
template <int R>
__device__ __forceinline__ void strip2_pairs(float v0, float v1, f32x2 (&Q)[2 * R + 1]) {
    if constexpr (R == 1) {
        const float l1 = shfl_up(v1, 1), r0 = shfl_dn(v0, 1);
        Q[0] = f2_pack(l1, v0);
        Q[1] = f2_pack(v0, v1);
        Q[2] = f2_pack(v1, r0);
    } else {
        const float l0 = shfl_up(v0, 1), l1 = shfl_up(v1, 1), r0 = shfl_dn(v0, 1), r1 = shfl_dn(v1, 1);
        Q[0] = f2_pack(l0, l1);
        Q[1] = f2_pack(l1, v0);
        Q[2] = f2_pack(v0, v1);
        Q[3] = f2_pack(v1, r0);
        Q[4] = f2_pack(r0, r1);
    }
}

// K1 for input row e entering ring slot U, both columns at once in paired
// FP32 (each half is the one-column arithmetic), in two stages:
//   stage A: level 1 of row e, then Eq. 1's A, b of window row e - R;
//   stage B: level 2 (box sums of A, b) and the output row e - 2R.
// INT: interior ring period.  stats non-null: stage A also writes
// (mu, nu, 1/(var + eps), A) for the segment's rows.
// Where stage A puts a window's statistics when the caller owns them (the
// fused backward); the default writes the segment's rows to `stats`.
struct NoStatsOut {
    __device__ __forceinline__ void put(int, int, float4) const {}
};

template <int R, bool INT, class SOut = NoStatsOut>
__device__ __forceinline__ void strip2_k1_stage_a(Strip2Ring<R>& q, const Strip2Lane<R>& ln, int U, float g0,
                                                  float g1, float p0, float p1, int e, int e_first, int xa,
                                                  float2* __restrict__ coef, float4* __restrict__ stats,
                                                  const StripGeom& s, f32x2 eps2, f32x2& A_out, f32x2& b_out,
                                                  const SOut* sout = nullptr) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW = 1.f / (float)W;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    // ---- level 1: centred statistics of row e over each column's window
    {
        f32x2 QG[W], QP[W];
        strip2_pairs<R>(g0, g1, QG);
        strip2_pairs<R>(p0, p1, QP);
        f32x2 s1 = QG[0], s2 = QP[0];
#pragma unroll
        for (int k = 1; k < W; ++k) {
            s1 = f2_add(s1, QG[k]);
            s2 = f2_add(s2, QP[k]);
        }
        const f32x2 inx = INT ? f2_splat(kInvW) : ln.inx;
        const f32x2 m1 = f2_mul(s1, inx), m2 = f2_mul(s2, inx);
        f32x2 a = 0ull, cc = 0ull;  // +0.0 in both halves
#pragma unroll
        for (int k = 0; k < W; ++k) {
            f32x2 dg = f2_sub(QG[k], m1);
            if (!INT) dg = f2_mul(ln.mk[k], dg);
            a = f2_fma(dg, dg, a);
            cc = f2_fma(dg, f2_sub(QP[k], m2), cc);
        }
        q.mg[U] = m1;
        q.mp[U] = m2;
        q.sgg[U] = a;
        q.sgp[U] = cc;
        q.vr[U] = (INT || (e >= 0 && e < s.h)) ? f2_splat(1.f) : 0ull;
    }
    // ---- Eq. 1's A, b of window row ce = e - R for both columns
    const int ce = e - R;
    f32x2 A2 = 0ull, b2 = 0ull;
    const int ny = INT ? W : min(ce + R, s.h - 1) - max(ce - R, 0) + 1;
    const bool rows_ok = INT || (ce >= 0 && ce < s.h && e - e_first >= 2 * R);
    if (rows_ok) {
        // ring slots in row order, oldest first (slot (U + 1) mod W): the
        // summation order, and so every bit of the result, does not depend on
        // where the segment starts
        const int k0 = ring_slot<W>(U, 0);
        f32x2 t1 = q.mg[k0], t2 = q.mp[k0], ta = q.sgg[k0], tc = q.sgp[k0];
#pragma unroll
        for (int j = 1; j < W; ++j) {
            const int k = ring_slot<W>(U, j);
            t1 = f2_add(t1, q.mg[k]);
            t2 = f2_add(t2, q.mp[k]);
            ta = f2_add(ta, q.sgg[k]);
            tc = f2_add(tc, q.sgp[k]);
        }
        const f32x2 iny = f2_splat(INT ? kInvW : inv_count(ny));
        const f32x2 mu = f2_mul(t1, iny), nu = f2_mul(t2, iny);
        f32x2 dgg = 0ull, dgp = 0ull;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = ring_slot<W>(U, j);
            f32x2 dg = f2_sub(q.mg[k], mu);
            if (!INT) dg = f2_mul(q.vr[k], dg);
            dgg = f2_fma(dg, dg, dgg);
            dgp = f2_fma(dg, f2_sub(q.mp[k], nu), dgp);
        }
        const f32x2 nxf = INT ? f2_splat((float)W) : ln.nx;
        const f32x2 inn = INT ? f2_splat(kInvW2)
                              : f2_pack(inv_count(ln.nx_i[0] * ny), inv_count(ln.nx_i[1] * ny));
        const f32x2 var = f2_mul(f2_fma(nxf, dgg, ta), inn);
        const f32x2 cov = f2_mul(f2_fma(nxf, dgp, tc), inn);
        float v0, v1;
        f2_unpack(f2_add(var, eps2), v0, v1);
        const f32x2 ive = f2_pack(rcp_approx(v0), rcp_approx(v1));
        A2 = f2_mul(cov, ive);
        // b = nu - A mu, as fma(-A, mu, nu)
        b2 = f2_fma(A2 ^ 0x8000000080000000ull, mu, nu);
        if (!INT) {  // columns outside the image hold A = b = 0
            A2 = f2_mul(A2, ln.xin2);
            b2 = f2_mul(b2, ln.xin2);
        }
        const bool seg_row = ce >= s.y0 && ce < s.y0 + s.seg;
        if (sout != nullptr) {
            float mu0, mu1, nu0, nu1, i0, i1, a0, a1;
            f2_unpack(mu, mu0, mu1);
            f2_unpack(nu, nu0, nu1);
            f2_unpack(ive, i0, i1);
            f2_unpack(A2, a0, a1);
            if (ln.out[0]) sout->put(ce, xa, make_float4(mu0, nu0, i0, a0));
            if (ln.out[1]) sout->put(ce, xa + 1, make_float4(mu1, nu1, i1, a1));
        } else if (stats != nullptr && seg_row) {
            float mu0, mu1, nu0, nu1, i0, i1, a0, a1;
            f2_unpack(mu, mu0, mu1);
            f2_unpack(nu, nu0, nu1);
            f2_unpack(ive, i0, i1);
            f2_unpack(A2, a0, a1);
            if (ln.out[0]) stats[(size_t)ce * s.w + xa] = make_float4(mu0, nu0, i0, a0);
            if (ln.out[1]) stats[(size_t)ce * s.w + xa + 1] = make_float4(mu1, nu1, i1, a1);
        }
        if (!s.mean && seg_row) {  // no box mean: A_l, b_l are the coefficients
            float a0, a1, bb0, bb1;
            f2_unpack(A2, a0, a1);
            f2_unpack(b2, bb0, bb1);
            if (ln.out[0]) coef[(size_t)ce * s.w + xa] = make_float2(a0, bb0);
            if (ln.out[1]) coef[(size_t)ce * s.w + xa + 1] = make_float2(a1, bb1);
        }
    }
    A_out = A2;
    b_out = b2;
}

// Where stage B puts (Abar, bbar) of output row co, column x: the plane's
// coefficient array (row pitch w).
struct CoefOut {
    float2* __restrict__ coef;
    int w;
    __device__ __forceinline__ void put(int co, int x, float2 v) const { coef[(size_t)co * w + x] = v; }
};

// Stage B for input row e (ring slot U): A2, b2 are stage A's result for it.
template <int R, bool INT, class Out = CoefOut>
__device__ __forceinline__ void strip2_k1_stage_b(Strip2Ring<R>& q, const Strip2Lane<R>& ln, int U, int e,
                                                  int e_first, int xa, const Out& dst, const StripGeom& s,
                                                  f32x2 A2, f32x2 b2) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    const int lane = threadIdx.x & 31;
    if (!s.mean) return;
    const int ce = e - R;
    // ---- level 2: horizontal box sums of A, b per column; vertical sum over the ring
    {
        float a0, a1, bb0, bb1;
        f2_unpack(A2, a0, a1);
        f2_unpack(b2, bb0, bb1);
        f32x2 QA[W], QB[W];
        strip2_pairs<R>(a0, a1, QA);
        strip2_pairs<R>(bb0, bb1, QB);
        f32x2 sa = QA[0], sb = QB[0];
#pragma unroll
        for (int k = 1; k < W; ++k) {
            sa = f2_add(sa, QA[k]);
            sb = f2_add(sb, QB[k]);
        }
        q.ha[U] = sa;
        q.hb[U] = sb;
    }
    const int co = ce - R;  // output row; level 2 holds window rows co - R .. co + R
    // (interior periods include the segment's first periods, whose rows only fill the rings)
    const bool row_out = INT ? e - e_first >= 4 * R
                             : (co >= s.y0 && co < s.y0 + s.seg && co < s.h && e - e_first >= 4 * R);
    if (row_out) {
        const int nyo = INT ? W : min(co + R, s.h - 1) - max(co - R, 0) + 1;
        f32x2 sa = q.ha[ring_slot<W>(U, 0)], sb = q.hb[ring_slot<W>(U, 0)];
#pragma unroll
        for (int j = 1; j < W; ++j) {  // row order, as in stage A
            sa = f2_add(sa, q.ha[ring_slot<W>(U, j)]);
            sb = f2_add(sb, q.hb[ring_slot<W>(U, j)]);
        }
        const f32x2 inn = INT ? f2_splat(kInvW2)
                              : f2_pack(inv_count(ln.nx_i[0] * nyo), inv_count(ln.nx_i[1] * nyo));
        float oa0, oa1, ob0, ob1;
        f2_unpack(f2_mul(sa, inn), oa0, oa1);
        f2_unpack(f2_mul(sb, inn), ob0, ob1);
        const bool w0 = INT ? (lane >= R && lane < 32 - R) : ln.out[0];
        const bool w1 = INT ? (lane >= R && lane < 32 - R) : ln.out[1];
        if (w0) dst.put(co, xa, make_float2(oa0, ob0));
        if (w1) dst.put(co, xa + 1, make_float2(oa1, ob1));
    }
}

template <typename TG, typename TP, int R>
__device__ __forceinline__ void strip2_ring_init(Strip2Ring<R>& q) {
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) q.vr[k] = q.mg[k] = q.mp[k] = q.sgg[k] = q.sgp[k] = q.ha[k] = q.hb[k] = 0ull;
}

// Strip geometry: x0 = strip (64 - 4R) - 2R, lane columns xa = x0 + 2 lane.
__host__ __device__ constexpr int strip2_out_cols(int R) { return 64 - 4 * R; }

// One ring period of the walk (rows base .. base + W - 1 with values gv, pv).
// Stage B's results go to `out` when given (the fused forward's shared-memory
// rows), else to the plane's coefficient array.
template <int R, bool INT, class Out = CoefOut, class SOut = NoStatsOut>
__device__ __forceinline__ void strip2_k1_period(Strip2Ring<R>& q, const Strip2Lane<R>& ln,
                                                 const float (&gv)[2][2 * R + 1], const float (&pv)[2][2 * R + 1],
                                                 int base, int e_first, int e_last, int xa, float2* __restrict__ coef,
                                                 float4* __restrict__ stats, const StripGeom& s, f32x2 eps2,
                                                 const Out* out = nullptr, const SOut* sout = nullptr) {
    constexpr int W = 2 * R + 1;
#pragma unroll
    for (int u = 0; u < W; ++u) {
        const int e = base + u;
        if (!INT && e >= e_last) break;  // uniform across the warp
        f32x2 A, b;
        strip2_k1_stage_a<R, INT, SOut>(q, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], e, e_first, xa, coef,
                                        stats, s, eps2, A, b, sout);
        if constexpr (std::is_same<Out, CoefOut>::value)
            strip2_k1_stage_b<R, INT>(q, ln, u, e, e_first, xa, CoefOut{coef, s.w}, s, A, b);
        else
            strip2_k1_stage_b<R, INT>(q, ln, u, e, e_first, xa, *out, s, A, b);
    }
}

// K1 for one strip segment, rows loaded one ring period ahead.
template <typename TG, typename TP, int R>
__device__ void coef_strip2(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                            const StripGeom& s, float eps, float4* __restrict__ stats = nullptr) {
    constexpr int W = 2 * R + 1;
    const f32x2 eps2 = f2_splat(eps);
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
        const bool row_int = cols_int && base >= 3 * R && base + W <= s.h && base + W <= e_last;
        if (row_int)
            strip2_k1_period<R, true>(q, ln, gv, pv, base, e_first, e_last, xa, coef, stats, s, eps2);
        else
            strip2_k1_period<R, false>(q, ln, gv, pv, base, e_first, e_last, xa, coef, stats, s, eps2);
    }
}

// ------------------------------------------------------------------- K4
// K4 from the window statistics the backward K1 pass saved, two columns per
// lane in paired FP32 (the strip geometry of the two-column K1: 64 - 4R
// outputs per strip, R lanes of halo per side for the two horizontal box
// levels).  Per window m (row ce, columns xa, xa + 1): dA = f_mu^T(d Abar),
// db = f_mu^T(d bbar) as box sums of d Abar / N, d bbar / N, then
//   gamma = (dA - db mu) / (var + eps),  beta = -gamma A,
// and four quantities whose box sums over the windows containing a pixel give
//   dP = G' S0 + S2,   dG = P' S0 + 2 G' S1 - S3
// (S0 = sum gamma / N, S1 = sum beta / N, S2 = sum (db - gamma mu') / N,
// S3 = sum (gamma nu' + 2 beta mu' + db A) / N; primes are shifts by the
// strip's constant, the mean of the segment's first output row).
template <int R>
struct Strip2BwdRing {
    static constexpr int W = 2 * R + 1;
    f32x2 hda[W], hdb[W];                  // row box sums of d Abar / N, d bbar / N (input rows)
    f32x2 hq0[W], hq1[W], hq2[W], hq3[W];  // row box sums of the four window quantities (window rows)
    f32x2 rg[W], rp[W];                    // raw G, P of the input rows
};

__device__ __forceinline__ f32x2 f2_neg(f32x2 v) { return v ^ 0x8000000080000000ull; }

// Row box sum of the pair (v0, v1)'s horizontal windows.
template <int R>
__device__ __forceinline__ f32x2 strip2_hsum(float v0, float v1) {
    constexpr int W = 2 * R + 1;
    f32x2 Q[W];
    strip2_pairs<R>(v0, v1, Q);
    f32x2 s = Q[0];
#pragma unroll
    for (int k = 1; k < W; ++k) s = f2_add(s, Q[k]);
    return s;
}

template <typename TP, typename TD, int R, bool INT>
__device__ __forceinline__ void strip2_k4s_row(Strip2BwdRing<R>& z, const Strip2Lane<R>& ln, int U, float g0,
                                               float g1, float p0, float p1, float2 d0, float2 d1, float4 st0,
                                               float4 st1, int e, int e_first, int xa, TP* __restrict__ dP,
                                               TD* __restrict__ dG, const StripGeom& s, f32x2 KG, f32x2 KP) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    const int lane = threadIdx.x & 31;
    const bool row_in = e >= 0 && e < s.h;
    z.rg[U] = f2_pack(g0, g1);
    z.rp[U] = f2_pack(p0, p1);
    if (s.mean) {
        // d Abar / N, d bbar / N at (e, xa), (e, xa + 1); zero outside the image
        float i0 = kInvW2, i1 = kInvW2;
        if (!INT) {
            const int ny = min(e + R, s.h - 1) - max(e - R, 0) + 1;
            i0 = (ln.xin[0] && row_in) ? inv_count(ln.nx_i[0] * ny) : 0.f;
            i1 = (ln.xin[1] && row_in) ? inv_count(ln.nx_i[1] * ny) : 0.f;
        }
        z.hda[U] = strip2_hsum<R>(d0.x * i0, d1.x * i1);
        z.hdb[U] = strip2_hsum<R>(d0.y * i0, d1.y * i1);
    } else {
        // no box mean of A, b: the window's own d Abar, d bbar (row e, read at row e - R below)
        z.hda[U] = f2_pack(d0.x, d1.x);
        z.hdb[U] = f2_pack(d0.y, d1.y);
    }
    const int ce = e - R;
    f32x2 q0 = 0ull, q1 = 0ull, q2 = 0ull, q3 = 0ull;
    if (INT || (ce >= 0 && ce < s.h && e - e_first >= 2 * R)) {
        const int ny = INT ? W : min(ce + R, s.h - 1) - max(ce - R, 0) + 1;
        f32x2 dA, db;
        if (s.mean) {
            dA = z.hda[ring_slot<W>(U, 0)];
            db = z.hdb[ring_slot<W>(U, 0)];
#pragma unroll
            for (int j = 1; j < W; ++j) {  // oldest row first
                dA = f2_add(dA, z.hda[ring_slot<W>(U, j)]);
                db = f2_add(db, z.hdb[ring_slot<W>(U, j)]);
            }
        } else {
            dA = z.hda[(U + W - R) % W];  // row ce = e - R
            db = z.hdb[(U + W - R) % W];
        }
        const f32x2 mu = f2_pack(st0.x, st1.x), nu = f2_pack(st0.y, st1.y);
        const f32x2 ive = f2_pack(st0.z, st1.z), A = f2_pack(st0.w, st1.w);
        const f32x2 gamma = f2_mul(f2_fma(f2_neg(db), mu, dA), ive);
        const f32x2 beta = f2_mul(f2_neg(gamma), A);
        const f32x2 inn = INT ? f2_splat(kInvW2)
                              : f2_pack(inv_count(ln.nx_i[0] * ny), inv_count(ln.nx_i[1] * ny));
        const f32x2 mus = f2_sub(mu, KG), nus = f2_sub(nu, KP);
        q0 = f2_mul(gamma, inn);
        q1 = f2_mul(beta, inn);
        q2 = f2_mul(f2_fma(f2_neg(gamma), mus, db), inn);
        q3 = f2_mul(f2_fma(gamma, nus, f2_fma(f2_add(beta, beta), mus, f2_mul(db, A))), inn);
        if (!INT) {  // windows of columns outside the image contribute nothing
            q0 = f2_mul(q0, ln.xin2);
            q1 = f2_mul(q1, ln.xin2);
            q2 = f2_mul(q2, ln.xin2);
            q3 = f2_mul(q3, ln.xin2);
        }
    }
    {
        float a[2];
        f2_unpack(q0, a[0], a[1]);
        z.hq0[U] = strip2_hsum<R>(a[0], a[1]);
        f2_unpack(q1, a[0], a[1]);
        z.hq1[U] = strip2_hsum<R>(a[0], a[1]);
        f2_unpack(q2, a[0], a[1]);
        z.hq2[U] = strip2_hsum<R>(a[0], a[1]);
        f2_unpack(q3, a[0], a[1]);
        z.hq3[U] = strip2_hsum<R>(a[0], a[1]);
    }
    const int co = ce - R;
    const bool rows = e - e_first >= 4 * R && (INT || (co >= s.y0 && co < s.y0 + s.seg && co < s.h));
    const bool w0 = rows && (INT ? (lane >= R && lane < 32 - R) : ln.out[0]);
    const bool w1 = rows && (INT ? (lane >= R && lane < 32 - R) : ln.out[1]);
    if (w0 || w1) {
        const int k0 = ring_slot<W>(U, 0);
        f32x2 S0 = z.hq0[k0], S1 = z.hq1[k0], S2 = z.hq2[k0], S3 = z.hq3[k0];
#pragma unroll
        for (int j = 1; j < W; ++j) {  // oldest row first
            const int k = ring_slot<W>(U, j);
            S0 = f2_add(S0, z.hq0[k]);
            S1 = f2_add(S1, z.hq1[k]);
            S2 = f2_add(S2, z.hq2[k]);
            S3 = f2_add(S3, z.hq3[k]);
        }
        const int V = ring_slot<W>(U, 0);  // row co = e - 2R, the oldest in the ring
        const f32x2 g = f2_sub(z.rg[V], KG), p = f2_sub(z.rp[V], KP);
        float vp0, vp1, vg0, vg1;
        f2_unpack(f2_fma(g, S0, S2), vp0, vp1);
        f2_unpack(f2_fma(p, S0, f2_fma(f2_add(g, g), S1, f2_neg(S3))), vg0, vg1);
        const size_t o = (size_t)co * s.w + xa;
        if (dP != nullptr) {
            if (w0) dP[o] = from_f32<TP>(vp0);
            if (w1) dP[o + 1] = from_f32<TP>(vp1);
        }
        if (dG != nullptr) {
            if (w0) dG[o] = from_f32<TD>(vg0);
            if (w1) dG[o + 1] = from_f32<TD>(vg1);
        }
    }
}

// K4 for one strip segment from saved statistics, rows loaded one ring period ahead.
template <typename TG, typename TP, typename TD, int R>
__device__ void lowres_bwd_strip2_stats(const TG* __restrict__ G, const TP* __restrict__ P,
                                        const float2* __restrict__ dcoef, const float4* __restrict__ stats,
                                        TP* __restrict__ dP, TD* __restrict__ dG, const StripGeom& s) {
    constexpr int W = 2 * R + 1;
    const int lane = threadIdx.x & 31;
    const int xa = s.x0 + 2 * lane;
    const Strip2Lane<R> ln = strip2_lane<R>(xa, s.w);
    // interior: every lane's columns and their windows inside the image
    const bool cols_int = s.x0 >= R && s.x0 + 64 + R <= s.w;
    Strip2BwdRing<R> z;
#pragma unroll
    for (int k = 0; k < W; ++k)
        z.hda[k] = z.hdb[k] = z.hq0[k] = z.hq1[k] = z.hq2[k] = z.hq3[k] = z.rg[k] = z.rp[k] = 0ull;
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, s.h) + 2 * R;
    float gn[2][W], pn[2][W];
    float2 dn[2][W];
    float4 sn[2][W];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u, ce = e - R;
            const bool row = e >= 0 && e < s.h && e < e_last;
            const bool srow = ce >= 0 && ce < s.h;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const bool ok = row && ln.xin[c];
                const size_t o = (size_t)e * s.w + xa + c;
                gn[c][u] = ok ? to_f32<TG>(G[o]) : 0.f;
                pn[c][u] = ok ? to_f32<TP>(P[o]) : 0.f;
                dn[c][u] = ok ? dcoef[o] : make_float2(0.f, 0.f);
                sn[c][u] = (srow && ln.xin[c]) ? stats[(size_t)ce * s.w + xa + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    load(e_first);
    // shift: mean of row y0 (the last row of the first period) over the output columns
    f32x2 KG, KP;
    {
        float sg = 0.f, sp = 0.f, cn = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (ln.out[c]) {
                sg += gn[c][2 * R];
                sp += pn[c][2 * R];
                cn += 1.f;
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sg += __shfl_xor_sync(0xffffffffu, sg, off);
            sp += __shfl_xor_sync(0xffffffffu, sp, off);
            cn += __shfl_xor_sync(0xffffffffu, cn, off);
        }
        KG = f2_splat(cn > 0.f ? sg / cn : 0.f);
        KP = f2_splat(cn > 0.f ? sp / cn : 0.f);
    }
    for (int base = e_first; base < e_last; base += W) {
        float gv[2][W], pv[2][W];
        float2 dv[2][W];
        float4 sv[2][W];
#pragma unroll
        for (int u = 0; u < W; ++u)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                gv[c][u] = gn[c][u];
                pv[c][u] = pn[c][u];
                dv[c][u] = dn[c][u];
                sv[c][u] = sn[c][u];
            }
        if (base + W < e_last) load(base + W);  // next period in flight while this one computes
        const bool row_int = cols_int && base >= 3 * R && base + W + R <= s.h && base + W <= e_last;
        if (row_int) {
#pragma unroll
            for (int u = 0; u < W; ++u)
                strip2_k4s_row<TP, TD, R, true>(z, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], dv[0][u], dv[1][u],
                                                sv[0][u], sv[1][u], base + u, e_first, xa, dP, dG, s, KG, KP);
        } else {
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (base + u >= e_last) break;  // uniform across the warp
                strip2_k4s_row<TP, TD, R, false>(z, ln, u, gv[0][u], gv[1][u], pv[0][u], pv[1][u], dv[0][u],
                                                 dv[1][u], sv[0][u], sv[1][u], base + u, e_first, xa, dP, dG, s, KG,
                                                 KP);
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
    const f32x2 eps2 = f2_splat(eps);
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
        if (!__all_sync(0xffffffffu, mbar_wait(bar_s + 8u * slot, (uint32_t)((m / NS) & 1), first_wait_limit(status)))) {
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
            const bool row_int = cols_int && base >= 3 * R && base + W <= s.h && base + W <= e_last;
            if (row_int)
                strip2_k1_period<R, true>(q, ln, gv, pv, base, e_first, e_last, xa, coef, stats, s, eps2);
            else
                strip2_k1_period<R, false>(q, ln, gv, pv, base, e_first, e_last, xa, coef, stats, s, eps2);
        }
    }
    if (!ok) {
        if (lane == 0) status_fail(status, kStatusTimeout);
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
