// Low-resolution stage as warp-strip column walks (radius R = 1 or 2): the
// shared pieces and the K4 strips that recompute the window statistics (one
// column per lane); K1 and the K4 that reads saved statistics hold two
// columns per lane (lowres_strip2.cuh).
//
// One warp owns a strip of 32 consecutive low-res columns and walks down a
// segment of rows.  Each lane holds one column: horizontal window terms come
// from the neighbouring lanes by warp shuffles, vertical window terms from a
// register ring of the last 2R + 1 rows (the walk is unrolled by 2R + 1 so
// every ring slot is a fixed register).  No shared memory, no barriers: the
// row loads of the next ring period are issued before the current one is
// processed.  Lanes [2R, 32 - 2R) produce outputs; the 2R lanes on each side
// are the strip's halo (neighbouring strips overlap by 4R columns), and the
// first 4R rows of a segment only fill the rings.
//
// A ring period whose rows and columns are all far enough from the image
// border takes the interior form: every window is full, so the masks and
// clipped counts drop out and the counts' reciprocals are constants (the
// same correctly rounded values the clipped form reads from its table), so a
// pixel's result does not depend on which form produced it.  The first periods of a segment,
// which only fill the rings, take the interior form too when their rows are
// inside the image: what they compute before the rings are full is never
// stored (a per-row predicate) and leaves the rings before any stored
// result reads it.
//
// Statistics are exactly centred as in the tile kernels: each row segment is
// centred on its own mean and rows are combined with Chan's update.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace dgf {

constexpr int kStripWarps = 4;    // warps per CTA of the single-call K1 strips (independent strips)
constexpr int kK4StripWarps = 4;  // warps per CTA of the K4 strips

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

// Ring slot of the j-th oldest row when the newest sits in slot U (rings of
// W = 2R + 1 rows).  Window sums run over the slots in this order, so their
// rounding does not depend on where a segment starts.
template <int W>
__host__ __device__ constexpr int ring_slot(int U, int j) { return (U + 1 + j) % W; }

struct StripGeom {
    int h, w;
    int x0;       // global column of lane 0 (first input column, may be negative)
    int y0;       // first output row of the segment
    int seg;      // output rows of the segment
    int mean = 1; // 1: box mean of A, b (fast guided filter); 0: A, b themselves (the layer as printed)
};

// Register rings of one strip: level 1 holds per-row statistics of the last
// 2R + 1 input rows, level 2 the horizontal box sums of A, b of the last
// 2R + 1 window rows.
template <int R>
struct StripRing {
    static constexpr int W = 2 * R + 1;
    float mg[W], mp[W], sgg[W], sgp[W], vr[W], ha[W], hb[W];
};

// Per-lane facts of the generic form (columns clipped at the image border).
template <int R>
struct StripLane {
    float mk[2 * R + 1];  // 1 where column x - R + k is inside the image
    int nx;               // clipped window width at this lane's column
    bool xin, out;        // column inside the image; lane writes an output
};

// Centred statistics (mu, nu, var, cov) of the window of row ce = e - R
// from the level-1 ring; ny = clipped window height.
template <int R, bool INT>
__device__ __forceinline__ void strip_window(const StripRing<R>& q, const StripLane<R>& ln, int U, int ny, float& mu,
                                             float& nu, float& var, float& cov) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW = 1.f / (float)W;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    float t1 = 0.f, t2 = 0.f, ta = 0.f, tc = 0.f;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int k = ring_slot<W>(U, j);
        t1 += q.mg[k];
        t2 += q.mp[k];
        ta += q.sgg[k];
        tc += q.sgp[k];
    }
    const float iny = INT ? kInvW : inv_count(ny);
    mu = t1 * iny;
    nu = t2 * iny;
    float dgg = 0.f, dgp = 0.f;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int k = ring_slot<W>(U, j);
        const float dg = INT ? q.mg[k] - mu : q.vr[k] * (q.mg[k] - mu);
        dgg = fmaf(dg, dg, dgg);
        dgp = fmaf(dg, q.mp[k] - nu, dgp);
    }
    const float nxf = INT ? (float)W : (float)ln.nx;
    const float inn = INT ? kInvW2 : inv_count(ln.nx * ny);
    var = fmaf(nxf, dgg, ta) * inn;
    cov = fmaf(nxf, dgp, tc) * inn;
}

// Level 1 for input row e: centred statistics of the row over this lane's
// window columns, stored in ring slot U.
template <int R, bool INT>
__device__ __forceinline__ void strip_row_stats(StripRing<R>& q, const StripLane<R>& ln, int U, float gvu,
                                                float pvu, bool row_in) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW = 1.f / (float)W;
    float g[W], p[W];
    g[R] = gvu;
    p[R] = pvu;
#pragma unroll
    for (int d = 1; d <= R; ++d) {
        g[R - d] = shfl_up(gvu, d);
        g[R + d] = shfl_dn(gvu, d);
        p[R - d] = shfl_up(pvu, d);
        p[R + d] = shfl_dn(pvu, d);
    }
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        s1 += g[k];
        s2 += p[k];
    }
    const float inx = INT ? kInvW : inv_count(ln.nx);
    const float m1 = s1 * inx, m2 = s2 * inx;
    float a = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const float dg = INT ? g[k] - m1 : ln.mk[k] * (g[k] - m1);
        a = fmaf(dg, dg, a);
        c = fmaf(dg, p[k] - m2, c);
    }
    q.mg[U] = m1;
    q.mp[U] = m2;
    q.sgg[U] = a;
    q.sgp[U] = c;
    q.vr[U] = (INT || row_in) ? 1.f : 0.f;
}

// Per-lane facts of the generic form, for column x.
template <int R>
__device__ __forceinline__ StripLane<R> strip_lane(int x, int w) {
    StripLane<R> ln;
    const int lane = threadIdx.x & 31;
    ln.xin = x >= 0 && x < w;
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) {
        const int xx = x - R + k;
        ln.mk[k] = (xx >= 0 && xx < w) ? 1.f : 0.f;
    }
    ln.nx = ln.xin ? min(x + R, w - 1) - max(x - R, 0) + 1 : 1;
    ln.out = lane >= 2 * R && lane < 32 - 2 * R && ln.xin;
    return ln;
}

// ------------------------------------------------- TMA staging of the strips
// A warp's rows arrive in blocks of RB rows (whole ring periods) through a
// ring of NS shared-memory slots, one mbarrier per slot.  Each input is one
// tiled copy per block: box (32 + U) columns x RB rows starting at the
// strip's first column rounded down to the 16-byte unit U (the lane reads at
// its offset inside the box); rows and columns outside the image read as
// zero, exactly what the plain loads supply.  The warp's lane 0 refills a
// slot once the warp has read it.  Waits are bounded: on a timeout the warp
// records it in the status word, waits (bounded) for its copies in flight
// and stops.
template <int R>
struct StripTmaCfg {
    static constexpr int RB = R == 1 ? 6 : 10;  // rows per block (2 ring periods)
    static constexpr int NS = 4;                // slots per warp
    // K4's slots also hold d Abar, d bbar; at R = 2 three slots keep a CTA's
    // ring under 56 KB, so four CTAs (16 warps) share an SM
    static constexpr int NS4 = R == 1 ? 4 : 3;
};

__host__ __device__ constexpr int strip_box_cols(int esize) { return 32 + 16 / esize; }
__host__ __device__ constexpr int align128i(int b) { return (b + 127) / 128 * 128; }
// bytes of one input's box in a slot (rounded to 128) for element size esize
__host__ __device__ constexpr int strip_box_bytes(int R, int esize, int rows) {
    return align128i(rows * strip_box_cols(esize) * esize);
}

__device__ __forceinline__ int floor_to(int x, int u) { return x >= 0 ? x / u * u : -((-x + u - 1) / u) * u; }

// ------------------------------------------------------------------- K4
// Algorithm 1 at low resolution for one strip segment.  Per window m (row
// ce, this lane's column): the statistics, dA = f_mu^T(d Abar) and
// db = f_mu^T(d bbar) as box sums of d Abar / N, d bbar / N, then
//   gamma = (dA - db mu) / (var + eps),  beta = -gamma A,
// and four quantities whose sums over the windows containing a pixel give
//   dP = G' S0 + S2,   dG = P' S0 + 2 G' S1 - S3,
// with S0 = sum gamma / N, S1 = sum beta / N, S2 = sum (db - gamma mu') / N,
// S3 = sum (gamma nu' + 2 beta mu' + db A) / N.  Primes are shifts by a
// per-strip constant (the mean of the segment's first output row), which
// conditions the separable sums; the result is the same in exact arithmetic.
template <int R>
struct StripBwdRing {
    static constexpr int W = 2 * R + 1;
    float hda[W], hdb[W];               // row box sums of d Abar / N, d bbar / N (input rows)
    float hq0[W], hq1[W], hq2[W], hq3[W];  // row box sums of the four window quantities (window rows)
    float rg[W], rp[W];                 // raw G, P of the input rows
};

template <typename TG, typename TP, typename TD, int R, bool INT>
__device__ __forceinline__ void strip_k4_row(StripRing<R>& q, StripBwdRing<R>& z, const StripLane<R>& ln, int U,
                                             float gvu, float pvu, float2 dvu, int e, int e_first, int x,
                                             TP* __restrict__ dP, TD* __restrict__ dG, const StripGeom& s,
                                             float eps, float KG, float KP) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    const int lane = threadIdx.x & 31;
    const bool row_in = e >= 0 && e < s.h;
    strip_row_stats<R, INT>(q, ln, U, gvu, pvu, row_in);
    z.rg[U] = gvu;
    z.rp[U] = pvu;
    if (s.mean) {
        // d Abar / N, d bbar / N at (e, x); zero outside the image
        const float inn = INT ? kInvW2
                              : ((ln.xin && row_in) ? inv_count(ln.nx * (min(e + R, s.h - 1) - max(e - R, 0) + 1))
                                                    : 0.f);
        z.hda[U] = hsum<R>(dvu.x * inn);
        z.hdb[U] = hsum<R>(dvu.y * inn);
    } else {
        // no box mean of A, b: the window's own d Abar, d bbar (row e, read at row e - R below)
        z.hda[U] = dvu.x;
        z.hdb[U] = dvu.y;
    }
    const int ce = e - R;
    float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
    if (INT || (ln.xin && ce >= 0 && ce < s.h && e - e_first >= 2 * R)) {
        const int ny = INT ? W : min(ce + R, s.h - 1) - max(ce - R, 0) + 1;
        float mu, nu, var, cov;
        strip_window<R, INT>(q, ln, U, ny, mu, nu, var, cov);
        float dA = 0.f, db = 0.f;
        if (s.mean) {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                dA += z.hda[ring_slot<W>(U, j)];
                db += z.hdb[ring_slot<W>(U, j)];
            }
        } else {
            dA = z.hda[(U + W - R) % W];  // row ce = e - R
            db = z.hdb[(U + W - R) % W];
        }
        const float ive = rcp_approx(var + eps);
        const float A = cov * ive;
        const float gamma = fmaf(-db, mu, dA) * ive;
        const float beta = -gamma * A;
        const float inn = INT ? kInvW2 : inv_count(ln.nx * ny);
        const float mus = mu - KG, nus = nu - KP;
        q0 = gamma * inn;
        q1 = beta * inn;
        q2 = fmaf(-gamma, mus, db) * inn;
        q3 = fmaf(gamma, nus, fmaf(2.f * beta, mus, db * A)) * inn;
    }
    z.hq0[U] = hsum<R>(q0);
    z.hq1[U] = hsum<R>(q1);
    z.hq2[U] = hsum<R>(q2);
    z.hq3[U] = hsum<R>(q3);
    const int co = ce - R;
    const bool write = INT ? (lane >= 2 * R && lane < 32 - 2 * R && e - e_first >= 4 * R)
                           : (ln.out && co >= s.y0 && co < s.y0 + s.seg && co < s.h && e - e_first >= 4 * R);
    if (write) {
        float S0 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = ring_slot<W>(U, j);
            S0 += z.hq0[k];
            S1 += z.hq1[k];
            S2 += z.hq2[k];
            S3 += z.hq3[k];
        }
        constexpr int kLag = 1;  // row co = e - 2R sits in slot (U + 1) mod W
        const int V = (U + kLag) % W;
        const float g = z.rg[V] - KG, p = z.rp[V] - KP;
        const size_t o = (size_t)co * s.w + x;
        if (dP != nullptr) dP[o] = from_f32<TP>(fmaf(g, S0, S2));
        if (dG != nullptr) dG[o] = from_f32<TD>(fmaf(p, S0, fmaf(2.f * g, S1, -S3)));
    }
}

template <typename TG, typename TP, typename TD, int R>
__device__ void lowres_bwd_strip(const TG* __restrict__ G, const TP* __restrict__ P,
                                 const float2* __restrict__ dcoef, TP* __restrict__ dP, TD* __restrict__ dG,
                                 const StripGeom& s, float eps) {
    constexpr int W = 2 * R + 1;
    const int lane = threadIdx.x & 31;
    const int x = s.x0 + lane;
    const StripLane<R> ln = strip_lane<R>(x, s.w);
    // interior columns: every lane's column and its count's window inside the image
    const bool cols_int = s.x0 >= R && s.x0 + 32 + R <= s.w;
    StripRing<R> q;
    StripBwdRing<R> z;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        q.mg[k] = q.mp[k] = q.sgg[k] = q.sgp[k] = q.vr[k] = 0.f;
        z.hda[k] = z.hdb[k] = z.hq0[k] = z.hq1[k] = z.hq2[k] = z.hq3[k] = z.rg[k] = z.rp[k] = 0.f;
    }
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, s.h) + 2 * R;
    float gn[W], pn[W];
    float2 dn[W];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            const bool ok = ln.xin && e >= 0 && e < s.h && e < e_last;
            const size_t o = (size_t)e * s.w + x;
            gn[u] = ok ? to_f32<TG>(G[o]) : 0.f;
            pn[u] = ok ? to_f32<TP>(P[o]) : 0.f;
            dn[u] = ok ? dcoef[o] : make_float2(0.f, 0.f);
        }
    };
    load(e_first);
    // shift: mean of row y0 (the last row of the first period) over the output lanes
    float KG, KP;
    {
        const bool use = ln.out;
        float sg = use ? gn[2 * R] : 0.f, sp = use ? pn[2 * R] : 0.f, cn = use ? 1.f : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sg += __shfl_xor_sync(0xffffffffu, sg, off);
            sp += __shfl_xor_sync(0xffffffffu, sp, off);
            cn += __shfl_xor_sync(0xffffffffu, cn, off);
        }
        KG = cn > 0.f ? sg / cn : 0.f;
        KP = cn > 0.f ? sp / cn : 0.f;
    }
    for (int base = e_first; base < e_last; base += W) {
        float gv[W], pv[W];
        float2 dv[W];
#pragma unroll
        for (int u = 0; u < W; ++u) {
            gv[u] = gn[u];
            pv[u] = pn[u];
            dv[u] = dn[u];
        }
        if (base + W < e_last) load(base + W);
        const bool row_int = cols_int && base >= 3 * R && base + W + R <= s.h &&
                             base + W <= e_last;
        if (row_int) {
#pragma unroll
            for (int u = 0; u < W; ++u)
                strip_k4_row<TG, TP, TD, R, true>(q, z, ln, u, gv[u], pv[u], dv[u], base + u, e_first, x, dP, dG,
                                                  s, eps, KG, KP);
        } else {
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (base + u >= e_last) break;  // uniform across the warp
                strip_k4_row<TG, TP, TD, R, false>(q, z, ln, u, gv[u], pv[u], dv[u], base + u, e_first, x, dP,
                                                   dG, s, eps, KG, KP);
            }
        }
    }
}


// K4 strip with TMA staging of G, P and d Abar, d bbar (same slots as K1's,
// one more box per slot).
template <typename TG, typename TP, typename TD, int R>
__device__ void lowres_bwd_strip_tma(const TmaTriple* maps, int plane, TP* __restrict__ dP, TD* __restrict__ dG,
                                     const StripGeom& s, float eps, unsigned char* ring, uint64_t* bars,
                                     uint32_t* status) {
    constexpr int W = 2 * R + 1, RB = StripTmaCfg<R>::RB, NS = StripTmaCfg<R>::NS4, NP = RB / W;
    constexpr int UG = 16 / (int)sizeof(TG), UP = 16 / (int)sizeof(TP);
    constexpr int BXG = 32 + UG, BXP = 32 + UP, BXD = 2 * (32 + 2);  // d: float pairs
    constexpr int BG = strip_box_bytes(R, (int)sizeof(TG), RB), BP = strip_box_bytes(R, (int)sizeof(TP), RB);
    constexpr int BD = align128i(RB * BXD * 4);
    constexpr int SLOT = BG + BP + BD;
    constexpr uint32_t TX =
        (uint32_t)(RB * BXG * (int)sizeof(TG) + RB * BXP * (int)sizeof(TP) + RB * BXD * 4);
    const int lane = threadIdx.x & 31;
    const int x = s.x0 + lane;
    const StripLane<R> ln = strip_lane<R>(x, s.w);
    const bool cols_int = s.x0 >= R && s.x0 + 32 + R <= s.w;
    StripRing<R> q;
    StripBwdRing<R> z;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        q.mg[k] = q.mp[k] = q.sgg[k] = q.sgp[k] = q.vr[k] = 0.f;
        z.hda[k] = z.hdb[k] = z.hq0[k] = z.hq1[k] = z.hq2[k] = z.hq3[k] = z.rg[k] = z.rp[k] = 0.f;
    }
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, s.h) + 2 * R;
    const int nblk = (e_last - e_first + RB - 1) / RB;
    const int xg = floor_to(s.x0, UG), xp = floor_to(s.x0, UP), xd = floor_to(s.x0, 2);
    const int og = s.x0 - xg + lane, op = s.x0 - xp + lane, od = 2 * (s.x0 - xd + lane);
    const uint32_t ring_s = smem_u32(ring), bar_s = smem_u32(bars);
    auto issue = [&](int m) {  // lane 0: block m into slot m % NS
        const int slot = m % NS;
        const uint32_t bar = bar_s + 8u * slot, dst = ring_s + (uint32_t)(slot * SLOT);
        const int y = e_first + m * RB;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(TX) : "memory");
        tma_load_3d(dst, &maps->a.map, xg, y, plane, bar);
        tma_load_3d(dst + BG, &maps->b.map, xp, y, plane, bar);
        tma_load_3d(dst + BG + BP, &maps->c.map, 2 * xd, y, plane, bar);
    };
    if (lane == 0) {
        for (int k = 0; k < NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * k) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int m = 0; m < min(NS, nblk); ++m) issue(m);
    }
    __syncwarp();
    float KG = 0.f, KP = 0.f;
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
        const float* sd = reinterpret_cast<const float*>(ring + slot * SLOT + BG + BP) + od;
        if (m == 0) {
            // shift: mean of row y0 (row 2R of the first block) over the output lanes
            const bool use = ln.out;
            float a = use ? to_f32<TG>(sg[2 * R * BXG]) : 0.f, b = use ? to_f32<TP>(sp[2 * R * BXP]) : 0.f;
            float cn = use ? 1.f : 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, off);
                b += __shfl_xor_sync(0xffffffffu, b, off);
                cn += __shfl_xor_sync(0xffffffffu, cn, off);
            }
            KG = cn > 0.f ? a / cn : 0.f;
            KP = cn > 0.f ? b / cn : 0.f;
        }
#pragma unroll 1  // one copy of the period's code (ring slots are fixed within a period)
        for (int pp = 0; pp < NP; ++pp) {
            const int base = e_first + m * RB + pp * W;
            float gv[W], pv[W];
            float2 dv[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                gv[u] = to_f32<TG>(sg[(pp * W + u) * BXG]);
                pv[u] = to_f32<TP>(sp[(pp * W + u) * BXP]);
                dv[u] = *reinterpret_cast<const float2*>(sd + (pp * W + u) * BXD);
            }
            if (pp == NP - 1) {
                __syncwarp();  // every lane has read the slot
                if (lane == 0 && m + NS < nblk) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(m + NS);
                }
            }
            if (base >= e_last) continue;  // uniform
            const bool row_int = cols_int && base >= 3 * R && base + W + R <= s.h &&
                                 base + W <= e_last;
            if (row_int) {
#pragma unroll
                for (int u = 0; u < W; ++u)
                    strip_k4_row<TG, TP, TD, R, true>(q, z, ln, u, gv[u], pv[u], dv[u], base + u, e_first, x, dP,
                                                      dG, s, eps, KG, KP);
            } else {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    if (base + u >= e_last) break;  // uniform across the warp
                    strip_k4_row<TG, TP, TD, R, false>(q, z, ln, u, gv[u], pv[u], dv[u], base + u, e_first, x, dP,
                                                       dG, s, eps, KG, KP);
                }
            }
        }
    }
    if (!ok) {
        if (lane == 0) status_fail(status, kStatusTimeout);
        for (int qb = m; qb < nblk && qb < m + NS; ++qb)
            mbar_wait(bar_s + 8u * (qb % NS), (uint32_t)((qb / NS) & 1), kWaitLimit);
    }
}

// shared memory of one CTA of K4 strips staged by TMA (kK4StripWarps warps)
template <typename TG, typename TP, int R>
__host__ __device__ constexpr int k4_strip_tma_smem() {
    return kK4StripWarps * StripTmaCfg<R>::NS4 *
               (strip_box_bytes(R, (int)sizeof(TG), StripTmaCfg<R>::RB) +
                strip_box_bytes(R, (int)sizeof(TP), StripTmaCfg<R>::RB) +
                align128i(StripTmaCfg<R>::RB * 2 * (32 + 2) * 4)) +
           kK4StripWarps * StripTmaCfg<R>::NS4 * 8;
}

}  // namespace dgf
