// Low-resolution stage with running (sliding) window sums: K1 and K4 at a
// cost per pixel that does not grow with the radius.  Used for 16-bit
// storage, where the parity gates leave room for the rounding of running
// sums over shifted data; FP32 storage keeps the exactly centred strips.
//
// One warp owns a strip of 32 lanes x V consecutive low-res columns and
// walks down a segment of rows.  The two box passes are separable:
//  * vertical: per column, a running sum over the last 2R + 1 rows; each
//    step adds the newest row and subtracts the row leaving the window,
//    whose terms are recomputed from its stored inputs with the same
//    operations, so the subtraction removes exactly the value that was
//    added.  The second pass (box of A, b in K1; of Algorithm 1's four
//    window quantities in K4) keeps its last 2R + 1 rows in a per-warp
//    shared-memory ring for the same purpose.
//  * staging: input rows reach each warp through a shared-memory ring of
//    2R + 1 + D rows filled D rows ahead by cp.async (each lane copies its
//    own V columns, so a lane reads only what it copied itself and no
//    barrier is needed); the leaving row and K4's output row are read from
//    the same ring.  Rows and columns outside the image are zero-filled.
//    Planes whose rows or pointers do not allow aligned copies fill the
//    ring with plain loads (same values, same arithmetic).
//  * horizontal: the vertical sums of a row, V per lane, slide along the
//    lane's columns; the R columns on each side come from the neighbouring
//    lanes by warp shuffles.
// The statistics use G' = G - K_G and P' = P - K_P, with K the mean of the
// segment's first output row over the strip (rounded to the guide's storage
// type, so G' is exact for 16-bit data): var = E[G'^2] - E[G']^2 and
// cov = E[G'P'] - E[G']E[P'] (the shift keeps both differences well
// conditioned; it cancels exactly in exact arithmetic).
//
// Geometry: a strip reads columns [x_base, x_base + 32 V), x_base = strip *
// OUTC - HB; columns [HB, HB + OUTC) of the strip are its outputs (HB >= 2R,
// a multiple of V, so every lane is wholly an output lane or wholly halo).
// A segment of S output rows walks input rows [y0 - 2R, y0 + S + 2R): the
// first 2R rows only fill the vertical sums of the first pass, the next 2R
// those of the second.  Values outside the image enter the sums as zero and
// window counts are clipped to the image.
#pragma once

#include "common.cuh"

namespace dgf {

template <int R, int V>
struct SlideGeom {
    static constexpr int W = 2 * R + 1;
    static constexpr int HB = V * ((2 * R + V - 1) / V);  // halo columns per side
    static constexpr int OUTC = 32 * V - 2 * HB;         // output columns per strip
    static_assert(OUTC > 0, "strip too narrow for the radius");
};

constexpr int kSlideWarps = 4;  // warps per CTA (independent strip segments)

// Warps per CTA (1 .. kSlideWarps): the count that keeps the most warps'
// rings resident on an SM (228 KB of shared memory, 1 KB reserved per CTA,
// at most 227 KB per CTA); the larger count on a tie.
template <int WARP_BYTES>
constexpr int slide_wpc() {
    int best = 1, most = 0;
    for (int wpc = 1; wpc <= kSlideWarps; ++wpc) {
        const int cta = wpc * WARP_BYTES + 1024;
        if (cta > 227 * 1024 + 1024) break;
        const int warps = (228 * 1024 / cta) * wpc;
        if (warps >= most) {
            most = warps;
            best = wpc;
        }
    }
    return best;
}


// Radius-R horizontal window sums of a row held V columns per lane, on
// pairs of quantities: out[j] = sum over k in [-R, R] of x at lane column
// j + k.  Lanes reach their neighbours by shuffles (each half moves on its
// own; the sums are paired instructions); results are meaningful for strip
// columns [R, 32 V - R) only (the others read across the warp's edge).
template <int R, int V>
__device__ __forceinline__ void hbox2(const f32x2 (&x)[V], f32x2 (&out)[V]) {
    f32x2 T[V + 2 * R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int o = -R + k;
        const int dl = -((-o + V - 1) / V);
        const int j = o - dl * V;
        float a, b;
        f2_unpack(x[j], a, b);
        T[k] = f2_pack(__shfl_up_sync(0xffffffffu, a, -dl), __shfl_up_sync(0xffffffffu, b, -dl));
    }
#pragma unroll
    for (int j = 0; j < V; ++j) T[R + j] = x[j];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int o = V + k;
        float a, b;
        f2_unpack(x[o % V], a, b);
        T[R + V + k] = f2_pack(__shfl_down_sync(0xffffffffu, a, o / V), __shfl_down_sync(0xffffffffu, b, o / V));
    }
    f32x2 s = T[0];
#pragma unroll
    for (int k = 1; k <= 2 * R; ++k) s = f2x_add(s, T[k]);
    out[0] = s;
#pragma unroll
    for (int j = 1; j < V; ++j) {
        s = f2x_sub(f2x_add(s, T[j + 2 * R]), T[j - 1]);
        out[j] = s;
    }
}

// Row e of one plane at the lane's V columns, as floats (zero outside the
// image).  vec: the whole vector is inside the image and aligned.
template <typename T, int V>
__device__ __forceinline__ void slide_load(const T* __restrict__ src, int e, int h, int w, int x0, bool vec,
                                           float (&out)[V]) {
    if (e < 0 || e >= h) {
#pragma unroll
        for (int j = 0; j < V; ++j) out[j] = 0.f;
        return;
    }
    const T* row = src + (size_t)e * w;
    if (vec) {
        const Vec<T, V> v = *reinterpret_cast<const Vec<T, V>*>(row + x0);
#pragma unroll
        for (int j = 0; j < V; ++j) out[j] = to_f32<T>(v.v[j]);
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int x = x0 + j;
            out[j] = (x >= 0 && x < w) ? to_f32<T>(row[x]) : 0.f;
        }
    }
}

// Per-lane column facts.
template <int R, int V>
struct SlideLane {
    float nx[V];     // clipped window width of each column (1 outside the image)
    float inx[V];    // 1 / nx, correctly rounded
    float xin[V];    // 1 inside the image, else 0
    bool col_int;    // every column of the lane has the full width 2R + 1
    bool out;        // the lane's columns are strip outputs
    bool vec;        // vector loads of the lane's columns are in bounds and aligned
    int x0;          // first column
};

template <int R, int V>
__device__ __forceinline__ SlideLane<R, V> slide_lane(int x_base, int w, bool aligned) {
    using Gm = SlideGeom<R, V>;
    SlideLane<R, V> L;
    const int lane = threadIdx.x & 31;
    L.x0 = x_base + lane * V;
    L.col_int = true;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int x = L.x0 + j;
        const bool in = x >= 0 && x < w;
        L.xin[j] = in ? 1.f : 0.f;
        const int n = in ? min(x + R, w - 1) - max(x - R, 0) + 1 : 1;
        L.nx[j] = (float)n;
        L.inx[j] = __frcp_rn((float)n);
        L.col_int = L.col_int && n == 2 * R + 1;
    }
    L.out = lane * V >= Gm::HB && lane * V < Gm::HB + Gm::OUTC;
    L.vec = aligned && L.x0 >= 0 && L.x0 + V <= w;
    return L;
}


// 1 / (window count) of the window of ny rows at column j: the product of
// the correctly rounded reciprocals of its width and height (one multiply
// per pixel; iny = 1 / ny is formed once per row).  Every use of a count
// in this file goes through it, so a term subtracted from a running sum is
// scaled exactly as it was when it was added.
template <int R, int V>
__device__ __forceinline__ float slide_inv(const SlideLane<R, V>& L, int j, float iny) {
    return L.inx[j] * iny;
}
__device__ __forceinline__ float slide_iny(int y, int h, int R) {
    return __frcp_rn((float)(min(y + R, h - 1) - max(y - R, 0) + 1));
}

// Shift constant: mean over the strip's in-image columns of row y (the
// segment's first output row), rounded to the storage type T.
template <typename T, int V>
__device__ __forceinline__ float slide_shift(const float (&v)[V], const float (&xin)[V]) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        s += v[j] * xin[j];
        c += xin[j];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    const float k = c > 0.f ? s / c : 0.f;
    return to_f32<T>(from_f32<T>(k));
}

// ---------------------------------------------------------------- staging
// Asynchronous copy of BYTES (4, 8 or 16) from global to shared memory; the
// bytes past `src_bytes` are zero-filled (src_bytes = 0: no read at all).
template <int BYTES>
__device__ __forceinline__ void slide_cp_async(uint32_t dst, const void* src, uint32_t src_bytes) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES),
                     "r"(src_bytes)
                     : "memory");
}
__device__ __forceinline__ void slide_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void slide_cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Prefetch depth (rows in flight ahead of the one being processed).
// K4 stages three inputs per row and keeps four quantities per column in
// its second-pass ring, so it prefetches fewer rows; at R = 8 K1's depth of
// 3 keeps the batched K1's eight warps of rings under 227 KB.
template <int R, bool K4 = false>
struct SlideStage {
    static constexpr int D = R > 4 ? 3 : (K4 ? 4 : 6);
    static constexpr int NR = 2 * R + 1 + D + 1;  // ring rows: the window, the rows in flight, the newest
};

// Copies the lane's V elements of row e of `src` (type T) to `dst` (its
// slot in shared memory): asynchronously when `async` (aligned rows), else
// by plain loads and stores.  Zero outside the image; with aligned rows a
// lane is wholly inside or outside (x0 and w are multiples of V).
template <typename T, int V>
__device__ __forceinline__ void stage_row(unsigned char* dst, const T* __restrict__ src, int e, int h, int w, int x0,
                                          bool async) {
    constexpr int BYTES = V * (int)sizeof(T);
    const bool in_row = e >= 0 && e < h;
    if (async) {
        const bool in = in_row && x0 >= 0 && x0 + V <= w;
        const T* p = in ? src + (size_t)e * w + x0 : src;
        constexpr int CH = BYTES < 16 ? BYTES : 16;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
#pragma unroll
        for (int c = 0; c < BYTES / CH; ++c)
            slide_cp_async<CH>(d + c * CH, reinterpret_cast<const char*>(p) + c * CH, in ? CH : 0);
    } else {
        Vec<T, V> v;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int x = x0 + j;
            v.v[j] = (in_row && x >= 0 && x < w) ? src[(size_t)e * w + x] : from_f32<T>(0.f);
        }
        *reinterpret_cast<Vec<T, V>*>(dst) = v;
    }
}

// The lane's V elements of a staged row, as floats.
template <typename T, int V>
__device__ __forceinline__ void unstage_row(const unsigned char* slot, float (&out)[V]) {
    const Vec<T, V> v = *reinterpret_cast<const Vec<T, V>*>(slot);
#pragma unroll
    for (int j = 0; j < V; ++j) out[j] = to_f32<T>(v.v[j]);
}

// ------------------------------------------------------------------- K1
// One strip segment: Abar, bbar of output rows [y0, y0 + S) (clipped to the
// plane).  ring: this warp's second-pass ring, (2R + 1) x 32 x V pairs, then
// its input ring, SlideStage<R>::NR rows of G and P (k1_slide_warp_bytes).
template <typename TG, typename TP, int R, int V>
__host__ __device__ constexpr int k1_slide_warp_bytes() {
    return (2 * R + 1) * 32 * V * 8 + SlideStage<R>::NR * 32 * V * ((int)sizeof(TG) + (int)sizeof(TP));
}

// AL: rows are V-element aligned (w a multiple of V, aligned bases): the
// lanes stage them by asynchronous copies, else by plain loads.
template <typename TG, typename TP, int R, int V, bool AL>
__device__ void k1_slide_segment_t(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                                   int h, int w, float eps, int x_base, int y0, int S, float4* __restrict__ ring) {
    constexpr bool aligned = AL;
    using Gm = SlideGeom<R, V>;
    constexpr int W = Gm::W;
    const int lane = threadIdx.x & 31;
    const SlideLane<R, V> L = slide_lane<R, V>(x_base, w, aligned);
    const int y1 = min(y0 + S, h);
    const int e0 = y0 - 2 * R, nrow = (y1 - y0) + 4 * R;
    float KG, KP;
    {
        float g[V], p[V];
        slide_load<TG, V>(G, y0, h, w, L.x0, L.vec, g);
        slide_load<TP, V>(P, y0, h, w, L.x0, L.vec, p);
        KG = slide_shift<TG, V>(g, L.xin);
        KP = slide_shift<TP, V>(p, L.xin);
    }
    // quantities held in pairs per column: (G', P') sums, (G'^2, G'P') sums,
    // and the second pass's (A, b) sums
    f32x2 a1[V], a2[V], ab[V];
    // the shift and the column mask as one paired FMA: (G', P') = (G, P) xin - (K_G, K_P) xin
    f32x2 xin2[V], nk[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        a1[j] = a2[j] = ab[j] = f2_splat(0.f);
        xin2[j] = f2_splat(L.xin[j]);
        nk[j] = f2_pack(-KG * L.xin[j], -KP * L.xin[j]);
    }
    const f32x2 K2 = f2_pack(KG, KP);
    // input rows through the ring, D rows ahead (the leaving row is still there)
    constexpr int D = SlideStage<R>::D, NR = SlideStage<R>::NR;
    constexpr int SLOT = 32 * V * ((int)sizeof(TG) + (int)sizeof(TP));
    unsigned char* rin = reinterpret_cast<unsigned char*>(ring + W * (V / 2) * 32);
    const int og = lane * V * (int)sizeof(TG), op = 32 * V * (int)sizeof(TG) + lane * V * (int)sizeof(TP);
    auto issue = [&](int tt, int slot) {  // row e0 + tt into ring slot `slot`
        unsigned char* sl = rin + slot * SLOT;
        stage_row<TG, V>(sl + og, G, e0 + tt, h, w, L.x0, aligned);
        stage_row<TP, V>(sl + op, P, e0 + tt, h, w, L.x0, aligned);
    };
    // a staged row's shifted (G', P') pairs
    auto shifted = [&](int slot, f32x2 (&sh)[V]) {
        const unsigned char* sl = rin + slot * SLOT;
        float g[V], p[V];
        unstage_row<TG, V>(sl + og, g);
        unstage_row<TP, V>(sl + op, p);
#pragma unroll
        for (int j = 0; j < V; ++j) sh[j] = f2x_fma(f2_pack(g[j], p[j]), xin2[j], nk[j]);
    };
#pragma unroll 1
    for (int tt = 0; tt < D; ++tt) {
        if (tt < nrow) issue(tt, tt);
        slide_cp_commit();
    }
    auto wrap = [](int k) { return k + 1 == NR ? 0 : k + 1; };
    int sn = 0, so = NR - W, sf = D;  // ring slots of rows t, t - W and t + D
    int u = 0;  // second-pass ring slot of the newest window row
    for (int t = 0; t < nrow; ++t) {
        const int e = e0 + t;
        if (t + D < nrow) issue(t + D, sf);
        slide_cp_commit();
        slide_cp_wait<D>();  // row e (and every older one) has landed
        // first pass, vertical: add row e ...
        if (e >= 0 && e < h) {
            f32x2 sh[V];
            shifted(sn, sh);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a1[j] = f2x_add(a1[j], sh[j]);
                a2[j] = f2x_add(a2[j], f2x_mul(f2_splat(f2_lo(sh[j])), sh[j]));
            }
        }
        // ... and subtract row e - W (zero when outside the image or before the walk)
        const int eo = e - W;
        if (t >= W && eo >= 0 && eo < h) {
            f32x2 sh[V];
            shifted(so, sh);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a1[j] = f2x_sub(a1[j], sh[j]);
                a2[j] = f2x_sub(a2[j], f2x_mul(f2_splat(f2_lo(sh[j])), sh[j]));
            }
        }
        sn = wrap(sn);
        so = wrap(so);
        sf = wrap(sf);
        if (t < 2 * R) continue;  // uniform: the first pass's sums are not full yet
        // first pass, horizontal, at window row c1 = e - R: statistics -> (A, b)
        const int c1 = e - R;
        f32x2 s1[V], s2[V], nab[V];
        hbox2<R, V>(a1, s1);
        hbox2<R, V>(a2, s2);
        const bool c1in = c1 >= 0 && c1 < h;
        const float iny1 = c1in ? slide_iny(c1, h, R) : 1.f;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const f32x2 inv2 = f2_splat(slide_inv<R, V>(L, j, iny1));
            const f32x2 m = f2x_mul(s1[j], inv2);                    // (mu', nu')
            const f32x2 q = f2x_mul(s2[j], inv2);                    // (E[G'^2], E[G'P'])
            const f32x2 vc = f2x_fma(f2_splat(-f2_lo(m)), m, q);     // (var, cov)
            const float var = fmaxf(f2_lo(vc), 0.f);
            const float a = f2_hi(vc) * rcp_approx(var + eps);
            const f32x2 mk = f2x_add(m, K2);                         // (mu, nu)
            const float b = fmaf(-a, f2_lo(mk), f2_hi(mk));
            nab[j] = (c1in && L.xin[j] != 0.f) ? f2_pack(a, b) : f2_splat(0.f);
        }
        // second pass, vertical: add window row c1, subtract row c1 - W from the ring
        float4* slot = ring + (size_t)u * (V / 2) * 32 + lane;
        if (t - 2 * R >= W) {
#pragma unroll
            for (int j = 0; j < V; j += 2) {
                const float4 o = slot[(j / 2) * 32];
                ab[j] = f2x_sub(f2x_add(ab[j], nab[j]), f2_pack(o.x, o.y));
                ab[j + 1] = f2x_sub(f2x_add(ab[j + 1], nab[j + 1]), f2_pack(o.z, o.w));
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) ab[j] = f2x_add(ab[j], nab[j]);
        }
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            float a0, b0, a1v, b1v;
            f2_unpack(nab[j], a0, b0);
            f2_unpack(nab[j + 1], a1v, b1v);
            slot[(j / 2) * 32] = make_float4(a0, b0, a1v, b1v);
        }
        u = (u + 1 == W) ? 0 : u + 1;
        if (t < 4 * R) continue;  // uniform: the second pass's sums are not full yet
        // second pass, horizontal, at output row c2 = e - 2R
        const int c2 = e - 2 * R;
        f32x2 sab[V];
        hbox2<R, V>(ab, sab);
        if (L.out) {
            const float iny2 = slide_iny(c2, h, R);
            float2* orow = coef + (size_t)c2 * w;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = L.x0 + j;
                if (x < w) {
                    float A, B;
                    f2_unpack(f2x_mul(sab[j], f2_splat(slide_inv<R, V>(L, j, iny2))), A, B);
                    orow[x] = make_float2(A, B);
                }
            }
        }
    }
    slide_cp_wait<0>();  // the last groups are empty; nothing is left in flight
}

// The segment with the row alignment as a compile-time choice (two
// specialised walks).
template <typename TG, typename TP, int R, int V>
__device__ __forceinline__ void k1_slide_segment(const TG* __restrict__ G, const TP* __restrict__ P,
                                                 float2* __restrict__ coef, int h, int w, float eps, int x_base,
                                                 int y0, int S, bool aligned, float4* __restrict__ ring) {
    if (aligned)
        k1_slide_segment_t<TG, TP, R, V, true>(G, P, coef, h, w, eps, x_base, y0, S, ring);
    else
        k1_slide_segment_t<TG, TP, R, V, false>(G, P, coef, h, w, eps, x_base, y0, S, ring);
}

// ------------------------------------------------------------------- K4
// Algorithm 1 at low resolution for one strip segment, from d Abar, d bbar
// (the K3 gather).  Per window m: the statistics and A; dA = f_mu^T(d Abar)
// and db = f_mu^T(d bbar) as window sums of d Abar / N, d bbar / N; then
//   gamma = (dA - db mu) / (var + eps),  beta = -gamma A,
// and the four window quantities
//   q0 = gamma / N, q1 = beta / N, q2 = (db - gamma mu') / N,
//   q3 = (gamma nu' + 2 beta mu' + db A) / N      (primes: shifted by K),
// whose window sums S0..S3 around a pixel give
//   dP = G' S0 + S2,   dG = P' S0 + 2 G' S1 - S3.
// ring: this warp's second-pass ring, (2R + 1) x 32 x V x 4 floats, then
// its input ring, SlideStage<R, true>::NR rows of G, P and d Abar, d bbar
// (k4_slide_warp_bytes).
template <typename TG, typename TP, int R, int V>
__host__ __device__ constexpr int k4_slide_warp_bytes() {
    return (2 * R + 1) * 32 * V * 16 + SlideStage<R, true>::NR * 32 * V * ((int)sizeof(TG) + (int)sizeof(TP) + 8);
}

template <typename TG, typename TP, typename TD, int R, int V>
__device__ void k4_slide_segment(const TG* __restrict__ G, const TP* __restrict__ P,
                                 const float2* __restrict__ dcoef, TP* __restrict__ dP, TD* __restrict__ dG, int h,
                                 int w, float eps, int x_base, int y0, int S, bool aligned, bool aligned_pairs,
                                 float4* __restrict__ ring) {
    using Gm = SlideGeom<R, V>;
    constexpr int W = Gm::W;
    const int lane = threadIdx.x & 31;
    const SlideLane<R, V> L = slide_lane<R, V>(x_base, w, aligned);
    const bool async = aligned && aligned_pairs;  // every input of the row copies asynchronously
    const int y1 = min(y0 + S, h);
    const int e0 = y0 - 2 * R, nrow = (y1 - y0) + 4 * R;
    float KG, KP;
    {
        float g[V], p[V];
        slide_load<TG, V>(G, y0, h, w, L.x0, L.vec, g);
        slide_load<TP, V>(P, y0, h, w, L.x0, L.vec, p);
        KG = slide_shift<TG, V>(g, L.xin);
        KP = slide_shift<TP, V>(p, L.xin);
    }
    // pairs per column: (G', P'), (G'^2, G'P') and (d Abar / N, d bbar / N)
    // sums of the first pass; (q0, q1), (q2, q3) sums of the second
    f32x2 a1[V], a2[V], a3[V], w01[V], w23[V], xin2[V], nk[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        a1[j] = a2[j] = a3[j] = w01[j] = w23[j] = f2_splat(0.f);
        xin2[j] = f2_splat(L.xin[j]);
        nk[j] = f2_pack(-KG * L.xin[j], -KP * L.xin[j]);
    }
    // input rows through the ring, D rows ahead (the leaving row and the
    // output row are still there)
    constexpr int D = SlideStage<R, true>::D, NR = SlideStage<R, true>::NR;
    constexpr int BG = 32 * V * (int)sizeof(TG), BP = 32 * V * (int)sizeof(TP), BD = 32 * V * 8;
    constexpr int SLOT = BG + BD + BP;  // pairs second, so they stay 16-byte aligned
    unsigned char* rin = reinterpret_cast<unsigned char*>(ring + W * V * 32);
    const int og = lane * V * (int)sizeof(TG), od = BG + lane * V * 8, op = BG + BD + lane * V * (int)sizeof(TP);
    const float* dflat = reinterpret_cast<const float*>(dcoef);
    auto issue = [&](int tt, int slot) {  // row e0 + tt into ring slot `slot`
        unsigned char* sl = rin + slot * SLOT;
        stage_row<TG, V>(sl + og, G, e0 + tt, h, w, L.x0, async);
        stage_row<float, 2 * V>(sl + od, dflat, e0 + tt, h, 2 * w, 2 * L.x0, async);
        stage_row<TP, V>(sl + op, P, e0 + tt, h, w, L.x0, async);
    };
    // a staged row's first-pass terms: (G', P') and (d Abar, d bbar) / N of
    // each pixel's own window
    auto terms = [&](int slot, int e, f32x2 (&sh)[V], f32x2 (&dd)[V]) {
        const unsigned char* sl = rin + slot * SLOT;
        float g[V], p[V], abv[2 * V];
        unstage_row<TG, V>(sl + og, g);
        unstage_row<TP, V>(sl + op, p);
        unstage_row<float, 2 * V>(sl + od, abv);
        const float iny = slide_iny(e, h, R);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            sh[j] = f2x_fma(f2_pack(g[j], p[j]), xin2[j], nk[j]);
            dd[j] = f2x_mul(f2_pack(abv[2 * j], abv[2 * j + 1]), f2_splat(slide_inv<R, V>(L, j, iny)));
        }
    };
#pragma unroll 1
    for (int tt = 0; tt < D; ++tt) {
        if (tt < nrow) issue(tt, tt);
        slide_cp_commit();
    }
    auto wrap = [](int k) { return k + 1 == NR ? 0 : k + 1; };
    int sn = 0, so = NR - W, sc = NR - 2 * R, sf = D;  // ring slots of rows t, t - W, t - 2R and t + D
    int u = 0;
    for (int t = 0; t < nrow; ++t) {
        const int e = e0 + t;
        if (t + D < nrow) issue(t + D, sf);
        slide_cp_commit();
        slide_cp_wait<D>();  // row e (and every older one) has landed
        if (e >= 0 && e < h) {
            f32x2 sh[V], dd[V];
            terms(sn, e, sh, dd);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a1[j] = f2x_add(a1[j], sh[j]);
                a2[j] = f2x_add(a2[j], f2x_mul(f2_splat(f2_lo(sh[j])), sh[j]));
                a3[j] = f2x_add(a3[j], dd[j]);
            }
        }
        const int eo = e - W;
        if (t >= W && eo >= 0 && eo < h) {
            f32x2 sh[V], dd[V];
            terms(so, eo, sh, dd);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a1[j] = f2x_sub(a1[j], sh[j]);
                a2[j] = f2x_sub(a2[j], f2x_mul(f2_splat(f2_lo(sh[j])), sh[j]));
                a3[j] = f2x_sub(a3[j], dd[j]);
            }
        }
        const int sc_now = sc;
        sn = wrap(sn);
        so = wrap(so);
        sc = wrap(sc);
        sf = wrap(sf);
        if (t < 2 * R) continue;  // uniform
        const int c1 = e - R;
        f32x2 s1[V], s2[V], s3[V];
        hbox2<R, V>(a1, s1);
        hbox2<R, V>(a2, s2);
        hbox2<R, V>(a3, s3);
        f32x2 q01[V], q23[V];
        const bool c1in = c1 >= 0 && c1 < h;
        const float iny1 = c1in ? slide_iny(c1, h, R) : 1.f;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const f32x2 inv2 = f2_splat(slide_inv<R, V>(L, j, iny1));
            const f32x2 m = f2x_mul(s1[j], inv2);                    // (mu', nu')
            const f32x2 q = f2x_mul(s2[j], inv2);                    // (E[G'^2], E[G'P'])
            const f32x2 vc = f2x_fma(f2_splat(-f2_lo(m)), m, q);     // (var, cov)
            const float mus = f2_lo(m), nus = f2_hi(m);
            const float ive = rcp_approx(fmaxf(f2_lo(vc), 0.f) + eps);
            const float A = f2_hi(vc) * ive;
            const float dA = f2_lo(s3[j]), db = f2_hi(s3[j]);
            const float gamma = fmaf(-db, mus + KG, dA) * ive;
            const float beta = -gamma * A;
            const bool in = c1in && L.xin[j] != 0.f;
            const f32x2 g01 = f2x_mul(f2_pack(gamma, beta), inv2);
            const f32x2 g23 = f2x_mul(f2_pack(fmaf(-gamma, mus, db), fmaf(gamma, nus, fmaf(2.f * beta, mus, db * A))),
                                      inv2);
            q01[j] = in ? g01 : f2_splat(0.f);
            q23[j] = in ? g23 : f2_splat(0.f);
        }
        float4* slot = ring + (size_t)u * V * 32 + lane;
        if (t - 2 * R >= W) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float4 o = slot[j * 32];
                w01[j] = f2x_sub(f2x_add(w01[j], q01[j]), f2_pack(o.x, o.y));
                w23[j] = f2x_sub(f2x_add(w23[j], q23[j]), f2_pack(o.z, o.w));
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                w01[j] = f2x_add(w01[j], q01[j]);
                w23[j] = f2x_add(w23[j], q23[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float x0, x1, x2, x3;
            f2_unpack(q01[j], x0, x1);
            f2_unpack(q23[j], x2, x3);
            slot[j * 32] = make_float4(x0, x1, x2, x3);
        }
        u = (u + 1 == W) ? 0 : u + 1;
        if (t < 4 * R) continue;  // uniform
        f32x2 S01[V], S23[V];
        hbox2<R, V>(w01, S01);
        hbox2<R, V>(w23, S23);
        if (L.out) {
            const int c2 = e - 2 * R;
            const unsigned char* sl = rin + sc_now * SLOT;  // row c2 = e - 2R
            float gc[V], pc[V];
            unstage_row<TG, V>(sl + og, gc);
            unstage_row<TP, V>(sl + op, pc);
            float outp[V], outg[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float gs = gc[j] - KG, ps = pc[j] - KP;
                float S0, S1, S2, S3;
                f2_unpack(S01[j], S0, S1);
                f2_unpack(S23[j], S2, S3);
                f2_unpack(f2x_fma(f2_pack(gs, ps), f2_splat(S0), f2_pack(S2, fmaf(2.f * gs, S1, -S3))), outp[j],
                          outg[j]);
            }
            const size_t o = (size_t)c2 * w + L.x0;
            if (L.vec) {
                if (dP != nullptr) store_vec<TP, V>(dP + o, outp);
                if (dG != nullptr) store_vec<TD, V>(dG + o, outg);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    if (L.x0 + j < w) {
                        if (dP != nullptr) dP[o + j] = from_f32<TP>(outp[j]);
                        if (dG != nullptr) dG[o + j] = from_f32<TD>(outg[j]);
                    }
                }
            }
        }
    }
    slide_cp_wait<0>();  // the last groups are empty; nothing is left in flight
}

}  // namespace dgf
