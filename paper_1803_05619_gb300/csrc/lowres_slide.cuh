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

// Radius-R horizontal window sums of a row held V columns per lane:
// out[j] = sum over k in [-R, R] of x at lane column j + k.  Lanes reach
// their neighbours by shuffles; results are meaningful for strip columns
// [R, 32 V - R) only (the others read across the warp's edge).
template <int R, int V>
__device__ __forceinline__ void hbox(const float (&x)[V], float (&out)[V]) {
    float T[V + 2 * R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int o = -R + k;                   // column offset left of the lane
        const int dl = -((-o + V - 1) / V);     // source lane offset (negative)
        const int j = o - dl * V;               // column inside the source lane
        T[k] = __shfl_up_sync(0xffffffffu, x[j], -dl);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) T[R + j] = x[j];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int o = V + k;
        T[R + V + k] = __shfl_down_sync(0xffffffffu, x[o % V], o / V);
    }
    float s = T[0];
#pragma unroll
    for (int k = 1; k <= 2 * R; ++k) s += T[k];
    out[0] = s;
#pragma unroll
    for (int j = 1; j < V; ++j) {
        s = (s + T[j + 2 * R]) - T[j - 1];
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

// d Abar, d bbar of row e at the lane's columns (zero outside the image).
template <int V>
__device__ __forceinline__ void slide_load_pairs(const float2* __restrict__ src, int e, int h, int w, int x0,
                                                 bool vec, float (&a)[V], float (&b)[V]) {
    if (e < 0 || e >= h) {
#pragma unroll
        for (int j = 0; j < V; ++j) a[j] = b[j] = 0.f;
        return;
    }
    const float2* row = src + (size_t)e * w;
    if (vec) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float4 q = *reinterpret_cast<const float4*>(row + x0 + j);
            a[j] = q.x;
            b[j] = q.y;
            a[j + 1] = q.z;
            b[j + 1] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int x = x0 + j;
            const float2 q = (x >= 0 && x < w) ? row[x] : make_float2(0.f, 0.f);
            a[j] = q.x;
            b[j] = q.y;
        }
    }
}

// Per-lane column facts.
template <int R, int V>
struct SlideLane {
    float nx[V];     // clipped window width of each column (1 outside the image)
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
        L.col_int = L.col_int && n == 2 * R + 1;
    }
    L.out = lane * V >= Gm::HB && lane * V < Gm::HB + Gm::OUTC;
    L.vec = aligned && L.x0 >= 0 && L.x0 + V <= w;
    return L;
}

__device__ __forceinline__ int slide_ny(int y, int h, int R) { return min(y + R, h - 1) - max(y - R, 0) + 1; }

// 1 / (window count) for a window of ny rows at column j: a compile-time
// constant for full windows, else the correctly rounded reciprocal.
template <int R, int V>
__device__ __forceinline__ float slide_inv(const SlideLane<R, V>& L, int j, int ny) {
    constexpr int W = 2 * R + 1;
    constexpr float kInvW2 = 1.f / (float)(W * W);
    if (L.col_int && ny == W) return kInvW2;
    return __frcp_rn(L.nx[j] * (float)ny);
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
__device__ __forceinline__ void cp_async_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES),
                     "r"(src_bytes)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
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
            cp_async_zfill<CH>(d + c * CH, reinterpret_cast<const char*>(p) + c * CH, in ? CH : 0);
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

template <typename TG, typename TP, int R, int V>
__device__ void k1_slide_segment(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                                 int h, int w, float eps, int x_base, int y0, int S, bool aligned,
                                 float4* __restrict__ ring) {
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
    float vg[V], vp[V], vgg[V], vgp[V], va[V], vb[V];
#pragma unroll
    for (int j = 0; j < V; ++j) vg[j] = vp[j] = vgg[j] = vgp[j] = va[j] = vb[j] = 0.f;
    // input rows through the ring, D rows ahead (the leaving row is still there)
    constexpr int D = SlideStage<R>::D, NR = SlideStage<R>::NR;
    constexpr int SLOT = 32 * V * ((int)sizeof(TG) + (int)sizeof(TP));
    unsigned char* rin = reinterpret_cast<unsigned char*>(ring + W * (V / 2) * 32);
    const int og = lane * V * (int)sizeof(TG), op = 32 * V * (int)sizeof(TG) + lane * V * (int)sizeof(TP);
    auto issue = [&](int tt) {  // row e0 + tt into its slot
        unsigned char* sl = rin + (tt % NR) * SLOT;
        stage_row<TG, V>(sl + og, G, e0 + tt, h, w, L.x0, aligned);
        stage_row<TP, V>(sl + op, P, e0 + tt, h, w, L.x0, aligned);
    };
#pragma unroll 1
    for (int tt = 0; tt < D; ++tt) {
        if (tt < nrow) issue(tt);
        cp_async_commit();
    }
    int u = 0;  // ring slot of the second pass's newest row
    for (int t = 0; t < nrow; ++t) {
        const int e = e0 + t;
        if (t + D < nrow) issue(t + D);
        cp_async_commit();
        cp_async_wait<D>();  // row e (and every older one) has landed
        float g[V], p[V], go[V], po[V];
        {
            const unsigned char* sl = rin + (t % NR) * SLOT;
            unstage_row<TG, V>(sl + og, g);
            unstage_row<TP, V>(sl + op, p);
        }
        // first pass, vertical: add row e
        const bool ein = e >= 0 && e < h;
        if (ein) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float gs = (g[j] - KG) * L.xin[j], ps = (p[j] - KP) * L.xin[j];
                vg[j] += gs;
                vp[j] += ps;
                vgg[j] += gs * gs;
                vgp[j] += gs * ps;
            }
        }
        // ... and subtract row e - W (zero when outside the image or before the walk)
        const int eo = e - W;
        if (t >= W && eo >= 0 && eo < h) {
            const unsigned char* sl = rin + ((t - W) % NR) * SLOT;
            unstage_row<TG, V>(sl + og, go);
            unstage_row<TP, V>(sl + op, po);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float gs = (go[j] - KG) * L.xin[j], ps = (po[j] - KP) * L.xin[j];
                vg[j] -= gs;
                vp[j] -= ps;
                vgg[j] -= gs * gs;
                vgp[j] -= gs * ps;
            }
        }
        if (t < 2 * R) continue;  // uniform: the first pass's sums are not full yet
        // first pass, horizontal, at window row c1 = e - R: statistics -> A, b
        const int c1 = e - R;
        float sg[V], sp[V], sgg[V], sgp[V];
        hbox<R, V>(vg, sg);
        hbox<R, V>(vp, sp);
        hbox<R, V>(vgg, sgg);
        hbox<R, V>(vgp, sgp);
        float A[V], B[V];
        const bool c1in = c1 >= 0 && c1 < h;
        const int ny1 = c1in ? slide_ny(c1, h, R) : 1;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const float inv = slide_inv<R, V>(L, j, ny1);
            const float mu = sg[j] * inv, nu = sp[j] * inv;
            const float var = fmaxf(fmaf(-mu, mu, sgg[j] * inv), 0.f);
            const float cov = fmaf(-mu, nu, sgp[j] * inv);
            const float a = cov * rcp_approx(var + eps);
            const float b = fmaf(-a, mu + KG, nu + KP);
            const bool in = c1in && L.xin[j] != 0.f;
            A[j] = in ? a : 0.f;
            B[j] = in ? b : 0.f;
        }
        // second pass, vertical: add row c1, subtract row c1 - W from the ring
        float4* slot = ring + (size_t)u * (V / 2) * 32 + lane;
        if (t - 2 * R >= W) {
#pragma unroll
            for (int j = 0; j < V; j += 2) {
                const float4 o = slot[(j / 2) * 32];
                va[j] = (va[j] + A[j]) - o.x;
                vb[j] = (vb[j] + B[j]) - o.y;
                va[j + 1] = (va[j + 1] + A[j + 1]) - o.z;
                vb[j + 1] = (vb[j + 1] + B[j + 1]) - o.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                va[j] += A[j];
                vb[j] += B[j];
            }
        }
#pragma unroll
        for (int j = 0; j < V; j += 2) slot[(j / 2) * 32] = make_float4(A[j], B[j], A[j + 1], B[j + 1]);
        u = (u + 1 == W) ? 0 : u + 1;
        if (t < 4 * R) continue;  // uniform: the second pass's sums are not full yet
        // second pass, horizontal, at output row c2 = e - 2R
        const int c2 = e - 2 * R;
        float sa[V], sb[V];
        hbox<R, V>(va, sa);
        hbox<R, V>(vb, sb);
        if (L.out) {
            const int ny2 = slide_ny(c2, h, R);
            float2* orow = coef + (size_t)c2 * w;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = L.x0 + j;
                if (x < w) {
                    const float inv = slide_inv<R, V>(L, j, ny2);
                    orow[x] = make_float2(sa[j] * inv, sb[j] * inv);
                }
            }
        }
    }
    cp_async_wait<0>();  // the last groups are empty; nothing is left in flight
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
    float vg[V], vp[V], vgg[V], vgp[V], vda[V], vdb[V], w0[V], w1[V], w2[V], w3[V];
#pragma unroll
    for (int j = 0; j < V; ++j) vg[j] = vp[j] = vgg[j] = vgp[j] = vda[j] = vdb[j] = w0[j] = w1[j] = w2[j] = w3[j] = 0.f;
    // the first pass's terms of row e at the lane's columns (zero outside),
    // from its raw values
    auto terms = [&](int e, const float (&g)[V], const float (&p)[V], float (&gs)[V], float (&ps)[V],
                     float (&da)[V], float (&db)[V]) {
        const int ny = slide_ny(e, h, R);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            gs[j] = (g[j] - KG) * L.xin[j];
            ps[j] = (p[j] - KP) * L.xin[j];
            const float inv = slide_inv<R, V>(L, j, ny);
            da[j] *= inv;
            db[j] *= inv;
        }
    };
    // input rows through the ring, D rows ahead (the leaving row and the
    // output row are still there)
    constexpr int D = SlideStage<R, true>::D, NR = SlideStage<R, true>::NR;
    constexpr int BG = 32 * V * (int)sizeof(TG), BP = 32 * V * (int)sizeof(TP), BD = 32 * V * 8;
    constexpr int SLOT = BG + BD + BP;  // pairs second, so they stay 16-byte aligned
    unsigned char* rin = reinterpret_cast<unsigned char*>(ring + W * V * 32);
    const int og = lane * V * (int)sizeof(TG), od = BG + lane * V * 8, op = BG + BD + lane * V * (int)sizeof(TP);
    const float* dflat = reinterpret_cast<const float*>(dcoef);
    auto issue = [&](int tt) {  // row e0 + tt into its slot
        unsigned char* sl = rin + (tt % NR) * SLOT;
        stage_row<TG, V>(sl + og, G, e0 + tt, h, w, L.x0, async);
        stage_row<float, 2 * V>(sl + od, dflat, e0 + tt, h, 2 * w, 2 * L.x0, async);
        stage_row<TP, V>(sl + op, P, e0 + tt, h, w, L.x0, async);
    };
    auto unstage = [&](int tt, float (&g)[V], float (&p)[V], float (&da)[V], float (&db)[V]) {
        const unsigned char* sl = rin + (tt % NR) * SLOT;
        unstage_row<TG, V>(sl + og, g);
        unstage_row<TP, V>(sl + op, p);
        float ab[2 * V];
        unstage_row<float, 2 * V>(sl + od, ab);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            da[j] = ab[2 * j];
            db[j] = ab[2 * j + 1];
        }
    };
#pragma unroll 1
    for (int tt = 0; tt < D; ++tt) {
        if (tt < nrow) issue(tt);
        cp_async_commit();
    }
    int u = 0;
    for (int t = 0; t < nrow; ++t) {
        const int e = e0 + t;
        if (t + D < nrow) issue(t + D);
        cp_async_commit();
        cp_async_wait<D>();  // row e (and every older one) has landed
        float g[V], p[V], da[V], db[V];
        unstage(t, g, p, da, db);
        if (e >= 0 && e < h) {
            float gs[V], ps[V];
            terms(e, g, p, gs, ps, da, db);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                vg[j] += gs[j];
                vp[j] += ps[j];
                vgg[j] += gs[j] * gs[j];
                vgp[j] += gs[j] * ps[j];
                vda[j] += da[j];
                vdb[j] += db[j];
            }
        }
        const int eo = e - W;
        if (t >= W && eo >= 0 && eo < h) {
            float go[V], po[V], ao[V], bo[V], gs[V], ps[V];
            unstage(t - W, go, po, ao, bo);
            terms(eo, go, po, gs, ps, ao, bo);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                vg[j] -= gs[j];
                vp[j] -= ps[j];
                vgg[j] -= gs[j] * gs[j];
                vgp[j] -= gs[j] * ps[j];
                vda[j] -= ao[j];
                vdb[j] -= bo[j];
            }
        }
        if (t < 2 * R) continue;  // uniform
        const int c1 = e - R;
        float sg[V], sp[V], sgg[V], sgp[V], sda[V], sdb[V];
        hbox<R, V>(vg, sg);
        hbox<R, V>(vp, sp);
        hbox<R, V>(vgg, sgg);
        hbox<R, V>(vgp, sgp);
        hbox<R, V>(vda, sda);
        hbox<R, V>(vdb, sdb);
        float q0[V], q1[V], q2[V], q3[V];
        const bool c1in = c1 >= 0 && c1 < h;
        const int ny1 = c1in ? slide_ny(c1, h, R) : 1;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const float inv = slide_inv<R, V>(L, j, ny1);
            const float mus = sg[j] * inv, nus = sp[j] * inv;
            const float var = fmaxf(fmaf(-mus, mus, sgg[j] * inv), 0.f);
            const float cov = fmaf(-mus, nus, sgp[j] * inv);
            const float ive = rcp_approx(var + eps);
            const float A = cov * ive;
            const float dA = sda[j], db = sdb[j];
            const float gamma = fmaf(-db, mus + KG, dA) * ive;
            const float beta = -gamma * A;
            const bool in = c1in && L.xin[j] != 0.f;
            q0[j] = in ? gamma * inv : 0.f;
            q1[j] = in ? beta * inv : 0.f;
            q2[j] = in ? fmaf(-gamma, mus, db) * inv : 0.f;
            q3[j] = in ? fmaf(gamma, nus, fmaf(2.f * beta, mus, db * A)) * inv : 0.f;
        }
        float4* slot = ring + (size_t)u * V * 32 + lane;
        if (t - 2 * R >= W) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float4 o = slot[j * 32];
                w0[j] = (w0[j] + q0[j]) - o.x;
                w1[j] = (w1[j] + q1[j]) - o.y;
                w2[j] = (w2[j] + q2[j]) - o.z;
                w3[j] = (w3[j] + q3[j]) - o.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                w0[j] += q0[j];
                w1[j] += q1[j];
                w2[j] += q2[j];
                w3[j] += q3[j];
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) slot[j * 32] = make_float4(q0[j], q1[j], q2[j], q3[j]);
        u = (u + 1 == W) ? 0 : u + 1;
        if (t < 4 * R) continue;  // uniform
        const int c2 = e - 2 * R;
        float S0[V], S1[V], S2[V], S3[V];
        hbox<R, V>(w0, S0);
        hbox<R, V>(w1, S1);
        hbox<R, V>(w2, S2);
        hbox<R, V>(w3, S3);
        if (L.out) {
            float gc[V], pc[V];
            {
                const unsigned char* sl = rin + ((t - 2 * R) % NR) * SLOT;  // row c2
                unstage_row<TG, V>(sl + og, gc);
                unstage_row<TP, V>(sl + op, pc);
            }
            float outp[V], outg[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float gs = gc[j] - KG, ps = pc[j] - KP;
                outp[j] = fmaf(gs, S0[j], S2[j]);
                outg[j] = fmaf(ps, S0[j], fmaf(2.f * gs, S1[j], -S3[j]));
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
    cp_async_wait<0>();  // the last groups are empty; nothing is left in flight
}

}  // namespace dgf
