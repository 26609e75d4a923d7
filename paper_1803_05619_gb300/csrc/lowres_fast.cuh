// Low-resolution stage, column-walking form for radius R known at compile
// time (R = 1, 2, 4, 8).
//
// A CTA owns a tile whose coefficient region E1 is CW columns x EY1 rows
// (outputs: (CW - 2R) x (EY1 - 2R)); its inputs E2 (E1 plus an R ring) are
// staged once in shared memory.  Threads are laid out as CW columns x
// (256 / CW) row groups.  Each thread owns one column and walks down its
// rows: at every row it forms the horizontal window quantity of that row
// from shared memory (2R + 1 reads), keeps the last 2R + 1 of them in a
// register ring, and emits the vertical window result for the row R above.
// The walk is unrolled by 2R + 1 so every ring slot is a fixed register.
// No integer division runs per element and every pass is one walk.
//
// Statistics are centred exactly: each row segment is centred on its own
// mean, and segments are combined with Chan's pairwise update (every term
// is a square or a product of deviations), so var and cov carry no
// E[x^2] - E[x]^2 cancellation.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace dgf {

constexpr int kLowThreads = 256;

// Per window m the backward needs four window sums over the windows that
// contain each pixel i (all divided by N_m; G' = G - K_G, P' = P - K_P,
// mu' = mu - K_G, nu' = nu - K_P for the tile shift K):
//   q0 = gamma, q1 = beta, q2 = db - gamma mu', q3 = gamma nu' + 2 beta mu' + db A,
// and then dP_i = G'_i S0 + S2,  dG_i = P'_i S0 + 2 G'_i S1 - S3,
// the regrouping of sum_m [gamma (G_i - mu) + db] / N_m and
// sum_m [gamma (P_i - nu) + 2 beta (G_i - mu) - db A] / N_m.
constexpr int kNQ = 4;

// The ring form (r <= 2) keeps the centred differences exact instead: per
// window it stores gamma~, beta~, mu, nu, db~ and (db A)~ (six planes) and
// forms gamma~ (G_i - mu_m) etc. per pixel, so large gamma in flat regions
// cannot cancel catastrophically.
constexpr int kNQD = 6;

__host__ __device__ inline int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

struct FastTile {
    int h, w;          // plane size
    int CW, EY1;       // coefficient region (columns, rows)
    int log2cw;        // CW = 1 << log2cw
    int tx0, ty0;      // output tile origin
    int TX, TY;        // output tile size
    float eps;
};

__device__ __forceinline__ int seg_count(int c, int n, int R) {
    return min(c + R, n - 1) - max(c - R, 0) + 1;
}

// Stage the E2 region (EY1 + 2R rows x CW + 2R columns) of one plane, FP32,
// zero outside the image.  Row-major, pitch EX2.
template <typename T, int R, bool INT = false>
__device__ __forceinline__ void fast_stage(const T* __restrict__ src, float* dst, const FastTile& t) {
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R;
    const int gx0 = t.tx0 - 2 * R, gy0 = t.ty0 - 2 * R;
    auto ld = [&](int e, int k) -> float {
        const int gy = gy0 + e, gx = gx0 + k;
        if (INT || (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w)) return to_f32<T>(src[(size_t)gy * t.w + gx]);
        return 0.f;
    };
    // columns [0, CW): flat index with shifts; 8 loads in flight per thread
    const int n = EY2 << t.log2cw;
    for (int base = threadIdx.x; base < n; base += 8 * kLowThreads) {
        float v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int idx = base + b * kLowThreads;
            if (idx < n) v[b] = ld(idx >> t.log2cw, idx & (t.CW - 1));
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int idx = base + b * kLowThreads;
            if (idx < n) dst[(idx >> t.log2cw) * EX2 + (idx & (t.CW - 1))] = v[b];
        }
    }
    // columns [CW, CW + 2R)
    constexpr int S = 2 * R;
    const int m = EY2 * S;
    for (int idx = threadIdx.x; idx < m; idx += kLowThreads) {
        const int e = idx / S, k = t.CW + idx % S;
        dst[e * EX2 + k] = ld(e, k);
    }
}

// TMA variant: the box starts at the 16-byte boundary at or left of the
// region's first column; `off` (per tile) skips the extra columns.
template <typename TA, typename TB, int R>
__device__ bool fast_stage_tma(const TmaPlane* ta, const TmaPlane* tb, int plane, const FastTile& t,
                               float* sA, float* sB, char* landing, uint32_t* status) {
    __shared__ __align__(8) uint64_t bar;
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R;
    const int xl = t.tx0 - 2 * R, yl = t.ty0 - 2 * R;
    const int ua = 16 / (int)sizeof(TA), ub = 16 / (int)sizeof(TB);
    const int offa = ((xl % ua) + ua) % ua, offb = ((xl % ub) + ub) % ub;
    char* la = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(landing) + 127) & ~uintptr_t(127));
    const uint32_t bytes_a = (uint32_t)(ta->bx * ta->by * (int)sizeof(TA));
    const uint32_t bytes_b = (uint32_t)(tb->bx * tb->by * (int)sizeof(TB));
    char* lb = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(la + bytes_a) + 127) & ~uintptr_t(127));
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes_a + bytes_b)
                     : "memory");
        tma_load_3d(smem_u32(la), &ta->map, xl - offa, yl, plane, b);
        tma_load_3d(smem_u32(lb), &tb->map, xl - offb, yl, plane, b);
    }
    __syncthreads();
    bool ok = mbar_wait(b, 0, first_wait_limit(status));
    if (!ok) {
        status_fail(status, kStatusTimeout);
        mbar_wait(b, 0, kWaitLimit);  // the copies land before the buffers are reused
    }
    ok = __syncthreads_and(ok) != 0;  // one decision for the whole CTA
    if (ok) {
        const TA* pa = reinterpret_cast<const TA*>(la);
        const TB* pb = reinterpret_cast<const TB*>(lb);
        const int cw = t.CW;
        const int c0 = threadIdx.x & (cw - 1), r0 = threadIdx.x >> t.log2cw, rstep = kLowThreads >> t.log2cw;
        for (int e = r0; e < EY2; e += rstep)
            for (int k = c0; k < EX2; k += cw) {
                sA[e * EX2 + k] = to_f32<TA>(pa[e * ta->bx + k + offa]);
                sB[e * EX2 + k] = to_f32<TB>(pb[e * tb->bx + k + offb]);
            }
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
    return ok;
}

// Row statistics of one E2 row at this thread's E1 column: segment mean and
// centred sums over the 2R + 1 columns (masked to the image).
template <int R>
__device__ __forceinline__ void fast_row_stats(const float* g, const float* p, const float (&mk)[2 * R + 1],
                                               float inx, float& mg, float& mp, float& sgg, float& sgp) {
    float gv[2 * R + 1], pv[2 * R + 1];
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        gv[k] = g[k];
        pv[k] = p[k];
        s1 += gv[k];
        s2 += pv[k];
    }
    mg = s1 * inx;
    mp = s2 * inx;
    float a = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        const float dg = mk[k] * (gv[k] - mg);
        a = fmaf(dg, dg, a);
        c = fmaf(dg, pv[k] - mp, c);
    }
    sgg = a;
    sgp = c;
}

// Window moments of E1 row e1 from the ring (all 2R + 1 slots), Chan's update.
// U: slot of the newest row; the slots are summed oldest first, so the
// rounding does not depend on where the walk started.
template <int R>
__device__ __forceinline__ void fast_window(const float (&mg)[2 * R + 1], const float (&mp)[2 * R + 1],
                                            const float (&sgg)[2 * R + 1], const float (&sgp)[2 * R + 1],
                                            const float (&vr)[2 * R + 1], int U, float nx, float iny, float inn,
                                            float& mu, float& nu, float& var, float& cov) {
    constexpr int W = 2 * R + 1;
    float s1 = 0.f, s2 = 0.f, a = 0.f, c = 0.f;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int k = (U + 1 + j) % W;
        s1 += mg[k];
        s2 += mp[k];
        a += sgg[k];
        c += sgp[k];
    }
    mu = s1 * iny;
    nu = s2 * iny;
    float dgg = 0.f, dgp = 0.f;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int k = (U + 1 + j) % W;
        const float dg = vr[k] * (mg[k] - mu);
        dgg = fmaf(dg, dg, dgg);
        dgp = fmaf(dg, mp[k] - nu, dgp);
    }
    var = fmaf(nx, dgg, a) * inn;
    cov = fmaf(nx, dgp, c) * inn;
}

// ------------------------------------------------------------------- K1
// Eq. 1's least-squares A, b per window (Sec. 3.2), then their box mean.
// smem: sG, sP (E2), sA, sB (E1); TMA landing (if used) overlaps sA, sB
// plus `extra` bytes after them.
template <typename TG, typename TP, int R, bool INT>
__device__ void coef_tile_ring(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                               const FastTile& t, float* smem, const TmaPlane* tg, const TmaPlane* tp,
                               int plane, uint32_t* status) {
    constexpr int W = 2 * R + 1;
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R, EX1 = t.CW;
    float* sG = smem;
    float* sP = sG + EX2 * EY2;
    float* sA = sP + EX2 * EY2;
    float* sB = sA + EX1 * t.EY1;
    bool staged = false;
    if (tg != nullptr && tp != nullptr)
        staged = fast_stage_tma<TG, TP, R>(tg, tp, plane, t, sG, sP, reinterpret_cast<char*>(sA), status);
    if (!staged) {
        fast_stage<TG, R, INT>(G, sG, t);
        fast_stage<TP, R, INT>(P, sP, t);
        __syncthreads();
    }
    const int c = threadIdx.x & (t.CW - 1), rg = threadIdx.x >> t.log2cw;
    const int ngroups = kLowThreads >> t.log2cw;
    // ---- pass A: E1 column c, E1 rows [ra, rb)
    {
        const int gx = t.tx0 - R + c;
        const bool colin = INT || (gx >= 0 && gx < t.w);
        float mk[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int x = gx - R + k;
            mk[k] = (INT || (x >= 0 && x < t.w)) ? 1.f : 0.f;
        }
        const float nx = INT ? (float)W : (colin ? (float)seg_count(gx, t.w, R) : 1.f);
        const float inx = INT ? 1.f / (float)W : inv_countf(nx);
        const int ra = (rg * t.EY1) / ngroups, rb = ((rg + 1) * t.EY1) / ngroups;
        float mg[W], mp[W], sgg[W], sgp[W], vr[W];
        // warm-up: E2 rows ra .. ra + 2R - 1 into slots 0 .. 2R - 1
#pragma unroll
        for (int s = 0; s < 2 * R; ++s) {
            const int e = ra + s;
            fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg[s], mp[s], sgg[s], sgp[s]);
            const int gy = t.ty0 - 2 * R + e;
            vr[s] = (INT || (gy >= 0 && gy < t.h)) ? 1.f : 0.f;
        }
        for (int base = ra; base < rb; base += W) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int e1 = base + s;
                if (e1 < rb) {
                    constexpr int dummy = 0;
                    (void)dummy;
                    const int slot = (s + 2 * R) % W;
                    const int e = e1 + 2 * R;
                    fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg[slot], mp[slot],
                                      sgg[slot], sgp[slot]);
                    const int gye = t.ty0 - 2 * R + e;
                    vr[slot] = (INT || (gye >= 0 && gye < t.h)) ? 1.f : 0.f;
                    const int gy = t.ty0 - R + e1;
                    float A = 0.f, b = 0.f;
                    if (INT || (colin && gy >= 0 && gy < t.h)) {
                        float mu, nu, var, cov;
                        const float ny = INT ? (float)W : (float)seg_count(gy, t.h, R);
                        const float iny = INT ? 1.f / (float)W : inv_countf(ny);
                        const float inn = INT ? 1.f / (float)(W * W) : inv_countf(nx * ny);
                        fast_window<R>(mg, mp, sgg, sgp, vr, slot, nx, iny, inn, mu, nu, var, cov);
                        A = cov * rcp_approx(var + t.eps);
                        b = fmaf(-A, mu, nu);
                    }
                    sA[e1 * EX1 + c] = A;
                    sB[e1 * EX1 + c] = b;
                }
            }
        }
    }
    __syncthreads();
    // ---- pass B: output column c < TX, output rows [ya, yb): box mean of A, b
    if (c < t.TX) {
        const int gx = t.tx0 + c;
        const int ya = (rg * t.TY) / ngroups, yb = ((rg + 1) * t.TY) / ngroups;
        const float nx = INT ? (float)W : ((gx < t.w) ? (float)seg_count(gx, t.w, R) : 1.f);
        float ha[W], hb[W];
#pragma unroll
        for (int s = 0; s < 2 * R; ++s) {
            const float* pa = sA + (ya + s) * EX1 + c;
            const float* pb = sB + (ya + s) * EX1 + c;
            float a = 0.f, bb = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                a += pa[k];
                bb += pb[k];
            }
            ha[s] = a;
            hb[s] = bb;
        }
        for (int base = ya; base < yb; base += W) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int y = base + s;
                if (y < yb) {
                    const int slot = (s + 2 * R) % W;
                    const float* pa = sA + (y + 2 * R) * EX1 + c;
                    const float* pb = sB + (y + 2 * R) * EX1 + c;
                    float a = 0.f, bb = 0.f;
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        a += pa[k];
                        bb += pb[k];
                    }
                    ha[slot] = a;
                    hb[slot] = bb;
                    const int gy = t.ty0 + y;
                    if (INT || (gx < t.w && gy < t.h)) {
                        float sa = 0.f, sb = 0.f;
#pragma unroll
                        for (int j = 0; j < W; ++j) {  // oldest row first
                            sa += ha[(slot + 1 + j) % W];
                            sb += hb[(slot + 1 + j) % W];
                        }
                        const float inn = INT ? 1.f / (float)(W * W) : inv_countf(nx * (float)seg_count(gy, t.h, R));
                        coef[(size_t)gy * t.w + gx] = make_float2(sa * inn, sb * inn);
                    }
                }
            }
        }
    }
    __syncthreads();
}

// Stage G, P and d Abar / N, d bbar / N (E2, zero outside the image), and
// compute the tile shift K = mean of the in-image output pixels.
template <typename TG, typename TP, int R, bool INT = false, bool SHIFT = true>
__device__ __forceinline__ void bwd_stage_and_shift(const TG* __restrict__ G, const TP* __restrict__ P,
                                                    const float2* __restrict__ dcoef, const FastTile& t, float* sG,
                                                    float* sP, float* sDA, float* sDB, float* red, float& KG_out,
                                                    float& KP_out) {
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R;
    fast_stage<TG, R, INT>(G, sG, t);
    fast_stage<TP, R, INT>(P, sP, t);
    {
        // d Abar / N, d bbar / N over E2 (zero outside the image), 8 loads in flight per thread
        const int gx0 = t.tx0 - 2 * R, gy0 = t.ty0 - 2 * R;
        auto ld = [&](int e, int k) -> float2 {
            const int gy = gy0 + e, gx = gx0 + k;
            if (INT || (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w)) {
                const float2 v = dcoef[(size_t)gy * t.w + gx];
                const float inn = INT ? 1.f / (float)((2 * R + 1) * (2 * R + 1))
                                      : inv_countf((float)seg_count(gy, t.h, R) * (float)seg_count(gx, t.w, R));
                return make_float2(v.x * inn, v.y * inn);
            }
            return make_float2(0.f, 0.f);
        };
        const int n = EY2 << t.log2cw;
        for (int base = threadIdx.x; base < n; base += 8 * kLowThreads) {
            float2 v[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int idx = base + b * kLowThreads;
                if (idx < n) v[b] = ld(idx >> t.log2cw, idx & (t.CW - 1));
            }
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int idx = base + b * kLowThreads;
                if (idx < n) {
                    const int o = (idx >> t.log2cw) * EX2 + (idx & (t.CW - 1));
                    sDA[o] = v[b].x;
                    sDB[o] = v[b].y;
                }
            }
        }
        constexpr int S = 2 * R;
        const int m = EY2 * S;
        for (int idx = threadIdx.x; idx < m; idx += kLowThreads) {
            const int e = idx / S, k = t.CW + idx % S;
            const float2 v = ld(e, k);
            sDA[e * EX2 + k] = v.x;
            sDB[e * EX2 + k] = v.y;
        }
    }
    __syncthreads();
    // tile shift K = mean of the in-image output pixels (conditioning only)
    float KG = 0.f, KP = 0.f;
    if (SHIFT) {
        float sg = 0.f, sp = 0.f, cn = 0.f;
        const int cw = t.CW;
        const int c0 = threadIdx.x & (cw - 1), r0 = threadIdx.x >> t.log2cw, rstep = kLowThreads >> t.log2cw;
        for (int y = r0; y < t.TY; y += rstep)
            if (c0 < t.TX && (INT || (t.ty0 + y < t.h && t.tx0 + c0 < t.w))) {
                const int o = (y + 2 * R) * EX2 + c0 + 2 * R;
                sg += sG[o];
                sp += sP[o];
                cn += 1.f;
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sg += __shfl_down_sync(0xffffffffu, sg, off);
            sp += __shfl_down_sync(0xffffffffu, sp, off);
            cn += __shfl_down_sync(0xffffffffu, cn, off);
        }
        if ((threadIdx.x & 31) == 0) {
            red[(threadIdx.x >> 5) * 3 + 0] = sg;
            red[(threadIdx.x >> 5) * 3 + 1] = sp;
            red[(threadIdx.x >> 5) * 3 + 2] = cn;
        }
        __syncthreads();
        sg = sp = cn = 0.f;
        for (int k = 0; k < kLowThreads / 32; ++k) {
            sg += red[k * 3 + 0];
            sp += red[k * 3 + 1];
            cn += red[k * 3 + 2];
        }
        if (cn > 0.f) {
            KG = sg / cn;
            KP = sp / cn;
        }
    }
    KG_out = KG;
    KP_out = KP;
}

// ------------------------------------------------------------------- K4
// Algorithm 1 at low resolution (see lowres.cu for the derivation):
// pass A forms, per window m of E1, the statistics, dA = f_mu^T(d Abar),
// db = f_mu^T(d bbar), gamma = (dA - db mu)/(var + eps), beta = -gamma A,
// and the seven quantities whose window sums give dP and dG; pass B sums
// them over the windows containing each output pixel.
// smem: sG, sP, sDA, sDB (E2), sQ (4 x E1), red (3 x warps).
template <typename TG, typename TP, typename TD, int R, bool INT>
__device__ void lowres_bwd_tile_ring(const TG* __restrict__ G, const TP* __restrict__ P,
                                     const float2* __restrict__ dcoef, TP* __restrict__ dP, TD* __restrict__ dG,
                                     const FastTile& t, float* smem) {
    constexpr int W = 2 * R + 1;
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R, EX1 = t.CW, n1 = t.CW * t.EY1;
    float* sG = smem;
    float* sP = sG + EX2 * EY2;
    float* sDA = sP + EX2 * EY2;
    float* sDB = sDA + EX2 * EY2;
    float* sQ = sDB + EX2 * EY2;
    float* red = sQ + (R == 1 ? kNQD : kNQ) * n1;
    // r = 1: every difference G_i - mu_m is formed exactly (9 windows per pixel);
    // r = 2: the four separable window sums, with G and P shifted by the tile mean
    constexpr bool DIRECT = (R == 1);
    constexpr int NQ = DIRECT ? kNQD : kNQ;
    float KG, KP;
    bwd_stage_and_shift<TG, TP, R, INT, !DIRECT>(G, P, dcoef, t, sG, sP, sDA, sDB, red, KG, KP);
    const int c = threadIdx.x & (t.CW - 1), rg = threadIdx.x >> t.log2cw;
    const int ngroups = kLowThreads >> t.log2cw;
    // ---- pass A
    {
        const int gx = t.tx0 - R + c;
        const bool colin = INT || (gx >= 0 && gx < t.w);
        float mk[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int x = gx - R + k;
            mk[k] = (INT || (x >= 0 && x < t.w)) ? 1.f : 0.f;
        }
        const float nx = INT ? (float)W : (colin ? (float)seg_count(gx, t.w, R) : 1.f);
        const float inx = INT ? 1.f / (float)W : inv_countf(nx);
        const int ra = (rg * t.EY1) / ngroups, rb = ((rg + 1) * t.EY1) / ngroups;
        float mg[W], mp[W], sgg[W], sgp[W], vr[W], hda[W], hdb[W];
#pragma unroll
        for (int s = 0; s < 2 * R; ++s) {
            const int e = ra + s;
            fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg[s], mp[s], sgg[s], sgp[s]);
            const int gy = t.ty0 - 2 * R + e;
            vr[s] = (INT || (gy >= 0 && gy < t.h)) ? 1.f : 0.f;
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                a += sDA[e * EX2 + c + k];
                b += sDB[e * EX2 + c + k];
            }
            hda[s] = a;
            hdb[s] = b;
        }
        for (int base = ra; base < rb; base += W) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int e1 = base + s;
                if (e1 < rb) {
                    const int slot = (s + 2 * R) % W;
                    const int e = e1 + 2 * R;
                    fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg[slot], mp[slot],
                                      sgg[slot], sgp[slot]);
                    const int gye = t.ty0 - 2 * R + e;
                    vr[slot] = (INT || (gye >= 0 && gye < t.h)) ? 1.f : 0.f;
                    {
                        float a = 0.f, b = 0.f;
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            a += sDA[e * EX2 + c + k];
                            b += sDB[e * EX2 + c + k];
                        }
                        hda[slot] = a;
                        hdb[slot] = b;
                    }
                    const int gy = t.ty0 - R + e1;
                    float q[NQ];
#pragma unroll
                    for (int k = 0; k < NQ; ++k) q[k] = 0.f;
                    if (INT || (colin && gy >= 0 && gy < t.h)) {
                        const float ny = INT ? (float)W : (float)seg_count(gy, t.h, R);
                        const float iny = INT ? 1.f / (float)W : inv_countf(ny);
                        const float inn = INT ? 1.f / (float)(W * W) : inv_countf(nx * ny);
                        float mu, nu, var, cov;
                        fast_window<R>(mg, mp, sgg, sgp, vr, slot, nx, iny, inn, mu, nu, var, cov);
                        const float ve = var + t.eps;
                        const float ive = rcp_approx(ve);
                        const float A = cov * ive;
                        float dA = 0.f, db = 0.f;
#pragma unroll
                        for (int j = 0; j < W; ++j) {  // oldest row first
                            dA += hda[(slot + 1 + j) % W];
                            db += hdb[(slot + 1 + j) % W];
                        }
                        const float alpha = fmaf(-db, mu, dA);
                        const float gamma = alpha * ive;
                        const float beta = -gamma * A;
                        q[0] = gamma * inn;
                        q[1] = beta * inn;
                        if constexpr (DIRECT) {
                            q[2] = mu;
                            q[3] = nu;
                            q[4] = db * inn;
                            q[5] = db * A * inn;
                        } else {
                            const float mus = mu - KG, nus = nu - KP;
                            q[2] = fmaf(-gamma, mus, db) * inn;
                            q[3] = fmaf(gamma, nus, fmaf(2.f * beta, mus, db * A)) * inn;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < NQ; ++k) sQ[k * n1 + e1 * EX1 + c] = q[k];
                }
            }
        }
    }
    __syncthreads();
    // ---- pass B (r = 2): four separable window sums; dP = G' S0 + S2,
    //   dG = P' S0 + 2 G' S1 - S3 (see kNQ)
    if (!DIRECT && c < t.TX) {
        const int gx = t.tx0 + c;
        const int ya = (rg * t.TY) / ngroups, yb = ((rg + 1) * t.TY) / ngroups;
        float hq[kNQ][W];
#pragma unroll
        for (int s = 0; s < 2 * R; ++s) {
#pragma unroll
            for (int m = 0; m < kNQ; ++m) {
                const float* pq = sQ + m * n1 + (ya + s) * EX1 + c;
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) a += pq[k];
                hq[m][s] = a;
            }
        }
        for (int base = ya; base < yb; base += W) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int y = base + s;
                if (y < yb) {
                    const int slot = (s + 2 * R) % W;
#pragma unroll
                    for (int m = 0; m < kNQ; ++m) {
                        const float* pq = sQ + m * n1 + (y + 2 * R) * EX1 + c;
                        float a = 0.f;
#pragma unroll
                        for (int k = 0; k < W; ++k) a += pq[k];
                        hq[m][slot] = a;
                    }
                    const int gy = t.ty0 + y;
                    if (INT || (gx < t.w && gy < t.h)) {
                        float S[kNQ];
#pragma unroll
                        for (int m = 0; m < kNQ; ++m) {
                            float a = 0.f;
#pragma unroll
                            for (int j = 0; j < W; ++j) a += hq[m][(slot + 1 + j) % W];  // oldest row first
                            S[m] = a;
                        }
                        const int o = (y + 2 * R) * EX2 + c + 2 * R;
                        const float g = sG[o] - KG, p = sP[o] - KP;
                        const size_t go = (size_t)gy * t.w + gx;
                        if (dP != nullptr) dP[go] = from_f32<TP>(fmaf(g, S[0], S[2]));
                        if (dG != nullptr) dG[go] = from_f32<TD>(fmaf(p, S[0], fmaf(2.f * g, S[1], -S[3])));
                    }
                }
            }
        }
    }
    // ---- pass B: exactly centred sums over the windows m containing pixel i,
    //   dP_i = sum gamma~_m (G_i - mu_m) + sum db~_m,
    //   dG_i = sum [gamma~_m (P_i - nu_m) + 2 beta~_m (G_i - mu_m)] - sum (db A)~_m,
    // (~ = divided by N_m).  The window data of the last 2R + 1 rows sit in a
    // register ring (W rows x W columns); only the two plain sums are separable.
    if (DIRECT && c < t.TX) {
        const int gx = t.tx0 + c;
        const int ya = (rg * t.TY) / ngroups, yb = ((rg + 1) * t.TY) / ngroups;
        float rg_[W][W], rb_[W][W], rm[W][W], rn[W][W], hd[W], he[W];
        auto load_row = [&](int e1, float (&g_)[W], float (&b_)[W], float (&m_)[W], float (&n_)[W], float& d_,
                            float& e_) {
            const float* q0 = sQ + e1 * EX1 + c;
            float sd = 0.f, se = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                g_[k] = q0[k];
                b_[k] = q0[n1 + k];
                m_[k] = q0[2 * n1 + k];
                n_[k] = q0[3 * n1 + k];
                sd += q0[4 * n1 + k];
                se += q0[5 * n1 + k];
            }
            d_ = sd;
            e_ = se;
        };
#pragma unroll
        for (int s = 0; s < 2 * R; ++s) load_row(ya + s, rg_[s], rb_[s], rm[s], rn[s], hd[s], he[s]);
        for (int base = ya; base < yb; base += W) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int y = base + s;
                if (y < yb) {
                    const int slot = (s + 2 * R) % W;
                    load_row(y + 2 * R, rg_[slot], rb_[slot], rm[slot], rn[slot], hd[slot], he[slot]);
                    const int gy = t.ty0 + y;
                    if (INT || (gx < t.w && gy < t.h)) {
                        const int o = (y + 2 * R) * EX2 + c + 2 * R;
                        const float g = sG[o], p = sP[o];
                        float aP = 0.f, aG = 0.f, sd = 0.f, se = 0.f;
#pragma unroll
                        for (int jj = 0; jj < W; ++jj) {
                            const int j = (slot + 1 + jj) % W;  // oldest row first
                            sd += hd[j];
                            se += he[j];
#pragma unroll
                            for (int k = 0; k < W; ++k) {
                                const float dg = g - rm[j][k], dp = p - rn[j][k];
                                aP = fmaf(rg_[j][k], dg, aP);
                                aG = fmaf(rg_[j][k], dp, fmaf(2.f * rb_[j][k], dg, aG));
                            }
                        }
                        const size_t go = (size_t)gy * t.w + gx;
                        if (dP != nullptr) dP[go] = from_f32<TP>(aP + sd);
                        if (dG != nullptr) dG[go] = from_f32<TD>(aG - se);
                    }
                }
            }
        }
    }
    __syncthreads();
}


// ------------------------------------------------------------ large radius
// For R >= 4 a register ring of 2R + 1 rows costs too many registers (and
// compile time); the walk instead writes each row's horizontal quantities
// to shared memory and a second walk sums 2R + 1 of them vertically.

template <int R>
__device__ __forceinline__ void fast_col_setup(const FastTile& t, int c, float (&mk)[2 * R + 1], float& nx,
                                               float& inx, bool& colin) {
    const int gx = t.tx0 - R + c;
    colin = gx >= 0 && gx < t.w;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        const int x = gx - R + k;
        mk[k] = (x >= 0 && x < t.w) ? 1.f : 0.f;
    }
    nx = colin ? (float)seg_count(gx, t.w, R) : 1.f;
    inx = inv_countf(nx);
}

// Window moments of E1 row e1, column c, from the row statistics stored in
// H (4 planes of EY2 x CW).
template <int R>
__device__ __forceinline__ void staged_window(const float* H, int plane_stride, int CW, int e1, int c,
                                              const FastTile& t, float nx, float ny, float& mu, float& nu,
                                              float& var, float& cov) {
    const float* hmg = H;
    const float* hmp = H + plane_stride;
    const float* hgg = H + 2 * plane_stride;
    const float* hgp = H + 3 * plane_stride;
    float s1 = 0.f, s2 = 0.f, a = 0.f, cc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        const int o = (e1 + k) * CW + c;
        s1 += hmg[o];
        s2 += hmp[o];
        a += hgg[o];
        cc += hgp[o];
    }
    const float iny = inv_countf(ny);
    mu = s1 * iny;
    nu = s2 * iny;
    float dgg = 0.f, dgp = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        const int gy = t.ty0 - 2 * R + e1 + k;
        const float v = (gy >= 0 && gy < t.h) ? 1.f : 0.f;
        const int o = (e1 + k) * CW + c;
        const float dg = v * (hmg[o] - mu);
        dgg = fmaf(dg, dg, dgg);
        dgp = fmaf(dg, hmp[o] - nu, dgp);
    }
    const float inn = inv_countf(nx * ny);
    var = fmaf(nx, dgg, a) * inn;
    cov = fmaf(nx, dgp, cc) * inn;
}

template <typename TG, typename TP, int R>
__device__ void coef_tile_staged(const TG* __restrict__ G, const TP* __restrict__ P, float2* __restrict__ coef,
                                 const FastTile& t, float* smem, const TmaPlane* tg, const TmaPlane* tp, int plane,
                                 uint32_t* status) {
    constexpr int W = 2 * R + 1;
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R, CW = t.CW;
    float* sG = smem;
    float* sP = sG + EX2 * EY2;
    float* sA = sP + EX2 * EY2;
    float* sB = sA + CW * t.EY1;
    float* H = sB + CW * t.EY1;  // 4 x EY2 x CW, later 2 x EY1 x CW
    bool staged = false;
    if (tg != nullptr && tp != nullptr)
        staged = fast_stage_tma<TG, TP, R>(tg, tp, plane, t, sG, sP, reinterpret_cast<char*>(sA), status);
    if (!staged) {
        fast_stage<TG, R>(G, sG, t);
        fast_stage<TP, R>(P, sP, t);
        __syncthreads();
    }
    const int c = threadIdx.x & (CW - 1), rg = threadIdx.x >> t.log2cw;
    const int ngroups = kLowThreads >> t.log2cw;
    const int hs = EY2 * CW;
    float mk[W], nx, inx;
    bool colin;
    fast_col_setup<R>(t, c, mk, nx, inx, colin);
    for (int e = rg; e < EY2; e += ngroups) {
        float mg, mp, sgg, sgp;
        fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg, mp, sgg, sgp);
        H[e * CW + c] = mg;
        H[hs + e * CW + c] = mp;
        H[2 * hs + e * CW + c] = sgg;
        H[3 * hs + e * CW + c] = sgp;
    }
    __syncthreads();
    for (int e1 = rg; e1 < t.EY1; e1 += ngroups) {
        const int gy = t.ty0 - R + e1;
        float A = 0.f, b = 0.f;
        if (colin && gy >= 0 && gy < t.h) {
            float mu, nu, var, cov;
            staged_window<R>(H, hs, CW, e1, c, t, nx, (float)seg_count(gy, t.h, R), mu, nu, var, cov);
            A = cov * rcp_approx(var + t.eps);
            b = fmaf(-A, mu, nu);
        }
        sA[e1 * CW + c] = A;
        sB[e1 * CW + c] = b;
    }
    __syncthreads();
    float* HA = H;
    float* HB = H + t.EY1 * CW;
    if (c < t.TX) {
        for (int e1 = rg; e1 < t.EY1; e1 += ngroups) {
            float a = 0.f, bb = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                a += sA[e1 * CW + c + k];
                bb += sB[e1 * CW + c + k];
            }
            HA[e1 * CW + c] = a;
            HB[e1 * CW + c] = bb;
        }
    }
    __syncthreads();
    if (c < t.TX) {
        const int gx = t.tx0 + c;
        const float nx0 = (gx < t.w) ? (float)seg_count(gx, t.w, R) : 1.f;
        for (int y = rg; y < t.TY; y += ngroups) {
            const int gy = t.ty0 + y;
            if (gx >= t.w || gy >= t.h) continue;
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                sa += HA[(y + k) * CW + c];
                sb += HB[(y + k) * CW + c];
            }
            const float inn = inv_countf(nx0 * (float)seg_count(gy, t.h, R));
            coef[(size_t)gy * t.w + gx] = make_float2(sa * inn, sb * inn);
        }
    }
    __syncthreads();
}

template <typename TG, typename TP, typename TD, int R>
__device__ void lowres_bwd_tile_staged(const TG* __restrict__ G, const TP* __restrict__ P,
                                       const float2* __restrict__ dcoef, TP* __restrict__ dP, TD* __restrict__ dG,
                                       const FastTile& t, float* smem) {
    constexpr int W = 2 * R + 1;
    const int EX2 = t.CW + 2 * R, EY2 = t.EY1 + 2 * R, CW = t.CW, n1 = t.CW * t.EY1;
    float* sG = smem;
    float* sP = sG + EX2 * EY2;
    float* sDA = sP + EX2 * EY2;
    float* sDB = sDA + EX2 * EY2;
    float* sQ = sDB + EX2 * EY2;
    float* red = sQ + kNQ * n1;
    float* H = red + 3 * (kLowThreads / 32) + 8;  // max(6 x EY2 x CW, kNQ x EY1 x CW)
    float KG, KP;
    bwd_stage_and_shift<TG, TP, R>(G, P, dcoef, t, sG, sP, sDA, sDB, red, KG, KP);
    const int c = threadIdx.x & (CW - 1), rg = threadIdx.x >> t.log2cw;
    const int ngroups = kLowThreads >> t.log2cw;
    const int hs = EY2 * CW;
    float mk[W], nx, inx;
    bool colin;
    fast_col_setup<R>(t, c, mk, nx, inx, colin);
    for (int e = rg; e < EY2; e += ngroups) {
        float mg, mp, sgg, sgp;
        fast_row_stats<R>(sG + e * EX2 + c, sP + e * EX2 + c, mk, inx, mg, mp, sgg, sgp);
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            a += sDA[e * EX2 + c + k];
            b += sDB[e * EX2 + c + k];
        }
        H[e * CW + c] = mg;
        H[hs + e * CW + c] = mp;
        H[2 * hs + e * CW + c] = sgg;
        H[3 * hs + e * CW + c] = sgp;
        H[4 * hs + e * CW + c] = a;
        H[5 * hs + e * CW + c] = b;
    }
    __syncthreads();
    for (int e1 = rg; e1 < t.EY1; e1 += ngroups) {
        const int gy = t.ty0 - R + e1;
        float q[kNQ] = {0.f, 0.f, 0.f, 0.f};
        if (colin && gy >= 0 && gy < t.h) {
            const float ny = (float)seg_count(gy, t.h, R);
            float mu, nu, var, cov;
            staged_window<R>(H, hs, CW, e1, c, t, nx, ny, mu, nu, var, cov);
            const float ve = var + t.eps;
            const float ive = rcp_approx(ve);
            const float A = cov * ive;
            float dA = 0.f, db = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                dA += H[4 * hs + (e1 + k) * CW + c];
                db += H[5 * hs + (e1 + k) * CW + c];
            }
            const float alpha = fmaf(-db, mu, dA);
            const float gamma = alpha * ive;
            const float beta = -gamma * A;
            const float inn = inv_countf(nx * ny);
            const float mus = mu - KG, nus = nu - KP;
            q[0] = gamma * inn;
            q[1] = beta * inn;
            q[2] = fmaf(-gamma, mus, db) * inn;
            q[3] = fmaf(gamma, nus, fmaf(2.f * beta, mus, db * A)) * inn;
        }
#pragma unroll
        for (int k = 0; k < kNQ; ++k) sQ[k * n1 + e1 * CW + c] = q[k];
    }
    __syncthreads();
    if (c < t.TX) {
        for (int e1 = rg; e1 < t.EY1; e1 += ngroups) {
#pragma unroll
            for (int m = 0; m < kNQ; ++m) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) a += sQ[m * n1 + e1 * CW + c + k];
                H[m * n1 + e1 * CW + c] = a;
            }
        }
    }
    __syncthreads();
    if (c < t.TX) {
        const int gx = t.tx0 + c;
        for (int y = rg; y < t.TY; y += ngroups) {
            const int gy = t.ty0 + y;
            if (gx >= t.w || gy >= t.h) continue;
            float S[kNQ];
#pragma unroll
            for (int m = 0; m < kNQ; ++m) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) a += H[m * n1 + (y + k) * CW + c];
                S[m] = a;
            }
            const int o = (y + 2 * R) * EX2 + c + 2 * R;
            const float g = sG[o] - KG, p = sP[o] - KP;
            const size_t go = (size_t)gy * t.w + gx;
            if (dP != nullptr) dP[go] = from_f32<TP>(fmaf(g, S[0], S[2]));
            if (dG != nullptr) dG[go] = from_f32<TD>(fmaf(p, S[0], fmaf(2.f * g, S[1], -S[3])));
        }
    }
    __syncthreads();
}

template <typename TG, typename TP, int R>
__device__ __forceinline__ void coef_tile_fast(const TG* __restrict__ G, const TP* __restrict__ P,
                                               float2* __restrict__ coef, const FastTile& t, float* smem,
                                               const TmaPlane* tg, const TmaPlane* tp, int plane, uint32_t* status) {
    if constexpr (R <= 2) {
        // tiles whose staged region lies inside the image skip every clip
        const bool interior = t.tx0 - 2 * R >= 0 && t.ty0 - 2 * R >= 0 && t.tx0 + t.CW <= t.w &&
                              t.ty0 + t.EY1 <= t.h;
        if (interior)
            coef_tile_ring<TG, TP, R, true>(G, P, coef, t, smem, tg, tp, plane, status);
        else
            coef_tile_ring<TG, TP, R, false>(G, P, coef, t, smem, tg, tp, plane, status);
    } else
        coef_tile_staged<TG, TP, R>(G, P, coef, t, smem, tg, tp, plane, status);
}

template <typename TG, typename TP, typename TD, int R>
__device__ __forceinline__ void lowres_bwd_tile_fast(const TG* __restrict__ G, const TP* __restrict__ P,
                                                     const float2* __restrict__ dcoef, TP* __restrict__ dP,
                                                     TD* __restrict__ dG, const FastTile& t, float* smem) {
    if constexpr (R <= 2) {
        // interior here also needs full window counts at every staged position
        // (d Abar / N is divided by the count of the window centred there), so
        // the staged region must stay R pixels inside the image
        const bool interior = t.tx0 - 3 * R >= 0 && t.ty0 - 3 * R >= 0 && t.tx0 + t.CW + R <= t.w &&
                              t.ty0 + t.EY1 + R <= t.h;
        if (interior)
            lowres_bwd_tile_ring<TG, TP, TD, R, true>(G, P, dcoef, dP, dG, t, smem);
        else
            lowres_bwd_tile_ring<TG, TP, TD, R, false>(G, P, dcoef, dP, dG, t, smem);
    } else
        lowres_bwd_tile_staged<TG, TP, TD, R>(G, P, dcoef, dP, dG, t, smem);
}

}  // namespace dgf
