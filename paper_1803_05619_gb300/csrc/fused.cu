// Forward as one kernel (K12): Eq. 1, the box means of A, b and Eq. 2 with
// the bilinear upsampler, per high-resolution warp strip, for r in {1, 2}
// and integer factors F with one low-res cell per lane.
//
// A warp owns 32 low-res columns J0 .. J0 + 31 (32 F high-res columns) of a
// segment of low-res rows of one plane.  Its lanes run the two-column K1
// walk (lowres_strip2.cuh, 64 - 4R coefficient columns) over the strip's
// coefficient footprint, columns J0 - 1 .. J0 + 32 (the bilinear taps), and
// put each finished row of (Abar, bbar) into a ring of D rows in the warp's
// shared memory instead of HBM.  After every ring period the same lanes run
// the K2 strip walk (hires_strip.cuh) over every row block whose taps are
// now available, reading them from the ring.  So the coefficients never make
// the HBM round trip, there is no stage boundary between the low-res and the
// high-res work, and the low-res arithmetic of a warp overlaps the high-res
// copies it has in flight.  The coefficient footprint costs a second K1
// column pass per strip (64 columns walked for 34 used) plus 4R + 2 halo rows
// per segment: extra arithmetic, no extra HBM bytes.
//
// Every step is the unfused kernels' arithmetic term for term (the K1 walk's
// sums run in row order and its pair arithmetic through non-contracting
// intrinsics, so other segment and strip offsets do not move a bit): the
// output equals the two-kernel forward's bit for bit.  Untuned, it serves
// r = 1; at r = 2 on large images the redundant K1 columns cost more than the
// saved Abar, bbar round trip, and the autotuner keeps the faster form.
#include "common.cuh"
#include "hires_strip.cuh"
#include "kernels.h"
#include "lowres_strip2.cuh"
#include "tma.cuh"

namespace dgf {

constexpr int kK12Warps = 4;   // warps per CTA
constexpr int kK12Cols = 34;   // coefficient columns of a strip: J0 - 1 .. J0 + 32

template <typename T, int R, int F>
struct K12Cfg {
    using A = K2Async<T, F, F>;                     // high-res row staging (per-lane cp.async)
    static constexpr int D = R == 1 ? 4 : 8;       // coefficient rows kept: more than one ring period
    static constexpr int RING_BYTES = A::NSB * A::SLOT;
    static constexpr int COEF_BYTES = D * kK12Cols * 8;
    static constexpr int WARP_BYTES = RING_BYTES + COEF_BYTES;
};

// Stage B's sink: the strip's coefficient columns of row co go to ring row co mod D.
template <int D>
struct CoefRing {
    float2* ring;
    int cx0;  // column of ring entry 0 (J0 - 1)
    __device__ __forceinline__ void put(int co, int x, float2 v) const {
        const int j = x - cx0;
        if (j >= 0 && j < kK12Cols) ring[(co & (D - 1)) * kK12Cols + j] = v;
    }
};

// K2's tap source: the same ring (rows and columns already clamped to the image).
template <int D>
struct CoefRingIn {
    const float2* ring;
    int cx0;
    __device__ __forceinline__ float2 at(int ii, int jj) const {
        return ring[(ii & (D - 1)) * kK12Cols + (jj - cx0)];
    }
};

// One warp: strip `strip`, high-res row blocks of low-res rows [ia, ib).
template <typename T, int R, int F>
__device__ void k12_strip(const T* __restrict__ G, const T* __restrict__ P, const T* __restrict__ in,
                          T* __restrict__ out, int h_l, int w_l, int h, int w, float eps, int strip, int ia, int ib,
                          unsigned char* wsm) {
    using C = K12Cfg<T, R, F>;
    using A = typename C::A;
    constexpr int VEC = F, W = 2 * R + 1, NSB = A::NSB, H0 = F / 2, VB = VEC * (int)sizeof(T), D = C::D;
    const int lane = threadIdx.x & 31;

    // ---- high-res side: blocks b0 .. ib - 1 of the K2 walk, rows staged by cp.async
    const K2Lane L = k2s_lane<VEC, F>(strip, w_l);
    const int b0 = ia == 0 ? -1 : ia;
    const int nblk = ib - b0;
    const uint32_t mine = smem_u32(wsm) + (uint32_t)(lane * VB);
    auto issue = [&](int m) {  // this lane's vectors of block b0 + m (partial lanes copy zeros; handled below)
        const uint32_t dst = mine + (uint32_t)((m % NSB) * A::SLOT);
#pragma unroll
        for (int t = 0; t < F; ++t) {
            const int y = F * (b0 + m) + H0 + t;
            const bool ok = L.full && y >= 0 && y < h;
            cp_async_zfill<VB>(dst + (uint32_t)(t * A::ROW * (int)sizeof(T)),
                               ok ? (const void*)(in + (size_t)y * w + L.x0) : (const void*)in, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int m = 0; m < NSB; ++m) {  // the first blocks' rows arrive while the low-res walk warms up
        if (m < nblk) issue(m);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // ---- low-res side: K1 walk producing coefficient rows ia .. c_hi
    float2* cring = reinterpret_cast<float2*>(wsm + C::RING_BYTES);
    const int cx0 = 32 * strip - 1;
    const int c_hi = min(ib + 1, h_l - 1);  // the last block reads row min(ib + 1, h_l - 1)
    StripGeom s;
    s.h = h_l;
    s.w = w_l;
    s.x0 = cx0 - 2 * R;
    s.y0 = ia;
    s.seg = c_hi - ia + 1;
    s.mean = 1;
    const CoefRing<D> sink{cring, cx0};
    const CoefRingIn<D> src{cring, cx0};
    const int xa = s.x0 + 2 * lane;
    const Strip2Lane<R> ln = strip2_lane<R>(xa, w_l);
    const bool cols_int = s.x0 >= 0 && s.x0 + 64 <= w_l;
    Strip2Ring<R> q;
    strip2_ring_init<T, T, R>(q);
    const f32x2 eps2 = f2_splat(eps);
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, h_l) + 2 * R;

    // ---- consumer: K2 steps (init, then blocks) as their tap rows become available
    K2Rows<VEC, F> kq;
    int step = -1;  // -1: k2s_init pending; then the number of blocks done
    const int need_init = min(max(b0, -1) + 1, h_l - 1);
    auto consume = [&](int have) {  // have: last coefficient row in the ring
        if (step < 0) {
            if (need_init > have) return;
            k2s_init<VEC, F>(kq, src, b0, L.J, h_l, w_l);
            step = 0;
        }
        while (step < nblk && min(b0 + step + 2, h_l - 1) <= have) {
            const int m = step, i = b0 + m;
            k2s_block<VEC, F>(kq, src, i, L.J, h_l, w_l);
            asm volatile("cp.async.wait_group %0;" ::"n"(NSB - 1) : "memory");
            const T* sr = reinterpret_cast<const T*>(wsm + (m % NSB) * A::SLOT) + lane * VEC;
#pragma unroll
            for (int t = 0; t < F; ++t) {
                const int y = F * i + H0 + t;
                float g[VEC];
                if (L.full) {
                    unpack_vec<T, VEC>(*reinterpret_cast<const Vec<T, VEC>*>(sr + t * A::ROW), g);
                } else {
#pragma unroll
                    for (int k = 0; k < VEC; ++k)
                        g[k] = (L.any && y >= 0 && y < h && L.x0 + k < w) ? to_f32<T>(in[(size_t)y * w + L.x0 + k])
                                                                         : 0.f;
                }
                if (L.any && y >= 0 && y < h) {
                    float o[VEC];
                    k2s_row<VEC, F>(kq, g, t, o);
                    k2s_store<T, VEC>(out, y, w, L, o);
                }
            }
            // the slot is read: refill it with block m + NSB (or an empty group)
            if (m + NSB < nblk) issue(m + NSB);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            ++step;
        }
    };

    float gn[2][W], pn[2][W];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            const bool row = e >= 0 && e < h_l && e < e_last;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const bool ok = row && ln.xin[c];
                gn[c][u] = ok ? to_f32<T>(G[(size_t)e * w_l + xa + c]) : 0.f;
                pn[c][u] = ok ? to_f32<T>(P[(size_t)e * w_l + xa + c]) : 0.f;
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
        const bool row_int = cols_int && base >= 3 * R && base + W <= h_l && base + W <= e_last;
        if (row_int)
            strip2_k1_period<R, true>(q, ln, gv, pv, base, e_first, e_last, xa, nullptr, nullptr, s, eps2, &sink);
        else
            strip2_k1_period<R, false>(q, ln, gv, pv, base, e_first, e_last, xa, nullptr, nullptr, s, eps2, &sink);
        __syncwarp();  // the period's coefficient rows are in the ring
        consume(min(base + W, e_last) - 1 - 2 * R);
        __syncwarp();  // every lane has read the taps it needs before the next period overwrites rows
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Warp w of the grid owns strip (w % nstrip) of segment (w / nstrip) % nseg
// (LS low-res rows each) of plane w / (nstrip nseg).
template <typename T, int R, int F>
__global__ void __launch_bounds__(kK12Warps * 32)
    k12_fused(const T* __restrict__ G, const T* __restrict__ P, const T* __restrict__ in, T* __restrict__ out,
              int h_l, int w_l, int h, int w, float eps, int LS, int nstrip, int nseg, int planes) {
    extern __shared__ __align__(128) unsigned char k12sm[];
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kK12Warps + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    k12_strip<T, R, F>(G + plane * lw, P + plane * lw, in + plane * hw, out + plane * hw, h_l, w_l, h, w, eps, strip,
                       sg * LS, min(sg * LS + LS, h_l), k12sm + (size_t)warp * K12Cfg<T, R, F>::WARP_BYTES);
}

template <typename T, int R, int F>
static cudaError_t k12_go(const void* G, const void* P, const void* in, void* out, int planes, int h_l, int w_l,
                          int h, int w, float eps, int LS, cudaStream_t s) {
    const int nstrip = (w_l + 31) / 32, nseg = (h_l + LS - 1) / LS;
    const long long warps = (long long)nstrip * nseg * planes;
    const size_t smem = (size_t)kK12Warps * K12Cfg<T, R, F>::WARP_BYTES;
    auto kern = k12_fused<T, R, F>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned ctas = (unsigned)((warps + kK12Warps - 1) / kK12Warps);
    kern<<<ctas, kK12Warps * 32, smem, s>>>(static_cast<const T*>(G), static_cast<const T*>(P),
                                            static_cast<const T*>(in), static_cast<T*>(out), h_l, w_l, h, w, eps, LS,
                                            nstrip, nseg, planes);
    return cudaGetLastError();
}

template <typename T, int F>
static cudaError_t k12_radius(const void* G, const void* P, const void* in, void* out, int planes, int h_l, int w_l,
                              int h, int w, int r, float eps, int LS, cudaStream_t s) {
    if (r == 1) return k12_go<T, 1, F>(G, P, in, out, planes, h_l, w_l, h, w, eps, LS, s);
    if (r == 2) return k12_go<T, 2, F>(G, P, in, out, planes, h_l, w_l, h, w, eps, LS, s);
    return cudaErrorInvalidValue;
}

// -------------------------------------------------------------------- K13
// Backward K1 + K3 in one kernel per high-res warp strip (r in {1, 2}; the
// K3 strips of 16-byte vectors with one low-res cell per lane: F32 F = 4,
// BF16/F16 F = 8).  The K3 strip's lanes read Abar at cells J0 .. J0 + 31
// (J0 = 30 strip - 1); the same lanes run the two-column K1 walk over those
// columns, put each finished row of Abar into a ring of D rows in the warp's
// shared memory for the K3 walk, and write the window statistics K4 reads to
// HBM for the cells the strip owns (its output columns J0 + 1 .. J0 + 30 and
// the segment's rows), as the backward K1 pass does.  Abar, bbar never reach
// HBM.  Term for term the two kernels' arithmetic: the same bits.
constexpr int kK13Cols = 32;
constexpr int kK13Warps = 4;

template <typename T, int R, int F>
struct K13Cfg {
    using B = K3Tma<T, F, F>;
    static constexpr int D = R == 1 ? 4 : 8;  // Abar rows kept: more than one ring period
    static constexpr int RING_BYTES = B::NSB * B::SLOT;
    static constexpr int COEF_BYTES = D * kK13Cols * 4;
    static constexpr int WARP_BYTES = RING_BYTES + COEF_BYTES;  // a multiple of 128
    static constexpr size_t CTA_BYTES = (size_t)kK13Warps * WARP_BYTES + (size_t)kK13Warps * B::NSB * 8;
};

template <int D>
struct AbarRing {
    float* ring;
    int cx0;  // column of ring entry 0 (J0)
    __device__ __forceinline__ void put(int co, int x, float2 v) const {
        const int j = x - cx0;
        if (j >= 0 && j < kK13Cols) ring[(co & (D - 1)) * kK13Cols + j] = v.x;
    }
};

template <int D>
struct AbarRingIn {
    const float* ring;
    int cx0;
    __device__ __forceinline__ float at(int ii, int jj) const { return ring[(ii & (D - 1)) * kK13Cols + (jj - cx0)]; }
};

// window statistics of the cells [x0, x1) x [y0, y1) this strip segment owns
struct StatsOwned {
    float4* stats;
    int w, x0, x1, y0, y1;
    __device__ __forceinline__ void put(int ce, int x, float4 v) const {
        if (stats != nullptr && ce >= y0 && ce < y1 && x >= x0 && x < x1) stats[(size_t)ce * w + x] = v;
    }
};

template <typename T, int R, int F>
__device__ void k13_strip(const T* __restrict__ G, const T* __restrict__ P, const K3Maps* maps, T* __restrict__ dG,
                          float2* __restrict__ dcoef, float4* __restrict__ stats, int h_l, int w_l, int h, int w,
                          float eps, int strip, int ia, int ib, int plane, unsigned char* wsm, uint64_t* bars,
                          uint32_t* status) {
    using C = K13Cfg<T, R, F>;
    using B = typename C::B;
    constexpr int VEC = F, W = 2 * R + 1, NSB = B::NSB, H0 = F / 2, D = C::D;
    const int lane = threadIdx.x & 31;

    // ---- high-res side: blocks ib0 .. ilast of the K3 walk, rows staged by TMA
    const K3Lane L = k3s_lane<VEC, F>(strip, w_l);
    const int ib0 = ia - 1, ilast = ib - 1;
    const int nblk = ilast - ib0 + 1;
    const int cx0 = K3Strip<VEC, F>::OUT * strip - 1;  // cell of lane 0
    const int xs = F * cx0;                            // 16-byte aligned (may be negative)
    const uint32_t ring_s = smem_u32(wsm), bar_s = smem_u32(bars);
    auto issue = [&](int m) {  // lane 0: block ib0 + m into slot m % NSB
        const int slot = m % NSB;
        const uint32_t bar = bar_s + 8u * slot, dst = ring_s + (uint32_t)(slot * B::SLOT);
        const int y = F * (ib0 + m) + H0;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)B::SLOT)
                     : "memory");
        tma_load_3d(dst, &maps->r, xs, y, plane, bar);
        tma_load_3d(dst + (uint32_t)B::BOX_BYTES, &maps->g, xs, y, plane, bar);
    };
    if (lane == 0) {  // the first blocks' rows arrive while the low-res walk warms up
        for (int k = 0; k < NSB; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * k) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int m = 0; m < min(NSB, nblk); ++m) issue(m);
    }
    __syncwarp();

    // ---- low-res side: K1 walk producing Abar rows c_lo .. c_hi
    float* cring = reinterpret_cast<float*>(wsm + C::RING_BYTES);
    const int c_lo = max(ia - 1, 0), c_hi = min(ib + 1, h_l - 1);
    StripGeom s;
    s.h = h_l;
    s.w = w_l;
    s.x0 = cx0 - 2 * R;
    s.y0 = c_lo;
    s.seg = c_hi - c_lo + 1;
    s.mean = 1;
    const AbarRing<D> sink{cring, cx0};
    const AbarRingIn<D> src{cring, cx0};
    const StatsOwned sown{stats, w_l, cx0 + 1, cx0 + 1 + K3Strip<VEC, F>::OUT, ia, ib};
    const int xa = s.x0 + 2 * lane;
    const Strip2Lane<R> ln = strip2_lane<R>(xa, w_l);
    const bool cols_int = s.x0 >= 0 && s.x0 + 64 <= w_l;
    Strip2Ring<R> q;
    strip2_ring_init<T, T, R>(q);
    const f32x2 eps2 = f2_splat(eps);
    const int e_first = s.y0 - 2 * R;
    const int e_last = min(s.y0 + s.seg, h_l) + 2 * R;

    // ---- consumer: K3 steps (init, then blocks) as their Abar rows become available
    K3State<VEC, F> st;
    int step = -1;  // -1: k3s_init pending; then the number of blocks done
    bool ok = true;
    const int need_init = min(max(ib0, -1) + 1, h_l - 1);
    auto consume = [&](int have) {  // have: last Abar row in the ring
        if (step < 0) {
            if (need_init > have) return;
            k3s_init<VEC, F>(st, src, ib0, L, h_l, w_l);
            step = 0;
        }
        while (step < nblk && min(ib0 + step + 2, h_l - 1) <= have) {
            const int m = step, slot = m % NSB, i = ib0 + m;
            k3s_block_start<VEC, F>(st, src, i, L, h_l, w_l);
            if (!__all_sync(0xffffffffu, mbar_wait(bar_s + 8u * slot, (uint32_t)((m / NSB) & 1), first_wait_limit(status)))) {
                ok = false;
                return;
            }
            const T* sr = reinterpret_cast<const T*>(wsm + slot * B::SLOT) + lane * VEC;
#pragma unroll
            for (int t = 0; t < F; ++t) {
                float r[VEC], g[VEC];
                unpack_vec<T, VEC>(*reinterpret_cast<const Vec<T, VEC>*>(sr + t * B::ROW), r);
                unpack_vec<T, VEC>(*reinterpret_cast<const Vec<T, VEC>*>(sr + F * B::ROW + t * B::ROW), g);
                if (t == F - 1) {
                    __syncwarp();  // every lane has read the slot
                    if (lane == 0 && m + NSB < nblk) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(m + NSB);
                    }
                }
                k3s_row<T, VEC, F>(st, r, g, t, i, ia, L, dG, h, w);
            }
            k3s_block_end<VEC, F>(st, i, ia, L, h_l, w_l, dcoef);
            ++step;
        }
    };

    float gn[2][W], pn[2][W];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int e = base + u;
            const bool row = e >= 0 && e < h_l && e < e_last;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const bool okc = row && ln.xin[c];
                gn[c][u] = okc ? to_f32<T>(G[(size_t)e * w_l + xa + c]) : 0.f;
                pn[c][u] = okc ? to_f32<T>(P[(size_t)e * w_l + xa + c]) : 0.f;
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
        const bool row_int = cols_int && base >= 3 * R && base + W <= h_l && base + W <= e_last;
        if (row_int)
            strip2_k1_period<R, true>(q, ln, gv, pv, base, e_first, e_last, xa, nullptr, nullptr, s, eps2, &sink,
                                      &sown);
        else
            strip2_k1_period<R, false>(q, ln, gv, pv, base, e_first, e_last, xa, nullptr, nullptr, s, eps2, &sink,
                                       &sown);
        __syncwarp();  // the period's Abar rows are in the ring
        consume(min(base + W, e_last) - 1 - 2 * R);
        __syncwarp();  // every lane has read the rows it needs before the next period overwrites rows
        if (!ok) break;  // uniform (the wait's result is the warp's)
    }
    if (!ok) {
        // record the timeout, then wait (bounded) for the copies still in flight
        if (lane == 0) status_fail(status, kStatusTimeout);
        for (int qb = step; qb < nblk && qb < step + NSB; ++qb)
            mbar_wait(bar_s + 8u * (qb % NSB), (uint32_t)((qb / NSB) & 1), kWaitLimit);
    }
}

template <typename T, int R, int F>
__global__ void __launch_bounds__(kK13Warps * 32)
    k13_fused_bwd(const T* __restrict__ G, const T* __restrict__ P, const __grid_constant__ K3Maps maps,
                  T* __restrict__ dG, float2* __restrict__ dcoef, float4* __restrict__ stats, int h_l, int w_l, int h,
                  int w, float eps, int LS, int nstrip, int nseg, int planes, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char k13sm[];
    using C = K13Cfg<T, R, F>;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kK13Warps + warp;
    if (gw >= nstrip * nseg * planes) return;  // whole warp leaves together
    const int strip = gw % nstrip, rest = gw / nstrip;
    const int sg = rest % nseg, plane = rest / nseg;
    const size_t hw = (size_t)h * w, lw = (size_t)h_l * w_l;
    uint64_t* bars = reinterpret_cast<uint64_t*>(k13sm + (size_t)kK13Warps * C::WARP_BYTES) + warp * C::B::NSB;
    k13_strip<T, R, F>(G + plane * lw, P + plane * lw, &maps, dG ? dG + plane * hw : nullptr, dcoef + plane * lw,
                       stats ? stats + plane * lw : nullptr, h_l, w_l, h, w, eps, strip, sg * LS,
                       min(sg * LS + LS, h_l), plane, k13sm + (size_t)warp * C::WARP_BYTES, bars, status);
}

template <typename T, int R, int F>
static cudaError_t k13_go(const void* G, const void* P, const K3Maps& maps, void* dG, float2* dcoef, float4* stats,
                          int planes, int h_l, int w_l, int h, int w, float eps, int LS, uint32_t* status,
                          cudaStream_t s) {
    using C = K13Cfg<T, R, F>;
    constexpr int OUT = K3Strip<F, F>::OUT;
    const int nstrip = (w_l + OUT - 1) / OUT, nseg = (h_l + LS - 1) / LS;
    const long long warps = (long long)nstrip * nseg * planes;
    auto kern = k13_fused_bwd<T, R, F>;
    if (C::CTA_BYTES > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::CTA_BYTES);
        if (e != cudaSuccess) return e;
    }
    const unsigned ctas = (unsigned)((warps + kK13Warps - 1) / kK13Warps);
    kern<<<ctas, kK13Warps * 32, C::CTA_BYTES, s>>>(static_cast<const T*>(G), static_cast<const T*>(P), maps,
                                                     static_cast<T*>(dG), dcoef, stats, h_l, w_l, h, w, eps, LS,
                                                     nstrip, nseg, planes, status);
    return cudaGetLastError();
}

template <typename T, int F>
static cudaError_t k13_radius(const void* G, const void* P, const K3Maps& maps, void* dG, float2* dcoef,
                              float4* stats, int planes, int h_l, int w_l, int h, int w, int r, float eps, int LS,
                              uint32_t* status, cudaStream_t s) {
    if (r == 1) return k13_go<T, 1, F>(G, P, maps, dG, dcoef, stats, planes, h_l, w_l, h, w, eps, LS, status, s);
    if (r == 2) return k13_go<T, 2, F>(G, P, maps, dG, dcoef, stats, planes, h_l, w_l, h, w, eps, LS, status, s);
    return cudaErrorInvalidValue;
}

bool k13_supported(dgf_dtype dt, int r, int F, int vec) {
    if (r != 1 && r != 2) return false;
    if (vec != F) return false;
    return dt == DGF_F32 ? F == 4 : F == 8;  // 16-byte vectors of F pixels
}

cudaError_t launch_k13(dgf_dtype dt, const void* G, const void* P, const K3Maps& maps, void* dG, float2* dcoef,
                       float4* stats, int planes, int h_l, int w_l, int h, int w, int r, int F, float eps, int LS,
                       uint32_t* status, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    if (!k13_supported(dt, r, F, F) || LS < 1) return cudaErrorInvalidValue;
    switch (dt) {
        case DGF_F32: return k13_radius<float, 4>(G, P, maps, dG, dcoef, stats, planes, h_l, w_l, h, w, r, eps, LS, status, s);
        case DGF_BF16:
            return k13_radius<__nv_bfloat16, 8>(G, P, maps, dG, dcoef, stats, planes, h_l, w_l, h, w, r, eps, LS, status, s);
        case DGF_F16: return k13_radius<__half, 8>(G, P, maps, dG, dcoef, stats, planes, h_l, w_l, h, w, r, eps, LS, status, s);
    }
    return cudaErrorInvalidValue;
}

bool k12_supported(dgf_dtype dt, int r, int F) {
    if (r != 1 && r != 2) return false;
    if (dt == DGF_F32) return F == 2 || F == 4;  // 8- and 16-byte vectors of F pixels
    return F == 4 || F == 8;
}

int k12_vec_bytes(dgf_dtype dt, int F) { return F * (dt == DGF_F32 ? 4 : 2); }

cudaError_t launch_k12(dgf_dtype dt, const void* G, const void* P, const void* in, void* out, int planes, int h_l,
                       int w_l, int h, int w, int r, int F, float eps, int LS, cudaStream_t s) {
    if (planes == 0) return cudaSuccess;
    if (!k12_supported(dt, r, F) || LS < 1) return cudaErrorInvalidValue;
    switch (dt) {
        case DGF_F32:
            return F == 2 ? k12_radius<float, 2>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s)
                          : k12_radius<float, 4>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s);
        case DGF_BF16:
            return F == 4 ? k12_radius<__nv_bfloat16, 4>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s)
                          : k12_radius<__nv_bfloat16, 8>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s);
        case DGF_F16:
            return F == 4 ? k12_radius<__half, 4>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s)
                          : k12_radius<__half, 8>(G, P, in, out, planes, h_l, w_l, h, w, r, eps, LS, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dgf
