// K3 as a warp-strip column walk (integer factor F, F | VEC).
//
// One warp owns a strip of 32 lanes x VEC high-res columns (K = VEC / F
// low-res cells per lane) and walks down the high-res rows of a segment of
// low-res rows.  Per high-res row y, with taps (i, i + 1) and weight lam_y:
//   d I_h(y, x)  = d O_h(y, x) * Abar_h(y, x),
//   Abar_h(y, .) = lerp(H_i, H_{i+1}, lam_y), H_i = row i of Abar
//                  interpolated along x at the lane's pixels (formed once per
//                  low-res row);
//   the transposed upsampler (Algorithm 1's first two lines): each pixel's
//   u = d O_h I_h and v = d O_h go to its two tap columns with the x weights
//   (in registers, then one shuffle from each neighbouring lane), and each
//   row's column sums go to the two tap rows with the y weights, into
//   register accumulators of low-res rows i and i + 1.
// Row i of d Abar, d bbar is complete once the rows of block i (the F rows
// whose first tap is i) are done; it is written then.  Virtual taps outside
// the image (row/column -1 and h_l / w_l) are accumulated like real ones and
// folded into the border row/column when written, as the clamp of the
// forward upsampler does.  Lanes 0 and 31 are the strip's halo (neighbouring
// strips overlap by 2K cells); the first block of a segment is its halo row.
// No atomics: every output is written once.  Rows reach the lanes either
// through a register ring filled one period (P rows) ahead, or (16-byte
// vectors) through a per-warp shared-memory ring filled by TMA.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace dgf {

template <int VEC, int F>
struct K3Strip {
    static constexpr int K = VEC / F;               // low-res cells per lane
    static constexpr int NB = F >= 4 ? 1 : 4 / F;   // blocks of F rows per period
    static constexpr int P = F * NB;                // rows per period (prefetch distance)
    static constexpr int OUT = 30 * K;              // output cells per strip (lanes 1 .. 30)
};

// Tap of lane pixel k (cell c = k / F, phase q = k % F): tap index lo (in the
// lane's tap columns J - 1 .. J + K, index 0 .. K + 1), weight of lo + 1.
template <int F>
__host__ __device__ constexpr int k3s_lo(int k) {
    return (k % F) < F / 2 ? k / F : k / F + 1;
}
template <int F>
__host__ __device__ constexpr float k3s_lam(int k) {
    return (k % F) < F / 2 ? (float)(2 * (k % F) + 1 + F) / (float)(2 * F)
                           : (float)(2 * (k % F) + 1 - F) / (float)(2 * F);
}

// Where K3 reads Abar of row ii, column jj from: the plane's coefficient array.
struct AbarIn {
    const float2* __restrict__ coef;
    int w_l;
    __device__ __forceinline__ float at(int ii, int jj) const {
        return reinterpret_cast<const float*>(coef)[2 * ((size_t)ii * w_l + jj)];
    }
};

// Abar of row ii at the lane's own K cells (columns clamped to the image).
template <int VEC, int F, class Src>
__device__ __forceinline__ void k3s_own(const Src& coef, int ii, int J, int w_l, float (&own)[VEC / F]) {
    constexpr int K = VEC / F;
#pragma unroll
    for (int c = 0; c < K; ++c) own[c] = coef.at(ii, clampi(J + c, 0, w_l - 1));
}

// A row of Abar interpolated along x at the lane's VEC pixels, from the
// lane's own cells and its neighbours' (columns clamp as in the forward).
template <int VEC, int F>
__device__ __forceinline__ void k3s_hrow_from(const float (&own)[VEC / F], int J, int w_l, float (&H)[VEC]) {
    constexpr int K = VEC / F;
    const float up = __shfl_up_sync(0xffffffffu, own[K - 1], 1);
    const float dn = __shfl_down_sync(0xffffffffu, own[0], 1);
    float tp[K + 2];
    tp[0] = (J - 1 < 0) ? own[0] : up;
#pragma unroll
    for (int c = 0; c < K; ++c) tp[c + 1] = own[c];
    tp[K + 1] = (J + K > w_l - 1) ? own[K - 1] : dn;
#pragma unroll
    for (int k = 0; k < VEC; ++k) H[k] = lerp(tp[k3s_lo<F>(k)], tp[k3s_lo<F>(k) + 1], k3s_lam<F>(k));
}

// Row y of R, G at the lane's pixels (zero outside the image or the segment).
template <typename T, int VEC>
__device__ __forceinline__ void k3s_load(const T* __restrict__ R, const T* __restrict__ G, int y, bool row_ok,
                                         int x0, int w, bool full, bool any, Vec<T, VEC>& r, Vec<T, VEC>& g) {
    if (row_ok && full) {
        r = ldg_vec<T, VEC>(R + (size_t)y * w + x0);
        g = ldg_vec<T, VEC>(G + (size_t)y * w + x0);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const bool ok = row_ok && any && x0 + k >= 0 && x0 + k < w;
            r.v[k] = ok ? R[(size_t)y * w + x0 + k] : from_f32<T>(0.f);
            g.v[k] = ok ? G[(size_t)y * w + x0 + k] : from_f32<T>(0.f);
        }
    }
}

// Per-lane state of a strip walk: Abar rows i, i + 1 along x at the lane's
// pixels, and the accumulators of d Abar, d bbar rows i (lo) and i + 1 (hi).
// PD: blocks ahead that the Abar cells are loaded (the fused backward,
// whose Abar rows are produced as it walks, uses 1).
template <int VEC, int F, int PD = 1>
struct K3State {
    static constexpr int K = VEC / F;
    float Hlo[VEC], Hhi[VEC];
    float alu[K], alv[K], ahu[K], ahv[K];
    float own_next[PD][K];  // Abar cells of the next PD blocks' second tap rows, oldest first
};

struct K3Lane {
    int J, x0;      // first cell and first high-res column of the lane
    bool full;      // all VEC pixels inside the image
    bool any;       // some pixel inside the image
    bool out;       // lane writes outputs (lanes 1 .. 30)
};

template <int VEC, int F>
__device__ __forceinline__ K3Lane k3s_lane(int strip, int w_l) {
    constexpr int K = VEC / F;
    const int lane = threadIdx.x & 31;
    K3Lane L;
    L.J = K3Strip<VEC, F>::OUT * strip - K + lane * K;
    L.x0 = F * L.J;
    L.full = L.J >= 0 && L.J + K <= w_l;
    L.any = L.J + K > 0 && L.J < w_l;
    L.out = lane >= 1 && lane <= 30;
    return L;
}

// Block i begins: Abar rows i and i + 1 (clamped) along x; the cells of row
// i + 1 + PD are loaded for later blocks.
template <int VEC, int F, int PD, class Src>
__device__ __forceinline__ void k3s_block_start(K3State<VEC, F, PD>& st, const Src& coef, int i, const K3Lane& L,
                                                int h_l, int w_l) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) st.Hlo[k] = st.Hhi[k];
    k3s_hrow_from<VEC, F>(st.own_next[0], L.J, w_l, st.Hhi);  // row min(i + 1, h_l - 1)
#pragma unroll
    for (int d = 0; d + 1 < PD; ++d)
#pragma unroll
        for (int c = 0; c < VEC / F; ++c) st.own_next[d][c] = st.own_next[d + 1][c];
    k3s_own<VEC, F>(coef, min(i + 1 + PD, h_l - 1), L.J, w_l, st.own_next[PD - 1]);
}

// High-res row y = F i + F/2 + t of block i (t compile-time after unrolling).
template <typename T, int VEC, int F, int PD>
__device__ __forceinline__ void k3s_row(K3State<VEC, F, PD>& st, const float (&r)[VEC], const float (&g)[VEC], int t,
                                        int i, int ia, const K3Lane& L, T* __restrict__ dG, int h, int w) {
    constexpr int K = VEC / F;
    const int y = F * i + F / 2 + t;
    const float lamy = (float)(2 * t + 1) / (float)(2 * F);
    // d I_h = d O_h * Abar_h (rows this segment owns)
    if (dG != nullptr && L.out && L.any && y >= 0 && y < h && (i >= ia || ia == 0)) {
        float o[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) o[k] = r[k] * lerp(st.Hlo[k], st.Hhi[k], lamy);
        if (L.full) {
            store_vec<T, VEC>(dG + (size_t)y * w + L.x0, o);
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (L.x0 + k >= 0 && L.x0 + k < w) dG[(size_t)y * w + L.x0 + k] = from_f32<T>(o[k]);
        }
    }
    // transposed upsampler: x weights onto the tap columns, lanes combined
    float pu[K + 2], pv[K + 2];
#pragma unroll
    for (int c = 0; c < K + 2; ++c) pu[c] = pv[c] = 0.f;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int lo = k3s_lo<F>(k);
        const float lx = k3s_lam<F>(k);
        const float u = r[k] * g[k];
        pu[lo] = fmaf(1.f - lx, u, pu[lo]);
        pu[lo + 1] = fmaf(lx, u, pu[lo + 1]);
        pv[lo] = fmaf(1.f - lx, r[k], pv[lo]);
        pv[lo + 1] = fmaf(lx, r[k], pv[lo + 1]);
    }
    const float lu = __shfl_up_sync(0xffffffffu, pu[K + 1], 1);
    const float lv = __shfl_up_sync(0xffffffffu, pv[K + 1], 1);
    const float ru = __shfl_down_sync(0xffffffffu, pu[0], 1);
    const float rv = __shfl_down_sync(0xffffffffu, pv[0], 1);
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float su = pu[c + 1], sv = pv[c + 1];
        if (c == 0) {
            su += lu;
            sv += lv;
        }
        if (c == K - 1) {
            su += ru;
            sv += rv;
        }
        // y weights onto the tap rows i, i + 1
        st.alu[c] = fmaf(1.f - lamy, su, st.alu[c]);
        st.alv[c] = fmaf(1.f - lamy, sv, st.alv[c]);
        st.ahu[c] = fmaf(lamy, su, st.ahu[c]);
        st.ahv[c] = fmaf(lamy, sv, st.ahv[c]);
    }
}

// Block i done: row i of d Abar, d bbar is complete; write it (rows this
// segment owns) and move the accumulators down one row.
template <int VEC, int F, int PD>
__device__ __forceinline__ void k3s_block_end(K3State<VEC, F, PD>& st, int i, int ia, const K3Lane& L, int h_l,
                                              int w_l, float2* __restrict__ dcoef) {
    constexpr int K = VEC / F;
    if (i == -1) {  // virtual row -1 folds into row 0
#pragma unroll
        for (int c = 0; c < K; ++c) {
            st.ahu[c] += st.alu[c];
            st.ahv[c] += st.alv[c];
        }
    }
    if (i == h_l - 1) {  // virtual row h_l folds into row h_l - 1
#pragma unroll
        for (int c = 0; c < K; ++c) {
            st.alu[c] += st.ahu[c];
            st.alv[c] += st.ahv[c];
        }
    }
    if (i >= ia && i >= 0) {
        // virtual columns -1 and w_l fold into columns 0 and w_l - 1
        const float fu = __shfl_up_sync(0xffffffffu, st.alu[K - 1], 1);
        const float fv = __shfl_up_sync(0xffffffffu, st.alv[K - 1], 1);
        const float gu = __shfl_down_sync(0xffffffffu, st.alu[0], 1);
        const float gv = __shfl_down_sync(0xffffffffu, st.alv[0], 1);
        if (L.J == 0) {
            st.alu[0] += fu;
            st.alv[0] += fv;
        }
#pragma unroll
        for (int c = 1; c < K; ++c)
            if (L.J + c == w_l) {
                st.alu[c - 1] += st.alu[c];
                st.alv[c - 1] += st.alv[c];
            }
        if (L.J + K == w_l) {
            st.alu[K - 1] += gu;
            st.alv[K - 1] += gv;
        }
        if (L.out) {
#pragma unroll
            for (int c = 0; c < K; ++c)
                if (L.J + c >= 0 && L.J + c < w_l)
                    dcoef[(size_t)i * w_l + L.J + c] = make_float2(st.alu[c], st.alv[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        st.alu[c] = st.ahu[c];
        st.alv[c] = st.ahv[c];
        st.ahu[c] = st.ahv[c] = 0.f;
    }
}

template <int VEC, int F, int PD, class Src>
__device__ __forceinline__ void k3s_init(K3State<VEC, F, PD>& st, const Src& coef, int ib0, const K3Lane& L, int h_l,
                                         int w_l) {
    constexpr int K = VEC / F;
    k3s_own<VEC, F>(coef, clampi(ib0, 0, h_l - 1), L.J, w_l, st.own_next[0]);
    k3s_hrow_from<VEC, F>(st.own_next[0], L.J, w_l, st.Hhi);
#pragma unroll
    for (int d = 0; d < PD; ++d) k3s_own<VEC, F>(coef, min(max(ib0, -1) + 1 + d, h_l - 1), L.J, w_l, st.own_next[d]);
#pragma unroll
    for (int c = 0; c < K; ++c) st.alu[c] = st.alv[c] = st.ahu[c] = st.ahv[c] = 0.f;
}

// Segment of low-res rows [ia, ib) of strip `strip` of one plane; rows are
// loaded one period ahead into a register ring.
template <typename T, int VEC, int F>
__device__ void k3_strip(const float2* __restrict__ coef, const T* __restrict__ R, const T* __restrict__ G,
                         T* __restrict__ dG, float2* __restrict__ dcoef, int h_l, int w_l, int h, int w, int strip,
                         int ia, int ib) {
    using S = K3Strip<VEC, F>;
    constexpr int NB = S::NB, P = S::P, H0 = F / 2;
    const K3Lane L = k3s_lane<VEC, F>(strip, w_l);
    const int ib0 = ia - 1, ilast = ib - 1;  // blocks ib0 .. ilast
    const int nper = (ilast - ib0 + 1 + NB - 1) / NB;
    auto row_of = [&](int pi, int s) { return F * (ib0 + pi * NB + s / F) + H0 + s % F; };
    auto row_ok = [&](int pi, int s) {
        const int y = row_of(pi, s);
        return ib0 + pi * NB + s / F <= ilast && y >= 0 && y < h;
    };
    Vec<T, VEC> rr[P], gg[P];
#pragma unroll
    for (int s = 0; s < P; ++s)
        k3s_load<T, VEC>(R, G, row_of(0, s), row_ok(0, s), L.x0, w, L.full, L.any, rr[s], gg[s]);
    K3State<VEC, F> st;
    k3s_init<VEC, F>(st, AbarIn{coef, w_l}, ib0, L, h_l, w_l);
    for (int pi = 0; pi < nper; ++pi) {
#pragma unroll
        for (int s = 0; s < P; ++s) {
            const int t = s % F;
            const int i = ib0 + pi * NB + s / F;
            if (i > ilast) break;  // uniform: past the segment's last block
            if (t == 0) k3s_block_start<VEC, F>(st, AbarIn{coef, w_l}, i, L, h_l, w_l);
            float r[VEC], g[VEC];
            unpack_vec<T, VEC>(rr[s], r);
            unpack_vec<T, VEC>(gg[s], g);
            if (pi + 1 < nper)
                k3s_load<T, VEC>(R, G, row_of(pi + 1, s), row_ok(pi + 1, s), L.x0, w, L.full, L.any, rr[s], gg[s]);
            k3s_row<T, VEC, F>(st, r, g, t, i, ia, L, dG, h, w);
            if (t == F - 1) k3s_block_end<VEC, F>(st, i, ia, L, h_l, w_l, dcoef);
        }
    }
}

// Same walk with the rows staged by TMA: per warp a ring of NSB slots, each
// holding one block (F rows) of R and of G as two tiled copies (box
// 32 VEC x F of a 3-D tensor map over columns, rows, planes; rows and
// columns outside the image read as zero, so edge strips and the segment's
// halo rows need no special case), one mbarrier per slot.  The warp's lane 0
// issues a block's two copies as soon as the warp has finished reading the
// slot.  Waits are bounded: on a timeout the warp records it in the status
// word, waits (bounded) for its copies in flight and stops.
template <typename T, int VEC, int F>
struct K3Tma {
    static constexpr int ROW = 32 * VEC;                           // box width (elements)
    static constexpr int NSB = F == 2 ? 6 : (F == 4 ? 3 : 2);      // slots (blocks) per warp
    static constexpr int WPC = F == 8 ? 4 : 8;                     // warps per CTA
    static constexpr int BOX_BYTES = ROW * F * (int)sizeof(T);     // one tensor, one block
    static constexpr int SLOT = 2 * BOX_BYTES;
    static constexpr size_t CTA_BYTES = (size_t)WPC * NSB * SLOT + (size_t)WPC * NSB * 8;
};


// Returns false after a timeout (recorded in the status word); the warp's
// copies have then landed or been waited for (bounded).  On success the slot
// barriers are invalidated, so a persistent warp can call it again with the
// same ring.
template <typename T, int VEC, int F>
__device__ bool k3_strip_tma(const float2* __restrict__ coef, const K3Maps* maps, T* __restrict__ dG,
                             float2* __restrict__ dcoef, int h_l, int w_l, int h, int w, int strip, int ia, int ib,
                             int plane, unsigned char* ring, uint64_t* bars, uint32_t* status) {
    using B = K3Tma<T, VEC, F>;
    static_assert(VEC * sizeof(T) == 16, "TMA staging needs 16-byte vectors");
    constexpr int NSB = B::NSB, H0 = F / 2;
    const int lane = threadIdx.x & 31;
    const K3Lane L = k3s_lane<VEC, F>(strip, w_l);
    const int ib0 = ia - 1, ilast = ib - 1;
    const int nblk = ilast - ib0 + 1;
    const int xs = F * (K3Strip<VEC, F>::OUT * strip - VEC / F);  // 16-byte aligned (may be negative)
    const uint32_t ring_s = smem_u32(ring), bar_s = smem_u32(bars);
    auto issue = [&](int m) {  // lane 0: block ib0 + m into slot m % NSB
        const int slot = m % NSB;
        const uint32_t bar = bar_s + 8u * slot, dst = ring_s + (uint32_t)(slot * B::SLOT);
        const int y = F * (ib0 + m) + H0;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)B::SLOT)
                     : "memory");
        tma_load_3d(dst, &maps->r, xs, y, plane, bar);
        tma_load_3d(dst + (uint32_t)B::BOX_BYTES, &maps->g, xs, y, plane, bar);
    };
    __syncwarp();  // a previous walk's reads of the ring are done
    if (lane == 0) {
        for (int s = 0; s < NSB; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int m = 0; m < min(NSB, nblk); ++m) issue(m);
    }
    __syncwarp();
    K3State<VEC, F> st;
    k3s_init<VEC, F>(st, AbarIn{coef, w_l}, ib0, L, h_l, w_l);
    int m = 0;
    bool ok = true;
    for (; m < nblk; ++m) {
        const int slot = m % NSB;
        const int i = ib0 + m;
        k3s_block_start<VEC, F>(st, AbarIn{coef, w_l}, i, L, h_l, w_l);
        if (!__all_sync(0xffffffffu, mbar_wait(bar_s + 8u * slot, (uint32_t)((m / NSB) & 1), first_wait_limit(status)))) {
            ok = false;
            break;
        }
        const T* sr = reinterpret_cast<const T*>(ring + slot * B::SLOT) + lane * VEC;
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
    }
    if (!ok) {
        // record the timeout, then wait (bounded) for the copies still in flight
        if (lane == 0) status_fail(status, kStatusTimeout);
        for (int q = m; q < nblk && q < m + NSB; ++q)
            mbar_wait(bar_s + 8u * (q % NSB), (uint32_t)((q / NSB) & 1), kWaitLimit);
        return false;
    }
    __syncwarp();  // every lane has passed its last wait
    if (lane == 0)
        for (int s = 0; s < NSB; ++s) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar_s + 8u * s) : "memory");
    return true;
}

// ------------------------------------------------------------- K2 strip
// Eq. 2 after the bilinear upsampler, as a strip walk: a lane holds VEC
// pixels (K = VEC / F cells).  Per low-res row block i (the F high-res rows
// whose first tap is row i) the lane forms once row i + 1 of Abar and bbar
// interpolated along x at its pixels (from its K + 2 tap columns, clamped)
// and the difference to row i; each high-res row of the block then costs one
// FMA per coefficient and one for the output.  Every lane writes its pixels
// (no halo).  Rows reach the lanes through per-warp shared-memory slots,
// filled by TMA (16-byte vectors, single calls) or by per-lane asynchronous
// copies.
// PD: blocks ahead that the coefficient taps are loaded (the fused forward,
// whose coefficient rows are produced as it walks, uses 1).
template <int VEC, int F, int PD = 1>
struct K2Rows {
    float A1[VEC], B1[VEC];       // row i + 1 (the block's second tap row) along x
    float DA[VEC], DB[VEC];       // row i + 1 minus row i
    float2 next[PD][VEC / F + 2]; // tap columns of the next PD blocks' second rows, oldest first
};

// Where K2 reads (Abar, bbar) of row ii, column jj from: the plane's
// coefficient array.
struct CoefIn {
    const float2* __restrict__ coef;
    int w_l;
    __device__ __forceinline__ float2 at(int ii, int jj) const { return coef[(size_t)ii * w_l + jj]; }
};

// The lane's K + 2 tap columns of coefficient row ii (clamped to the image).
template <int VEC, int F, class Src>
__device__ __forceinline__ void k2s_taps(const Src& coef, int ii, int J, int w_l, float2 (&tp)[VEC / F + 2]) {
    constexpr int K = VEC / F;
#pragma unroll
    for (int c = 0; c < K + 2; ++c) tp[c] = coef.at(ii, clampi(J - 1 + c, 0, w_l - 1));
}

template <int VEC, int F>
__device__ __forceinline__ void k2s_hrow_from(const float2 (&tp)[VEC / F + 2], float (&HA)[VEC], float (&HB)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        HA[k] = lerp(tp[k3s_lo<F>(k)].x, tp[k3s_lo<F>(k) + 1].x, k3s_lam<F>(k));
        HB[k] = lerp(tp[k3s_lo<F>(k)].y, tp[k3s_lo<F>(k) + 1].y, k3s_lam<F>(k));
    }
}

// Before the first block b0: row clamp(b0) becomes the "second tap" row;
// the taps of rows b0 + 1 .. b0 + PD (clamped) are loaded ahead.
template <int VEC, int F, int PD, class Src>
__device__ __forceinline__ void k2s_init(K2Rows<VEC, F, PD>& q, const Src& coef, int b0, int J, int h_l, int w_l) {
    k2s_taps<VEC, F>(coef, clampi(b0, 0, h_l - 1), J, w_l, q.next[0]);
    k2s_hrow_from<VEC, F>(q.next[0], q.A1, q.B1);
#pragma unroll
    for (int d = 0; d < PD; ++d) k2s_taps<VEC, F>(coef, min(max(b0, -1) + 1 + d, h_l - 1), J, w_l, q.next[d]);
}

// Block i begins: taps rows clamp(i) (the previous second row) and clamp(i + 1);
// the taps of row i + 1 + PD are loaded for later blocks.
template <int VEC, int F, int PD, class Src>
__device__ __forceinline__ void k2s_block(K2Rows<VEC, F, PD>& q, const Src& coef, int i, int J, int h_l, int w_l) {
    float a[VEC], b[VEC];
    k2s_hrow_from<VEC, F>(q.next[0], a, b);  // row min(i + 1, h_l - 1)
#pragma unroll
    for (int d = 0; d + 1 < PD; ++d)
#pragma unroll
        for (int c = 0; c < VEC / F + 2; ++c) q.next[d][c] = q.next[d + 1][c];
    k2s_taps<VEC, F>(coef, min(i + 1 + PD, h_l - 1), J, w_l, q.next[PD - 1]);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        q.DA[k] = a[k] - q.A1[k];
        q.DB[k] = b[k] - q.B1[k];
        q.A1[k] = a[k];
        q.B1[k] = b[k];
    }
}

// O_h at row t of the block: lerp along y written from the second row,
// A1 + (lam_y - 1) DA with lam_y = (2t + 1) / 2F.
template <int VEC, int F, int PD>
__device__ __forceinline__ void k2s_row(const K2Rows<VEC, F, PD>& q, const float (&g)[VEC], int t, float (&o)[VEC]) {
    const float lm1 = (float)(2 * t + 1 - 2 * F) / (float)(2 * F);
#pragma unroll
    for (int k = 0; k < VEC; ++k) o[k] = fmaf(fmaf(lm1, q.DA[k], q.A1[k]), g[k], fmaf(lm1, q.DB[k], q.B1[k]));
}

struct K2Lane {
    int J, x0;
    bool full, any;
};

template <int VEC, int F>
__device__ __forceinline__ K2Lane k2s_lane(int strip, int w_l) {
    constexpr int K = VEC / F;
    K2Lane L;
    L.J = 32 * K * strip + (int)(threadIdx.x & 31) * K;
    L.x0 = F * L.J;
    L.full = L.J + K <= w_l;
    L.any = L.J < w_l;
    return L;
}

template <typename T, int VEC>
__device__ __forceinline__ void k2s_store(T* __restrict__ out, int y, int w, const K2Lane& L, const float (&o)[VEC]) {
    if (L.full) {
        store_vec<T, VEC>(out + (size_t)y * w + L.x0, o);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if (L.x0 + k < w) out[(size_t)y * w + L.x0 + k] = from_f32<T>(o[k]);
    }
}

template <typename T, int VEC, int F>
struct K2Tma {
    static constexpr int ROW = 32 * VEC;
    static constexpr int NSB = F == 2 ? 8 : (F == 4 ? 4 : 2);   // slots (blocks) per warp
    static constexpr int WPC = 8;                               // warps per CTA
    static constexpr int SLOT = ROW * F * (int)sizeof(T);
    static constexpr size_t CTA_BYTES = (size_t)WPC * NSB * SLOT + (size_t)WPC * NSB * 8;
};

// Same walk with the input rows staged per block by TMA (16-byte vectors).
// Returns false after a timeout (recorded in the status word); on success
// the slot barriers are invalidated, so a persistent warp can call it again
// with the same ring.
template <typename T, int VEC, int F>
__device__ bool k2_strip_tma(const float2* __restrict__ coef, const CUtensorMap* map, T* __restrict__ out, int h_l,
                             int w_l, int h, int w, int strip, int ia, int ib, int plane, unsigned char* ring,
                             uint64_t* bars, uint32_t* status) {
    using B = K2Tma<T, VEC, F>;
    static_assert(VEC * sizeof(T) == 16, "TMA staging needs 16-byte vectors");
    constexpr int NSB = B::NSB, H0 = F / 2;
    const int lane = threadIdx.x & 31;
    const K2Lane L = k2s_lane<VEC, F>(strip, w_l);
    const int b0 = ia == 0 ? -1 : ia;
    const int nblk = ib - b0;
    const int xs = B::ROW * strip;
    const uint32_t ring_s = smem_u32(ring), bar_s = smem_u32(bars);
    auto issue = [&](int m) {  // lane 0: block b0 + m into slot m % NSB
        const int slot = m % NSB;
        const uint32_t bar = bar_s + 8u * slot;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)B::SLOT)
                     : "memory");
        tma_load_3d(ring_s + (uint32_t)(slot * B::SLOT), map, xs, F * (b0 + m) + H0, plane, bar);
    };
    __syncwarp();  // a previous walk's reads of the ring are done
    if (lane == 0) {
        for (int s = 0; s < NSB; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int m = 0; m < min(NSB, nblk); ++m) issue(m);
    }
    __syncwarp();
    K2Rows<VEC, F> q;
    k2s_init<VEC, F>(q, CoefIn{coef, w_l}, b0, L.J, h_l, w_l);
    int m = 0;
    bool ok = true;
    for (; m < nblk; ++m) {
        const int slot = m % NSB;
        const int i = b0 + m;
        k2s_block<VEC, F>(q, CoefIn{coef, w_l}, i, L.J, h_l, w_l);
        if (!__all_sync(0xffffffffu, mbar_wait(bar_s + 8u * slot, (uint32_t)((m / NSB) & 1), first_wait_limit(status)))) {
            ok = false;
            break;
        }
        const T* sr = reinterpret_cast<const T*>(ring + slot * B::SLOT) + lane * VEC;
#pragma unroll
        for (int t = 0; t < F; ++t) {
            float g[VEC];
            unpack_vec<T, VEC>(*reinterpret_cast<const Vec<T, VEC>*>(sr + t * B::ROW), g);
            if (t == F - 1) {
                __syncwarp();  // every lane has read the slot
                if (lane == 0 && m + NSB < nblk) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(m + NSB);
                }
            }
            const int y = F * i + H0 + t;
            if (L.any && y >= 0 && y < h) {
                float o[VEC];
                k2s_row<VEC, F>(q, g, t, o);
                k2s_store<T, VEC>(out, y, w, L, o);
            }
        }
    }
    if (!ok) {
        if (lane == 0) status_fail(status, kStatusTimeout);
        for (int qb = m; qb < nblk && qb < m + NSB; ++qb)
            mbar_wait(bar_s + 8u * (qb % NSB), (uint32_t)((qb / NSB) & 1), kWaitLimit);
        return false;
    }
    __syncwarp();  // every lane has passed its last wait
    if (lane == 0)
        for (int s = 0; s < NSB; ++s) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar_s + 8u * s) : "memory");
    return true;
}

// Same walk with the input rows staged by per-lane asynchronous copies
// (cp.async, 16 or 8 bytes per lane and row, zero-filled outside the image)
// into a per-warp ring of NSB blocks, one commit group per block; no tensor
// map is needed, so the persistent batched kernel uses this form.  Each lane
// reads back only what it copied, so no barrier is involved.
template <typename T, int VEC, int F>
struct K2Async {
    static constexpr int ROW = 32 * VEC;
    static constexpr int NSB = F == 2 ? 6 : (F == 4 ? 3 : 2);
    static constexpr int SLOT = ROW * F * (int)sizeof(T);
    static constexpr size_t WARP_BYTES = (size_t)NSB * SLOT;
};

template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(uint32_t dst, const void* src, bool ok) {
    const uint32_t n = ok ? BYTES : 0;  // 0 source bytes: the destination is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES), "r"(n)
                 : "memory");
}

template <typename T, int VEC, int F>
__device__ void k2_strip_async(const float2* __restrict__ coef, const T* __restrict__ in, T* __restrict__ out,
                               int h_l, int w_l, int h, int w, int strip, int ia, int ib, unsigned char* ring) {
    using B = K2Async<T, VEC, F>;
    constexpr int NSB = B::NSB, H0 = F / 2, VB = VEC * (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const K2Lane L = k2s_lane<VEC, F>(strip, w_l);
    const int b0 = ia == 0 ? -1 : ia;
    const int nblk = ib - b0;
    const uint32_t mine = smem_u32(ring) + (uint32_t)(lane * VB);
    auto issue = [&](int m) {  // this lane's vectors of block b0 + m (partial lanes copy zeros; handled below)
        const uint32_t dst = mine + (uint32_t)((m % NSB) * B::SLOT);
#pragma unroll
        for (int t = 0; t < F; ++t) {
            const int y = F * (b0 + m) + H0 + t;
            const bool ok = L.full && y >= 0 && y < h;
            cp_async_zfill<VB>(dst + (uint32_t)(t * B::ROW * (int)sizeof(T)),
                               ok ? (const void*)(in + (size_t)y * w + L.x0) : (const void*)in, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int m = 0; m < NSB; ++m) {
        if (m < nblk) issue(m);
        else asm volatile("cp.async.commit_group;" ::: "memory");  // keep the group count uniform
    }
    K2Rows<VEC, F> q;
    k2s_init<VEC, F>(q, CoefIn{coef, w_l}, b0, L.J, h_l, w_l);
    for (int m = 0; m < nblk; ++m) {
        const int i = b0 + m;
        k2s_block<VEC, F>(q, CoefIn{coef, w_l}, i, L.J, h_l, w_l);
        asm volatile("cp.async.wait_group %0;" ::"n"(NSB - 1) : "memory");
        const T* sr = reinterpret_cast<const T*>(ring + (m % NSB) * B::SLOT) + lane * VEC;
#pragma unroll
        for (int t = 0; t < F; ++t) {
            const int y = F * i + H0 + t;
            float g[VEC];
            if (L.full) {
                unpack_vec<T, VEC>(*reinterpret_cast<const Vec<T, VEC>*>(sr + t * B::ROW), g);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    g[k] = (L.any && y >= 0 && y < h && L.x0 + k < w) ? to_f32<T>(in[(size_t)y * w + L.x0 + k]) : 0.f;
            }
            if (L.any && y >= 0 && y < h) {
                float o[VEC];
                k2s_row<VEC, F>(q, g, t, o);
                k2s_store<T, VEC>(out, y, w, L, o);
            }
        }
        // the slot is read: refill it with block m + NSB (or an empty group)
        if (m + NSB < nblk) issue(m + NSB);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace dgf
