// Generic-radius tile of K1 (any r up to the shared-memory limit), shared by
// the per-call kernel and the persistent batched kernel.
#pragma once

#include "lowres.cuh"
#include "tma.cuh"

namespace dgf {

// --------------------------------------------------------------------- K1
// Eq. 1 (least-squares A, b per window, Sec. 3.2) followed by the box mean
// of A and b (Sec. 3.3's f_mu applied once more at low resolution).
template <typename TG, typename TP>
__device__ void coef_tile(const TG* __restrict__ G, const TP* __restrict__ P,
                          float2* __restrict__ coef, const LowresTile& t, float* smem,
                          const TmaPlane* tg, const TmaPlane* tp, int plane, uint32_t* status) {
    const int n2 = t.EY2 * t.EX2;
    float* sG = smem;
    float* sP = sG + n2;
    float* hbuf = sP + n2;
    bool staged = false;
    if (tg != nullptr && tp != nullptr)
        staged = tma_stage_pair<TG, TP>(tg, tp, plane, t, sG, sP, hbuf, status);
    if (!staged) {
        stage_plane<TG>(G, sG, t);
        stage_plane<TP>(P, sP, t);
    }
    __syncthreads();
    const int nh = t.EY2 * t.EX1;
    stats_rows(sG, sP, hbuf, hbuf + nh, hbuf + 2 * nh, hbuf + 3 * nh, t);
    __syncthreads();
    // A, b on E1 (zero outside the image); the staged inputs are dead now
    const int n1 = t.EY1 * t.EX1;
    float* sA = smem;
    float* sB = smem + n1;
    for (int idx = threadIdx.x; idx < n1; idx += kThreads) {
        const int ey1 = idx / t.EX1, ex = idx - ey1 * t.EX1;
        const int gy = t.ty0 - t.r + ey1, gx = t.tx0 - t.r + ex;
        float A = 0.f, b = 0.f;
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const Moments m = stats_window(hbuf, hbuf + nh, hbuf + 2 * nh, hbuf + 3 * nh, ey1, ex, t);
            A = m.cov / (m.var + t.eps);
            b = fmaf(-A, m.mu, m.nu);
        }
        sA[idx] = A;
        sB[idx] = b;
    }
    __syncthreads();
    if (!t.mean) {
        // no box mean: the output pixels' own A, b (the layer as Sec. 3.2 prints it)
        for (int idx = threadIdx.x; idx < t.TY * t.TX; idx += kThreads) {
            const int y = idx / t.TX, x = idx - y * t.TX;
            const int gy = t.ty0 + y, gx = t.tx0 + x;
            if (gy >= t.h || gx >= t.w) continue;
            const int o = (y + t.r) * t.EX1 + x + t.r;
            coef[(size_t)gy * t.w + gx] = make_float2(sA[o], sB[o]);
        }
        __syncthreads();
        return;
    }
    float* rA = hbuf;
    float* rB = hbuf + t.EY1 * t.TX;
    box_rows(sA, t.EX1, t.EY1, t.tx0 - t.r, rA, t.TX, t.tx0, t.TX, t.w, t.r);
    box_rows(sB, t.EX1, t.EY1, t.tx0 - t.r, rB, t.TX, t.tx0, t.TX, t.w, t.r);
    __syncthreads();
    const int n0 = t.TY * t.TX;
    for (int idx = threadIdx.x; idx < n0; idx += kThreads) {
        const int y = idx / t.TX, x = idx - y * t.TX;
        const int gy = t.ty0 + y, gx = t.tx0 + x;
        if (gy >= t.h || gx >= t.w) continue;
        const int lo = max(gy - t.r, 0), hi = min(gy + t.r, t.h - 1);
        float sa = 0.f, sb = 0.f;
        for (int k = lo; k <= hi; ++k) {
            const int o = (k - (t.ty0 - t.r)) * t.TX + x;
            sa += rA[o];
            sb += rB[o];
        }
        const float n = (float)((hi - lo + 1) * t.cnt(gx, t.w));
        coef[(size_t)gy * t.w + gx] = make_float2(sa / n, sb / n);
    }
    __syncthreads();
}

}  // namespace dgf
