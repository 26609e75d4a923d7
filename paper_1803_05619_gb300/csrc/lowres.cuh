// Low-resolution stage of the guided filtering layer: window statistics,
// the local linear model and its box mean (forward), and the recomputation
// plus Algorithm 1's low-resolution gradient steps (backward).
//
// One CTA owns a TY x TX tile of one plane.  The tile's inputs plus a 2r
// halo are staged in shared memory (by TMA when the tensor-map alignment
// rules allow, else by coalesced loads; both leave identical contents), and
// every window sum is a separable pass over shared memory:
//   * E2 = tile + 2r ring: staged inputs;
//   * E1 = tile + r ring:  A, b (their box mean reaches r outside the tile);
//   * E0 = tile:           outputs.
// Windows are clipped to the image and divided by the in-image count.
#pragma once

#include "common.cuh"

namespace dgf {

struct LowresTile {
    int h, w, r;     // low-res plane size and radius
    int ty0, tx0;    // tile origin
    int TY, TX;      // tile size
    int EY2, EX2;    // staged region (TY + 4r) x (TX + 4r)
    int EY1, EX1;    // coefficient region (TY + 2r) x (TX + 2r)
    float eps;
    int mean;        // 1: box mean of A, b; 0: A, b themselves (the layer as printed)

    __device__ __forceinline__ void init(int h_, int w_, int r_, float eps_, int ty0_, int tx0_,
                                         int TY_, int TX_) {
        h = h_; w = w_; r = r_; eps = eps_; ty0 = ty0_; tx0 = tx0_; TY = TY_; TX = TX_; mean = 1;
        EY2 = TY + 4 * r; EX2 = TX + 4 * r; EY1 = TY + 2 * r; EX1 = TX + 2 * r;
    }
    // number of in-image samples of the clipped 1-D window [c - r, c + r]
    __device__ __forceinline__ int cnt(int c, int n) const {
        return min(c + r, n - 1) - max(c - r, 0) + 1;
    }
};

// Stage one plane's (TY+4r) x (TX+4r) halo tile as FP32 (zero outside the image).
template <typename T>
__device__ __forceinline__ void stage_plane(const T* __restrict__ src, float* dst, const LowresTile& t) {
    const int n = t.EY2 * t.EX2;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
        const int ey = idx / t.EX2, ex = idx - ey * t.EX2;
        const int gy = t.ty0 - 2 * t.r + ey, gx = t.tx0 - 2 * t.r + ex;
        float v = 0.f;
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) v = to_f32<T>(src[(size_t)gy * t.w + gx]);
        dst[idx] = v;
    }
}

// Horizontal pass of the centred statistics.  For every row of E2 and every
// column of E1: the clipped row segment's means (mg, mp) and its centred
// sums sgg = sum (g - mg)^2, sgp = sum (g - mg)(p - mp)  (two passes).
__device__ __forceinline__ void stats_rows(const float* sG, const float* sP, float* hMG, float* hMP,
                                           float* hSGG, float* hSGP, const LowresTile& t) {
    const int n = t.EY2 * t.EX1;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
        const int ey = idx / t.EX1, ex = idx - ey * t.EX1;
        const int gy = t.ty0 - 2 * t.r + ey, gx = t.tx0 - t.r + ex;
        float mg = 0.f, mp = 0.f, sgg = 0.f, sgp = 0.f;
        if (gy >= 0 && gy < t.h && gx >= 0 && gx < t.w) {
            const int lo = max(gx - t.r, 0), hi = min(gx + t.r, t.w - 1);
            const float* g = sG + ey * t.EX2 + (lo - (t.tx0 - 2 * t.r));
            const float* p = sP + ey * t.EX2 + (lo - (t.tx0 - 2 * t.r));
            const int len = hi - lo + 1;
            float s1 = 0.f, s2 = 0.f;
            for (int k = 0; k < len; ++k) { s1 += g[k]; s2 += p[k]; }
            const float inv = 1.f / (float)len;
            mg = s1 * inv;
            mp = s2 * inv;
            for (int k = 0; k < len; ++k) {
                const float dg = g[k] - mg;
                sgg = fmaf(dg, dg, sgg);
                sgp = fmaf(dg, p[k] - mp, sgp);
            }
        }
        hMG[idx] = mg; hMP[idx] = mp; hSGG[idx] = sgg; hSGP[idx] = sgp;
    }
}

// Vertical pass: combine the clipped column of row segments into the window
// moments (Chan's pairwise update, every term centred):
//   mu = mean of segment means, var N = sum sgg + nx sum (mg - mu)^2,
//   cov N = sum sgp + nx sum (mg - mu)(mp - nu).
// Returns in-image flag; outputs mu, nu, var, cov of window (gy, gx).
struct Moments {
    float mu, nu, var, cov;
    int n;
};

__device__ __forceinline__ Moments stats_window(const float* hMG, const float* hMP, const float* hSGG,
                                                const float* hSGP, int ey1, int ex,
                                                const LowresTile& t) {
    const int gy = t.ty0 - t.r + ey1, gx = t.tx0 - t.r + ex;
    const int lo = max(gy - t.r, 0), hi = min(gy + t.r, t.h - 1);
    const int ny = hi - lo + 1, nx = t.cnt(gx, t.w);
    const int e0 = lo - (t.ty0 - 2 * t.r);
    float s1 = 0.f, s2 = 0.f;
    for (int k = 0; k < ny; ++k) {
        s1 += hMG[(e0 + k) * t.EX1 + ex];
        s2 += hMP[(e0 + k) * t.EX1 + ex];
    }
    const float invy = 1.f / (float)ny;
    Moments m;
    m.mu = s1 * invy;
    m.nu = s2 * invy;
    float sgg = 0.f, sgp = 0.f, dgg = 0.f, dgp = 0.f;
    for (int k = 0; k < ny; ++k) {
        const int o = (e0 + k) * t.EX1 + ex;
        const float dg = hMG[o] - m.mu;
        sgg += hSGG[o];
        sgp += hSGP[o];
        dgg = fmaf(dg, dg, dgg);
        dgp = fmaf(dg, hMP[o] - m.nu, dgp);
    }
    const float fx = (float)nx;
    m.n = nx * ny;
    const float invn = 1.f / (float)m.n;
    m.var = fmaf(fx, dgg, sgg) * invn;
    m.cov = fmaf(fx, dgp, sgp) * invn;
    return m;
}

// Box sum of `src` (pitch sp, region rows x cols with origin (oy, ox) in
// image coordinates) along x with radius r, clipped to the image; output
// for columns [dx0, dx0 + dcols) of the same rows.  Values outside the image
// must be zero in src; the clip only saves reads.
__device__ __forceinline__ void box_rows(const float* src, int sp, int rows, int ox, float* dst,
                                         int dp, int dx0, int dcols, int w, int r) {
    const int n = rows * dcols;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
        const int y = idx / dcols, x = idx - y * dcols;
        const int gx = dx0 + x;
        float s = 0.f;
        if (gx >= 0 && gx < w) {
            const int lo = max(gx - r, 0), hi = min(gx + r, w - 1);
            const float* p = src + y * sp + (lo - ox);
            for (int k = 0; k <= hi - lo; ++k) s += p[k];
        }
        dst[y * dp + x] = s;
    }
}

}  // namespace dgf
