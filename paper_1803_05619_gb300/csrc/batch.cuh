// Descriptor table of a batched call: passed by value as one kernel
// parameter (__grid_constant__), so a CUDA-graph replay updates it in place
// with cudaGraphExecKernelNodeSetParams and no device copy.
#pragma once

#include "../../include/dgf.h"

namespace dgf {

struct BatchImage {
    const void* p_l;
    const void* I_l;
    const void* I_h;
    void* O_h;
    float2* coef;     // Abar, bbar of this image (C planes), in the workspace
    int C, h_l, w_l, h, w, r;
    float eps;
    int F;            // integer upsampling factor, 0 = general ratio
    int vec;          // elements per vector access of the high-res pass
    int k1_fast;      // 1: column-walking kernel (k1_ty = EY1, k1_tx = CW), 0: generic tile
    int k1_ty, k1_tx; // low-res tile
    int k2_th;        // high-res rows per tile
    int k1_nx, k1_ny; // low-res tiles per plane
    int k2_nx, k2_ny; // high-res tiles per plane
};

struct BatchParams {
    int n;
    int k1_total, k2_total;
    int k1_start[DGF_MAX_BATCH + 1];  // prefix sums of tiles (all planes) per image
    int k2_start[DGF_MAX_BATCH + 1];
    BatchImage img[DGF_MAX_BATCH];
};

static_assert(sizeof(BatchParams) < 32000, "kernel parameter limit");

// image owning flat tile t: largest i with start[i] <= t
__device__ __forceinline__ int batch_find(const int* start, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace dgf
