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
    const void* k2_map; // K2Map of I_h in device memory (TMA-staged strips), or null
};

struct BatchParams {
    int n;
    int k1_total, k2_total;
    int k1_start[DGF_MAX_BATCH + 1];  // prefix sums of tiles (all planes) per image
    int k2_start[DGF_MAX_BATCH + 1];
    BatchImage img[DGF_MAX_BATCH];
};

static_assert(sizeof(BatchParams) < 32000, "kernel parameter limit");

// One image of the batched backward (16-bit storage): its K3 strip walk and
// sliding K4 work lists.
struct BwdImage {
    const void* dO;       // d O_h (C planes)
    const void* p_l;      // P
    const void* I_l;      // G_l
    const void* I_h;      // G_h
    void* dp;             // d p_l (nullable)
    void* dIl;            // d I_l (nullable)
    void* dIh;            // d I_h (nullable)
    const float2* coef;   // Abar, bbar (from the K1 stage)
    float2* dcoef;        // d Abar, d bbar (K3 writes, K4 reads)
    int C, h_l, w_l, h, w;
    float eps;
    int k3_ls, k3_nx;     // K3: low-res rows per segment; work items per plane
    int k4_S, k4_nx;      // K4: output rows per segment; work items per plane
    int k4_aligned, k4_pairs;
    const void* k3_maps;  // K3Maps of d O_h and G_h in device memory (TMA staging), or null: plain loads
};

struct BwdParams {
    int n;
    int total;
    int start[DGF_MAX_BATCH + 1];  // prefix sums of work items (all planes) per image
    BwdImage img[DGF_MAX_BATCH];
};

static_assert(sizeof(BwdParams) < 32000, "kernel parameter limit");

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
