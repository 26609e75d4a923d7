// Host-side launchers of the guided-filtering kernels (internal interface
// between the C ABI in api.cu and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <initializer_list>

#include "../../include/dgf.h"

namespace dgf {

struct TmaPair;
struct TmaTriple;
struct K3Maps;
struct K2Map;
constexpr int kStripWarpsPerCta = 8;

// Shared-memory pitch (float2 columns) of a K2 tile row.
__host__ __device__ inline int k2_pitch(int vec, int F, int w_l, int w) {
    const int TW = 32 * vec;
    if (F > 0) return TW / F + 2;
    const long long span = ((long long)TW * w_l + w - 1) / w;
    return (int)span + 3;
}

// Low-resolution tile configuration: fast = 1: column-walking tile kernels
// (r in {1, 2, 4, 8}; a = CW columns, b = EY1 rows of the coefficient
// region); fast = 2: warp-strip K1 (r in {1, 2}; a = rows per segment,
// b = 0); fast = 3: sliding-sum warp strips for 16-bit storage (r in
// {1, 2, 4, 8}; a = output rows per segment, 0 = slide_auto_seg; b = columns
// per lane V); fast = 0: generic tile kernels (a = TY, b = TX output tile).
struct LowCfg {
    int fast;
    int a, b;
    int mean = 1;  // 1: box mean of A, b (fast guided filter); 0: A_l, b_l as Sec. 3.2 prints them
};

// Sliding-sum strips (lowres_slide.cuh): radii built, default columns per
// lane, default output rows per segment (a function of the plane height and
// r only, so a plane's bits do not depend on how many planes a call holds),
// output columns per strip.
bool slide_radius(int r);
int slide_k1_v(int r);
int slide_k4_v(int r);
bool slide_v_built(int r, int V, bool k4);
int slide_auto_seg(int h, int r);
int slide_out_cols(int r, int V);
size_t k1_slide_smem_bytes(int r, int V, int warps);
template <int R>
cudaError_t launch_k1_slide_r(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes, int h,
                              int w, float eps, int S, int V, cudaStream_t s);
template <int R>
cudaError_t launch_k4_slide_r(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP,
                              void* dG, int planes, int h, int w, float eps, int S, int V, cudaStream_t s);
extern template cudaError_t launch_k1_slide_r<1>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                                 float, int, int, cudaStream_t);
extern template cudaError_t launch_k1_slide_r<2>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                                 float, int, int, cudaStream_t);
extern template cudaError_t launch_k1_slide_r<4>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                                 float, int, int, cudaStream_t);
extern template cudaError_t launch_k1_slide_r<8>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                                 float, int, int, cudaStream_t);
extern template cudaError_t launch_k4_slide_r<1>(dgf_dtype, bool, const void*, const void*, const float2*, void*,
                                                 void*, int, int, int, float, int, int, cudaStream_t);
extern template cudaError_t launch_k4_slide_r<2>(dgf_dtype, bool, const void*, const void*, const float2*, void*,
                                                 void*, int, int, int, float, int, int, cudaStream_t);
extern template cudaError_t launch_k4_slide_r<4>(dgf_dtype, bool, const void*, const void*, const float2*, void*,
                                                 void*, int, int, int, float, int, int, cudaStream_t);
extern template cudaError_t launch_k4_slide_r<8>(dgf_dtype, bool, const void*, const void*, const float2*, void*,
                                                 void*, int, int, int, float, int, int, cudaStream_t);

size_t k1_smem_bytes(int r, int TY, int TX);
size_t k4_smem_bytes(int r, int TY, int TX);
bool low_fast_radius(int r);
size_t k1_fast_smem_bytes(int r, int CW, int EY1, size_t tma_landing);
size_t k4_fast_smem_bytes(int r, int CW, int EY1);
size_t k1_cfg_smem(const LowCfg& c, int r, size_t tma_landing);
size_t k4_cfg_smem(const LowCfg& c, int r);
void low_grid(const LowCfg& c, int r, int h, int w, int& gx, int& gy);
size_t k2_smem_bytes(int vec, int F, int h_l, int h, int w_l, int w, int TH);
bool k3_fast_ok(int vec, int F);

cudaError_t launch_k1(dgf_dtype dt, bool guide_f32, const void* G, const void* P, float2* coef, int planes,
                      int h, int w, int r, float eps, const LowCfg& c, const TmaPair& tma, size_t smem,
                      uint32_t* status, float4* stats, cudaStream_t s);
cudaError_t launch_k4(dgf_dtype dt, bool guide_f32, const void* G, const void* P, const float2* dcoef,
                      void* dP, void* dG, int planes, int h, int w, int r, float eps, const LowCfg& c,
                      const TmaTriple* tma, uint32_t* status, const float4* stats, cudaStream_t s);
// K2 as warp strips (mode 0, integer F in {2, 4, 8} dividing vec); LS =
// low-res rows per segment; map: TMA staging of `in` (16-byte vectors) or null.
bool k2_strip_ok(int vec, int F);
// shared memory of the persistent batched K2 in strip form (its slot rings)
size_t k2_strip_batched_smem(int esize, int vec, int F);
cudaError_t launch_k2_strip(dgf_dtype dt, const float2* coef, const void* in, void* out, int planes, int h_l,
                            int w_l, int h, int w, int vec, int F, int LS, const K2Map* map, uint32_t* status,
                            cudaStream_t s);
cudaError_t launch_k2(dgf_dtype dt, int mode, const float2* coef, const void* in, void* out, int planes,
                      int h_l, int w_l, int h, int w, int vec, int F, int TH, cudaStream_t s);
cudaError_t launch_k3(dgf_dtype dt, const float2* coef, const void* R, const void* G, void* dG,
                      float2* dcoef, int planes, int h_l, int w_l, int h, int w, int vec, int F, int LS,
                      const K3Maps* maps, uint32_t* status, cudaStream_t s);
// guide_f32: G is FP32 while R is stored in dt (a grey guide over 16-bit data)
cudaError_t launch_k3_general(dgf_dtype dt, const void* R, const void* G, float2* dcoef, int planes,
                              int h_l, int w_l, int h, int w, cudaStream_t s, bool guide_f32 = false);
// K2 tiles (MODE 0) with an FP32 guide and O_h stored in dt
cudaError_t launch_k2_guide_f32(dgf_dtype dt, const float2* coef, const float* in, void* out, int planes, int h_l,
                                int w_l, int h, int w, int vec, int F, int TH, cudaStream_t s);

// Fused forward (K1 + K2 in one kernel per high-res warp strip; r in {1, 2};
// one low-res cell per lane: F-pixel vectors of 8 or 16 bytes).  LS =
// low-res rows per segment.  in/out must be aligned to k12_vec_bytes.
bool k12_supported(dgf_dtype dt, int r, int F);
int k12_vec_bytes(dgf_dtype dt, int F);
cudaError_t launch_k12(dgf_dtype dt, const void* G, const void* P, const void* in, void* out, int planes, int h_l,
                       int w_l, int h, int w, int r, int F, float eps, int LS, cudaStream_t s);

// Fused backward K1 + K3 (r in {1, 2}; K3 strips of 16-byte vectors with one
// low-res cell per lane: F32 F = 4, BF16/F16 F = 8, vec == F); `maps` the K3
// tensor maps of d O_h and the guide; stats: the window statistics of every
// cell for K4 (or null).  LS = low-res rows per segment.
bool k13_supported(dgf_dtype dt, int r, int F, int vec);
cudaError_t launch_k13(dgf_dtype dt, const void* G, const void* P, const K3Maps& maps, void* dG, float2* dcoef,
                       float4* stats, int planes, int h_l, int w_l, int h, int w, int r, int F, float eps, int LS,
                       uint32_t* status, cudaStream_t s);

// Guidance transform (Sec. 3.4): weights staged to constant memory first.
constexpr int kMaxK6Blocks = 1024;   // rows of weight-gradient partials
constexpr int kWGradPadded = 99;     // padded [dw1 16x3 | dw2 3x16 | db2 3]
cudaError_t guide_upload(const float* w1, const float* w2, const float* b2, int hidden, cudaStream_t s);
bool guided_supported(dgf_dtype dt, int w, int F);
// G_h (or null): F(I_h) of every high-res pixel, FP32, also written there
cudaError_t launch_k5(dgf_dtype dt, const void* I_h, float* G_l, int N, int h_l, int w_l, int h, int w,
                      int F, float slope, cudaStream_t s, float* G_h = nullptr);
cudaError_t launch_k2_guided(dgf_dtype dt, const float2* coef, const void* I_h, void* O_h, int N,
                             int h_l, int w_l, int h, int w, int F, int TH, float slope, cudaStream_t s);
// G_h (or null): F(I_h) in FP32 as the forward's K5 kept it, read instead of evaluating F
cudaError_t launch_k3_guided(dgf_dtype dt, const void* R, const void* I_h, float2* dcoef, int N,
                             int h_l, int w_l, int h, int w, int F, float slope, cudaStream_t s,
                             const float* G_h = nullptr);
// F applied to the low-res guide itself (G_l = F(I_l), I_l: N x 3 x h_l x w_l):
// K5L forms G_l (FP32); K6L chains d G_l through F to d I_l (nullable) and
// writes k6_low_blocks(...) weight-gradient partial rows from `partials`.
cudaError_t launch_k5_low(dgf_dtype dt, const void* I_l, float* G_l, int N, int h_l, int w_l, float slope,
                          cudaStream_t s);
int k6_low_blocks(int N, int h_l, int w_l);
cudaError_t launch_k6_low(dgf_dtype dt, const float* dG_l, const void* I_l, void* dI_l, float* partials, int N,
                          int h_l, int w_l, float slope, cudaStream_t s);
int k6_blocks(int N, int h, int w);
cudaError_t launch_k6(dgf_dtype dt, const float2* coef, const float* dG_l, const void* R, const void* I_h,
                      void* dI_h, float* partials, int N, int h_l, int w_l, int h, int w, int F, float slope,
                      cudaStream_t s);
cudaError_t launch_wreduce(const float* partials, int nblocks, float* dW, int hidden, cudaStream_t s);

// Grey guide (channel mean of an n_in-channel guide, Sec. 4.2, DGF_b): G
// (N x C planes, FP32) = the mean of I's n_in planes of each image (stored in
// dt), repeated C times; and its adjoint d I (N x n_in planes) = the sum of
// d G's C planes / n_in, repeated n_in times (both in dt).  `plane` = pixels
// per plane.
cudaError_t launch_grey_mean(dgf_dtype dt, const void* I, float* G, int N, int n_in, int C, size_t plane,
                             cudaStream_t s);
// src_f32: d G is FP32 (else stored in dt)
cudaError_t launch_grey_adjoint(dgf_dtype dt, bool src_f32, const void* dG, void* dI, int N, int n_in, int C,
                                size_t plane, cudaStream_t s);
// The high-resolution kernels with the grey guide formed in registers from
// I_h's n_in channels (integer factor F; N images of C output channels).
// grey_fold_vec: the vector width they use for these sizes and pointers, or
// 0 when they do not serve them.  K2grey writes O_h; K3grey writes d Abar,
// d bbar (dcoef) and, when dI_h is not null, d I_h (n_in planes per image)
// from Abar (coef).
int grey_fold_vec(dgf_dtype dt, int F, int C, int w, std::initializer_list<const void*> ptrs);
cudaError_t launch_k2_grey(dgf_dtype dt, const float2* coef, const void* I_h, void* O_h, int N, int C, int n_in,
                           int h_l, int w_l, int h, int w, int F, int vec, cudaStream_t s);
cudaError_t launch_k3_grey(dgf_dtype dt, const void* R, const void* I_h, const float2* coef, float2* dcoef,
                           void* dI_h, int N, int C, int n_in, int h_l, int w_l, int h, int w, int F, int vec,
                           cudaStream_t s);

// Column-walking low-resolution kernels, one translation unit per radius.
template <int R>
cudaError_t launch_k1_fast(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes,
                           int h, int w, float eps, const LowCfg& c, const TmaPair& tma, size_t smem,
                           uint32_t* status, float4* stats, cudaStream_t s);
template <int R>
cudaError_t launch_k4_fast(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP,
                           void* dG, int planes, int h, int w, float eps, const LowCfg& c, const TmaTriple* tma,
                           uint32_t* status, const float4* stats, cudaStream_t s);
extern template cudaError_t launch_k1_fast<1>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                              float, const LowCfg&, const TmaPair&, size_t, uint32_t*, float4*, cudaStream_t);
extern template cudaError_t launch_k1_fast<2>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                              float, const LowCfg&, const TmaPair&, size_t, uint32_t*, float4*, cudaStream_t);
extern template cudaError_t launch_k1_fast<4>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                              float, const LowCfg&, const TmaPair&, size_t, uint32_t*, float4*, cudaStream_t);
extern template cudaError_t launch_k1_fast<8>(dgf_dtype, bool, const void*, const void*, float2*, int, int, int,
                                              float, const LowCfg&, const TmaPair&, size_t, uint32_t*, float4*, cudaStream_t);
extern template cudaError_t launch_k4_fast<1>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*,
                                              int, int, int, float, const LowCfg&, const TmaTriple*, uint32_t*, const float4*,
                                              cudaStream_t);
extern template cudaError_t launch_k4_fast<2>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*,
                                              int, int, int, float, const LowCfg&, const TmaTriple*, uint32_t*, const float4*,
                                              cudaStream_t);
extern template cudaError_t launch_k4_fast<4>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*,
                                              int, int, int, float, const LowCfg&, const TmaTriple*, uint32_t*, const float4*,
                                              cudaStream_t);
extern template cudaError_t launch_k4_fast<8>(dgf_dtype, bool, const void*, const void*, const float2*, void*, void*,
                                              int, int, int, float, const LowCfg&, const TmaTriple*, uint32_t*, const float4*,
                                              cudaStream_t);

// Persistent kernels of the batched backward (batch_bwd.cuh), 16-bit storage:
// K3 strips per (vector width, factor, TMA staging or plain loads); sliding K4 per (radius, columns per
// lane), with the dynamic shared memory and threads of its CTA.
cudaError_t k3_batched_kernel(dgf_dtype dt, int vec, int F, bool tma, void** fn, size_t* smem, int* threads);
cudaError_t k4_batched_kernel(dgf_dtype dt, int r, int V, void** fn, size_t* smem, int* threads);
int slide_out_cols(int r, int V);

// Persistent batched kernels (function pointers for graph nodes).
// V: columns per lane of the sliding form (mode 3), else ignored; threads:
// the CTA size of the kernel (the sliding form's single-call warps per CTA,
// else kThreads), if not null
cudaError_t k1_batched_kernel(dgf_dtype dt, int r, int mode, size_t smem, void** fn, int V = 0,
                              int* threads = nullptr);
int k1_slide_batched_wpc(int r, int V);
cudaError_t k2_batched_kernel(dgf_dtype dt, int vec, int F, size_t smem, void** fn);
// K2 strips staged by TMA (16-byte vectors, integer F dividing vec): the
// kernel, its dynamic shared memory and threads per CTA
cudaError_t k2_batched_tma_kernel(dgf_dtype dt, int vec, int F, void** fn, size_t* smem, int* threads);

}  // namespace dgf
