// Shared device helpers of the guided-filtering kernels: storage-type
// conversion, vector access and the bilinear source coordinate.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgf {

constexpr int kThreads = 256;  // threads per CTA of every tiled kernel
constexpr int kWarps = kThreads / 32;

// ------------------------------------------------------------ reciprocals
// 1/x from the special-function unit (PTX rcp.approx.ftz.f32: relative error
// within about one unit in the last place; subnormal arguments flush to
// zero).  Used for 1/(var + eps): var >= 0 and eps >= FLT_MIN (checked at the
// entry points) keep the argument normal.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------ paired FP32
// Two values per register pair (a 64-bit f32x2: low half, high half), as the
// two-column strips hold their columns.  The arithmetic on a pair is two
// scalar round-to-nearest operations through the __fadd_rn / __fmul_rn /
// __fmaf_rn intrinsics, which the compiler never contracts or reassociates:
// every bit of a result is fixed by the source, whatever the surrounding
// code.  (Blackwell's paired add/mul/fma.rn.f32x2 instructions were measured
// to round differently depending on the code around them, which made the
// low-res results depend on the strip and segment shapes the autotuner
// picks; they are kept for the guidance transform's 1x1 convolutions as
// f2x_mul / f2x_fma, where no such shape dependence arises.)
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_splat(float a) { return f2_pack(a, a); }
__device__ __forceinline__ void f2_unpack(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return f2_pack(__fadd_rn(a0, b0), __fadd_rn(a1, b1));
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return f2_pack(__fsub_rn(a0, b0), __fsub_rn(a1, b1));
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return f2_pack(__fmul_rn(a0, b0), __fmul_rn(a1, b1));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    float a0, a1, b0, b1, c0, c1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    f2_unpack(c, c0, c1);
    return f2_pack(__fmaf_rn(a0, b0, c0), __fmaf_rn(a1, b1, c1));
}
// Blackwell's paired instructions (one instruction for both halves, each
// half rounded to nearest as its scalar instruction would be).
__device__ __forceinline__ f32x2 f2x_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2x_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float f2_lo(f32x2 v) {
    float a, b;
    f2_unpack(v, a, b);
    return a;
}
__device__ __forceinline__ float f2_hi(f32x2 v) {
    float a, b;
    f2_unpack(v, a, b);
    return b;
}
__device__ __forceinline__ f32x2 f2x_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2x_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Correctly rounded 1/k for window counts k = 1 .. kInvCountMax (the largest
// clipped window, (2 r + 1)^2 at r = 16), built by the compiler.  Entry 0 is
// unused.  Window counts come from integer clipping, so a table load replaces
// a division.
constexpr int kInvCountMax = 33 * 33;
struct InvCountTable {
    float v[kInvCountMax + 1];
    constexpr InvCountTable() : v() {
        for (int k = 1; k <= kInvCountMax; ++k) v[k] = 1.f / (float)k;
    }
};
static __constant__ InvCountTable kInvCount = InvCountTable();
__device__ __forceinline__ float inv_count(int k) { return kInvCount.v[k]; }
__device__ __forceinline__ float inv_countf(float k) { return kInvCount.v[(int)k]; }  // k integral

// ---------------------------------------------------------------- storage
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// VEC consecutive elements moved as one aligned access (16, 8, 4 or 2 bytes).
template <typename T, int VEC>
struct __align__(sizeof(T) * VEC) Vec {
    T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, float (&out)[VEC]) {
    Vec<T, VEC> x = *reinterpret_cast<const Vec<T, VEC>*>(p);
#pragma unroll
    for (int k = 0; k < VEC; ++k) out[k] = to_f32<T>(x.v[k]);
}

// Raw vector load through the read-only path (kept packed until used).
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldg_vec(const T* __restrict__ p) {
    return *reinterpret_cast<const Vec<T, VEC>*>(p);
}

template <typename T, int VEC>
__device__ __forceinline__ void unpack_vec(const Vec<T, VEC>& x, float (&out)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) out[k] = to_f32<T>(x.v[k]);
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const float (&in)[VEC]) {
    Vec<T, VEC> x;
#pragma unroll
    for (int k = 0; k < VEC; ++k) x.v[k] = from_f32<T>(in[k]);
    *reinterpret_cast<Vec<T, VEC>*>(p) = x;
}

// ------------------------------------------------------------- upsampler
// Bilinear source position of output sample y when n_in samples are
// stretched over n_out (half-pixel centres, align_corners = False):
// t = (y + 1/2) n_in / n_out - 1/2, clamped below at 0.  `i0` is floor(t);
// the second tap is i0 + 1, which callers clamp to n_in - 1 by replicating
// the last sample.  Exact integer arithmetic for i0; lam = remainder / (2 n_out).
struct Tap {
    int i0;
    float lam;
};

__device__ __forceinline__ Tap tap_general(int y, int n_in, int n_out) {
    long long num = (long long)(2 * y + 1) * n_in - n_out;  // = 2 n_out t
    Tap t;
    if (num <= 0) {
        t.i0 = 0;
        t.lam = 0.f;
        return t;
    }
    long long den = 2LL * n_out;
    long long i0 = num / den;
    t.i0 = (int)i0;
    t.lam = (float)(num - i0 * den) / (float)den;
    return t;
}

// Integer factor F (n_out = F n_in): y = F j + q gives t = j + (2q + 1 - F) / (2F).
// i0 may be -1 at the left border; callers replicate sample 0 there, which is
// the same as clamping t at 0.
template <int F>
__device__ __forceinline__ Tap tap_int(int y) {
    static_assert(F > 0, "integer factor");
    const int j = y / F, q = y - (y / F) * F;
    const int t2 = 2 * q + 1 - F;
    Tap t;
    if (t2 < 0) {
        t.i0 = j - 1;
        t.lam = (float)(t2 + 2 * F) / (float)(2 * F);
    } else {
        t.i0 = j;
        t.lam = (float)t2 / (float)(2 * F);
    }
    return t;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ float lerp(float a, float b, float lam) { return fmaf(lam, b - a, a); }

}  // namespace dgf
