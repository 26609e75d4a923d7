// TMA (cp.async.bulk.tensor) staging of the low-resolution halo tiles.
//
// A 3-D tensor map (x = column, y = row, z = plane) per input describes the
// whole N*C stack of low-resolution planes.  One elected thread arms an
// mbarrier with the expected byte count and issues one tiled bulk copy per
// input; the box starts at a column rounded down to the 16-byte boundary
// (loads may start at negative or out-of-range coordinates, which read as
// zero, exactly like the plain staging path).  Waits are bounded: when the
// limit runs out the kernel records DGF_ERR_TIMEOUT in the status word,
// waits once more (bounded) for its copies, and falls back to plain loads.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "lowres.cuh"

namespace dgf {

struct TmaPlane {
    CUtensorMap map;  // 64-byte aligned opaque descriptor
    int off;          // column offset of the halo inside the box
    int bx, by;       // box extent (elements, rows)
    int esize;        // bytes per element
};

struct TmaPair {
    TmaPlane a, b;
    int enabled;
};

// K4 strips: G, P and d Abar, d bbar (the float2 pairs as a float tensor of
// twice the width).
struct TmaTriple {
    TmaPlane a, b, c;
    int enabled;
};

// Tensor maps of K3's two high-resolution inputs (d O_h, I_h): 3-D (column,
// row, plane), box of one strip row segment x one block of rows.
struct K3Maps {
    CUtensorMap r, g;  // 64-byte aligned opaque descriptors
};

// Tensor map of K2's high-resolution input (I_h), boxes as for K3.
struct K2Map {
    CUtensorMap m;
};

constexpr long long kWaitLimit = 1LL << 22;  // try_wait polls before giving up
constexpr uint32_t kStatusTimeout = 1u;

// The library's status block (one per device, in api.cu), passed to the
// kernels as `uint32_t* status`:
//   status[0]      error bits (kStatusTimeout: a bounded wait ran out);
//   status[1]      polls of a first wait on a copy (kWaitLimit unless a test
//                  lowers it to make the wait run out); the second wait, for
//                  the copies still in flight, always polls kWaitLimit times,
//                  so every copy has landed before its shared memory is
//                  reused or the kernel exits;
//   status[2..3]   address of a pinned host word mirroring the error bits
//                  (0 when the host has not set one up), written only when an
//                  error is recorded, so the host sees it at its next call
//                  without synchronising.
__device__ __forceinline__ long long first_wait_limit(const uint32_t* status) {
    return status != nullptr ? (long long)status[1] : kWaitLimit;
}

__device__ __forceinline__ void status_fail(uint32_t* status, uint32_t bits) {
    if (status == nullptr) return;
    atomicOr(status, bits);
    uint32_t* host = *reinterpret_cast<uint32_t* const volatile*>(status + 2);
    if (host != nullptr) {
        *reinterpret_cast<volatile uint32_t*>(host) = bits;  // the only bit there is
        __threadfence_system();
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Before a tensor map written by a host copy into global memory is used:
// acquire it into the tensor-map proxy (system scope: the writer was a copy
// from the host).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :
        : "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

template <typename TS>
__device__ __forceinline__ void tma_unpack(const void* land, const TmaPlane* tp, float* dst,
                                           const LowresTile& t) {
    const TS* src = static_cast<const TS*>(land);
    const int n = t.EY2 * t.EX2;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
        const int ey = idx / t.EX2, ex = idx - ey * t.EX2;
        dst[idx] = to_f32<TS>(src[ey * tp->bx + ex + tp->off]);
    }
}

// Stage the E2 halo tiles of two planes with TMA into a landing area inside
// `scratch` (checked large enough on the host), then widen to FP32 sG, sP.
// Returns false only when the copies did not complete in time.
template <typename TA, typename TB>
__device__ bool tma_stage_pair(const TmaPlane* ta, const TmaPlane* tb, int plane, const LowresTile& t,
                               float* sA, float* sB, float* scratch, uint32_t* status) {
    __shared__ __align__(8) uint64_t bar;
    char* la = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(scratch) + 127) & ~uintptr_t(127));
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
        const int ya = t.ty0 - 2 * t.r;
        tma_load_3d(smem_u32(la), &ta->map, t.tx0 - 2 * t.r - ta->off, ya, plane, b);
        tma_load_3d(smem_u32(lb), &tb->map, t.tx0 - 2 * t.r - tb->off, ya, plane, b);
    }
    __syncthreads();
    bool ok = mbar_wait(b, 0, first_wait_limit(status));
    if (!ok) {
        status_fail(status, kStatusTimeout);
        mbar_wait(b, 0, kWaitLimit);  // the copies land before the buffers are reused
    }
    ok = __syncthreads_and(ok) != 0;  // one decision for the whole CTA
    if (ok) {
        tma_unpack<TA>(la, ta, sA, t);
        tma_unpack<TB>(lb, tb, sB, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
    return ok;
}

// Extra dynamic shared memory the TMA path may need beyond the region it
// borrows (alignment slack of the two landing buffers).
inline size_t tma_extra_bytes(int, int, int) { return 256; }

}  // namespace dgf
