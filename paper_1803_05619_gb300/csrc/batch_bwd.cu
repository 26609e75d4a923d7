// Persistent kernels of the batched backward (batch_bwd.cuh): function
// pointers and launch shapes for the graph nodes, per node class.
#include "batch_bwd.cuh"
#include "kernels.h"

namespace dgf {

template <typename K>
static cudaError_t bwd_prep(K kernel, size_t smem) {
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) cudaGetLastError();
        return e;
    }
    return cudaSuccess;
}

template <typename T, int VEC, int F, bool TMA>
static cudaError_t k3b_one(void** fn, size_t* smem, int* threads) {
    using Sh = K3BatchShape<T, VEC, F, TMA>;
    *fn = (void*)k3_batched<T, VEC, F, TMA>;
    *smem = Sh::SMEM;
    *threads = Sh::WPC * 32;
    return bwd_prep(k3_batched<T, VEC, F, TMA>, *smem);
}

template <typename T>
static cudaError_t k3b_get(int vec, int F, bool tma, void** fn, size_t* smem, int* threads) {
#define DGF_K3B(VV, FF)                                                   \
    if (vec == VV && F == FF) {                                           \
        if constexpr (VV * sizeof(T) == 16)                               \
            if (tma) return k3b_one<T, VV, FF, true>(fn, smem, threads);  \
        if (!tma) return k3b_one<T, VV, FF, false>(fn, smem, threads);    \
        return cudaErrorInvalidValue;                                     \
    }
    DGF_K3B(8, 8)
    DGF_K3B(8, 4)
    DGF_K3B(4, 4)
    DGF_K3B(4, 2)
#undef DGF_K3B
    return cudaErrorInvalidValue;
}

cudaError_t k3_batched_kernel(dgf_dtype dt, int vec, int F, bool tma, void** fn, size_t* smem, int* threads) {
    switch (dt) {
        case DGF_BF16: return k3b_get<__nv_bfloat16>(vec, F, tma, fn, smem, threads);
        case DGF_F16: return k3b_get<__half>(vec, F, tma, fn, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int R, int V>
static cudaError_t k4b_one(void** fn, size_t* smem, int* threads) {
    constexpr int WPC = slide_wpc<k4_slide_warp_bytes<T, T, R, V>()>();
    *fn = (void*)k4_batched<T, R, V>;
    *smem = (size_t)WPC * k4_slide_warp_bytes<T, T, R, V>();
    *threads = WPC * 32;
    return bwd_prep(k4_batched<T, R, V>, *smem);
}

template <typename T>
static cudaError_t k4b_get(int r, int V, void** fn, size_t* smem, int* threads) {
#define DGF_K4B(RR, VV) \
    if (r == RR && V == VV) return k4b_one<T, RR, VV>(fn, smem, threads);
    DGF_K4B(1, 2)
    DGF_K4B(1, 4)
    DGF_K4B(1, 8)
    DGF_K4B(2, 2)
    DGF_K4B(2, 4)
    DGF_K4B(2, 8)
    DGF_K4B(4, 4)
    DGF_K4B(8, 4)
#undef DGF_K4B
    return cudaErrorInvalidValue;
}

cudaError_t k4_batched_kernel(dgf_dtype dt, int r, int V, void** fn, size_t* smem, int* threads) {
    switch (dt) {
        case DGF_BF16: return k4b_get<__nv_bfloat16>(r, V, fn, smem, threads);
        case DGF_F16: return k4b_get<__half>(r, V, fn, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dgf
