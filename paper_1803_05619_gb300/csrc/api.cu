// C ABI of the guided filtering layer (include/dgf.h): argument validation,
// workspace layout, tile planning, kernel sequencing, the graph-replayed
// batched path, launch counting and optional per-kernel event timing.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <tuple>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dgf.h"
#include "batch.cuh"
#include "kernels.h"
#include "tma.cuh"
#include "tune.h"

namespace dgf {

// -------------------------------------------------------------- errors
static thread_local std::string t_err;

static dgf_status fail(dgf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

static dgf_status cuda_fail(cudaError_t e, const char* what) {
    // consume the runtime's record of a non-sticky error (a launch or
    // attribute call the runtime refused), so that it is reported once, by
    // this call, and not again by a later launch check
    cudaGetLastError();
    return fail(DGF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------- launch count + profiling
static std::atomic<long long> g_launches{0};

struct ProfEntry {
    double ms = 0.0;
    long long n = 0;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::map<std::string, ProfEntry> g_prof;

struct Pending {
    const char* name;
    cudaEvent_t a, b;
};

class Launcher {
   public:
    explicit Launcher(cudaStream_t s) : s_(s) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        prof_ = g_prof_on;
    }
    template <class Fn>
    cudaError_t run(const char* name, Fn&& fn) {
        g_launches.fetch_add(1);
        if (!prof_) return fn();
        Pending p{name, nullptr, nullptr};
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        cudaEventRecord(p.a, s_);
        cudaError_t e = fn();
        cudaEventRecord(p.b, s_);
        pend_.push_back(p);
        return e;
    }
    ~Launcher() {
        if (pend_.empty()) return;
        cudaStreamSynchronize(s_);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& p : pend_) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                ProfEntry& e = g_prof[p.name];
                e.ms += ms;
                e.n += 1;
            }
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    }

   private:
    cudaStream_t s_;
    bool prof_ = false;
    std::vector<Pending> pend_;
};

// --------------------------------------------------------------- status word
// The status block of tma.cuh, one per device: error bits, the polls of a
// first wait on a copy, and the address of the pinned host word that
// mirrors the error bits (set up by the first call of a workspace entry
// point on the device).
__device__ uint32_t g_status_block[4] = {0u, (uint32_t)kWaitLimit, 0u, 0u};

// Device address of the status block on the current device, resolved once
// per device under a lock (concurrent first calls from several host threads).
static std::mutex g_status_mu;
static uint32_t* g_status_dev[64] = {nullptr};
static volatile uint32_t* g_status_host[64] = {nullptr};

static uint32_t* status_ptr() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (g_status_dev[dev] == nullptr) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_status_block) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_dev[dev] = static_cast<uint32_t*>(a);
    }
    return g_status_dev[dev];
}

// The pinned host mirror of the current device's error bits: allocated and
// published to the device block on the first call (a synchronous copy, so
// that first call must not come during a stream capture).
static void status_mirror_setup() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return;
    uint32_t* blk = status_ptr();
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (blk == nullptr || g_status_host[dev] != nullptr) return;
    // (a failure leaves no mirror and clears the runtime's last error, so
    // the calls that follow see only their own errors)
    void* h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    memset(h, 0, 64);
    void* hd = nullptr;
    if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) {
        cudaFreeHost(h);
        cudaGetLastError();
        return;
    }
    uint32_t bits = 0;  // bits a kernel recorded before the mirror existed
    if (cudaMemcpy(&bits, blk, sizeof bits, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(blk + 2, &hd, sizeof hd, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFreeHost(h);
        cudaGetLastError();
        return;
    }
    static_cast<uint32_t*>(h)[0] = bits;
    g_status_host[dev] = static_cast<volatile uint32_t*>(h);
}

// Every entry point starts here: an error a kernel recorded in an earlier
// call on this device (visible in the host mirror without synchronising)
// makes every later call fail until dgf_clear_device_status().
static dgf_status entry_check(bool setup) {
    if (setup) status_mirror_setup();
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return DGF_OK;
    volatile uint32_t* m = g_status_host[dev];
    if (m != nullptr && *m != 0u)
        return fail(DGF_ERR_TIMEOUT,
                    "a bounded device wait ran out in an earlier call on this device (its results are "
                    "invalid); dgf_clear_device_status() resets the error");
    return DGF_OK;
}

// ------------------------------------------------------------------ sizes
static size_t esize(dgf_dtype dt) { return dt == DGF_F32 ? 4 : 2; }
static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr int kMaxRadius = 16;

struct Layout {
    size_t coef, dcoef, stats, gl, dgl, partials, gh, total;
};

// hi: high-res pixel-channels (N C h w): with the guidance transform the
// forward keeps F(I_h) there in FP32 (K5 writes it, K2 reads it).
static Layout layout(int N, int C, int h_l, int w_l, bool guided, size_t hi = 0) {
    const size_t lo = (size_t)N * C * h_l * w_l;
    Layout L{};
    size_t off = 0;
    L.coef = off;
    off += align256(lo * sizeof(float2));
    L.dcoef = off;
    off += align256(lo * sizeof(float2));
    L.stats = off;  // window statistics kept from the backward K1 pass for K4
    off += align256(lo * sizeof(float4));
    if (guided) {
        L.gl = off;
        off += align256(lo * sizeof(float));
        L.dgl = off;
        off += align256(lo * sizeof(float));
        L.partials = off;
        off += align256((size_t)kMaxK6Blocks * kWGradPadded * sizeof(float));
        L.gh = off;
        off += align256(hi * sizeof(float));
    }
    L.total = off;
    return L;
}

static bool bad_eps(float eps) { return !(eps >= FLT_MIN) || !std::isfinite(eps); }

static int integer_factor(int h_l, int w_l, int h, int w) {
    if (h % h_l != 0 || w % w_l != 0) return 0;
    const int fy = h / h_l, fx = w / w_l;
    return fy == fx ? fy : 0;
}

// Vector width (elements) of the high-res passes: 16-byte vectors, else
// 8-byte vectors, else scalars; the width must divide w and keep every
// pointer aligned.
static int pick_vec(dgf_dtype dt, int w, std::initializer_list<const void*> ptrs) {
    const int esz = (int)esize(dt);
    for (int v = 16 / esz; v >= 8 / esz; v >>= 1) {
        if (w % v != 0) continue;
        bool ok = true;
        for (const void* p : ptrs)
            if (p != nullptr && (reinterpret_cast<uintptr_t>(p) % (size_t)(v * esz)) != 0) ok = false;
        if (ok) return v;
    }
    return 1;
}

static bool aligned16(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (p != nullptr && reinterpret_cast<uintptr_t>(p) % 16 != 0) return false;
    return true;
}

struct Plan {
    int F = 0;      // integer factor (0 = general ratio)
    int vec = 1;    // K2 / K3 vector width
    LowCfg k1{0, 32, 32};
    LowCfg k4{0, 16, 16};
    int k2_th = 32;        // K2 tiles: high-res rows per tile
    bool k2_strip = false; // K2 as warp strips (integer F in {2, 4, 8} dividing vec)
    int k2_ls = 8;         // K2 strips: low-res rows per segment
    int k3_lth = 8;
    bool k3_fast = false;
    bool k12 = false;      // forward as the fused K12 kernel
    bool k12_ok = false;   // K12 can serve this call (the tuner may still prefer K1 + K2)
    int k12_ls = 32;       // K12: low-res rows per segment
    bool k13 = false;      // backward K1 + K3 as the fused K13 kernel
    bool k13_ok = false;
    int k13_ls = 16;       // K13: low-res rows per segment
    int sc = 0;            // the plane's size class in the autotuner's keys
};

static bool g_fused_allowed = true;

static bool aligned_to(std::initializer_list<const void*> ptrs, int bytes) {
    for (const void* p : ptrs)
        if (p != nullptr && reinterpret_cast<uintptr_t>(p) % (uintptr_t)bytes != 0) return false;
    return true;
}

static size_t g_smem_optin = 0;
static size_t smem_limit() {
    if (g_smem_optin == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 227 * 1024;
        g_smem_optin = (size_t)v;
    }
    return g_smem_optin;
}

// Default low-resolution tiles: the column-walking kernels for r in
// {1, 2, 4, 8} (CW columns x EY1 rows of coefficients per CTA), else the
// generic tile kernels with the largest square tile that fits.
static bool pick_lowres_tiles(int r, Plan& p) {
    const size_t lim = smem_limit();
    bool ok1 = false, ok4 = false;
    if (low_fast_radius(r)) {
        // defaults from timing every shape on GB300 (BF16, 2 x 3 x 540 x 960 at r = 4,
        // 8 x 3 x 256^2 at r = 8); the autotuner refines them per call shape
        const LowCfg k1 = r <= 2 ? LowCfg{2, 32, 0} : (r == 4 ? LowCfg{1, 64, 32} : LowCfg{1, 64, 64});
        const LowCfg k4 = r <= 2 ? LowCfg{2, 32, 0} : (r == 4 ? LowCfg{1, 64, 16} : LowCfg{1, 64, 32});
        if (k1_cfg_smem(k1, r, 0) <= lim) {
            p.k1 = k1;
            ok1 = true;
        }
        if (k4_cfg_smem(k4, r) <= lim) {
            p.k4 = k4;
            ok4 = true;
        }
    }
    static const int cand[] = {32, 16, 8};
    for (int t : cand) {
        if (ok1) break;
        if (k1_smem_bytes(r, t, t) <= lim) {
            p.k1 = LowCfg{0, t, t};
            ok1 = true;
        }
    }
    for (int t : cand) {
        if (ok4) break;
        if (t <= 16 && k4_smem_bytes(r, t, t) <= lim) {
            p.k4 = LowCfg{0, t, t};
            ok4 = true;
        }
    }
    return ok1 && ok4;
}

// K3 strip segments: low-res rows per segment
static int default_k3_lth(int) { return 32; }

// Small planes: the strip kernels' segment length (rows per warp) is shrunk
// until one plane alone gives a warp per SM, so a small image is not
// a handful of warps walking long row chains.  The rule looks at the plane
// shape only, never at the number of planes in a call, so a plane's bits do
// not depend on the call it is in (and every kernel it is applied to gives
// the same bits at every segment length except K4, whose shift constant
// comes from the segment's first row).
static int g_sms = 0;
static int sm_count() {
    if (g_sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        g_sms = v;
    }
    return g_sms;
}
static int fill_ls(int ls, int nstrip, int rows, int min_ls) {
    const long long want = sm_count();  // warps of one plane: one per SM
    while (ls > min_ls && (long long)nstrip * ((rows + ls - 1) / ls) < want) ls = std::max(min_ls, ls / 2);
    return ls;
}

static std::vector<LowCfg> low_candidates(int r, bool k4, dgf_dtype dt);
static bool in_candidates(const LowCfg& c, int r, bool k4, dgf_dtype dt) {
    for (const LowCfg& x : low_candidates(r, k4, dt))
        if (x.fast == c.fast && x.a == c.a && x.b == c.b) return true;
    return false;
}

// Sliding-sum low-res strips for 16-bit storage (dgf_set_lowres_slide).
static bool g_slide_allowed = true;
// Batched backward as one graph of persistent kernels where it applies
// (dgf_set_batched_graph_backward).
static bool g_batched_graph_bwd = true;

// Table entries of the low-res kernels: b > 0 column-walking tiles (CW = a,
// EY1 = b), b == 0 strips (a rows per segment), b < 0 sliding strips (a rows
// per segment, -b columns per lane).
static LowCfg low_from_table(int a, int b) {
    if (b < 0) return LowCfg{3, a, -b};
    return LowCfg{b == 0 ? 2 : 1, a, b};
}
static void low_to_table(const LowCfg& c, int& a, int& b) {
    a = c.a;
    b = c.fast == 3 ? -c.b : c.b;
}

// Shapes from the autotuner's table override the defaults (whether or not
// tuning is enabled now), so every call with the same key uses one shape.
static Plan make_plan(dgf_dtype dt, int h_l, int w_l, int h, int w, int r, bool gf32,
                      std::initializer_list<const void*> hires_ptrs, bool mean_ab = true) {
    Plan p;
    p.sc = tune_size_class(h_l, w_l);
    p.F = integer_factor(h_l, w_l, h, w);
    p.vec = pick_vec(dt, w, hires_ptrs);
    pick_lowres_tiles(r, p);
    // 16-bit storage: the sliding-sum strips (FP32 storage keeps the
    // exactly centred forms, which its tighter gates need)
    if (g_slide_allowed && dt != DGF_F32 && slide_radius(r)) {
        p.k1 = LowCfg{3, 0, slide_k1_v(r)};
        p.k4 = LowCfg{3, 0, slide_k4_v(r)};
    }
    p.k3_fast = p.F > 0 && k3_fast_ok(p.vec, p.F);
    p.k2_strip = p.F > 0 && k2_strip_ok(p.vec, p.F);
    p.k3_lth = default_k3_lth(p.F);
    int a, b;
    // a table entry (tuned, pinned or read from a cache file) is used only if
    // it is one of the shapes the kernels are built for
    if (low_fast_radius(r)) {
        if (tune_lookup(TuneKey{1, (int)dt, r, 0, 0, gf32 ? 1 : 0, p.sc}, a, b)) {
            const LowCfg c = low_from_table(a, b);
            if (in_candidates(c, r, false, dt)) p.k1 = c;
        }
        if (tune_lookup(TuneKey{4, (int)dt, r, 0, 0, gf32 ? 1 : 0, p.sc}, a, b)) {
            const LowCfg c = low_from_table(a, b);
            if (in_candidates(c, r, true, dt)) p.k4 = c;
        }
    }
    if (tune_lookup(TuneKey{2, (int)dt, 0, p.F, p.vec, 0, p.sc}, a, b) && a >= 1 && a <= 256) {
        if (p.k2_strip)
            p.k2_ls = a;
        else
            p.k2_th = a;
    }
    if (p.k3_fast && tune_lookup(TuneKey{3, (int)dt, 0, p.F, p.vec, 0, p.sc}, a, b) && a >= 1 && a <= 256)
        p.k3_lth = a;
    // fused forward: plain guide, box mean of A, b, r in {1, 2}, a factor with
    // one low-res cell per lane; a table entry a = 0 means the tuner found
    // K1 + K2 faster for this key
    // (the fused kernel's K1 part is the strip walk: it stands in for the
    // strip K1 + K2 pair only, so a tile-form K1 keeps the two kernels)
    p.k12_ok = g_fused_allowed && !gf32 && mean_ab && p.F > 0 && k12_supported(dt, r, p.F) &&
               aligned_to(hires_ptrs, k12_vec_bytes(dt, p.F)) && p.k1.fast == 2;
    // untuned default: fused at r = 1, where it measured faster than K1 + K2
    // on large images too (at r = 2 its redundant K1 columns cost more)
    p.k12 = p.k12_ok && r == 1;
    if (p.k12_ok && tune_lookup(TuneKey{5, (int)dt, r, p.F, 0, 0, p.sc}, a, b) && a >= 0 && a <= 256) {
        p.k12 = a > 0;
        if (a > 0) p.k12_ls = a;
    }
    // fused backward K1 + K3: likewise for the strip K1 and the 16-byte K3
    // strips with one low-res cell per lane
    p.k13_ok = g_fused_allowed && !gf32 && mean_ab && p.k3_fast && k13_supported(dt, r, p.F, p.vec) &&
               aligned_to(hires_ptrs, 16) && p.k1.fast == 2;
    p.k13 = p.k13_ok && r == 1;
    if (p.k13_ok && tune_lookup(TuneKey{6, (int)dt, r, p.F, p.vec, 0, p.sc}, a, b) && a >= 0 && a <= 256) {
        p.k13 = a > 0;
        if (a > 0) p.k13_ls = a;
    }
    if (!mean_ab) {
        // the layer as printed (no box mean of A, b): warp strips for r in
        // {1, 2}, generic tiles otherwise (the column-walking tiles always
        // box-average A, b)
        if (r == 1 || r == 2) {
            p.k1 = LowCfg{2, 32, 0};
            p.k4 = LowCfg{2, 32, 0};
        } else {
            for (int tt : {32, 16, 8})
                if (k1_smem_bytes(r, tt, tt) <= smem_limit()) {
                    p.k1 = LowCfg{0, tt, tt};
                    break;
                }
            for (int tt : {16, 8})
                if (k4_smem_bytes(r, tt, tt) <= smem_limit()) {
                    p.k4 = LowCfg{0, tt, tt};
                    break;
                }
        }
        p.k1.mean = 0;
        p.k4.mean = 0;
    }
    return p;
}

static std::vector<LowCfg> low_candidates(int r, bool k4, dgf_dtype dt) {
    std::vector<LowCfg> v;
    if (!low_fast_radius(r)) return v;
    if (g_slide_allowed && dt != DGF_F32 && slide_radius(r))
        for (int V : {2, 4, 8})
            if (slide_v_built(r, V, k4))
                for (int seg : {8, 12, 16, 24, 32, 48, 64})
                    if (seg >= 2 * r) v.push_back(LowCfg{3, seg, V});
    if (r <= 2)
        for (int seg : {8, 16, 24, 32, 48, 64, 128}) v.push_back(LowCfg{2, seg, 0});
    static const int cws[] = {64, 128, 256};
    static const int eys[] = {16, 32, 64};
    for (int cw : cws)
        for (int ey : eys) {
            if (cw <= 2 * r + 1 || ey <= 2 * r + 1) continue;
            const size_t sm = k4 ? k4_fast_smem_bytes(r, cw, ey) : k1_fast_smem_bytes(r, cw, ey, 0);
            if (sm <= smem_limit()) v.push_back(LowCfg{1, cw, ey});
        }
    return v;
}

// --------------------------------------------------------------- TMA maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

static bool g_tma_allowed = true;

// Tensor map over one plane stack (planes x h x w, element size esz) with
// a bx x by box.  False when the TMA alignment rules do not hold.
static bool make_tma(TmaPlane& tp, const void* base, CUtensorMapDataType ty, int esz, int planes, int h, int w,
                     int bx, int by, int off) {
    EncodeTiledFn enc = encode_fn();
    if (enc == nullptr) return false;
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    if (((size_t)w * esz) % 16 != 0) return false;
    if (((size_t)bx * esz) % 16 != 0) return false;
    if (bx > 256 || by > 256 || bx < 1 || by < 1) return false;
    tp.off = off;
    tp.bx = bx;
    tp.by = by;
    tp.esize = esz;
    cuuint64_t gdim[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)planes};
    cuuint64_t gstride[2] = {(cuuint64_t)w * esz, (cuuint64_t)w * h * esz};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult rc = enc(&tp.map, ty, 3, const_cast<void*>(base), gdim, gstride, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return rc == CUDA_SUCCESS;
}

static CUtensorMapDataType tma_type(dgf_dtype dt) {
    return dt == DGF_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                         : (dt == DGF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
}

// K3's tensor maps (d O_h, I_h): box of one strip row (32 vec columns) x F
// rows.  Only for 16-byte vectors; returns false (plain loads) otherwise or
// when the maps cannot be made.
static bool make_k3_maps(K3Maps& m, const void* R, const void* G, dgf_dtype dt, int planes, int h, int w, int vec,
                         int F) {
    if (!g_tma_allowed || F <= 0 || vec * (int)esize(dt) != 16) return false;
    TmaPlane a, b;
    if (!make_tma(a, R, tma_type(dt), (int)esize(dt), planes, h, w, 32 * vec, F, 0)) return false;
    if (!make_tma(b, G, tma_type(dt), (int)esize(dt), planes, h, w, 32 * vec, F, 0)) return false;
    m.r = a.map;
    m.g = b.map;
    return true;
}

// Box of one input for K1's halo tile.  Generic tiles start on a 16-byte
// column boundary (TX a multiple of the 16-byte unit), so the offset is a
// constant; column-walking tiles start anywhere, so the box is one unit
// wider and the kernel computes the offset per tile.
static bool k1_box(const LowCfg& c, int r, int esz, int& bx, int& by, int& off) {
    const int U = 16 / esz;
    if (c.fast == 3) return false;  // the sliding strips read rows directly
    if (c.fast == 2) {
        // warp strips (two columns per lane): 64 columns plus one 16-byte
        // unit (the strip's first column is rounded down to it), whole
        // blocks of ring periods
        bx = 64 + U;
        by = r == 1 ? 6 : 10;
        off = 0;
        return true;
    }
    if (c.fast) {
        const int EX2 = c.a + 2 * r;
        bx = (EX2 + U - 1 + U - 1) / U * U;
        by = c.b + 2 * r;
        off = 0;
        return true;
    }
    const int TY = c.a, TX = c.b;
    if (TX % U != 0) return false;
    const int lead = (2 * r + U - 1) / U * U;  // box starts on a 16-byte column boundary
    off = lead - 2 * r;
    bx = (off + TX + 4 * r + U - 1) / U * U;
    by = TY + 4 * r;
    return true;
}

// TMA pair for K1's (G, P) staging; `landing` returns the bytes the two
// landing buffers need (with alignment slack).
static TmaPair make_tma_pair(const void* G, dgf_dtype dg, const void* P, dgf_dtype dp, int planes, int h, int w,
                             int r, const LowCfg& c, size_t& landing) {
    TmaPair t;
    memset(&t, 0, sizeof t);
    t.enabled = 0;
    landing = 0;
    if (!g_tma_allowed) return t;
    int bxa, bya, offa, bxb, byb, offb;
    if (!k1_box(c, r, (int)esize(dg), bxa, bya, offa) || !k1_box(c, r, (int)esize(dp), bxb, byb, offb)) return t;
    if (!make_tma(t.a, G, tma_type(dg), (int)esize(dg), planes, h, w, bxa, bya, offa)) return t;
    if (!make_tma(t.b, P, tma_type(dp), (int)esize(dp), planes, h, w, bxb, byb, offb)) return t;
    const size_t need = (size_t)bxa * bya * esize(dg) + (size_t)bxb * byb * esize(dp) + 256;
    if (c.fast == 2) {
        // the strip kernel sizes its own slot rings (well under the limit)
    } else if (c.fast) {
        if (k1_fast_smem_bytes(r, c.a, c.b, need) > smem_limit()) return t;
        landing = need;
    } else {
        // landing buffers live in the generic K1's row-statistics region (4 EY2 EX1 floats)
        const size_t region = (size_t)4 * (c.a + 4 * r) * (c.b + 2 * r) * sizeof(float);
        if (need > region + tma_extra_bytes(r, c.a, c.b)) return t;
    }
    t.enabled = 1;
    return t;
}

// K2's tensor map (I_h), same box as K3's.
static bool make_k2_map(K2Map& m, const void* in, dgf_dtype dt, int planes, int h, int w, int vec, int F) {
    if (!g_tma_allowed || F <= 0 || vec * (int)esize(dt) != 16) return false;
    TmaPlane a;
    if (!make_tma(a, in, tma_type(dt), (int)esize(dt), planes, h, w, 32 * vec, F, 0)) return false;
    m.m = a.map;
    return true;
}

// K2 (mode 0: O_h = Abar_h I_h + bbar_h) in the plan's form.
static cudaError_t launch_k2_plan(dgf_dtype dt, const float2* coef, const void* in, void* out, int planes, int h_l,
                                  int w_l, int h, int w, const Plan& p, int shape, cudaStream_t s) {
    if (p.k2_strip) {
        const int K = p.vec / p.F;
        shape = fill_ls(shape, (w_l + 32 * K - 1) / (32 * K), h_l, 2);
        K2Map map;
        const bool tma = make_k2_map(map, in, dt, planes, h, w, p.vec, p.F);
        return launch_k2_strip(dt, coef, in, out, planes, h_l, w_l, h, w, p.vec, p.F, shape, tma ? &map : nullptr,
                               status_ptr(), s);
    }
    return launch_k2(dt, 0, coef, in, out, planes, h_l, w_l, h, w, p.vec, p.F, shape, s);
}

// K4 strips' tensor maps: G, P (box 32 + U columns x RB rows) and d Abar,
// d bbar as float pairs (box 2 x 34 floats).  Disabled when any map cannot
// be made (alignment) or for the tile forms.
static TmaTriple make_k4_maps(const void* G, dgf_dtype dg, const void* P, dgf_dtype dp, const float2* dcoef,
                              int planes, int h, int w, int r, const LowCfg& c) {
    TmaTriple t;
    memset(&t, 0, sizeof t);
    t.enabled = 0;
    if (!g_tma_allowed || c.fast != 2) return t;
    const int rb = r == 1 ? 6 : 10;
    const int eg = (int)esize(dg), ep = (int)esize(dp);
    if (!make_tma(t.a, G, tma_type(dg), eg, planes, h, w, 32 + 16 / eg, rb, 0)) return t;
    if (!make_tma(t.b, P, tma_type(dp), ep, planes, h, w, 32 + 16 / ep, rb, 0)) return t;
    if (!make_tma(t.c, dcoef, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, planes, h, 2 * w, 2 * 34, rb, 0)) return t;
    t.enabled = 1;
    return t;
}

// stats: window statistics saved by the backward K1 pass (strip forms), or null
static LowCfg low_fill(LowCfg c, int r, int h_l, int w_l, bool k4);

static cudaError_t run_k4(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP,
                          void* dG, int planes, int h_l, int w_l, int r, float eps, const LowCfg& c0, cudaStream_t s,
                          const float4* stats = nullptr) {
    const LowCfg c = low_fill(c0, r, h_l, w_l, true);
    const TmaTriple tma = make_k4_maps(G, gf32 ? DGF_F32 : dt, P, dt, dcoef, planes, h_l, w_l, r, c);
    return launch_k4(dt, gf32, G, P, dcoef, dP, dG, planes, h_l, w_l, r, eps, c, &tma, status_ptr(), stats, s);
}

// --------------------------------------------------------------- validation
static dgf_status check_sizes(int N, int C, int h_l, int w_l, int h, int w, int r, float eps, dgf_dtype dt) {
    if ((int)dt < 0 || (int)dt > 2) return fail(DGF_ERR_INVALID, "dtype %d is not FP32, BF16 or FP16", (int)dt);
    if (N < 0) return fail(DGF_ERR_INVALID, "N = %d < 0", N);
    if (C < 1) return fail(DGF_ERR_INVALID, "C = %d < 1", C);
    if (h_l < 1 || w_l < 1 || h < 1 || w < 1)
        return fail(DGF_ERR_INVALID, "sizes must be >= 1 (h_l=%d w_l=%d h=%d w=%d)", h_l, w_l, h, w);
    if (h_l > h || w_l > w) return fail(DGF_ERR_INVALID, "low-res %dx%d larger than high-res %dx%d", h_l, w_l, h, w);
    if (r < 0) return fail(DGF_ERR_INVALID, "radius r = %d < 0", r);
    if (r > kMaxRadius) return fail(DGF_ERR_UNSUPPORTED, "radius r = %d > %d", r, kMaxRadius);
    if (bad_eps(eps)) return fail(DGF_ERR_INVALID, "eps must be finite and >= FLT_MIN (the smallest normal float)");
    if ((long long)N * C > 65535) return fail(DGF_ERR_UNSUPPORTED, "N*C = %lld planes > 65535", (long long)N * C);
    if ((long long)h * w >= (1LL << 40)) return fail(DGF_ERR_UNSUPPORTED, "plane too large");
    return DGF_OK;
}

static dgf_status check_guide(const dgf_guide* g, int C, int h_l, int w_l, int h, int w, dgf_dtype dt) {
    if (g == nullptr) return DGF_OK;
    if (g->w1 == nullptr || g->w2 == nullptr || g->b2 == nullptr)
        return fail(DGF_ERR_INVALID, "guide weights must be non-NULL");
    if (g->hidden < 1 || g->hidden > 16) return fail(DGF_ERR_INVALID, "guide hidden = %d not in [1, 16]", g->hidden);
    if (!std::isfinite(g->slope)) return fail(DGF_ERR_INVALID, "guide slope not finite");
    if (C != 3) return fail(DGF_ERR_UNSUPPORTED, "guidance transform needs C = 3 (got %d)", C);
    const int F = integer_factor(h_l, w_l, h, w);
    if (F == 0) return fail(DGF_ERR_INVALID, "guidance transform needs h = f h_l and w = f w_l");
    if (!guided_supported(dt, w, F))
        return fail(DGF_ERR_UNSUPPORTED, "guidance transform: factor %d with width %d not supported", F, w);
    return DGF_OK;
}

static dgf_status check_ws(void* ws, size_t ws_bytes, size_t need) {
    if (need == 0) return DGF_OK;
    if (ws == nullptr) return fail(DGF_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(DGF_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (ws_bytes < need) return fail(DGF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    return DGF_OK;
}

// ---------------------------------------------------------------- autotune
// Each helper times its candidates on the call's own buffers (the real
// launch that follows overwrites every output) and records the fastest.
// Small planes (size class 1) are not tuned: their kernels are a few walks
// bound by latency, which back-to-back timing of one kernel does not
// measure (on a 64 x 64 plane it picked K1 tiles, which rule out the fused
// kernels, and the step got slower); they keep the default shapes, with
// segments shrunk until a plane gives a warp per SM, unless pinned.
static void tune_k1(dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef, int planes, int h_l,
                    int w_l, int r, float eps, cudaStream_t s, Plan& p) {
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{1, (int)dt, r, 0, 0, gf32 ? 1 : 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    float best = 1e30f;
    LowCfg bc = p.k1;
    for (const LowCfg& c : low_candidates(r, false, dt)) {
        size_t landing = 0;
        TmaPair tma = make_tma_pair(G, gf32 ? DGF_F32 : dt, P, dt, planes, h_l, w_l, r, c, landing);
        const size_t smem = k1_cfg_smem(c, r, tma.enabled ? landing : 0);
        const float ms = time_launch(s, [&] {
            return launch_k1(dt, gf32, G, P, coef, planes, h_l, w_l, r, eps, c, tma, smem, status_ptr(), nullptr, s);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bc = c;
        }
    }
    if (best < 1e30f) {
        int ta, tb;
        low_to_table(bc, ta, tb);
        tune_store(key, ta, tb);
        p.k1 = bc;
    }
}

static void tune_k4(dgf_dtype dt, bool gf32, const void* G, const void* P, const float2* dcoef, void* dP, void* dG,
                    int planes, int h_l, int w_l, int r, float eps, cudaStream_t s, Plan& p,
                    const float4* stats = nullptr) {
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{4, (int)dt, r, 0, 0, gf32 ? 1 : 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    float best = 1e30f;
    LowCfg bc = p.k4;
    for (const LowCfg& c : low_candidates(r, true, dt)) {
        const float ms = time_launch(s, [&] {
            return run_k4(dt, gf32, G, P, dcoef, dP, dG, planes, h_l, w_l, r, eps, c, s, c.fast == 2 ? stats : nullptr);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bc = c;
        }
    }
    if (best < 1e30f) {
        int ta, tb;
        low_to_table(bc, ta, tb);
        tune_store(key, ta, tb);
        p.k4 = bc;
    }
}

static void tune_k2(dgf_dtype dt, const float2* coef, const void* in, void* out, int planes, int h_l, int w_l,
                    int h, int w, cudaStream_t s, Plan& p) {
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{2, (int)dt, 0, p.F, p.vec, 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    float best = 1e30f;
    int bt = p.k2_strip ? p.k2_ls : p.k2_th;
    const std::initializer_list<int> strip_cand = {4, 6, 8, 12, 16, 24, 32}, tile_cand = {8, 16, 32, 64};
    for (int th : p.k2_strip ? strip_cand : tile_cand) {
        if (!p.k2_strip && k2_smem_bytes(p.vec, p.F, h_l, h, w_l, w, th) > smem_limit()) continue;
        const float ms = time_launch(s, [&] {
            return launch_k2_plan(dt, coef, in, out, planes, h_l, w_l, h, w, p, th, s);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bt = th;
        }
    }
    if (best < 1e30f) {
        tune_store(key, bt, 0);
        if (p.k2_strip)
            p.k2_ls = bt;
        else
            p.k2_th = bt;
    }
}

static void tune_k3(dgf_dtype dt, const float2* coef, const void* R, const void* G, void* dG, float2* dcoef,
                    int planes, int h_l, int w_l, int h, int w, cudaStream_t s, Plan& p) {
    if (!p.k3_fast) return;
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{3, (int)dt, 0, p.F, p.vec, 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    float best = 1e30f;
    int bl = p.k3_lth;
    K3Maps maps;
    const bool tma = make_k3_maps(maps, R, G, dt, planes, h, w, p.vec, p.F);
    for (int lth : {8, 12, 16, 20, 24, 32, 48, 64}) {  // intermediate lengths let a grid fill whole waves
        const float ms = time_launch(s, [&] {
            return launch_k3(dt, coef, R, G, dG, dcoef, planes, h_l, w_l, h, w, p.vec, p.F, lth,
                             tma ? &maps : nullptr, status_ptr(), s);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bl = lth;
        }
    }
    if (best < 1e30f) {
        tune_store(key, bl, 0);
        p.k3_lth = bl;
    }
}

// Whether the autotuner's table already holds the backward's shapes for this key.
static bool tune_has_low(dgf_dtype dt, int r, const Plan& p) {
    int a, b;
    if (!low_fast_radius(r)) return true;
    return tune_lookup(TuneKey{1, (int)dt, r, 0, 0, 0, p.sc}, a, b) &&
           tune_lookup(TuneKey{4, (int)dt, r, 0, 0, 0, p.sc}, a, b);
}
static bool tune_has_k3(dgf_dtype dt, const Plan& p) {
    int a, b;
    return !p.k3_fast || tune_lookup(TuneKey{3, (int)dt, 0, p.F, p.vec, 0, p.sc}, a, b);
}

// The fused forward against the two-kernel forward with its tuned shapes:
// records the fastest K12 segment length, or 0 when K1 + K2 win.
static void tune_k12(dgf_dtype dt, const void* G, const void* P, float2* coef, const void* in, void* out,
                     int planes, int h_l, int w_l, int h, int w, int r, float eps, cudaStream_t s, Plan& p) {
    if (!p.k12_ok) return;
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{5, (int)dt, r, p.F, 0, 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    size_t landing = 0;
    TmaPair tma = make_tma_pair(G, dt, P, dt, planes, h_l, w_l, r, p.k1, landing);
    const size_t smem = k1_cfg_smem(p.k1, r, tma.enabled ? landing : 0);
    float best = time_launch(s, [&] {
        cudaError_t e = launch_k1(dt, false, G, P, coef, planes, h_l, w_l, r, eps, p.k1, tma, smem, status_ptr(),
                                  nullptr, s);
        if (e != cudaSuccess) return e;
        return launch_k2_plan(dt, coef, in, out, planes, h_l, w_l, h, w, p, p.k2_strip ? p.k2_ls : p.k2_th, s);
    }, 3);
    if (best <= 0.f) best = 1e30f;
    int bl = 0;
    for (int ls : {8, 16, 32, 64}) {
        const float ms = time_launch(s, [&] {
            return launch_k12(dt, G, P, in, out, planes, h_l, w_l, h, w, r, p.F, eps, ls, s);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bl = ls;
        }
    }
    tune_store(key, bl, 0);
    p.k12 = bl > 0;
    if (bl > 0) p.k12_ls = bl;
}

// The fused backward K13 against K1 (with the statistics when K4 reads them)
// + K3 at their tuned shapes: records the fastest K13 segment length, or 0.
static void tune_k13(dgf_dtype dt, const void* G, const void* P, float2* coef, float4* stats, const void* R,
                     const void* Gh, void* dGh, float2* dcoef, int planes, int h_l, int w_l, int h, int w, int r,
                     float eps, const K3Maps& maps, cudaStream_t s, Plan& p) {
    if (!p.k13_ok) return;
    if (p.sc != 0) return;  // small planes keep the default shapes
    TuneKey key{6, (int)dt, r, p.F, p.vec, 0, p.sc};
    int a, b;
    if (tune_lookup(key, a, b)) return;
    size_t landing = 0;
    TmaPair tma = make_tma_pair(G, dt, P, dt, planes, h_l, w_l, r, p.k1, landing);
    const size_t smem = k1_cfg_smem(p.k1, r, tma.enabled ? landing : 0);
    float best = time_launch(s, [&] {
        cudaError_t e = launch_k1(dt, false, G, P, coef, planes, h_l, w_l, r, eps, p.k1, tma, smem, status_ptr(),
                                  stats, s);
        if (e != cudaSuccess) return e;
        return launch_k3(dt, coef, R, Gh, dGh, dcoef, planes, h_l, w_l, h, w, p.vec, p.F, p.k3_lth, &maps,
                         status_ptr(), s);
    }, 3);
    if (best <= 0.f) best = 1e30f;
    int bl = 0;
    for (int ls : {8, 12, 16, 24, 32}) {
        const float ms = time_launch(s, [&] {
            return launch_k13(dt, G, P, maps, dGh, dcoef, stats, planes, h_l, w_l, h, w, r, p.F, eps, ls,
                              status_ptr(), s);
        }, 3);
        if (ms > 0.f && ms < best) {
            best = ms;
            bl = ls;
        }
    }
    tune_store(key, bl, 0);
    p.k13 = bl > 0;
    if (bl > 0) p.k13_ls = bl;
}

// the strip forms' segment rows for this plane shape (fill_ls)
static LowCfg low_fill(LowCfg c, int r, int h_l, int w_l, bool k4) {
    if (c.fast == 2 && r >= 1) {
        const int out = k4 ? 32 - 4 * r : 64 - 4 * r;
        if (out > 0) c.a = fill_ls(c.a, (w_l + out - 1) / out, h_l, 4);
    }
    return c;
}

static cudaError_t run_k1(Launcher& L, dgf_dtype dt, bool gf32, const void* G, const void* P, float2* coef,
                          int planes, int h_l, int w_l, int r, float eps, const Plan& p, cudaStream_t s,
                          float4* stats = nullptr) {
    const LowCfg c = low_fill(p.k1, r, h_l, w_l, false);
    size_t landing = 0;
    TmaPair tma = make_tma_pair(G, gf32 ? DGF_F32 : dt, P, dt, planes, h_l, w_l, r, c, landing);
    const size_t smem = k1_cfg_smem(c, r, tma.enabled ? landing : 0);
    uint32_t* st = status_ptr();
    return L.run("k1_lowres_coef", [&] {
        return launch_k1(dt, gf32, G, P, coef, planes, h_l, w_l, r, eps, c, tma, smem, st, stats, s);
    });
}

}  // namespace dgf

// ------------------------------------------------------------------ batched
namespace dgf {

// One K1 node per radius present in the batch (each with the shared memory
// and grid of its own tile shape, so small radii keep full occupancy), all
// feeding one K2 node.  Keyed by (device, dtype, radii present).
struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> n1, n2;
};

std::mutex g_batch_mu;
// key: device, dtype, K1 classes (radius, form, lane width), K2 classes (staging, vector width, factor)
std::map<std::tuple<int, int, std::vector<int>, std::vector<int>>, BatchGraph> g_batch;

struct BatchPrep {
    BatchParams bp;
    size_t smem1 = 0, smem2 = 0;
    size_t maps = 0;  // workspace offset of the K2 tensor maps (one per image)
    size_t ws = 0;
};

dgf_status prepare_batch(const dgf_image* imgs, int n, dgf_dtype dt, char* ws_base, BatchPrep& out) {
    if (n < 0 || n > DGF_MAX_BATCH) return fail(DGF_ERR_INVALID, "batch size %d not in [0, %d]", n, DGF_MAX_BATCH);
    if (n > 0 && imgs == nullptr) return fail(DGF_ERR_INVALID, "image table is NULL");
    BatchParams& bp = out.bp;
    memset(&bp, 0, sizeof bp);
    bp.n = n;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const dgf_image& im = imgs[i];
        dgf_status st = check_sizes(1, im.C, im.h_l, im.w_l, im.h, im.w, im.r, im.eps, dt);
        if (st != DGF_OK) {
            const std::string why = t_err;
            return fail(st, "image %d: %s", i, why.c_str());
        }
        if (ws_base != nullptr &&
            (im.p_l == nullptr || im.I_l == nullptr || im.I_h == nullptr || im.O_h == nullptr))
            return fail(DGF_ERR_INVALID, "image %d: NULL pointer", i);
        if (reinterpret_cast<uintptr_t>(im.coef) % alignof(float2) != 0)
            return fail(DGF_ERR_INVALID, "image %d: coef must be 8-byte aligned", i);
        BatchImage& b = bp.img[i];
        b.p_l = im.p_l;
        b.I_l = im.I_l;
        b.I_h = im.I_h;
        b.O_h = im.O_h;
        b.C = im.C;
        b.h_l = im.h_l;
        b.w_l = im.w_l;
        b.h = im.h;
        b.w = im.w;
        b.r = im.r;
        b.eps = im.eps;
        Plan p = make_plan(dt, im.h_l, im.w_l, im.h, im.w, im.r, false, {im.I_h, im.O_h});
        // the persistent K2 runs strips where the single call does, else tiles
        // with fast taps for factors 4 and 8 only
        b.F = p.k2_strip ? p.F : ((p.F == 4 || p.F == 8) ? p.F : 0);
        b.vec = p.vec;
        if (p.k1.fast == 3) {  // sliding strips: the single call's segment rows and columns per lane
            if (p.k1.a == 0) p.k1.a = slide_auto_seg(im.h_l, im.r);
            if (p.k1.b == 0) p.k1.b = slide_k1_v(im.r);
        }
        b.k1_fast = p.k1.fast;
        b.k1_ty = p.k1.fast ? p.k1.b : p.k1.a;  // tiles: EY1; generic: TY; strips: 0; sliding: V
        b.k1_tx = p.k1.fast ? p.k1.a : p.k1.b;  // tiles: CW;  generic: TX; strips, sliding: rows per segment
        low_grid(p.k1, im.r, im.h_l, im.w_l, b.k1_nx, b.k1_ny);
        if (p.k2_strip) {
            // work items of kWarps strip segments (one per warp); k2_th = low-res rows per segment
            b.k2_th = p.k2_ls;
            const int K = b.vec / b.F;
            const int nstrip = (im.w_l + 32 * K - 1) / (32 * K), nseg = (im.h_l + b.k2_th - 1) / b.k2_th;
            b.k2_nx = (nstrip * nseg + kWarps - 1) / kWarps;
            b.k2_ny = 1;
        } else {
            b.k2_th = p.k2_th;
            b.k2_nx = (im.w + 32 * b.vec - 1) / (32 * b.vec);
            b.k2_ny = (im.h + b.k2_th - 1) / b.k2_th;
        }
        // the image's coefficients: in the caller's buffer when it keeps them, else a workspace slot
        b.coef = im.coef != nullptr ? static_cast<float2*>(im.coef)
                                    : (ws_base ? reinterpret_cast<float2*>(ws_base + off) : nullptr);
        off += align256((size_t)im.C * im.h_l * im.w_l * sizeof(float2));
        bp.k1_start[i + 1] = bp.k1_start[i] + b.k1_nx * b.k1_ny * im.C;
        bp.k2_start[i + 1] = bp.k2_start[i] + b.k2_nx * b.k2_ny * im.C;
        out.smem1 = std::max(out.smem1, k1_cfg_smem(p.k1, b.r, 0));
        out.smem2 = std::max(out.smem2, p.k2_strip ? k2_strip_batched_smem((int)esize(dt), b.vec, b.F)
                                                   : k2_smem_bytes(b.vec, b.F, b.h_l, b.h, b.w_l, b.w, b.k2_th));
    }
    bp.k1_total = bp.k1_start[n];
    bp.k2_total = bp.k2_start[n];
    out.maps = off;
    if (n > 0) off += align256((size_t)n * sizeof(K2Map));
    out.ws = off;
    return DGF_OK;
}

}  // namespace dgf


using namespace dgf;

// ====================================================================== ABI
namespace dgf {
// ----------------------------------------------------- plane-group pipeline
// One call's planes in G groups on two streams forked from the caller's: the
// low-resolution kernels (latency-bound, few warps per SM) on a stream of the
// greatest priority, the high-resolution kernels (HBM-bound) on a stream of
// the least, ordered per group by events.  The low-res pass of one group then
// runs while the high-res pass of another streams from HBM, instead of
// between them.  Every kernel sees exactly the planes and pointers it would
// in the one-stream order, so the results are the same bits.  Off by default
// (dgf_set_pipeline): the low-res walks are latency-bound, so a group's pass
// is nearly as long as the whole call's and the overlap does not pay.
constexpr int kPipeGroups = 3;
struct PipePool {
    int dev = -1;
    cudaStream_t lo = nullptr, hi = nullptr;
    cudaEvent_t fork = nullptr, join_lo = nullptr, join_hi = nullptr;
    cudaEvent_t k1[kPipeGroups] = {}, k3[kPipeGroups] = {};
};
static std::mutex g_pipe_mu;
static std::map<int, PipePool> g_pipe_pools;
static bool g_pipeline = false;

static cudaError_t pipe_pool(PipePool*& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    PipePool& p = g_pipe_pools[dev];
    if (p.dev < 0) {
        int least = 0, greatest = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&p.lo, cudaStreamNonBlocking, greatest)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&p.hi, cudaStreamNonBlocking, least)) != cudaSuccess) return e;
        cudaEvent_t* evs[] = {&p.fork, &p.join_lo, &p.join_hi};
        for (cudaEvent_t* ev : evs)
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        for (int g = 0; g < kPipeGroups; ++g) {
            if ((e = cudaEventCreateWithFlags(&p.k1[g], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.k3[g], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        p.dev = dev;
    }
    out = &p;
    return cudaSuccess;
}

// groups for a call of `planes` planes (1: no pipeline)
static int pipe_groups(int planes) {
    if (!g_pipeline) return 1;
    return planes >= 6 ? 3 : (planes >= 2 ? 2 : 1);
}

static cudaError_t pipe_fork(PipePool& p, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaEventRecord(p.fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(p.lo, p.fork, 0)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(p.hi, p.fork, 0);
}

static cudaError_t pipe_join(PipePool& p, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaEventRecord(p.join_lo, p.lo)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(p.join_hi, p.hi)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, p.join_lo, 0)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, p.join_hi, 0);
}

template <typename Ptr>
static Ptr* plane_off(Ptr* base, size_t elems) {
    return base == nullptr ? nullptr : base + elems;
}
static const void* byte_off(const void* base, size_t bytes) {
    return base == nullptr ? nullptr : static_cast<const char*>(base) + bytes;
}
static void* byte_off(void* base, size_t bytes) { return base == nullptr ? nullptr : static_cast<char*>(base) + bytes; }
}  // namespace dgf

extern "C" {

size_t dgf_workspace_size(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt, const dgf_guide* g) {
    if (check_sizes(N, C, h_l, w_l, h, w, r, 1.f, dt) != DGF_OK) return 0;
    return layout(N, C, h_l, w_l, g != nullptr, (size_t)N * C * h * w).total;
}

// The kept values of a call (dgf_options.coef): N C h_l w_l (Abar, bbar)
// pairs, then, with a guidance transform (C = 3), from the next 256-byte
// boundaries the low-res guide G_l and the high-res guide F(I_h) (FP32).
static float* kept_guide(float2* coef, int planes, int h_l, int w_l) {
    return reinterpret_cast<float*>(reinterpret_cast<char*>(coef) + align256((size_t)planes * h_l * w_l * sizeof(float2)));
}
static float* kept_guide_h(float2* coef, int planes, int h_l, int w_l) {
    const size_t lo = (size_t)planes * h_l * w_l;
    return reinterpret_cast<float*>(reinterpret_cast<char*>(coef) + align256(lo * sizeof(float2)) +
                                    align256(lo * sizeof(float)));
}

static dgf_status forward_impl(const void* p_l, const void* I_l, const void* I_h, void* O_h, int N, int C, int h_l,
                               int w_l, int h, int w, int r, float eps, dgf_dtype dt, const dgf_guide* g,
                               void* workspace, size_t ws_bytes, dgf_stream_t stream, bool mean_ab,
                               bool guide_low = false, bool guide_f32 = false, float2* coef_out = nullptr) {
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if ((st = check_guide(g, C, h_l, w_l, h, w, dt)) != DGF_OK) return st;
    if (guide_low && g == nullptr) return fail(DGF_ERR_INVALID, "guide_low needs a guidance transform");
    if (N == 0) return DGF_OK;
    if (p_l == nullptr || I_h == nullptr || O_h == nullptr || ((g == nullptr || guide_low) && I_l == nullptr))
        return fail(DGF_ERR_INVALID, "NULL input or output pointer");
    const Layout lay = layout(N, C, h_l, w_l, g != nullptr, (size_t)N * C * h * w);
    if ((st = check_ws(workspace, ws_bytes, lay.total)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    // the coefficients go to the caller's buffer when it keeps them for the
    // backward (the fused forward never writes them: the two kernels then)
    float2* coef = coef_out != nullptr ? coef_out : reinterpret_cast<float2*>(ws + lay.coef);
    const int planes = N * C;
    // an FP32 guide over 16-bit data (the grey guide): FP32 guide reads in K1
    // and the K2 tiles; the strip and fused forms read guides in dt
    const bool gf = guide_f32 && dt != DGF_F32;
    Plan p = make_plan(dt, h_l, w_l, h, w, r, g != nullptr || gf, {I_h, O_h}, mean_ab);
    if (coef_out != nullptr) p.k12_ok = p.k12 = false;
    Launcher L(s);
    cudaError_t e;
    const bool tuning = tune_enabled() && !stream_capturing(s) && mean_ab && !gf;
    if (gf) {
        // K1 over the FP32 grey guide: its own tuning key (guide_f32 = 1)
        if (tune_enabled() && !stream_capturing(s) && mean_ab)
            tune_k1(dt, true, I_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
        e = run_k1(L, dt, true, I_l, p_l, coef, planes, h_l, w_l, r, eps, p, s);
        if (e != cudaSuccess) return cuda_fail(e, "k1");
        e = L.run("k2_hires_apply", [&] {
            return launch_k2_guide_f32(dt, coef, static_cast<const float*>(I_h), O_h, planes, h_l, w_l, h, w, p.vec,
                                       p.F, p.k2_th, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k2");
        return DGF_OK;
    }
    if (g == nullptr) {
        if (tuning && p.k12_ok) {
            // shapes of the two-kernel forward first: K12 is timed against it
            tune_k1(dt, false, I_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
            tune_k2(dt, coef, I_h, O_h, planes, h_l, w_l, h, w, s, p);
            if (p.k1.fast == 2)
                tune_k12(dt, I_l, p_l, coef, I_h, O_h, planes, h_l, w_l, h, w, r, eps, s, p);
            else
                p.k12_ok = p.k12 = false;  // the tuner chose K1 tiles
        }
        if (p.k12) {
            const int ls = fill_ls(p.k12_ls, (w_l + 31) / 32, h_l, 2);
            e = L.run("k12_fused_forward", [&] {
                return launch_k12(dt, I_l, p_l, I_h, O_h, planes, h_l, w_l, h, w, r, p.F, eps, ls, s);
            });
            if (e != cudaSuccess) return cuda_fail(e, "k12");
            return DGF_OK;
        }
        if (tuning) {
            tune_k1(dt, false, I_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
            tune_k2(dt, coef, I_h, O_h, planes, h_l, w_l, h, w, s, p);
        }
        const int G = pipe_groups(planes);
        if (G == 1) {
            e = run_k1(L, dt, false, I_l, p_l, coef, planes, h_l, w_l, r, eps, p, s);
            if (e != cudaSuccess) return cuda_fail(e, "k1");
            e = L.run("k2_hires_apply", [&] {
                return launch_k2_plan(dt, coef, I_h, O_h, planes, h_l, w_l, h, w, p, p.k2_strip ? p.k2_ls : p.k2_th,
                                      s);
            });
            if (e != cudaSuccess) return cuda_fail(e, "k2");
            return DGF_OK;
        }
        // K1 of every group on the low-res stream, K2 of group g on the
        // high-res stream once K1 of group g is done
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        PipePool* pp = nullptr;
        if ((e = pipe_pool(pp)) != cudaSuccess) return cuda_fail(e, "pipeline streams");
        if ((e = pipe_fork(*pp, s)) != cudaSuccess) return cuda_fail(e, "pipeline fork");
        const size_t es = esize(dt), lw = (size_t)h_l * w_l, hw = (size_t)h * w;
        {
            Launcher Llo(pp->lo), Lhi(pp->hi);
            for (int gi = 0; gi < G; ++gi) {
                const int p0 = gi * planes / G, n = (gi + 1) * planes / G - p0;
                e = run_k1(Llo, dt, false, byte_off(I_l, p0 * lw * es), byte_off(p_l, p0 * lw * es), coef + p0 * lw, n,
                           h_l, w_l, r, eps, p, pp->lo);
                if (e != cudaSuccess) return cuda_fail(e, "k1");
                if ((e = cudaEventRecord(pp->k1[gi], pp->lo)) != cudaSuccess) return cuda_fail(e, "pipeline event");
            }
            for (int gi = 0; gi < G; ++gi) {
                const int p0 = gi * planes / G, n = (gi + 1) * planes / G - p0;
                if ((e = cudaStreamWaitEvent(pp->hi, pp->k1[gi], 0)) != cudaSuccess) return cuda_fail(e, "pipeline wait");
                e = Lhi.run("k2_hires_apply", [&] {
                    return launch_k2_plan(dt, coef + p0 * lw, byte_off(I_h, p0 * hw * es), byte_off(O_h, p0 * hw * es), n,
                                          h_l, w_l, h, w, p, p.k2_strip ? p.k2_ls : p.k2_th, pp->hi);
                });
                if (e != cudaSuccess) return cuda_fail(e, "k2");
            }
        }
        if ((e = pipe_join(*pp, s)) != cudaSuccess) return cuda_fail(e, "pipeline join");
        return DGF_OK;
    }
    // G_l goes to the caller's buffer after the coefficients when it keeps them
    float* G_l = coef_out != nullptr ? kept_guide(coef_out, planes, h_l, w_l) : reinterpret_cast<float*>(ws + lay.gl);
    // with G_l the block mean of F(I_h), K5 also keeps F(I_h) in FP32 and K2
    // reads that guide instead of evaluating F again per pixel (kept for the
    // backward's K3g when the caller keeps the forward's values)
    float* G_h = guide_low ? nullptr
                           : (coef_out != nullptr ? kept_guide_h(coef_out, planes, h_l, w_l)
                                                  : reinterpret_cast<float*>(ws + lay.gh));
    if (!aligned16({I_h, O_h})) return fail(DGF_ERR_UNSUPPORTED, "guidance transform needs 16-byte aligned I_h, O_h");
    e = guide_upload(g->w1, g->w2, g->b2, g->hidden, s);
    if (e != cudaSuccess) return cuda_fail(e, "guide weights");
    if (guide_low)
        e = L.run("k5_guide_low", [&] { return launch_k5_low(dt, I_l, G_l, N, h_l, w_l, g->slope, s); });
    else
        e = L.run("k5_guide_down",
                  [&] { return launch_k5(dt, I_h, G_l, N, h_l, w_l, h, w, p.F, g->slope, s, G_h); });
    if (e != cudaSuccess) return cuda_fail(e, "k5");
    // K1 over the FP32 low-res guide: its own tuning key (guide_f32 = 1)
    if (tune_enabled() && !stream_capturing(s) && mean_ab)
        tune_k1(dt, true, G_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
    e = run_k1(L, dt, true, G_l, p_l, coef, planes, h_l, w_l, r, eps, p, s);
    if (e != cudaSuccess) return cuda_fail(e, "k1");
    if (G_h != nullptr) {
        e = L.run("k2_hires_apply", [&] {
            return launch_k2_guide_f32(dt, coef, G_h, O_h, planes, h_l, w_l, h, w, p.vec, p.F, p.k2_th, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k2");
        return DGF_OK;
    }
    e = L.run("k2_hires_apply_guided", [&] {
        return launch_k2_guided(dt, coef, I_h, O_h, N, h_l, w_l, h, w, p.F, 8, g->slope, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "k2g");
    return DGF_OK;
}

// Backward without the guidance transform for one call (N C planes): K1
// (coefficients, and the window statistics when both low-res stages are
// strips) -> K3 -> K4, on stream s, in the workspace slice `ws` laid out by
// `lay`.  Shared by dgf_backward and dgf_backward_batched.
static dgf_status backward_plain(Launcher& L, dgf_dtype dt, const void* dO_h, const void* p_l, const void* I_l,
                                 const void* I_h, void* dp_l, void* dI_l, void* dI_h, int planes, int h_l, int w_l,
                                 int h, int w, int r, float eps, Plan& p, char* ws, const Layout& lay, cudaStream_t s,
                                 bool tuning, bool gf = false, const float2* coef_in = nullptr) {
    float2* coef = reinterpret_cast<float2*>(ws + lay.coef);
    float2* dcoef = reinterpret_cast<float2*>(ws + lay.dcoef);
    cudaError_t e;
    // coefficients are recomputed unless the forward's are given; with
    // both low-res stages in strip form the K1 pass also keeps each
    // window's statistics for K4, which then skips recomputing them (and
    // the K1 pass runs whether or not the coefficients are given)
    const bool need_k4 = dp_l != nullptr || dI_l != nullptr;
    if (tuning && (dI_h != nullptr || need_k4)) tune_k1(dt, gf, I_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
    // K4's form decides whether the K1 pass saves statistics, so it is tuned
    // before that pass, on whatever the workspace holds (timing only; the
    // real K4 launch below overwrites its outputs): the first call of a key
    // then runs exactly the kernels of every later call
    if (tuning && need_k4)
        tune_k4(dt, gf, I_l, p_l, dcoef, dp_l, dI_l, planes, h_l, w_l, r, eps, s, p,
                p.k1.fast == 2 ? reinterpret_cast<float4*>(ws + lay.stats) : nullptr);
    const bool use_stats = need_k4 && p.k1.fast == 2 && p.k4.fast == 2;
    float4* stats = use_stats ? reinterpret_cast<float4*>(ws + lay.stats) : nullptr;
    // the forward's coefficients stand in for a K1 pass that would compute nothing else
    const bool reuse = coef_in != nullptr && !use_stats;
    if (reuse) p.k13_ok = p.k13 = false;
    float2* cf = reuse ? const_cast<float2*>(coef_in) : coef;  // read only from here on
    bool fused = false;
    if (p.k13_ok && p.k3_fast) {
        // K1 + K3 as one kernel (the tuner, when on, times it against the pair)
        K3Maps maps;
        if (make_k3_maps(maps, dO_h, I_h, dt, planes, h, w, p.vec, p.F)) {
            if (tuning) {
                tune_k3(dt, coef, dO_h, I_h, dI_h, dcoef, planes, h_l, w_l, h, w, s, p);
                tune_k13(dt, I_l, p_l, coef, stats, dO_h, I_h, dI_h, dcoef, planes, h_l, w_l, h, w, r, eps, maps, s,
                         p);
            }
            if (p.k13) {
                const int ls = fill_ls(p.k13_ls, (w_l + 29) / 30, h_l, 2);
                e = L.run("k13_fused_backward", [&] {
                    return launch_k13(dt, I_l, p_l, maps, dI_h, dcoef, stats, planes, h_l, w_l, h, w, r, p.F, eps,
                                      ls, status_ptr(), s);
                });
                if (e != cudaSuccess) return cuda_fail(e, "k13");
                fused = true;
            }
        }
    }
    if (!fused && !reuse && (dI_h != nullptr || use_stats)) {
        e = run_k1(L, dt, gf, I_l, p_l, coef, planes, h_l, w_l, r, eps, p, s, stats);
        if (e != cudaSuccess) return cuda_fail(e, "k1");
    }
    if (fused) {
        // K13 wrote d Abar, d bbar (and the statistics)
    } else if (p.k3_fast) {
        if (tuning) tune_k3(dt, cf, dO_h, I_h, dI_h, dcoef, planes, h_l, w_l, h, w, s, p);
        K3Maps maps;
        const bool tma = make_k3_maps(maps, dO_h, I_h, dt, planes, h, w, p.vec, p.F);
        e = L.run("k3_hires_bwd", [&] {
            return launch_k3(dt, cf, dO_h, I_h, dI_h, dcoef, planes, h_l, w_l, h, w, p.vec, p.F,
                             fill_ls(p.k3_lth, (w_l + 30 * (p.vec / p.F) - 1) / (30 * (p.vec / p.F)), h_l, 2),
                             tma ? &maps : nullptr, status_ptr(), s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k3");
    } else {
        if (dI_h != nullptr) {
            e = L.run("k2_hires_scale", [&] {
                return launch_k2(dt, 1, cf, dO_h, dI_h, planes, h_l, w_l, h, w, p.vec, p.F, p.k2_th, s);
            });
            if (e != cudaSuccess) return cuda_fail(e, "k2 scale");
        }
        e = L.run("k3_gather_general", [&] {
            return launch_k3_general(dt, dO_h, I_h, dcoef, planes, h_l, w_l, h, w, s, gf);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k3 general");
    }
    if (need_k4) {
        const float4* k4_stats = p.k4.fast == 2 ? stats : nullptr;
        e = L.run("k4_lowres_bwd", [&] {
            return run_k4(dt, gf, I_l, p_l, dcoef, dp_l, dI_l, planes, h_l, w_l, r, eps, p.k4, s, k4_stats);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k4");
    }
    return DGF_OK;
}

// backward_plain with the planes in groups on the two pipeline streams:
// K1 (low-res stream) -> K3 (high-res stream) -> K4 (low-res stream) per group.
static dgf_status backward_pipelined(dgf_dtype dt, const void* dO_h, const void* p_l, const void* I_l,
                                     const void* I_h, void* dp_l, void* dI_l, void* dI_h, int planes, int h_l, int w_l,
                                     int h, int w, int r, float eps, const Plan& p, char* ws, const Layout& lay,
                                     cudaStream_t s, int G, const float2* coef_in) {
    float2* coef = reinterpret_cast<float2*>(ws + lay.coef);
    float2* dcoef = reinterpret_cast<float2*>(ws + lay.dcoef);
    const bool need_k4 = dp_l != nullptr || dI_l != nullptr;
    const bool use_stats = need_k4 && p.k1.fast == 2 && p.k4.fast == 2;
    float4* stats = use_stats ? reinterpret_cast<float4*>(ws + lay.stats) : nullptr;
    const bool reuse = coef_in != nullptr && !use_stats;  // the forward's coefficients stand in for K1's
    const float2* cf = reuse ? coef_in : coef;
    const bool need_k1 = !reuse && (dI_h != nullptr || use_stats);
    const size_t es = esize(dt), lw = (size_t)h_l * w_l, hw = (size_t)h * w;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    PipePool* pp = nullptr;
    cudaError_t e;
    if ((e = pipe_pool(pp)) != cudaSuccess) return cuda_fail(e, "pipeline streams");
    if ((e = pipe_fork(*pp, s)) != cudaSuccess) return cuda_fail(e, "pipeline fork");
    {
        Launcher Llo(pp->lo), Lhi(pp->hi);
        auto grp = [&](int gi, int& p0, int& n) {
            p0 = gi * planes / G;
            n = (gi + 1) * planes / G - p0;
        };
        for (int gi = 0; gi < G; ++gi) {
            int p0, n;
            grp(gi, p0, n);
            if (need_k1) {
                e = run_k1(Llo, dt, false, byte_off(I_l, p0 * lw * es), byte_off(p_l, p0 * lw * es), coef + p0 * lw, n,
                           h_l, w_l, r, eps, p, pp->lo, plane_off(stats, p0 * lw));
                if (e != cudaSuccess) return cuda_fail(e, "k1");
            }
            if ((e = cudaEventRecord(pp->k1[gi], pp->lo)) != cudaSuccess) return cuda_fail(e, "pipeline event");
        }
        for (int gi = 0; gi < G; ++gi) {
            int p0, n;
            grp(gi, p0, n);
            if ((e = cudaStreamWaitEvent(pp->hi, pp->k1[gi], 0)) != cudaSuccess) return cuda_fail(e, "pipeline wait");
            const void* dO = byte_off(dO_h, p0 * hw * es);
            const void* G_h = byte_off(I_h, p0 * hw * es);
            void* dG_h = byte_off(dI_h, p0 * hw * es);
            K3Maps maps;
            const bool tma = make_k3_maps(maps, dO, G_h, dt, n, h, w, p.vec, p.F);
            e = Lhi.run("k3_hires_bwd", [&] {
                return launch_k3(dt, cf + p0 * lw, dO, G_h, dG_h, dcoef + p0 * lw, n, h_l, w_l, h, w, p.vec, p.F,
                                 fill_ls(p.k3_lth, (w_l + 30 * (p.vec / p.F) - 1) / (30 * (p.vec / p.F)), h_l, 2),
                                 tma ? &maps : nullptr, status_ptr(), pp->hi);
            });
            if (e != cudaSuccess) return cuda_fail(e, "k3");
            if ((e = cudaEventRecord(pp->k3[gi], pp->hi)) != cudaSuccess) return cuda_fail(e, "pipeline event");
        }
        if (need_k4) {
            const float4* k4_stats = p.k4.fast == 2 ? stats : nullptr;
            for (int gi = 0; gi < G; ++gi) {
                int p0, n;
                grp(gi, p0, n);
                if ((e = cudaStreamWaitEvent(pp->lo, pp->k3[gi], 0)) != cudaSuccess) return cuda_fail(e, "pipeline wait");
                e = Llo.run("k4_lowres_bwd", [&] {
                    return run_k4(dt, false, byte_off(I_l, p0 * lw * es), byte_off(p_l, p0 * lw * es), dcoef + p0 * lw,
                                  byte_off(dp_l, p0 * lw * es), byte_off(dI_l, p0 * lw * es), n, h_l, w_l, r, eps,
                                  p.k4, pp->lo, plane_off(k4_stats, p0 * lw));
                });
                if (e != cudaSuccess) return cuda_fail(e, "k4");
            }
        }
    }
    if ((e = pipe_join(*pp, s)) != cudaSuccess) return cuda_fail(e, "pipeline join");
    return DGF_OK;
}

static dgf_status backward_impl(const void* dO_h, const void* p_l, const void* I_l, const void* I_h, void* dp_l,
                                void* dI_l, void* dI_h, float* dW, int N, int C, int h_l, int w_l, int h, int w,
                                int r, float eps, dgf_dtype dt, const dgf_guide* g, void* workspace,
                                size_t ws_bytes, dgf_stream_t stream, bool mean_ab, bool guide_low = false,
                                bool guide_f32 = false, const float2* coef_in = nullptr) {
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if ((st = check_guide(g, C, h_l, w_l, h, w, dt)) != DGF_OK) return st;
    if (guide_low && g == nullptr) return fail(DGF_ERR_INVALID, "guide_low needs a guidance transform");
    if (g != nullptr && dI_l != nullptr && !guide_low)
        return fail(DGF_ERR_INVALID, "dI_l must be NULL with a guidance transform (unless guide_low)");
    if (g == nullptr && dW != nullptr) return fail(DGF_ERR_INVALID, "dW needs a guidance transform");
    if (N == 0) {
        if (g != nullptr && dW != nullptr) {
            cudaError_t e = cudaMemsetAsync(dW, 0, sizeof(float) * (6 * g->hidden + 3),
                                            reinterpret_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return cuda_fail(e, "memset dW");
        }
        return DGF_OK;
    }
    if (dO_h == nullptr || p_l == nullptr || I_h == nullptr || ((g == nullptr || guide_low) && I_l == nullptr))
        return fail(DGF_ERR_INVALID, "NULL input pointer");
    const Layout lay = layout(N, C, h_l, w_l, g != nullptr, (size_t)N * C * h * w);
    if ((st = check_ws(workspace, ws_bytes, lay.total)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    float2* coef = reinterpret_cast<float2*>(ws + lay.coef);
    float2* dcoef = reinterpret_cast<float2*>(ws + lay.dcoef);
    const int planes = N * C;
    const bool gf = guide_f32 && dt != DGF_F32;  // FP32 guide over 16-bit data (the grey guide)
    Plan p = make_plan(dt, h_l, w_l, h, w, r, g != nullptr || gf, {dO_h, I_h, dI_h}, mean_ab);
    Launcher L(s);
    cudaError_t e;
    if (gf) {
        // K1 and K4 read the FP32 guide; the high-res gradients come from the
        // general K2 (d I_h = d O_h * Abar_h) and K3 gather (FP32 guide reads)
        p.k3_fast = false;
        p.k13_ok = p.k13 = false;
        if (dp_l == nullptr && dI_l == nullptr && dI_h == nullptr) return DGF_OK;
        return backward_plain(L, dt, dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, planes, h_l, w_l, h, w, r, eps, p, ws,
                              lay, s, tune_enabled() && !stream_capturing(s) && mean_ab, true, coef_in);
    }
    if (g == nullptr) {
        if (dp_l == nullptr && dI_l == nullptr && dI_h == nullptr) return DGF_OK;
        const bool tuning = tune_enabled() && !stream_capturing(s) && mean_ab;
        const int G = p.k3_fast ? pipe_groups(planes) : 1;
        const bool tuned = !tuning || (tune_has_low(dt, r, p) && tune_has_k3(dt, p));
        if (G == 1 || !tuned)  // the first call of a key tunes (one stream), later calls pipeline
            return backward_plain(L, dt, dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, planes, h_l, w_l, h, w, r, eps, p, ws,
                                  lay, s, tuning, false, coef_in);
        return backward_pipelined(dt, dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, planes, h_l, w_l, h, w, r, eps, p, ws, lay,
                                  s, G, coef_in);
    }
    // with the guidance transform; G_l is the forward's when it kept it
    float* G_l = coef_in != nullptr ? kept_guide(const_cast<float2*>(coef_in), planes, h_l, w_l)
                                    : reinterpret_cast<float*>(ws + lay.gl);
    float* dG_l = reinterpret_cast<float*>(ws + lay.dgl);
    float* partials = reinterpret_cast<float*>(ws + lay.partials);
    const bool need_hi = dI_h != nullptr || dW != nullptr;
    // with F applied to I_l, d G_l goes back through F at low resolution (K6L)
    // instead of into K6's d G_h
    const bool need_lo = guide_low && (dI_l != nullptr || dW != nullptr);
    if (!aligned16({dO_h, I_h, dI_h}))
        return fail(DGF_ERR_UNSUPPORTED, "guidance transform needs 16-byte aligned dO_h, I_h, dI_h");
    e = guide_upload(g->w1, g->w2, g->b2, g->hidden, s);
    if (e != cudaSuccess) return cuda_fail(e, "guide weights");
    if (coef_in != nullptr)
        e = cudaSuccess;  // G_l kept by the forward
    else if (guide_low)
        e = L.run("k5_guide_low", [&] { return launch_k5_low(dt, I_l, G_l, N, h_l, w_l, g->slope, s); });
    else
        e = L.run("k5_guide_down", [&] { return launch_k5(dt, I_h, G_l, N, h_l, w_l, h, w, p.F, g->slope, s); });
    if (e != cudaSuccess) return cuda_fail(e, "k5");
    const bool gtune = tune_enabled() && !stream_capturing(s) && mean_ab;
    // Abar for K6: the forward's when given, else recomputed
    if (coef_in != nullptr) {
        coef = const_cast<float2*>(coef_in);  // read only from here on
    } else {
        if (gtune) tune_k1(dt, true, G_l, p_l, coef, planes, h_l, w_l, r, eps, s, p);
        e = run_k1(L, dt, true, G_l, p_l, coef, planes, h_l, w_l, r, eps, p, s);
        if (e != cudaSuccess) return cuda_fail(e, "k1");
    }
    e = L.run("k3_hires_bwd_guided", [&] {
        return launch_k3_guided(dt, dO_h, I_h, dcoef, N, h_l, w_l, h, w, p.F, g->slope, s,
                                (coef_in != nullptr && !guide_low)
                                    ? kept_guide_h(const_cast<float2*>(coef_in), planes, h_l, w_l)
                                    : nullptr);
    });
    if (e != cudaSuccess) return cuda_fail(e, "k3g");
    const bool want_dgl = guide_low ? need_lo : need_hi;
    if (dp_l != nullptr || want_dgl) {
        // timing only: the K4 launch below overwrites what the candidates wrote
        if (gtune) tune_k4(dt, true, G_l, p_l, dcoef, dp_l, want_dgl ? dG_l : nullptr, planes, h_l, w_l, r, eps, s, p);
        e = L.run("k4_lowres_bwd", [&] {
            return run_k4(dt, true, G_l, p_l, dcoef, dp_l, want_dgl ? dG_l : nullptr, planes, h_l, w_l, r, eps,
                          p.k4, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k4");
    }
    int rows = 0;  // weight-gradient partial rows written
    if (need_hi) {
        e = L.run("k6_guide_bwd", [&] {
            return launch_k6(dt, coef, guide_low ? nullptr : dG_l, dO_h, I_h, dI_h, partials, N, h_l, w_l, h, w,
                             p.F, g->slope, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k6");
        rows = k6_blocks(N, h, w);
    }
    if (need_lo) {
        if (rows + k6_low_blocks(N, h_l, w_l) > kMaxK6Blocks)
            return fail(DGF_ERR_UNSUPPORTED, "weight-gradient partial rows exceed %d", kMaxK6Blocks);
        e = L.run("k6_guide_low", [&] {
            return launch_k6_low(dt, dG_l, I_l, dI_l, partials + (size_t)rows * kWGradPadded, N, h_l, w_l,
                                 g->slope, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k6l");
        rows += k6_low_blocks(N, h_l, w_l);
    }
    if (dW != nullptr) {
        e = L.run("k6_weight_reduce", [&] { return launch_wreduce(partials, rows, dW, g->hidden, s); });
        if (e != cudaSuccess) return cuda_fail(e, "k6 reduce");
    }
    return DGF_OK;
}

dgf_status dgf_forward(const void* p_l, const void* I_l, const void* I_h, void* O_h, int N, int C, int h_l,
                       int w_l, int h, int w, int r, float eps, dgf_dtype dt, const dgf_guide* g, void* workspace,
                       size_t ws_bytes, dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    return forward_impl(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, workspace, ws_bytes, stream, true);
}

// Grey guide (Sec. 4.2, DGF_b): the guide's channel count when it differs from the
// output's C (its channel mean then guides every output channel); 0 when the
// guide has the output's channels (F the identity).
static int grey_channels(const dgf_options* opt, int C) {
    if (opt == nullptr) return 0;
    const int n = opt->guide_channels;
    return (n == 0 || n == C) ? 0 : n;
}

// Workspace of a grey-guide call: the plain layout, then the grey guide at
// both resolutions repeated over the C output channels, then their gradients.
struct GreyLayout {
    size_t gl, gh, dgl, dgh, total;
};

static GreyLayout grey_layout(int N, int C, int h_l, int w_l, int h, int w, dgf_dtype dt) {
    GreyLayout L;
    size_t off = layout(N, C, h_l, w_l, false).total;
    const size_t lo = (size_t)N * C * h_l * w_l, hi = (size_t)N * C * h * w;
    L.gl = off;  // the grey guides, FP32
    off += align256(lo * 4);
    L.gh = off;
    off += align256(hi * 4);
    L.dgl = off;  // their gradients per output channel: FP32 at low res (K4 with an FP32 guide), dt at high res
    off += align256(lo * 4);
    L.dgh = off;
    off += align256(hi * esize(dt));
    L.total = off;
    return L;
}

static dgf_status check_grey(int n_in, int N, const dgf_guide* g) {
    if (n_in < 1) return fail(DGF_ERR_INVALID, "guide_channels = %d < 0", n_in);
    if ((long long)N * n_in > 65535) return fail(DGF_ERR_UNSUPPORTED, "N*guide_channels > 65535 planes");
    if (g != nullptr) return fail(DGF_ERR_INVALID, "a grey guide and a guidance transform exclude each other");
    return DGF_OK;
}

static bool g_grey_fold = true;

// The folded grey-guide forms (the high-resolution guide formed in the
// kernels' registers) serve an integer factor F in {2, 4, 8} with vector
// access to the high-resolution tensors; their vector width, else 0.
static int grey_fold(dgf_dtype dt, int C, int h_l, int w_l, int h, int w, std::initializer_list<const void*> ptrs) {
    if (!g_grey_fold) return 0;
    const int F = integer_factor(h_l, w_l, h, w);
    return F > 0 ? grey_fold_vec(dt, F, C, w, ptrs) : 0;
}

static dgf_status forward_grey(const void* p_l, const void* I_l, const void* I_h, void* O_h, int N, int C, int h_l,
                               int w_l, int h, int w, int r, float eps, dgf_dtype dt, const dgf_guide* g,
                               void* workspace, size_t ws_bytes, dgf_stream_t stream, bool mean_ab, int n_in,
                               float2* coef_out) {
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if ((st = check_grey(n_in, N, g)) != DGF_OK) return st;
    if (N == 0) return DGF_OK;
    if (p_l == nullptr || I_l == nullptr || I_h == nullptr || O_h == nullptr)
        return fail(DGF_ERR_INVALID, "NULL input or output pointer");
    const GreyLayout gl = grey_layout(N, C, h_l, w_l, h, w, dt);
    if ((st = check_ws(workspace, ws_bytes, gl.total)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    Launcher L(s);
    float* Gl = reinterpret_cast<float*>(ws + gl.gl);
    float* Gh = reinterpret_cast<float*>(ws + gl.gh);
    cudaError_t e = L.run("grey_guide", [&] {
        return launch_grey_mean(dt, I_l, Gl, N, n_in, C, (size_t)h_l * w_l, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "grey guide");
    if (const int vec = grey_fold(dt, C, h_l, w_l, h, w, {I_h, O_h}); vec != 0) {
        // K1 over the low-res grey guide (FP32), then K2 forming G_h itself
        const int planes = N * C;
        float2* coef = coef_out != nullptr ? coef_out : reinterpret_cast<float2*>(ws + layout(N, C, h_l, w_l, false).coef);
        Plan p = make_plan(dt, h_l, w_l, h, w, r, true, {I_h, O_h}, mean_ab);
        if (tune_enabled() && !stream_capturing(s) && mean_ab)
            tune_k1(dt, true, Gl, p_l, coef, planes, h_l, w_l, r, eps, s, p);
        e = run_k1(L, dt, true, Gl, p_l, coef, planes, h_l, w_l, r, eps, p, s);
        if (e != cudaSuccess) return cuda_fail(e, "k1");
        e = L.run("k2_grey_apply",
                  [&] { return launch_k2_grey(dt, coef, I_h, O_h, N, C, n_in, h_l, w_l, h, w, p.F, vec, s); });
        if (e != cudaSuccess) return cuda_fail(e, "k2 grey");
        return DGF_OK;
    }
    e = L.run("grey_guide", [&] { return launch_grey_mean(dt, I_h, Gh, N, n_in, C, (size_t)h * w, s); });
    if (e != cudaSuccess) return cuda_fail(e, "grey guide");
    return forward_impl(p_l, Gl, Gh, O_h, N, C, h_l, w_l, h, w, r, eps, dt, nullptr, workspace, ws_bytes, stream,
                        mean_ab, false, true, coef_out);
}

// opt->coef as the call's buffer of kept values: NULL, or 256-byte aligned
static dgf_status opt_coef(const dgf_options* opt, float2*& coef) {
    coef = opt != nullptr ? static_cast<float2*>(opt->coef) : nullptr;
    if (reinterpret_cast<uintptr_t>(coef) % 256 != 0)
        return fail(DGF_ERR_INVALID, "coef must be 256-byte aligned");
    return DGF_OK;
}

dgf_status dgf_forward_opt(const void* p_l, const void* I_l, const void* I_h, void* O_h, int N, int C, int h_l,
                           int w_l, int h, int w, int r, float eps, dgf_dtype dt, const dgf_guide* g,
                           void* workspace, size_t ws_bytes, dgf_stream_t stream, const dgf_options* opt) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    const bool mean_ab = opt == nullptr || opt->mean_ab != 0;
    const int n_in = grey_channels(opt, C);
    float2* coef = nullptr;
    if (dgf_status st = opt_coef(opt, coef); st != DGF_OK) return st;
    if (n_in != 0)
        return forward_grey(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, workspace, ws_bytes, stream,
                            mean_ab, n_in, coef);
    return forward_impl(p_l, I_l, I_h, O_h, N, C, h_l, w_l, h, w, r, eps, dt, g, workspace, ws_bytes, stream,
                        mean_ab, opt != nullptr && opt->guide_low != 0, false, coef);
}

dgf_status dgf_backward(const void* dO_h, const void* p_l, const void* I_l, const void* I_h, void* dp_l, void* dI_l,
                        void* dI_h, float* dW, int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                        dgf_dtype dt, const dgf_guide* g, void* workspace, size_t ws_bytes, dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    return backward_impl(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps, dt, g, workspace,
                         ws_bytes, stream, true);
}

static dgf_status backward_grey(const void* dO_h, const void* p_l, const void* I_l, const void* I_h, void* dp_l,
                                void* dI_l, void* dI_h, float* dW, int N, int C, int h_l, int w_l, int h, int w,
                                int r, float eps, dgf_dtype dt, const dgf_guide* g, void* workspace,
                                size_t ws_bytes, dgf_stream_t stream, bool mean_ab, int n_in,
                                const float2* coef_in) {
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if ((st = check_grey(n_in, N, g)) != DGF_OK) return st;
    if (dW != nullptr) return fail(DGF_ERR_INVALID, "dW needs a guidance transform");
    if (N == 0 || (dp_l == nullptr && dI_l == nullptr && dI_h == nullptr)) return DGF_OK;
    if (dO_h == nullptr || p_l == nullptr || I_l == nullptr || I_h == nullptr)
        return fail(DGF_ERR_INVALID, "NULL input pointer");
    const GreyLayout gl = grey_layout(N, C, h_l, w_l, h, w, dt);
    if ((st = check_ws(workspace, ws_bytes, gl.total)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    if (const int vec = grey_fold(dt, C, h_l, w_l, h, w, {dO_h, I_h, dI_h}); vec != 0) {
        // the low-res grey guide (FP32); K1 (Abar, bbar, for d I_h only) ->
        // K3 forming G_h itself and writing d I_h -> K4 (d p_l and d G_l per
        // output channel) -> d I_l from the d G_l sums
        Launcher L(s);
        const int planes = N * C;
        const Layout lay = layout(N, C, h_l, w_l, false);
        float2* coef = reinterpret_cast<float2*>(ws + lay.coef);
        float2* dcoef = reinterpret_cast<float2*>(ws + lay.dcoef);
        float* Gl = reinterpret_cast<float*>(ws + gl.gl);
        float* dGl = reinterpret_cast<float*>(ws + gl.dgl);
        Plan p = make_plan(dt, h_l, w_l, h, w, r, true, {dO_h, I_h, dI_h}, mean_ab);
        const bool tuning = tune_enabled() && !stream_capturing(s) && mean_ab;
        const bool need_k4 = dp_l != nullptr || dI_l != nullptr;
        cudaError_t e = L.run("grey_guide", [&] {
            return launch_grey_mean(dt, I_l, Gl, N, n_in, C, (size_t)h_l * w_l, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "grey guide");
        if (coef_in != nullptr) {
            coef = const_cast<float2*>(coef_in);  // the forward's Abar: read only
        } else if (dI_h != nullptr) {
            if (tuning) tune_k1(dt, true, Gl, p_l, coef, planes, h_l, w_l, r, eps, s, p);
            e = run_k1(L, dt, true, Gl, p_l, coef, planes, h_l, w_l, r, eps, p, s);
            if (e != cudaSuccess) return cuda_fail(e, "k1");
        }
        e = L.run("k3_grey_bwd", [&] {
            return launch_k3_grey(dt, dO_h, I_h, coef, dcoef, dI_h, N, C, n_in, h_l, w_l, h, w, p.F, vec, s);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k3 grey");
        if (need_k4) {
            // timing only: the K4 launch below overwrites what the candidates wrote
            if (tuning) tune_k4(dt, true, Gl, p_l, dcoef, dp_l, dI_l ? dGl : nullptr, planes, h_l, w_l, r, eps, s, p);
            e = L.run("k4_lowres_bwd", [&] {
                return run_k4(dt, true, Gl, p_l, dcoef, dp_l, dI_l ? dGl : nullptr, planes, h_l, w_l, r, eps, p.k4, s);
            });
            if (e != cudaSuccess) return cuda_fail(e, "k4");
        }
        if (dI_l != nullptr) {
            e = L.run("grey_guide_adjoint", [&] {
                return launch_grey_adjoint(dt, true, dGl, dI_l, N, n_in, C, (size_t)h_l * w_l, s);
            });
            if (e != cudaSuccess) return cuda_fail(e, "grey guide adjoint");
        }
        return DGF_OK;
    }
    {
        Launcher L(s);
        cudaError_t e = L.run("grey_guide", [&] {
            return launch_grey_mean(dt, I_l, reinterpret_cast<float*>(ws + gl.gl), N, n_in, C, (size_t)h_l * w_l, s);
        });
        if (e == cudaSuccess)
            e = L.run("grey_guide", [&] {
                return launch_grey_mean(dt, I_h, reinterpret_cast<float*>(ws + gl.gh), N, n_in, C, (size_t)h * w, s);
            });
        if (e != cudaSuccess) return cuda_fail(e, "grey guide");
    }
    // Algorithm 1 per output channel with the repeated grey guide, its guide
    // gradients into the workspace, then their sum over the channels / n_I
    st = backward_impl(dO_h, p_l, ws + gl.gl, ws + gl.gh, dp_l, dI_l ? ws + gl.dgl : nullptr,
                       dI_h ? ws + gl.dgh : nullptr, nullptr, N, C, h_l, w_l, h, w, r, eps, dt, nullptr, workspace,
                       ws_bytes, stream, mean_ab, false, true, coef_in);
    if (st != DGF_OK) return st;
    Launcher L(s);
    cudaError_t e = cudaSuccess;
    if (dI_l != nullptr)
        e = L.run("grey_guide_adjoint", [&] {
            return launch_grey_adjoint(dt, true, ws + gl.dgl, dI_l, N, n_in, C, (size_t)h_l * w_l, s);
        });
    if (e == cudaSuccess && dI_h != nullptr)
        e = L.run("grey_guide_adjoint",
                  [&] { return launch_grey_adjoint(dt, false, ws + gl.dgh, dI_h, N, n_in, C, (size_t)h * w, s); });
    if (e != cudaSuccess) return cuda_fail(e, "grey guide adjoint");
    return DGF_OK;
}

dgf_status dgf_backward_opt(const void* dO_h, const void* p_l, const void* I_l, const void* I_h, void* dp_l,
                            void* dI_l, void* dI_h, float* dW, int N, int C, int h_l, int w_l, int h, int w, int r,
                            float eps, dgf_dtype dt, const dgf_guide* g, void* workspace, size_t ws_bytes,
                            dgf_stream_t stream, const dgf_options* opt) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    const bool mean_ab = opt == nullptr || opt->mean_ab != 0;
    const int n_in = grey_channels(opt, C);
    float2* coef = nullptr;
    if (dgf_status st = opt_coef(opt, coef); st != DGF_OK) return st;
    if (n_in != 0)
        return backward_grey(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps, dt, g,
                             workspace, ws_bytes, stream, mean_ab, n_in, coef);
    return backward_impl(dO_h, p_l, I_l, I_h, dp_l, dI_l, dI_h, dW, N, C, h_l, w_l, h, w, r, eps, dt, g, workspace,
                         ws_bytes, stream, mean_ab, opt != nullptr && opt->guide_low != 0, false, coef);
}

size_t dgf_workspace_size_opt(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt, const dgf_guide* g,
                              const dgf_options* opt) {
    if (check_sizes(N, C, h_l, w_l, h, w, r, 1.f, dt) != DGF_OK) return 0;
    const int n_in = grey_channels(opt, C);
    if (n_in == 0) return layout(N, C, h_l, w_l, g != nullptr, (size_t)N * C * h * w).total;
    if (check_grey(n_in, N, g) != DGF_OK) return 0;
    return grey_layout(N, C, h_l, w_l, h, w, dt).total;
}

size_t dgf_coef_bytes(int N, int C, int h_l, int w_l, int h, int w, const dgf_guide* g) {
    if (N < 0 || C < 1 || h_l < 1 || w_l < 1 || h < h_l || w < w_l || (long long)N * C > 65535) return 0;
    const size_t lo = (size_t)N * C * h_l * w_l;
    if (g == nullptr) return lo * sizeof(float2);
    return align256(lo * sizeof(float2)) + align256(lo * sizeof(float)) + (size_t)N * C * h * w * sizeof(float);
}

int dgf_backward_reuses_coef(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt, const dgf_guide* g,
                             const dgf_options* opt) {
    if (check_sizes(N, C, h_l, w_l, h, w, r, 1.f, dt) != DGF_OK) return 0;
    if (g != nullptr) return 1;  // its K1 pass computes Abar for K6 alone
    const bool mean_ab = opt == nullptr || opt->mean_ab != 0;
    const int n_in = grey_channels(opt, C);
    if (n_in != 0 && grey_fold(dt, C, h_l, w_l, h, w, {}) != 0) return 1;
    // the plain backward (and the grey guide's streaming form): its K1 pass
    // also writes the window statistics when both low-res stages are strips
    const Plan p = make_plan(dt, h_l, w_l, h, w, r, n_in != 0 && dt != DGF_F32, {}, mean_ab);
    return (p.k1.fast == 2 && p.k4.fast == 2) ? 0 : 1;
}

extern "C" size_t dgf_workspace_size_batched(const dgf_image* imgs, int n, dgf_dtype dt) {
    static thread_local BatchPrep prep;
    if (prepare_batch(imgs, n, dt, nullptr, prep) != DGF_OK) return 0;
    return prep.ws;
}

extern "C" dgf_status dgf_forward_batched(const dgf_image* imgs, int n, dgf_dtype dt, void* workspace,
                                          size_t ws_bytes, dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    static thread_local BatchPrep prep;
    if ((int)dt < 0 || (int)dt > 2) return fail(DGF_ERR_INVALID, "dtype %d", (int)dt);
    dgf_status st = prepare_batch(imgs, n, dt, nullptr, prep);
    if (st != DGF_OK) return st;
    if (n == 0) return DGF_OK;
    if ((st = check_ws(workspace, ws_bytes, prep.ws)) != DGF_OK) return st;
    st = prepare_batch(imgs, n, dt, static_cast<char*>(workspace), prep);
    if (st != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Node classes: K1 by (radius, kernel form), one tile shape each,
    // K2 by (vector width, factor).  Every node is a persistent kernel
    // specialised for its class, so it keeps the registers and occupancy of
    // the single-call kernel; its images keep their workspace slots.
    std::vector<int> c1, c2;
    // K2 strips of 16-byte vectors are staged by TMA as in the single call:
    // tensor maps of I_h in the workspace's map region, copied there on the
    // stream ahead of the graph
    static thread_local std::vector<K2Map> k2maps;
    k2maps.assign(n, K2Map{});
    std::vector<char> tma2(n, 0);
    K2Map* maps_dev = reinterpret_cast<K2Map*>(static_cast<char*>(workspace) + prep.maps);
    // (a capture cannot hold the maps' copy from pageable host memory: the
    // plain-load strips then serve; the same bits)
    const bool capturing = stream_capturing(s);
    bool any_map = false;
    for (int i = 0; i < n && !capturing; ++i) {
        const BatchImage& im = prep.bp.img[i];
        void* f = nullptr;
        size_t sm = 0;
        int th = 0;
        tma2[i] = im.F > 0 && k2_strip_ok(im.vec, im.F) &&
                  make_k2_map(k2maps[i], im.I_h, dt, im.C, im.h, im.w, im.vec, im.F) &&
                  k2_batched_tma_kernel(dt, im.vec, im.F, &f, &sm, &th) == cudaSuccess;
        any_map = any_map || tma2[i];
    }
    // K1 class: radius, form and (sliding form) columns per lane
    auto k1class = [](const BatchImage& im) { return (im.r * 4 + im.k1_fast) * 16 + (im.k1_fast == 3 ? im.k1_ty : 0); };
    // K2 class: staging, vector width, factor
    auto k2class = [&](int i) { return (tma2[i] ? 10000 : 0) + prep.bp.img[i].vec * 100 + prep.bp.img[i].F; };
    for (int i = 0; i < n; ++i) {
        const BatchImage& im = prep.bp.img[i];
        if (std::find(c1.begin(), c1.end(), k1class(im)) == c1.end()) c1.push_back(k1class(im));
        if (std::find(c2.begin(), c2.end(), k2class(i)) == c2.end()) c2.push_back(k2class(i));
    }
    std::sort(c1.begin(), c1.end());
    std::sort(c2.begin(), c2.end());
    static thread_local std::vector<BatchParams> bp1, bp2;
    bp1.resize(c1.size());
    bp2.resize(c2.size());
    std::vector<size_t> sm1(c1.size(), 0), sm2(c2.size(), 0);
    std::vector<int> fast1(c1.size(), 0);
    for (size_t q = 0; q < c1.size(); ++q) {
        BatchParams& b = bp1[q];
        memset(&b, 0, sizeof b);
        for (int i = 0; i < n; ++i) {
            const BatchImage& im = prep.bp.img[i];
            if (k1class(im) != c1[q]) continue;
            const int j = b.n++;
            b.img[j] = im;
            b.k1_start[j + 1] = b.k1_start[j] + im.k1_nx * im.k1_ny * im.C;
            const LowCfg c{im.k1_fast, im.k1_fast ? im.k1_tx : im.k1_ty, im.k1_fast ? im.k1_ty : im.k1_tx};
            sm1[q] = std::max(sm1[q], k1_cfg_smem(c, im.r, 0));
            fast1[q] = im.k1_fast;
        }
        b.k1_total = b.k1_start[b.n];
    }
    std::vector<void*> f2(c2.size(), nullptr);
    std::vector<int> th2(c2.size(), kThreads), occ2(c2.size(), 0);
    cudaError_t e;
    for (size_t q = 0; q < c2.size(); ++q) {
        BatchParams& b = bp2[q];
        memset(&b, 0, sizeof b);
        const bool tma = c2[q] >= 10000;
        const int vec = c2[q] % 10000 / 100, F = c2[q] % 100;
        std::vector<int> members;
        for (int i = 0; i < n; ++i)
            if (k2class(i) == c2[q]) members.push_back(i);
        if (tma) {
            // one segment length for the class (the strip walk's bits do not
            // depend on it): whole waves of CTA slots, few halo rows
            if ((e = k2_batched_tma_kernel(dt, vec, F, &f2[q], &sm2[q], &th2[q])) != cudaSuccess)
                return cuda_fail(e, "k2 batched tma");
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2[q], f2[q], th2[q], sm2[q]);
            const double slots = (double)sms * std::max(occ2[q], 1);
            const int wpc = th2[q] / 32, OUT = 32 * (vec / F);
            auto items = [&](int ls) {
                long long t = 0;
                for (int i : members) {
                    const BatchImage& im = prep.bp.img[i];
                    const int nstrip = (im.w_l + OUT - 1) / OUT, nseg = (im.h_l + ls - 1) / ls;
                    t += (long long)((nstrip * nseg + wpc - 1) / wpc) * im.C;
                }
                return t;
            };
            int ls = 32;
            double best = 1e30;
            for (int c = 8; c <= 64; ++c) {
                const double waves = (double)items(c) / slots, eff = waves / std::ceil(waves);
                const double cost = (c + 0.25) / c / eff;
                if (cost < best - 1e-9) {
                    best = cost;
                    ls = c;
                }
            }
            for (int i : members) {
                const int j = b.n++;
                b.img[j] = prep.bp.img[i];
                BatchImage& im = b.img[j];
                const int nstrip = (im.w_l + OUT - 1) / OUT, nseg = (im.h_l + ls - 1) / ls;
                im.k2_th = ls;
                im.k2_nx = (nstrip * nseg + wpc - 1) / wpc;
                im.k2_ny = 1;
                im.k2_map = maps_dev + i;
                b.k2_start[j + 1] = b.k2_start[j] + im.k2_nx * im.C;
            }
        } else {
            for (int i : members) {
                const BatchImage& im = prep.bp.img[i];
                const int j = b.n++;
                b.img[j] = im;
                b.k2_start[j + 1] = b.k2_start[j] + im.k2_nx * im.k2_ny * im.C;
                sm2[q] = std::max(sm2[q], (im.F > 0 && k2_strip_ok(im.vec, im.F))
                                              ? k2_strip_batched_smem((int)esize(dt), im.vec, im.F)
                                              : k2_smem_bytes(im.vec, im.F, im.h_l, im.h, im.w_l, im.w, im.k2_th));
            }
            if ((e = k2_batched_kernel(dt, vec, F, sm2[q], &f2[q])) != cudaSuccess)
                return cuda_fail(e, "k2 batched attr");
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2[q], f2[q], kThreads, sm2[q]);
        }
        b.k2_total = b.k2_start[b.n];
    }
    uint32_t* stw = status_ptr();
    std::vector<cudaKernelNodeParams> p1(c1.size()), p2(c2.size());
    std::vector<std::array<void*, 2>> a1(c1.size()), a2(c2.size());
    for (size_t q = 0; q < c1.size(); ++q) {
        void* f = nullptr;
        int threads = kThreads;
        if ((e = k1_batched_kernel(dt, c1[q] / 64, fast1[q], sm1[q], &f, c1[q] % 16, &threads)) != cudaSuccess)
            return cuda_fail(e, "k1 batched attr");
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, threads, sm1[q]);
        a1[q] = {&bp1[q], &stw};
        p1[q] = cudaKernelNodeParams{};
        p1[q].func = f;
        // the sliding form takes one work item per CTA (the whole list), the
        // others loop over it
        p1[q].gridDim = dim3(std::max(1, fast1[q] == 3 ? bp1[q].k1_total
                                                       : std::min(bp1[q].k1_total, sms * std::max(occ, 1))));
        p1[q].blockDim = dim3(threads);
        p1[q].sharedMemBytes = (unsigned)sm1[q];
        p1[q].kernelParams = a1[q].data();
    }
    for (size_t q = 0; q < c2.size(); ++q) {
        a2[q] = {&bp2[q], &stw};
        p2[q] = cudaKernelNodeParams{};
        p2[q].func = f2[q];
        p2[q].gridDim = dim3(std::max(1, std::min(bp2[q].k2_total, sms * std::max(occ2[q], 1))));
        p2[q].blockDim = dim3(th2[q]);
        p2[q].sharedMemBytes = (unsigned)sm2[q];
        p2[q].kernelParams = a2[q].data();
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchGraph& bg = g_batch[std::make_tuple(dev, (int)dt, c1, c2)];
    if (bg.exec == nullptr) {
        if ((e = cudaGraphCreate(&bg.graph, 0)) != cudaSuccess) return cuda_fail(e, "graph create");
        bg.n1.resize(c1.size());
        bg.n2.resize(c2.size());
        for (size_t q = 0; q < c1.size(); ++q)
            if ((e = cudaGraphAddKernelNode(&bg.n1[q], bg.graph, nullptr, 0, &p1[q])) != cudaSuccess)
                return cuda_fail(e, "graph node k1");
        // the stage boundary: every K2 node waits for every K1 node
        for (size_t q = 0; q < c2.size(); ++q)
            if ((e = cudaGraphAddKernelNode(&bg.n2[q], bg.graph, bg.n1.data(), bg.n1.size(), &p2[q])) != cudaSuccess)
                return cuda_fail(e, "graph node k2");
        if ((e = cudaGraphInstantiate(&bg.exec, bg.graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
    } else {
        for (size_t q = 0; q < c1.size(); ++q)
            if ((e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.n1[q], &p1[q])) != cudaSuccess)
                return cuda_fail(e, "graph update k1");
        for (size_t q = 0; q < c2.size(); ++q)
            if ((e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.n2[q], &p2[q])) != cudaSuccess)
                return cuda_fail(e, "graph update k2");
    }
    if (any_map &&
        (e = cudaMemcpyAsync(maps_dev, k2maps.data(), (size_t)n * sizeof(K2Map), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return cuda_fail(e, "k2 maps");
    Launcher L(s);
    e = L.run("batched_graph(k1,k2)", [&] {
        g_launches.fetch_add((long long)(c1.size() + c2.size()) - 1);  // every node of the replay
        return cudaGraphLaunch(bg.exec, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return DGF_OK;
}

// ------------------------------------------------------- batched backward
// Images are independent: each image's backward (K1 -> K3 -> K4, exactly the
// kernels and shapes of its single call) runs as one chain on one of a few
// library-owned streams forked from and joined back to the caller's stream,
// so small images run concurrently and large ones fill the GPU by
// themselves.  Results are those of the single calls.
namespace dgf {
constexpr int kBwdStreams = 8;
struct BwdPool {
    int dev = -1;
    cudaStream_t st[kBwdStreams] = {};
    cudaEvent_t fork = nullptr, join[kBwdStreams] = {};
};
std::mutex g_bwd_mu;
std::map<int, BwdPool> g_bwd_pools;

static cudaError_t bwd_pool(int dev, BwdPool*& out) {
    BwdPool& p = g_bwd_pools[dev];
    if (p.dev < 0) {
        cudaError_t e;
        for (int i = 0; i < kBwdStreams; ++i) {
            if ((e = cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        p.dev = dev;
    }
    out = &p;
    return cudaSuccess;
}

// Streams of dgf_host_step: host -> device copies, kernels, device -> host
// copies, with one event per group and stage.
constexpr int kHostMaxGroups = 16;
struct HostPool {
    int dev = -1;
    cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t copied[kHostMaxGroups] = {}, done[kHostMaxGroups] = {};
};
std::mutex g_host_mu;
std::map<int, HostPool> g_host_pools;

static cudaError_t host_pool(int dev, HostPool*& out) {
    HostPool& p = g_host_pools[dev];
    if (p.dev < 0) {
        cudaError_t e;
        cudaStream_t* sts[] = {&p.in, &p.comp, &p.out};
        for (cudaStream_t* st : sts)
            if ((e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&p.join, cudaEventDisableTiming)) != cudaSuccess) return e;
        for (int g = 0; g < kHostMaxGroups; ++g) {
            if ((e = cudaEventCreateWithFlags(&p.copied[g], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.done[g], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        p.dev = dev;
    }
    out = &p;
    return cudaSuccess;
}

static void host_pools_free() {
    std::lock_guard<std::mutex> lk(g_host_mu);
    for (auto& kv : g_host_pools) {
        HostPool& p = kv.second;
        cudaStream_t sts[] = {p.in, p.comp, p.out};
        for (cudaStream_t st : sts)
            if (st) cudaStreamDestroy(st);
        if (p.fork) cudaEventDestroy(p.fork);
        if (p.join) cudaEventDestroy(p.join);
        for (int g = 0; g < kHostMaxGroups; ++g) {
            if (p.copied[g]) cudaEventDestroy(p.copied[g]);
            if (p.done[g]) cudaEventDestroy(p.done[g]);
        }
    }
    g_host_pools.clear();
}

static dgf_status check_grad_images(const dgf_image_grad* imgs, int n, dgf_dtype dt, size_t* ws_total) {
    if ((int)dt < 0 || (int)dt > 2) return fail(DGF_ERR_INVALID, "dtype %d", (int)dt);
    if (n < 0 || n > DGF_MAX_BATCH) return fail(DGF_ERR_INVALID, "n = %d outside [0, %d]", n, DGF_MAX_BATCH);
    if (n > 0 && imgs == nullptr) return fail(DGF_ERR_INVALID, "NULL image array");
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const dgf_image_grad& im = imgs[i];
        dgf_status st = check_sizes(1, im.C, im.h_l, im.w_l, im.h, im.w, im.r, im.eps, dt);
        if (st != DGF_OK) {
            const std::string why = t_err;
            return fail(st, "image %d: %s", i, why.c_str());
        }
        if (im.dO_h == nullptr || im.p_l == nullptr || im.I_l == nullptr || im.I_h == nullptr)
            return fail(DGF_ERR_INVALID, "image %d: NULL input pointer", i);
        if (reinterpret_cast<uintptr_t>(im.coef) % alignof(float2) != 0)
            return fail(DGF_ERR_INVALID, "image %d: coef must be 8-byte aligned", i);
        off += align256(layout(1, im.C, im.h_l, im.w_l, false).total);
    }
    // 16-bit storage: the K3 tensor maps of the one-graph form
    if (dt != DGF_F32 && n > 0) off += align256((size_t)n * sizeof(K3Maps));
    *ws_total = off;
    return DGF_OK;
}
}  // namespace dgf

// ------------------------------------------------ batched backward as a graph
// For 16-bit storage, when every image's backward runs the sliding K1/K4 and
// the strip K3: one CUDA graph of persistent kernels, one per node class,
// K1 classes (radius, columns per lane) -> K3 classes (vector width,
// factor) -> K4 classes (radius, columns per lane); every edge is a stage
// boundary and each image keeps its workspace slot.  Each image runs its
// single call's arithmetic (same segment lengths for the sliding kernels; the
// K3 walk gives the same bits at any segment length), so the results equal
// the single calls bit for bit.
namespace dgf {

struct BwdGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> n1, n3, n4;
};
static std::mutex g_bwdg_mu;
static std::map<std::tuple<int, int, std::vector<int>, std::vector<int>, std::vector<int>>, BwdGraph> g_bwdg;

static dgf_status backward_batched_graph(const dgf_image_grad* imgs, int n, dgf_dtype dt, char* ws, cudaStream_t s,
                                         bool& done) {
    done = false;
    if (dt == DGF_F32 || n <= 0 || stream_capturing(s)) return DGF_OK;
    struct Item {
        Plan p;
        int S1, V1, S4, V4;
        bool k4, tma;
        int k3c;  // K3 class: vector width, factor, staging
    };
    std::vector<Item> it(n);
    // K3 tensor maps (the single call's TMA staging) go to the workspace's map
    // region, copied there on the stream ahead of the graph
    static thread_local std::vector<K3Maps> maps;
    maps.assign(n, K3Maps{});
    std::vector<size_t> off(n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        const dgf_image_grad& im = imgs[i];
        off[i] = o;
        o += align256(layout(1, im.C, im.h_l, im.w_l, false).total);
        Item& t = it[i];
        t.p = make_plan(dt, im.h_l, im.w_l, im.h, im.w, im.r, false, {im.dO_h, im.I_h, im.dI_h});
        const Plan& p = t.p;
        if (p.k1.fast != 3 || p.k4.fast != 3 || !p.k3_fast || p.F <= 0) return DGF_OK;
        void* f = nullptr;
        size_t sm3 = 0;
        int th3 = 0;
        t.tma = make_k3_maps(maps[i], im.dO_h, im.I_h, dt, im.C, im.h, im.w, p.vec, p.F);
        t.k3c = (t.tma ? 10000 : 0) + p.vec * 100 + p.F;
        if (k3_batched_kernel(dt, p.vec, p.F, t.tma, &f, &sm3, &th3) != cudaSuccess) return DGF_OK;
        t.S1 = p.k1.a > 0 ? p.k1.a : slide_auto_seg(im.h_l, im.r);
        t.V1 = p.k1.b > 0 ? p.k1.b : slide_k1_v(im.r);
        t.S4 = p.k4.a > 0 ? p.k4.a : slide_auto_seg(im.h_l, im.r);
        t.V4 = p.k4.b > 0 ? p.k4.b : slide_k4_v(im.r);
        t.k4 = im.dp_l != nullptr || im.dI_l != nullptr;
        size_t sm4 = 0;
        int th4 = 0;
        if (t.k4 && k4_batched_kernel(dt, im.r, t.V4, &f, &sm4, &th4) != cudaSuccess) return DGF_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = sm_count();
    // node classes
    std::vector<int> c1, c3, c4;
    auto add = [](std::vector<int>& v, int k) {
        if (std::find(v.begin(), v.end(), k) == v.end()) v.push_back(k);
    };
    // as in the single call, K1 runs only for the images that want d I_h
    // (d Abar and d bbar do not depend on the coefficients) and have not
    // brought the forward's
    for (int i = 0; i < n; ++i) {
        const dgf_image_grad& im = imgs[i];
        if (im.dp_l == nullptr && im.dI_l == nullptr && im.dI_h == nullptr) continue;
        if (im.dI_h != nullptr && im.coef == nullptr) add(c1, im.r * 16 + it[i].V1);
        add(c3, it[i].k3c);
        if (it[i].k4) add(c4, im.r * 16 + it[i].V4);
    }
    if (c3.empty()) {
        done = true;
        return DGF_OK;
    }
    std::sort(c1.begin(), c1.end());
    std::sort(c3.begin(), c3.end());
    std::sort(c4.begin(), c4.end());
    static thread_local std::vector<BatchParams> bp1;
    static thread_local std::vector<BwdParams> bp3, bp4;
    bp1.resize(c1.size());
    bp3.resize(c3.size());
    bp4.resize(c4.size());
    std::vector<cudaKernelNodeParams> p1(c1.size()), p3(c3.size()), p4(c4.size());
    std::vector<std::array<void*, 2>> a1(c1.size()), a3(c3.size());
    std::vector<std::array<void*, 1>> a4(c4.size());
    uint32_t* stw = status_ptr();
    cudaError_t e;
    auto bwd_image = [&](int i, BwdImage& b) {
        const dgf_image_grad& im = imgs[i];
        const Layout lay = layout(1, im.C, im.h_l, im.w_l, false);
        memset(&b, 0, sizeof b);
        b.dO = im.dO_h;
        b.p_l = im.p_l;
        b.I_l = im.I_l;
        b.I_h = im.I_h;
        b.dp = im.dp_l;
        b.dIl = im.dI_l;
        b.dIh = im.dI_h;
        b.coef = im.coef != nullptr ? static_cast<const float2*>(im.coef)
                                    : reinterpret_cast<const float2*>(ws + off[i] + lay.coef);
        b.dcoef = reinterpret_cast<float2*>(ws + off[i] + lay.dcoef);
        b.C = im.C;
        b.h_l = im.h_l;
        b.w_l = im.w_l;
        b.h = im.h;
        b.w = im.w;
        b.eps = im.eps;
    };
    for (size_t q = 0; q < c1.size(); ++q) {  // K1: the forward's persistent sliding K1
        BatchParams& b = bp1[q];
        memset(&b, 0, sizeof b);
        const int r = c1[q] / 16, V = c1[q] % 16;
        size_t smem = 0;
        for (int i = 0; i < n; ++i) {
            const dgf_image_grad& im = imgs[i];
            if (im.dI_h == nullptr || im.coef != nullptr || im.r * 16 + it[i].V1 != c1[q]) continue;
            const int j = b.n++;
            BatchImage& bi = b.img[j];
            bi.p_l = im.p_l;
            bi.I_l = im.I_l;
            bi.I_h = im.I_h;
            bi.coef = reinterpret_cast<float2*>(ws + off[i] + layout(1, im.C, im.h_l, im.w_l, false).coef);
            bi.C = im.C;
            bi.h_l = im.h_l;
            bi.w_l = im.w_l;
            bi.h = im.h;
            bi.w = im.w;
            bi.r = im.r;
            bi.eps = im.eps;
            bi.k1_fast = 3;
            bi.k1_ty = V;
            bi.k1_tx = it[i].S1;
            const LowCfg c{3, it[i].S1, V};
            low_grid(c, im.r, im.h_l, im.w_l, bi.k1_nx, bi.k1_ny);
            b.k1_start[j + 1] = b.k1_start[j] + bi.k1_nx * bi.k1_ny * im.C;
            smem = std::max(smem, k1_cfg_smem(c, im.r, 0));
        }
        b.k1_total = b.k1_start[b.n];
        void* f = nullptr;
        int threads = kThreads;
        if ((e = k1_batched_kernel(dt, r, 3, smem, &f, V, &threads)) != cudaSuccess)
            return cuda_fail(e, "k1 batched attr");
        a1[q] = {&bp1[q], &stw};
        p1[q] = cudaKernelNodeParams{};
        p1[q].func = f;
        p1[q].gridDim = dim3(std::max(1, b.k1_total));  // one work item per CTA
        p1[q].blockDim = dim3(threads);
        p1[q].sharedMemBytes = (unsigned)smem;
        p1[q].kernelParams = a1[q].data();
    }
    K3Maps* maps_dev = reinterpret_cast<K3Maps*>(ws + o);
    for (size_t q = 0; q < c3.size(); ++q) {  // K3 strips
        BwdParams& b = bp3[q];
        memset(&b, 0, sizeof b);
        const bool tma = c3[q] >= 10000;
        const int vec = c3[q] % 10000 / 100, F = c3[q] % 100, OUT = 30 * (vec / F);
        void* f = nullptr;
        size_t smem = 0;
        int threads = 0;
        if ((e = k3_batched_kernel(dt, vec, F, tma, &f, &smem, &threads)) != cudaSuccess)
            return cuda_fail(e, "k3 batched");
        const int wpc = threads / 32;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, threads, smem);
        const double slots = (double)sms * std::max(occ, 1);
        // one segment length for the class (the walk's bits do not depend on
        // it), chosen like the single call's: whole waves of CTA slots, few
        // halo blocks
        std::vector<int> members;
        for (int i = 0; i < n; ++i) {
            const dgf_image_grad& im = imgs[i];
            if (im.dp_l == nullptr && im.dI_l == nullptr && im.dI_h == nullptr) continue;
            if (it[i].k3c == c3[q]) members.push_back(i);
        }
        auto items = [&](int ls) {
            long long t = 0;
            for (int i : members) {
                const dgf_image_grad& im = imgs[i];
                const int nstrip = (im.w_l + OUT - 1) / OUT, nseg = (im.h_l + ls - 1) / ls;
                t += (long long)((nstrip * nseg + wpc - 1) / wpc) * im.C;
            }
            return t;
        };
        int ls = 32;
        double best = 1e30;
        for (int c = 8; c <= 64; ++c) {
            const double waves = (double)items(c) / slots, eff = waves / std::ceil(waves);
            const double cost = (c + 1.0) / c / eff;
            if (cost < best - 1e-9) {
                best = cost;
                ls = c;
            }
        }
        for (int i : members) {
            const dgf_image_grad& im = imgs[i];
            const int j = b.n++;
            bwd_image(i, b.img[j]);
            b.img[j].k3_ls = ls;
            const int nstrip = (im.w_l + OUT - 1) / OUT, nseg = (im.h_l + ls - 1) / ls;
            b.img[j].k3_nx = (nstrip * nseg + wpc - 1) / wpc;
            b.img[j].k3_maps = tma ? maps_dev + i : nullptr;
            b.start[j + 1] = b.start[j] + b.img[j].k3_nx * im.C;
        }
        b.total = b.start[b.n];
        a3[q] = {&bp3[q], &stw};
        p3[q] = cudaKernelNodeParams{};
        p3[q].func = f;
        p3[q].gridDim = dim3(std::max(1, b.total));  // one work item per CTA
        p3[q].blockDim = dim3(threads);
        p3[q].sharedMemBytes = (unsigned)smem;
        p3[q].kernelParams = a3[q].data();
    }
    for (size_t q = 0; q < c4.size(); ++q) {  // sliding K4
        BwdParams& b = bp4[q];
        memset(&b, 0, sizeof b);
        const int r = c4[q] / 16, V = c4[q] % 16;
        void* f = nullptr;
        size_t smem = 0;
        int threads = 0;
        if ((e = k4_batched_kernel(dt, r, V, &f, &smem, &threads)) != cudaSuccess) return cuda_fail(e, "k4 batched");
        const int wpc = threads / 32, outc = slide_out_cols(r, V);
        for (int i = 0; i < n; ++i) {
            const dgf_image_grad& im = imgs[i];
            if (!it[i].k4 || im.r * 16 + it[i].V4 != c4[q]) continue;
            const int j = b.n++;
            bwd_image(i, b.img[j]);
            BwdImage& bi = b.img[j];
            bi.k4_S = it[i].S4;
            const int nstrip = (im.w_l + outc - 1) / outc, nseg = (im.h_l + bi.k4_S - 1) / bi.k4_S;
            bi.k4_nx = (nstrip * nseg + wpc - 1) / wpc;
            const size_t a = (size_t)V * 2;  // bytes of V 16-bit elements
            auto al = [a](const void* ptr) { return ptr == nullptr || reinterpret_cast<uintptr_t>(ptr) % a == 0; };
            bi.k4_aligned = im.w_l % V == 0 && al(im.I_l) && al(im.p_l) && al(im.dp_l) && al(im.dI_l);
            bi.k4_pairs = im.w_l % 2 == 0 && reinterpret_cast<uintptr_t>(bi.dcoef) % 16 == 0;
            b.start[j + 1] = b.start[j] + bi.k4_nx * im.C;
        }
        b.total = b.start[b.n];
        a4[q] = {&bp4[q]};
        p4[q] = cudaKernelNodeParams{};
        p4[q].func = f;
        p4[q].gridDim = dim3(std::max(1, b.total));  // one work item per CTA
        p4[q].blockDim = dim3(threads);
        p4[q].sharedMemBytes = (unsigned)smem;
        p4[q].kernelParams = a4[q].data();
    }
    std::lock_guard<std::mutex> lk(g_bwdg_mu);
    BwdGraph& bg = g_bwdg[std::make_tuple(dev, (int)dt, c1, c3, c4)];
    if (bg.exec == nullptr) {
        if ((e = cudaGraphCreate(&bg.graph, 0)) != cudaSuccess) return cuda_fail(e, "graph create");
        bg.n1.resize(c1.size());
        bg.n3.resize(c3.size());
        bg.n4.resize(c4.size());
        for (size_t q = 0; q < c1.size(); ++q)
            if ((e = cudaGraphAddKernelNode(&bg.n1[q], bg.graph, nullptr, 0, &p1[q])) != cudaSuccess)
                return cuda_fail(e, "graph node k1");
        for (size_t q = 0; q < c3.size(); ++q)
            if ((e = cudaGraphAddKernelNode(&bg.n3[q], bg.graph, bg.n1.data(), bg.n1.size(), &p3[q])) != cudaSuccess)
                return cuda_fail(e, "graph node k3");
        for (size_t q = 0; q < c4.size(); ++q)
            if ((e = cudaGraphAddKernelNode(&bg.n4[q], bg.graph, bg.n3.data(), bg.n3.size(), &p4[q])) != cudaSuccess)
                return cuda_fail(e, "graph node k4");
        if ((e = cudaGraphInstantiate(&bg.exec, bg.graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
    } else {
        for (size_t q = 0; q < c1.size(); ++q)
            if ((e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.n1[q], &p1[q])) != cudaSuccess)
                return cuda_fail(e, "graph update k1");
        for (size_t q = 0; q < c3.size(); ++q)
            if ((e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.n3[q], &p3[q])) != cudaSuccess)
                return cuda_fail(e, "graph update k3");
        for (size_t q = 0; q < c4.size(); ++q)
            if ((e = cudaGraphExecKernelNodeSetParams(bg.exec, bg.n4[q], &p4[q])) != cudaSuccess)
                return cuda_fail(e, "graph update k4");
    }
    bool any_map = false;
    for (int i = 0; i < n; ++i) any_map = any_map || it[i].tma;
    if (any_map &&
        (e = cudaMemcpyAsync(maps_dev, maps.data(), (size_t)n * sizeof(K3Maps), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return cuda_fail(e, "k3 maps");
    Launcher L(s);
    e = L.run("batched_bwd_graph(k1,k3,k4)", [&] {
        g_launches.fetch_add((long long)(c1.size() + c3.size() + c4.size()) - 1);  // every node of the replay
        return cudaGraphLaunch(bg.exec, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    done = true;
    return DGF_OK;
}

}  // namespace dgf

extern "C" size_t dgf_workspace_size_batched_backward(const dgf_image_grad* imgs, int n, dgf_dtype dt) {
    size_t total = 0;
    if (check_grad_images(imgs, n, dt, &total) != DGF_OK) return 0;
    return total;
}

// The batched backward; mean_ab = false (the layer as printed, Sec. 3.2 and
// Algorithm 1 without the box mean of A, b) runs every image's chain.
static dgf_status backward_batched_impl(const dgf_image_grad* imgs, int n, dgf_dtype dt, void* workspace,
                                        size_t ws_bytes, dgf_stream_t stream, bool mean_ab) {
    size_t total = 0;
    dgf_status st = check_grad_images(imgs, n, dt, &total);
    if (st != DGF_OK) return st;
    if (n == 0) return DGF_OK;
    if ((st = check_ws(workspace, ws_bytes, total)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bool done = false;
    if (g_batched_graph_bwd && mean_ab) {
        st = backward_batched_graph(imgs, n, dt, static_cast<char*>(workspace), s, done);
        if (st != DGF_OK || done) return st;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bwd_mu);
    BwdPool* pool = nullptr;
    cudaError_t e = bwd_pool(dev, pool);
    if (e != cudaSuccess) return cuda_fail(e, "backward stream pool");
    const int ns = std::min(n, kBwdStreams);
    if ((e = cudaEventRecord(pool->fork, s)) != cudaSuccess) return cuda_fail(e, "fork");
    for (int k = 0; k < ns; ++k)
        if ((e = cudaStreamWaitEvent(pool->st[k], pool->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    char* ws = static_cast<char*>(workspace);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const dgf_image_grad& im = imgs[i];
        cudaStream_t si = pool->st[i % ns];
        const Layout lay = layout(1, im.C, im.h_l, im.w_l, false);
        Plan p = make_plan(dt, im.h_l, im.w_l, im.h, im.w, im.r, false, {im.dO_h, im.I_h, im.dI_h}, mean_ab);
        if (im.dp_l != nullptr || im.dI_l != nullptr || im.dI_h != nullptr) {
            Launcher L(si);
            st = backward_plain(L, dt, im.dO_h, im.p_l, im.I_l, im.I_h, im.dp_l, im.dI_l, im.dI_h, im.C, im.h_l,
                                im.w_l, im.h, im.w, im.r, im.eps, p, ws + off, lay, si, false, false,
                                static_cast<const float2*>(im.coef));
            if (st != DGF_OK) return st;
        }
        off += align256(lay.total);
    }
    for (int k = 0; k < ns; ++k) {
        if ((e = cudaEventRecord(pool->join[k], pool->st[k])) != cudaSuccess) return cuda_fail(e, "join");
        if ((e = cudaStreamWaitEvent(s, pool->join[k], 0)) != cudaSuccess) return cuda_fail(e, "join wait");
    }
    return DGF_OK;
}

extern "C" dgf_status dgf_backward_batched(const dgf_image_grad* imgs, int n, dgf_dtype dt, void* workspace,
                                           size_t ws_bytes, dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    return backward_batched_impl(imgs, n, dt, workspace, ws_bytes, stream, true);
}

// Options of the batched and host-memory calls: the box mean of A, b only.
static dgf_status batch_options(const dgf_options* opt, bool& mean_ab) {
    mean_ab = opt == nullptr || opt->mean_ab != 0;
    if (opt != nullptr && (opt->guide_channels != 0 || opt->guide_low != 0))
        return fail(DGF_ERR_UNSUPPORTED, "the batched and host-memory calls take the mean_ab option only");
    return DGF_OK;
}

extern "C" dgf_status dgf_backward_batched_opt(const dgf_image_grad* imgs, int n, dgf_dtype dt, void* workspace,
                                               size_t ws_bytes, dgf_stream_t stream, const dgf_options* opt) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    bool mean_ab = true;
    if (dgf_status st = batch_options(opt, mean_ab); st != DGF_OK) return st;
    return backward_batched_impl(imgs, n, dt, workspace, ws_bytes, stream, mean_ab);
}

// The layer as printed over a batch: each image's K1 (A, b without their box
// mean) and K2 on one of the library streams, in the image's coefficient
// slot of the batched workspace.
static dgf_status forward_batched_chains(const dgf_image* imgs, int n, dgf_dtype dt, void* workspace,
                                         size_t ws_bytes, dgf_stream_t stream) {
    static thread_local BatchPrep prep;
    if ((int)dt < 0 || (int)dt > 2) return fail(DGF_ERR_INVALID, "dtype %d", (int)dt);
    dgf_status st = prepare_batch(imgs, n, dt, nullptr, prep);
    if (st != DGF_OK) return st;
    if (n == 0) return DGF_OK;
    if ((st = check_ws(workspace, ws_bytes, prep.ws)) != DGF_OK) return st;
    if ((st = prepare_batch(imgs, n, dt, static_cast<char*>(workspace), prep)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bwd_mu);
    BwdPool* pool = nullptr;
    cudaError_t e = bwd_pool(dev, pool);
    if (e != cudaSuccess) return cuda_fail(e, "batch stream pool");
    const int ns = std::min(n, kBwdStreams);
    if ((e = cudaEventRecord(pool->fork, s)) != cudaSuccess) return cuda_fail(e, "fork");
    for (int k = 0; k < ns; ++k)
        if ((e = cudaStreamWaitEvent(pool->st[k], pool->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    for (int i = 0; i < n; ++i) {
        const dgf_image& im = imgs[i];
        cudaStream_t si = pool->st[i % ns];
        float2* coef = prep.bp.img[i].coef;
        Plan p = make_plan(dt, im.h_l, im.w_l, im.h, im.w, im.r, false, {im.I_h, im.O_h}, false);
        Launcher L(si);
        e = run_k1(L, dt, false, im.I_l, im.p_l, coef, im.C, im.h_l, im.w_l, im.r, im.eps, p, si);
        if (e != cudaSuccess) return cuda_fail(e, "k1");
        e = L.run("k2_hires_apply", [&] {
            return launch_k2_plan(dt, coef, im.I_h, im.O_h, im.C, im.h_l, im.w_l, im.h, im.w, p,
                                  p.k2_strip ? p.k2_ls : p.k2_th, si);
        });
        if (e != cudaSuccess) return cuda_fail(e, "k2");
    }
    for (int k = 0; k < ns; ++k) {
        if ((e = cudaEventRecord(pool->join[k], pool->st[k])) != cudaSuccess) return cuda_fail(e, "join");
        if ((e = cudaStreamWaitEvent(s, pool->join[k], 0)) != cudaSuccess) return cuda_fail(e, "join wait");
    }
    return DGF_OK;
}

extern "C" dgf_status dgf_forward_batched_opt(const dgf_image* imgs, int n, dgf_dtype dt, void* workspace,
                                              size_t ws_bytes, dgf_stream_t stream, const dgf_options* opt) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    bool mean_ab = true;
    if (dgf_status st = batch_options(opt, mean_ab); st != DGF_OK) return st;
    if (mean_ab) return dgf_forward_batched(imgs, n, dt, workspace, ws_bytes, stream);
    return forward_batched_chains(imgs, n, dt, workspace, ws_bytes, stream);
}

extern "C" const char* dgf_last_error(void) { return t_err.c_str(); }

extern "C" void dgf_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
}

extern "C" void dgf_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.clear();
}

extern "C" int dgf_profile_read(const char** names, double* total_ms, long long* launches, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int i = 0;
    for (auto& kv : g_prof) {
        if (i < cap) {
            if (names) names[i] = kv.first.c_str();
            if (total_ms) total_ms[i] = kv.second.ms;
            if (launches) launches[i] = kv.second.n;
        }
        ++i;
    }
    return i;
}

extern "C" long long dgf_launch_count(void) { return g_launches.load(); }

extern "C" int dgf_device_status(void) {
    uint32_t* p = status_ptr();
    if (p == nullptr) return -1;
    uint32_t v = 0;
    if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return (int)v;
}

extern "C" dgf_status dgf_clear_device_status(void) {
    uint32_t* p = status_ptr();
    if (p == nullptr) return fail(DGF_ERR_CUDA, "status word unavailable");
    const uint32_t z = 0;
    cudaError_t e = cudaMemcpy(p, &z, sizeof z, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_status_host[dev] != nullptr) *g_status_host[dev] = 0u;
    return DGF_OK;
}

extern "C" dgf_status dgf_set_wait_polls(long long polls) {
    if (polls < 0 || polls > kWaitLimit) return fail(DGF_ERR_INVALID, "polls %lld not in [0, %lld]", polls, kWaitLimit);
    uint32_t* p = status_ptr();
    if (p == nullptr) return fail(DGF_ERR_CUDA, "status word unavailable");
    const uint32_t v = (uint32_t)polls;
    cudaError_t e = cudaMemcpy(p + 1, &v, sizeof v, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "set wait polls");
    return DGF_OK;
}

extern "C" void dgf_set_tma(int on) { g_tma_allowed = on != 0; }

extern "C" void dgf_set_fused(int on) { g_fused_allowed = on != 0; }
extern "C" void dgf_set_lowres_slide(int on) { g_slide_allowed = on != 0; }
extern "C" void dgf_set_grey_fold(int on) { g_grey_fold = on != 0; }
extern "C" void dgf_set_batched_graph_backward(int on) { g_batched_graph_bwd = on != 0; }

extern "C" void dgf_set_pipeline(int on) { g_pipeline = on != 0; }

extern "C" void dgf_autotune(int on) { tune_set_enabled(on != 0); }

extern "C" int dgf_autotune_entries(void) { return tune_count(); }

extern "C" dgf_status dgf_autotune_pin(int kind, dgf_dtype dt, int r, int F, int vec, int guide_f32, int a,
                                       int b) {
    const int bmin = (kind == 1 || kind == 4) ? -8 : 0;  // b < 0: sliding strips with -b columns per lane
    if (kind < 1 || kind > 6 || (int)dt < 0 || (int)dt > 2 || r < 0 || F < 0 || vec < 0 || a < 0 ||
        (a == 0 && kind < 5) || a > 4096 || b < bmin || b > 4096 || (guide_f32 != 0 && guide_f32 != 1))
        return fail(DGF_ERR_INVALID, "autotune_pin: bad key or shape");
    // a pin serves planes of both size classes
    tune_store(TuneKey{kind, (int)dt, r, F, vec, guide_f32, 0}, a, b);
    tune_store(TuneKey{kind, (int)dt, r, F, vec, guide_f32, 1}, a, b);
    return DGF_OK;
}

extern "C" void dgf_autotune_reset(void) { tune_clear(); }

extern "C" void dgf_shutdown(void) {
    {
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        for (auto& kv : g_pipe_pools) {
            PipePool& p = kv.second;
            if (p.lo) cudaStreamDestroy(p.lo);
            if (p.hi) cudaStreamDestroy(p.hi);
            cudaEvent_t evs[] = {p.fork, p.join_lo, p.join_hi};
            for (cudaEvent_t ev : evs)
                if (ev) cudaEventDestroy(ev);
            for (int g = 0; g < kPipeGroups; ++g) {
                if (p.k1[g]) cudaEventDestroy(p.k1[g]);
                if (p.k3[g]) cudaEventDestroy(p.k3[g]);
            }
        }
        g_pipe_pools.clear();
    }
    {
        std::lock_guard<std::mutex> lk(g_bwd_mu);
        for (auto& kv : g_bwd_pools) {
            for (int k = 0; k < kBwdStreams; ++k) {
                if (kv.second.st[k]) cudaStreamDestroy(kv.second.st[k]);
                if (kv.second.join[k]) cudaEventDestroy(kv.second.join[k]);
            }
            if (kv.second.fork) cudaEventDestroy(kv.second.fork);
        }
        g_bwd_pools.clear();
    }
    host_pools_free();
    {
        std::lock_guard<std::mutex> lk(g_bwdg_mu);
        for (auto& kv : g_bwdg) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        g_bwdg.clear();
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& kv : g_batch) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    g_batch.clear();
}

}  // extern "C"

// =========================================== forward pass without allocation
// Some callers cannot allocate device memory at call time: cudaMalloc may
// synchronise the device and may fail under memory pressure, so latency-
// critical loops and host frameworks that own every byte of device memory
// forbid it, and such callers cannot provide the workspace dgf_forward
// needs.  dgf_forward_noalloc keeps its FP32 (Abar, bbar) scratch in a
// fixed device array of this translation unit instead; the caller still
// passes inputs and outputs.
namespace dgf {

constexpr size_t kNoAllocPairs = size_t(1) << 20;  // (Abar, bbar) pairs: 8 MiB per device
static __device__ __align__(256) float2 g_noalloc_coef[kNoAllocPairs];
static std::mutex g_noalloc_mu;
static float2* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch on the current device; resolved once per
// device (host code cannot pass the array's name to a kernel: on the host
// it only stands in for the symbol).
static dgf_status noalloc_scratch(float2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(DGF_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_coef);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = static_cast<float2*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return DGF_OK;
}

}  // namespace dgf

extern "C" size_t dgf_noalloc_max_pairs(void) { return kNoAllocPairs; }

extern "C" dgf_status dgf_forward_noalloc(const void* p_l, const void* I_l, const void* I_h, void* O_h, int N,
                                          int C, int h_l, int w_l, int h, int w, int r, float eps, dgf_dtype dt,
                                          dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(false); st0 != DGF_OK) return st0;
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if (N == 0) return DGF_OK;
    if (p_l == nullptr || I_l == nullptr || I_h == nullptr || O_h == nullptr)
        return fail(DGF_ERR_INVALID, "NULL input or output pointer");
    const size_t pairs = (size_t)N * C * h_l * w_l;
    if (pairs > kNoAllocPairs)
        return fail(DGF_ERR_UNSUPPORTED,
                    "N*C*h_l*w_l = %zu exceeds the fixed scratch of %zu low-resolution pixels (8 MiB); "
                    "use dgf_forward with a workspace", pairs, kNoAllocPairs);
    float2* coef = nullptr;
    if ((st = noalloc_scratch(&coef)) != DGF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int planes = N * C;
    const Plan p = make_plan(dt, h_l, w_l, h, w, r, false, {I_h, O_h});
    // K1 overwrites every scratch entry the call reads, so stale contents
    // from an earlier call never reach the output.
    size_t landing = 0;
    TmaPair tma = make_tma_pair(I_l, dt, p_l, dt, planes, h_l, w_l, r, p.k1, landing);
    const size_t smem = k1_cfg_smem(p.k1, r, tma.enabled ? landing : 0);
    g_launches.fetch_add(1);
    cudaError_t e =
        launch_k1(dt, false, I_l, p_l, coef, planes, h_l, w_l, r, eps, p.k1, tma, smem, status_ptr(), nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "k1");
    g_launches.fetch_add(1);
    e = launch_k2_plan(dt, coef, I_h, O_h, planes, h_l, w_l, h, w, p, p.k2_strip ? p.k2_ls : p.k2_th, s);
    if (e != cudaSuccess) return cuda_fail(e, "k2");
    return DGF_OK;
}

// ====================================================== host-memory batches
// dgf_host_step: the planes of one batch in groups, each group's inputs
// copied in on one stream, its forward and backward on a second and its
// results copied out on a third, so copies in both directions overlap the
// kernels of the neighbouring groups.  Each group runs dgf_forward and
// dgf_backward on its planes (N = planes, C = 1: without a guidance
// transform the planes are independent), in device copies that sit at the
// planes' offsets of full-size device tensors.
namespace dgf {

struct HostLayout {
    size_t off[8];  // p_l, I_l, I_h, dO_h, O_h, dp_l, dI_l, dI_h
    size_t ws, total;
};

static int host_groups(int planes, int groups) {
    int G = groups > 0 ? groups : 6;
    G = std::min(G, kHostMaxGroups);
    return std::max(1, std::min(G, planes));
}

static HostLayout host_layout(int N, int C, int h_l, int w_l, int h, int w, dgf_dtype dt, int G) {
    HostLayout L;
    const size_t planes = (size_t)N * C, esz = esize(dt);
    const size_t lo = planes * h_l * w_l * esz, hi = planes * h * w * esz;
    const size_t sizes[8] = {lo, lo, hi, hi, hi, lo, lo, hi};
    size_t o = 0;
    for (int k = 0; k < 8; ++k) {
        L.off[k] = o;
        o += align256(sizes[k]);
    }
    const int gmax = (int)((planes + G - 1) / G);
    L.ws = o;
    L.total = o + align256(layout(gmax, 1, h_l, w_l, false).total);
    return L;
}

}  // namespace dgf

extern "C" size_t dgf_host_step_device_bytes(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt,
                                             int groups) {
    if (check_sizes(N, C, h_l, w_l, h, w, r, 1.f, dt) != DGF_OK) return 0;
    if (groups < 0 || groups > kHostMaxGroups) return 0;
    return host_layout(N, C, h_l, w_l, h, w, dt, host_groups(std::max(N * C, 1), groups)).total;
}

static dgf_status host_step_impl(const dgf_host_step_io* io, int N, int C, int h_l, int w_l, int h, int w, int r,
                                 float eps, dgf_dtype dt, int groups, void* device, size_t device_bytes,
                                 dgf_stream_t stream, bool mean_ab) {
    dgf_status st = check_sizes(N, C, h_l, w_l, h, w, r, eps, dt);
    if (st != DGF_OK) return st;
    if (io == nullptr) return fail(DGF_ERR_INVALID, "NULL io descriptor");
    if (groups < 0 || groups > kHostMaxGroups)
        return fail(DGF_ERR_INVALID, "groups = %d outside [0, %d]", groups, kHostMaxGroups);
    const bool bwd = io->dp_l != nullptr || io->dI_l != nullptr || io->dI_h != nullptr;
    if (io->p_l == nullptr || io->I_l == nullptr || io->I_h == nullptr || (bwd && io->dO_h == nullptr))
        return fail(DGF_ERR_INVALID, "NULL host input pointer");
    if (N == 0 || (io->O_h == nullptr && !bwd)) return DGF_OK;
    const int planes = N * C;
    const int G = host_groups(planes, groups);
    const HostLayout lay = host_layout(N, C, h_l, w_l, h, w, dt, G);
    if ((st = check_ws(device, device_bytes, lay.total)) != DGF_OK) return st;
    if (stream_capturing(reinterpret_cast<cudaStream_t>(stream)))
        return fail(DGF_ERR_UNSUPPORTED, "dgf_host_step under stream capture");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_host_mu);
    HostPool* hp = nullptr;
    if ((e = host_pool(dev, hp)) != cudaSuccess) return cuda_fail(e, "host-step streams");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(device);
    const size_t esz = esize(dt);
    const size_t lo_plane = (size_t)h_l * w_l * esz, hi_plane = (size_t)h * w * esz;
    const size_t plane_bytes[8] = {lo_plane, lo_plane, hi_plane, hi_plane, hi_plane, lo_plane, lo_plane, hi_plane};
    const void* hin[4] = {io->p_l, io->I_l, io->I_h, bwd ? io->dO_h : nullptr};
    void* hout[4] = {io->O_h, io->dp_l, io->dI_l, io->dI_h};
    void* ws = base + lay.ws;
    const size_t ws_bytes = lay.total - lay.ws;

    // fork: the three streams start after the caller's earlier work
    if ((e = cudaEventRecord(hp->fork, s)) != cudaSuccess) return cuda_fail(e, "fork");
    cudaStream_t sts[3] = {hp->in, hp->comp, hp->out};
    for (cudaStream_t x : sts)
        if ((e = cudaStreamWaitEvent(x, hp->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    dgf_status result = DGF_OK;
    for (int g = 0; g < G && result == DGF_OK; ++g) {
        const int p0 = (int)((size_t)planes * g / G), p1 = (int)((size_t)planes * (g + 1) / G);
        const int n = p1 - p0;
        auto dptr = [&](int k) { return base + lay.off[k] + (size_t)p0 * plane_bytes[k]; };
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (hin[k] != nullptr)
                e = cudaMemcpyAsync(dptr(k), static_cast<const char*>(hin[k]) + (size_t)p0 * plane_bytes[k],
                                    (size_t)n * plane_bytes[k], cudaMemcpyHostToDevice, hp->in);
        if (e == cudaSuccess) e = cudaEventRecord(hp->copied[g], hp->in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->comp, hp->copied[g], 0);
        if (e != cudaSuccess) {
            result = cuda_fail(e, "host-to-device copy");
            break;
        }
        dgf_stream_t cs = reinterpret_cast<dgf_stream_t>(hp->comp);
        if (io->O_h != nullptr)
            result = forward_impl(dptr(0), dptr(1), dptr(2), dptr(4), n, 1, h_l, w_l, h, w, r, eps, dt, nullptr, ws,
                                  ws_bytes, cs, mean_ab);
        if (result == DGF_OK && bwd)
            result = backward_impl(dptr(3), dptr(0), dptr(1), dptr(2), io->dp_l ? dptr(5) : nullptr,
                                   io->dI_l ? dptr(6) : nullptr, io->dI_h ? dptr(7) : nullptr, nullptr, n, 1, h_l,
                                   w_l, h, w, r, eps, dt, nullptr, ws, ws_bytes, cs, mean_ab);
        if (result != DGF_OK) break;
        if ((e = cudaEventRecord(hp->done[g], hp->comp)) == cudaSuccess)
            e = cudaStreamWaitEvent(hp->out, hp->done[g], 0);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (hout[k] != nullptr)
                e = cudaMemcpyAsync(static_cast<char*>(hout[k]) + (size_t)p0 * plane_bytes[4 + k], dptr(4 + k),
                                    (size_t)n * plane_bytes[4 + k], cudaMemcpyDeviceToHost, hp->out);
        if (e != cudaSuccess) result = cuda_fail(e, "device-to-host copy");
    }
    // join: the caller's stream waits for all three (also after an error)
    for (cudaStream_t x : sts) {
        cudaError_t ej = cudaEventRecord(hp->join, x);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, hp->join, 0);
        if (ej != cudaSuccess && result == DGF_OK) result = cuda_fail(ej, "join");
    }
    return result;
}

extern "C" dgf_status dgf_host_step(const dgf_host_step_io* io, int N, int C, int h_l, int w_l, int h, int w,
                                    int r, float eps, dgf_dtype dt, int groups, void* device, size_t device_bytes,
                                    dgf_stream_t stream) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    return host_step_impl(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream, true);
}

extern "C" dgf_status dgf_host_step_opt(const dgf_host_step_io* io, int N, int C, int h_l, int w_l, int h, int w,
                                        int r, float eps, dgf_dtype dt, int groups, void* device,
                                        size_t device_bytes, dgf_stream_t stream, const dgf_options* opt) {
    if (dgf_status st0 = entry_check(true); st0 != DGF_OK) return st0;
    bool mean_ab = true;
    if (dgf_status st = batch_options(opt, mean_ab); st != DGF_OK) return st;
    return host_step_impl(io, N, C, h_l, w_l, h, w, r, eps, dt, groups, device, device_bytes, stream, mean_ab);
}
