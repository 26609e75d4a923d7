// Autotuner of the tile shapes: per (kernel, storage type, radius or
// factor, vector width, guide type) it times every candidate shape on the
// call's own buffers with CUDA events and keeps the fastest.  The choice is
// cached in memory and, when DGF_TUNE_CACHE names a file, persisted there
// as text lines "version/device kind dt r F vec gf32 sc a b": keyed also by the
// device name and by the cache version of this library (kTuneVersion, raised
// whenever the kernels' shapes or their encoding change), so entries written
// by another build or for another GPU are never used.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "tune.h"

namespace dgf {

namespace {

std::mutex g_mu;
using FullKey = std::tuple<std::string, int, int, int, int, int, int, int>;
std::map<FullKey, std::pair<int, int>> g_table;
bool g_loaded = false;
int g_enabled = -1;  // -1: read DGF_AUTOTUNE on first use

constexpr const char* kTuneVersion = "dgf3";

std::string device_name() {
    int dev = 0;
    cudaDeviceProp p;
    std::string s = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
        s = p.name;
    } else {
        cudaGetLastError();  // no device here: leave no error behind for later calls
    }
    for (auto& ch : s)
        if (ch == ' ' || ch == '/') ch = '_';
    return std::string(kTuneVersion) + "/" + s;
}

// a table entry the plan code can read: shapes are positive except b of the
// low-res kernels (kinds 1, 4), where b < 0 names the sliding strips
bool entry_ok(int kind, int dt, int r, int F, int vec, int gf32, int sc, int a, int b) {
    if (kind < 1 || kind > 6 || dt < 0 || dt > 2 || r < 0 || r > 64 || F < 0 || F > 64 || vec < 0 || vec > 64)
        return false;
    if ((gf32 != 0 && gf32 != 1) || (sc != 0 && sc != 1)) return false;
    if (a < 0 || a > 4096 || (a == 0 && kind < 5)) return false;
    const int bmin = (kind == 1 || kind == 4) ? -8 : 0;
    return b >= bmin && b <= 4096;
}

FullKey full_key(const TuneKey& k) {
    return std::make_tuple(device_name(), k.kind, k.dt, k.r, k.F, k.vec, k.gf32, k.sc);
}

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = getenv("DGF_TUNE_CACHE");
    if (path == nullptr || *path == 0) return;
    FILE* f = fopen(path, "r");
    if (f == nullptr) return;
    char line[512], name[256];
    int kind, dt, r, F, vec, gf32, sc, a, b;
    // malformed, out-of-range or truncated lines are skipped one by one: a
    // corrupt cache only costs a re-tune of the keys it held; lines of
    // another version or device stay in the file but never match a key
    while (fgets(line, sizeof line, f) != nullptr) {
        char tail = 0;
        const int n = sscanf(line, "%255s %d %d %d %d %d %d %d %d %d %c", name, &kind, &dt, &r, &F, &vec, &gf32,
                             &sc, &a, &b, &tail);
        if (n != 10 || !entry_ok(kind, dt, r, F, vec, gf32, sc, a, b)) continue;
        g_table[std::make_tuple(std::string(name), kind, dt, r, F, vec, gf32, sc)] = {a, b};
    }
    fclose(f);
}

void save_locked() {
    const char* path = getenv("DGF_TUNE_CACHE");
    if (path == nullptr || *path == 0) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (f == nullptr) return;
    for (auto& kv : g_table) {
        const auto& k = kv.first;
        fprintf(f, "%s %d %d %d %d %d %d %d %d %d\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k),
                std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), kv.second.first,
                kv.second.second);
    }
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

bool tune_enabled() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_enabled < 0) {
        const char* e = getenv("DGF_AUTOTUNE");
        g_enabled = (e != nullptr && strcmp(e, "1") == 0) ? 1 : 0;
    }
    return g_enabled == 1;
}

void tune_set_enabled(bool on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled = on ? 1 : 0;
}

bool tune_lookup(const TuneKey& k, int& a, int& b) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_table.find(full_key(k));
    if (it == g_table.end()) return false;
    a = it->second.first;
    b = it->second.second;
    return true;
}

void tune_store(const TuneKey& k, int a, int b) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_table[full_key(k)] = {a, b};
    save_locked();
}

void tune_clear() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
    g_loaded = true;
}

// entries this device and library version would use
int tune_count() {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    const std::string me = device_name();
    int n = 0;
    for (auto& kv : g_table) n += std::get<0>(kv.first) == me;
    return n;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return true;
    return st != cudaStreamCaptureStatusNone;
}

float time_launch(cudaStream_t s, const std::function<cudaError_t()>& fn, int reps) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    if (fn() == cudaSuccess) {  // warm-up (attributes, first-touch)
        cudaEventRecord(a, s);
        bool ok = true;
        for (int i = 0; i < reps && ok; ++i) ok = fn() == cudaSuccess;
        cudaEventRecord(b, s);
        if (ok && cudaEventSynchronize(b) == cudaSuccess) {
            cudaEventElapsedTime(&ms, a, b);
            ms /= reps;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace dgf
