// Tile-shape autotuner (host side).
#pragma once

#include <cuda_runtime.h>

#include <functional>

namespace dgf {

// kind: 1 = K1 low-res coefficients, 2 = K2 high-res apply, 3 = K3 high-res
// backward, 4 = K4 low-res backward, 5 = fused forward K12, 6 = fused
// backward K13.  The value (a, b) is the kernel's shape: K1/K4 tiles as
// a = CW and b = EY1; K1 warp strips as a = rows per segment and b = 0
// (b < 0: the sliding strips with -b columns per lane); K2: a = rows per
// tile; K3: a = low-res rows per strip segment; K12/K13: a = low-res rows
// per segment, or 0 when the two-kernel form is faster for the key.
// sc: the plane's size class (1: a low-res plane under 128 x 128 pixels,
// whose kernels are bound by the latency of a few short walks; 0: larger),
// so shapes tuned on small images never serve large ones or the reverse.
struct TuneKey {
    int kind, dt, r, F, vec, gf32, sc;
};

inline int tune_size_class(int h_l, int w_l) { return (long long)h_l * w_l < 128 * 128 ? 1 : 0; }

bool tune_enabled();
void tune_set_enabled(bool on);
bool tune_lookup(const TuneKey& k, int& a, int& b);
void tune_store(const TuneKey& k, int a, int b);
void tune_clear();
int tune_count();
bool stream_capturing(cudaStream_t s);
// Average milliseconds of `reps` launches after one warm-up; -1 on error.
float time_launch(cudaStream_t s, const std::function<cudaError_t()>& fn, int reps);

}  // namespace dgf
