// internal.h -- declarations shared between the C-ABI layer (capi.cu) and
// the kernel translation units.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>

#include "../../include/mdn.h"
#include <nvtx3/nvToolsExt.h>

namespace mdn {

// NVTX range over the lifetime of the object (a named span of host time on a
// profiler's timeline; free when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Per-thread error message; returns `code` for convenient `return fail(...)`.
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int check_launch(const char* where);

// Device-side selector parameters (FP32 thresholds, angle-sector boundary
// vectors), built on the host from mdn_bucket_params.
struct SelParams {
    int n_angle, n_strength, n_coherence;
    int nthr_s, nthr_c;
    float strength_thr[MDN_MAX_THR];
    float coherence_thr[MDN_MAX_THR];
    float coh_eps;
    // boundary unit vectors of the doubled orientation angle psi in [0, pi):
    // (cos, sin) of 2 pi k / n_angle for k = 1 .. n_angle/2 - 1
    float bcos[32];
    float bsin[32];
    // squared-domain forms of the thresholds (FP32 roundings of FP64 values):
    // strength_q = T^2, coherence_r = 2C / (1 + C^2) (1 for C = 1, +inf above),
    // eps2 = coh_eps^2
    float strength_q[MDN_MAX_THR];
    float coherence_r[MDN_MAX_THR];
    float eps2;
};
int make_sel_params(const mdn_bucket_params* bp, SelParams* out);

// 1-D normalised Gaussian (sigma 1.5, 5 taps), FP32, computed on the host.
void gauss5_weights(float w[5]);

struct LevelArgs {
    const void* z;        // [n][3][h][w] storage type
    const void* coarse;   // [n][3][hc][wc] or nullptr
    void* out;            // [n][3][h][w] or nullptr (select-only)
    void* buckets;        // [n][h][w] or nullptr, u8 (K <= 256) or u16
    const void* bank;     // [K][3][D], or prepared row slots when bank_rows
    int64_t n, h, w, hc, wc;
    int dtype, bank_dtype;   // bank_dtype: element type (MDN_F32 / MDN_F16)
    bool bank_rows;          // bank in the row-slot layout of mdn_prepare_bank_rows
    int K;
    mdn_geometry geom;
    SelParams sel;
    int variant = -1;        // level-kernel variant (LV_*), -1: autotune table, else the static rule
};
int launch_level(const LevelArgs& a, cudaStream_t s);

// Level-kernel variants of the per-image path (mdn_autotune_level times them).
enum LevelVariant {
    LV_FUSED_SMEM = 0,   // warp-specialised fused kernel, bank in shared memory (K <= 256, if it fits)
    LV_FUSED_L2 = 1,     // fused kernel reading a prepared bank through L2
    LV_STRIP = 2,        // strip kernel, bank in shared memory (K <= 256, if it fits)
    LV_TILE_SMEM = 3,    // one pixel per thread, bank in shared memory (if it fits)
    LV_TILE_L2 = 4,      // one pixel per thread, taps read through L2
    LV_FUSED_CLUSTER = 5,   // fused kernel on CTA pairs, FP32 bank split between their shared memories
    LV_COUNT = 6
};
// Autotune table (tune.cu): the variant recorded for this call's geometry,
// storage / bank types, K and image-size class, or -1.  Thread-safe.
int tune_lookup(const LevelArgs& a);
// Server entries: the level-kernel variant for a server geometry and bank width, or -1.
int tune_server_lookup(const mdn_geometry& g, bool wide);
void tune_server_store(const mdn_geometry& g, bool wide, int variant, float ms);
// variant forced on the calling thread's level calls (the tuner), -1 = none
extern thread_local int g_force_variant;
int launch_pyramid_down(const void* in, void* out, int dtype, int64_t n, int64_t h, int64_t w,
                        cudaStream_t s);

// ---- training ----
struct TrainArgs {
    const void* z;        // noisy level [n][3][h][w]
    const void* coarse;   // [n][3][hc][wc] or nullptr
    const void* target;   // clean level [n][3][h][w]
    int dtype;
    int64_t n, h, w, hc, wc;
    mdn_geometry geom;
    int K, D, G, T, Dp;
    int precision;
    double* gram;         // [K][G][Dp][Dp]
    int64_t* counts;      // [K]
    const void* buckets;  // [n][h][w] (computed beforehand), u8 (K <= 256) or u16
    void* ws;
    size_t ws_bytes;
};
size_t train_ws_bytes(int64_t n, int64_t h, int64_t w, int P, bool coarse, int K, int G, int Dp, int precision);
int launch_gram(const TrainArgs& a, cudaStream_t s);
size_t solve_ws_bytes(int K, int G, int D, int T);
int launch_solve(const double* gram, const int64_t* counts, int K, int G, int D, int T,
                 double lambda, float* bank_out, int32_t* status, void* ws, size_t ws_bytes,
                 cudaStream_t s);

int num_sms();
// image sizes: h, w <= 2^20 and n * 3 * h * w < 2^31, checked without overflow
bool dims_ok(int64_t n, int64_t h, int64_t w);
int check_img(const void* p, int dtype, int64_t n, int64_t h, int64_t w, const char* what);
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// bytes per pixel of a bucket map of K buckets
inline int bucket_bytes(int K) { return K <= 256 ? 1 : 2; }
inline int regressor_len(const mdn_geometry& g) {
    int pf = (2 * g.r_fine + 1) * (2 * g.r_fine + 1);
    int pc = g.r_coarse >= 0 ? (2 * g.r_coarse + 1) * (2 * g.r_coarse + 1) : 0;
    return (g.cross_channel ? 3 : 1) * (pf + pc);
}

}  // namespace mdn
