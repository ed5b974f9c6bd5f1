// train_common.cuh -- regressor gather shared by the Gram kernels
// (SIMT and tcgen05): row r of A = [regressor | target] for the pixel
// sorted[r], in the FP32 working colour space.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace mdn {

constexpr int SORT_CHUNK = 4096;    // pixels per histogram/scatter block
constexpr int GRAM_CHUNK = 16384;   // max rows of one Gram work item (FP32 partial)
constexpr int GRAM_RB = 32;         // rows gathered per step (SIMT)
constexpr int GRAM_MAX_DP = 160;

// Working channel of Gram feature i (regressor tap or target) of group g:
// per-channel geometry uses channel g throughout; cross-channel features are
// ordered coarse (c, dy, dx), fine (c, dy, dx), then the three targets.
__host__ __device__ inline int feature_channel(int i, int g, int D, int rf, int rc, int cross) {
    if (!cross) return g;
    const int pc = rc >= 0 ? (2 * rc + 1) * (2 * rc + 1) : 0, pf = (2 * rf + 1) * (2 * rf + 1);
    if (i < 3 * pc) return i / pc;
    if (i < D) return (i - 3 * pc) / pf;
    return i - D;
}

// Centring constant of a working channel: luma (or any RGB channel) lies in
// [0, 1] and is shifted by 0.5, chroma is already centred.
__host__ __device__ inline double channel_center(int c, int color) {
    return (color == MDN_RGB || c == 0) ? 0.5 : 0.0;
}

struct GatherArgs {
    const float* zw;   // [n][3][h][w] working space, level l
    const float* tw;   // [n][3][h][w] working space, clean level l
    const float* cw;   // [n][3][hc][wc] working space, coarse output, or nullptr
    int h, w, hc, wc;
    int rf, rc, cross, color;
    int D, T, G, Dp, Dp4;   // Dp4: SIMT row stride, >= Dp + 1, multiple of 4
};

// Column codes of the SIMT Gram rows: src (0 coarse, 1 fine, 2 target,
// 3 ones) | c << 2 | (dy + 8) << 4 | (dx + 8) << 9.  Rows have Dq = Dp + 1
// columns: the regressor taps and targets, shifted by the channel's centring
// constant, then a ones column (see k_reduce_centered).
__device__ __forceinline__ void build_coltab(const GatherArgs& ga, int* coltab) {
    const int Dq = ga.Dp + 1;
    for (int e = threadIdx.x; e < ga.G * Dq; e += blockDim.x) {
        int g = e / Dq, j = e % Dq;
        int nch = ga.cross ? 3 : 1;
        int pc = ga.rc >= 0 ? (2 * ga.rc + 1) * (2 * ga.rc + 1) : 0;
        int pf = (2 * ga.rf + 1) * (2 * ga.rf + 1);
        int code;
        if (j < nch * pc) {
            int c = ga.cross ? j / pc : g, idx = j % pc;
            int dy = idx / (2 * ga.rc + 1) - ga.rc, dx = idx % (2 * ga.rc + 1) - ga.rc;
            code = 0 | (c << 2) | ((dy + 8) << 4) | ((dx + 8) << 9);
        } else if (j < ga.D) {
            int jj = j - nch * pc;
            int c = ga.cross ? jj / pf : g, idx = jj % pf;
            int dy = idx / (2 * ga.rf + 1) - ga.rf, dx = idx % (2 * ga.rf + 1) - ga.rf;
            code = 1 | (c << 2) | ((dy + 8) << 4) | ((dx + 8) << 9);
        } else if (j < ga.Dp) {
            int c = ga.cross ? j - ga.D : g;
            code = 2 | (c << 2) | (8 << 4) | (8 << 9);
        } else {
            code = 3;
        }
        coltab[e] = code;
    }
}

__device__ __forceinline__ float gather_value(const GatherArgs& ga, int code, int pix) {
    const int src = code & 3, c = (code >> 2) & 3;
    if (src == 3) return 1.f;
    const int hw = ga.h * ga.w;
    const int img = pix / hw, rem = pix % hw;
    const int y = rem / ga.w, x = rem % ga.w;
    const int dy = ((code >> 4) & 31) - 8, dx = ((code >> 9) & 31) - 8;
    const float cen = (float)channel_center(c, ga.color);
    if (src == 1) {
        int yy = clampi(y + dy, 0, ga.h - 1), xx = clampi(x + dx, 0, ga.w - 1);
        return __ldg(ga.zw + ((int64_t)img * 3 + c) * hw + (int64_t)yy * ga.w + xx) - cen;
    } else if (src == 0) {
        int yy = clampi(y / 2 + dy, 0, ga.hc - 1), xx = clampi(x / 2 + dx, 0, ga.wc - 1);
        return __ldg(ga.cw + ((int64_t)img * 3 + c) * ga.hc * ga.wc + (int64_t)yy * ga.wc + xx) - cen;
    }
    return __ldg(ga.tw + ((int64_t)img * 3 + c) * hw + rem) - cen;
}

// As[g][r][j] for r < nr (rows >= nr and columns >= Dq are zeroed), row
// stride DPs floats, RB rows per group.
__device__ __forceinline__ void gather_rows(const GatherArgs& ga, const int* coltab, const int* rows, int nr,
                                            float* As, int DPs, int RB) {
    const int per_g = RB * DPs, Dq = ga.Dp + 1;
    for (int e = threadIdx.x; e < ga.G * per_g; e += blockDim.x) {
        int g = e / per_g, r = (e / DPs) % RB, j = e % DPs;
        float v = 0.f;
        if (r < nr && j < Dq) v = gather_value(ga, coltab[g * Dq + j], rows[r]);
        As[e] = v;
    }
}

int gram_tc_error(int* out);
int launch_gram_tc(const GatherArgs& ga, int precision, const int4* chunks, int maxch, const int* sorted,
                   float* partial, cudaStream_t s);

}  // namespace mdn
