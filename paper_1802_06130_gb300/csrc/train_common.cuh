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

struct GatherArgs {
    const float* zw;   // [n][3][h][w] working space, level l
    const float* tw;   // [n][3][h][w] working space, clean level l
    const float* cw;   // [n][3][hc][wc] working space, coarse output, or nullptr
    int h, w, hc, wc;
    int rf, rc, cross;
    int D, T, G, Dp, Dp4;
};

// column code: src (0 coarse, 1 fine, 2 target) | c << 2 | (dy + 8) << 4 | (dx + 8) << 9
__device__ __forceinline__ void build_coltab(const GatherArgs& ga, int* coltab) {
    for (int e = threadIdx.x; e < ga.G * ga.Dp; e += blockDim.x) {
        int g = e / ga.Dp, j = e % ga.Dp;
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
        } else {
            int c = ga.cross ? j - ga.D : g;
            code = 2 | (c << 2) | (8 << 4) | (8 << 9);
        }
        coltab[e] = code;
    }
}

__device__ __forceinline__ float gather_value(const GatherArgs& ga, int code, int pix) {
    const int hw = ga.h * ga.w;
    const int img = pix / hw, rem = pix % hw;
    const int y = rem / ga.w, x = rem % ga.w;
    const int src = code & 3, c = (code >> 2) & 3;
    const int dy = ((code >> 4) & 31) - 8, dx = ((code >> 9) & 31) - 8;
    if (src == 1) {
        int yy = clampi(y + dy, 0, ga.h - 1), xx = clampi(x + dx, 0, ga.w - 1);
        return __ldg(ga.zw + ((int64_t)img * 3 + c) * hw + (int64_t)yy * ga.w + xx);
    } else if (src == 0) {
        int yy = clampi(y / 2 + dy, 0, ga.hc - 1), xx = clampi(x / 2 + dx, 0, ga.wc - 1);
        return __ldg(ga.cw + ((int64_t)img * 3 + c) * ga.hc * ga.wc + (int64_t)yy * ga.wc + xx);
    }
    return __ldg(ga.tw + ((int64_t)img * 3 + c) * hw + rem);
}

// As[g][r][j] for r < nr (rows >= nr and columns >= Dp are zeroed), row
// stride DPs floats, RB rows per group.
__device__ __forceinline__ void gather_rows(const GatherArgs& ga, const int* coltab, const int* rows, int nr,
                                            float* As, int DPs, int RB) {
    const int per_g = RB * DPs;
    for (int e = threadIdx.x; e < ga.G * per_g; e += blockDim.x) {
        int g = e / per_g, r = (e / DPs) % RB, j = e % DPs;
        float v = 0.f;
        if (r < nr && j < ga.Dp) v = gather_value(ga, coltab[g * ga.Dp + j], rows[r]);
        As[e] = v;
    }
}

int launch_gram_tc(const GatherArgs& ga, int precision, const int4* chunks, int maxch, const int* sorted,
                   float* partial, cudaStream_t s);

}  // namespace mdn
