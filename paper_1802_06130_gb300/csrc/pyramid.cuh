// pyramid.cuh -- one 64x16 output tile of one channel of a 2x downsampling
// step (Section 4, "Multiscale filtering"): 5-tap binomial [1 4 6 4 1]/16,
// clamped borders, FP32 in a fixed order (horizontal fma chain over the
// clamped input rows, then the vertical chain), rounded to the storage type.
// Shared by the per-image pyramid kernel and the serving batch kernel.
#pragma once
#include "common.cuh"

namespace mdn {
namespace pyr {

constexpr int PTX = 64, PTY = 16, PNT = 256;
constexpr int PIW = 2 * PTX + 3, PIH = 2 * PTY + 3;
constexpr int PLOADS = (PIW * PIH + PNT - 1) / PNT;

// src/dst: one channel plane.  Loads are issued in register batches so that
// every thread keeps ~18 requests in flight (the step is HBM-bound).
template <typename TS>
__device__ __forceinline__ void tile_down(const TS* __restrict__ src, TS* __restrict__ dst, int H, int W, int Ho,
                                          int Wo, int ox0, int oy0, float (*tile)[PIW], float (*hs)[PTX + 1]) {
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const int tid = threadIdx.x;
    const int ix0 = 2 * ox0 - 2, iy0 = 2 * oy0 - 2;
    float v[PLOADS];
#pragma unroll
    for (int j = 0; j < PLOADS; ++j) {
        int i = tid + j * PNT;
        if (i < PIH * PIW) {
            int r = i / PIW, c = i % PIW;
            int gy = clampi(iy0 + r, 0, H - 1), gx = clampi(ix0 + c, 0, W - 1);
            const int64_t o = (int64_t)gy * W + gx;
            v[j] = mdn_in(o, (int64_t)H * W, 301) ? ld_f(src, o) : 0.f;
        }
    }
#pragma unroll
    for (int j = 0; j < PLOADS; ++j) {
        int i = tid + j * PNT;
        if (i < PIH * PIW) tile[i / PIW][i % PIW] = v[j];
    }
    __syncthreads();
    for (int i = tid; i < PIH * PTX; i += PNT) {
        int r = i / PTX, c = i % PTX;
        const float* p = &tile[r][mdn_in(2 * c + 4, PIW, 302) ? 2 * c : 0];
        float acc = __fmul_rn(b0, p[0]);
        acc = __fmaf_rn(b1, p[1], acc);
        acc = __fmaf_rn(b2, p[2], acc);
        acc = __fmaf_rn(b1, p[3], acc);
        acc = __fmaf_rn(b0, p[4], acc);
        hs[r][c] = acc;
    }
    __syncthreads();
    for (int i = tid; i < PTY * PTX; i += PNT) {
        int ty = i / PTX, tx = i % PTX;
        int ox = ox0 + tx, oy = oy0 + ty;
        if (ox < Wo && oy < Ho && mdn_in(2 * ty + 4, PIH, 303)) {
            float acc = __fmul_rn(b0, hs[2 * ty][tx]);
            acc = __fmaf_rn(b1, hs[2 * ty + 1][tx], acc);
            acc = __fmaf_rn(b2, hs[2 * ty + 2][tx], acc);
            acc = __fmaf_rn(b1, hs[2 * ty + 3][tx], acc);
            acc = __fmaf_rn(b0, hs[2 * ty + 4][tx], acc);
            st_f(dst, (int64_t)oy * Wo + ox, acc);
        }
    }
}

}  // namespace pyr
}  // namespace mdn
