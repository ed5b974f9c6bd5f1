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
template <typename TS, int NT = PNT>
__device__ __forceinline__ void tile_down(const TS* __restrict__ src, TS* __restrict__ dst, int H, int W, int Ho,
                                          int Wo, int ox0, int oy0, float (*tile)[PIW], float (*hs)[PTX + 1]) {
    constexpr int NLOADS = (PIW * PIH + NT - 1) / NT;
    constexpr int BATCH = NLOADS < 9 ? NLOADS : 9;            // loads in flight per thread
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const int tid = threadIdx.x;
    const int ix0 = 2 * ox0 - 2, iy0 = 2 * oy0 - 2;
    for (int j0 = 0; j0 < NLOADS; j0 += BATCH) {
        float v[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            int i = tid + (j0 + j) * NT;
            if (i < PIH * PIW) {
                int r = i / PIW, c = i % PIW;
                int gy = clampi(iy0 + r, 0, H - 1), gx = clampi(ix0 + c, 0, W - 1);
                const int64_t o = (int64_t)gy * W + gx;
                v[j] = mdn_in(o, (int64_t)H * W, 301) ? ld_f(src, o) : 0.f;
            }
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            int i = tid + (j0 + j) * NT;
            if (i < PIH * PIW) tile[i / PIW][i % PIW] = v[j];
        }
    }
    __syncthreads();
    for (int i = tid; i < PIH * PTX; i += NT) {
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
    for (int i = tid; i < PTY * PTX; i += NT) {
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

// Per-image fast path (k_pyramid_fast): 64 x 32 output tiles of images whose
// rows start on 16-byte boundaries, 256 threads.  The 131 x 67 input window
// of a tile is copied raw (storage type) into one of two shared-memory
// stages as an aligned superset of whole 16-byte vectors (VE elements each:
// columns xa .. xa + NV*VE - 1 with xa = ix0 rounded down to VE), by
// cp.async so that the next tile's copies are in flight while the current
// tile is computed; rows are clamped to the image, and with W and xa
// multiples of VE a vector lies wholly inside its row or wholly outside it,
// one outside being filled with the row's edge element (the clamped columns
// of tile_down).  Output column c's horizontal taps p[2c .. 2c + 4] are the
// staged elements off + 2c .. off + 2c + 4 (off = ix0 - xa is even), i.e.
// three consecutive element pairs starting at pair o2 + c (o2 = off / 2):
// one 32-bit word of two FP16 values or one 8-byte pair of FP32 values each,
// consecutive across the lanes.  Thread (c, seg) makes output column c of
// the FRY = 8 rows FRY seg .. FRY seg + FRY - 1: the 2 FRY + 3 horizontal
// sums of its input rows in turn, with the vertical 5-tap window in
// registers.  The values and the two FP32 chains are those of tile_down, so
// the outputs are bit-identical.
constexpr int FTY = 32, FNT = 256, FSEG = FNT / PTX, FRY = FTY / FSEG;   // FRY output rows per thread
constexpr int FIH = 2 * FTY + 3;                                   // staged input rows
template <typename TS> struct Fast {
    static constexpr int VE = 16 / (int)sizeof(TS);              // elements per 16-byte vector
    static constexpr int NV = (PIW + VE - 1 + VE - 1) / VE;       // vectors per window row (any ix0 - xa < VE)
    static constexpr int PITCH = NV * VE;                          // staged elements per row
    static constexpr size_t STAGE_BYTES = (size_t)FIH * PITCH * sizeof(TS);
    static constexpr size_t SMEM_BYTES = 2 * STAGE_BYTES;
};

// Starts the copies of one tile's window into `stage` (cp.async, then one
// commit group per call); vectors outside a row are stored directly.
template <typename TS>
__device__ __forceinline__ void raw_issue(const TS* __restrict__ src, int H, int W, int iy0, int xa,
                                          TS* __restrict__ stage) {
    using F = Fast<TS>;
    for (int i = threadIdx.x; i < FIH * F::NV; i += FNT) {
        const int r = i / F::NV, q = i - r * F::NV;
        const int gy = clampi(iy0 + r, 0, H - 1), x = xa + q * F::VE;
        TS* dst = stage + r * F::PITCH + q * F::VE;
        if (x >= 0 && x + F::VE <= W) {
            const int64_t o = (int64_t)gy * W + x;
            const TS* g = src + (mdn_in(o + F::VE - 1, (int64_t)H * W, 304) ? o : 0);
            const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
        } else {
            const int64_t o = (int64_t)gy * W + (x < 0 ? 0 : W - 1);
            const TS e = src[mdn_in(o, (int64_t)H * W, 306) ? o : 0];
            uint32_t b;
            if constexpr (sizeof(TS) == 2) {
                const uint32_t h = __half_as_ushort(e);
                b = h | (h << 16);
            } else {
                b = __float_as_uint(e);
            }
            *reinterpret_cast<uint4*>(dst) = make_uint4(b, b, b, b);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// element pair k of a staged row as two floats
template <typename TS> __device__ __forceinline__ float2 pair_at(const TS* row, int k) {
    if constexpr (sizeof(TS) == 2) return __half22float2(reinterpret_cast<const __half2*>(row)[k]);
    else return reinterpret_cast<const float2*>(row)[k];
}

// Outputs of one staged tile: thread (c, seg) makes column c of rows
// FRY seg .. FRY seg + FRY - 1; o2 = (ix0 - xa) / 2.
template <typename TS>
__device__ __forceinline__ void raw_compute(const TS* __restrict__ stage, TS* __restrict__ dst, int Ho, int Wo,
                                            int ox0, int oy0, int o2) {
    using F = Fast<TS>;
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const int c = threadIdx.x % PTX, seg = threadIdx.x / PTX;
    const int k0 = mdn_in(2 * (o2 + c + 2) + 1, F::PITCH, 305) ? o2 + c : 0;
    auto hrow = [&](int r) {   // horizontal sum of staged input row r at output column c
        const TS* row = stage + r * F::PITCH;
        const float2 p0 = pair_at<TS>(row, k0), p1 = pair_at<TS>(row, k0 + 1), p2 = pair_at<TS>(row, k0 + 2);
        float acc = __fmul_rn(b0, p0.x);
        acc = __fmaf_rn(b1, p0.y, acc);
        acc = __fmaf_rn(b2, p1.x, acc);
        acc = __fmaf_rn(b1, p1.y, acc);
        acc = __fmaf_rn(b0, p2.x, acc);
        return acc;
    };
    const int r0 = 2 * FRY * seg;   // first staged row of this segment's window
    float h0 = hrow(r0), h1 = hrow(r0 + 1), h2 = hrow(r0 + 2);
    const int ox = ox0 + c;
#pragma unroll
    for (int k = 0; k < FRY; ++k) {
        const float h3 = hrow(r0 + 2 * k + 3), h4 = hrow(r0 + 2 * k + 4);
        float acc = __fmul_rn(b0, h0);
        acc = __fmaf_rn(b1, h1, acc);
        acc = __fmaf_rn(b2, h2, acc);
        acc = __fmaf_rn(b1, h3, acc);
        acc = __fmaf_rn(b0, h4, acc);
        const int oy = oy0 + FRY * seg + k;
        if (ox < Wo && oy < Ho) st_f(dst, (int64_t)oy * Wo + ox, acc);
        h0 = h2;
        h1 = h3;
        h2 = h4;
    }
}

}  // namespace pyr
}  // namespace mdn
