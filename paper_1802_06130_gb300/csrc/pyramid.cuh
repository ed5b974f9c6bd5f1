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
// rows start on 16-byte boundaries, 256 threads.  The 131 x 67 input
// window is loaded as an aligned superset of whole 16-byte vectors (VE
// elements each, columns xa .. xa + NV*VE - 1 with xa = ix0 rounded down to
// VE) and staged with its even and odd columns in separate rows E and O, so
// that output column c's horizontal taps E[o2+c], O[o2+c], E[o2+c+1],
// O[o2+c+1], E[o2+c+2] are consecutive across the lanes (no bank
// conflicts).  Thread (c, seg) then makes output column c of the FRY = 8
// rows FRY seg .. FRY seg + FRY - 1: the 2 FRY + 3 horizontal sums of its
// input rows in turn, with the vertical 5-tap window held in registers.  The values and the two
// FP32 chains are those of tile_down, so the outputs are bit-identical.
constexpr int FTY = 32, FNT = 256, FSEG = FNT / PTX, FRY = FTY / FSEG;   // FRY output rows per thread
constexpr int FIH = 2 * FTY + 3;                                   // staged input rows
template <typename TS> struct Fast {
    static constexpr int VE = 16 / (int)sizeof(TS);              // elements per 16-byte vector
    static constexpr int NV = (PIW + VE - 1 + VE - 1) / VE;       // vectors per window row (any ix0 - xa < VE)
    static constexpr int PITCH = NV * VE;                          // staged columns per row
    static constexpr int HP = PITCH / 2;                           // floats per E or O row
    static constexpr int NLD = (FIH * NV + FNT - 1) / FNT;        // vector loads per thread
    static constexpr int SMEM_FLOATS = 2 * FIH * HP;
};

// Staged window of one tile: FIH input rows of NV 16-byte vectors from
// (iy0, xa), rows clamped to the image.  With W a multiple of VE and xa a
// multiple of VE, a vector lies wholly inside its row or wholly outside it;
// one outside holds the row's edge element VE times (the clamped columns of
// tile_down).  Thread tid's share is vectors tid, tid + FNT, ...
template <typename TS>
__device__ __forceinline__ void fast_fetch(const TS* __restrict__ src, int H, int W, int iy0, int xa,
                                           uint4 (&v)[Fast<TS>::NLD]) {
    using F = Fast<TS>;
#pragma unroll
    for (int j = 0; j < F::NLD; ++j) {
        const int i = threadIdx.x + j * FNT;
        if (i < FIH * F::NV) {
            const int r = i / F::NV, q = i - r * F::NV;
            const int gy = clampi(iy0 + r, 0, H - 1), x = xa + q * F::VE;
            if (x >= 0 && x + F::VE <= W) {
                const int64_t o = (int64_t)gy * W + x;
                v[j] = mdn_in(o + F::VE - 1, (int64_t)H * W, 304) ? __ldg(reinterpret_cast<const uint4*>(src + o))
                                                                  : make_uint4(0, 0, 0, 0);
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
                v[j] = make_uint4(b, b, b, b);
            }
        }
    }
}

// The fetched vectors into the E (even staged columns) and O (odd) rows.
template <typename TS>
__device__ __forceinline__ void fast_stage(const uint4 (&v)[Fast<TS>::NLD], float* __restrict__ sm) {
    using F = Fast<TS>;
    float* E = sm;
    float* O = sm + FIH * F::HP;
#pragma unroll
    for (int j = 0; j < F::NLD; ++j) {
        const int i = threadIdx.x + j * FNT;
        if (i < FIH * F::NV) {
            const int r = i / F::NV, q = i - r * F::NV;
            if constexpr (sizeof(TS) == 2) {
                const uint32_t w4[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
                float f[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 p2 = __half22float2(*reinterpret_cast<const __half2*>(&w4[k]));
                    f[2 * k] = p2.x;
                    f[2 * k + 1] = p2.y;
                }
                *reinterpret_cast<float4*>(E + r * F::HP + 4 * q) = make_float4(f[0], f[2], f[4], f[6]);
                *reinterpret_cast<float4*>(O + r * F::HP + 4 * q) = make_float4(f[1], f[3], f[5], f[7]);
            } else {
                *reinterpret_cast<float2*>(E + r * F::HP + 2 * q) =
                    make_float2(__uint_as_float(v[j].x), __uint_as_float(v[j].z));
                *reinterpret_cast<float2*>(O + r * F::HP + 2 * q) =
                    make_float2(__uint_as_float(v[j].y), __uint_as_float(v[j].w));
            }
        }
    }
}

// Outputs of one staged interior tile: thread (c, seg) makes column c of
// rows FRY seg .. FRY seg + FRY - 1; o2 = (ix0 - xa) / 2.
template <typename TS>
__device__ __forceinline__ void fast_compute(const float* __restrict__ sm, TS* __restrict__ dst, int Ho, int Wo,
                                             int ox0, int oy0, int o2) {
    using F = Fast<TS>;
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const float* E = sm;
    const float* O = sm + FIH * F::HP;
    const int c = threadIdx.x % PTX, seg = threadIdx.x / PTX;
    const int k0 = mdn_in(o2 + c + 2, F::HP, 305) ? o2 + c : 0;
    auto hrow = [&](int r) {   // horizontal sum of staged input row r at output column c
        const float* e = E + r * F::HP + k0;
        const float* od = O + r * F::HP + k0;
        float acc = __fmul_rn(b0, e[0]);
        acc = __fmaf_rn(b1, od[0], acc);
        acc = __fmaf_rn(b2, e[1], acc);
        acc = __fmaf_rn(b1, od[1], acc);
        acc = __fmaf_rn(b0, e[2], acc);
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
