// k_pyramid.cu -- A1: one 2x downsampling step of the image pyramid
// (Section 4, "Multiscale filtering"; 5-tap binomial kernel, clamped borders).
//
// Arithmetic order (fixed, so that the result is reproducible bit for bit):
// for every input row r of the 5-row window, H_r = b0*p[2x-2] then
// fma(b1,p[2x-1]), fma(b2,p[2x]), fma(b3,p[2x+1]), fma(b4,p[2x+2]) in FP32;
// then out = b0*H_0, fma(b1,H_1) ... fma(b4,H_4); finally rounded to the
// storage type (RN-even for FP16).  b = [1 4 6 4 1]/16 is exact in FP32.
//
// Tiling: a CTA makes a 64x16 output tile of one channel; the 131x35 input
// window (clamped coordinates) is staged in shared memory with coalesced,
// register-batched loads, the horizontal pass writes 35x64 row sums to shared
// memory and the vertical pass produces the outputs.  HBM-bound: each input
// element is read once from DRAM (neighbouring tiles' halos hit L2).
#include "common.cuh"
#include "internal.h"

namespace mdn {
namespace {

// Output tile 64 x 16 of one channel per CTA (256 threads); input window
// 131 x 35 (clamped).  Loads are issued in register batches so that every
// thread keeps ~18 requests in flight (the kernel is HBM-bound).
constexpr int PTX = 64, PTY = 16, PNT = 256;
constexpr int PIW = 2 * PTX + 3, PIH = 2 * PTY + 3;
constexpr int PLOADS = (PIW * PIH + PNT - 1) / PNT;

template <typename TS>
__global__ void __launch_bounds__(PNT) k_pyramid_down(const TS* __restrict__ in, TS* __restrict__ out, int H, int W,
                                                      int Ho, int Wo) {
    __shared__ float tile[PIH][PIW];
    __shared__ float hs[PIH][PTX + 1];
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const int tid = threadIdx.x;
    const int ox0 = blockIdx.x * PTX, oy0 = blockIdx.y * PTY;
    const int ix0 = 2 * ox0 - 2, iy0 = 2 * oy0 - 2;
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    const TS* src = in + ((int64_t)img * 3 + ch) * (int64_t)H * W;
    TS* dst = out + ((int64_t)img * 3 + ch) * (int64_t)Ho * Wo;
    float v[PLOADS];
#pragma unroll
    for (int j = 0; j < PLOADS; ++j) {
        int i = tid + j * PNT;
        if (i < PIH * PIW) {
            int r = i / PIW, c = i % PIW;
            int gy = clampi(iy0 + r, 0, H - 1), gx = clampi(ix0 + c, 0, W - 1);
            v[j] = ld_f(src, (int64_t)gy * W + gx);
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
        const float* p = &tile[r][2 * c];
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
        if (ox < Wo && oy < Ho) {
            float acc = __fmul_rn(b0, hs[2 * ty][tx]);
            acc = __fmaf_rn(b1, hs[2 * ty + 1][tx], acc);
            acc = __fmaf_rn(b2, hs[2 * ty + 2][tx], acc);
            acc = __fmaf_rn(b1, hs[2 * ty + 3][tx], acc);
            acc = __fmaf_rn(b0, hs[2 * ty + 4][tx], acc);
            st_f(dst, (int64_t)oy * Wo + ox, acc);
        }
    }
}

}  // namespace

int launch_pyramid_down(const void* in, void* out, int dtype, int64_t n, int64_t h, int64_t w,
                        cudaStream_t s) {
    int64_t ho = (h + 1) / 2, wo = (w + 1) / 2;
    dim3 block(PNT);
    dim3 grid((unsigned)((wo + PTX - 1) / PTX), (unsigned)((ho + PTY - 1) / PTY), (unsigned)(n * 3));
    if (grid.y > 65535 || grid.z > 65535) return fail(MDN_ESHAPE, "pyramid: image too large");
    if (dtype == MDN_F32)
        k_pyramid_down<float><<<grid, block, 0, s>>>((const float*)in, (float*)out, (int)h, (int)w, (int)ho, (int)wo);
    else
        k_pyramid_down<__half><<<grid, block, 0, s>>>((const __half*)in, (__half*)out, (int)h, (int)w, (int)ho, (int)wo);
    return check_launch("k_pyramid_down");
}

}  // namespace mdn
