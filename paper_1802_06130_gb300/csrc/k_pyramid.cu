// k_pyramid.cu -- A1: one 2x downsampling step of the image pyramid
// (Section 4, "Multiscale filtering"; 5-tap binomial kernel, clamped borders).
//
// Arithmetic order (fixed, so that the result is reproducible bit for bit):
// for every input row r of the 5-row window, H_r = b0*p[2x-2] then
// fma(b1,p[2x-1]), fma(b2,p[2x]), fma(b3,p[2x+1]), fma(b4,p[2x+2]) in FP32;
// then out = b0*H_0, fma(b1,H_1) ... fma(b4,H_4); finally rounded to the
// storage type (RN-even for FP16).  b = [1 4 6 4 1]/16 is exact in FP32.
//
// Tiling: a CTA of 32x8 threads makes a 32x8 output tile; the 67x19 input
// window (clamped coordinates) of one channel is staged in shared memory with
// coalesced row loads, the horizontal pass writes 19x32 row sums to shared
// memory and the vertical pass produces the outputs.  HBM-bound: each input
// element is read once from DRAM (neighbouring tiles' halos hit L2).
#include "common.cuh"
#include "internal.h"

namespace mdn {
namespace {

constexpr int PTX = 32, PTY = 8;
constexpr int PIW = 2 * PTX + 3, PIH = 2 * PTY + 3;

template <typename TS>
__global__ void __launch_bounds__(PTX * PTY) k_pyramid_down(const TS* __restrict__ in, TS* __restrict__ out,
                                                            int H, int W, int Ho, int Wo) {
    __shared__ float tile[PIH][PIW + 1];
    __shared__ float hs[PIH][PTX + 1];
    const float b0 = 0.0625f, b1 = 0.25f, b2 = 0.375f;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PTX + tx;
    const int ox0 = blockIdx.x * PTX, oy0 = blockIdx.y * PTY;
    const int ix0 = 2 * ox0 - 2, iy0 = 2 * oy0 - 2;
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    const TS* src = in + ((int64_t)img * 3 + ch) * (int64_t)H * W;
    TS* dst = out + ((int64_t)img * 3 + ch) * (int64_t)Ho * Wo;
    for (int i = tid; i < PIH * PIW; i += PTX * PTY) {
        int r = i / PIW, c = i % PIW;
        int gy = clampi(iy0 + r, 0, H - 1), gx = clampi(ix0 + c, 0, W - 1);
        tile[r][c] = ld_f(src, (int64_t)gy * W + gx);
    }
    __syncthreads();
    for (int i = tid; i < PIH * PTX; i += PTX * PTY) {
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

}  // namespace

int launch_pyramid_down(const void* in, void* out, int dtype, int64_t n, int64_t h, int64_t w,
                        cudaStream_t s) {
    int64_t ho = (h + 1) / 2, wo = (w + 1) / 2;
    dim3 block(PTX, PTY);
    dim3 grid((unsigned)((wo + PTX - 1) / PTX), (unsigned)((ho + PTY - 1) / PTY), (unsigned)(n * 3));
    if (grid.y > 65535 || grid.z > 65535) return fail(MDN_ESHAPE, "pyramid: image too large");
    if (dtype == MDN_F32)
        k_pyramid_down<float><<<grid, block, 0, s>>>((const float*)in, (float*)out, (int)h, (int)w, (int)ho, (int)wo);
    else
        k_pyramid_down<__half><<<grid, block, 0, s>>>((const __half*)in, (__half*)out, (int)h, (int)w, (int)ho, (int)wo);
    return check_launch("k_pyramid_down");
}

}  // namespace mdn
