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
#include "pyramid.cuh"

namespace mdn {
namespace {

template <typename TS>
__global__ void __launch_bounds__(pyr::PNT) k_pyramid_down(const TS* __restrict__ in, TS* __restrict__ out, int H,
                                                           int W, int Ho, int Wo) {
    __shared__ float tile[pyr::PIH][pyr::PIW];
    __shared__ float hs[pyr::PIH][pyr::PTX + 1];
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    pyr::tile_down(in + ((int64_t)img * 3 + ch) * (int64_t)H * W, out + ((int64_t)img * 3 + ch) * (int64_t)Ho * Wo, H,
                   W, Ho, Wo, blockIdx.x * pyr::PTX, blockIdx.y * pyr::PTY, tile, hs);
}

}  // namespace

int launch_pyramid_down(const void* in, void* out, int dtype, int64_t n, int64_t h, int64_t w,
                        cudaStream_t s) {
    int64_t ho = (h + 1) / 2, wo = (w + 1) / 2;
    dim3 block(pyr::PNT);
    dim3 grid((unsigned)((wo + pyr::PTX - 1) / pyr::PTX), (unsigned)((ho + pyr::PTY - 1) / pyr::PTY), (unsigned)(n * 3));
    if (grid.y > 65535 || grid.z > 65535) return fail(MDN_ESHAPE, "pyramid: image too large");
    if (dtype == MDN_F32)
        k_pyramid_down<float><<<grid, block, 0, s>>>((const float*)in, (float*)out, (int)h, (int)w, (int)ho, (int)wo);
    else
        k_pyramid_down<__half><<<grid, block, 0, s>>>((const __half*)in, (__half*)out, (int)h, (int)w, (int)ho, (int)wo);
    return check_launch("k_pyramid_down");
}

}  // namespace mdn
