// k_pyramid.cu -- A1: one 2x downsampling step of the image pyramid
// (Section 4, "Multiscale filtering"; 5-tap binomial kernel, clamped borders).
//
// Arithmetic order (fixed, so that the result is reproducible bit for bit):
// for every input row r of the 5-row window, H_r = b0*p[2x-2] then
// fma(b1,p[2x-1]), fma(b2,p[2x]), fma(b3,p[2x+1]), fma(b4,p[2x+2]) in FP32;
// then out = b0*H_0, fma(b1,H_1) ... fma(b4,H_4); finally rounded to the
// storage type (RN-even for FP16).  b = [1 4 6 4 1]/16 is exact in FP32.
//
// Tiling: 64x32 output tiles of one channel.  Images whose rows start on
// 16-byte boundaries (W a multiple of 8 for FP16, 4 for FP32, aligned base)
// go to the persistent kernel k_pyramid_fast: each CTA walks its tiles with
// the next tile's window copying (cp.async, 16-byte vectors, rows clamped,
// vectors outside a row filled with its edge element) into one of two
// shared-memory stages while the current one is computed from the other
// (per-thread output columns reading element pairs, the vertical window in
// registers; see pyramid.cuh), so DRAM latency overlaps the arithmetic.  Other images go to
// k_pyramid_down, which stages the clamped 131x35 windows of the two 64x16
// halves with scalar loads.  Both give the same FP32 chains on the same
// clamped values, so every tile follows the fixed FP32 order above bit for
// bit.  Each input element is read once from DRAM (neighbouring tiles'
// halos hit L2).
#include "common.cuh"
#include "internal.h"
#include "pyramid.cuh"

namespace mdn {
namespace {

// Every tile of every plane (ntx x nty per plane), persistent CTAs, the
// next tile's window copying into the other shared-memory stage while the
// current one is computed.
template <typename TS>
__global__ void __launch_bounds__(pyr::FNT) k_pyramid_fast(const TS* __restrict__ in, TS* __restrict__ out, int H,
                                                           int W, int Ho, int Wo, int nplanes, int ntx, int nty) {
    using F = pyr::Fast<TS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto stage = [&](int k) { return reinterpret_cast<TS*>(smem_raw + (k & 1) * F::STAGE_BYTES); };
    const int64_t per_plane = (int64_t)ntx * nty, ntiles = per_plane * nplanes;
    // ix0 = 128 tx - 2 and xa = floor(ix0 / VE) VE = 128 tx - VE, so (ix0 - xa) / 2 is the same for all tiles
    constexpr int O2 = (F::VE - 2) / 2;
    auto where = [&](int64_t t, const TS*& src, TS*& dst, int& ox0, int& oy0) {
        const int plane = (int)(t / per_plane), rem = (int)(t - (int64_t)plane * per_plane);
        const int tx = rem % ntx, ty = rem / ntx;
        src = in + (int64_t)plane * H * W;
        dst = out + (int64_t)plane * Ho * Wo;
        ox0 = tx * pyr::PTX;
        oy0 = ty * pyr::FTY;
    };
    int64_t t = blockIdx.x;
    if (t < ntiles) {
        const TS* src; TS* dst; int ox0, oy0;
        where(t, src, dst, ox0, oy0);
        pyr::raw_issue<TS>(src, H, W, 2 * oy0 - 2, 2 * ox0 - F::VE, stage(0));
    }
    for (int i = 0; t < ntiles; t += gridDim.x, ++i) {
        const TS* src; TS* dst; int ox0, oy0;
        where(t, src, dst, ox0, oy0);
        if (t + gridDim.x < ntiles) {   // the next tile into the other stage (read two iterations ago)
            const TS* s2; TS* d2; int x2, y2;
            where(t + gridDim.x, s2, d2, x2, y2);
            pyr::raw_issue<TS>(s2, H, W, 2 * y2 - 2, 2 * x2 - F::VE, stage(i + 1));
            asm volatile("cp.async.wait_group 1;" ::: "memory");   // this tile's copies landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();   // every thread's copies and edge stores of this tile are visible
        pyr::raw_compute<TS>(stage(i), dst, Ho, Wo, ox0, oy0, O2);
        __syncthreads();   // the stage is read before it is refilled
    }
}

// Images whose rows are not 16-byte aligned: two scalar 64x16 halves per tile.
template <typename TS>
__global__ void __launch_bounds__(pyr::FNT) k_pyramid_down(const TS* __restrict__ in, TS* __restrict__ out, int H,
                                                           int W, int Ho, int Wo) {
    __shared__ float tile[pyr::PIH][pyr::PIW];
    __shared__ float hs[pyr::PIH][pyr::PTX + 1];
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    const TS* src = in + ((int64_t)img * 3 + ch) * (int64_t)H * W;
    TS* dst = out + ((int64_t)img * 3 + ch) * (int64_t)Ho * Wo;
    for (int half = 0; half < pyr::FTY / pyr::PTY; ++half) {
        if (half) __syncthreads();   // the previous half is done with the buffers
        pyr::tile_down<TS, pyr::FNT>(src, dst, H, W, Ho, Wo, tx * pyr::PTX, ty * pyr::FTY + half * pyr::PTY, tile,
                                     hs);
    }
}

template <typename TS>
int launch_typed(const TS* in, TS* out, int64_t n, int64_t h, int64_t w, cudaStream_t s) {
    using F = pyr::Fast<TS>;
    const int64_t ho = (h + 1) / 2, wo = (w + 1) / 2;
    const int64_t ntx_all = (wo + pyr::PTX - 1) / pyr::PTX, nty_all = (ho + pyr::FTY - 1) / pyr::FTY;
    if (nty_all > 65535 || n * 3 > 65535) return fail(MDN_ESHAPE, "pyramid: image too large");
    if (w % F::VE == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
        auto kern = k_pyramid_fast<TS>;
        const int bytes = (int)F::SMEM_BYTES;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "k_pyramid_fast: smem attribute");
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, pyr::FNT, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "k_pyramid_fast: occupancy");
        const int64_t ntiles = ntx_all * nty_all * n * 3;
        int64_t grid = (int64_t)num_sms() * (occ > 0 ? occ : 1);
        if (grid > ntiles) grid = ntiles;
        kern<<<(unsigned)grid, pyr::FNT, bytes, s>>>(in, out, (int)h, (int)w, (int)ho, (int)wo, (int)(n * 3),
                                                 (int)ntx_all, (int)nty_all);
        return check_launch("k_pyramid_fast");
    }
    dim3 grid((unsigned)ntx_all, (unsigned)nty_all, (unsigned)(n * 3));
    k_pyramid_down<TS><<<grid, pyr::FNT, 0, s>>>(in, out, (int)h, (int)w, (int)ho, (int)wo);
    return check_launch("k_pyramid_down");
}

}  // namespace

int launch_pyramid_down(const void* in, void* out, int dtype, int64_t n, int64_t h, int64_t w,
                        cudaStream_t s) {
    if (dtype == MDN_F32) return launch_typed<float>((const float*)in, (float*)out, n, h, w, s);
    return launch_typed<__half>((const __half*)in, (__half*)out, n, h, w, s);
}

}  // namespace mdn
