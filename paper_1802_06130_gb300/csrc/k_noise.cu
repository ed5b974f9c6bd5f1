// k_noise.cu -- noise-level estimate of an input image, to choose the bank set
// trained for the nearest noise level (the paper assumes the level is known
// and names estimating it as the way to select the filter set, Section 6).
// Estimator (Donoho and Johnstone's robust wavelet estimate): the finest
// diagonal Haar detail d = (a - b - c + e) / 2 of each 2x2 block
// [a b; c e] of every channel has variance sigma^2 under i.i.d. Gaussian noise
// and is small on smooth image content, so sigma = median(|d|) / 0.6745
// (0.6745 = the median of |N(0, 1)|).  The median is taken from a histogram
// of NOISE_BINS bins over [0, NOISE_MAX) with linear interpolation inside the
// median bin (within half a bin, NOISE_MAX / NOISE_BINS / 2, of the exact median).
#include "common.cuh"
#include "internal.h"

namespace mdn {
namespace noise {

constexpr int NOISE_BINS = 16384;
constexpr float NOISE_MAX = 0.5f;   // |d| at or above this counts in the last bin
constexpr int TB = 256;

template <typename TS>
__global__ void __launch_bounds__(TB) k_noise_hist(const TS* __restrict__ img, int64_t h, int64_t w,
                                                   unsigned* __restrict__ hist) {
    extern __shared__ unsigned sh[];
    for (int i = threadIdx.x; i < NOISE_BINS; i += TB) sh[i] = 0;
    __syncthreads();
    const int64_t bh = h / 2, bw = w / 2, nb = bh * bw;
    const TS* im = img + (int64_t)blockIdx.y * 3 * h * w;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < 3 * nb; e += (int64_t)gridDim.x * TB) {
        const int c = (int)(e / nb);
        const int64_t q = e % nb;
        const int64_t y = 2 * (q / bw), x = 2 * (q % bw);
        const TS* p = im + (int64_t)c * h * w + y * w + x;
        const float a = ld_f(p, 0), b = ld_f(p, 1), cc = ld_f(p, w), d = ld_f(p, w + 1);
        const float v = fabsf(0.5f * ((a - b) - (cc - d)));
        int bin = (int)(v * (NOISE_BINS / NOISE_MAX));
        bin = bin < NOISE_BINS ? bin : NOISE_BINS - 1;
        atomicAdd(&sh[bin], 1u);
    }
    __syncthreads();
    unsigned* hg = hist + (int64_t)blockIdx.y * NOISE_BINS;
    for (int i = threadIdx.x; i < NOISE_BINS; i += TB)
        if (sh[i]) atomicAdd(&hg[i], sh[i]);
}

// One CTA per image: prefix sums over the histogram, the bin holding the
// median, linear interpolation inside it.
__global__ void __launch_bounds__(1024) k_noise_median(const unsigned* __restrict__ hist, int64_t count,
                                                        float* __restrict__ sigma) {
    constexpr int PER = NOISE_BINS / 1024;
    __shared__ unsigned long long part[1024];
    const unsigned* hg = hist + (int64_t)blockIdx.x * NOISE_BINS;
    const int t = threadIdx.x;
    unsigned long long s = 0;
    for (int i = 0; i < PER; ++i) s += hg[t * PER + i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // inclusive scan
        const unsigned long long add = t >= d ? part[t - d] : 0ull;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    // median position: the (count - 1) / 2-th value (0-based), i.e. the lower
    // median; the bin where the cumulative count first exceeds it
    const double target = 0.5 * (double)count;
    const unsigned long long before = t > 0 ? part[t - 1] : 0ull;
    if ((double)before < target && (double)part[t] >= target) {
        unsigned long long cum = before;
        for (int i = 0; i < PER; ++i) {
            const unsigned cnt = hg[t * PER + i];
            if ((double)(cum + cnt) >= target) {
                const double frac = cnt ? (target - (double)cum) / (double)cnt : 0.5;
                const double med = ((double)(t * PER + i) + frac) * (double)NOISE_MAX / NOISE_BINS;
                sigma[blockIdx.x] = (float)(med / 0.6744897501960817);
                break;
            }
            cum += cnt;
        }
    }
}

}  // namespace noise
}  // namespace mdn

using namespace mdn;

extern "C" size_t mdn_noise_workspace_bytes(int64_t n) {
    return n > 0 ? (size_t)n * noise::NOISE_BINS * sizeof(unsigned) : 0;
}

extern "C" int mdn_estimate_noise(const void* img, int32_t dtype, int64_t n, int64_t h, int64_t w, float* sigma_out,
                                  void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("mdn_estimate_noise");
    if (!img || !sigma_out || (n > 0 && !ws)) return fail(MDN_EINVAL, "estimate_noise: null pointer");
    if (dtype != MDN_F32 && dtype != MDN_F16) return fail(MDN_EINVAL, "estimate_noise: dtype must be F32 or F16");
    if (n < 0 || n > 65535 || h < 2 || w < 2 || h > (1 << 20) || w > (1 << 20))
        return fail(MDN_ESHAPE, "estimate_noise: need 0 <= n <= 65535 and h, w in 2 .. 2^20");
    if (ws_bytes < mdn_noise_workspace_bytes(n)) return fail(MDN_EWORKSPACE, "estimate_noise: workspace too small");
    if (n == 0) return MDN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(ws, 0, mdn_noise_workspace_bytes(n), s);
    if (e != cudaSuccess) return cuda_fail(e, "estimate_noise: clear");
    const int64_t work = 3 * (h / 2) * (w / 2);
    unsigned gx = (unsigned)std::min<int64_t>((work + noise::TB * 8 - 1) / (noise::TB * 8), 304);
    const size_t smem = noise::NOISE_BINS * sizeof(unsigned);
    dim3 grid(gx, (unsigned)n);
    if (dtype == MDN_F32) {
        e = cudaFuncSetAttribute(noise::k_noise_hist<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            noise::k_noise_hist<float><<<grid, noise::TB, smem, s>>>((const float*)img, h, w, (unsigned*)ws);
    } else {
        e = cudaFuncSetAttribute(noise::k_noise_hist<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            noise::k_noise_hist<__half><<<grid, noise::TB, smem, s>>>((const __half*)img, h, w, (unsigned*)ws);
    }
    if (e != cudaSuccess) return cuda_fail(e, "estimate_noise: smem attribute");
    noise::k_noise_median<<<(unsigned)n, 1024, 0, s>>>((const unsigned*)ws, work, sigma_out);
    return check_launch("k_noise");
}
