// k_augment.cu -- training-set augmentation by the 8 dihedral transforms of
// the pairs (Section 5: flips and 90-degree rotations), applied to the
// accumulated per-bucket Gram sums.  A transform of the image permutes the
// taps of every patch and moves the orientation bin of every pixel (the
// structure tensor turns with the image), so the augmented sums are permuted
// copies of the original ones; no patch is gathered again.
#include <cuda_fp16.h>

#include "internal.h"
#include "train_common.cuh"

namespace mdn {
namespace aug {

// Tap of the original patch that transform t puts at row i, column j of the
// transformed (n x n) patch: undo the mirror (columns), then undo the 90-degree
// rotations (a rotated patch holds at (i, j) the entry (j, n-1-i) of the patch
// before the rotation).
__device__ __forceinline__ int tap_source(int tap, int n, int t) {
    int i = tap / n, j = tap % n;
    if (t >= 4) j = n - 1 - j;
    for (int r = 0; r < (t & 3); ++r) {
        const int ni = j, nj = n - 1 - i;
        i = ni;
        j = nj;
    }
    return i * n + j;
}

// Feature of the original regressor that transform t puts at feature f
// (fine taps only: cross-channel features are channel-major (c, tap); the
// targets after the D regressor entries are unchanged).
__device__ __forceinline__ int feature_source(int f, int D, int n, int cross, int t) {
    if (f >= D) return f;
    const int nn = n * n;
    if (cross) return (f / nn) * nn + tap_source(f % nn, n, t);
    return tap_source(f, n, t);
}

// Bucket whose pixels transform t sends to bucket kp.
__device__ __forceinline__ int bucket_source(int kp, int n_angle, int m, int t) {
    const int ap = kp / m, rest = kp % m;
    int a = t >= 4 ? n_angle - 1 - ap : ap;
    a = ((a - (t & 3) * (n_angle / 2)) % n_angle + n_angle) % n_angle;
    return a * m + rest;
}

// One thread per output entry (k', g, i, j); the 8 transforms are summed in a
// fixed order (deterministic).
__global__ void k_dihedral(const double* __restrict__ gin, const int64_t* __restrict__ cin, int K, int G, int Dp,
                           int D, int n, int cross, int n_angle, int m, double* __restrict__ gout,
                           int64_t* __restrict__ cout) {
    const int64_t per = (int64_t)G * Dp * Dp;
    const int64_t total = (int64_t)K * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int kp = (int)(e / per);
        const int64_t r = e % per;
        const int g = (int)(r / ((int64_t)Dp * Dp));
        const int i = (int)((r / Dp) % Dp), j = (int)(r % Dp);
        double acc = 0.0;
        for (int t = 0; t < 8; ++t) {
            const int k = bucket_source(kp, n_angle, m, t);
            const int si = feature_source(i, D, n, cross, t), sj = feature_source(j, D, n, cross, t);
            acc += gin[(int64_t)k * per + ((int64_t)g * Dp + si) * Dp + sj];
        }
        gout[e] = acc;
        if (r == 0) {
            int64_t c = 0;
            for (int t = 0; t < 8; ++t) c += cin[bucket_source(kp, n_angle, m, t)];
            cout[kp] = c;
        }
    }
}

// Image form of transform t (for multiscale training, whose pyramids do not
// commute with the mirror): out = mirror_columns_if(t >= 4)(rot90^(t mod 4)(in))
// per channel, where rot90 of an (h x w) image is the (w x h) image r with
// r[i][j] = in[j][w - 1 - i].  One thread per output value.
template <typename TS>
__global__ void k_dihedral_img(const TS* __restrict__ in, TS* __restrict__ out, int64_t n, int h, int w, int t) {
    const bool swap = (t & 1) != 0;
    const int ho = swap ? w : h, wo = swap ? h : w;
    const int64_t plane = (int64_t)ho * wo;
    const int64_t total = n * 3 * plane;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ch = e / plane, q = e % plane;
        int i = (int)(q / wo), j = (int)(q % wo);
        int cw = wo, chh = ho;   // shape of the image the coordinates refer to
        if (t >= 4) j = cw - 1 - j;
        for (int r = 0; r < (t & 3); ++r) {
            // (i, j) in a rotated image of shape (chh, cw) comes from (j, chh - 1 - i) of shape (cw, chh)
            const int ni = j, nj = chh - 1 - i;
            i = ni;
            j = nj;
            const int tmp = cw;
            cw = chh;
            chh = tmp;
        }
        out[e] = in[ch * (int64_t)h * w + (int64_t)i * w + j];
    }
}

}  // namespace aug
}  // namespace mdn

using namespace mdn;

extern "C" int mdn_augment_dihedral(const double* gram_in, const int64_t* counts_in, const mdn_geometry* geom,
                                    const mdn_bucket_params* bp, double* gram_out, int64_t* counts_out,
                                    void* stream) {
    NvtxRange nvtx_range("mdn_augment_dihedral");
    if (!gram_in || !counts_in || !geom || !bp || !gram_out || !counts_out)
        return fail(MDN_EINVAL, "augment_dihedral: null argument");
    if (gram_out == gram_in || counts_out == counts_in)
        return fail(MDN_EINVAL, "augment_dihedral: outputs must not alias the inputs");
    if (geom->r_coarse >= 0)
        return fail(MDN_ESHAPE, "augment_dihedral: single-level geometry only (r_coarse < 0)");
    if (geom->r_fine < 0 || geom->r_fine > 8) return fail(MDN_ESHAPE, "augment_dihedral: r_fine must be 0..8");
    if (bp->n_angle < 2 || bp->n_angle % 2 || bp->n_strength < 1 || bp->n_coherence < 1)
        return fail(MDN_EINVAL, "augment_dihedral: n_angle must be even and the grid non-empty");
    const int K = bp->n_angle * bp->n_strength * bp->n_coherence;
    if (K > MDN_MAX_K) return fail(MDN_EINVAL, "augment_dihedral: more than 4096 buckets");
    const int D = regressor_len(*geom);
    const int G = geom->cross_channel ? 1 : 3, T = geom->cross_channel ? 3 : 1, Dp = D + T;
    const int64_t total = (int64_t)K * G * Dp * Dp;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
    aug::k_dihedral<<<grid, 256, 0, (cudaStream_t)stream>>>(gram_in, counts_in, K, G, Dp, D, 2 * geom->r_fine + 1,
                                                             geom->cross_channel, bp->n_angle,
                                                             bp->n_strength * bp->n_coherence, gram_out, counts_out);
    return check_launch("k_dihedral");
}

extern "C" int mdn_dihedral_images(const void* in, int32_t dtype, int64_t n, int64_t h, int64_t w, int32_t t, void* out,
                                   void* stream) {
    NvtxRange nvtx_range("mdn_dihedral_images");
    if (!in || !out) return fail(MDN_EINVAL, "dihedral_images: null pointer");
    if (in == out) return fail(MDN_EINVAL, "dihedral_images: out must not alias in");
    if (dtype != MDN_F32 && dtype != MDN_F16) return fail(MDN_EINVAL, "dihedral_images: dtype must be F32 or F16");
    if (t < 0 || t > 7) return fail(MDN_EINVAL, "dihedral_images: t must be 0..7");
    if (n < 0 || h < 1 || w < 1 || h > (1 << 20) || w > (1 << 20)) return fail(MDN_ESHAPE, "dihedral_images: bad shape");
    const int64_t total = n * 3 * h * w;
    if (total == 0) return MDN_OK;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == MDN_F32)
        aug::k_dihedral_img<float><<<grid, 256, 0, s>>>((const float*)in, (float*)out, n, (int)h, (int)w, t);
    else
        aug::k_dihedral_img<__half><<<grid, 256, 0, s>>>((const __half*)in, (__half*)out, n, (int)h, (int)w, t);
    return check_launch("k_dihedral_img");
}
