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
constexpr int GRAM_MAX_CTAS = 160;  // tensor-core Gram: at most one CTA per SM, row quantum per CTA
constexpr int GRAM_MIN_QUANTUM = 1024;
// Fixed cost of one tensor-core chunk (accumulator drain and read-back) in
// rows of gather work, used to balance the CTAs' shares of a pixel group.
constexpr int GRAM_RUN_COST = 128;
constexpr int GRAM_MAX_GROUPS = 64;  // pixel groups processed one after the other (L2-sized working set)
constexpr double GRAM_GROUP_BYTES = 40e6;   // target working-plane bytes of one pixel group
// Above 256 buckets every group has about K chunks, each with a fixed cost and
// an FP32 partial: larger groups (fewer chunks) win until the planes leave L2
// (16 x 1 MP, 4096 buckets, 7x7 + 5x5: 40 MB 22.0 ms, 100 MB 18.5, 250 MB 21.5).
constexpr double GRAM_GROUP_BYTES_WIDE = 100e6;

// Pixel groups of the Gram accumulation: the tensor-core path walks the
// sorted rows group by group (pixel-index ranges of GB pixels, GB a multiple
// of SORT_CHUNK) so that the working planes it gathers from stay in L2; the
// SIMT path uses one group.  cap = chunk-table entries per group.
struct GramGroups {
    int64_t GB;
    int ngroups, cap;
};
inline GramGroups gram_groups(int64_t n, int64_t h, int64_t w, int P, bool coarse, int K, bool tensor) {
    GramGroups q;
    const int64_t npix = n * h * w;
    if (!tensor || npix == 0) {
        q.GB = npix > 0 ? (npix + SORT_CHUNK - 1) / SORT_CHUNK * SORT_CHUNK : SORT_CHUNK;
        q.ngroups = 1;
        q.cap = (int)(npix / GRAM_CHUNK + K + 1);
        return q;
    }
    const double hw = (double)h * w, hc = (double)((h + 1) / 2), wc = (double)((w + 1) / 2);
    const double bpp = 12.0 * ((h + 2.0 * P) * (w + 2.0 * P) / hw + 1.0 + (coarse ? (hc + 2 * P) * (wc + 2 * P) / hw : 0.0));
    int64_t gb = (int64_t)((K > 256 ? GRAM_GROUP_BYTES_WIDE : GRAM_GROUP_BYTES) / bpp) / SORT_CHUNK * SORT_CHUNK;
    if (gb < SORT_CHUNK) gb = SORT_CHUNK;
    if ((npix + gb - 1) / gb > GRAM_MAX_GROUPS) gb = ((npix + GRAM_MAX_GROUPS - 1) / GRAM_MAX_GROUPS + SORT_CHUNK - 1) / SORT_CHUNK * SORT_CHUNK;
    q.GB = gb;
    q.ngroups = (int)((npix + gb - 1) / gb);
    q.cap = GRAM_MAX_CTAS + K + 1;
    return q;
}

// Working channel of Gram feature i (regressor tap or target) of group g:
// per-channel geometry uses channel g throughout; cross-channel features are
// ordered coarse (c, dy, dx), fine (c, dy, dx), then the three targets.
__host__ __device__ inline int feature_channel(int i, int g, int D, int rf, int rc, int cross) {
    if (!cross) return g;
    const int pc = rc >= 0 ? (2 * rc + 1) * (2 * rc + 1) : 0, pf = (2 * rf + 1) * (2 * rf + 1);
    if (i < 3 * pc) return i / pc;
    if (i < D) return (i - 3 * pc) / pf;
    return i - D;
}

// Centring constant of a working channel: luma (or any RGB channel) lies in
// [0, 1] and is shifted by 0.5, chroma is already centred.
__host__ __device__ inline double channel_center(int c, int color) {
    return (color == MDN_RGB || c == 0) ? 0.5 : 0.0;
}

// The working planes hold each value already shifted by its channel's centring
// constant (and, for the TF32 Gram, already rounded to TF32; for the BF16 Gram
// they hold 16-bit BF16 values, the operands themselves).  The regressor
// planes are stored with a replicated border of P = max(rf, rc) pixels, so
// that every tap of every pixel is an in-range load and clamping to the image
// (the border rule of the filter) needs no per-tap test.
struct GatherArgs {
    const float* zw;   // [n][3][Hp][Wp] working space, level l, border P replicated
    const float* tw;   // [n][3][h][w] working space, clean level l (centre taps only, no border)
    const float* cw;   // [n][3][Hcp][Wcp] working space, coarse output, border P replicated, or nullptr
    int h, w, hc, wc;
    int n;                     // images
    int P, Hp, Wp, Hcp, Wcp;   // Hp = h + 2P, Wp = w + 2P, Hcp = hc + 2P, Wcp = wc + 2P
    int rf, rc, cross, color;
    int D, T, G, Dp, Dp4;   // Dp4: SIMT row stride, >= Dp + 1, multiple of 4
};

// Column codes of the SIMT Gram rows: src (0 coarse, 1 fine, 2 target,
// 3 ones) | c << 2 | (dy + 8) << 4 | (dx + 8) << 9.  Rows have Dq = Dp + 1
// columns: the regressor taps and targets, shifted by the channel's centring
// constant, then a ones column (see k_reduce_sum and k_center).
__device__ __forceinline__ void build_coltab(const GatherArgs& ga, int* coltab) {
    const int Dq = ga.Dp + 1;
    for (int e = threadIdx.x; e < ga.G * Dq; e += blockDim.x) {
        int g = e / Dq, j = e % Dq;
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
        } else if (j < ga.Dp) {
            int c = ga.cross ? j - ga.D : g;
            code = 2 | (c << 2) | (8 << 4) | (8 << 9);
        } else {
            code = 3;
        }
        coltab[e] = code;
    }
}

__device__ __forceinline__ float gather_value(const GatherArgs& ga, int code, int pix) {
    const int src = code & 3, c = (code >> 2) & 3;
    if (src == 3) return 1.f;
    const int hw = ga.h * ga.w;
    const int img = pix / hw, rem = pix % hw;
    const int y = rem / ga.w, x = rem % ga.w;
    const int dy = ((code >> 4) & 31) - 8, dx = ((code >> 9) & 31) - 8;
    if (src == 1) {
        const int yy = y + ga.P + dy, xx = x + ga.P + dx;
        return __ldg(ga.zw + ((int64_t)img * 3 + c) * ga.Hp * ga.Wp + (int64_t)yy * ga.Wp + xx);
    } else if (src == 0) {
        const int yy = y / 2 + ga.P + dy, xx = x / 2 + ga.P + dx;
        return __ldg(ga.cw + ((int64_t)img * 3 + c) * ga.Hcp * ga.Wcp + (int64_t)yy * ga.Wcp + xx);
    }
    return __ldg(ga.tw + ((int64_t)img * 3 + c) * hw + rem);
}

// As[g][r][j] for r < nr (rows >= nr and columns >= Dq are zeroed), row
// stride DPs floats, RB rows per group.
__device__ __forceinline__ void gather_rows(const GatherArgs& ga, const int* coltab, const int* rows, int nr,
                                            float* As, int DPs, int RB) {
    const int per_g = RB * DPs, Dq = ga.Dp + 1;
    for (int e = threadIdx.x; e < ga.G * per_g; e += blockDim.x) {
        int g = e / per_g, r = (e / DPs) % RB, j = e % DPs;
        float v = 0.f;
        if (r < nr && j < Dq) v = gather_value(ga, coltab[g * Dq + j], rows[r]);
        As[e] = v;
    }
}

// Border width of the working planes and the padded extents.
inline int gram_border(const mdn_geometry& g) { return g.r_coarse > g.r_fine ? g.r_coarse : g.r_fine; }

int gram_tc_error(int* out);
void gram_tc_set_wait(unsigned long long ns);
void gram_tc_expire_next(int enable);
// Tensor-core Gram over the per-group chunk tables: CTA b accumulates, group
// after group, the chunks whose owner field (w) is b; ncta CTAs.
int launch_gram_tc(const GatherArgs& ga, int precision, const int4* chunks, const int* gcount, int ngroups, int cap,
                   const int* sorted, float* partial, int ncta, cudaStream_t s);

}  // namespace mdn
