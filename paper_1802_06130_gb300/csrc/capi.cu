// capi.cu -- the extern "C" entry points of libmdn (include/mdn.h):
// argument validation, parameter marshalling and launch sequencing.  Every
// arithmetic step of the method runs in the kernels of the other
// translation units.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"
#include "train_common.cuh"

namespace mdn {

#ifdef MDN_CHECK
__device__ unsigned long long g_mdn_check;   // first bounds violation (see common.cuh)
#endif

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return MDN_ECUDA;
}
int check_launch(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, where);
    return MDN_OK;
}

int num_sms() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        cached_dev = dev;
    }
    return cached > 0 ? cached : 1;
}

void gauss5_weights(float w[5]) {
    double d[5], s = 0.0;
    for (int u = -2; u <= 2; ++u) {
        d[u + 2] = std::exp(-(double)(u * u) / (2.0 * 1.5 * 1.5));
        s += d[u + 2];
    }
    for (int u = 0; u < 5; ++u) w[u] = (float)(d[u] / s);
}

int make_sel_params(const mdn_bucket_params* bp, SelParams* sp) {
    if (!bp) return fail(MDN_EINVAL, "bucket params: null");
    if (bp->n_angle < 2 || bp->n_angle > 64 || (bp->n_angle & 1))
        return fail(MDN_EINVAL, "bucket params: n_angle must be even, 2..64");
    if (bp->n_strength < 1 || bp->n_strength > MDN_MAX_THR + 1 || bp->n_coherence < 1 ||
        bp->n_coherence > MDN_MAX_THR + 1)
        return fail(MDN_EINVAL, "bucket params: n_strength/n_coherence out of range 1..17");
    int K = bp->n_angle * bp->n_strength * bp->n_coherence;
    if (K > MDN_MAX_K) return fail(MDN_EINVAL, "bucket params: more than 4096 buckets");
    std::memset(sp, 0, sizeof(*sp));
    sp->n_angle = bp->n_angle;
    sp->n_strength = bp->n_strength;
    sp->n_coherence = bp->n_coherence;
    sp->nthr_s = bp->n_strength - 1;
    sp->nthr_c = bp->n_coherence - 1;
    for (int i = 0; i < sp->nthr_s; ++i) sp->strength_thr[i] = bp->strength_thr[i];
    for (int i = 0; i < sp->nthr_c; ++i) sp->coherence_thr[i] = bp->coherence_thr[i];
    sp->coh_eps = bp->coh_eps;
    for (int i = 0; i < sp->nthr_s; ++i) sp->strength_q[i] = (float)((double)bp->strength_thr[i] * bp->strength_thr[i]);
    for (int i = 0; i < sp->nthr_c; ++i) {
        const double C = (double)bp->coherence_thr[i];
        sp->coherence_r[i] = C < 1.0 ? (float)(2.0 * C / (1.0 + C * C)) : (C == 1.0 ? 1.0f : INFINITY);
    }
    sp->eps2 = (float)((double)bp->coh_eps * bp->coh_eps);
    const double PI = 3.14159265358979323846;
    for (int k = 1; k < bp->n_angle / 2; ++k) {
        double a = 2.0 * PI * k / bp->n_angle;
        sp->bcos[k - 1] = (float)std::cos(a);
        sp->bsin[k - 1] = (float)std::sin(a);
    }
    return MDN_OK;
}

static int check_geom(const mdn_geometry* g) {
    if (!g) return fail(MDN_EINVAL, "geometry: null");
    if (g->r_fine < 1 || g->r_fine > 3) return fail(MDN_ESHAPE, "geometry: r_fine must be 1..3");
    if (g->r_coarse < -1 || g->r_coarse > 3) return fail(MDN_ESHAPE, "geometry: r_coarse must be -1..3");
    if (g->color != MDN_YCBCR601 && g->color != MDN_RGB) return fail(MDN_EINVAL, "geometry: bad color");
    return MDN_OK;
}

bool dims_ok(int64_t n, int64_t h, int64_t w) {
    // each factor is bounded before any product is formed: h, w <= 2^20 keeps
    // 3*h*w below 2^63, and n is then bounded by division
    if (n < 0 || h < 0 || w < 0 || h > (int64_t(1) << 20) || w > (int64_t(1) << 20)) return false;
    const int64_t per = 3 * h * w;
    return per == 0 || n <= ((int64_t(1) << 31) - 1) / per;
}

int check_img(const void* p, int dtype, int64_t n, int64_t h, int64_t w, const char* what) {
    if (dtype != MDN_F32 && dtype != MDN_F16) return fail(MDN_EINVAL, std::string(what) + ": bad dtype");
    if (n < 0 || h < 0 || w < 0) return fail(MDN_ESHAPE, std::string(what) + ": negative size");
    if (!dims_ok(n, h, w))
        return fail(MDN_ESHAPE, std::string(what) + ": image too large (h, w <= 2^20 and n*3*h*w < 2^31)");
    if (!p && n * h * w > 0) return fail(MDN_EINVAL, std::string(what) + ": null pointer");
    return MDN_OK;
}

static size_t esize(int dtype) { return dtype == MDN_F16 ? 2 : 4; }

// bank dtype code -> element type and layout (plain [K][3][D] or prepared row slots)
static int bank_kind(int32_t bank_dtype, int* elem, bool* rows, const char* what) {
    switch (bank_dtype) {
        case MDN_F32: *elem = MDN_F32; *rows = false; return MDN_OK;
        case MDN_F16: *elem = MDN_F16; *rows = false; return MDN_OK;
        case MDN_F32_ROWS: *elem = MDN_F32; *rows = true; return MDN_OK;
        case MDN_F16_ROWS: *elem = MDN_F16; *rows = true; return MDN_OK;
        default: return fail(MDN_EINVAL, std::string(what) + ": bad bank dtype");
    }
}

int launch_level_f32_f32(const LevelArgs& a, cudaStream_t s);
int launch_level_f32_f16(const LevelArgs& a, cudaStream_t s);
int launch_level_f16_f32(const LevelArgs& a, cudaStream_t s);
int launch_level_f16_f16(const LevelArgs& a, cudaStream_t s);
int launch_select_f32(const LevelArgs& a, cudaStream_t s);
int launch_select_f16(const LevelArgs& a, cudaStream_t s);

int launch_level(const LevelArgs& a, cudaStream_t s) {
    if (a.n == 0 || a.h == 0 || a.w == 0) return MDN_OK;
    if (!a.out) return a.dtype == MDN_F32 ? launch_select_f32(a, s) : launch_select_f16(a, s);
    if (a.dtype == MDN_F32)
        return a.bank_dtype == MDN_F32 ? launch_level_f32_f32(a, s) : launch_level_f32_f16(a, s);
    return a.bank_dtype == MDN_F32 ? launch_level_f16_f32(a, s) : launch_level_f16_f16(a, s);
}

}  // namespace mdn

using namespace mdn;

extern "C" {

int mdn_version(void) { return 10000; }

const char* mdn_last_error(void) { return g_last_error.c_str(); }

int mdn_regressor_len(const mdn_geometry* geom) {
    if (!geom || geom->r_fine < 0 || geom->r_fine > 3 || geom->r_coarse < -1 || geom->r_coarse > 3) return -1;
    return regressor_len(*geom);
}

int mdn_bucket_elem_bytes(int32_t K) { return K < 1 || K > MDN_MAX_K ? 0 : bucket_bytes(K); }

size_t mdn_pyramid_bytes(int64_t n, int64_t h, int64_t w, int32_t levels, int32_t dtype) {
    if (!dims_ok(n, h, w) || levels > 8) return SIZE_MAX;   // no size is large enough: calls will be rejected
    size_t tot = 0;
    for (int l = 1; l < levels; ++l) {
        h = (h + 1) / 2;
        w = (w + 1) / 2;
        tot += align256((size_t)n * 3 * h * w * esize(dtype));
    }
    return tot;
}

int mdn_build_pyramid(const void* img, int32_t dtype, int64_t n, int64_t h, int64_t w, int32_t levels,
                      void* const* out_levels, void* stream) {
    NvtxRange nvtx_range("mdn_build_pyramid");
    int rc = check_img(img, dtype, n, h, w, "build_pyramid");
    if (rc) return rc;
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "build_pyramid: levels must be 1..8");
    if (levels > 1 && !out_levels) return fail(MDN_EINVAL, "build_pyramid: out_levels null");
    for (int l = 1; l < levels; ++l)
        if (!out_levels[l - 1]) return fail(MDN_EINVAL, "build_pyramid: null level pointer");
    if (n == 0 || h == 0 || w == 0) return MDN_OK;
    const void* src = img;
    for (int l = 1; l < levels; ++l) {
        rc = launch_pyramid_down(src, out_levels[l - 1], dtype, n, h, w, (cudaStream_t)stream);
        if (rc) return rc;
        src = out_levels[l - 1];
        h = (h + 1) / 2;
        w = (w + 1) / 2;
    }
    return MDN_OK;
}

int mdn_select_buckets(const void* z, int32_t dtype, int64_t n, int64_t h, int64_t w,
                       const mdn_bucket_params* bp, void* buckets, void* stream) {
    NvtxRange nvtx_range("mdn_select_buckets");
    int rc = check_img(z, dtype, n, h, w, "select_buckets");
    if (rc) return rc;
    if (!buckets) return fail(MDN_EINVAL, "select_buckets: null output");
    LevelArgs a{};
    rc = make_sel_params(bp, &a.sel);
    if (rc) return rc;
    a.z = z; a.out = nullptr; a.buckets = buckets; a.n = n; a.h = h; a.w = w;
    a.dtype = dtype; a.K = bp->n_angle * bp->n_strength * bp->n_coherence;
    a.geom = mdn_geometry{3, -1, 0, MDN_YCBCR601};
    return launch_level(a, (cudaStream_t)stream);
}

int mdn_filter_level(const void* z, const void* coarse, int32_t dtype, int64_t n, int64_t h, int64_t w,
                     const void* bank, int32_t bank_dtype, const mdn_geometry* geom,
                     const mdn_bucket_params* bp, void* out, void* buckets_out, void* stream) {
    NvtxRange nvtx_range("mdn_filter_level");
    int rc = check_img(z, dtype, n, h, w, "filter_level");
    if (rc) return rc;
    if ((rc = check_geom(geom))) return rc;
    if (!out) return fail(MDN_EINVAL, "filter_level: null output");
    if (!bank) return fail(MDN_EINVAL, "filter_level: null bank");
    int bank_elem = 0;
    bool bank_rows = false;
    if ((rc = bank_kind(bank_dtype, &bank_elem, &bank_rows, "filter_level"))) return rc;
    if (geom->r_coarse >= 0 && !coarse) return fail(MDN_EINVAL, "filter_level: coarse level required");
    if (out == z || (coarse && out == coarse)) return fail(MDN_EINVAL, "filter_level: out aliases an input");
    LevelArgs a{};
    if ((rc = make_sel_params(bp, &a.sel))) return rc;
    a.z = z; a.coarse = geom->r_coarse >= 0 ? coarse : nullptr; a.out = out; a.buckets = buckets_out;
    a.bank = bank; a.n = n; a.h = h; a.w = w; a.hc = (h + 1) / 2; a.wc = (w + 1) / 2;
    a.dtype = dtype; a.bank_dtype = bank_elem; a.bank_rows = bank_rows; a.variant = g_force_variant;
    a.K = bp->n_angle * bp->n_strength * bp->n_coherence;
    a.geom = *geom;
    return launch_level(a, (cudaStream_t)stream);
}

size_t mdn_denoise_workspace_bytes(int64_t n, int64_t h, int64_t w, int32_t levels, int32_t dtype) {
    // pyramid levels 1..L-1 plus outputs u^1..u^{L-2}
    if (!dims_ok(n, h, w) || levels > 8) return SIZE_MAX;
    size_t tot = mdn_pyramid_bytes(n, h, w, levels, dtype);
    int64_t hh = h, ww = w;
    for (int l = 1; l <= levels - 2; ++l) {
        hh = (hh + 1) / 2;
        ww = (ww + 1) / 2;
        tot += align256((size_t)n * 3 * hh * ww * esize(dtype));
    }
    return tot;
}

int mdn_denoise_multiscale(const void* noisy, int32_t dtype, int64_t n, int64_t h, int64_t w, int32_t levels,
                           const void* const* banks, int32_t bank_dtype, const mdn_geometry* geom,
                           const mdn_bucket_params* bparams, void* out, void* const* bucket_maps, void* ws,
                           size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("mdn_denoise_multiscale");
    int rc = check_img(noisy, dtype, n, h, w, "denoise_multiscale");
    if (rc) return rc;
    if ((rc = check_geom(geom))) return rc;
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "denoise_multiscale: levels must be 1..8");
    if ((levels == 1) != (geom->r_coarse < 0))
        return fail(MDN_ESHAPE, "denoise_multiscale: levels = 1 needs r_coarse = -1 and levels > 1 needs r_coarse >= 0");
    if (!banks || !bparams || (!out && n * h * w > 0))
        return fail(MDN_EINVAL, "denoise_multiscale: null banks/bparams/out");
    if (out == noisy && n * h * w > 0) return fail(MDN_EINVAL, "denoise_multiscale: out aliases the input");
    int bank_elem = 0;
    bool bank_rows = false;
    if ((rc = bank_kind(bank_dtype, &bank_elem, &bank_rows, "denoise_multiscale"))) return rc;
    const int nb = levels > 1 ? levels - 1 : 1;
    for (int l = 0; l < nb; ++l)
        if (!banks[l] && n * h * w > 0) return fail(MDN_EINVAL, "denoise_multiscale: null bank pointer");
    size_t need = mdn_denoise_workspace_bytes(n, h, w, levels, dtype);
    if (ws_bytes < need || (need && !ws)) return fail(MDN_EWORKSPACE, "denoise_multiscale: workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0 || h == 0 || w == 0) return MDN_OK;
    // carve workspace: z^1..z^{L-1}, then u^1..u^{L-2}
    const void* zl[9];
    void* ul[9];
    int64_t hl[9], wl[9];
    hl[0] = h; wl[0] = w; zl[0] = noisy;
    char* p = (char*)ws;
    for (int l = 1; l < levels; ++l) {
        hl[l] = (hl[l - 1] + 1) / 2;
        wl[l] = (wl[l - 1] + 1) / 2;
        zl[l] = p;
        p += align256((size_t)n * 3 * hl[l] * wl[l] * esize(dtype));
    }
    for (int l = 1; l <= levels - 2; ++l) {
        ul[l] = p;
        p += align256((size_t)n * 3 * hl[l] * wl[l] * esize(dtype));
    }
    ul[0] = out;
    {
        NvtxRange r("pyramid");
        for (int l = 1; l < levels; ++l) {
            rc = launch_pyramid_down(zl[l - 1], (void*)zl[l], dtype, n, hl[l - 1], wl[l - 1], s);
            if (rc) return rc;
        }
    }
    const void* coarse = levels > 1 ? zl[levels - 1] : nullptr;   // base case u^{L-1} = z^{L-1}
    for (int l = nb - 1; l >= 0; --l) {
        LevelArgs a{};
        if ((rc = make_sel_params(&bparams[l], &a.sel))) return rc;
        a.z = zl[l]; a.coarse = coarse; a.out = ul[l];
        a.buckets = bucket_maps ? bucket_maps[l] : nullptr;
        a.bank = banks[l]; a.n = n; a.h = hl[l]; a.w = wl[l]; a.hc = (hl[l] + 1) / 2; a.wc = (wl[l] + 1) / 2;
        a.dtype = dtype; a.bank_dtype = bank_elem; a.bank_rows = bank_rows; a.variant = g_force_variant; a.variant = g_force_variant;
        a.K = bparams[l].n_angle * bparams[l].n_strength * bparams[l].n_coherence;
        a.geom = *geom;
        NvtxRange r(l == 0 ? "level 0" : l == 1 ? "level 1" : l == 2 ? "level 2" : "level 3+");
        if ((rc = launch_level(a, s))) return rc;
        coarse = ul[l];
    }
    return MDN_OK;
}

size_t mdn_gram_state_bytes(const mdn_geometry* geom, int32_t K) {
    if (!geom) return 0;
    int D = regressor_len(*geom);
    int G = geom->cross_channel ? 1 : 3, T = geom->cross_channel ? 3 : 1;
    return (size_t)K * G * (D + T) * (D + T) * sizeof(double);
}

size_t mdn_train_workspace_bytes(int64_t n, int64_t h, int64_t w, const mdn_geometry* geom, int32_t K,
                                 int32_t gram_precision) {
    if (!geom) return 0;
    int D = regressor_len(*geom);
    int G = geom->cross_channel ? 1 : 3, T = geom->cross_channel ? 3 : 1;
    size_t solve = solve_ws_bytes(K, G, D, T);
    const int P = geom->r_coarse > geom->r_fine ? geom->r_coarse : geom->r_fine;
    size_t tr = align256((size_t)n * h * w * bucket_bytes(K)) +                 // bucket map
                train_ws_bytes(n, h, w, P, geom->r_coarse >= 0, K, G, D + T, gram_precision);  // working planes, sort, partials
    return tr > solve + 256 ? tr : solve + 256;
}

size_t mdn_solve_workspace_bytes(const mdn_geometry* geom, int32_t K) {
    if (!geom) return 0;
    int D = regressor_len(*geom);
    int G = geom->cross_channel ? 1 : 3, T = geom->cross_channel ? 3 : 1;
    return solve_ws_bytes(K, G, D, T);
}

int mdn_train_level_filters(const void* noisy_lvl, const void* coarse_out, const void* clean_lvl, int32_t dtype,
                            int64_t n, int64_t h, int64_t w, const mdn_geometry* geom,
                            const mdn_bucket_params* bp, int32_t gram_precision, int32_t accumulate,
                            double* gram, int64_t* counts, double lambda, float* bank_out, void* ws,
                            size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("mdn_train_level_filters");
    int rc = check_img(noisy_lvl, dtype, n, h, w, "train_level_filters");
    if (rc) return rc;
    if ((rc = check_img(clean_lvl, dtype, n, h, w, "train_level_filters (clean)"))) return rc;
    if ((rc = check_geom(geom))) return rc;
    if (geom->r_coarse >= 0 && !coarse_out) return fail(MDN_EINVAL, "train_level_filters: coarse level required");
    if (!gram || !counts) return fail(MDN_EINVAL, "train_level_filters: null gram/counts");
    if (gram_precision < MDN_GRAM_FP32 || gram_precision > MDN_GRAM_SPLIT_BF16)
        return fail(MDN_EINVAL, "train_level_filters: bad gram precision");
    if (!(lambda >= 0.0)) return fail(MDN_EINVAL, "train_level_filters: lambda must be >= 0");
    SelParams sp;
    if ((rc = make_sel_params(bp, &sp))) return rc;
    const int K = bp->n_angle * bp->n_strength * bp->n_coherence;
    size_t need = mdn_train_workspace_bytes(n, h, w, geom, K, gram_precision);
    if (ws_bytes < need || !ws) return fail(MDN_EWORKSPACE, "train_level_filters: workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    TrainArgs t{};
    t.z = noisy_lvl; t.coarse = geom->r_coarse >= 0 ? coarse_out : nullptr; t.target = clean_lvl;
    t.dtype = dtype; t.n = n; t.h = h; t.w = w; t.hc = (h + 1) / 2; t.wc = (w + 1) / 2;
    t.geom = *geom; t.K = K; t.D = regressor_len(*geom);
    t.G = geom->cross_channel ? 1 : 3; t.T = geom->cross_channel ? 3 : 1; t.Dp = t.D + t.T;
    t.precision = gram_precision; t.gram = gram; t.counts = counts;
    void* bmap = ws;
    t.buckets = bmap;
    const size_t bmap_bytes = align256((size_t)n * h * w * bucket_bytes(K));
    t.ws = (char*)ws + bmap_bytes;
    t.ws_bytes = ws_bytes - bmap_bytes;
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(gram, 0, mdn_gram_state_bytes(geom, K), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * K, s);
        if (e != cudaSuccess) return cuda_fail(e, "train_level_filters: clear");
    }
    if (n > 0 && h > 0 && w > 0) {
        LevelArgs a{};
        a.sel = sp; a.z = noisy_lvl; a.out = nullptr; a.buckets = bmap; a.n = n; a.h = h; a.w = w;
        a.dtype = dtype; a.K = K; a.geom = mdn_geometry{3, -1, 0, MDN_YCBCR601};
        {
            NvtxRange r("select");
            if ((rc = launch_level(a, s))) return rc;
        }
        NvtxRange r("gram");
        if ((rc = launch_gram(t, s))) return rc;
    }
    if (bank_out) {
        int32_t* status = (int32_t*)ws;   // reuse the start of the workspace
        rc = launch_solve(gram, counts, K, t.G, t.D, t.T, lambda, bank_out, status,
                          (char*)ws + 256, ws_bytes - 256, s);
        if (rc) return rc;
    }
    return MDN_OK;
}

int mdn_solve_bank(const double* gram, const int64_t* counts, const mdn_geometry* geom, int32_t K, double lambda,
                   float* bank_out, int32_t* status_out, void* ws, size_t ws_bytes, void* stream) {
    NvtxRange nvtx_range("mdn_solve_bank");
    int rc;
    if ((rc = check_geom(geom))) return rc;
    if (!gram || !counts || !bank_out || !status_out) return fail(MDN_EINVAL, "solve_bank: null pointer");
    if (K < 1 || K > MDN_MAX_K) return fail(MDN_EINVAL, "solve_bank: K must be 1..4096");
    if (!(lambda >= 0.0)) return fail(MDN_EINVAL, "solve_bank: lambda must be >= 0");
    int D = regressor_len(*geom);
    int G = geom->cross_channel ? 1 : 3, T = geom->cross_channel ? 3 : 1;
    if (ws_bytes < solve_ws_bytes(K, G, D, T) || !ws) return fail(MDN_EWORKSPACE, "solve_bank: workspace too small");
    return launch_solve(gram, counts, K, G, D, T, lambda, bank_out, status_out, ws, ws_bytes, (cudaStream_t)stream);
}

int mdn_check_status(int32_t* site, int64_t* index) {
    if (!site || !index) return fail(MDN_EINVAL, "check_status: null");
#ifdef MDN_CHECK
    unsigned long long v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_mdn_check, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_mdn_check, &zero, sizeof(zero));
    if (e != cudaSuccess) return cuda_fail(e, "check_status");
    if (v >> 63) {
        *site = (int32_t)((v >> 48) & 0x7fff);
        int64_t i = (int64_t)(v & 0xffffffffffffull);
        if (i & (int64_t(1) << 47)) i -= int64_t(1) << 48;   // sign of the recorded 48-bit index
        *index = i;
    } else {
        *site = 0;
        *index = 0;
    }
#else
    *site = -1;
    *index = 0;
#endif
    return MDN_OK;
}

int mdn_set_gram_wait_limit(uint64_t ns) {
    gram_tc_set_wait((unsigned long long)ns);
    return MDN_OK;
}

int mdn_gram_expire_next_wait(int32_t enable) {
    gram_tc_expire_next(enable);
    return MDN_OK;
}

double mdn_pyramid_noise_factor(int32_t level) {
    if (level < 0 || level > 7) return -1.0;
    // composed kernel of `level` binomial downsamplings, in input samples:
    // c_0 = delta, c_{l+1}[m] = sum_u b[u] c_l[m - 2^l u], b = [1 4 6 4 1] / 16
    static const double b[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    double c[1024] = {1.0}, nxt[1024];
    int len = 1;
    for (int l = 0; l < level; ++l) {
        const int step = 1 << l, nlen = len + 4 * step;
        for (int m = 0; m < nlen; ++m) nxt[m] = 0.0;
        for (int u = 0; u < 5; ++u)
            for (int m = 0; m < len; ++m) nxt[m + u * step] += b[u] * c[m];
        for (int m = 0; m < nlen; ++m) c[m] = nxt[m];
        len = nlen;
    }
    // separable 2-D kernel: the variance factor is (sum_m c[m]^2)^2, its root sum_m c[m]^2
    double ss = 0.0;
    for (int m = 0; m < len; ++m) ss += c[m] * c[m];
    return ss;
}

int32_t mdn_levels_for_sigma(double sigma, double coarsest_sigma, int32_t min_levels, int32_t max_levels) {
    if (!(sigma >= 0.0) || !(coarsest_sigma > 0.0) || min_levels < 1 || max_levels > 8 || min_levels > max_levels)
        return -1;
    int32_t L = 1;
    while (L < max_levels && sigma * mdn_pyramid_noise_factor(L - 1) >= coarsest_sigma) ++L;
    return L < min_levels ? min_levels : L;
}

int mdn_train_status(int32_t* flag) {
    if (!flag) return fail(MDN_EINVAL, "train_status: null");
    int v = 0;
    int rc = gram_tc_error(&v);
    if (rc) return rc;
    *flag = v;
    return MDN_OK;
}

}  // extern "C"
