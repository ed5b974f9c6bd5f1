// tensor.cu -- tensor-descriptor forms of the hot-path entry points
// (mdn_t_*): every argument is an mdn_tensor (dtype, rank, shape, strides in
// elements, device data), checked against the shapes the operation implies
// before the pointer form is called.  The kernels read dense row-major
// buffers, so the strides must be the dense ones; anything else (a view with
// a step, a transposed or broadcast tensor) is refused with MDN_ESHAPE,
// naming the argument, as is a wrong dtype, rank or extent.
#include <cstdio>
#include <string>

#include "internal.h"

namespace mdn {
namespace {

const char* dtype_name(int d) {
    switch (d) {
        case MDN_F32: return "f32";
        case MDN_F16: return "f16";
        case MDN_F16_ROWS: return "f16 row slots";
        case MDN_F32_ROWS: return "f32 row slots";
        case MDN_U8: return "u8";
        case MDN_U16: return "u16";
        case MDN_F64: return "f64";
        case MDN_I64: return "i64";
        default: return "unknown";
    }
}

// t must be a dense row-major tensor of dtype `dtype` (one of `dtype` or
// `alt` when alt >= 0) and exactly the given shape; -1 in shape: any extent.
int want(const mdn_tensor* t, const char* what, int dtype, int alt, int ndim, const int64_t* shape) {
    char msg[256];
    if (!t) {
        snprintf(msg, sizeof msg, "%s: null tensor", what);
        return fail(MDN_EINVAL, msg);
    }
    if (!t->data) {
        snprintf(msg, sizeof msg, "%s: null data", what);
        return fail(MDN_EINVAL, msg);
    }
    if (t->dtype != dtype && t->dtype != alt) {
        snprintf(msg, sizeof msg, "%s: dtype %s, expected %s%s%s", what, dtype_name(t->dtype), dtype_name(dtype),
                 alt >= 0 ? " or " : "", alt >= 0 ? dtype_name(alt) : "");
        return fail(MDN_ESHAPE, msg);
    }
    if (t->ndim != ndim) {
        snprintf(msg, sizeof msg, "%s: rank %d, expected %d", what, t->ndim, ndim);
        return fail(MDN_ESHAPE, msg);
    }
    int64_t dense = 1;
    for (int i = ndim - 1; i >= 0; --i) {
        if (t->shape[i] < 0 || (shape[i] >= 0 && t->shape[i] != shape[i])) {
            snprintf(msg, sizeof msg, "%s: extent %lld in dimension %d, expected %lld", what,
                     (long long)t->shape[i], i, (long long)shape[i]);
            return fail(MDN_ESHAPE, msg);
        }
        if (t->shape[i] > 1 && t->strides[i] != dense) {
            snprintf(msg, sizeof msg, "%s: stride %lld in dimension %d, the kernels need the dense %lld", what,
                     (long long)t->strides[i], i, (long long)dense);
            return fail(MDN_ESHAPE, msg);
        }
        dense *= t->shape[i] > 0 ? t->shape[i] : 1;
    }
    return MDN_OK;
}

// an image batch [N][3][H][W] of F32 or F16; its sizes are returned
int image(const mdn_tensor* t, const char* what, int64_t* n, int64_t* h, int64_t* w) {
    const int64_t any[4] = {-1, 3, -1, -1};
    if (int rc = want(t, what, MDN_F32, MDN_F16, 4, any)) return rc;
    *n = t->shape[0];
    *h = t->shape[2];
    *w = t->shape[3];
    return MDN_OK;
}

int same_image(const mdn_tensor* t, const char* what, int dtype, int64_t n, int64_t h, int64_t w) {
    const int64_t s[4] = {n, 3, h, w};
    return want(t, what, dtype, -1, 4, s);
}

int kcount(const mdn_bucket_params* bp) {
    return bp ? bp->n_angle * bp->n_strength * bp->n_coherence : 0;
}

// a bank for K buckets of geometry g: dense [K][3][D] F32 / F16, or the
// 1-D byte image of its prepared row slots (dtype MDN_F16_ROWS / _F32_ROWS)
int bank(const mdn_tensor* t, const char* what, const mdn_geometry* g, int K, int* code) {
    if (t && (t->dtype == MDN_F16_ROWS || t->dtype == MDN_F32_ROWS)) {
        const int64_t s[1] = {(int64_t)mdn_bank_rows_bytes(g, K, t->dtype == MDN_F16_ROWS ? MDN_F16 : MDN_F32)};
        if (int rc = want(t, what, t->dtype, -1, 1, s)) return rc;
        *code = t->dtype;
        return MDN_OK;
    }
    const int64_t s[3] = {K, 3, mdn_regressor_len(g)};
    if (int rc = want(t, what, MDN_F32, MDN_F16, 3, s)) return rc;
    *code = t->dtype;
    return MDN_OK;
}

// an optional bucket map [N][H][W], u8 for K <= 256, else u16
int bucket_map(const mdn_tensor* t, const char* what, int K, int64_t n, int64_t h, int64_t w) {
    const int64_t s[3] = {n, h, w};
    return want(t, what, K <= 256 ? MDN_U8 : MDN_U16, -1, 3, s);
}

}  // namespace
}  // namespace mdn

using namespace mdn;

extern "C" {

int mdn_t_build_pyramid(const mdn_tensor* img, int32_t levels, mdn_tensor* out, void* stream) {
    int64_t n, h, w;
    if (int rc = image(img, "build_pyramid: img", &n, &h, &w)) return rc;
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "build_pyramid: levels must be 1..8");
    if (levels > 1 && !out) return fail(MDN_EINVAL, "build_pyramid: null output array");
    void* ptrs[8] = {};
    int64_t hl = h, wl = w;
    for (int l = 1; l < levels; ++l) {
        hl = (hl + 1) / 2;
        wl = (wl + 1) / 2;
        char what[64];
        snprintf(what, sizeof what, "build_pyramid: out[%d]", l - 1);
        if (int rc = same_image(&out[l - 1], what, img->dtype, n, hl, wl)) return rc;
        ptrs[l - 1] = out[l - 1].data;
    }
    return mdn_build_pyramid(img->data, img->dtype, n, h, w, levels, ptrs, stream);
}

int mdn_t_filter_level(const mdn_tensor* z, const mdn_tensor* coarse, const mdn_tensor* bank_t,
                       const mdn_geometry* geom, const mdn_bucket_params* bp, mdn_tensor* out,
                       mdn_tensor* buckets_out, void* stream) {
    int64_t n, h, w;
    if (!geom || !bp) return fail(MDN_EINVAL, "filter_level: null geometry or bucket parameters");
    if (int rc = image(z, "filter_level: z", &n, &h, &w)) return rc;
    if (geom->r_coarse >= 0)
        if (int rc = same_image(coarse, "filter_level: coarse", z->dtype, n, (h + 1) / 2, (w + 1) / 2)) return rc;
    const int K = kcount(bp);
    int code = 0;
    if (int rc = bank(bank_t, "filter_level: bank", geom, K, &code)) return rc;
    if (int rc = same_image(out, "filter_level: out", z->dtype, n, h, w)) return rc;
    if (buckets_out)
        if (int rc = bucket_map(buckets_out, "filter_level: buckets_out", K, n, h, w)) return rc;
    return mdn_filter_level(z->data, geom->r_coarse >= 0 ? coarse->data : nullptr, z->dtype, n, h, w, bank_t->data,
                            code, geom, bp, out->data, buckets_out ? buckets_out->data : nullptr, stream);
}

int mdn_t_denoise_multiscale(const mdn_tensor* noisy, int32_t levels, const mdn_tensor* banks,
                             const mdn_geometry* geom, const mdn_bucket_params* bparams, mdn_tensor* out,
                             mdn_tensor* bucket_maps, void* ws, size_t ws_bytes, void* stream) {
    int64_t n, h, w;
    if (!geom || !bparams || !banks) return fail(MDN_EINVAL, "denoise_multiscale: null argument");
    if (int rc = image(noisy, "denoise_multiscale: noisy", &n, &h, &w)) return rc;
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "denoise_multiscale: levels must be 1..8");
    const int nb = geom->r_coarse < 0 ? 1 : levels - 1;
    if (nb < 1) return fail(MDN_EINVAL, "denoise_multiscale: a multiscale geometry needs levels >= 2");
    const void* bptr[8] = {};
    void* mptr[8] = {};
    int code0 = -1;
    int64_t hl = h, wl = w;
    for (int l = 0; l < nb; ++l) {
        char what[64];
        snprintf(what, sizeof what, "denoise_multiscale: banks[%d]", l);
        int code = 0;
        if (int rc = bank(&banks[l], what, geom, kcount(&bparams[l]), &code)) return rc;
        if (code0 >= 0 && code != code0) return fail(MDN_ESHAPE, "denoise_multiscale: banks differ in dtype");
        code0 = code;
        bptr[l] = banks[l].data;
        if (bucket_maps && bucket_maps[l].data) {
            snprintf(what, sizeof what, "denoise_multiscale: bucket_maps[%d]", l);
            if (int rc = bucket_map(&bucket_maps[l], what, kcount(&bparams[l]), n, hl, wl)) return rc;
            mptr[l] = bucket_maps[l].data;
        }
        hl = (hl + 1) / 2;
        wl = (wl + 1) / 2;
    }
    if (int rc = same_image(out, "denoise_multiscale: out", noisy->dtype, n, h, w)) return rc;
    return mdn_denoise_multiscale(noisy->data, noisy->dtype, n, h, w, levels, bptr, code0, geom, bparams, out->data,
                                  bucket_maps ? mptr : nullptr, ws, ws_bytes, stream);
}

int mdn_t_train_level_filters(const mdn_tensor* noisy_lvl, const mdn_tensor* coarse_out,
                              const mdn_tensor* clean_lvl, const mdn_geometry* geom, const mdn_bucket_params* bp,
                              int32_t gram_precision, int32_t accumulate, mdn_tensor* gram, mdn_tensor* counts,
                              double lambda, mdn_tensor* bank_out, void* ws, size_t ws_bytes, void* stream) {
    int64_t n, h, w;
    if (!geom || !bp) return fail(MDN_EINVAL, "train_level_filters: null geometry or bucket parameters");
    if (int rc = image(noisy_lvl, "train_level_filters: noisy_lvl", &n, &h, &w)) return rc;
    if (geom->r_coarse >= 0)
        if (int rc = same_image(coarse_out, "train_level_filters: coarse_out", noisy_lvl->dtype, n, (h + 1) / 2,
                                (w + 1) / 2))
            return rc;
    if (int rc = same_image(clean_lvl, "train_level_filters: clean_lvl", noisy_lvl->dtype, n, h, w)) return rc;
    const int K = kcount(bp), D = mdn_regressor_len(geom);
    if (D <= 0) return fail(MDN_ESHAPE, "train_level_filters: geometry");
    const bool cross = geom->cross_channel != 0;
    const int64_t gs[4] = {K, cross ? 1 : 3, cross ? D + 3 : D + 1, cross ? D + 3 : D + 1};
    if (int rc = want(gram, "train_level_filters: gram", MDN_F64, -1, 4, gs)) return rc;
    const int64_t cs[1] = {K};
    if (int rc = want(counts, "train_level_filters: counts", MDN_I64, -1, 1, cs)) return rc;
    if (bank_out) {
        const int64_t bs[3] = {K, 3, D};
        if (int rc = want(bank_out, "train_level_filters: bank_out", MDN_F32, -1, 3, bs)) return rc;
    }
    return mdn_train_level_filters(noisy_lvl->data, geom->r_coarse >= 0 ? coarse_out->data : nullptr,
                                   clean_lvl->data, noisy_lvl->dtype, n, h, w, geom, bp, gram_precision, accumulate,
                                   (double*)gram->data, (int64_t*)counts->data, lambda,
                                   bank_out ? (float*)bank_out->data : nullptr, ws, ws_bytes, stream);
}

}  // extern "C"
