/*
 * mdn_oracle.c -- plain, slow, FP64 CPU oracle for trainable multiscale
 * denoising (Choi, Isidoro, Getreuer, Milanfar, "Fast, Trainable, Multiscale
 * Denoising", arXiv 1802.06130).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code with the
 * CUDA path and is written straight from the paper's definitions:
 *
 *   pyramid           Section 4 "Multiscale filtering" (2x downsampling)
 *   structure tensor  Section 3 "Filter selection", tensor T_i equation
 *   features/buckets  Section 3 "Filter selection" (orientation, strength,
 *                     coherence) -> s(i)
 *   filtering         Eq. 1 (single scale) and the multiscale equation of
 *                     Section 4 (h = [f; g] over [R_{i/2} u^{l+1}; R_i z^l])
 *   colour            Section 3 footnote 1: YCbCr (ITU-R BT.601) per channel
 *   training          Eqs. 5-6 (train1/train2): per-bucket linear least
 *                     squares, solved through the normal equations
 *
 * Readings of places where the paper is silent (each also listed in the
 * design notes): clamp-to-edge borders; 5-tap binomial downsampling;
 * central-difference gradients; 5x5 normalised Gaussian (sigma 1.5) spatial
 * weights on clamped product fields; orientation = minor-eigenvector angle in
 * [0, pi) with x to the right and y down; lower-inclusive thresholds;
 * coherence := 0 when sqrt(l1)+sqrt(l2) < coh_eps; coarse index floor(i/2)
 * (or, with `align`, the coarse patch sampled bilinearly at i/2: the
 * half-pixel-aligned variant of the coarse term);
 * ridge (G/n + lambda I) h = b/n; empty buckets take the pooled filter.
 *
 * Precision modes.  Everything is FP64 unless `mirror32` is set, in which
 * case the pyramid and the structure tensor/features follow the documented
 * FP32 evaluation order (explicit fmaf, -ffp-contract=off) so that bucket
 * indices can be compared bit for bit.  Stored planes can be rounded to FP32
 * or FP16 (round-to-nearest-even) to mirror a storage precision.
 *
 * All images are planar [C][H][W], row-major.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP loops (the filter and Gram loops over rows): set
 * (n > 0) and query.  Used to time the oracle single-threaded and on all
 * host cores. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_MAX_THR 16
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t n_angle, n_strength, n_coherence;
    float strength_thr[ORC_MAX_THR];
    float coherence_thr[ORC_MAX_THR];
    float coh_eps;
} orc_bparams;

static inline long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ */
/* Storage rounding                                                    */
/* ------------------------------------------------------------------ */

/* Round to the nearest IEEE binary16 value, ties to even (IEEE 754-2008
 * round-to-nearest-even).  Finite results only up to 65504; larger
 * magnitudes go to +-inf as RN does at >= 65520. */
double orc_round_f16(double x)
{
    if (isnan(x)) return x;
    double a = fabs(x);
    if (a >= 65520.0) return copysign(INFINITY, x);
    if (a == 0.0) return x;
    int e;
    frexp(a, &e);                /* a = m * 2^e, m in [0.5, 1) */
    /* binary16: 11 significant bits for normals (exponent >= -14),
     * fixed quantum 2^-24 for subnormals. */
    int q = (e - 1 >= -14) ? (e - 1 - 10) : -24;
    double scaled = ldexp(a, -q);
    double r = nearbyint(scaled); /* default rounding mode: nearest-even */
    return copysign(ldexp(r, q), x);
}

void orc_round_storage(double* x, long n, int storage)
{
    /* storage: 0 = keep FP64, 1 = FP32, 2 = FP16 */
    if (storage == 1) {
        for (long i = 0; i < n; ++i) x[i] = (double)(float)x[i];
    } else if (storage == 2) {
        for (long i = 0; i < n; ++i) x[i] = orc_round_f16(x[i]);
    }
}

/* ------------------------------------------------------------------ */
/* A1: 2x downsampling (Section 4, "Multiscale filtering")             */
/* ------------------------------------------------------------------ */

static const double BINOM5[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};

/* out[c][y][x] = sum_{u,v=-2..2} b_u b_v in[c][clamp(2y+v)][clamp(2x+u)],
 * out size ceil(H/2) x ceil(W/2).  mirror32 = 0: direct 25-tap FP64 sum.
 * mirror32 = 1: FP32, horizontal pass first (fmaf chain u = -2..2 at every
 * clamped input row), then the vertical pass (fmaf chain v = -2..2). */
void orc_pyramid_down(const double* in, int C, int H, int W, double* out, int mirror32)
{
    int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    for (int c = 0; c < C; ++c) {
        const double* p = in + (long)c * H * W;
        double* q = out + (long)c * Ho * Wo;
        for (int y = 0; y < Ho; ++y)
            for (int x = 0; x < Wo; ++x) {
                if (!mirror32) {
                    double s = 0.0;
                    for (int v = -2; v <= 2; ++v)
                        for (int u = -2; u <= 2; ++u) {
                            long yy = clampl(2L * y + v, 0, H - 1);
                            long xx = clampl(2L * x + u, 0, W - 1);
                            s += BINOM5[v + 2] * BINOM5[u + 2] * p[yy * W + xx];
                        }
                    q[(long)y * Wo + x] = s;
                } else {
                    float hrow[5];
                    for (int v = -2; v <= 2; ++v) {
                        long yy = clampl(2L * y + v, 0, H - 1);
                        float acc = (float)BINOM5[0] * (float)p[yy * W + clampl(2L * x - 2, 0, W - 1)];
                        for (int u = -1; u <= 2; ++u)
                            acc = fmaf((float)BINOM5[u + 2], (float)p[yy * W + clampl(2L * x + u, 0, W - 1)], acc);
                        hrow[v + 2] = acc;
                    }
                    float acc = (float)BINOM5[0] * hrow[0];
                    for (int v = 1; v < 5; ++v) acc = fmaf((float)BINOM5[v], hrow[v], acc);
                    q[(long)y * Wo + x] = (double)acc;
                }
            }
    }
}

/* ------------------------------------------------------------------ */
/* A2: colour structure tensor (Section 3, "Filter selection")         */
/* ------------------------------------------------------------------ */

/* Spatial weights w_j: 5x5 Gaussian, sigma = 1.5, normalised to sum 1; it is
 * separable, w_{u,v} = w_u w_v with the 1-D weights normalised. */
static void gauss5(double w[5])
{
    double s = 0.0;
    for (int u = -2; u <= 2; ++u) { w[u + 2] = exp(-(double)(u * u) / (2.0 * 1.5 * 1.5)); s += w[u + 2]; }
    for (int u = 0; u < 5; ++u) w[u] /= s;
}

/* T_i = sum_c sum_j w_j g^c_j (g^c_j)^T with g^c = ((z[x+1]-z[x-1])/2,
 * (z[y+1]-z[y-1])/2) per RGB channel c, neighbours clamped to the image; the
 * sum over j runs over the 5x5 window with clamped positions.
 * Output T planar [3][H][W] = (Txx, Txy, Tyy). */
void orc_structure_tensor(const double* z, int H, int W, int mirror32, double* T)
{
    long HW = (long)H * W;
    double w[5];
    gauss5(w);
    /* products per pixel */
    double* P = (double*)malloc(sizeof(double) * 3 * HW);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long xm = clampl(x - 1, 0, W - 1), xp = clampl(x + 1, 0, W - 1);
            long ym = clampl(y - 1, 0, H - 1), yp = clampl(y + 1, 0, H - 1);
            if (!mirror32) {
                double pxx = 0, pxy = 0, pyy = 0;
                for (int c = 0; c < 3; ++c) {
                    const double* zc = z + c * HW;
                    double gx = (zc[(long)y * W + xp] - zc[(long)y * W + xm]) / 2.0;
                    double gy = (zc[yp * W + x] - zc[ym * W + x]) / 2.0;
                    pxx += gx * gx; pxy += gx * gy; pyy += gy * gy;
                }
                P[(long)y * W + x] = pxx; P[HW + (long)y * W + x] = pxy; P[2 * HW + (long)y * W + x] = pyy;
            } else {
                float gx[3], gy[3];
                for (int c = 0; c < 3; ++c) {
                    const double* zc = z + c * HW;
                    gx[c] = ((float)zc[(long)y * W + xp] - (float)zc[(long)y * W + xm]) * 0.5f;
                    gy[c] = ((float)zc[yp * W + x] - (float)zc[ym * W + x]) * 0.5f;
                }
                float pxx = gx[0] * gx[0], pxy = gx[0] * gy[0], pyy = gy[0] * gy[0];
                for (int c = 1; c < 3; ++c) {
                    pxx = fmaf(gx[c], gx[c], pxx);
                    pxy = fmaf(gx[c], gy[c], pxy);
                    pyy = fmaf(gy[c], gy[c], pyy);
                }
                P[(long)y * W + x] = pxx; P[HW + (long)y * W + x] = pxy; P[2 * HW + (long)y * W + x] = pyy;
            }
        }
    if (!mirror32) {
        for (int f = 0; f < 3; ++f)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    double s = 0.0;
                    for (int v = -2; v <= 2; ++v)
                        for (int u = -2; u <= 2; ++u)
                            s += w[v + 2] * w[u + 2] * P[f * HW + clampl(y + v, 0, H - 1) * W + clampl(x + u, 0, W - 1)];
                    T[f * HW + (long)y * W + x] = s;
                }
    } else {
        float wf[5];
        for (int u = 0; u < 5; ++u) wf[u] = (float)w[u];
        float* Hs = (float*)malloc(sizeof(float) * HW);
        for (int f = 0; f < 3; ++f) {
            /* horizontal pass (u = -2..2 fmaf chain), then vertical */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    float acc = wf[0] * (float)P[f * HW + (long)y * W + clampl(x - 2, 0, W - 1)];
                    for (int u = -1; u <= 2; ++u)
                        acc = fmaf(wf[u + 2], (float)P[f * HW + (long)y * W + clampl(x + u, 0, W - 1)], acc);
                    Hs[(long)y * W + x] = acc;
                }
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    float acc = wf[0] * Hs[clampl(y - 2, 0, H - 1) * W + x];
                    for (int v = -1; v <= 2; ++v)
                        acc = fmaf(wf[v + 2], Hs[clampl(y + v, 0, H - 1) * W + x], acc);
                    T[f * HW + (long)y * W + x] = (double)acc;
                }
        }
        free(Hs);
    }
    free(P);
}

/* ------------------------------------------------------------------ */
/* A3: eigen-features and the bucket index s(i)                        */
/* ------------------------------------------------------------------ */

/* Eigenvalues l1 >= l2 of T = [[a,b],[b,c]]; strength = sqrt(l1);
 * coherence = (sqrt l1 - sqrt l2)/(sqrt l1 + sqrt l2), := 0 when the
 * denominator is below coh_eps; orientation = angle of the eigenvector of the
 * smaller eigenvalue, theta = atan2(2b, a - c)/2 + pi/2 reduced to [0, pi)
 * (atan2(0,0) = 0, so an isotropic T gives theta = pi/2).
 * feat planar [3][H][W] = (theta/pi, strength, coherence).
 * mirror32: l1, l2, strength and coherence in FP32 with the documented order;
 * theta from the FP32 pair (a - c, 2b) evaluated in FP64. */
void orc_features(const double* T, int H, int W, int mirror32, float coh_eps, double* feat)
{
    long HW = (long)H * W;
    for (long i = 0; i < HW; ++i) {
        double a = T[i], b = T[HW + i], c = T[2 * HW + i];
        double th, st, co;
        if (!mirror32) {
            double ht = (a + c) / 2.0, hd = (a - c) / 2.0;
            double disc = sqrt(hd * hd + b * b);
            double l1 = ht + disc, l2 = ht - disc;
            if (l2 < 0) l2 = 0;
            if (l1 < 0) l1 = 0;
            double s1 = sqrt(l1), s2 = sqrt(l2);
            st = s1;
            co = (s1 + s2 < (double)coh_eps) ? 0.0 : (s1 - s2) / (s1 + s2);
            th = 0.5 * atan2(2.0 * b, a - c) + M_PI / 2.0;
        } else {
            float af = (float)a, bf = (float)b, cf = (float)c;
            float ht = (af + cf) * 0.5f, hd = (af - cf) * 0.5f;
            float disc = sqrtf(fmaf(hd, hd, bf * bf));
            float l1 = ht + disc, l2 = ht - disc;
            if (l2 < 0.0f) l2 = 0.0f;
            float s1 = sqrtf(l1), s2 = sqrtf(l2);
            float den = s1 + s2;
            st = (double)s1;
            co = (den < coh_eps) ? 0.0 : (double)((s1 - s2) / den);
            float X = af - cf, Y = bf + bf;
            th = 0.5 * atan2((double)Y, (double)X) + M_PI / 2.0;
        }
        if (th >= M_PI) th -= M_PI;
        if (th < 0) th += M_PI;
        feat[i] = th / M_PI;
        feat[HW + i] = st;
        feat[2 * HW + i] = co;
    }
}

static int count_le(const float* thr, int n, double v)
{
    int k = 0;
    for (int t = 0; t < n; ++t) if ((double)thr[t] <= v) ++k;
    return k;
}

/* s(i) = (a * n_strength + s) * n_coherence + c with a = floor(n_angle *
 * theta/pi) (clamped to n_angle-1), s and c = number of thresholds <= value.
 * band[i] = 1 when any feature lies within `band_eps` of a decision threshold
 * (angle boundaries k/n_angle incl. 0 and 1, strength and coherence
 * thresholds, and coh_eps for sqrt(l1)+sqrt(l2), approximated here by the
 * strength feature). */
void orc_buckets(const double* feat, int H, int W, const orc_bparams* bp, double band_eps,
                 int32_t* bucket, uint8_t* band)
{
    long HW = (long)H * W;
    int ns = bp->n_strength - 1, nc = bp->n_coherence - 1;
    for (long i = 0; i < HW; ++i) {
        double t = feat[i], st = feat[HW + i], co = feat[2 * HW + i];
        int a = (int)floor(t * bp->n_angle);
        if (a >= bp->n_angle) a = bp->n_angle - 1;
        if (a < 0) a = 0;
        int s = count_le(bp->strength_thr, ns, st);
        int c = count_le(bp->coherence_thr, nc, co);
        bucket[i] = (a * bp->n_strength + s) * bp->n_coherence + c;
        if (band) {
            int bd = 0;
            double ta = t * bp->n_angle;
            double fr = ta - floor(ta);
            if (fr * (1.0 / bp->n_angle) < band_eps || (1.0 - fr) * (1.0 / bp->n_angle) < band_eps) bd = 1;
            for (int k = 0; k < ns; ++k) if (fabs(st - (double)bp->strength_thr[k]) < band_eps) bd = 1;
            for (int k = 0; k < nc; ++k) if (fabs(co - (double)bp->coherence_thr[k]) < band_eps) bd = 1;
            if (st < (double)bp->coh_eps + band_eps) bd = 1;
            band[i] = (uint8_t)bd;
        }
    }
}

/* FP32 bucket decisions (the `mirror32` reading used to pin the GPU's bucket
 * maps bit for bit).  The strength and coherence bins are decided on the
 * FP32 tensor (a, b, c) without square roots or divisions, by comparisons
 * that are equivalent in exact arithmetic to thresholding the features:
 *   ht = (a + c) / 2, hd = (a - c) / 2, d2 = hd^2 + b^2 (= disc^2), so
 *   lambda1 = ht + disc and lambda2 = ht - disc;
 *   sqrt(lambda1) >= T  <=>  disc >= T^2 - ht
 *                       <=>  u <= 0  or  d2 >= u^2,   u = T^2 - ht;
 *   coherence >= C (0 <= C < 1)  <=>  disc >= ht * 2C / (1 + C^2)
 *                       <=>  d2 >= (ht R)^2,          R = 2C / (1 + C^2)
 *   (C = 1: R = 1; C > 1 never passes);
 *   coherence := 0 (bin 0) when lambda1 < eps^2 <=> v > 0 and d2 < v^2, v = eps^2 - ht.
 * Every quantity is an FP32 operation in this order (T^2, R and eps^2 are
 * computed in FP64 from the FP32 thresholds and rounded to FP32), so a
 * decision differs from thresholding the exact features only for features
 * within a few ulps of a threshold.  The angle bin is floor(n_angle theta/pi)
 * with theta from atan2 in FP64 on the FP32 pair (a - c, 2b). */
void orc_buckets_fp32(const double* T, int H, int W, const orc_bparams* bp, int32_t* bucket)
{
    long HW = (long)H * W;
    int ns = bp->n_strength - 1, nc = bp->n_coherence - 1;
    float q[16], r[16];
    for (int t = 0; t < ns; ++t) q[t] = (float)((double)bp->strength_thr[t] * (double)bp->strength_thr[t]);
    for (int t = 0; t < nc; ++t) {
        double C = (double)bp->coherence_thr[t];
        r[t] = C < 1.0 ? (float)(2.0 * C / (1.0 + C * C)) : (C == 1.0 ? 1.0f : INFINITY);
    }
    const float e2 = (float)((double)bp->coh_eps * (double)bp->coh_eps);
    for (long i = 0; i < HW; ++i) {
        float af = (float)T[i], bf = (float)T[HW + i], cf = (float)T[2 * HW + i];
        float ht = (af + cf) * 0.5f, hd = (af - cf) * 0.5f;
        float d2 = fmaf(hd, hd, bf * bf);
        int s = 0, c = 0;
        for (int t = 0; t < ns; ++t) {
            float u = q[t] - ht;
            if (u <= 0.0f || d2 >= u * u) ++s;
        }
        float v = e2 - ht;
        int zero = v > 0.0f && d2 < v * v;
        if (!zero)
            for (int t = 0; t < nc; ++t) {
                float w = ht * r[t];
                if (d2 >= w * w) ++c;
            }
        float X = af - cf, Y = bf + bf;
        double th = 0.5 * atan2((double)Y, (double)X) + M_PI / 2.0;
        if (th >= M_PI) th -= M_PI;
        if (th < 0) th += M_PI;
        int a = (int)floor(th / M_PI * bp->n_angle);
        if (a >= bp->n_angle) a = bp->n_angle - 1;
        if (a < 0) a = 0;
        bucket[i] = (a * bp->n_strength + s) * bp->n_coherence + c;
    }
}

/* ------------------------------------------------------------------ */
/* Colour transform (Section 3 footnote 1): zero-offset ITU-R BT.601   */
/* ------------------------------------------------------------------ */

static void rgb_to_ycc(double r, double g, double b, double* y, double* cb, double* cr)
{
    double Y = 0.299 * r + 0.587 * g + 0.114 * b;
    *y = Y;
    *cb = (b - Y) / 1.772;
    *cr = (r - Y) / 1.402;
}

static void ycc_to_rgb(double y, double cb, double cr, double* r, double* g, double* b)
{
    double R = y + 1.402 * cr;
    double B = y + 1.772 * cb;
    *r = R;
    *b = B;
    *g = (y - 0.299 * R - 0.114 * B) / 0.587;
}

/* planar RGB <-> YCbCr (color = 0: YCbCr, 1: identity / RGB filtering) */
void orc_to_work(const double* rgb, long HW, int color, double* out)
{
    for (long i = 0; i < HW; ++i) {
        if (color == 1) { out[i] = rgb[i]; out[HW + i] = rgb[HW + i]; out[2 * HW + i] = rgb[2 * HW + i]; }
        else rgb_to_ycc(rgb[i], rgb[HW + i], rgb[2 * HW + i], out + i, out + HW + i, out + 2 * HW + i);
    }
}

void orc_from_work(const double* w, long HW, int color, double* out)
{
    for (long i = 0; i < HW; ++i) {
        if (color == 1) { out[i] = w[i]; out[HW + i] = w[HW + i]; out[2 * HW + i] = w[2 * HW + i]; }
        else ycc_to_rgb(w[i], w[HW + i], w[2 * HW + i], out + i, out + HW + i, out + 2 * HW + i);
    }
}

/* ------------------------------------------------------------------ */
/* Regressor vector (patch operator R_i, Section 3; [R_{i/2}u; R_i z],  */
/* Section 4)                                                          */
/* ------------------------------------------------------------------ */

/* Coarse sample of channel plane u (Hc x Wc) for fine pixel (y, x) and tap
 * (dy, dx).  align = 0: u at (floor(y/2) + dy, floor(x/2) + dx) (reading of
 * the paper's i/2).  align = 1: u sampled bilinearly at (y/2 + dy, x/2 + dx)
 * -- coarse pixel (Y, X) sits at fine (2Y, 2X), so an odd fine coordinate
 * falls half way between two coarse samples and takes their mean; each of the
 * (up to four) samples is clamped to the plane on its own. */
static double coarse_sample(const double* u, int Hc, int Wc, int y, int x, int dy, int dx, int align)
{
    int y0 = y / 2 + dy, x0 = x / 2 + dx;
    int ny = (align && (y & 1)) ? 2 : 1, nx = (align && (x & 1)) ? 2 : 1;
    double s = 0.0;
    for (int a = 0; a < ny; ++a)
        for (int b = 0; b < nx; ++b)
            s += u[clampl(y0 + a, 0, Hc - 1) * Wc + clampl(x0 + b, 0, Wc - 1)];
    return s / (double)(ny * nx);
}

/* Regressor for output channel oc at pixel (y, x): coarse taps first (when
 * rc >= 0), then fine taps.  Within each block: (channel, dy, dx) row-major,
 * the channel loop covering the output channel only (per-channel geometry) or
 * all three (cross-channel).  zw is the working-space (YCbCr or RGB) image of
 * level l, uw the working-space image of level l+1 of size Hc x Wc; align
 * selects the coarse sampling (coarse_sample). */
static int regressor(const double* zw, int H, int W, const double* uw, int Hc, int Wc,
                     int rf, int rc, int cross, int align, int oc, int y, int x, double* r)
{
    int n = 0;
    long HW = (long)H * W, HWc = (long)Hc * Wc;
    int c0 = cross ? 0 : oc, c1 = cross ? 3 : oc + 1;
    if (rc >= 0) {
        for (int c = c0; c < c1; ++c)
            for (int dy = -rc; dy <= rc; ++dy)
                for (int dx = -rc; dx <= rc; ++dx)
                    r[n++] = coarse_sample(uw + c * HWc, Hc, Wc, y, x, dy, dx, align);
    }
    for (int c = c0; c < c1; ++c)
        for (int dy = -rf; dy <= rf; ++dy)
            for (int dx = -rf; dx <= rf; ++dx)
                r[n++] = zw[c * HW + clampl(y + dy, 0, H - 1) * W + clampl(x + dx, 0, W - 1)];
    return n;
}

int orc_regressor_len(int rf, int rc, int cross)
{
    int pf = (2 * rf + 1) * (2 * rf + 1), pc = rc >= 0 ? (2 * rc + 1) * (2 * rc + 1) : 0;
    return (cross ? 3 : 1) * (pf + pc);
}

/* ------------------------------------------------------------------ */
/* A4: spatially-adaptive filtering, Eq. 1 and the multiscale equation  */
/* ------------------------------------------------------------------ */

/* out (RGB, [3][H][W]) = from_work( (h^{s(i)}_oc)^T [R_{i/2} u ; R_i z] ).
 * z: level-l RGB image; uc: level-(l+1) RGB image (Hc x Wc) or NULL when
 * rc < 0; bank: [K][3][D] (D = orc_regressor_len). */
void orc_filter_level(const double* z, int H, int W, const double* uc, int Hc, int Wc,
                      const int32_t* bucket, const double* bank, int K,
                      int rf, int rc, int cross, int color, int align, double* out)
{
    long HW = (long)H * W;
    int D = orc_regressor_len(rf, rc, cross);
    double* zw = (double*)malloc(sizeof(double) * 3 * HW);
    double* uw = NULL;
    orc_to_work(z, HW, color, zw);
    if (rc >= 0) {
        uw = (double*)malloc(sizeof(double) * 3 * (long)Hc * Wc);
        orc_to_work(uc, (long)Hc * Wc, color, uw);
    }
    double* ow = (double*)malloc(sizeof(double) * 3 * HW);
#pragma omp parallel
    {
        double* r = (double*)malloc(sizeof(double) * D);
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int k = bucket[(long)y * W + x];
                if (k >= K) k = K - 1;
                for (int oc = 0; oc < 3; ++oc) {
                    regressor(zw, H, W, uw, Hc, Wc, rf, rc, cross, align, oc, y, x, r);
                    const double* h = bank + ((long)k * 3 + oc) * D;
                    double s = 0.0;
                    for (int j = 0; j < D; ++j) s += h[j] * r[j];
                    ow[oc * HW + (long)y * W + x] = s;
                }
            }
        free(r);
    }
    orc_from_work(ow, HW, color, out);
    free(ow);
    free(zw);
    free(uw);
}

/* ------------------------------------------------------------------ */
/* A5: per-bucket normal equations (Eqs. 5-6)                          */
/* ------------------------------------------------------------------ */

/* Accumulates, for every pixel i with s(i) = k, the Gram matrix of the
 * augmented row a = [x ; y] into gram[k][g] (size Dp x Dp, Dp = D + T):
 * per-channel geometry: G = 3 groups (one per working channel), T = 1 target;
 * cross-channel: G = 1 group, T = 3 targets.  counts[k] += 1 per pixel.
 * target: level-l clean RGB image. */
void orc_gram_accumulate(const double* z, int H, int W, const double* uc, int Hc, int Wc,
                         const double* target, const int32_t* bucket, int K,
                         int rf, int rc, int cross, int color, int align, double* gram, int64_t* counts)
{
    long HW = (long)H * W;
    int D = orc_regressor_len(rf, rc, cross);
    int G = cross ? 1 : 3, Tn = cross ? 3 : 1, Dp = D + Tn;
    double* zw = (double*)malloc(sizeof(double) * 3 * HW);
    double* tw = (double*)malloc(sizeof(double) * 3 * HW);
    double* uw = NULL;
    orc_to_work(z, HW, color, zw);
    orc_to_work(target, HW, color, tw);
    if (rc >= 0) {
        uw = (double*)malloc(sizeof(double) * 3 * (long)Hc * Wc);
        orc_to_work(uc, (long)Hc * Wc, color, uw);
    }
    double* a = (double*)malloc(sizeof(double) * Dp);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int k = bucket[(long)y * W + x];
            if (k >= K) continue;
            counts[k] += 1;
            for (int g = 0; g < G; ++g) {
                regressor(zw, H, W, uw, Hc, Wc, rf, rc, cross, align, g, y, x, a);
                if (cross) for (int t = 0; t < 3; ++t) a[D + t] = tw[t * HW + (long)y * W + x];
                else a[D] = tw[g * HW + (long)y * W + x];
                double* Gm = gram + ((long)k * G + g) * Dp * Dp;
                for (int p = 0; p < Dp; ++p)
                    for (int q = 0; q < Dp; ++q) Gm[(long)p * Dp + q] += a[p] * a[q];
            }
        }
    free(a);
    free(zw);
    free(tw);
    free(uw);
}

/* ------------------------------------------------------------------ */
/* A6: ridge solve by Cholesky (FP64)                                  */
/* ------------------------------------------------------------------ */

/* Solves (A) X = B in place for SPD A (n x n, row-major) and m right-hand
 * sides B (n x m, row-major) by A = L L^T, forward then back substitution.
 * Returns 0, or -1 when a pivot is not positive. */
int orc_cholesky_solve(double* A, int n, double* B, int m)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(long)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(long)j * n + k] * A[(long)j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        A[(long)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(long)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(long)i * n + k] * A[(long)j * n + k];
            A[(long)i * n + j] = s / ljj;
        }
    }
    for (int c = 0; c < m; ++c) {
        for (int i = 0; i < n; ++i) {           /* L y = b */
            double s = B[(long)i * m + c];
            for (int k = 0; k < i; ++k) s -= A[(long)i * n + k] * B[(long)k * m + c];
            B[(long)i * m + c] = s / A[(long)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {      /* L^T x = y */
            double s = B[(long)i * m + c];
            for (int k = i + 1; k < n; ++k) s -= A[(long)k * n + i] * B[(long)k * m + c];
            B[(long)i * m + c] = s / A[(long)i * n + i];
        }
    }
    return 0;
}

/* h_k = (G_k^{XX}/n_k + lambda I)^{-1} G_k^{XY}/n_k for every bucket and
 * group; a bucket with n_k = 0 takes the pooled filter solved from the sum
 * of all buckets' Gram matrices with the same ridge.  bank_out: [K][3][D].
 * Returns the number of failed solves. */
int orc_solve_bank(const double* gram, const int64_t* counts, int K, int D, int cross,
                   double lambda, double* bank_out)
{
    int G = cross ? 1 : 3, Tn = cross ? 3 : 1, Dp = D + Tn;
    long gsz = (long)Dp * Dp;
    int fails = 0;
    double* pooled = (double*)calloc((size_t)G * gsz, sizeof(double));
    int64_t ntot = 0;
    for (int k = 0; k < K; ++k) {
        ntot += counts[k];
        for (int g = 0; g < G; ++g)
            for (long e = 0; e < gsz; ++e) pooled[g * gsz + e] += gram[((long)k * G + g) * gsz + e];
    }
    double* A = (double*)malloc(sizeof(double) * D * D);
    double* B = (double*)malloc(sizeof(double) * D * Tn);
    double* pooled_h = (double*)calloc((size_t)3 * D, sizeof(double));
    /* k = -1 solves the pooled system first; empty buckets then copy it */
    {
        for (int k = -1; k < K; ++k) {
            const double* Gk;
            double n;
            if (k < 0) { Gk = pooled; n = (double)ntot; }
            else {
                if (counts[k] == 0) {
                    memcpy(bank_out + (long)k * 3 * D, pooled_h, sizeof(double) * 3 * D);
                    continue;
                }
                Gk = gram + (long)k * G * gsz; n = (double)counts[k];
            }
            for (int g = 0; g < G; ++g) {
                const double* Gm = Gk + g * gsz;
                if (n == 0) { fails++; continue; }
                for (int p = 0; p < D; ++p) {
                    for (int q = 0; q < D; ++q) A[(long)p * D + q] = Gm[(long)p * Dp + q] / n;
                    A[(long)p * D + p] += lambda;
                    for (int t = 0; t < Tn; ++t) B[(long)p * Tn + t] = Gm[(long)p * Dp + D + t] / n;
                }
                if (orc_cholesky_solve(A, D, B, Tn) != 0) { fails++; continue; }
                double* dst = (k < 0) ? pooled_h : bank_out + (long)k * 3 * D;
                for (int t = 0; t < Tn; ++t) {
                    int oc = cross ? t : g;
                    for (int p = 0; p < D; ++p) dst[(long)oc * D + p] = B[(long)p * Tn + t];
                }
            }
        }
    }
    free(pooled_h);
    free(A);
    free(B);
    free(pooled);
    return fails;
}
