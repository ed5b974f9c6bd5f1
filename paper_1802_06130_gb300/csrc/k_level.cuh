// k_level.cuh -- A2+A3+A4: the fused per-level kernel.
//
// For every output pixel i of level l, in one pass over a tile:
//   * colour structure tensor T_i (Section 3, "Filter selection"): central
//     differences per RGB channel, products summed over channels, separable
//     5x5 Gaussian (sigma 1.5) on the clamped product field;
//   * eigen-features (strength sqrt(l1), coherence, orientation of the minor
//     eigenvector) and the bucket s(i);
//   * the selected filter applied to [R_{i/2} u^{l+1} ; R_i z^l] in the
//     working colour space (multiscale equation of Section 4; Eq. 1 when
//     there is no coarse term), converted back to RGB and stored.
//
// Arithmetic of the selector (fixed, reproducible bit for bit):
//   g = (z[+1] - z[-1]) * 0.5 per axis and channel;
//   Pxx = gxR*gxR, fma(gxG,gxG,.), fma(gxB,gxB,.)  (same for Pxy, Pyy);
//   H = w0*P[x-2], fma(w1,P[x-1]) ... fma(w4,P[x+2]);  T = same over rows;
//   ht = (a+c)*0.5, hd = (a-c)*0.5, disc = sqrt(fma(hd,hd,b*b)),
//   l1 = ht+disc, l2 = max(ht-disc, 0), s1 = sqrt(l1), s2 = sqrt(l2),
//   coherence = (s1-s2)/(s1+s2) or 0 if s1+s2 < coh_eps, strength = s1
//   (IEEE round-to-nearest square roots and division throughout, so that the
//   FP32 reference evaluated in the same order gives the same buckets).
// Orientation bin: the doubled angle psi = 2 theta of the minor eigenvector
// is the angle of v = (c-a, -2b); psi is placed in one of n_angle sectors of
// width 2 pi / n_angle by sign tests against the sector boundary vectors (no
// arctangent), with v = 0 mapped to theta = pi/2.
//
// Tiling and memory: a persistent CTA (grid = SMs x resident CTAs) loads the
// whole filter bank into shared memory once (when it fits; otherwise taps are
// read through the read-only cache), then loops over TW x TH tiles: the RGB
// tile with a 3-pixel halo and the coarse tile with an r_coarse halo are
// staged in shared memory with coalesced, clamped loads, the tensor fields
// are computed in shared memory, and every thread filters its pixels with
// taps and patch values from shared memory.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace mdn {
namespace lvl {

constexpr int TW = 32, TH = 16, NT = 256;
constexpr int HZ = 3;                      // tensor halo (1 gradient + 2 smoothing)
constexpr int ZW = TW + 2 * HZ, ZH = TH + 2 * HZ;
constexpr int PW = TW + 4, PH = TH + 4;

template <int RC> struct Coarse {
    static constexpr int UW = RC >= 0 ? TW / 2 + 2 * RC : 0;
    static constexpr int UH = RC >= 0 ? TH / 2 + 2 * RC : 0;
};

template <typename TB> struct BankVec;
template <> struct BankVec<float> { static constexpr int V = 4; };
template <> struct BankVec<__half> { static constexpr int V = 8; };

template <int RF, int RC, bool CROSS> struct Geo {
    static constexpr int PF = (2 * RF + 1) * (2 * RF + 1);
    static constexpr int PC = RC >= 0 ? (2 * RC + 1) * (2 * RC + 1) : 0;
    static constexpr int NCH = CROSS ? 3 : 1;
    static constexpr int D = NCH * (PF + PC);
};

template <typename TB, int D> struct BankLayout {
    static constexpr int V = BankVec<TB>::V;
    static constexpr int DP = (D + V - 1) / V * V;   // padded row length
};

// shared-memory footprint of the tile buffers (bytes; the bucket tile is u16)
template <int RC> constexpr size_t tile_bytes() {
    return sizeof(float) * (3 * ZH * ZW + 3 * PH * PW + 3 * PH * TW + 3 * Coarse<RC>::UH * Coarse<RC>::UW) +
           sizeof(uint16_t) * TH * TW;
}

__device__ __forceinline__ void rgb_to_work(float r, float g, float b, int color, float& y, float& cb, float& cr) {
    if (color == MDN_RGB) { y = r; cb = g; cr = b; return; }
    // zero-offset ITU-R BT.601: Y = .299R + .587G + .114B, Cb = (B-Y)/1.772, Cr = (R-Y)/1.402
    y = 0.299f * r + 0.587f * g + 0.114f * b;
    cb = -0.168735892f * r - 0.331264108f * g + 0.5f * b;
    cr = 0.5f * r - 0.418687589f * g - 0.081312411f * b;
}
__device__ __forceinline__ void work_to_rgb(float y, float cb, float cr, int color, float& r, float& g, float& b) {
    if (color == MDN_RGB) { r = y; g = cb; b = cr; return; }
    r = y + 1.402f * cr;
    g = y - 0.344136286f * cb - 0.714136286f * cr;
    b = y + 1.772f * cb;
}

// Orientation/strength/coherence -> bucket index for N pixels at once (the
// N computations are independent and free of branches and divisions, so
// they overlap).  Strength and coherence bins are decided in the squared
// domain, equivalent in exact arithmetic to thresholding the features:
//   ht = (a+c)/2, hd = (a-c)/2, d2 = hd^2 + b^2 = disc^2
//   (lambda1 = ht + disc, lambda2 = ht - disc);
//   sqrt(lambda1) >= T      <=>  u <= 0 or d2 >= u^2, u = T^2 - ht;
//   coherence >= C (C < 1)  <=>  d2 >= (ht R)^2, R = 2C / (1 + C^2);
//   coherence := 0 when lambda1 < eps^2 <=> v > 0 and d2 < v^2, v = eps^2 - ht
// (T^2, R, eps^2: FP32 roundings of FP64 values, made on the host).  Each
// step is the FP32 operation shown, so a decision differs from thresholding
// the exact features only for features within a few ulps of a threshold.
// Orientation: the doubled angle of the minor eigenvector is the angle of
// v = (c - a, -2b); it is placed in one of n_angle sectors by counting the
// sector boundaries b_k (k < n_angle/2 - 1) with cross(b_k, v) >= 0, after
// folding v into the upper half plane; v = 0 gives theta = pi/2.
template <int N>
__device__ __forceinline__ void buckets_of(const float (&a)[N], const float (&b)[N], const float (&c)[N],
                                           const SelParams& sp, int (&k)[N]) {
    float ht[N], d2[N], vx[N], vy[N];
    int ab[N], sb[N], cb[N];
    bool zero[N];
    const int half = sp.n_angle >> 1;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        ht[n] = __fmul_rn(__fadd_rn(a[n], c[n]), 0.5f);
        const float hd = __fmul_rn(__fsub_rn(a[n], c[n]), 0.5f);
        d2[n] = __fmaf_rn(hd, hd, __fmul_rn(b[n], b[n]));
        float x = __fsub_rn(c[n], a[n]), y = -__fadd_rn(b[n], b[n]);
        const bool upper = (y > 0.f) || (y == 0.f && x > 0.f);
        const bool vz = (x == 0.f && y == 0.f);
        vx[n] = upper ? x : -x;
        vy[n] = upper ? y : -y;
        ab[n] = vz ? half : (upper ? 0 : half);
        zero[n] = vz;
        sb[n] = 0;
        cb[n] = 0;
    }
    for (int t = 0; t < half - 1; ++t) {
        const float bc = sp.bcos[t], bs = sp.bsin[t];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float cr = __fmaf_rn(bc, vy[n], -__fmul_rn(bs, vx[n]));
            ab[n] += (!zero[n] && cr >= 0.f) ? 1 : 0;
        }
    }
    for (int t = 0; t < sp.nthr_s; ++t) {
        const float q = sp.strength_q[t];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float u = __fsub_rn(q, ht[n]);
            sb[n] += (u <= 0.f || d2[n] >= __fmul_rn(u, u)) ? 1 : 0;
        }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) {
        const float v = __fsub_rn(sp.eps2, ht[n]);
        zero[n] = v > 0.f && d2[n] < __fmul_rn(v, v);
    }
    for (int t = 0; t < sp.nthr_c; ++t) {
        const float r = sp.coherence_r[t];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float w = __fmul_rn(ht[n], r);
            cb[n] += (!zero[n] && d2[n] >= __fmul_rn(w, w)) ? 1 : 0;
        }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) k[n] = (ab[n] * sp.n_strength + sb[n]) * sp.n_coherence + cb[n];
}
__device__ __forceinline__ int bucket_of(float a, float b, float c, const SelParams& sp) {
    const float A[1] = {a}, B[1] = {b}, Cc[1] = {c};
    int k[1];
    buckets_of<1>(A, B, Cc, sp, k);
    return k[0];
}

// One output channel of the level filter for the pixel whose fine-patch
// centre is zc (shared tile, working space) and coarse-patch centre uc.
// Two consecutive taps of a bank row read from global memory as one 4-byte
// (FP16) or 8-byte (FP32) load; the caller guarantees the alignment.
__device__ __forceinline__ void ld_pair(const __half* p, float& a, float& b) {
    const float2 f = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
    a = f.x; b = f.y;
}
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b) {
    const float2 f = __ldg(reinterpret_cast<const float2*>(p));
    a = f.x; b = f.y;
}

// pair_ok: the bank is read through the cache (SMEM = false) and every row
// start is aligned for ld_pair (even D and an aligned base pointer).
template <int RF, int RC, bool CROSS, typename TB, bool SMEM>
__device__ __forceinline__ float apply_filter(const TB* __restrict__ hb, const float* __restrict__ zc,
                                              const float* __restrict__ uc, int oc_const, bool pair_ok) {
    using G = Geo<RF, RC, CROSS>;
    constexpr int V = BankVec<TB>::V;
    constexpr int UW = Coarse<RC>::UW, UH = Coarse<RC>::UH;
    constexpr int NCOARSE = G::NCH * G::PC;
    float acc = 0.f;
    float h[V];
#pragma unroll
    for (int t = 0; t < G::D; ++t) {
        if (t % V == 0) {
            if constexpr (SMEM) {
                if constexpr (V == 4) {
                    float4 q = reinterpret_cast<const float4*>(hb)[t / V];
                    h[0] = q.x; h[1] = q.y; h[2] = q.z; h[3] = q.w;
                } else {
                    uint4 q = reinterpret_cast<const uint4*>(hb)[t / V];
                    const __half2* hp = reinterpret_cast<const __half2*>(&q);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float2 f = __half22float2(hp[e]);
                        h[2 * e] = f.x; h[2 * e + 1] = f.y;
                    }
                }
            } else if (G::D % 2 == 0 && pair_ok) {
#pragma unroll
                for (int e = 0; e < V; e += 2)
                    if (t + e < G::D) ld_pair(hb + t + e, h[e], h[e + 1]);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (t + e < G::D) h[e] = ld_f(hb, t + e);
            }
        }
        const float hv = h[t % V];
        if (t < NCOARSE) {
            constexpr int PCs = G::PC > 0 ? G::PC : 1, RCs = RC > 0 ? RC : 0;
            const int cc = t / PCs, idx = t % PCs;
            const int dy = idx / (2 * RCs + 1) - RCs, dx = idx % (2 * RCs + 1) - RCs;
            const int c = CROSS ? cc : oc_const;
            acc = fmaf(hv, uc[c * UH * UW + dy * UW + dx], acc);
        } else {
            const int tt = t - NCOARSE;
            const int cc = tt / G::PF, idx = tt % G::PF;
            const int dy = idx / (2 * RF + 1) - RF, dx = idx % (2 * RF + 1) - RF;
            const int c = CROSS ? cc : oc_const;
            acc = fmaf(hv, zc[c * ZH * ZW + dy * ZW + dx], acc);
        }
    }
    return acc;
}

template <int RF, int RC, bool CROSS, typename TS, typename TB, bool SMEM, bool FILTER>
__global__ void __launch_bounds__(NT) k_level(const TS* __restrict__ z, const TS* __restrict__ coarse,
                                              TS* __restrict__ out, void* __restrict__ bmap,
                                              const TB* __restrict__ bank, int H, int W, int Hc, int Wc,
                                              int nimg, int K, int color, SelParams sp, float w0, float w1,
                                              float w2, bool pair_ok) {
    using G = Geo<RF, RC, CROSS>;
    using BL = BankLayout<TB, G::D>;
    constexpr int UW = Coarse<RC>::UW, UH = Coarse<RC>::UH;
    extern __shared__ __align__(16) unsigned char smem[];
    float* zs = reinterpret_cast<float*>(smem);             // [3][ZH][ZW]
    float* ps = zs + 3 * ZH * ZW;                            // [3][PH][PW]
    float* hs = ps + 3 * PH * PW;                            // [3][PH][TW]
    float* us = hs + 3 * PH * TW;                            // [3][UH][UW]
    uint16_t* bk = reinterpret_cast<uint16_t*>(us + 3 * UH * UW);  // [TH][TW]
    TB* bank_s = reinterpret_cast<TB*>(smem + ((tile_bytes<RC>() + 15) & ~size_t(15)));
    const bool wide = K > 256;   // bucket map element: u8, or u16 above 256 buckets
    const int tid = threadIdx.x;
    const float wv[5] = {w0, w1, w2, w1, w0};

    if constexpr (FILTER && SMEM) {
        // bank -> shared memory, rows padded to BL::DP (pad taps are zero)
        const int rows = K * 3;
        for (int i = tid; i < rows * BL::DP; i += NT) {
            int r = i / BL::DP, t = i % BL::DP;
            bank_s[i] = t < G::D ? bank[(int64_t)r * G::D + t] : TB(0.f);
        }
    }

    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int64_t ntiles = (int64_t)tiles_x * tiles_y * nimg;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int img = (int)(tile / ((int64_t)tiles_x * tiles_y));
        const int trem = (int)(tile % ((int64_t)tiles_x * tiles_y));
        const int x0 = (trem % tiles_x) * TW, y0 = (trem / tiles_x) * TH;
        const TS* zi = z + (int64_t)img * 3 * H * W;
        __syncthreads();  // previous tile finished with the shared buffers
        // ---- stage the RGB tile (clamped) ----
        for (int i = tid; i < 3 * ZH * ZW; i += NT) {
            int c = i / (ZH * ZW), r = (i / ZW) % ZH, q = i % ZW;
            int gy = clampi(y0 - HZ + r, 0, H - 1), gx = clampi(x0 - HZ + q, 0, W - 1);
            const int64_t o = ((int64_t)c * H + gy) * W + gx;
            zs[i] = mdn_in(o, 3 * (int64_t)H * W, 201) && mdn_in(img, nimg, 202) ? ld_f(zi, o) : 0.f;
        }
        if constexpr (FILTER && RC >= 0) {
            const TS* ci = coarse + (int64_t)img * 3 * Hc * Wc;
            const int cx0 = x0 / 2 - RC, cy0 = y0 / 2 - RC;
            for (int i = tid; i < UH * UW; i += NT) {
                int r = i / UW, q = i % UW;
                int gy = clampi(cy0 + r, 0, Hc - 1), gx = clampi(cx0 + q, 0, Wc - 1);
                int64_t o = (int64_t)gy * Wc + gx;
                if (!mdn_in(o, (int64_t)Hc * Wc, 203)) o = 0;
                float cr, cg, cb;
                rgb_to_work(ld_f(ci, o), ld_f(ci, o + (int64_t)Hc * Wc), ld_f(ci, o + 2 * (int64_t)Hc * Wc), color,
                            cr, cg, cb);
                us[i] = cr; us[UH * UW + i] = cg; us[2 * UH * UW + i] = cb;
            }
        }
        __syncthreads();
        // ---- products of central-difference gradients at clamped positions ----
        for (int i = tid; i < PH * PW; i += NT) {
            int r = i / PW, q = i % PW;
            int cy = clampi(y0 - 2 + r, 0, H - 1), cx = clampi(x0 - 2 + q, 0, W - 1);
            int ly = cy - (y0 - HZ), lx = cx - (x0 - HZ);
            int lxm = clampi(cx - 1, 0, W - 1) - (x0 - HZ), lxp = clampi(cx + 1, 0, W - 1) - (x0 - HZ);
            int lym = clampi(cy - 1, 0, H - 1) - (y0 - HZ), lyp = clampi(cy + 1, 0, H - 1) - (y0 - HZ);
            float gx[3], gy[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float* zc = zs + c * ZH * ZW;
                gx[c] = __fmul_rn(__fsub_rn(zc[ly * ZW + lxp], zc[ly * ZW + lxm]), 0.5f);
                gy[c] = __fmul_rn(__fsub_rn(zc[lyp * ZW + lx], zc[lym * ZW + lx]), 0.5f);
            }
            float pxx = __fmul_rn(gx[0], gx[0]), pxy = __fmul_rn(gx[0], gy[0]), pyy = __fmul_rn(gy[0], gy[0]);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                pxx = __fmaf_rn(gx[c], gx[c], pxx);
                pxy = __fmaf_rn(gx[c], gy[c], pxy);
                pyy = __fmaf_rn(gy[c], gy[c], pyy);
            }
            ps[i] = pxx; ps[PH * PW + i] = pxy; ps[2 * PH * PW + i] = pyy;
        }
        __syncthreads();
        // ---- horizontal smoothing pass; RGB tile -> working colour space ----
        for (int i = tid; i < 3 * PH * TW; i += NT) {
            int f = i / (PH * TW), r = (i / TW) % PH, q = i % TW;
            const float* p = ps + f * PH * PW + r * PW + q;
            float acc = __fmul_rn(wv[0], p[0]);
#pragma unroll
            for (int u = 1; u < 5; ++u) acc = __fmaf_rn(wv[u], p[u], acc);
            hs[i] = acc;
        }
        if constexpr (FILTER) {
            for (int i = tid; i < ZH * ZW; i += NT) {
                float a, b, c;
                rgb_to_work(zs[i], zs[ZH * ZW + i], zs[2 * ZH * ZW + i], color, a, b, c);
                zs[i] = a; zs[ZH * ZW + i] = b; zs[2 * ZH * ZW + i] = c;
            }
        }
        __syncthreads();
        // ---- vertical pass, features, bucket ----
        for (int i = tid; i < TH * TW; i += NT) {
            int r = i / TW, q = i % TW;
            float t3[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const float* p = hs + f * PH * TW + r * TW + q;
                float acc = __fmul_rn(wv[0], p[0]);
#pragma unroll
                for (int v = 1; v < 5; ++v) acc = __fmaf_rn(wv[v], p[v * TW], acc);
                t3[f] = acc;
            }
            int k = bucket_of(t3[0], t3[1], t3[2], sp);
            k = k < K ? k : K - 1;
            bk[i] = (uint16_t)k;
            int gy = y0 + r, gx = x0 + q;
            if (bmap && gy < H && gx < W && mdn_in(((int64_t)img * H + gy) * W + gx, (int64_t)nimg * H * W, 204)) {
                const int64_t o = ((int64_t)img * H + gy) * W + gx;
                if (wide) static_cast<uint16_t*>(bmap)[o] = (uint16_t)k;
                else static_cast<uint8_t*>(bmap)[o] = (uint8_t)k;
            }
        }
        if constexpr (FILTER) {
            __syncthreads();
            // ---- filtering ----
            TS* oi = out + (int64_t)img * 3 * H * W;
            for (int i = tid; i < TH * TW; i += NT) {
                int r = i / TW, q = i % TW;
                int gy = y0 + r, gx = x0 + q;
                if (gy >= H || gx >= W) continue;
                if (!mdn_in((int64_t)img * H * W + (int64_t)gy * W + gx, (int64_t)nimg * H * W, 205)) continue;
                const int k = mdn_in(bk[i], K, 206) ? bk[i] : 0;
                const float* zc = zs + (r + HZ) * ZW + (q + HZ);
                const float* uc = us + (r / 2 + (RC > 0 ? RC : 0)) * UW + (q / 2 + (RC > 0 ? RC : 0));
                float o[3];
#pragma unroll
                for (int oc = 0; oc < 3; ++oc) {
                    const TB* hb = SMEM ? bank_s + ((int64_t)k * 3 + oc) * BL::DP
                                        : bank + ((int64_t)k * 3 + oc) * G::D;
                    o[oc] = apply_filter<RF, RC, CROSS, TB, SMEM>(hb, zc, uc, oc, pair_ok);
                }
                float R, Gc, B;
                work_to_rgb(o[0], o[1], o[2], color, R, Gc, B);
                int64_t po = (int64_t)gy * W + gx;
                st_f(oi, po, R);
                st_f(oi, (int64_t)H * W + po, Gc);
                st_f(oi, 2 * (int64_t)H * W + po, B);
            }
        }
    }
}

template <int RF, int RC, bool CROSS, typename TS, typename TB, bool SMEM, bool FILTER>
int run(const LevelArgs& a, cudaStream_t s) {
    using G = Geo<RF, RC, CROSS>;
    using BL = BankLayout<TB, G::D>;
    auto kern = k_level<RF, RC, CROSS, TS, TB, SMEM, FILTER>;
    size_t bytes = ((tile_bytes<RC>() + 15) & ~size_t(15));
    if (FILTER && SMEM) bytes += sizeof(TB) * (size_t)a.K * 3 * BL::DP;
    int occ = 1;
    {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "k_level: set smem attribute");
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "k_level: occupancy");
        if (o < 1) return fail(MDN_ESHAPE, "k_level: shared memory footprint too large");
        occ = o;
    }
    const int64_t tiles = ((a.w + TW - 1) / TW) * ((a.h + TH - 1) / TH) * a.n;
    int64_t grid = (int64_t)num_sms() * occ;
    if (grid > tiles) grid = tiles;
    float w[5];
    gauss5_weights(w);
    kern<<<(unsigned)grid, NT, bytes, s>>>((const TS*)a.z, (const TS*)a.coarse, (TS*)a.out, a.buckets,
                                           (const TB*)a.bank, (int)a.h, (int)a.w, (int)a.hc, (int)a.wc,
                                           (int)a.n, a.K, a.geom.color, a.sel, w[0], w[1], w[2],
                                           G::D % 2 == 0 && (uintptr_t)a.bank % (2 * sizeof(TB)) == 0);
    return check_launch("k_level");
}

// bytes of shared memory the SMEM variant needs for K buckets
template <int RF, int RC, bool CROSS, typename TB> size_t smem_need(int K) {
    using G = Geo<RF, RC, CROSS>;
    using BL = BankLayout<TB, G::D>;
    return ((tile_bytes<RC>() + 15) & ~size_t(15)) + sizeof(TB) * (size_t)K * 3 * BL::DP;
}

// dynamic shared memory a kernel may use: the 227 KB opt-in maximum less
// what the kernels declare statically (sector boundary tables)
constexpr size_t SMEM_LIMIT = 232448 - 512;

// ==========================================================================
// Strip variant (v2): same selector stage; the filter stage gives every
// thread a vertical strip of PY pixels of one column, so that each loaded
// column of patch values (PY + 2r values) serves PY pixels and 2r+1 taps.
// Shared-memory bank layout: for bucket k, output channel oc, block b (the
// coarse then the fine patch of each input channel) and column dx, one
// 8-element slot holding the 2r+1 taps of that column (dy = -r..r, zero
// padded).  A slot is one 16-byte (FP16) or two 16-byte (FP32) loads; the
// per-bucket stride is an odd number of 16-byte units so that lanes with
// different buckets hit different bank groups.
// ==========================================================================
namespace v2 {

#ifndef MDN_V2_NT
#define MDN_V2_NT 384
#endif
#ifndef MDN_V2_PY
#define MDN_V2_PY 4
#endif

// Tile shape: 32 columns (one warp), NT threads, PY rows per thread strip.
template <int NT_, int PY_> struct Shape {
    static constexpr int TW = 32, NT = NT_, PY = PY_, NW = NT / 32, TH = NW * PY;
    static constexpr int HZ = 3;
    static constexpr int ZW = TW + 2 * HZ + 1, ZH = TH + 2 * HZ;   // row stride 39 (column 38 unused)
    static constexpr int PW = TW + 4, PH = TH + 4;
};
using DefShape = Shape<MDN_V2_NT, MDN_V2_PY>;

template <class SH, int RC> struct Coarse {
    static constexpr int UWD = RC >= 0 ? SH::TW / 2 + 2 * RC : 0;   // columns staged
    static constexpr int UW = RC >= 0 ? 27 : 0;                     // row stride (see the v3 consumer)
    static constexpr int UH = RC >= 0 ? SH::TH / 2 + 2 * RC : 0;
    static_assert(UWD <= 27, "coarse tile wider than its row stride");
};

template <int RF, int RC, bool CROSS> struct Slots {
    static constexpr int NCH = CROSS ? 3 : 1;
    static constexpr int PER_OC = NCH * ((RC >= 0 ? 2 * RC + 1 : 0) + (2 * RF + 1));
    static constexpr int S = 3 * PER_OC;    // slots per bucket
};

template <typename TB> struct SlotBytes;
template <> struct SlotBytes<float> { static constexpr int B = 32; };
template <> struct SlotBytes<__half> { static constexpr int B = 16; };

// per-bucket stride in 16-byte units: odd
template <int RF, int RC, bool CROSS, typename TB> constexpr int bucket_units() {
    int u = Slots<RF, RC, CROSS>::S * SlotBytes<TB>::B / 16;
    return (u % 2 == 1) ? u : u + 1;
}

template <class SH, int RC> constexpr size_t tile_bytes() {
    return sizeof(float) * (3 * SH::ZH * SH::ZW + 3 * SH::PH * SH::PW + 3 * SH::PH * SH::TW +
                            3 * Coarse<SH, RC>::UH * Coarse<SH, RC>::UW) +
           SH::TH * SH::TW;
}

template <class SH, int RF, int RC, bool CROSS, typename TB> size_t smem_need_s(int K) {
    return ((tile_bytes<SH, RC>() + 15) & ~size_t(15)) + (size_t)K * bucket_units<RF, RC, CROSS, TB>() * 16;
}
template <int RF, int RC, bool CROSS, typename TB> size_t smem_need(int K) {
    return smem_need_s<DefShape, RF, RC, CROSS, TB>(K);
}

// 8 taps of one slot as floats
template <typename TB> __device__ __forceinline__ void load_slot(const unsigned char* p, float h[8]);
template <> __device__ __forceinline__ void load_slot<__half>(const unsigned char* p, float h[8]) {
    uint4 q = *reinterpret_cast<const uint4*>(p);
    const __half2* hp = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float2 f = __half22float2(hp[e]);
        h[2 * e] = f.x; h[2 * e + 1] = f.y;
    }
}
template <> __device__ __forceinline__ void load_slot<float>(const unsigned char* p, float h[8]) {
    float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 16);
    h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w; h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
}

// bank [K][3][D] (regressor order) -> shared-memory slots, by nthreads
// threads; bucket k goes to slot block pos[k] (pos == nullptr: block k)
template <int RF, int RC, bool CROSS, typename TB>
__device__ __forceinline__ void load_bank_slots(const TB* __restrict__ bank, int K, unsigned char* bank_s, int tid,
                                                int nthreads, const uint8_t* pos = nullptr) {
    using G = Geo<RF, RC, CROSS>;
    using SL = Slots<RF, RC, CROSS>;
    constexpr int SB = SlotBytes<TB>::B;
    constexpr int BSTRIDE = bucket_units<RF, RC, CROSS, TB>() * 16;
    constexpr int NCX = RC >= 0 ? 2 * RC + 1 : 0;
    constexpr int NFX = 2 * RF + 1;
    constexpr int E = SB / (int)sizeof(TB);   // 8 elements per slot
    const int total = K * SL::S * E;
    for (int i = tid; i < total; i += nthreads) {
        const int e = i % E, slot = (i / E) % SL::S, k = i / (E * SL::S);
        const int oc = slot / SL::PER_OC, sr = slot % SL::PER_OC;
        int src = -1;
        if (sr < G::NCH * NCX) {                    // coarse block of channel cc
            const int cc = sr / (NCX > 0 ? NCX : 1), dx = sr % (NCX > 0 ? NCX : 1);
            if (e < NCX) src = cc * G::PC + e * NCX + dx;
        } else {
            const int t = sr - G::NCH * NCX;
            const int cc = t / NFX, dx = t % NFX;
            if (e < NFX) src = G::NCH * G::PC + cc * G::PF + e * NFX + dx;
        }
        TB v = src >= 0 ? bank[((int64_t)k * 3 + oc) * G::D + src] : TB(0.f);
        const int kp = pos ? pos[k] : k;
        reinterpret_cast<TB*>(bank_s + (size_t)kp * BSTRIDE + slot * SB)[e] = v;
    }
}

// Placement of bucket k = (a * ns + s) * nc + c in the shared-memory bank:
// with a per-bucket stride of 43 x 16 bytes, block p starts in 16-byte bank
// group 3p mod 8.  Choosing p = pi(k) with pi(k) = 3 g mod 8 (mod 8), g = a + 2s
// + 4c, puts every two buckets within +-1 of each other in angle, strength and
// coherence bin (the ones that sit side by side in a quarter-warp) in
// different bank groups.  pi is a bijection when every residue of 3g mod 8 has
// K/8 buckets (true for n_angle divisible by 8, ns, nc <= 3); otherwise the
// identity is used.  Built once per CTA by `nthreads` threads into pos[256].
__device__ __forceinline__ void build_bucket_placement(const SelParams& sp, int K, uint8_t* pos, int tid,
                                                       int nthreads) {
    const int ns = sp.n_strength, nc = sp.n_coherence;
    const bool ok = (sp.n_angle % 8 == 0) && ns <= 3 && nc <= 3 && K % 8 == 0 && K <= 256;
    for (int k = tid; k < K; k += nthreads) {
        if (!ok) { pos[k] = (uint8_t)k; continue; }
        auto cls = [&](int q) {
            const int a = q / (ns * nc), s = (q / nc) % ns, c = q % nc;
            return (3 * ((a + 2 * s + 4 * c) & 7)) & 7;
        };
        const int r = cls(k);
        int rank = 0;
        for (int q = 0; q < k; ++q) rank += cls(q) == r ? 1 : 0;
        pos[k] = (uint8_t)(8 * rank + r);
    }
}

}  // namespace v2
namespace v3 {
template <int RF, int RC, bool CROSS, typename TB, bool GLOBAL = false, bool CL = false>
__device__ __forceinline__ void filter_group(const float* __restrict__ zb, int zpl, int zst,
                                             const float* __restrict__ ub, int upl, int ust,
                                             const unsigned char* __restrict__ bank_s, const int (&kb)[8], int j,
                                             float o[3], uint32_t cb0 = 0, uint32_t cb1 = 0, int ckh = 0);
}  // namespace v3
namespace v2 {

// One TW x TH tile at (x0, y0) of one image: stage, select, filter, store.
// ROWS = false: strip filter on the column-slot bank (load_bank_slots);
// ROWS = true: the lane-group filter of v3 (v3::filter_group) on the row-slot
// bank (v3::load_bank_rows), whose outputs are bit-identical to k_level3's.
// smem: tile buffers (tile_bytes<SH, RC>()); bank_s: the bank's slots.
// zi/ci/oi: this image's planes; bmap_img: its bucket map or nullptr.
template <class SH, int RF, int RC, bool CROSS, typename TS, typename TB, bool ROWS = false>
__device__ __forceinline__ void tile_v2(unsigned char* smem, const unsigned char* bank_s, const TS* __restrict__ zi,
                                        const TS* __restrict__ ci, TS* __restrict__ oi, uint8_t* __restrict__ bmap_img,
                                        int H, int W, int Hc, int Wc, int x0, int y0, int K, int color,
                                        const SelParams& sp, const float wv[5]) {
    using G = Geo<RF, RC, CROSS>;
    using SL = Slots<RF, RC, CROSS>;
    constexpr int TW = SH::TW, TH = SH::TH, NT = SH::NT, PY = SH::PY, HZ = SH::HZ;
    constexpr int ZW = SH::ZW, ZH = SH::ZH, PW = SH::PW, PH = SH::PH;
    constexpr int UW = Coarse<SH, RC>::UW, UH = Coarse<SH, RC>::UH;
    constexpr int SB = SlotBytes<TB>::B;
    constexpr int BSTRIDE = bucket_units<RF, RC, CROSS, TB>() * 16;
    float* zs = reinterpret_cast<float*>(smem);             // [3][ZH][ZW]
    float* ps = zs + 3 * ZH * ZW;                            // [3][PH][PW]
    float* hs = ps + 3 * PH * PW;                            // [3][PH][TW]
    float* us = hs + 3 * PH * TW;                            // [3][UH][UW]
    uint8_t* bk = reinterpret_cast<uint8_t*>(us + 3 * UH * UW);  // [TH][TW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 3 * ZH * ZW; i += NT) {
        int c = i / (ZH * ZW), r = (i / ZW) % ZH, q = i % ZW;
        int gy = clampi(y0 - HZ + r, 0, H - 1), gx = clampi(x0 - HZ + q, 0, W - 1);
        const int64_t o = ((int64_t)c * H + gy) * W + gx;
        zs[i] = mdn_in(o, 3 * (int64_t)H * W, 401) ? ld_f(zi, o) : 0.f;
    }
    if constexpr (RC >= 0) {
        constexpr int UWD = Coarse<SH, RC>::UWD;
        const int cx0 = x0 / 2 - RC, cy0 = y0 / 2 - RC;
        for (int i = tid; i < UH * UWD; i += NT) {
            int r = i / UWD, q = i % UWD;
            int gy = clampi(cy0 + r, 0, Hc - 1), gx = clampi(cx0 + q, 0, Wc - 1);
            int64_t o = (int64_t)gy * Wc + gx;
            if (!mdn_in(o, (int64_t)Hc * Wc, 402)) o = 0;
            float a, b, c;
            rgb_to_work(ld_f(ci, o), ld_f(ci, o + (int64_t)Hc * Wc), ld_f(ci, o + 2 * (int64_t)Hc * Wc), color, a, b,
                        c);
            const int e = r * UW + q;
            us[e] = a; us[UH * UW + e] = b; us[2 * UH * UW + e] = c;
        }
    }
    __syncthreads();
    for (int i = tid; i < PH * PW; i += NT) {
        int r = i / PW, q = i % PW;
        int cy = clampi(y0 - 2 + r, 0, H - 1), cx = clampi(x0 - 2 + q, 0, W - 1);
        int ly = cy - (y0 - HZ), lx = cx - (x0 - HZ);
        int lxm = clampi(cx - 1, 0, W - 1) - (x0 - HZ), lxp = clampi(cx + 1, 0, W - 1) - (x0 - HZ);
        int lym = clampi(cy - 1, 0, H - 1) - (y0 - HZ), lyp = clampi(cy + 1, 0, H - 1) - (y0 - HZ);
        float gx[3], gy[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* zc = zs + c * ZH * ZW;
            gx[c] = __fmul_rn(__fsub_rn(zc[ly * ZW + lxp], zc[ly * ZW + lxm]), 0.5f);
            gy[c] = __fmul_rn(__fsub_rn(zc[lyp * ZW + lx], zc[lym * ZW + lx]), 0.5f);
        }
        float pxx = __fmul_rn(gx[0], gx[0]), pxy = __fmul_rn(gx[0], gy[0]), pyy = __fmul_rn(gy[0], gy[0]);
#pragma unroll
        for (int c = 1; c < 3; ++c) {
            pxx = __fmaf_rn(gx[c], gx[c], pxx);
            pxy = __fmaf_rn(gx[c], gy[c], pxy);
            pyy = __fmaf_rn(gy[c], gy[c], pyy);
        }
        ps[i] = pxx; ps[PH * PW + i] = pxy; ps[2 * PH * PW + i] = pyy;
    }
    __syncthreads();
    for (int i = tid; i < 3 * PH * TW; i += NT) {
        int f = i / (PH * TW), r = (i / TW) % PH, q = i % TW;
        const float* p = ps + f * PH * PW + r * PW + q;
        float acc = __fmul_rn(wv[0], p[0]);
#pragma unroll
        for (int u = 1; u < 5; ++u) acc = __fmaf_rn(wv[u], p[u], acc);
        hs[i] = acc;
    }
    for (int i = tid; i < ZH * ZW; i += NT) {
        float a, b, c;
        rgb_to_work(zs[i], zs[ZH * ZW + i], zs[2 * ZH * ZW + i], color, a, b, c);
        zs[i] = a; zs[ZH * ZW + i] = b; zs[2 * ZH * ZW + i] = c;
    }
    __syncthreads();
    for (int i = tid; i < TH * TW; i += NT) {
        int r = i / TW, q = i % TW;
        float t3[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const float* p = hs + f * PH * TW + r * TW + q;
            float acc = __fmul_rn(wv[0], p[0]);
#pragma unroll
            for (int v = 1; v < 5; ++v) acc = __fmaf_rn(wv[v], p[v * TW], acc);
            t3[f] = acc;
        }
        int k = bucket_of(t3[0], t3[1], t3[2], sp);
        k = k < K ? k : K - 1;
        bk[i] = (uint8_t)k;
        int gy = y0 + r, gx = x0 + q;
        if (bmap_img && gy < H && gx < W) bmap_img[(int64_t)gy * W + gx] = (uint8_t)k;
    }
    __syncthreads();
    if constexpr (ROWS) {
        // ---- filtering: warps cover 2 rows x 16 columns per pass, lane groups of 8 ----
        constexpr int NW = NT / 32;
        static_assert(NW % 2 == 0 && TH % NW == 0, "passes of NW rows must cover the tile");
        const int g = lane >> 3, j = lane & 7, ro = g >> 1, c0 = 16 * (warp & 1) + 8 * (g & 1);
#pragma unroll 1
        for (int pass = 0; pass < TH / NW; ++pass) {
            const int r = 2 * ((warp >> 1) + (NW / 2) * pass) + ro;
            const uint2 kbw = *reinterpret_cast<const uint2*>(bk + r * TW + c0);
            int kb[8];
#pragma unroll
            for (int p = 0; p < 8; ++p) kb[p] = (int)(((p < 4 ? kbw.x : kbw.y) >> (8 * (p & 3))) & 0xffu);
#ifdef MDN_CHECK
            const bool ok = mdn_in(r + HZ + RF, ZH, 403) && mdn_in(c0 + HZ + RF + 7, ZW, 404) &&
                            (RC < 0 || (mdn_in(r / 2 + 2 * (RC > 0 ? RC : 0), UH, 405) &&
                                        mdn_in(c0 / 2 + 3 + 2 * (RC > 0 ? RC : 0), UW, 406)));
            for (int p = 0; p < 8; ++p)
                if (!mdn_in(kb[p], K, 407)) kb[p] = 0;
            const int rr_ = ok ? r : 0, cc_ = ok ? c0 : 0;
#else
            const int rr_ = r, cc_ = c0;
#endif
            float o[3];
            v3::filter_group<RF, RC, CROSS, TB>(zs + (rr_ + HZ - RF) * ZW + cc_ + HZ - RF, ZH * ZW, ZW,
                                                 us + (rr_ / 2) * UW + cc_ / 2, UH * UW, UW, bank_s, kb, j, o);
            const int gy = y0 + r, gx = x0 + c0 + j;
            if (gy < H && gx < W) {
                float R, Gc, B;
                work_to_rgb(o[0], o[1], o[2], color, R, Gc, B);
                const int64_t po = (int64_t)gy * W + gx;
                st_f(oi, po, R);
                st_f(oi, (int64_t)H * W + po, Gc);
                st_f(oi, 2 * (int64_t)H * W + po, B);
            }
        }
        return;
    }
    // ---- filtering: lane = column, warp = strip of PY rows ----
    const int q = lane, r0 = warp * PY;
    const unsigned char* hb[PY];
#pragma unroll
    for (int p = 0; p < PY; ++p) hb[p] = bank_s + (size_t)bk[(r0 + p) * TW + q] * BSTRIDE;
    float o[3][PY];
#pragma unroll
    for (int oc = 0; oc < 3; ++oc) {
        float acc[PY];
#pragma unroll
        for (int p = 0; p < PY; ++p) acc[p] = 0.f;
        int slot = oc * SL::PER_OC;
        if constexpr (RC >= 0) {
            constexpr int NCR = PY / 2 + 2 * RC;     // coarse rows touched by the strip
#pragma unroll
            for (int cc = 0; cc < G::NCH; ++cc) {
                const int c = CROSS ? cc : oc;
                const float* ub = us + c * UH * UW + (r0 / 2) * UW + (q / 2) + RC;
#pragma unroll
                for (int dx = -RC; dx <= RC; ++dx, ++slot) {
                    float col[NCR];
#pragma unroll
                    for (int j = 0; j < NCR; ++j) col[j] = ub[j * UW + dx];
#pragma unroll
                    for (int p = 0; p < PY; ++p) {
                        float h[8];
                        load_slot<TB>(hb[p] + slot * SB, h);
#pragma unroll
                        for (int dy = 0; dy < 2 * RC + 1; ++dy) acc[p] = fmaf(h[dy], col[p / 2 + dy], acc[p]);
                    }
                }
            }
        }
#pragma unroll
        for (int cc = 0; cc < G::NCH; ++cc) {
            const int c = CROSS ? cc : oc;
            const float* zb = zs + c * ZH * ZW + (r0 + HZ - RF) * ZW + q + HZ;
#pragma unroll
            for (int dx = -RF; dx <= RF; ++dx, ++slot) {
                float col[PY + 2 * RF];
#pragma unroll
                for (int j = 0; j < PY + 2 * RF; ++j) col[j] = zb[j * ZW + dx];
#pragma unroll
                for (int p = 0; p < PY; ++p) {
                    float h[8];
                    load_slot<TB>(hb[p] + slot * SB, h);
#pragma unroll
                    for (int dy = 0; dy < 2 * RF + 1; ++dy) acc[p] = fmaf(h[dy], col[p + dy], acc[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PY; ++p) o[oc][p] = acc[p];
    }
    const int gx = x0 + q;
#pragma unroll
    for (int p = 0; p < PY; ++p) {
        const int gy = y0 + r0 + p;
        if (gy < H && gx < W) {
            float R, Gc, B;
            work_to_rgb(o[0][p], o[1][p], o[2][p], color, R, Gc, B);
            int64_t po = (int64_t)gy * W + gx;
            st_f(oi, po, R);
            st_f(oi, (int64_t)H * W + po, Gc);
            st_f(oi, 2 * (int64_t)H * W + po, B);
        }
    }
}

template <class SH, int RF, int RC, bool CROSS, typename TS, typename TB>
__global__ void __launch_bounds__(SH::NT, 1) k_level2(const TS* __restrict__ z, const TS* __restrict__ coarse,
                                                      TS* __restrict__ out, uint8_t* __restrict__ bmap,
                                                      const TB* __restrict__ bank, int H, int W, int Hc, int Wc,
                                                      int nimg, int K, int color, SelParams sp, float w0, float w1,
                                                      float w2) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* bank_s = smem + ((tile_bytes<SH, RC>() + 15) & ~size_t(15));
    const float wv[5] = {w0, w1, w2, w1, w0};
    load_bank_slots<RF, RC, CROSS, TB>(bank, K, bank_s, threadIdx.x, SH::NT);
    const int tiles_x = (W + SH::TW - 1) / SH::TW, tiles_y = (H + SH::TH - 1) / SH::TH;
    const int64_t ntiles = (int64_t)tiles_x * tiles_y * nimg;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int img = (int)(tile / ((int64_t)tiles_x * tiles_y));
        const int trem = (int)(tile % ((int64_t)tiles_x * tiles_y));
        const int x0 = (trem % tiles_x) * SH::TW, y0 = (trem / tiles_x) * SH::TH;
        __syncthreads();   // bank slots loaded / previous tile finished with the shared buffers
        tile_v2<SH, RF, RC, CROSS, TS, TB>(smem, bank_s, z + (int64_t)img * 3 * H * W,
                                           RC >= 0 ? coarse + (int64_t)img * 3 * Hc * Wc : nullptr,
                                           out + (int64_t)img * 3 * H * W,
                                           bmap ? bmap + (int64_t)img * H * W : nullptr, H, W, Hc, Wc, x0, y0, K,
                                           color, sp, wv);
    }
}

template <int RF, int RC, bool CROSS, typename TS, typename TB>
int run2(const LevelArgs& a, cudaStream_t s) {
    using SH = DefShape;
    auto kern = k_level2<SH, RF, RC, CROSS, TS, TB>;
    const size_t bytes = smem_need_s<SH, RF, RC, CROSS, TB>(a.K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_level2: set smem attribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SH::NT, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_level2: occupancy");
    if (occ < 1) return fail(MDN_ESHAPE, "k_level2: shared memory footprint too large");
    const int64_t tiles = ((a.w + SH::TW - 1) / SH::TW) * ((a.h + SH::TH - 1) / SH::TH) * a.n;
    int64_t grid = (int64_t)num_sms() * occ;
    if (grid > tiles) grid = tiles;
    float w[5];
    gauss5_weights(w);
    kern<<<(unsigned)grid, SH::NT, bytes, s>>>((const TS*)a.z, (const TS*)a.coarse, (TS*)a.out, (uint8_t*)a.buckets,
                                               (const TB*)a.bank, (int)a.h, (int)a.w, (int)a.hc, (int)a.wc,
                                               (int)a.n, a.K, a.geom.color, a.sel, w[0], w[1], w[2]);
    return check_launch("k_level2");
}

}  // namespace v2

// ==========================================================================
// Warp-specialised variant (v3).  Producer warps (8) stage tile t+1 (global
// loads, tensor, features, buckets, RGB -> working space) into one of two
// shared-memory stages while consumer warps (8) filter tile t from the other
// stage.
//
// Consumer mapping (conflict-free by construction).  A consumer warp covers
// 2 tile rows x 16 columns; its 4 groups of 8 lanes take (row offset g >> 1,
// columns 8 (g & 1) .. + 7), and lane j of a group is filter row dy = j - r
// of a block of radius r (lanes j > 2r idle).  The bank holds one 16-byte
// ROW slot per (bucket, output channel, block, dy) with the 2r+1 taps of
// that row (dx = -r..r), so at every coefficient load the active lanes of a
// group read consecutive 16-byte slots of one bucket -- one wavefront per
// group whatever the buckets of the neighbouring pixels.  Each lane keeps its
// patch row (8 + 2r values; coarse: 4 + 2r) in registers for the group's 8
// pixels; the row strides (39 fine, 27 coarse floats) put the rows and
// column groups a warp reads in distinct banks, and the two row offsets of a
// warp read the same coarse row (broadcast).  The per-lane partial sums of
// the 8 pixels x 3 channels are reduce-scattered over the group with
// shuffles, leaving pixel j's three channels in lane j, so a warp's stores
// cover 2 rows x 16 consecutive columns.
// Hand-off uses named barriers:
//   FULL[s]  : producers bar.arrive, consumers bar.sync   (128 + 256 threads)
//   EMPTY[s] : consumers bar.arrive, producers bar.sync   (256 + 128 threads)
//   PROD     : producer-internal bar.sync (128 threads)
// Every CTA computes the same tile count T for both roles; producers wait on
// EMPTY[i%2] only for i >= 2 and consumers arrive on EMPTY[i%2] only when
// i + 2 < T, so every barrier generation receives exactly 384 threads and
// generations are ordered (a consumer reaches tile i's arrival only after
// tile i's FULL, which follows the producer's EMPTY wait for tile i).
// ==========================================================================
namespace v3 {

constexpr int TW = 32, TH = 32;
constexpr int NCW = 8, NPW = 8;                 // consumer / producer warps
constexpr int NC = NCW * 32, NP = NPW * 32, NT = NC + NP;
constexpr int HZ = 3;
constexpr int ZW = TW + 2 * HZ + 1, ZH = TH + 2 * HZ;   // row stride 39 (odd; column 38 is not read)
constexpr int PW = TW + 4, PH = TH + 4;
constexpr int PX = 8;                           // pixels per lane group
static_assert(NCW * 32 == 8 * TW && TH % 8 == 0, "a consumer pass (8 warps x 2 rows x 16 columns) covers 8 tile rows");

enum { BAR_FULL0 = 1, BAR_EMPTY0 = 3, BAR_PROD = 5 };

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

template <int RC> struct Coarse {
    static constexpr int UWD = RC >= 0 ? TW / 2 + 2 * RC : 0;   // columns staged
    static constexpr int UW = RC >= 0 ? 27 : 0;                 // row stride (conflict-free coarse rows)
    static constexpr int UH = RC >= 0 ? TH / 2 + 2 * RC : 0;
    static_assert(UWD <= 27, "coarse radius too large for the row stride");
};

// Row-slot bank layout: for bucket k, output channel oc, the coarse blocks of
// the input channels, then their fine blocks; one slot per block row dy
// holding taps dx = -r..r (zero padded to 8 elements).
template <int RF, int RC, bool CROSS> struct RowSlots {
    static constexpr int NCH = CROSS ? 3 : 1;
    static constexpr int NCR = RC >= 0 ? 2 * RC + 1 : 0, NFR = 2 * RF + 1;
    static constexpr int PER_OC = NCH * (NCR + NFR);
    static constexpr int S = 3 * PER_OC;                  // slots per bucket
};
template <int RF, int RC, bool CROSS, typename TB> constexpr int bucket_bytes_rows() {
    return RowSlots<RF, RC, CROSS>::S * v2::SlotBytes<TB>::B;
}

template <int RF, int RC, bool CROSS, typename TB>
__device__ __forceinline__ void load_bank_rows(const TB* __restrict__ bank, int K, unsigned char* bank_s, int tid,
                                               int nthreads) {
    using G = Geo<RF, RC, CROSS>;
    using SL = RowSlots<RF, RC, CROSS>;
    constexpr int SB = v2::SlotBytes<TB>::B;
    constexpr int E = SB / (int)sizeof(TB);   // 8 elements per slot
    constexpr int BB = bucket_bytes_rows<RF, RC, CROSS, TB>();
    const int total = K * SL::S * E;
    for (int i = tid; i < total; i += nthreads) {
        const int e = i % E, slot = (i / E) % SL::S, k = i / (E * SL::S);
        const int oc = slot / SL::PER_OC, sr = slot % SL::PER_OC;
        int src = -1;
        if (sr < SL::NCH * SL::NCR) {              // coarse block of channel cc, row dyi
            const int cc = sr / (SL::NCR > 0 ? SL::NCR : 1), dyi = sr % (SL::NCR > 0 ? SL::NCR : 1);
            if (e < SL::NCR) src = cc * G::PC + dyi * SL::NCR + e;
        } else {
            const int t = sr - SL::NCH * SL::NCR;
            const int cc = t / SL::NFR, dyi = t % SL::NFR;
            if (e < SL::NFR) src = SL::NCH * G::PC + cc * G::PF + dyi * SL::NFR + e;
        }
        const int64_t gi = ((int64_t)k * 3 + oc) * G::D + src;
        const TB v = src >= 0 && mdn_in(gi, (int64_t)K * 3 * G::D, 127) ? bank[gi] : TB(0.f);
        reinterpret_cast<TB*>(bank_s + (size_t)k * BB + slot * SB)[e] = v;
    }
}


// Filter of one lane group (8 consecutive pixels of one row, the calling
// lane being j = lane & 7): the per-lane partial sums over each block row
// dy = j - r, then a reduce-scatter over the group with shuffles, after which
// o[] holds the three working-space outputs of pixel j.  Every lane of the
// warp must call it (the shuffles use the full mask).
//   zb:  fine plane of input channel 0 at (patch row 0, patch column 0) of the
//        group's first pixel, i.e. (row r - RF, column c0 - RF) of the pixel
//        grid; zpl: plane stride; zst: row stride (floats, working space)
//   ub:  coarse plane of channel 0 at (row r/2, column c0/2) of the coarse
//        stage (whose origin is RC rows and columns before the coarse pixel of
//        the tile origin); upl, ust: plane and row strides
//   kb:  the 8 pixels' buckets
//   GLOBAL: the row-slot bank is in global memory (read through the
//        read-only cache, 16-byte loads) instead of shared memory
// The arithmetic (FMA order within a lane, reduction tree) is fixed, so any
// kernel calling this gives bit-identical outputs for the same inputs.
template <typename TB, bool GLOBAL> __device__ __forceinline__ void group_slot(const unsigned char* p, float h[8]) {
    if constexpr (!GLOBAL) {
        v2::load_slot<TB>(p, h);
    } else if constexpr (sizeof(TB) == 2) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
        const __half2* hp = reinterpret_cast<const __half2*>(&q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(hp[e]);
            h[2 * e] = f.x; h[2 * e + 1] = f.y;
        }
    } else {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p + 16));
        h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w; h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
    }
}

// An FP32 slot (8 floats, 32 bytes) of a bank held in the shared memory of
// a CTA of this cluster, by its shared::cluster address.
__device__ __forceinline__ void cluster_slot(uint32_t a, float h[8]) {
    uint32_t v[8];
    asm("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(a));
    asm("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(a + 16));
#pragma unroll
    for (int e = 0; e < 8; ++e) h[e] = __uint_as_float(v[e]);
}

// CL: the bank is split over the two CTAs of a cluster by bucket (buckets
// below ckh in CTA 0, the rest in CTA 1, each at the start of its bank
// area), cb0 / cb1 the shared::cluster addresses of the two areas.
template <int RF, int RC, bool CROSS, typename TB, bool GLOBAL, bool CL>
__device__ __forceinline__ void filter_group(const float* __restrict__ zb, int zpl, int zst,
                                             const float* __restrict__ ub, int upl, int ust,
                                             const unsigned char* __restrict__ bank_s, const int (&kb)[8], int j,
                                             float o[3], uint32_t cb0, uint32_t cb1, int ckh) {
    using SL = RowSlots<RF, RC, CROSS>;
    constexpr int SB = v2::SlotBytes<TB>::B;
    constexpr int BSTRIDE = bucket_bytes_rows<RF, RC, CROSS, TB>();
    static_assert(!CL || (sizeof(TB) == 4 && !GLOBAL), "cluster banks: FP32 slots in shared memory");
    const unsigned FULL = 0xffffffffu;
    const unsigned char* hb[PX];
    uint32_t hc[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        if constexpr (CL) hc[p] = kb[p] < ckh ? cb0 + kb[p] * BSTRIDE : cb1 + (kb[p] - ckh) * BSTRIDE;
        else hb[p] = bank_s + (size_t)kb[p] * BSTRIDE;
    }
    float acc[3][PX];
#pragma unroll
    for (int oc = 0; oc < 3; ++oc)
#pragma unroll
        for (int p = 0; p < PX; ++p) acc[oc][p] = 0.f;
#pragma unroll
    for (int oc = 0; oc < 3; ++oc) {
        int slot = oc * SL::PER_OC;
        if constexpr (RC >= 0) {
            constexpr int NCOL = PX / 2 + 2 * RC;
#pragma unroll
            for (int cc = 0; cc < SL::NCH; ++cc, slot += SL::NCR) {
                const int c = CROSS ? cc : oc;
                if (j < SL::NCR) {
                    // coarse row r/2 + RC + dy (dy = j - RC); tap dx of pixel p at column k = p/2 + RC + dx
                    const float* src = ub + c * upl + j * ust;
                    float col[NCOL];
#pragma unroll
                    for (int k = 0; k < NCOL; ++k) col[k] = src[k];
#pragma unroll
                    for (int p = 0; p < PX; ++p) {
                        float h[8];
                        if constexpr (CL) cluster_slot(hc[p] + (slot + j) * SB, h);
                        else group_slot<TB, GLOBAL>(hb[p] + (slot + j) * SB, h);
#pragma unroll
                        for (int d = 0; d < SL::NCR; ++d) acc[oc][p] = fmaf(h[d], col[p / 2 + d], acc[oc][p]);
                    }
                }
            }
        }
        constexpr int NCOL = PX + 2 * RF;
#pragma unroll
        for (int cc = 0; cc < SL::NCH; ++cc, slot += SL::NFR) {
            const int c = CROSS ? cc : oc;
            if (j < SL::NFR) {
                // fine row r + dy (dy = j - RF); tap dx of pixel p at column k = p + RF + dx
                const float* src = zb + c * zpl + j * zst;
                float col[NCOL];
#pragma unroll
                for (int k = 0; k < NCOL; ++k) col[k] = src[k];
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    float h[8];
                    if constexpr (CL) cluster_slot(hc[p] + (slot + j) * SB, h);
                    else group_slot<TB, GLOBAL>(hb[p] + (slot + j) * SB, h);
#pragma unroll
                    for (int d = 0; d < SL::NFR; ++d) acc[oc][p] = fmaf(h[d], col[p + d], acc[oc][p]);
                }
            }
        }
    }
    // reduce-scatter over the group's 8 lanes: lane j keeps pixel j
    float w4[3][4], w2[3][2];
    const bool b2 = j & 4, b1 = j & 2, b0 = j & 1;
#pragma unroll
    for (int oc = 0; oc < 3; ++oc)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float keep = b2 ? acc[oc][q + 4] : acc[oc][q];
            const float send = b2 ? acc[oc][q] : acc[oc][q + 4];
            w4[oc][q] = keep + __shfl_xor_sync(FULL, send, 4);
        }
#pragma unroll
    for (int oc = 0; oc < 3; ++oc)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float keep = b1 ? w4[oc][q + 2] : w4[oc][q];
            const float send = b1 ? w4[oc][q] : w4[oc][q + 2];
            w2[oc][q] = keep + __shfl_xor_sync(FULL, send, 2);
        }
#pragma unroll
    for (int oc = 0; oc < 3; ++oc) {
        const float keep = b0 ? w2[oc][1] : w2[oc][0];
        const float send = b0 ? w2[oc][0] : w2[oc][1];
        o[oc] = keep + __shfl_xor_sync(FULL, send, 1);
    }
}

// stage: zs [3][ZH][ZW], us [3][UH][UW], then the bucket tile [TH][TW] of
// BTB-byte indices at a 16-byte aligned offset (8 indices = one vector load)
template <int RC> constexpr size_t bk_offset() {
    return (sizeof(float) * (3 * ZH * ZW + 3 * Coarse<RC>::UH * Coarse<RC>::UW) + 15) & ~size_t(15);
}
template <int RC, int BTB = 1> constexpr size_t stage_bytes() {
    return (bk_offset<RC>() + (size_t)TH * TW * BTB + 15) & ~size_t(15);
}
constexpr size_t scratch_bytes() { return sizeof(float) * (3 * PH * PW + 3 * PH * TW); }
template <int RC, int BTB = 1> constexpr size_t front_bytes() {
    return ((2 * stage_bytes<RC, BTB>() + scratch_bytes()) + 15) & ~size_t(15);
}
// GB: the bank stays in global memory (prepared row slots read through L2);
// BTB: bytes per bucket index in the stage (1, or 2 above 256 buckets)
template <int RF, int RC, bool CROSS, typename TB, bool GB = false, int BTB = 1> size_t smem_need(int K) {
    return front_bytes<RC, BTB>() + (GB ? 0 : (size_t)K * bucket_bytes_rows<RF, RC, CROSS, TB>());
}

// One TW x TH tile as the kernel sees it: the image it lies in (bases of
// the [3][H][W] input and output, the [3][Hc][Wc] coarse input, the [H][W]
// bucket map or null), its origin, and the bank and colour space of its item.
template <typename TS, typename BT> struct TileRef {
    const TS* z;
    const TS* coarse;
    TS* out;
    BT* bmap;
    const unsigned char* bank;   // prepared row slots (bank read through L2), else unused
    int H, W, Hc, Wc, x0, y0, K, color, item;
};

// Tile source of a batch of n equal-size images with one bank: tiles in
// image-major, row-major order.
template <typename TS, typename BT> struct BatchTiles {
    const TS* z;
    const TS* coarse;
    TS* out;
    BT* bmap;
    const unsigned char* bank;
    int H, W, Hc, Wc, nimg, K, color, tiles_x, tiles_y;
    SelParams sp;
    __device__ __forceinline__ int64_t count() const { return (int64_t)tiles_x * tiles_y * nimg; }
    __device__ __forceinline__ TileRef<TS, BT> at(int64_t tile) const {
        const int img = (int)(tile / ((int64_t)tiles_x * tiles_y));
        const int trem = (int)(tile % ((int64_t)tiles_x * tiles_y));
        TileRef<TS, BT> t;
        t.z = z + (int64_t)img * 3 * H * W;
        t.coarse = coarse ? coarse + (int64_t)img * 3 * Hc * Wc : nullptr;
        t.out = out + (int64_t)img * 3 * H * W;
        t.bmap = bmap ? bmap + (int64_t)img * H * W : nullptr;
        t.bank = bank;
        t.H = H; t.W = W; t.Hc = Hc; t.Wc = Wc;
        t.x0 = (trem % tiles_x) * TW;
        t.y0 = (trem / tiles_x) * TH;
        t.K = mdn_in(img, nimg, 104) ? K : 0;
        t.color = color;
        t.item = 0;
        return t;
    }
    __device__ __forceinline__ const SelParams& sel(int) const { return sp; }
};

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// CL: launched in clusters of two CTAs, the (FP32) bank split between them
// by bucket; each CTA loads its half, and the consumers read every slot by
// its shared::cluster address.  Every CTA passes the same two cluster
// barriers (after the load, before exit), whatever its tile count.
template <int RF, int RC, bool CROSS, typename TS, typename TB, bool GB, typename BT, class SRC, bool CL = false>
__global__ void __launch_bounds__(NT, 1) k_level3(const __grid_constant__ SRC src, const TB* __restrict__ bank,
                                                  float w0, float w1, float w2, int rows_in) {
    using SL = RowSlots<RF, RC, CROSS>;
    constexpr int UW = Coarse<RC>::UW, UH = Coarse<RC>::UH, UWD = Coarse<RC>::UWD;
    constexpr int SB = v2::SlotBytes<TB>::B;
    constexpr int BSTRIDE = bucket_bytes_rows<RF, RC, CROSS, TB>();
    constexpr size_t SBY = stage_bytes<RC, (int)sizeof(BT)>();
    extern __shared__ __align__(16) unsigned char smem[];
    float* ps = reinterpret_cast<float*>(smem + 2 * SBY);   // producer scratch [3][PH][PW]
    float* hs = ps + 3 * PH * PW;                             // [3][PH][TW]
    unsigned char* bank_sm = smem + front_bytes<RC, (int)sizeof(BT)>();   // bank in shared memory (!GB)
    const int tid = threadIdx.x;

    if constexpr (!GB) {
        int K = src.K;   // shared-memory banks: batch sources only
        const TB* b = bank;
        int skip = 0;    // buckets before this CTA's part (CL: the other CTA's half)
        if constexpr (CL) {
            uint32_t rank;
            asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
            const int kh = (K + 1) / 2;
            skip = rank ? kh : 0;
            K = rank ? K - kh : kh;
            b = bank + (size_t)skip * 3 * Geo<RF, RC, CROSS>::D;
        }
        if (rows_in) {   // prepared row slots: a straight 16-byte copy
            const uint4* r = reinterpret_cast<const uint4*>(bank) + (size_t)skip * BSTRIDE / 16;
            for (int i = tid; i < K * BSTRIDE / 16; i += NT) reinterpret_cast<uint4*>(bank_sm)[i] = __ldg(r + i);
        } else {
            load_bank_rows<RF, RC, CROSS, TB>(b, K, bank_sm, tid, NT);
        }
    }   // once per persistent CTA
    __syncthreads();
    uint32_t cb0 = 0, cb1 = 0;
    int ckh = 0;
    if constexpr (CL) {
        cluster_sync_all();   // both halves are loaded before any CTA reads the other's
        const uint32_t local = (uint32_t)__cvta_generic_to_shared(bank_sm);
        asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(cb0) : "r"(local));
        asm volatile("mapa.shared::cluster.u32 %0, %1, 1;" : "=r"(cb1) : "r"(local));
        ckh = (src.K + 1) / 2;
    }

    const int64_t ntiles = src.count();
    const int64_t T = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int warp = tid >> 5, lane = tid & 31;

    if (warp >= NCW) {
        // =============================== producer ===============================
        const int pt = tid - NC;
        const int pw = pt >> 5;                       // producer warp 0..NPW-1
        const float wv[5] = {w0, w1, w2, w1, w0};
        // Register prefetch: the inputs of tile i+1 are loaded while tile i's
        // selector runs, so global latency overlaps shared-memory work.
        // Interior tiles (halo inside the image, rows 8-byte aligned) load
        // 4-element chunks covering columns x0-4 .. x0+35 without clamping;
        // border tiles use clamped scalar loads.
        constexpr int NCHUNK = 10;                    // 4-element chunks per staged row
        constexpr int NZV = (3 * ZH * NCHUNK + NP - 1) / NP;
        constexpr int NZS = (3 * ZH * ZW + NP - 1) / NP;
        constexpr int NZ = NZV * 4 > NZS ? NZV * 4 : NZS;
        constexpr int NU = RC >= 0 ? (UH * UWD + NP - 1) / NP : 0;
        float zreg[NZ];
        float ureg[NU > 0 ? NU : 1][3];
        // vector loads need 4-element-aligned rows and an aligned image base
        auto interior = [&](const TileRef<TS, BT>& t) {
            const bool rows_aligned = (t.W % 4) == 0 && (reinterpret_cast<uintptr_t>(t.z) & 15) == 0;
            return rows_aligned && t.x0 - 4 >= 0 && t.x0 + TW + 4 <= t.W && t.y0 - HZ >= 0 && t.y0 + TH + HZ <= t.H;
        };
        auto fetch = [&](int64_t tile) {
            const TileRef<TS, BT> t = src.at(tile);
            const int x0 = t.x0, y0 = t.y0, H = t.H, W = t.W, Hc = t.Hc, Wc = t.Wc;
            const TS* zi = t.z;
            if (interior(t)) {
#pragma unroll
                for (int j = 0; j < NZV; ++j) {
                    const int e = pt + j * NP;
                    if (e < 3 * ZH * NCHUNK) {
                        const int c = e / (ZH * NCHUNK), r = (e / NCHUNK) % ZH, k = e % NCHUNK;
                        const TS* src = zi + ((int64_t)c * H + (y0 - HZ + r)) * W + (x0 - 4 + 4 * k);
                        if (mdn_in(y0 - HZ + r, H, 101) && mdn_in(x0 - 4 + 4 * k, W - 3, 102)) ld4(src, zreg + 4 * j);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < NZS; ++j) {
                    const int e = pt + j * NP;
                    if (e < 3 * ZH * ZW) {
                        int c = e / (ZH * ZW), r = (e / ZW) % ZH, q = e % ZW;
                        int gy = clampi(y0 - HZ + r, 0, H - 1), gx = clampi(x0 - HZ + q, 0, W - 1);
                        const int64_t o = ((int64_t)c * H + gy) * W + gx;
                        zreg[j] = mdn_in(o, 3 * (int64_t)H * W, 103) && t.K > 0 ? ld_f(zi, o) : 0.f;
                    }
                }
            }
            if constexpr (RC >= 0) {
                const TS* ci = t.coarse;
                const int cx0 = x0 / 2 - RC, cy0 = y0 / 2 - RC;
#pragma unroll
                for (int j = 0; j < NU; ++j) {
                    const int e = pt + j * NP;
                    if (e < UH * UWD) {
                        int r = e / UWD, q = e % UWD;
                        int gy = clampi(cy0 + r, 0, Hc - 1), gx = clampi(cx0 + q, 0, Wc - 1);
                        int64_t o = (int64_t)gy * Wc + gx;
                        if (!mdn_in(o, (int64_t)Hc * Wc, 105)) o = 0;
                        ureg[j][0] = ld_f(ci, o);
                        ureg[j][1] = ld_f(ci, o + (int64_t)Hc * Wc);
                        ureg[j][2] = ld_f(ci, o + 2 * (int64_t)Hc * Wc);
                    }
                }
            }
        };
        if (T > 0) fetch(blockIdx.x);
        for (int64_t i = 0; i < T; ++i) {
            const int s = (int)(i & 1);
            if (i >= 2) bar_sync(BAR_EMPTY0 + s, NT);
            float* zs = reinterpret_cast<float*>(smem + s * SBY);
            float* us = zs + 3 * ZH * ZW;
            BT* bk = reinterpret_cast<BT*>(smem + s * SBY + bk_offset<RC>());
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const TileRef<TS, BT> t = src.at(tile);
            const int x0 = t.x0, y0 = t.y0, H = t.H, W = t.W, K = t.K, color = t.color;
            const SelParams& sp = src.sel(t.item);
            const bool inner = interior(t);
            if (inner) {
                // chunk k covers staged columns 4k-1 .. 4k+2 (column -1 and >= ZW dropped)
#pragma unroll
                for (int j = 0; j < NZV; ++j) {
                    const int e = pt + j * NP;
                    if (e < 3 * ZH * NCHUNK) {
                        const int cr = e / NCHUNK, k = e % NCHUNK;
                        float* row = zs + cr * ZW;
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int q = 4 * k - 1 + t;
                            if (q >= 0 && q < ZW && mdn_in(cr * ZW + q, 3 * ZH * ZW, 106)) row[q] = zreg[4 * j + t];
                        }
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < NZS; ++j) {
                    const int e = pt + j * NP;
                    if (e < 3 * ZH * ZW && mdn_in(e, 3 * ZH * ZW, 107)) zs[e] = zreg[j];
                }
            }
            if constexpr (RC >= 0) {
#pragma unroll
                for (int j = 0; j < NU; ++j) {
                    const int e = pt + j * NP;
                    if (e < UH * UWD) {
                        float a, b, c;
                        rgb_to_work(ureg[j][0], ureg[j][1], ureg[j][2], color, a, b, c);
                        const int o = (e / UWD) * UW + e % UWD;
                        if (mdn_in(o, UH * UW, 108)) { us[o] = a; us[UH * UW + o] = b; us[2 * UH * UW + o] = c; }
                    }
                }
            }
            if (i + 1 < T) fetch(tile + gridDim.x);
            bar_sync(BAR_PROD, NP);
            // products of central-difference gradients at the PH x PW positions,
            // spread flat over the producer threads (consecutive lanes along x).
            // Interior tiles: a thread takes the two positions (2m, q), (2m+1, q),
            // whose gradients share four of their twelve staged values
            auto prod = [&](const float (&gx)[3], const float (&gy)[3], int e) {
                float pxx = __fmul_rn(gx[0], gx[0]), pxy = __fmul_rn(gx[0], gy[0]), pyy = __fmul_rn(gy[0], gy[0]);
#pragma unroll
                for (int c = 1; c < 3; ++c) {
                    pxx = __fmaf_rn(gx[c], gx[c], pxx);
                    pxy = __fmaf_rn(gx[c], gy[c], pxy);
                    pyy = __fmaf_rn(gy[c], gy[c], pyy);
                }
                if (mdn_in(e, PH * PW, 109)) { ps[e] = pxx; ps[PH * PW + e] = pxy; ps[2 * PH * PW + e] = pyy; }
            };
            if (inner) {
                static_assert(PH % 2 == 0, "row pairs");
                for (int e0 = pt; e0 < (PH / 2) * PW; e0 += NP) {
                    const int m = e0 / PW, q = e0 - m * PW;
                    int ly = 2 * m + 1, lx = q + 1;   // staged position of product (2m, q)
                    if (!(mdn_in(ly - 1, ZH - 2, 110) && mdn_in(lx - 1, ZW - 2, 111))) ly = lx = 1;
                    float gx0[3], gy0[3], gx1[3], gy1[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float* zc = zs + c * ZH * ZW + ly * ZW + lx;
                        const float um = zc[-ZW], c0v = zc[0], c1v = zc[ZW], dn = zc[2 * ZW];
                        gx0[c] = __fmul_rn(__fsub_rn(zc[1], zc[-1]), 0.5f);
                        gy0[c] = __fmul_rn(__fsub_rn(c1v, um), 0.5f);
                        gx1[c] = __fmul_rn(__fsub_rn(zc[ZW + 1], zc[ZW - 1]), 0.5f);
                        gy1[c] = __fmul_rn(__fsub_rn(dn, c0v), 0.5f);
                    }
                    prod(gx0, gy0, 2 * m * PW + q);
                    prod(gx1, gy1, (2 * m + 1) * PW + q);
                }
            }
            for (int e0 = pt; !inner && e0 < PH * PW; e0 += NP) {   // border tiles: clamped positions
                {
                    const int r = e0 / PW, q = e0 - r * PW;
                    const int cy = clampi(y0 - 2 + r, 0, H - 1), cx = clampi(x0 - 2 + q, 0, W - 1);
                    const int ly = cy - (y0 - HZ), lx = cx - (x0 - HZ);
                    const int lxm = clampi(cx - 1, 0, W - 1) - (x0 - HZ), lxp = clampi(cx + 1, 0, W - 1) - (x0 - HZ);
                    int lym = clampi(cy - 1, 0, H - 1) - (y0 - HZ), lyp = clampi(cy + 1, 0, H - 1) - (y0 - HZ);
                    int lyc = ly, lxc = lx, lxmc = lxm, lxpc = lxp;
                    if (!(mdn_in(lym, ZH, 112) && mdn_in(lyp, ZH, 112) && mdn_in(lyc, ZH, 112) &&
                          mdn_in(lxmc, ZW, 113) && mdn_in(lxpc, ZW, 113) && mdn_in(lxc, ZW, 113)))
                        lym = lyp = lyc = lxc = lxmc = lxpc = 0;
                    float gx[3], gy[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float* zc = zs + c * ZH * ZW;
                        gx[c] = __fmul_rn(__fsub_rn(zc[lyc * ZW + lxpc], zc[lyc * ZW + lxmc]), 0.5f);
                        gy[c] = __fmul_rn(__fsub_rn(zc[lyp * ZW + lxc], zc[lym * ZW + lxc]), 0.5f);
                    }
                    prod(gx, gy, e0);
                }
            }
            bar_sync(BAR_PROD, NP);
            // horizontal smoothing pass: each thread makes 4 consecutive outputs
            // of one (field, row) from two 16-byte loads of its 8 inputs
            static_assert(PW % 4 == 0 && TW % 4 == 0, "16-byte rows");
            for (int e = pt; e < 3 * PH * (TW / 4); e += NP) {
                int fr = e / (TW / 4), q = 4 * (e - fr * (TW / 4));
                if (!(mdn_in(fr * PW + q + 7, 3 * PH * PW, 114) && mdn_in(fr * TW + q + 3, 3 * PH * TW, 115))) fr = q = 0;
                const float4 a4 = *reinterpret_cast<const float4*>(ps + fr * PW + q);
                const float4 b4 = *reinterpret_cast<const float4*>(ps + fr * PW + q + 4);
                const float p8[8] = {a4.x, a4.y, a4.z, a4.w, b4.x, b4.y, b4.z, b4.w};
                float o4[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float acc = __fmul_rn(wv[0], p8[t]);
#pragma unroll
                    for (int u = 1; u < 5; ++u) acc = __fmaf_rn(wv[u], p8[t + u], acc);
                    o4[t] = acc;
                }
                *reinterpret_cast<float4*>(hs + fr * TW + q) = make_float4(o4[0], o4[1], o4[2], o4[3]);
            }
            // RGB tile -> working colour space, flat over the producer threads
            // (the unused pad column is converted too)
            for (int e = pt; e < ZH * ZW; e += NP) {
                if (!mdn_in(e, ZH * ZW, 116)) continue;
                float a, b, c;
                rgb_to_work(zs[e], zs[ZH * ZW + e], zs[2 * ZH * ZW + e], color, a, b, c);
                zs[e] = a; zs[ZH * ZW + e] = b; zs[2 * ZH * ZW + e] = c;
            }
            bar_sync(BAR_PROD, NP);
            // vertical pass, features, bucket: producer warp pw takes the 4
            // consecutive rows 4 pw .. 4 pw + 3, lanes along x, with the five
            // smoothing rows of each field held in a sliding register window
            // (same products and sums, in the same order, as five loads)
            static_assert(TH == 4 * NPW, "4 output rows per producer warp");
            float win[3][4];
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    win[f][v] = mdn_in(4 * pw + v + 4, PH, 117) ? hs[f * PH * TW + (4 * pw + v) * TW + lane] : 0.f;
            float ta[4], tb[4], tc[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int r = 4 * pw + rr;
                float t3[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float nxt = mdn_in(r + 4, PH, 118) ? hs[f * PH * TW + (r + 4) * TW + lane] : 0.f;
                    float acc = __fmul_rn(wv[0], win[f][0]);
#pragma unroll
                    for (int v = 1; v < 4; ++v) acc = __fmaf_rn(wv[v], win[f][v], acc);
                    acc = __fmaf_rn(wv[4], nxt, acc);
                    t3[f] = acc;
#pragma unroll
                    for (int v = 0; v < 3; ++v) win[f][v] = win[f][v + 1];
                    win[f][3] = nxt;
                }
                ta[rr] = t3[0]; tb[rr] = t3[1]; tc[rr] = t3[2];
            }
            int kk[4];
            buckets_of<4>(ta, tb, tc, sp, kk);   // the four rows' selectors overlap
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int r = 4 * pw + rr;
                const int k = kk[rr] < K ? kk[rr] : (K > 0 ? K - 1 : 0);
                if (mdn_in(r * TW + lane, TH * TW, 119)) bk[r * TW + lane] = (BT)k;
                const int gy = y0 + r, gx = x0 + lane;
                const int64_t mo = (int64_t)gy * W + gx;
                if (t.bmap && gy < H && gx < W && mdn_in(mo, (int64_t)H * W, 120)) t.bmap[mo] = (BT)k;
            }
            bar_arrive(BAR_FULL0 + s, NT);
        }
    } else {
        // =============================== consumer ===============================
        const int g = lane >> 3, j = lane & 7;
        const int ro = g >> 1, c0 = 16 * (warp & 1) + 8 * (g & 1);   // row offset, first column of the group
        for (int64_t i = 0; i < T; ++i) {
            const int s = (int)(i & 1);
            bar_sync(BAR_FULL0 + s, NT);
            const float* zs = reinterpret_cast<const float*>(smem + s * SBY);
            const float* us = zs + 3 * ZH * ZW;
            const BT* bk = reinterpret_cast<const BT*>(smem + s * SBY + bk_offset<RC>());
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const TileRef<TS, BT> t = src.at(tile);
            const int x0 = t.x0, y0 = t.y0, H = t.H, W = t.W;
            TS* oi = t.out;
            const unsigned char* bank_s = GB ? t.bank : bank_sm;
            const int K = t.K;
#pragma unroll 1
            for (int pass = 0; pass < TH / 8; ++pass) {
                const int r = 2 * ((warp >> 1) + 4 * pass) + ro;          // tile row of this group
                int kb[8];
                if constexpr (sizeof(BT) == 1) {
                    const uint2 w8 = *reinterpret_cast<const uint2*>(bk + r * TW + c0);
#pragma unroll
                    for (int p = 0; p < 8; ++p) kb[p] = (int)(((p < 4 ? w8.x : w8.y) >> (8 * (p & 3))) & 0xffu);
                } else {
                    const uint4 w16 = *reinterpret_cast<const uint4*>(bk + r * TW + c0);
                    const uint32_t wv4[4] = {w16.x, w16.y, w16.z, w16.w};
#pragma unroll
                    for (int p = 0; p < 8; ++p) kb[p] = (int)((wv4[p >> 1] >> (16 * (p & 1))) & 0xffffu);
                }
#ifdef MDN_CHECK
                // every patch row and column the group reads, and its buckets
                const bool fine_ok = mdn_in(r + HZ + RF, ZH, 121) && mdn_in(c0 + HZ + RF + PX - 1, ZW, 122);
                const bool coarse_ok = RC < 0 || (mdn_in(r / 2 + 2 * (RC > 0 ? RC : 0), UH, 123) &&
                                                  mdn_in(c0 / 2 + PX / 2 + 2 * (RC > 0 ? RC : 0) - 1, UW, 124));
                for (int p = 0; p < 8; ++p)
                    if (!mdn_in(kb[p], K, 125)) kb[p] = 0;
                const int rr_ = fine_ok && coarse_ok ? r : 0, cc_ = fine_ok && coarse_ok ? c0 : 0;
#else
                const int rr_ = r, cc_ = c0;
#endif
                float o[3];
                filter_group<RF, RC, CROSS, TB, GB, CL>(zs + (rr_ + HZ - RF) * ZW + cc_ + HZ - RF, ZH * ZW, ZW,
                                                     us + (rr_ / 2) * UW + cc_ / 2, UH * UW, UW, bank_s, kb, j, o,
                                                     cb0, cb1, ckh);
                if (pass == TH / 8 - 1 && i + 2 < T) bar_arrive(BAR_EMPTY0 + s, NT);   // stage s no longer read
                const int gy = y0 + r, gx = x0 + c0 + j;
                if (gy < H && gx < W && mdn_in((int64_t)gy * W + gx, (int64_t)H * W, 126)) {
                    float R, Gc, B;
                    work_to_rgb(o[0], o[1], o[2], t.color, R, Gc, B);
                    const int64_t po = (int64_t)gy * W + gx;
                    st_f(oi, po, R);
                    st_f(oi, (int64_t)H * W + po, Gc);
                    st_f(oi, 2 * (int64_t)H * W + po, B);
                }
            }
        }
    }
    if constexpr (CL) cluster_sync_all();   // no CTA leaves while its partner may still read its half
}

template <int RF, int RC, bool CROSS, typename TS, typename TB, bool GB = false, typename BT = uint8_t>
int run3(const LevelArgs& a, cudaStream_t s) {
    using SRC = BatchTiles<TS, BT>;
    auto kern = k_level3<RF, RC, CROSS, TS, TB, GB, BT, SRC>;
    const size_t bytes = smem_need<RF, RC, CROSS, TB, GB, (int)sizeof(BT)>(a.K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_level3: set smem attribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_level3: occupancy");
    if (occ < 1) return fail(MDN_ESHAPE, "k_level3: shared memory footprint too large");
    const int64_t tiles = ((a.w + TW - 1) / TW) * ((a.h + TH - 1) / TH) * a.n;
    int64_t grid = (int64_t)num_sms() * occ;
    if (grid > tiles) grid = tiles;
    float w[5];
    gauss5_weights(w);
    SRC src;
    src.z = (const TS*)a.z;
    src.coarse = (const TS*)a.coarse;
    src.out = (TS*)a.out;
    src.bmap = (BT*)a.buckets;
    src.bank = (const unsigned char*)a.bank;
    src.H = (int)a.h; src.W = (int)a.w; src.Hc = (int)a.hc; src.Wc = (int)a.wc;
    src.nimg = (int)a.n; src.K = a.K; src.color = a.geom.color;
    src.tiles_x = (int)((a.w + TW - 1) / TW);
    src.tiles_y = (int)((a.h + TH - 1) / TH);
    src.sp = a.sel;
    kern<<<(unsigned)grid, NT, bytes, s>>>(src, (const TB*)a.bank, w[0], w[1], w[2], a.bank_rows ? 1 : 0);
    return check_launch("k_level3");
}

// Shared memory of the cluster form: the stages plus half the FP32 bank (rounded up).
template <int RF, int RC, bool CROSS> size_t smem_need_cluster(int K) {
    return front_bytes<RC, 1>() + (size_t)((K + 1) / 2) * bucket_bytes_rows<RF, RC, CROSS, float>();
}

// The fused kernel in clusters of two CTAs with an FP32 bank split between them.
template <int RF, int RC, bool CROSS, typename TS>
int run3_cluster(const LevelArgs& a, cudaStream_t s) {
    using SRC = BatchTiles<TS, uint8_t>;
    auto kern = k_level3<RF, RC, CROSS, TS, float, false, uint8_t, SRC, true>;
    const size_t bytes = smem_need_cluster<RF, RC, CROSS>(a.K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_level3 (cluster): set smem attribute");
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * (unsigned)num_sms());
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return cuda_fail(e, "k_level3 (cluster): occupancy");
    if (nclusters < 1) return fail(MDN_ESHAPE, "k_level3 (cluster): no cluster of two fits");
    const int64_t tiles = ((a.w + TW - 1) / TW) * ((a.h + TH - 1) / TH) * a.n;
    int64_t grid = 2 * (int64_t)nclusters;
    if (grid > tiles + (tiles & 1)) grid = tiles + (tiles & 1);   // whole clusters; a CTA may get no tile
    cfg.gridDim = dim3((unsigned)grid);
    float w[5];
    gauss5_weights(w);
    SRC src;
    src.z = (const TS*)a.z;
    src.coarse = (const TS*)a.coarse;
    src.out = (TS*)a.out;
    src.bmap = (uint8_t*)a.buckets;
    src.bank = (const unsigned char*)a.bank;
    src.H = (int)a.h; src.W = (int)a.w; src.Hc = (int)a.hc; src.Wc = (int)a.wc;
    src.nimg = (int)a.n; src.K = a.K; src.color = a.geom.color;
    src.tiles_x = (int)((a.w + TW - 1) / TW);
    src.tiles_y = (int)((a.h + TH - 1) / TH);
    src.sp = a.sel;
    e = cudaLaunchKernelEx(&cfg, kern, src, (const float*)a.bank, w[0], w[1], w[2], a.bank_rows ? 1 : 0);
    if (e != cudaSuccess) return cuda_fail(e, "k_level3 (cluster): launch");
    return check_launch("k_level3 (cluster)");
}

}  // namespace v3


#ifndef MDN_USE_V3
#define MDN_USE_V3 1
#endif

// Whether level-kernel variant v applies to this call.
template <int RF, int RC, bool CROSS, typename TB> bool variant_ok(const LevelArgs& a, int v) {
    const bool small = a.K <= 256;
    switch (v) {
        case LV_FUSED_SMEM: return small && v3::smem_need<RF, RC, CROSS, TB>(a.K) <= SMEM_LIMIT;
        case LV_FUSED_L2: return a.bank_rows;
        case LV_STRIP: return !a.bank_rows && small && v2::smem_need<RF, RC, CROSS, TB>(a.K) <= SMEM_LIMIT;
        case LV_TILE_SMEM: return !a.bank_rows && smem_need<RF, RC, CROSS, TB>(a.K) <= SMEM_LIMIT;
        case LV_TILE_L2: return !a.bank_rows;
        case LV_FUSED_CLUSTER:
            return sizeof(TB) == 4 && a.K >= 2 && small && v3::smem_need_cluster<RF, RC, CROSS>(a.K) <= SMEM_LIMIT;
        default: return false;
    }
}

template <int RF, int RC, bool CROSS, typename TS, typename TB>
int run_variant(const LevelArgs& a, int v, cudaStream_t s) {
    switch (v) {
        case LV_FUSED_SMEM: return v3::run3<RF, RC, CROSS, TS, TB, false, uint8_t>(a, s);   // plain or prepared bank
        case LV_FUSED_L2:
            return a.K <= 256 ? v3::run3<RF, RC, CROSS, TS, TB, true, uint8_t>(a, s)
                              : v3::run3<RF, RC, CROSS, TS, TB, true, uint16_t>(a, s);
        case LV_STRIP: return v2::run2<RF, RC, CROSS, TS, TB>(a, s);
        case LV_TILE_SMEM: return run<RF, RC, CROSS, TS, TB, true, true>(a, s);
        case LV_FUSED_CLUSTER:
            if constexpr (sizeof(TB) == 4) return v3::run3_cluster<RF, RC, CROSS, TS>(a, s);
            return fail(MDN_ESHAPE, "filter_level: cluster banks are FP32");
        default: return run<RF, RC, CROSS, TS, TB, false, true>(a, s);
    }
}

// One compiled geometry: the forced variant (the tuner), else the autotune
// table's entry, else the static rule.  Plain banks ([K][3][D]): the fused
// kernel with the bank in shared memory when it fits, else the strip or tile
// kernels.  Prepared banks (row slots, mdn_prepare_bank_rows): the fused
// kernel, with the bank copied to shared memory when it fits and read
// through L2 otherwise.  The cluster form (an FP32 bank split over two CTAs)
// runs only when forced or chosen by the autotuner.
template <int RF, int RC, bool CROSS, typename TS, typename TB>
int dispatch_geo(const LevelArgs& a, cudaStream_t s) {
    if (a.variant >= 0) {
        if (!variant_ok<RF, RC, CROSS, TB>(a, a.variant))
            return fail(MDN_ESHAPE, "filter_level: this level-kernel variant does not apply to the call");
        return run_variant<RF, RC, CROSS, TS, TB>(a, a.variant, s);
    }
    const int t = tune_lookup(a);
    if (t >= 0 && variant_ok<RF, RC, CROSS, TB>(a, t)) return run_variant<RF, RC, CROSS, TS, TB>(a, t, s);
    // (the cluster form of FP32 banks is the tuner's to choose: reading every
    // slot across the pair, it measured 4x slower than the L2 form)
    if (a.bank_rows)
        return run_variant<RF, RC, CROSS, TS, TB>(
            a, variant_ok<RF, RC, CROSS, TB>(a, LV_FUSED_SMEM) ? LV_FUSED_SMEM : LV_FUSED_L2, s);
    for (int v : {LV_FUSED_SMEM, LV_STRIP, LV_TILE_SMEM})
        if ((v != LV_FUSED_SMEM || MDN_USE_V3) && variant_ok<RF, RC, CROSS, TB>(a, v))
            return run_variant<RF, RC, CROSS, TS, TB>(a, v, s);
    return run_variant<RF, RC, CROSS, TS, TB>(a, LV_TILE_L2, s);
}

// Geometry dispatch for one (storage, bank) type pair.
template <typename TS, typename TB> int dispatch(const LevelArgs& a, cudaStream_t s) {
    const mdn_geometry& g = a.geom;
#define MDN_GEO(RF_, RC_, CR_)                                                   \
    if (g.r_fine == RF_ && g.r_coarse == RC_ && (g.cross_channel != 0) == CR_) \
        return dispatch_geo<RF_, RC_, CR_, TS, TB>(a, s);
    MDN_GEO(2, -1, false)
    MDN_GEO(3, 3, false)
    MDN_GEO(3, 2, false)
    MDN_GEO(3, -1, true)
    MDN_GEO(2, 1, false)
#undef MDN_GEO
    return fail(MDN_ESHAPE, "filter_level: geometry not compiled (supported: r_fine/r_coarse/cross = "
                            "2/-1/0, 3/3/0, 3/2/0, 3/-1/1, 2/1/0)");
}

}  // namespace lvl
}  // namespace mdn
