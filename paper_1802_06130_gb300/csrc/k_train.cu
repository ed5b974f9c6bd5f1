// k_train.cu -- A5/A6: bucketed least-squares training (Eqs. 5-6).
//
// Pipeline for one level (all on the stream, no host synchronisation):
//   k_to_work      storage RGB -> FP32 working colour space (z, coarse, target)
//   k_hist         per-block bucket histograms of the bucket map
//   k_scan         bucket-major exclusive scan -> stable scatter offsets and
//                  the chunk table (bucket, begin, end), chunks <= CHUNK rows
//   k_scatter      stable counting-sort scatter of pixel indices by bucket
//   Gram           per chunk: A^T A of the gathered rows A = [regressor|target
//                  shifted by a per-channel constant | 1] (SIMT FP32 here,
//                  tcgen05 variants in k_gram_tc.cu), written as FP32 partials
//   k_reduce_centered  FP64 sum of a bucket's partials in chunk order
//                  (deterministic) with the exact centring correction, added
//                  into gram[k][g]; counts[k] += n_k
//   k_pool/k_chol  ridge solve (G_xx/n + lambda I) h = G_xy/n by Cholesky in
//                  FP64 shared memory, one CTA per (bucket, group); empty
//                  buckets copy the pooled solution
#include "common.cuh"
#include "internal.h"
#include "train_common.cuh"

namespace mdn {
namespace trn {

// ---------------------------------------------------------------- helpers

template <typename TS>
__global__ void k_to_work(const TS* __restrict__ in, float* __restrict__ out, int64_t hw, int64_t n, int color) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= hw * n) return;
    int64_t img = i / hw, p = i % hw;
    const TS* s = in + img * 3 * hw + p;
    float r = ld_f(s, 0), g = ld_f(s, hw), b = ld_f(s, 2 * hw);
    float y, cb, cr;
    if (color == MDN_RGB) { y = r; cb = g; cr = b; }
    else {
        y = 0.299f * r + 0.587f * g + 0.114f * b;
        cb = -0.168735892f * r - 0.331264108f * g + 0.5f * b;
        cr = 0.5f * r - 0.418687589f * g - 0.081312411f * b;
    }
    float* d = out + img * 3 * hw + p;
    d[0] = y; d[hw] = cb; d[2 * hw] = cr;
}

__global__ void k_hist(const uint8_t* __restrict__ bmap, int64_t npix, int K, int* __restrict__ blockhist) {
    __shared__ int h[MDN_MAX_K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) h[k] = 0;
    __syncthreads();
    int64_t b0 = (int64_t)blockIdx.x * SORT_CHUNK;
    int64_t e = b0 + SORT_CHUNK < npix ? b0 + SORT_CHUNK : npix;
    for (int64_t i = b0 + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&h[bmap[i]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) blockhist[(int64_t)blockIdx.x * K + k] = h[k];
}

// One CTA.  offs[b][k] = start of block b's bucket-k run in the sorted list;
// bstart[k], bcount[k]; chunk table entries (k, begin, end); nchunks_out.
__global__ void k_scan(const int* __restrict__ blockhist, int nblk, int K, int* __restrict__ offs,
                       int64_t* __restrict__ bstart, int64_t* __restrict__ bcount, int4* __restrict__ chunks,
                       int maxchunks, int chunk_rows, int* __restrict__ nchunks_out) {
    __shared__ int64_t tot[MDN_MAX_K];
    __shared__ int64_t cstart[MDN_MAX_K + 1];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int64_t s = 0;
        for (int b = 0; b < nblk; ++b) s += blockhist[(int64_t)b * K + k];
        tot[k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0, c = 0;
        for (int k = 0; k < K; ++k) {
            bstart[k] = run;
            bcount[k] = tot[k];
            cstart[k] = c;
            run += tot[k];
            c += (tot[k] + chunk_rows - 1) / chunk_rows;
        }
        cstart[K] = c;
        *nchunks_out = (int)c;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int64_t run = bstart[k];
        for (int b = 0; b < nblk; ++b) {
            offs[(int64_t)b * K + k] = (int)run;
            run += blockhist[(int64_t)b * K + k];
        }
        int64_t c = cstart[k];
        for (int64_t r = 0; r < tot[k]; r += chunk_rows, ++c) {
            if (c >= maxchunks) break;
            int64_t e = r + chunk_rows < tot[k] ? r + chunk_rows : tot[k];
            chunks[c] = make_int4(k, (int)(bstart[k] + r), (int)(bstart[k] + e), 0);
        }
    }
    // unused tail entries
    for (int64_t c = cstart[K] + threadIdx.x; c < maxchunks; c += blockDim.x) chunks[c] = make_int4(-1, 0, 0, 0);
}

// Stable scatter: pixels of a block are ranked in index order within their
// bucket (warp match + per-warp counts), so the sorted list is deterministic.
__global__ void __launch_bounds__(256) k_scatter(const uint8_t* __restrict__ bmap, int64_t npix, int K,
                                                 const int* __restrict__ offs, int* __restrict__ sorted) {
    __shared__ int run[MDN_MAX_K];
    __shared__ int wcnt[8][MDN_MAX_K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < K; k += blockDim.x) run[k] = offs[(int64_t)blockIdx.x * K + k];
    int64_t b0 = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int64_t base = b0; base < b0 + SORT_CHUNK; base += blockDim.x) {
        for (int i = threadIdx.x; i < 8 * MDN_MAX_K; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        int64_t i = base + threadIdx.x;
        bool valid = i < npix;
        int k = valid ? bmap[i] : 0x7fffffff - lane;   // invalid lanes never match a bucket
        unsigned m = __match_any_sync(0xffffffffu, k);
        int rank = __popc(m & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][k] = __popc(m);
        __syncthreads();
        if (valid) {
            int pos = run[k] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][k];
            sorted[pos] = (int)i;
        }
        __syncthreads();
        for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += wcnt[w][kk];
            run[kk] += s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- SIMT Gram

// Gram of one chunk, FP32 products/accumulation, 4x4 register blocks of the
// upper triangle of every group's Dp x Dp matrix.
__global__ void __launch_bounds__(256) k_gram_simt(GatherArgs ga, const int4* __restrict__ chunks,
                                                    const int* __restrict__ sorted, float* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 ch = chunks[blockIdx.x];
    if (ch.x < 0) return;
    const int Dq = ga.Dp + 1, G = ga.G, DPs = ga.Dp4;   // Dq: features + ones column
    float* As = reinterpret_cast<float*>(smem);        // [G][RB][DPs]
    int* coltab = reinterpret_cast<int*>(As + (size_t)G * GRAM_RB * DPs);   // [G][Dq]
    build_coltab(ga, coltab);
    const int nb = (Dq + 3) / 4;
    const int nblk_g = nb * (nb + 1) / 2;
    const int total = G * nblk_g;
    constexpr int MB = 8;   // max blocks per thread
    float acc[MB][16];
#pragma unroll
    for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[m][e] = 0.f;
    int bg[MB], bi[MB], bj[MB];
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        int id = threadIdx.x + m * blockDim.x;
        if (id < total) {
            int g = id / nblk_g, r = id % nblk_g;
            int i = 0;
            while (r >= nb - i) { r -= nb - i; ++i; }
            bg[m] = g; bi[m] = i; bj[m] = i + r;
        } else {
            bg[m] = -1; bi[m] = bj[m] = 0;
        }
    }
    __syncthreads();
    for (int r0 = ch.y; r0 < ch.z; r0 += GRAM_RB) {
        const int nr = ch.z - r0 < GRAM_RB ? ch.z - r0 : GRAM_RB;
        __syncthreads();
        gather_rows(ga, coltab, sorted + r0, nr, As, DPs, GRAM_RB);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            if (bg[m] < 0) continue;
            const float* Ab = As + (size_t)bg[m] * GRAM_RB * DPs;
            for (int r = 0; r < nr; ++r) {
                float4 a = *reinterpret_cast<const float4*>(Ab + r * DPs + bi[m] * 4);
                float4 b = *reinterpret_cast<const float4*>(Ab + r * DPs + bj[m] * 4);
                float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[m][p * 4 + q] = fmaf(av[p], bv[q], acc[m][p * 4 + q]);
            }
        }
    }
    float* out = partial + (size_t)blockIdx.x * G * Dq * Dq;
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        if (bg[m] < 0) continue;
        for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) {
                int i = bi[m] * 4 + p, j = bj[m] * 4 + q;
                if (i < Dq && j < Dq && i <= j) out[((size_t)bg[m] * Dq + i) * Dq + j] = acc[m][p * 4 + q];
            }
    }
}

// FP64 reduction of a bucket's chunk partials in chunk order (deterministic):
// partials are (Dq = Dp + 1)^2 upper triangles of the shifted rows with the
// ones column last; the exact centring correction is
// G_ij = S_ij + c_i s_j + c_j s_i + n c_i c_j, s_i = S_{i,ones}, n = S_{ones,ones}.
__global__ void k_reduce_centered(const float* __restrict__ partial, const int4* __restrict__ chunks,
                                  const int* __restrict__ nchunks, const int64_t* __restrict__ bcount, int K, int G,
                                  int Dp, int D, int rf, int rc, int cross, int color, double* __restrict__ gram,
                                  int64_t* __restrict__ counts) {
    const int k = blockIdx.y;
    const int Dq = Dp + 1;
    const int64_t entq = (int64_t)G * Dq * Dq;
    __shared__ int c0, c1;
    if (threadIdx.x == 0) {
        int nc = *nchunks, lo = 0, hi = nc;
        while (lo < hi) { int mid = (lo + hi) / 2; if (chunks[mid].x < k) lo = mid + 1; else hi = mid; }
        c0 = lo;
        hi = nc;
        while (lo < hi) { int mid = (lo + hi) / 2; if (chunks[mid].x <= k) lo = mid + 1; else hi = mid; }
        c1 = lo;
    }
    __syncthreads();
    const int64_t ent = (int64_t)G * Dp * Dp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ent; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / ((int64_t)Dp * Dp));
        const int i = (int)((e / Dp) % Dp), j = (int)(e % Dp);
        if (i > j) continue;
        double sij = 0.0, si = 0.0, sj = 0.0, n = 0.0;
        const size_t base = (size_t)g * Dq * Dq;
        for (int c = c0; c < c1; ++c) {
            const float* P = partial + (size_t)c * entq + base;
            sij += (double)P[(size_t)i * Dq + j];
            si += (double)P[(size_t)i * Dq + Dp];
            sj += (double)P[(size_t)j * Dq + Dp];
            n += (double)P[(size_t)Dp * Dq + Dp];
        }
        const double ci = channel_center(feature_channel(i, g, D, rf, rc, cross), color);
        const double cj = channel_center(feature_channel(j, g, D, rf, rc, cross), color);
        const double v = sij + ci * sj + cj * si + n * ci * cj;
        double* G0 = gram + (size_t)k * ent + (size_t)g * Dp * Dp;
        G0[(size_t)i * Dp + j] += v;
        if (i != j) G0[(size_t)j * Dp + i] += v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[k] += bcount[k];
}

// ---------------------------------------------------------------- solve

__global__ void k_pool(const double* __restrict__ gram, const int64_t* __restrict__ counts, int K, int64_t ent,
                       double* __restrict__ pooled, double* __restrict__ ntot) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ent; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += gram[(size_t)k * ent + e];
        pooled[e] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (double)counts[k];
        *ntot = s;
    }
}

// One CTA per (bucket, group); pooled_mode: solve only the pooled system
// (blockIdx.x == group) into pooled_h.  Otherwise buckets with n_k = 0 copy
// pooled_h.  bank_out FP32 [K][3][D].
__global__ void __launch_bounds__(256) k_chol(const double* __restrict__ gram, const int64_t* __restrict__ counts,
                                              const double* __restrict__ pooled, const double* __restrict__ ntot,
                                              int G, int D, int T, double lambda, int pooled_mode,
                                              double* __restrict__ pooled_h, float* __restrict__ bank_out,
                                              int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* A = reinterpret_cast<double*>(smem);   // [D][D]
    double* B = A + (size_t)D * D;                  // [D][T]
    const int Dp = D + T;
    int k, g;
    const double* Gm;
    double n;
    if (pooled_mode) {
        k = -1; g = blockIdx.x;
        Gm = pooled + (size_t)g * Dp * Dp;
        n = *ntot;
    } else {
        k = blockIdx.x / G; g = blockIdx.x % G;
        n = (double)counts[k];
        if (counts[k] == 0) {
            // pooled filter
            for (int t = 0; t < T; ++t) {
                int oc = T == 1 ? g : t;
                for (int p = threadIdx.x; p < D; p += blockDim.x)
                    bank_out[((size_t)k * 3 + oc) * D + p] = (float)pooled_h[(size_t)oc * D + p];
            }
            return;
        }
        Gm = gram + ((size_t)k * G + g) * Dp * Dp;
    }
    if (!(n > 0.0)) {
        if (threadIdx.x == 0) atomicAdd(status, 1);
        return;
    }
    const double inv = 1.0 / n;
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
        int p = e / D, q = e % D;
        A[e] = Gm[(size_t)p * Dp + q] * inv + (p == q ? lambda : 0.0);
    }
    for (int e = threadIdx.x; e < D * T; e += blockDim.x) {
        int p = e / T, t = e % T;
        B[e] = Gm[(size_t)p * Dp + D + t] * inv;
    }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // right-looking Cholesky, lower triangle: A = L L^T
    for (int j = 0; j < D; ++j) {
        if (threadIdx.x == 0) {
            double d = A[(size_t)j * D + j];
            if (!(d > 0.0)) { bad = 1; d = 1.0; }
            A[(size_t)j * D + j] = sqrt(d);
        }
        __syncthreads();
        const double ljj = A[(size_t)j * D + j];
        for (int i = j + 1 + threadIdx.x; i < D; i += blockDim.x) A[(size_t)i * D + j] /= ljj;
        __syncthreads();
        const int m = D - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = j + 1 + e / m, c = j + 1 + e % m;
            if (c <= i) A[(size_t)i * D + c] -= A[(size_t)i * D + j] * A[(size_t)c * D + j];
        }
        __syncthreads();
    }
    // L y = b, then L^T x = y, column by column
    for (int i = 0; i < D; ++i) {
        if (threadIdx.x < T) B[(size_t)i * T + threadIdx.x] /= A[(size_t)i * D + i];
        __syncthreads();
        for (int e = threadIdx.x; e < (D - i - 1) * T; e += blockDim.x) {
            int r = i + 1 + e / T, t = e % T;
            B[(size_t)r * T + t] -= A[(size_t)r * D + i] * B[(size_t)i * T + t];
        }
        __syncthreads();
    }
    for (int i = D - 1; i >= 0; --i) {
        if (threadIdx.x < T) B[(size_t)i * T + threadIdx.x] /= A[(size_t)i * D + i];
        __syncthreads();
        for (int e = threadIdx.x; e < i * T; e += blockDim.x) {
            int r = e / T, t = e % T;
            B[(size_t)r * T + t] -= A[(size_t)i * D + r] * B[(size_t)i * T + t];
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicAdd(status, 1);
    for (int t = 0; t < T; ++t) {
        int oc = T == 1 ? g : t;
        for (int p = threadIdx.x; p < D; p += blockDim.x) {
            double v = bad ? 0.0 : B[(size_t)p * T + t];
            if (pooled_mode) pooled_h[(size_t)oc * D + p] = v;
            else bank_out[((size_t)k * 3 + oc) * D + p] = (float)v;
        }
    }
}

}  // namespace trn

using namespace trn;

size_t train_ws_bytes(int64_t npix, int K, int G, int Dp, int precision) {
    (void)precision;
    int64_t nblk = (npix + SORT_CHUNK - 1) / SORT_CHUNK;
    int64_t maxch = npix / GRAM_CHUNK + K + 1;
    size_t b = 0;
    b += align256(sizeof(int) * nblk * K) * 2;        // blockhist, offs
    b += align256(sizeof(int64_t) * K) * 2;           // bstart, bcount
    b += align256(sizeof(int4) * maxch) + 256;        // chunks, nchunks
    b += align256(sizeof(int) * (npix > 0 ? npix : 1));   // sorted
    b += align256(sizeof(float) * maxch * G * (Dp + 1) * (Dp + 1));  // partials (tensor-core layout is Dp+1)
    return b;
}

int launch_gram(const TrainArgs& a, cudaStream_t s) {
    const int64_t hw = a.h * a.w, npix = a.n * hw;
    const int64_t hwc = a.hc * a.wc;
    if (a.Dp + 1 > GRAM_MAX_DP) return fail(MDN_ESHAPE, "train: regressor too long (D + T must be <= 159)");
    // carve the workspace
    char* p = (char*)a.ws;
    auto take = [&](size_t bytes) { char* r = p; p += align256(bytes); return r; };
    float* zw = (float*)take(sizeof(float) * 3 * npix);
    float* tw = (float*)take(sizeof(float) * 3 * npix);
    float* cw = (float*)take(sizeof(float) * 3 * a.n * hwc);
    int64_t nblk = (npix + SORT_CHUNK - 1) / SORT_CHUNK;
    int64_t maxch = npix / GRAM_CHUNK + a.K + 1;
    int* blockhist = (int*)take(sizeof(int) * nblk * a.K);
    int* offs = (int*)take(sizeof(int) * nblk * a.K);
    int64_t* bstart = (int64_t*)take(sizeof(int64_t) * a.K);
    int64_t* bcount = (int64_t*)take(sizeof(int64_t) * a.K);
    int4* chunks = (int4*)take(sizeof(int4) * maxch);
    int* nchunks = (int*)take(sizeof(int));
    int* sorted = (int*)take(sizeof(int) * (npix > 0 ? npix : 1));
    float* partial = (float*)take(sizeof(float) * maxch * a.G * (a.Dp + 1) * (a.Dp + 1));
    if ((size_t)(p - (char*)a.ws) > a.ws_bytes) return fail(MDN_EWORKSPACE, "train: workspace too small");

    const int TB = 256;
    auto conv = [&](const void* in, float* out, int64_t hw_, int64_t cnt) {
        unsigned g = (unsigned)((hw_ * cnt + TB - 1) / TB);
        if (a.dtype == MDN_F32) k_to_work<float><<<g, TB, 0, s>>>((const float*)in, out, hw_, cnt, a.geom.color);
        else k_to_work<__half><<<g, TB, 0, s>>>((const __half*)in, out, hw_, cnt, a.geom.color);
    };
    conv(a.z, zw, hw, a.n);
    conv(a.target, tw, hw, a.n);
    if (a.coarse) conv(a.coarse, cw, hwc, a.n);
    k_hist<<<(unsigned)nblk, TB, 0, s>>>(a.buckets, npix, a.K, blockhist);
    k_scan<<<1, TB, 0, s>>>(blockhist, (int)nblk, a.K, offs, bstart, bcount, chunks, (int)maxch, GRAM_CHUNK, nchunks);
    k_scatter<<<(unsigned)nblk, TB, 0, s>>>(a.buckets, npix, a.K, offs, sorted);
    int rc = check_launch("train: sort");
    if (rc) return rc;

    GatherArgs ga{};
    ga.zw = zw; ga.tw = tw; ga.cw = a.coarse ? cw : nullptr;
    ga.h = (int)a.h; ga.w = (int)a.w; ga.hc = (int)a.hc; ga.wc = (int)a.wc;
    ga.rf = a.geom.r_fine; ga.rc = a.geom.r_coarse; ga.cross = a.geom.cross_channel; ga.color = a.geom.color;
    ga.D = a.D; ga.T = a.T; ga.G = a.G; ga.Dp = a.Dp; ga.Dp4 = (a.Dp + 1 + 3) / 4 * 4;
    if (a.precision == MDN_GRAM_FP32) {
        size_t sm = sizeof(float) * (size_t)a.G * GRAM_RB * ga.Dp4 + sizeof(int) * a.G * (a.Dp + 1);
        const int nb = (a.Dp + 1 + 3) / 4;
        if (a.G * nb * (nb + 1) / 2 > 8 * 256) return fail(MDN_ESHAPE, "train: Gram too large for the SIMT path");
        cudaError_t ea = cudaFuncSetAttribute(k_gram_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (ea != cudaSuccess) return cuda_fail(ea, "k_gram_simt: shared memory attribute");
        k_gram_simt<<<(unsigned)maxch, 256, sm, s>>>(ga, chunks, sorted, partial);
        if ((rc = check_launch("k_gram_simt"))) return rc;
    } else {
        rc = launch_gram_tc(ga, a.precision, chunks, (int)maxch, sorted, partial, s);
        if (rc) return rc;
    }
    dim3 rg((unsigned)((a.G * a.Dp * a.Dp + 255) / 256), (unsigned)a.K);
    k_reduce_centered<<<rg, 256, 0, s>>>(partial, chunks, nchunks, bcount, a.K, a.G, a.Dp, a.D, a.geom.r_fine,
                                         a.geom.r_coarse, a.geom.cross_channel, a.geom.color, a.gram, a.counts);
    return check_launch("k_reduce_centered");
}

size_t solve_ws_bytes(int K, int G, int D, int T) {
    (void)K;
    size_t Dp = D + T;
    return align256(sizeof(double) * G * Dp * Dp) + align256(sizeof(double)) + align256(sizeof(double) * 3 * D);
}

int launch_solve(const double* gram, const int64_t* counts, int K, int G, int D, int T, double lambda,
                 float* bank_out, int32_t* status, void* ws, size_t ws_bytes, cudaStream_t s) {
    const int Dp = D + T;
    if (ws_bytes < solve_ws_bytes(K, G, D, T)) return fail(MDN_EWORKSPACE, "solve: workspace too small");
    char* p = (char*)ws;
    double* pooled = (double*)p; p += align256(sizeof(double) * G * Dp * Dp);
    double* ntot = (double*)p; p += align256(sizeof(double));
    double* pooled_h = (double*)p;
    size_t sm = sizeof(double) * ((size_t)D * D + (size_t)D * T);
    if (sm > 200 * 1024) return fail(MDN_ESHAPE, "solve: D too large for shared-memory Cholesky");
    cudaError_t ea = cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ea != cudaSuccess) return cuda_fail(ea, "solve: shared memory attribute");
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "solve: clear status");
    int64_t ent = (int64_t)G * Dp * Dp;
    k_pool<<<(unsigned)((ent + 255) / 256), 256, 0, s>>>(gram, counts, K, ent, pooled, ntot);
    k_chol<<<G, 256, sm, s>>>(gram, counts, pooled, ntot, G, D, T, lambda, 1, pooled_h, bank_out, status);
    k_chol<<<K * G, 256, sm, s>>>(gram, counts, pooled, ntot, G, D, T, lambda, 0, pooled_h, bank_out, status);
    return check_launch("k_chol");
}

}  // namespace mdn
