// k_train.cu -- A5/A6: bucketed least-squares training (Eqs. 5-6).
//
// Pipeline for one level (all on the stream, no host synchronisation):
//   k_to_work      storage RGB -> working colour space (z, coarse, target),
//                  centred; FP32, TF32-rounded or BF16 by the Gram precision
//   k_hist         per-block bucket histograms of the bucket map
//   k_scan         bucket-major exclusive scan -> stable scatter offsets and
//                  the chunk table (bucket, begin, end), chunks <= CHUNK rows
//   k_scatter      stable counting-sort scatter of pixel indices by bucket
//   Gram           per chunk: A^T A of the gathered rows A = [regressor|target
//                  shifted by a per-channel constant | 1] (SIMT FP32 here,
//                  tcgen05 variants in k_gram_tc.cu), written as FP32 partials
//   k_reduce_sum / k_center  FP64 sum of a bucket's partials in group and
//                  chunk order (deterministic), then the exact centring
//                  correction, added into gram[k][g]; counts[k] += n_k
//   k_pool/k_chol  ridge solve (G_xx/n + lambda I) h = G_xy/n by Cholesky in
//                  FP64 shared memory, one CTA per (bucket, group); empty
//                  buckets copy the pooled solution
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "train_common.cuh"

namespace mdn {
namespace trn {

// ---------------------------------------------------------------- helpers

// Storage RGB -> FP32 working colour space, shifted by each channel's centring
// constant, written with a replicated border of P pixels: out is
// [n][3][h + 2P][w + 2P] and out(y + P, x + P) takes the input at
// (clamp(y, 0, h-1), clamp(x, 0, w-1)).  round_tf32: round the shifted value
// to TF32 (nearest, ties away), the operand precision of the TF32 Gram (the
// tensor core would otherwise drop the low mantissa bits, a bias that does not
// average out over many rows).
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// mode: 0 FP32 value, 1 rounded to TF32 (nearest, ties away), 2 rounded to
// BF16 (nearest even) and stored as 16-bit BF16 (the BF16 Gram's operands)
template <typename TS>
__global__ void k_to_work(const TS* __restrict__ in, void* __restrict__ outv, int h, int w, int64_t n, int P,
                          int color, int mode) {
    const int Hp = h + 2 * P, Wp = w + 2 * P;
    const int64_t hwp = (int64_t)Hp * Wp, hw = (int64_t)h * w;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= hwp * n) return;
    const int64_t img = i / hwp, q = i % hwp;
    const int yp = (int)(q / Wp), xp = (int)(q % Wp);
    const int y = clampi(yp - P, 0, h - 1), x = clampi(xp - P, 0, w - 1);
    const TS* s = in + img * 3 * hw + (int64_t)y * w + x;
    float r = ld_f(s, 0), g = ld_f(s, hw), b = ld_f(s, 2 * hw);
    float yy, cb, cr;
    if (color == MDN_RGB) { yy = r; cb = g; cr = b; }
    else {
        yy = 0.299f * r + 0.587f * g + 0.114f * b;
        cb = -0.168735892f * r - 0.331264108f * g + 0.5f * b;
        cr = 0.5f * r - 0.418687589f * g - 0.081312411f * b;
    }
    yy -= (float)channel_center(0, color);
    cb -= (float)channel_center(1, color);
    cr -= (float)channel_center(2, color);
    const int64_t o = img * 3 * hwp + q;
    if (mode == 2) {
        __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(outv) + o;
        d[0] = __float2bfloat16_rn(yy); d[hwp] = __float2bfloat16_rn(cb); d[2 * hwp] = __float2bfloat16_rn(cr);
        return;
    }
    if (mode == 1) { yy = round_tf32(yy); cb = round_tf32(cb); cr = round_tf32(cr); }
    float* d = reinterpret_cast<float*>(outv) + o;
    d[0] = yy; d[hwp] = cb; d[2 * hwp] = cr;
}

// Per-block bucket histograms; TK = uint8_t (K <= 256) or uint16_t.
template <typename TK>
__global__ void k_hist(const TK* __restrict__ bmap, int64_t npix, int K, int* __restrict__ blockhist) {
    __shared__ int h[MDN_MAX_K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) h[k] = 0;
    __syncthreads();
    int64_t b0 = (int64_t)blockIdx.x * SORT_CHUNK;
    int64_t e = b0 + SORT_CHUNK < npix ? b0 + SORT_CHUNK : npix;
    for (int64_t i = b0 + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&h[bmap[i]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) blockhist[(int64_t)blockIdx.x * K + k] = h[k];
}

// Bucket offsets in three short passes over the per-block histograms
// (blocks of SORT_CHUNK pixels, grouped into SCAN_SEGS segments):
//   k_segsum  segsum[s][k] = sum of blockhist over segment s's blocks
//   k_scan    bstart[k], bcount[k] and segoff[s][k] = start of segment s's
//             bucket-k run in the sorted list (one CTA, below)
//   k_offs    offs[b][k] = start of block b's bucket-k run
constexpr int SCAN_SEGS = 64;

__global__ void k_segsum(const int* __restrict__ blockhist, int nblk, int K, int seglen, int* __restrict__ segsum) {
    const int sg = blockIdx.x, b0 = sg * seglen, b1 = min(b0 + seglen, nblk);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int t = 0;
        for (int b = b0; b < b1; ++b) t += blockhist[(int64_t)b * K + k];
        segsum[sg * K + k] = t;
    }
}

__global__ void k_offs(const int* __restrict__ blockhist, const int* __restrict__ segoff, int nblk, int K, int seglen,
                       int* __restrict__ offs) {
    const int sg = blockIdx.x, b0 = sg * seglen, b1 = min(b0 + seglen, nblk);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int run = segoff[sg * K + k];
        for (int b = b0; b < b1; ++b) {
            offs[(int64_t)b * K + k] = run;
            run += blockhist[(int64_t)b * K + k];
        }
    }
}

// exclusive prefix sum over the threads of a CTA (blockDim.x <= 256)
__device__ int block_exclusive_scan(int v, int* tmp, int* total) {
    const int t = threadIdx.x;
    tmp[t] = v;
    __syncthreads();
    for (int d = 1; d < blockDim.x; d <<= 1) {
        const int add = t >= d ? tmp[t - d] : 0;
        __syncthreads();
        tmp[t] += add;
        __syncthreads();
    }
    const int incl = tmp[t];
    *total = tmp[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

// One CTA (256 threads); thread t owns the contiguous buckets
// [t * per, (t + 1) * per), per = ceil(K / 256), so any K <= MDN_MAX_K works.
__global__ void __launch_bounds__(256) k_scan(const int* __restrict__ segsum, int nseg, int K,
                                              int64_t* __restrict__ bstart, int64_t* __restrict__ bcount,
                                              int* __restrict__ segoff) {
    __shared__ int tmp[256];
    __shared__ int total;
    const int per = (K + blockDim.x - 1) / blockDim.x;
    const int k0 = min((int)threadIdx.x * per, K), k1 = min(k0 + per, K);
    int mine = 0;
    for (int k = k0; k < k1; ++k) {
        int t = 0;
        for (int sg = 0; sg < nseg; ++sg) t += segsum[sg * K + k];
        bcount[k] = t;
        mine += t;
    }
    int run = block_exclusive_scan(mine, tmp, &total);   // pixel counts are < 2^31
    for (int k = k0; k < k1; ++k) {
        bstart[k] = run;
        for (int sg = 0; sg < nseg; ++sg) {
            segoff[sg * K + k] = run;
            run += segsum[sg * K + k];
        }
    }
}

// Chunk table of one pixel group (CTA per group).  A group is the pixel-index
// range [g * GB, (g + 1) * GB): since the sorted list is ordered by bucket and
// then by pixel index, the group's rows of bucket k form one contiguous run.
// Group g's chunks, in bucket order, go to chunks[g * cap ...], each
// (k, begin, end, w), and crange[g][k] gets bucket k's chunk range.
// Quantum mode (tensor cores) balances the CTAs by cost: a non-empty run costs
// its rows plus run_cost rows (the fixed work of a chunk: draining and
// reading back the accumulator), the runs are laid end to end in that cost
// space, cut at every multiple of Q = max(ceil(total cost / ncta), minq), and
// each chunk records w = the CTA that owns it (cost position of its first row
// / Q).  Otherwise runs are cut into pieces of at most chunk_rows rows (w = 0).
__global__ void __launch_bounds__(256) k_chunks(const int* __restrict__ offs, const int64_t* __restrict__ bstart,
                                                const int64_t* __restrict__ bcount, int K, int nblk, int bpg,
                                                int quantum_mode, int ncta, int minq, int run_cost,
                                                int chunk_rows, int cap, int4* __restrict__ chunks,
                                                int* __restrict__ gcount, int2* __restrict__ crange) {
    __shared__ int tmp[256];
    __shared__ int total;
    const int g = blockIdx.x;
    const int b0 = g * bpg, b1 = b0 + bpg;
    // thread t handles the contiguous buckets [k0, k1) (one bucket when K <= 256)
    const int per = (K + blockDim.x - 1) / blockDim.x;
    const int k0 = min((int)threadIdx.x * per, K), k1 = min(k0 + per, K);
    const int A = quantum_mode ? run_cost : 0;
    auto run_of = [&](int k, int& start, int& len) {
        start = offs[(int64_t)b0 * K + k];
        const int end = b1 < nblk ? offs[(int64_t)b1 * K + k] : (int)(bstart[k] + bcount[k]);
        len = end - start;
    };
    auto cost_of = [&](int len) { return len > 0 ? len + A : 0; };
    int mine = 0;
    for (int k = k0; k < k1; ++k) {
        int st, ln;
        run_of(k, st, ln);
        mine += cost_of(ln);
    }
    const int vbase = block_exclusive_scan(mine, tmp, &total);   // cost position of bucket k0's run
    const int ctot = total;
    int Q = chunk_rows;
    if (quantum_mode) {
        const int q = (ctot + ncta - 1) / ncta;
        Q = q > minq ? q : minq;
    }
    // a run's rows sit at cost positions [v, v + len), v = run start + A
    auto chunks_of = [&](int v, int len) {
        if (len <= 0) return 0;
        if (quantum_mode) {
            const int inner = (v + len + Q - 1) / Q - 1 - v / Q;   // multiples of Q in (v, v + len)
            return (inner > 0 ? inner : 0) + 1;
        }
        return (len + Q - 1) / Q;
    };
    int nmine = 0;
    for (int k = k0, c = vbase; k < k1; ++k) {
        int st, ln;
        run_of(k, st, ln);
        nmine += chunks_of(c + A, ln);
        c += cost_of(ln);
    }
    const int cbase = block_exclusive_scan(nmine, tmp, &total);
    int j = cbase;
    for (int k = k0, c = vbase; k < k1; ++k) {
        int start, len;
        run_of(k, start, len);
        const int j0 = j, v = c + A;
        for (int r = v; r < v + len && j < cap; ++j) {
            int e = quantum_mode ? (r / Q + 1) * Q : r + Q;
            if (e > v + len) e = v + len;
            chunks[(int64_t)g * cap + j] = make_int4(k, start + (r - v), start + (e - v), quantum_mode ? r / Q : 0);
            r = e;
        }
        crange[(int64_t)g * K + k] = make_int2(g * cap + j0, g * cap + j);   // bucket k's chunks in group g
        c += cost_of(len);
    }
    if (threadIdx.x == 0) gcount[g] = total < cap ? total : cap;   // the capacity bounds the total by construction
}

// Stable scatter: pixels of a block are ranked in index order within their
// bucket (warp match + per-warp counts), so the sorted list is deterministic.
// K <= 256 (u8 maps).
__global__ void __launch_bounds__(256) k_scatter(const uint8_t* __restrict__ bmap, int64_t npix, int K,
                                                 const int* __restrict__ offs, int* __restrict__ sorted) {
    constexpr int NK = 256;
    __shared__ int run[NK];
    __shared__ int wcnt[8][NK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < K; k += blockDim.x) run[k] = offs[(int64_t)blockIdx.x * K + k];
    int64_t b0 = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int64_t base = b0; base < b0 + SORT_CHUNK; base += blockDim.x) {
        for (int i = threadIdx.x; i < 8 * NK; i += blockDim.x) (&wcnt[0][0])[i] = 0;
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

// The same stable scatter for K > 256 (u16 maps): one warp per block walks the
// block's pixels 32 at a time in index order; lanes holding the same bucket
// are ranked by lane, and the leader advances the bucket's run offset after
// the warp has read it.
__global__ void __launch_bounds__(32) k_scatter_wide(const uint16_t* __restrict__ bmap, int64_t npix, int K,
                                                     const int* __restrict__ offs, int* __restrict__ sorted) {
    __shared__ int run[MDN_MAX_K];
    const int lane = threadIdx.x;
    for (int k = lane; k < K; k += 32) run[k] = offs[(int64_t)blockIdx.x * K + k];
    __syncwarp();
    const int64_t b0 = (int64_t)blockIdx.x * SORT_CHUNK;
    const int64_t e = b0 + SORT_CHUNK < npix ? b0 + SORT_CHUNK : npix;
    for (int64_t base = b0; base < e; base += 32) {
        const int64_t i = base + lane;
        const bool valid = i < e;
        const int k = valid ? (int)bmap[i] : 0x7fffffff - lane;   // invalid lanes never match a bucket
        const unsigned m = __match_any_sync(0xffffffffu, k);
        const int rank = __popc(m & ((1u << lane) - 1u));
        const int pos = valid ? run[k] + rank : 0;
        __syncwarp();
        if (valid) {
            sorted[pos] = (int)i;
            if (rank == 0) run[k] += __popc(m);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- SIMT Gram

// Gram of one chunk, FP32 products/accumulation, 4x4 register blocks of the
// upper triangle of every group's Dp x Dp matrix, written to the partial in the
// lower-triangle layout k_reduce_sum reads.
__global__ void __launch_bounds__(256) k_gram_simt(GatherArgs ga, const int4* __restrict__ chunks,
                                                    const int* __restrict__ nchunks, const int* __restrict__ sorted,
                                                    float* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem[];
    if ((int)blockIdx.x >= *nchunks) return;
    const int4 ch = chunks[blockIdx.x];
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
                if (i < Dq && j < Dq && i <= j) out[((size_t)bg[m] * Dq + j) * Dq + i] = acc[m][p * 4 + q];
            }
    }
}

// FP64 reduction of a bucket's chunk partials in group order, then chunk order
// (deterministic), in two passes.  Partials are (Dq = Dp + 1)^2 symmetric
// matrices of the shifted rows with the ones column last, of which the lower
// triangle (row-major: entry (a, b), a >= b, at a * Dq + b) is written.
// crange[g][k] = bucket k's chunk range in group g (from k_chunks).
//   k_reduce_sum  S[k][g] = sum of the bucket's partials (lower triangle)
//   k_center      the exact centring correction
//                 G_ij = S_ij + c_i s_j + c_j s_i + n c_i c_j,
//                 s_i = S_{ones,i}, n = S_{ones,ones}, added into gram[k][g]
__global__ void k_reduce_sum(const float* __restrict__ partial, const int2* __restrict__ crange, int ngroups,
                             int K, int G, int Dq, double* __restrict__ S) {
    const int k = blockIdx.y;
    const int64_t entq = (int64_t)G * Dq * Dq;
    __shared__ int2 rg[GRAM_MAX_GROUPS];
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) rg[g] = crange[(int64_t)g * K + k];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < entq; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)((e / Dq) % Dq), b = (int)(e % Dq);
        if (a < b) continue;
        double acc = 0.0;
        for (int gr = 0; gr < ngroups; ++gr)
            for (int c = rg[gr].x; c < rg[gr].y; ++c) acc += (double)__ldcs(partial + (size_t)c * entq + e);
        S[(size_t)k * entq + e] = acc;
    }
}

__global__ void k_center(const double* __restrict__ S, const int64_t* __restrict__ bcount, int G, int Dp, int D,
                         int rf, int rc, int cross, int color, double* __restrict__ gram,
                         int64_t* __restrict__ counts) {
    const int k = blockIdx.y;
    const int Dq = Dp + 1;
    const int64_t ent = (int64_t)G * Dp * Dp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ent; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / ((int64_t)Dp * Dp));
        const int i = (int)((e / Dp) % Dp), j = (int)(e % Dp);
        if (i > j) continue;
        const double* Sq = S + ((size_t)k * G + g) * Dq * Dq;   // lower triangle
        const double sij = Sq[(size_t)j * Dq + i], si = Sq[(size_t)Dp * Dq + i], sj = Sq[(size_t)Dp * Dq + j];
        const double n = Sq[(size_t)Dp * Dq + Dp];
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

size_t train_ws_bytes(int64_t n, int64_t h, int64_t w, int P, bool coarse, int K, int G, int Dp, int precision) {
    const int64_t npix = n * h * w, hc = (h + 1) / 2, wc = (w + 1) / 2;
    const GramGroups gq = gram_groups(n, h, w, P, coarse, K, precision != MDN_GRAM_FP32);
    const int64_t nblk = (npix + SORT_CHUNK - 1) / SORT_CHUNK;
    const int64_t nent = (int64_t)gq.ngroups * gq.cap;
    size_t b = 0;
    b += align256(sizeof(float) * 3 * n * (h + 2 * P) * (w + 2 * P));    // z, border P
    b += align256(sizeof(float) * 3 * npix);                               // target
    b += align256(sizeof(float) * 3 * n * (hc + 2 * P) * (wc + 2 * P));  // coarse, border P
    b += align256(sizeof(int) * nblk * K) * 2;        // blockhist, offs
    b += align256(sizeof(int) * SCAN_SEGS * K) * 2;   // segsum, segoff
    b += align256(sizeof(int64_t) * K) * 2;           // bstart, bcount
    b += align256(sizeof(int4) * nent) + align256(sizeof(int) * gq.ngroups);   // chunk tables, counts
    b += align256(sizeof(int2) * gq.ngroups * K);                                // per (group, bucket) chunk ranges
    b += align256(sizeof(int) * (npix > 0 ? npix : 1));   // sorted
    b += align256(sizeof(float) * nent * G * (Dp + 1) * (Dp + 1));  // partials (Dp + 1 with the ones column)
    b += align256(sizeof(double) * K * G * (Dp + 1) * (Dp + 1));    // FP64 bucket sums
    return b;
}

int launch_gram(const TrainArgs& a, cudaStream_t s) {
    const int64_t hw = a.h * a.w, npix = a.n * hw;
    const int P = gram_border(a.geom);
    const int64_t Hp = a.h + 2 * P, Wp = a.w + 2 * P, Hcp = a.hc + 2 * P, Wcp = a.wc + 2 * P;
    if (a.Dp + 1 > GRAM_MAX_DP) return fail(MDN_ESHAPE, "train: regressor too long (D + T must be <= 159)");
    if (3 * a.n * Hp * Wp >= (int64_t(1) << 31))
        return fail(MDN_ESHAPE, "train: padded working planes exceed 2^31 elements");
    const bool tensor = a.precision != MDN_GRAM_FP32;
    const GramGroups gq = gram_groups(a.n, a.h, a.w, P, a.coarse != nullptr, a.K, tensor);
    // carve the workspace (the layout of train_ws_bytes)
    char* p = (char*)a.ws;
    auto take = [&](size_t bytes) { char* r = p; p += align256(bytes); return r; };
    float* zw = (float*)take(sizeof(float) * 3 * a.n * Hp * Wp);
    float* tw = (float*)take(sizeof(float) * 3 * npix);
    float* cw = (float*)take(sizeof(float) * 3 * a.n * Hcp * Wcp);
    const int64_t nblk = (npix + SORT_CHUNK - 1) / SORT_CHUNK;
    const int64_t nent = (int64_t)gq.ngroups * gq.cap;
    int* blockhist = (int*)take(sizeof(int) * nblk * a.K);
    int* offs = (int*)take(sizeof(int) * nblk * a.K);
    int* segsum = (int*)take(sizeof(int) * SCAN_SEGS * a.K);
    int* segoff = (int*)take(sizeof(int) * SCAN_SEGS * a.K);
    int64_t* bstart = (int64_t*)take(sizeof(int64_t) * a.K);
    int64_t* bcount = (int64_t*)take(sizeof(int64_t) * a.K);
    int4* chunks = (int4*)take(sizeof(int4) * nent);
    int* gcount = (int*)take(sizeof(int) * gq.ngroups);
    int2* crange = (int2*)take(sizeof(int2) * gq.ngroups * a.K);
    int* sorted = (int*)take(sizeof(int) * (npix > 0 ? npix : 1));
    float* partial = (float*)take(sizeof(float) * nent * a.G * (a.Dp + 1) * (a.Dp + 1));
    double* bsum = (double*)take(sizeof(double) * a.K * a.G * (a.Dp + 1) * (a.Dp + 1));
    if ((size_t)(p - (char*)a.ws) > a.ws_bytes) return fail(MDN_EWORKSPACE, "train: workspace too small");

    constexpr int TB = 256;
    auto conv = [&](const void* in, float* out, int64_t hh, int64_t ww, int pad) {
        const int64_t cnt = a.n * (hh + 2 * pad) * (ww + 2 * pad);
        unsigned g = (unsigned)((cnt + TB - 1) / TB);
        const int mode = a.precision == MDN_GRAM_TF32 ? 1 : (a.precision == MDN_GRAM_BF16 ? 2 : 0);
        if (a.dtype == MDN_F32)
            k_to_work<float><<<g, TB, 0, s>>>((const float*)in, out, (int)hh, (int)ww, a.n, pad, a.geom.color, mode);
        else
            k_to_work<__half><<<g, TB, 0, s>>>((const __half*)in, out, (int)hh, (int)ww, a.n, pad, a.geom.color, mode);
    };
    conv(a.z, zw, a.h, a.w, P);
    conv(a.target, tw, a.h, a.w, 0);
    if (a.coarse) conv(a.coarse, cw, a.hc, a.wc, P);
    // sort: per-block histograms, bucket offsets, stable scatter
    const int seglen = (int)((nblk + SCAN_SEGS - 1) / SCAN_SEGS);
    const int nseg = (int)((nblk + seglen - 1) / seglen);
    const bool wide = a.K > 256;   // u16 bucket map
    if (wide) k_hist<uint16_t><<<(unsigned)nblk, TB, 0, s>>>((const uint16_t*)a.buckets, npix, a.K, blockhist);
    else k_hist<uint8_t><<<(unsigned)nblk, TB, 0, s>>>((const uint8_t*)a.buckets, npix, a.K, blockhist);
    k_segsum<<<nseg, TB, 0, s>>>(blockhist, (int)nblk, a.K, seglen, segsum);
    k_scan<<<1, TB, 0, s>>>(segsum, nseg, a.K, bstart, bcount, segoff);
    k_offs<<<nseg, TB, 0, s>>>(blockhist, segoff, (int)nblk, a.K, seglen, offs);
    if (wide) k_scatter_wide<<<(unsigned)nblk, 32, 0, s>>>((const uint16_t*)a.buckets, npix, a.K, offs, sorted);
    else k_scatter<<<(unsigned)nblk, TB, 0, s>>>((const uint8_t*)a.buckets, npix, a.K, offs, sorted);
    // chunk tables: tensor cores one CTA per SM, each taking a share of every group
    const int ncta = num_sms() < GRAM_MAX_CTAS ? num_sms() : GRAM_MAX_CTAS;
    k_chunks<<<gq.ngroups, TB, 0, s>>>(offs, bstart, bcount, a.K, (int)nblk, (int)(gq.GB / SORT_CHUNK),
                                       tensor ? 1 : 0, ncta, GRAM_MIN_QUANTUM, GRAM_RUN_COST, GRAM_CHUNK, gq.cap,
                                       chunks, gcount, crange);
    int rc = check_launch("train: sort");
    if (rc) return rc;

    GatherArgs ga{};
    ga.zw = zw; ga.tw = tw; ga.cw = a.coarse ? cw : nullptr;
    ga.h = (int)a.h; ga.w = (int)a.w; ga.hc = (int)a.hc; ga.wc = (int)a.wc; ga.n = (int)a.n;
    ga.P = P; ga.Hp = (int)Hp; ga.Wp = (int)Wp; ga.Hcp = (int)Hcp; ga.Wcp = (int)Wcp;
    ga.rf = a.geom.r_fine; ga.rc = a.geom.r_coarse; ga.cross = a.geom.cross_channel; ga.color = a.geom.color;
    ga.D = a.D; ga.T = a.T; ga.G = a.G; ga.Dp = a.Dp; ga.Dp4 = (a.Dp + 1 + 3) / 4 * 4;
    if (!tensor) {
        size_t sm = sizeof(float) * (size_t)a.G * GRAM_RB * ga.Dp4 + sizeof(int) * a.G * (a.Dp + 1);
        const int nb = (a.Dp + 1 + 3) / 4;
        if (a.G * nb * (nb + 1) / 2 > 8 * 256) return fail(MDN_ESHAPE, "train: Gram too large for the SIMT path");
        cudaError_t ea = cudaFuncSetAttribute(k_gram_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (ea != cudaSuccess) return cuda_fail(ea, "k_gram_simt: shared memory attribute");
        k_gram_simt<<<(unsigned)gq.cap, 256, sm, s>>>(ga, chunks, gcount, sorted, partial);
        if ((rc = check_launch("k_gram_simt"))) return rc;
    } else {
        rc = launch_gram_tc(ga, a.precision, chunks, gcount, gq.ngroups, gq.cap, sorted, partial, ncta, s);
        if (rc) return rc;
    }
    const int Dq = a.Dp + 1;
    dim3 rg1((unsigned)((a.G * Dq * Dq + 255) / 256), (unsigned)a.K);
    k_reduce_sum<<<rg1, 256, 0, s>>>(partial, crange, gq.ngroups, a.K, a.G, Dq, bsum);
    dim3 rg2((unsigned)((a.G * a.Dp * a.Dp + 255) / 256), (unsigned)a.K);
    k_center<<<rg2, 256, 0, s>>>(bsum, bcount, a.G, a.Dp, a.D, a.geom.r_fine, a.geom.r_coarse, a.geom.cross_channel,
                                 a.geom.color, a.gram, a.counts);
    return check_launch("k_reduce_sum / k_center");
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
