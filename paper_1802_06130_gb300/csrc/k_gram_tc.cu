// k_gram_tc.cu -- A5 on the 5th-generation tensor cores: per-chunk Gram
// matrices G = A^T A of the gathered rows A = [regressor | target] of one
// bucket (Eqs. 5-6 normal equations), with tcgen05.mma and the accumulator in
// tensor memory.
//
// Formulation.  With X^T the (features x pixels) transpose of a K-step of A,
// G += X^T (X^T)^T: both MMA operands are the same shared-memory matrix,
// K-major (pixels contiguous), 128-byte swizzled (8-row x 128-byte atoms,
// 16-byte chunk c of row r stored at c ^ (r mod 8)).  Per K-step of KB pixels
// (one 128-byte atom: 32 TF32 or 64 BF16 values) four MMAs of K = 32 bytes
// advance the descriptor start address by 32 bytes.
//   Dp <= 128:      M = 128, N = round16(Dp)            (one MMA per group)
//   128 < Dp <= 160: M = 128 x N = 160 (rows 0..127) and M = 128 x N = 32
//                   (rows 32..159 x cols 128..159), which together cover the
//                   upper triangle.
// Centring: each feature is shifted by a constant c_f (0.5 for luma or RGB
// channels, 0 for chroma) and a ones column is appended, so the accumulated
// Gram S of the shifted rows also holds their column sums s and the count n;
// the FP64 reduction restores G = S + c s^T + s c^T + n c c^T exactly.  This
// removes the large DC eigenvalue that would otherwise amplify the operand
// rounding in the ridge solve.  TF32 operands are rounded to nearest.
// Precisions: TF32 (kind::tf32), BF16 (kind::f16, BF16 operands) and split
// BF16 (x = hi + lo, G ~ hi hi^T + hi lo^T + lo hi^T, three MMAs).  FP32
// accumulation in TMEM; each chunk's upper triangle is written as an FP32
// partial and reduced in FP64 by k_reduce (k_train.cu).
//
// Pipeline: 512 threads gather K-step t into stage t%2 (each thread owns a
// feature and a quarter of the step's pixels, two 16-byte stores per feature
// row), fence the async proxy, then thread 0 issues the MMAs and commits them
// to the stage's mbarrier; the loads of step t+1 are issued immediately and
// overlap the MMAs of step t and the barrier waits.  Waits on mbarriers are bounded: on expiry the CTA records
// an error, waits (bounded) for its issued MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "train_common.cuh"

namespace mdn {
namespace tc {

constexpr int NTHREADS = 512;
constexpr int TMEM_COLS = 512;
constexpr unsigned long long WAIT_LIMIT = 1ull << 24;   // try_wait polls before giving up

__device__ int g_gram_error;   // set to 1 when a bounded wait expired

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle,
// stride between 8-row groups = 1024 bytes (SBO), leading offset unused.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}

// instruction descriptor for kind::f16 / kind::tf32: D = F32, A/B format,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t make_idesc(int ab_format, int M, int N) {
    return (1u << 4) | ((uint32_t)ab_format << 7) | ((uint32_t)ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    if constexpr (TF32) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum));
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier; true on success
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity) {
    for (unsigned long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 operand: round to nearest (the tensor core would otherwise drop the
// low mantissa bits, a bias that does not average out over many rows)
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ float center_of(int c, int color) { return (float)channel_center(c, color); }

// Precision modes
enum { P_TF32 = 0, P_BF16 = 1, P_SPLIT = 2 };

template <int MODE> struct Cfg {
    static constexpr bool TF32 = MODE == P_TF32;
    static constexpr int KB = TF32 ? 32 : 64;          // pixels per K-step (one 128-byte atom)
    static constexpr int PER_CHUNK = TF32 ? 4 : 8;     // pixels per 16-byte chunk
    static constexpr int NBUF = MODE == P_SPLIT ? 2 : 1;  // hi (+ lo) operand copies
    static constexpr int FMT = TF32 ? 2 : 1;           // TF32 = 2, BF16 = 1
};

// Per-pixel information of one K-step, staged in shared memory:
// [0] image index (-1 = padding row), [1] y, [2] x, [3] y/2, [4] x/2.
constexpr int PIX_FIELDS = 5;

// Shared memory: [2 stages][G][NBUF][ROWS x 128 B] operand tiles (1024-B
// aligned), then pixel info [2][PIX_FIELDS][KB], mbarriers, TMEM slot, flag.
//
// Thread t owns feature fA = t mod 128 (and fB = fA + 128 when the tile has
// 160 rows) of every group, for the quarter t / 128 of the K-step's pixels:
// PPT = KB/4 consecutive pixels, i.e. two 16-byte chunks per feature row.
// Software pipeline: the loads of step t+1 are issued right after step t's
// MMAs, so they are in flight while the stage and MMA barriers are waited on.
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) k_gram_tc(GatherArgs ga, const int4* __restrict__ chunks,
                                                         const int* __restrict__ sorted, float* __restrict__ partial,
                                                         int rows) {
    using C = Cfg<MODE>;
    constexpr int PPT = C::KB / 4;                 // pixels per thread per feature
    constexpr int NSLOT = 3;                       // (feature, group) slots per thread
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int G = ga.G, Dp = ga.Dp, Dq = ga.Dp + 1;   // Dq: features + the ones column
    const size_t tile_bytes = (size_t)rows * 128;
    const size_t stage_bytes = tile_bytes * C::NBUF * G;
    int* pix = reinterpret_cast<int*>(smem + 2 * stage_bytes);                      // [2][PIX_FIELDS][KB]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(pix + 2 * PIX_FIELDS * C::KB);      // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
    int* flag = reinterpret_cast<int*>(tmem_slot + 1);                              // [0]: abort
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 ch = chunks[blockIdx.x];
    if (ch.x < 0) return;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        flag[0] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }

    // ---- this thread's (feature, group) slots and their column codes ----
    // code: src (0 coarse, 1 fine, 2 target, 3 ones) | c << 2 | (dy+8) << 4 | (dx+8) << 9; -1 = zero row
    const int fA = tid & 127, quarter = tid >> 7;
    int sf[NSLOT], sg[NSLOT], code[NSLOT];
    float cen[NSLOT];
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
        const int f = G > 1 ? fA : fA + 128 * j;
        const int g = G > 1 ? j : 0;
        sf[j] = f;
        sg[j] = g;
        int cd = -1;
        const bool live = (G > 1 ? j < G : j < 2) && f < rows;
        if (live && f < Dp) {
            const int nch = ga.cross ? 3 : 1;
            const int pc = ga.rc >= 0 ? (2 * ga.rc + 1) * (2 * ga.rc + 1) : 0;
            const int pf = (2 * ga.rf + 1) * (2 * ga.rf + 1);
            if (f < nch * pc) {
                const int c = ga.cross ? f / pc : g, idx = f % pc;
                cd = 0 | (c << 2) | ((idx / (2 * ga.rc + 1) - ga.rc + 8) << 4) | ((idx % (2 * ga.rc + 1) - ga.rc + 8) << 9);
            } else if (f < ga.D) {
                const int jj = f - nch * pc;
                const int c = ga.cross ? jj / pf : g, idx = jj % pf;
                cd = 1 | (c << 2) | ((idx / (2 * ga.rf + 1) - ga.rf + 8) << 4) | ((idx % (2 * ga.rf + 1) - ga.rf + 8) << 9);
            } else {
                const int c = ga.cross ? f - ga.D : g;
                cd = 2 | (c << 2) | (8 << 4) | (8 << 9);
            }
        } else if (live && f == Dp) {
            cd = 3;
        }
        if (!live) sf[j] = -1;
        code[j] = cd;
        cen[j] = (cd >= 0 && (cd & 3) != 3) ? center_of((cd >> 2) & 3, ga.color) : 0.f;
    }

    const int nrows = ch.z - ch.y;
    const int nsteps = (nrows + C::KB - 1) / C::KB;
    const int hw = ga.h * ga.w;

    // per-pixel info of step t into pix buffer b (threads < KB)
    auto decode = [&](int t, int b) {
        if (tid < C::KB) {
            const int r = ch.y + t * C::KB + tid;
            int* pb = pix + b * PIX_FIELDS * C::KB;
            if (t < nsteps && r < ch.z) {
                const int p = sorted[r];
                const int img = p / hw, rem = p % hw;
                const int y = rem / ga.w, x = rem % ga.w;
                pb[tid] = img; pb[C::KB + tid] = y; pb[2 * C::KB + tid] = x;
                pb[3 * C::KB + tid] = y >> 1; pb[4 * C::KB + tid] = x >> 1;
            } else {
                pb[tid] = -1; pb[C::KB + tid] = 0; pb[2 * C::KB + tid] = 0; pb[3 * C::KB + tid] = 0;
                pb[4 * C::KB + tid] = 0;
            }
        }
    };
    float vals[NSLOT][PPT];
    // issue the loads of one step (pixel info in buffer b), branch-free per pixel
    auto load_step = [&](int b) {
        const int* pb = pix + b * PIX_FIELDS * C::KB;
#pragma unroll
        for (int j = 0; j < NSLOT; ++j) {
            const int cd = code[j];
            const int src = cd & 3, c = (cd >> 2) & 3;
            const int dy = ((cd >> 4) & 31) - 8, dx = ((cd >> 9) & 31) - 8;
            const float* plane;
            int ph, pw;
            if (src == 0) { plane = ga.cw; ph = ga.hc; pw = ga.wc; }
            else if (src == 1) { plane = ga.zw; ph = ga.h; pw = ga.w; }
            else { plane = ga.tw; ph = ga.h; pw = ga.w; }
            const int yo = src == 0 ? 3 : 1, xo = src == 0 ? 4 : 2;   // pixel-info field of y, x
            const bool fetch = cd >= 0 && src != 3;
#pragma unroll
            for (int e = 0; e < PPT; ++e) {
                const int rr = quarter * PPT + e;
                const int img = pb[rr];
                float v = 0.f;
                if (fetch && img >= 0) {
                    const int yy = clampi(pb[yo * C::KB + rr] + dy, 0, ph - 1);
                    const int xx = clampi(pb[xo * C::KB + rr] + dx, 0, pw - 1);
                    v = __ldg(plane + ((int64_t)img * 3 + c) * ph * pw + (int64_t)yy * pw + xx);
                }
                vals[j][e] = v;
            }
        }
    };
    // store the held values (centred, ones column, zero padding) into stage s
    auto store_step = [&](int s, int b) {
        const int* pb = pix + b * PIX_FIELDS * C::KB;
        unsigned char* stage = smem + s * stage_bytes;
#pragma unroll
        for (int j = 0; j < NSLOT; ++j) {
            if (sf[j] < 0) continue;
            const int f = sf[j];
            unsigned char* rowp = stage + (size_t)sg[j] * C::NBUF * tile_bytes + (size_t)(f >> 3) * 1024 + (f & 7) * 128;
            float v[PPT];
#pragma unroll
            for (int e = 0; e < PPT; ++e) {
                const bool valid = pb[quarter * PPT + e] >= 0 && code[j] >= 0;
                const float x = (code[j] & 3) == 3 ? 1.f : vals[j][e] - cen[j];
                v[e] = valid ? x : 0.f;
            }
#pragma unroll
            for (int hq = 0; hq < 2; ++hq) {
                const int chunk = (quarter * 2 + hq) ^ (f & 7);
                if constexpr (MODE == P_TF32) {
                    *reinterpret_cast<float4*>(rowp + chunk * 16) =
                        make_float4(to_tf32(v[4 * hq]), to_tf32(v[4 * hq + 1]), to_tf32(v[4 * hq + 2]),
                                    to_tf32(v[4 * hq + 3]));
                } else {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * hq + 2 * e], v[8 * hq + 2 * e + 1]);
                        hi[e] = *reinterpret_cast<uint32_t*>(&h2);
                        if constexpr (MODE == P_SPLIT) {
                            float2 hf = __bfloat1622float2(h2);
                            __nv_bfloat162 l2 =
                                __floats2bfloat162_rn(v[8 * hq + 2 * e] - hf.x, v[8 * hq + 2 * e + 1] - hf.y);
                            lo[e] = *reinterpret_cast<uint32_t*>(&l2);
                        }
                    }
                    *reinterpret_cast<uint4*>(rowp + chunk * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    if constexpr (MODE == P_SPLIT)
                        *reinterpret_cast<uint4*>(rowp + tile_bytes + chunk * 16) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
        }
    };

    // MMA shapes
    const bool two = Dq > 128;
    const int N1 = two ? 160 : ((Dq + 15) / 16) * 16;
    const uint32_t idesc1 = make_idesc(C::FMT, 128, N1);
    const uint32_t idesc2 = make_idesc(C::FMT, 128, 32);
    const int cols_per_group = two ? 192 : N1;

    // prologue: pixel info of step 0, its loads
    decode(0, 0);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (nsteps > 0) load_step(0);

    int committed = 0;   // steps whose MMAs were issued and committed
    for (int t = 0; t < nsteps; ++t) {
        const int s = t & 1;
        // stage s is free once the MMAs of step t-2 completed
        if (t >= 2 && tid == 0 && !wait_parity(smem_u32(&mbar[s]), (uint32_t)(((t - 2) >> 1) & 1))) flag[0] = 1;
        decode(t + 1, (t + 1) & 1);
        __syncthreads();
        if (flag[0]) break;
        store_step(s, s);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* stage = smem + s * stage_bytes;
            for (int g = 0; g < G; ++g) {
                const uint32_t base_hi = smem_u32(stage + (size_t)g * C::NBUF * tile_bytes);
                const uint32_t base_lo = base_hi + (uint32_t)tile_bytes;
                const uint32_t d1 = tmem + g * cols_per_group;
                const uint32_t d2 = d1 + 160;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t acc = (t > 0 || k > 0) ? 1u : 0u;
                    const uint32_t ko = 32 * k;
                    const int npairs = MODE == P_SPLIT ? 3 : 1;
                    for (int pr = 0; pr < npairs; ++pr) {
                        const uint32_t ab = pr == 2 ? base_lo : base_hi;
                        const uint32_t bb = pr == 1 ? base_lo : base_hi;
                        const uint32_t accp = (pr > 0) ? 1u : acc;
                        mma<C::TF32>(d1, make_desc(ab + ko), make_desc(bb + ko), idesc1, accp);
                        if (two)
                            mma<C::TF32>(d2, make_desc(ab + 4 * 1024 + ko), make_desc(bb + 16 * 1024 + ko), idesc2, accp);
                    }
                }
            }
            commit(smem_u32(&mbar[s]));
        }
        committed = t + 1;
        if (t + 1 < nsteps) load_step((t + 1) & 1);
    }

    // wait for the last commit of each stage (bounded), then read back
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            // last committed step that used stage s
            const int last = (committed - 1 - s) >= 0 ? ((committed - 1 - s) / 2) * 2 + s : -1;
            if (last >= 0 && !wait_parity(smem_u32(&mbar[s]), (uint32_t)((last >> 1) & 1))) flag[0] = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = flag[0] == 0;
    if (!ok && tid == 0) atomicExch(&g_gram_error, 1);
    if (ok && warp < 4) {
        // warp w reads TMEM lanes 32w..32w+31 = accumulator rows
        const int row = 32 * warp + lane;
        float* out = partial + (size_t)blockIdx.x * G * Dq * Dq;
        for (int g = 0; g < G; ++g) {
            float* og = out + (size_t)g * Dq * Dq;
            const uint32_t d1 = tmem + g * cols_per_group + ((uint32_t)(32 * warp) << 16);
            for (int c0 = 0; c0 < N1; c0 += 16) {
                float v[16];
                tmem_ld16(d1 + c0, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int j = c0 + e;
                    if (row < Dq && j < Dq && row <= j) og[(size_t)row * Dq + j] = v[e];
                }
            }
            if (two) {
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    float v[16];
                    tmem_ld16(d1 + 160 + c0, v);
                    const int i = 32 + row;      // accumulator row m -> feature 32 + m
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = 128 + c0 + e;
                        if (i >= 128 && i < Dq && j < Dq && i <= j) og[(size_t)i * Dq + j] = v[e];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

template <int MODE> size_t smem_bytes(int G, int rows) {
    using C = Cfg<MODE>;
    size_t b = 1024;                                        // alignment slack
    b += 2 * (size_t)rows * 128 * C::NBUF * G;              // operand stages
    b += sizeof(int) * 2 * PIX_FIELDS * C::KB + 2 * sizeof(uint64_t) + 16;
    // at least 120 KB so that one CTA (and its 512 TMEM columns) owns the SM
    return b < 120 * 1024 ? 120 * 1024 : b;
}

template <int MODE>
int run(const GatherArgs& ga, const int4* chunks, int maxch, const int* sorted, float* partial, cudaStream_t s) {
    const int rows = ga.Dp + 1 > 128 ? 160 : 128;
    const size_t bytes = smem_bytes<MODE>(ga.G, rows);
    if (bytes > 232448) return fail(MDN_ESHAPE, "train: tensor-core Gram tile does not fit in shared memory");
    if (ga.G * (ga.Dp + 1 > 128 ? 192 : ((ga.Dp + 1 + 15) / 16) * 16) > TMEM_COLS)
        return fail(MDN_ESHAPE, "train: Gram accumulators exceed tensor memory");
    auto kern = k_gram_tc<MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_gram_tc: smem attribute");
    kern<<<maxch, NTHREADS, bytes, s>>>(ga, chunks, sorted, partial, rows);
    return check_launch("k_gram_tc");
}

}  // namespace tc

int launch_gram_tc(const GatherArgs& ga, int precision, const int4* chunks, int maxch, const int* sorted,
                   float* partial, cudaStream_t s) {
    if (ga.Dp + 1 > 160) return fail(MDN_ESHAPE, "train: tensor-core Gram supports D + T <= 159");
    switch (precision) {
        case MDN_GRAM_TF32: return tc::run<tc::P_TF32>(ga, chunks, maxch, sorted, partial, s);
        case MDN_GRAM_BF16: return tc::run<tc::P_BF16>(ga, chunks, maxch, sorted, partial, s);
        case MDN_GRAM_SPLIT_BF16: return tc::run<tc::P_SPLIT>(ga, chunks, maxch, sorted, partial, s);
        default: return fail(MDN_EINVAL, "train: bad Gram precision");
    }
}

int gram_tc_error(int* out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, tc::g_gram_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tc::g_gram_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "gram error flag");
    *out = v;
    return MDN_OK;
}

}  // namespace mdn
