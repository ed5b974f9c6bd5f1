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
//   Dq <= 128:      M = 128, N = round16(Dq)            (one MMA per group)
//   128 < Dq <= 160: M = 128 x N = 160 (rows 0..127) and M = 128 x N = 32
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
// accumulation in TMEM; each chunk's symmetric matrix is written as an FP32
// partial (lower triangle, row-major) and reduced in FP64 by k_reduce_sum
// and k_center (k_train.cu).
//
// Work split.  The sorted rows are walked in pixel groups (pixel-index ranges
// whose working planes fit in L2); each group's rows are cut into one share
// per CTA (one CTA per SM), and the CTAs go through the groups in the same
// order, so that at any time they gather from one group's planes.  A CTA
// accumulates the chunks (bucket runs) of its shares one after the other and
// writes one partial per chunk.
//
// Warp roles (512 threads), connected by mbarrier rings of S stages:
//   warp 5        decode: sorted row -> per-pixel base offsets of the coarse,
//                 fine and target planes (pixel slot s), arrive pixfull[s]
//   warps 6..15   gather: a warp owns blocks of 8 feature rows and fills the
//                 K-step's 8 16-byte chunks (4 TF32 or 8 BF16 pixels each)
//                 for them, lane = (row, 4-byte word);
//                 base + per-feature offset addresses (the planes carry a
//                 replicated border, so no tap needs clamping, and hold
//                 centred values, pre-rounded for TF32).  TF32: 4-byte
//                 cp.async copies straight into the swizzled tile, two K-steps
//                 in flight; BF16: the loads of two row blocks are issued
//                 before they are rounded and stored as bf16x2 words.  Then
//                 fence the async proxy, arrive full[s]
//   warp 4        one thread waits full[s], issues the MMAs of the K-step and
//                 commits them to empty[s] (which frees stage and pixel slot
//                 s); at a chunk end it commits acc_full
//   warps 0..3    wait acc_full, read the accumulator (TMEM lane quarter w),
//                 write the chunk's partial, arrive acc_empty.  Lane = row i
//                 of the accumulator, so entry (i, j) goes to the lower
//                 triangle at j * Dq + i: a warp's 32 rows are 32 consecutive
//                 floats (one coalesced store per column).  The stores are
//                 streaming (evict-first): with many buckets the partials of a
//                 pixel group exceed L2 and must not evict the group's planes
// Every wait is bounded by a time limit: on expiry the CTA raises a shared
// abort flag that ends every role's loop, waits (bounded) for its issued MMAs,
// frees its TMEM, and reports the error through g_gram_error.
#include <atomic>

#include <cuda_bf16.h>

#include "train_common.cuh"

namespace mdn {
namespace tc {

constexpr int NTHREADS = 512;
constexpr int EPI_WARPS = 4;                  // warps 0..3
constexpr int MMA_WARP = 4;
constexpr int DEC_WARP = 5;
constexpr int GATHER0 = 6;                    // warps 6..15
constexpr int NG = NTHREADS / 32 - GATHER0;   // gather warps
constexpr int TMEM_COLS = 512;
constexpr int PGS = 8;                        // 16-byte chunks (pixel groups) per 128-byte K atom
constexpr int MAX_STAGES = 4;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // default bound of one wait: 2 s

__device__ int g_gram_error;   // set to 1 when a bounded wait expired
__device__ float g_one = 1.0f;                 // the ones column reads this value
__device__ unsigned short g_one_bf16 = 0x3F80;  // 1.0 in BF16 (the BF16 planes' ones column)

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

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the completion of phase `parity`: gives up after limit_ns
// (and raises the abort flag), or, when honour_abort is set, as soon as
// another role raised it.  sleep_ns > 0 backs off between polls (for roles
// whose waits are long and not latency-critical).
__device__ __noinline__ bool wait_bar(uint32_t mbar, uint32_t parity, volatile int* abortf,
                                      unsigned long long limit_ns, bool honour_abort = true, unsigned sleep_ns = 0) {
    unsigned long long t0 = 0;   // the clock is read only once a wait is long
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (try_wait(mbar, parity)) return true;
        if (sleep_ns) __nanosleep(sleep_ns);
        if ((it & 15) == 15) {
            if (honour_abort && *abortf) return false;
            if ((it & 255) == 255) {
                const unsigned long long t = global_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > limit_ns) break;
            }
        }
    }
    *abortf = 1;
    return false;
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// 4-byte asynchronous global -> shared copy; zero fill when !valid
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
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

// Precision modes
enum { P_TF32 = 0, P_BF16 = 1, P_SPLIT = 2 };

template <int MODE> struct Cfg {
    static constexpr bool TF32 = MODE == P_TF32;
    static constexpr int KB = TF32 ? 32 : 64;          // pixels per K-step (one 128-byte atom)
    static constexpr int NBUF = MODE == P_SPLIT ? 2 : 1;  // hi (+ lo) operand copies
    static constexpr int FMT = TF32 ? 2 : 1;           // TF32 = 2, BF16 = 1
    static constexpr int BSTR = KB + 4;                // ints per base array (16-byte pad: no bank aliasing)
    static constexpr int SLOT_INTS = 4 * BSTR + 4;     // bases[4][BSTR] (coarse, fine, target, zero), count
};

// One feature row of the gather: the plane pointer already offset by the
// tap's (channel, dy, dx), the row's byte offset in a stage and its swizzle.
// (The planes hold centred values, so a row is a plain copy of its taps.)
struct __align__(16) Item {
    const float* ptr;
    uint32_t meta;   // bit 0 live, bits 1-2 source (0 coarse, 1 fine, 2 target, 3 ones), bits 3-5 row mod 8, bits 8.. row byte offset
    uint32_t pad;
};

// This CTA's chunks, group after group: chunk-table indices
// [rng[2g], rng[2g + 1]) of group g.
struct ChunkIter {
    const int* rng;
    int ng, g, c;
    __device__ void skip() {
        while (g < ng && c >= rng[2 * g + 1]) {
            ++g;
            if (g < ng) c = rng[2 * g];
        }
    }
    __device__ void begin() { g = 0; c = ng > 0 ? rng[0] : 0; skip(); }
    __device__ void next() { ++c; skip(); }
    __device__ bool done() const { return g >= ng; }
};

struct Layout {
    uint32_t stage_bytes, off_pix, off_items, off_bars, total;
};

template <int MODE> __host__ __device__ inline Layout layout(int G, int rows, int S) {
    using C = Cfg<MODE>;
    Layout L;
    L.stage_bytes = (uint32_t)(G * C::NBUF * rows * 128);
    L.off_pix = S * L.stage_bytes;
    L.off_items = L.off_pix + S * C::SLOT_INTS * 4;
    L.off_bars = L.off_items + G * rows * (uint32_t)sizeof(Item);
    L.total = L.off_bars + (3 * S + 3) * 8 + 8 + 8 * GRAM_MAX_GROUPS;
    return L;
}

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gram_tc(GatherArgs ga, const int4* __restrict__ chunks, const int* __restrict__ gcount, int ngroups, int cap,
              const int* __restrict__ sorted, float* __restrict__ partial, int rows, int S,
              unsigned long long wait_ns, int expire_test) {
    using C = Cfg<MODE>;
    constexpr int KB = C::KB, BSTR = C::BSTR;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int G = ga.G, Dp = ga.Dp, Dq = ga.Dp + 1;   // Dq: features + the ones column
    const int RBG = (Dq + 7) / 8, RB = G * RBG;        // row blocks (8 feature rows) per group, in all
    const Layout L = layout<MODE>(G, rows, S);
    const uint32_t tile_bytes = (uint32_t)rows * 128;
    int* pix = reinterpret_cast<int*>(smem + L.off_pix);
    Item* items = reinterpret_cast<Item*>(smem + L.off_items);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint64_t* empty = full + S;
    uint64_t* pixfull = full + 2 * S;
    uint64_t* acc_full = full + 3 * S;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* fin = acc_full + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abortf = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int* rng = reinterpret_cast<int*>(tmem_slot + 2);   // [2 * ngroups]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up: zero stages and pixel slots, item table, barriers, TMEM
    for (uint32_t i = tid; i < L.off_items / 16; i += NTHREADS)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    for (int e = tid; e < G * rows; e += NTHREADS) {
        const int g = e / rows, f = e % rows;
        Item it;
        it.ptr = MODE == P_BF16 ? reinterpret_cast<const float*>(&g_one_bf16) : &g_one;
        it.meta = 0;
        it.pad = 0;
        if (f < Dq) {
            int src = 3, c = 0, dy = 0, dx = 0;
            if (f < Dp) {
                const int nch = ga.cross ? 3 : 1;
                const int wc = 2 * ga.rc + 1, wf = 2 * ga.rf + 1;
                const int pc = ga.rc >= 0 ? wc * wc : 0, pf = wf * wf;
                if (f < nch * pc) {
                    const int idx = f % pc;
                    src = 0; c = ga.cross ? f / pc : g; dy = idx / wc - ga.rc; dx = idx % wc - ga.rc;
                } else if (f < ga.D) {
                    const int jj = f - nch * pc, idx = jj % pf;
                    src = 1; c = ga.cross ? jj / pf : g; dy = idx / wf - ga.rf; dx = idx % wf - ga.rf;
                } else {
                    src = 2; c = ga.cross ? f - ga.D : g;
                }
            }
            // the address arithmetic is done on integers: a tap offset may be
            // negative, the base of every pixel makes the sum non-negative
            intptr_t off = 0;
            const float* plane = MODE == P_BF16 ? reinterpret_cast<const float*>(&g_one_bf16) : &g_one;
            constexpr intptr_t ESZ = MODE == P_BF16 ? 2 : 4;   // the BF16 Gram's planes hold 16-bit values
            if (src == 0) { plane = ga.cw; off = (intptr_t)c * ga.Hcp * ga.Wcp + (intptr_t)dy * ga.Wcp + dx; }
            else if (src == 1) { plane = ga.zw; off = (intptr_t)c * ga.Hp * ga.Wp + (intptr_t)dy * ga.Wp + dx; }
            else if (src == 2) { plane = ga.tw; off = (intptr_t)c * ga.h * ga.w; }
            it.ptr = reinterpret_cast<const float*>(reinterpret_cast<intptr_t>(plane) + off * ESZ);
            const uint32_t rowoff = (uint32_t)g * C::NBUF * tile_bytes + (uint32_t)(f >> 3) * 1024 + (uint32_t)(f & 7) * 128;
            it.meta = 1u | ((uint32_t)src << 1) | ((uint32_t)(f & 7) << 3) | (rowoff << 8);
        }
        items[e] = it;
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(&full[s], NG);
            bar_init(&empty[s], 1);
            bar_init(&pixfull[s], 1);
        }
        bar_init(acc_full, 1);
        bar_init(acc_empty, EPI_WARPS);
        bar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abortf = 0;
    }
    // this CTA's chunks in every group (the owner field w is non-decreasing)
    for (int g = tid; g < ngroups; g += NTHREADS) {
        const int base = g * cap, nc = gcount[g], b = blockIdx.x;
        int lo = 0, hi = nc;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (chunks[base + mid].w < b) lo = mid + 1; else hi = mid; }
        const int first = lo;
        hi = nc;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (chunks[base + mid].w <= b) lo = mid + 1; else hi = mid; }
        rng[2 * g] = base + first;
        rng[2 * g + 1] = base + lo;
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // zeroed stages visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    ChunkIter cit0;
    cit0.rng = rng;
    cit0.ng = ngroups;
    cit0.begin();


    // MMA shapes
    const bool two = Dq > 128;
    const int N1 = two ? 160 : ((Dq + 15) / 16) * 16;
    const uint32_t cols_per_group = two ? 192 : (uint32_t)N1;

    if (warp == DEC_WARP) {
        // ---------------------------------------------------------- decode
        // the sorted indices of the next K-step are loaded while this one is decoded
        const int hw = ga.h * ga.w;
        const int inv_f = ga.P * ga.Wp + ga.P;                   // pixel (0, 0): every tap in range
        const int inv_c = ga.cw ? ga.P * ga.Wcp + ga.P : 0;
        constexpr int PL = KB / 32;                              // pixels per lane
        int s = 0;
        uint32_t ph = 0;
        long long T = 0;
        ChunkIter it = cit0;
        int r0 = 0, cz = 0;
        int nxt[PL];
        auto fetch = [&](int rr0, int zz, int* dst) {
#pragma unroll
            for (int j = 0; j < PL; ++j) {
                const int e = lane + 32 * j;
                dst[j] = rr0 + e < zz ? __ldg(sorted + rr0 + e) : -1;
            }
        };
        if (!it.done()) {
            const int4 ch = chunks[it.c];
            r0 = ch.y;
            cz = ch.z;
            fetch(r0, cz, nxt);
        }
        while (!it.done()) {
            int cur[PL];
#pragma unroll
            for (int j = 0; j < PL; ++j) cur[j] = nxt[j];
            const int nv = cz - r0 < KB ? cz - r0 : KB;
            // advance to the next K-step (possibly of the next chunk) and prefetch it
            ChunkIter nx = it;
            int r1 = r0 + KB, z_n = cz;
            if (r1 >= cz) {
                nx.next();
                if (!nx.done()) { const int4 ch = chunks[nx.c]; r1 = ch.y; z_n = ch.z; }
            }
            if (!nx.done()) fetch(r1, z_n, nxt);
            if (T >= S && !wait_bar(smem_u32(&empty[s]), ph ^ 1u, abortf, wait_ns)) break;
            int* pb = pix + s * C::SLOT_INTS;
#pragma unroll
            for (int j = 0; j < PL; ++j) {
                const int e = lane + 32 * j;
                int bc = inv_c, bf = inv_f, bt = 0;
                int p = cur[j];
                if (p >= 0 && !mdn_in(p, (int64_t)ga.n * hw, 601)) p = -1;   // a pixel index past the images
                if (p >= 0) {
                    const int img = p / hw, rem = p - img * hw;
                    const int y = rem / ga.w, x = rem - y * ga.w;
                    bf = img * 3 * ga.Hp * ga.Wp + (y + ga.P) * ga.Wp + x + ga.P;
                    bt = img * 3 * hw + rem;
                    if (ga.cw) bc = img * 3 * ga.Hcp * ga.Wcp + ((y >> 1) + ga.P) * ga.Wcp + (x >> 1) + ga.P;
                }
                pb[e] = bc;
                pb[BSTR + e] = bf;
                pb[2 * BSTR + e] = bt;
            }
            if (lane == 0) pb[4 * BSTR] = nv;
            __syncwarp();
            if (lane == 0) bar_arrive(&pixfull[s]);
            ++T;
            if (++s == S) { s = 0; ph ^= 1u; }
            it = nx;
            r0 = r1;
            cz = z_n;
        }
    } else if (warp >= GATHER0) {
        // ---------------------------------------------------------- gather
        // Gather warp gw owns row blocks rb = gw, gw + NG, ... (8 feature rows
        // each) and fills all 8 pixel chunks of every K-step for them.  Lane
        // (r, e) = (lane / 4, lane % 4) handles row r of a block and the e-th
        // 4-byte word of each 16-byte chunk (one TF32 pixel or two BF16
        // pixels), so the 32 lanes of a store cover 8 rows x 16 bytes: 8
        // distinct swizzled chunks.
        const int gw = warp - GATHER0;
        const int lr = lane >> 2, le = lane & 3;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        auto item_of = [&](int rb) -> Item {
            const int g = rb / RBG, f = (rb - g * RBG) * 8 + lr;
            return items[g * rows + f];
        };
        // TF32 gathers with cp.async: on 16 x 1 MP of cross-channel 7x7x3
        // patches a whole level took 5.8 ms this way and 6.2 ms through the
        // register path below (which BF16 and split BF16 use).
        if constexpr (MODE == P_TF32) {
            // TF32: the planes already hold the rounded operands, so each lane
            // copies one value per chunk with a 4-byte cp.async straight into
            // the swizzled tile (zero fill past the chunk end).  Two K-steps
            // are in flight: step n's stage is published once step n - 1's
            // copies landed.
            int pend = -1;   // stage of the previous, still unpublished step
            for (ChunkIter it = cit0; !it.done() && ok; it.next()) {
                const int4 ch = chunks[it.c];
                for (int r0 = ch.y; r0 < ch.z; r0 += KB) {
                    if (!wait_bar(smem_u32(&pixfull[s]), ph, abortf, wait_ns)) { ok = false; break; }
                    const int* pb = pix + s * C::SLOT_INTS;
                    const int nv = pb[4 * BSTR];
                    const uint32_t stage = smem_u32(smem + s * L.stage_bytes);
                    for (int rb = gw; rb < RB; rb += NG) {
                        const Item it2 = item_of(rb);
                        if (!(it2.meta & 1u)) continue;
                        const int* bsrc = pb + ((it2.meta >> 1) & 3u) * BSTR + le;
                        const uint32_t rowb = stage + (it2.meta >> 8) + 4 * le;
                        const uint32_t sw = (it2.meta >> 3) & 7u;
#pragma unroll
                        for (int pg = 0; pg < PGS; ++pg)
                            cp_async4(rowb + ((pg ^ sw) << 4), it2.ptr + bsrc[4 * pg], 4 * pg + le < nv);
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    if (pend >= 0) {
                        asm volatile("cp.async.wait_group 1;" ::: "memory");
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) bar_arrive(&full[pend]);
                    }
                    pend = s;
                    if (++s == S) { s = 0; ph ^= 1u; }
                }
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (pend >= 0 && ok) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) bar_arrive(&full[pend]);
            }
        } else {
            // Register path: lane (r, e) loads pixel e (TF32) or pixels 2e, 2e+1
            // (BF16) of each chunk and stores them as one 4-byte word; the loads
            // of two row blocks (16 or 32 per lane) are issued before any of
            // them is stored.
            constexpr int PPL = MODE == P_TF32 ? 1 : 2;
            for (ChunkIter it = cit0; !it.done() && ok; it.next()) {
                const int4 ch = chunks[it.c];
                for (int r0 = ch.y; r0 < ch.z; r0 += KB) {
                    if (!wait_bar(smem_u32(&pixfull[s]), ph, abortf, wait_ns)) { ok = false; break; }
                    const int* pb = pix + s * C::SLOT_INTS;
                    const int nv = pb[4 * BSTR];
                    unsigned char* stage = smem + s * L.stage_bytes;
                    for (int rb0 = gw; rb0 < RB; rb0 += 2 * NG) {
                        float v0[2][PGS], v1[2][PGS];
                        uint32_t rowb[2], sw[2];
                        bool live[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int rb = rb0 + h * NG;
                            live[h] = false;
                            rowb[h] = 0;
                            sw[h] = 0;
#pragma unroll
                            for (int pg = 0; pg < PGS; ++pg) v0[h][pg] = v1[h][pg] = 0.f;
                            if (rb < RB) {
                                const Item it2 = item_of(rb);
                                if (it2.meta & 1u) {
                                    live[h] = true;
                                    const int* bsrc = pb + ((it2.meta >> 1) & 3u) * BSTR + PPL * le;
                                    rowb[h] = (it2.meta >> 8) + 4 * le;
                                    sw[h] = (it2.meta >> 3) & 7u;
#pragma unroll
                                    for (int pg = 0; pg < PGS; ++pg) {
                                        if constexpr (MODE == P_TF32) {
                                            v0[h][pg] = __ldg(it2.ptr + bsrc[4 * pg]);
                                        } else {
                                            const int2 b = *reinterpret_cast<const int2*>(bsrc + 8 * pg);
                                            if constexpr (MODE == P_BF16) {
                                                // BF16 planes: the operands themselves, kept as bit patterns
                                                const unsigned short* p16 = reinterpret_cast<const unsigned short*>(it2.ptr);
                                                v0[h][pg] = __uint_as_float((uint32_t)__ldg(p16 + b.x));
                                                v1[h][pg] = __uint_as_float((uint32_t)__ldg(p16 + b.y));
                                            } else {
                                                v0[h][pg] = __ldg(it2.ptr + b.x);
                                                v1[h][pg] = __ldg(it2.ptr + b.y);
                                            }
                                        }
                                    }
                                }
                            }
                        }
                        if (nv < KB) {   // ragged last K-step of a chunk
#pragma unroll
                            for (int h = 0; h < 2; ++h)
#pragma unroll
                                for (int pg = 0; pg < PGS; ++pg) {
                                    const int px = 4 * PPL * pg + PPL * le;
                                    if (px >= nv) v0[h][pg] = 0.f;
                                    if (px + 1 >= nv) v1[h][pg] = 0.f;
                                }
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (!live[h]) continue;
#pragma unroll
                            for (int pg = 0; pg < PGS; ++pg) {
                                unsigned char* dst = stage + rowb[h] + ((pg ^ sw[h]) << 4);
                                if constexpr (MODE == P_TF32) {
                                    *reinterpret_cast<float*>(dst) = v0[h][pg];   // the plane holds TF32 values
                                } else if constexpr (MODE == P_BF16) {
                                    // two 16-bit patterns (zero past the chunk end) -> one bf16x2 word
                                    *reinterpret_cast<uint32_t*>(dst) =
                                        __float_as_uint(v0[h][pg]) | (__float_as_uint(v1[h][pg]) << 16);
                                } else {
                                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0[h][pg], v1[h][pg]);
                                    *reinterpret_cast<__nv_bfloat162*>(dst) = h2;
                                    const float2 hf = __bfloat1622float2(h2);
                                    *reinterpret_cast<__nv_bfloat162*>(dst + tile_bytes) =
                                        __floats2bfloat162_rn(v0[h][pg] - hf.x, v1[h][pg] - hf.y);
                                }
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) bar_arrive(&full[s]);
                    if (++s == S) { s = 0; ph ^= 1u; }
                }
            }
        }
    } else if (warp == MMA_WARP) {
        // ---------------------------------------------------------- MMA issue
        if (lane == 0) {
            const uint32_t idesc1 = make_idesc(C::FMT, 128, N1);
            const uint32_t idesc2 = make_idesc(C::FMT, 128, 32);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            int q = 0;
            // failure-detection test: wait on phase 0 of `fin`, on which nothing
            // arrives before this thread's own commit below, so the wait runs
            // out after wait_ns and takes the abort path (no MMA issued yet)
            if (expire_test && !wait_bar(smem_u32(fin), 0u, abortf, wait_ns)) ok = false;
            for (ChunkIter it = cit0; !it.done() && ok; it.next(), ++q) {
                const int4 ch = chunks[it.c];
                if (q > 0) {
                    if (!wait_bar(smem_u32(acc_empty), (uint32_t)((q - 1) & 1), abortf, wait_ns)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                for (int r0 = ch.y; r0 < ch.z; r0 += KB) {
                    if (!wait_bar(smem_u32(&full[s]), ph, abortf, wait_ns)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sbase = smem_u32(smem + s * L.stage_bytes);
                    const bool first = r0 == ch.y;
                    for (int g = 0; g < G; ++g) {
                        // descriptors of the group's hi (and lo) tiles; the start address field
                        // (address / 16) advances by 2 per 32-byte K slice, by 256 per 4 KB
                        // (32 rows) and by 1024 per 16 KB (128 rows)
                        const uint64_t dhi = make_desc(sbase + (uint32_t)g * C::NBUF * tile_bytes);
                        const uint64_t dlo = dhi + (tile_bytes >> 4);
                        const uint32_t d1 = tmem + (uint32_t)g * cols_per_group;
                        const uint32_t d2 = d1 + 160;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t acc = (!first || k > 0) ? 1u : 0u;
                            constexpr int npairs = MODE == P_SPLIT ? 3 : 1;
#pragma unroll
                            for (int pr = 0; pr < npairs; ++pr) {
                                const uint64_t da = (pr == 2 ? dlo : dhi) + 2 * k;
                                const uint64_t db = (pr == 1 ? dlo : dhi) + 2 * k;
                                const uint32_t accp = pr > 0 ? 1u : acc;
                                mma<C::TF32>(d1, da, db, idesc1, accp);
                                if (two) mma<C::TF32>(d2, da + 256, db + 1024, idesc2, accp);
                            }
                        }
                    }
                    commit(smem_u32(&empty[s]));
                    if (++s == S) { s = 0; ph ^= 1u; }
                }
                if (!ok) break;
                commit(smem_u32(acc_full));
            }
            // all issued MMAs complete before TMEM is released (always with the
            // default 2 s bound, whatever the wait limit of the launch)
            commit(smem_u32(fin));
            wait_bar(smem_u32(fin), 0u, abortf, WAIT_NS, false);
        }
    } else {
        // ---------------------------------------------------------- read-back (warps 0..3)
        const int row = 32 * warp + lane;   // TMEM lane = accumulator row
        int q = 0;
        for (ChunkIter it = cit0; !it.done(); it.next(), ++q) {
            if (!wait_bar(smem_u32(acc_full), (uint32_t)(q & 1), abortf, wait_ns, true, 500)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float* out = partial + (size_t)it.c * G * Dq * Dq;
            for (int g = 0; g < G; ++g) {
                float* og = out + (size_t)g * Dq * Dq;
                const uint32_t d1 = tmem + (uint32_t)g * cols_per_group + ((uint32_t)(32 * warp) << 16);
                for (int c0_ = 0; c0_ < N1; c0_ += 16) {
                    float v[16];
                    tmem_ld16(d1 + c0_, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = c0_ + e;
                        if (row < Dq && j < Dq && row <= j) __stcs(og + (size_t)j * Dq + row, v[e]);   // lanes: consecutive
                    }
                }
                if (two) {
                    for (int c0_ = 0; c0_ < 32; c0_ += 16) {
                        float v[16];
                        tmem_ld16(d1 + 160 + c0_, v);
                        const int i = 32 + row;      // accumulator row m -> feature 32 + m
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int j = 128 + c0_ + e;
                            if (i >= 128 && i < Dq && j < Dq && i <= j) __stcs(og + (size_t)j * Dq + i, v[e]);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(acc_empty);
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abortf) atomicExch(&g_gram_error, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Wait bound of the next launches (0 = the default) and the one-shot
// expiry test (see mdn_set_gram_wait_limit / mdn_gram_expire_next_wait).
static std::atomic<unsigned long long> g_wait_ns{0};
static std::atomic<int> g_expire_next{0};

template <int MODE>
int run(const GatherArgs& ga, const int4* chunks, const int* gcount, int ngroups, int cap, const int* sorted,
        float* partial, int ncta, cudaStream_t s) {
    const int Dq = ga.Dp + 1;
    const int rows = Dq > 128 ? 160 : 128;
    if (ga.G * (Dq > 128 ? 192 : ((Dq + 15) / 16) * 16) > TMEM_COLS)
        return fail(MDN_ESHAPE, "train: Gram accumulators exceed tensor memory");
    if (ngroups > GRAM_MAX_GROUPS) return fail(MDN_ESHAPE, "train: too many pixel groups");
    constexpr int SMEM_MAX = 232448 - 1024;   // opt-in maximum less the alignment slack
    int S = MAX_STAGES;
    while (S > 2 && (int)layout<MODE>(ga.G, rows, S).total > SMEM_MAX) --S;
    const Layout L = layout<MODE>(ga.G, rows, S);
    if ((int)L.total > SMEM_MAX) return fail(MDN_ESHAPE, "train: tensor-core Gram tile does not fit in shared memory");
    // at least 120 KB so that one CTA (and its 512 TMEM columns) owns the SM
    size_t bytes = (size_t)L.total + 1024;
    if (bytes < 120 * 1024) bytes = 120 * 1024;
    auto kern = k_gram_tc<MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "k_gram_tc: smem attribute");
    if (ncta <= 0 || ngroups <= 0) return MDN_OK;
    const unsigned long long wait_ns = g_wait_ns.load() ? g_wait_ns.load() : WAIT_NS;
    const int expire = g_expire_next.exchange(0);
    kern<<<(unsigned)ncta, NTHREADS, bytes, s>>>(ga, chunks, gcount, ngroups, cap, sorted, partial, rows, S, wait_ns,
                                                 expire);
    return check_launch("k_gram_tc");
}

}  // namespace tc

int launch_gram_tc(const GatherArgs& ga, int precision, const int4* chunks, const int* gcount, int ngroups, int cap,
                   const int* sorted, float* partial, int ncta, cudaStream_t s) {
    if (ga.Dp + 1 > 160) return fail(MDN_ESHAPE, "train: tensor-core Gram supports D + T <= 159");
    switch (precision) {
        case MDN_GRAM_TF32: return tc::run<tc::P_TF32>(ga, chunks, gcount, ngroups, cap, sorted, partial, ncta, s);
        case MDN_GRAM_BF16: return tc::run<tc::P_BF16>(ga, chunks, gcount, ngroups, cap, sorted, partial, ncta, s);
        case MDN_GRAM_SPLIT_BF16:
            return tc::run<tc::P_SPLIT>(ga, chunks, gcount, ngroups, cap, sorted, partial, ncta, s);
        default: return fail(MDN_EINVAL, "train: bad Gram precision");
    }
}

void gram_tc_set_wait(unsigned long long ns) { tc::g_wait_ns.store(ns); }
void gram_tc_expire_next(int enable) { tc::g_expire_next.store(enable ? 1 : 0); }

int gram_tc_error(int* out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, tc::g_gram_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tc::g_gram_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "gram error flag");
    *out = v;
    return MDN_OK;
}

}  // namespace mdn
