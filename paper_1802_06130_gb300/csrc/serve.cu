// serve.cu -- continuous-batching denoise server (A8): native scheduler,
// device arena, batched per-stage kernels replayed from CUDA graphs, and a
// level-kernel autotuner.
//
// A request is upload -> pyramid level 1 .. L-1 -> filter level L-2 .. 0 ->
// download.  The scheduler thread forms a tick from queued requests when a
// tick context (its own upload, compute and download streams, device work
// list and captured graph) is free and the arena has room: all of the tick's
// requests run their whole chain in one replay of the context's graph, whose
// nodes are one batched pyramid launch per level and one batched filter
// launch per level (filter items sorted by bank); every launch reads its
// stage's items from the device work list, so the graph never changes.
//
// Requests come in two size classes.  Large ones (at least LARGE_PIXELS
// finest-level pixels, e.g. 12 MP camera frames) run one per tick on the
// large contexts, whose compute streams have the lowest priority; small
// ones are batched (up to ~4 MP a tick) on the small contexts, whose compute
// streams have the highest priority, so their kernels start as soon as SMs
// free up between a large tick's launches.  Because every context has its own
// streams, a small tick's upload, kernels and download never queue behind a
// large tick's in a stream (on Grace hosts a 73 MB copy to or from a pinned
// buffer the GPU has not used recently can take 10-30x its usual 0.4 ms;
// with one download stream every later request waited for it).  Within a
// class, requests are admitted in FIFO order.  The scheduler polls each
// in-flight tick's download event and then releases the tick's arena space.
// Per-pixel arithmetic is that of the per-image path, so results do not
// depend on the batch or the class.
//
// Host transfers are SM copy kernels, not copy-engine copies.  On the Grace
// host a copy-engine transfer to or from a pinned buffer that the GPU has not
// used for a second or more runs at ~7-10 GB/s instead of ~190 (7-10 ms for
// a 12 MP FP16 frame), and serving rotates through many user buffers; SM
// loads and stores of the same memory overlap their address translations
// across many warps (1.3-3 ms when cold, the copy engines' speed when hot).
// The level and pyramid kernels leave COPY_SMS SMs free, which is enough for
// a copy kernel to run the host link at full speed while they compute.
// Buffers that are not pinned or not 16-byte aligned use the copy engines.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "k_level.cuh"
#include "pyramid.cuh"

struct mdn_server;   // defined below (outside the namespace, as declared in mdn.h)

namespace mdn {
namespace srv {
namespace v2 = lvl::v2;

constexpr int MAX_ITEMS = 256;      // requests per tick
constexpr int MAX_LEVELS = 8;
constexpr int MAX_STAGE_ITEMS = MAX_ITEMS * (MAX_LEVELS - 1);
constexpr int MAX_BANKS = 64;
constexpr int NCTX_LARGE = 2, NCTX_SMALL = 4;   // tick contexts per size class
constexpr int NCTX = NCTX_LARGE + NCTX_SMALL;
constexpr int64_t TICK_PIXELS = 4200000;    // a small tick takes more requests only while under this (finest) size
constexpr int64_t LARGE_PIXELS = 4000000;   // requests of at least this many pixels are large
constexpr int RF = 3, RC = 3;       // geometry of the tile kernels (variants 0-2)
constexpr bool CROSS = false;
constexpr int NVAR = 4;             // level-kernel variants: 0-2 tile kernels, 3 the fused kernel
constexpr int COPY_SMS = 8;         // SMs the level and pyramid kernels leave to the host copies
constexpr int COPY_NT = 256, COPY_BLOCKS = 4 * COPY_SMS;
// SMs the server's compute kernels are sized for (all but COPY_SMS, at least one)
inline int compute_sms() { return num_sms() > COPY_SMS ? num_sms() - COPY_SMS : 1; }

struct PyrItem {
    const __half* in;
    __half* out;
    int H, W, Ho, Wo, tiles_x, tile_start;
};
struct LvlItem {
    const __half* z;
    const __half* coarse;
    __half* out;
    int H, W, Hc, Wc, bank, tiles_x, tile_start, pad;
};
// Items of stage l: pyr[pyr_begin[l] .. pyr_begin[l] + pyr_n[l]) builds
// pyramid level l (1..7); lvl[lvl_begin[l] .. + lvl_n[l]) filters level l
// (0..6).  tile_start is relative to the stage.
// one host <-> device transfer of whole 16-byte units (the tail goes by copy engine)
struct CopyItem {
    const uint4* src;
    uint4* dst;
    int64_t n16;
};
struct WorkList {
    int pyr_begin[MAX_LEVELS], pyr_n[MAX_LEVELS], pyr_tiles[MAX_LEVELS];
    int lvl_begin[MAX_LEVELS], lvl_n[MAX_LEVELS], lvl_tiles[MAX_LEVELS];
    int n_up, n_down;
    PyrItem pyr[MAX_STAGE_ITEMS];
    LvlItem lvl[MAX_STAGE_ITEMS];
    CopyItem up[MAX_ITEMS], down[MAX_ITEMS];
};
struct Tables {
    const __half* bank[MAX_BANKS];
    const unsigned char* rows[MAX_BANKS];   // the same banks as prepared row slots (fused kernel)
    int K[MAX_BANKS];
    int color[MAX_BANKS];
    SelParams sel[MAX_BANKS];
    float w[3];
};

// ---------------------------------------------------------------- kernels

__global__ void __launch_bounds__(pyr::PNT) k_serve_pyr(const WorkList* __restrict__ wl, int stage) {
    __shared__ float tile[pyr::PIH][pyr::PIW];
    __shared__ float hs[pyr::PIH][pyr::PTX + 1];
    const int n = wl->pyr_n[stage], T = wl->pyr_tiles[stage], b = wl->pyr_begin[stage];
    for (int gt = blockIdx.x; gt < 3 * T; gt += gridDim.x) {
        const int ch = gt / T, t = gt % T;
        int lo = 0, hi = n - 1;   // last item with tile_start <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (wl->pyr[b + mid].tile_start <= t) lo = mid; else hi = mid - 1;
        }
        const PyrItem& it = wl->pyr[mdn_in(b + lo, MAX_STAGE_ITEMS, 501) ? b + lo : 0];
        const int lt = t - it.tile_start;
        __syncthreads();   // shared buffers free
        pyr::tile_down(it.in + (int64_t)ch * it.H * it.W, it.out + (int64_t)ch * it.Ho * it.Wo, it.H, it.W, it.Ho,
                       it.Wo, (lt % it.tiles_x) * pyr::PTX, (lt / it.tiles_x) * pyr::PTY, tile, hs);
    }
}

template <class SH>
__global__ void __launch_bounds__(SH::NT, 1) k_serve_level(const WorkList* __restrict__ wl,
                                                           const Tables* __restrict__ tb, int stage) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* bank_s = smem + ((v2::tile_bytes<SH, RC>() + 15) & ~size_t(15));
    __shared__ SelParams sp;
    const int T = wl->lvl_tiles[stage], n = wl->lvl_n[stage];
    const LvlItem* items = wl->lvl + wl->lvl_begin[stage];
    const int per = (T + gridDim.x - 1) / gridDim.x;
    const int begin = blockIdx.x * per, end = min(T, begin + per);
    const float wv[5] = {tb->w[0], tb->w[1], tb->w[2], tb->w[1], tb->w[0]};
    int cur_bank = -1, item = 0;
    for (int t = begin; t < end; ++t) {
        while (item + 1 < n && items[item + 1].tile_start <= t) ++item;
        const LvlItem& it = items[mdn_in(wl->lvl_begin[stage] + item, MAX_STAGE_ITEMS, 502) ? item : 0];
        __syncthreads();   // previous tile finished with the shared buffers
        if (!mdn_in(it.bank, MAX_BANKS, 503)) continue;
        if (it.bank != cur_bank) {
            // items are sorted by bank: a CTA's contiguous tile range rarely switches
            lvl::v3::load_bank_rows<RF, RC, CROSS, __half>(tb->bank[it.bank], tb->K[it.bank], bank_s, threadIdx.x,
                                                           SH::NT);
            if (threadIdx.x == 0) sp = tb->sel[it.bank];
            cur_bank = it.bank;
            __syncthreads();
        }
        const int lt = t - it.tile_start;
        v2::tile_v2<SH, RF, RC, CROSS, __half, __half, true>(smem, bank_s, it.z, it.coarse, it.out, nullptr, it.H, it.W,
                                                       it.Hc, it.Wc, (lt % it.tiles_x) * SH::TW,
                                                       (lt / it.tiles_x) * SH::TH, tb->K[it.bank],
                                                       tb->color[it.bank], sp, wv);
    }
}

// A tick's uploads (down = 0) or downloads (down = 1): every item copied by
// the whole grid, four independent 16-byte loads in flight per thread.
__global__ void __launch_bounds__(COPY_NT) k_host_copy(const WorkList* __restrict__ wl, int down) {
    const int n = down ? wl->n_down : wl->n_up;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int k = 0; k < n; ++k) {
        const CopyItem it = (down ? wl->down : wl->up)[mdn_in(k, MAX_ITEMS, 506) ? k : 0];
        const uint4* __restrict__ src = it.src;
        uint4* __restrict__ dst = it.dst;
        const size_t m = (size_t)it.n16;
        size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
        for (; i + 3 * stride < m; i += 4 * stride) {
            const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
            dst[i] = a;
            dst[i + stride] = b;
            dst[i + 2 * stride] = c;
            dst[i + 3 * stride] = d;
        }
        for (; i < m; i += stride) dst[i] = src[i];
    }
}

// deterministic structured test pattern for the autotuner (no host data)
__global__ void k_fill_pattern(__half* p, int H, int W) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * (int64_t)H * W) return;
    int c = (int)(i / ((int64_t)H * W)), r = (int)(i % ((int64_t)H * W));
    int y = r / W, x = r % W;
    uint32_t hsh = (uint32_t)i * 2654435761u;
    hsh ^= hsh >> 13;
    float noise = ((hsh & 0xffff) / 65535.f - 0.5f) * 0.3f;
    float v = 0.5f + 0.3f * __sinf(0.05f * x + 0.07f * y + c) + noise;
    p[i] = __float2half_rn(v);
}

// ---------------------------------------------------------------- tile shapes

using S0 = v2::Shape<256, 4>;
using S1 = v2::Shape<384, 4>;
using S2 = v2::Shape<512, 2>;

template <class SH> size_t level_smem(int Kmax) {
    return ((v2::tile_bytes<SH, RC>() + 15) & ~size_t(15)) +
           (size_t)Kmax * lvl::v3::bucket_bytes_rows<RF, RC, CROSS, __half>();
}

template <class SH> int launch_level(const WorkList* wl, const Tables* tb, int Kmax, int stage, cudaStream_t s) {
    auto kern = k_serve_level<SH>;
    const size_t bytes = level_smem<SH>(Kmax);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "server: level kernel smem attribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SH::NT, bytes);
    if (e != cudaSuccess || occ < 1) return fail(MDN_ESHAPE, "server: level kernel does not fit");
    kern<<<compute_sms() * occ, SH::NT, bytes, s>>>(wl, tb, stage);
    return check_launch("k_serve_level");
}

// Tile source of one filter stage of a tick for the fused kernel: the
// stage's items (requests of any size and bank set, sorted by bank) in the
// device work list, each item's 32 x 32 tiles row-major after those of the
// items before it; every tile reads its own item's prepared bank and
// selector parameters.
template <typename BT> struct StageTiles {
    const WorkList* wl;
    const Tables* tb;
    int stage;
    __device__ __forceinline__ int64_t count() const { return wl->lvl_tiles[stage]; }
    __device__ __forceinline__ lvl::v3::TileRef<__half, BT> at(int64_t tile) const {
        const int n = wl->lvl_n[stage], b = wl->lvl_begin[stage];
        int lo = 0, hi = n - 1;   // last item with tile_start <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (wl->lvl[b + mid].tile_start <= tile) lo = mid; else hi = mid - 1;
        }
        const LvlItem& it = wl->lvl[mdn_in(b + lo, MAX_STAGE_ITEMS, 504) ? b + lo : 0];
        const int bk = mdn_in(it.bank, MAX_BANKS, 505) ? it.bank : 0;
        const int lt = (int)tile - it.tile_start;
        lvl::v3::TileRef<__half, BT> t;
        t.z = it.z;
        t.coarse = it.coarse;
        t.out = it.out;
        t.bmap = nullptr;
        t.bank = tb->rows[bk];
        t.H = it.H; t.W = it.W; t.Hc = it.Hc; t.Wc = it.Wc;
        t.x0 = (lt % it.tiles_x) * lvl::v3::TW;
        t.y0 = (lt / it.tiles_x) * lvl::v3::TH;
        t.K = tb->K[bk];
        t.color = tb->color[bk];
        t.item = bk;
        return t;
    }
    __device__ __forceinline__ const SelParams& sel(int bk) const { return tb->sel[bk]; }
};

// the fused warp-specialised level kernel over a stage's work list, banks read through L2
template <int RF_, int RC_, bool CROSS_, typename BT>
int launch_fused(const WorkList* wl, const Tables* tb, int stage, cudaStream_t s) {
    using SRC = StageTiles<BT>;
    auto kern = lvl::v3::k_level3<RF_, RC_, CROSS_, __half, __half, true, BT, SRC>;
    const size_t bytes = lvl::v3::smem_need<RF_, RC_, CROSS_, __half, true, (int)sizeof(BT)>(0);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "server: fused level kernel smem attribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, lvl::v3::NT, bytes);
    if (e != cudaSuccess || occ < 1) return fail(MDN_ESHAPE, "server: fused level kernel does not fit");
    SRC src{wl, tb, stage};
    float w[5];
    gauss5_weights(w);
    kern<<<compute_sms() * occ, lvl::v3::NT, bytes, s>>>(src, nullptr, w[0], w[1], w[2], 1);
    return check_launch("k_level3 (server)");
}

// geometry of the server's banks (7x7 + 7x7 or 7x7 + 5x5 per channel) and bucket-index width
int launch_fused_geom(const mdn_geometry& g, int Kmax, const WorkList* wl, const Tables* tb, int stage,
                      cudaStream_t s) {
    if (g.r_fine == 3 && g.r_coarse == 3)
        return Kmax <= 256 ? launch_fused<3, 3, false, uint8_t>(wl, tb, stage, s)
                           : launch_fused<3, 3, false, uint16_t>(wl, tb, stage, s);
    return Kmax <= 256 ? launch_fused<3, 2, false, uint8_t>(wl, tb, stage, s)
                       : launch_fused<3, 2, false, uint16_t>(wl, tb, stage, s);
}

int launch_variant(int v, const mdn_geometry& g, const WorkList* wl, const Tables* tb, int Kmax, int stage,
                   cudaStream_t s) {
    switch (v) {
        case 0: return launch_level<S0>(wl, tb, Kmax, stage, s);
        case 1: return launch_level<S1>(wl, tb, Kmax, stage, s);
        case 2: return launch_level<S2>(wl, tb, Kmax, stage, s);
        default: return launch_fused_geom(g, Kmax, wl, tb, stage, s);
    }
}
int variant_threads(int v) { return v == 0 ? S0::NT : v == 1 ? S1::NT : v == 2 ? S2::NT : lvl::v3::NT; }
int variant_rows(int v) { return v == 0 ? S0::TH : v == 1 ? S1::TH : v == 2 ? S2::TH : lvl::v3::TH; }
int variant_tile_rows(int v) { return variant_rows(v); }

// ---------------------------------------------------------------- arena

// First-fit allocator over one device block; free ranges coalesce.
class Arena {
  public:
    void init(char* base, size_t bytes) {
        base_ = base;
        size_ = bytes;
        free_.clear();
        free_[0] = bytes;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* ptr(size_t off) const { return base_ + off; }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    char* base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t id;
    const void* host_in;
    void* host_out;
    int h, w, set, levels;
    size_t off = 0, bytes = 0;
    __half* z[9] = {};   // z[0] = input, z[l] = pyramid level l
    __half* u[9] = {};   // u[l] = level-l output (u[0] = output)
    int hl[9], wl[9];
    double t_submit = 0, t_admit = 0, t_done = 0;
    const void* dev_in = nullptr;   // device addresses of pinned, 16-byte aligned host buffers (SM copies),
    void* dev_out = nullptr;        // else null (copy engines)
};

size_t request_bytes(int h, int w, int levels) {
    size_t tot = 0;
    int hh = h, ww = w;
    tot += 2 * align256((size_t)3 * h * w * 2);   // input + output
    for (int l = 1; l < levels; ++l) {
        hh = (hh + 1) / 2;
        ww = (ww + 1) / 2;
        tot += align256((size_t)3 * hh * ww * 2);                       // z^l
        if (l <= levels - 2) tot += align256((size_t)3 * hh * ww * 2);  // u^l
    }
    return tot;
}

}  // namespace srv
}  // namespace mdn

using namespace mdn;
using namespace mdn::srv;

struct TickCtx {
    cudaStream_t stream = nullptr;   // capture stream of this context's graph
    cudaStream_t s_up = nullptr, s_comp = nullptr, s_down = nullptr;
    bool large = false;              // size class served by this context
    cudaEvent_t ev_up = nullptr, ev_comp = nullptr, ev_done = nullptr;
    // tracing only (MDN_SERVER_TRACE): starts of the upload, compute and download phases
    cudaEvent_t ev_t0 = nullptr, ev_cstart = nullptr, ev_dstart = nullptr;
    double t_launch = 0;
    int64_t pixels = 0;
    uint64_t tick_id = 0;
    WorkList* d_wl = nullptr;
    WorkList* h_wl = nullptr;   // pinned staging
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
};

struct mdn_server {
    int device = 0;
    char* arena_mem = nullptr;
    Arena arena;
    Tables* d_tb = nullptr;
    TickCtx ctx[NCTX];
    int max_active = 16;
    int max_levels = 2;
    int variant = 3;
    float variant_ms[NVAR] = {-1, -1, -1, -1};
    int Kmax = 0;
    mdn_geometry geom{3, 3, 0, MDN_YCBCR601};   // bank geometry (7x7 + 7x7 or 7x7 + 5x5 per channel)
    bool tile_ok = true;          // tile kernels (variants 0-2) apply: 7x7 + 7x7 and K <= 256
    unsigned char* rows_mem = nullptr;   // prepared row slots of every bank
    bool copy_engines = false;           // MDN_SERVER_COPY_ENGINES=1: host transfers by copy engine only
    struct Set {
        int levels;
        int bank_index[8];   // table index of level l's bank
    };
    std::vector<Set> sets;
    // scheduling state (guarded by mu)
    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-up: submissions, tick completions, stop
    std::condition_variable cv_done;  // pollers
    std::deque<Request> queue[2];     // [0] small, [1] large requests
    int inflight = 0;
    std::deque<mdn_result> done;
    std::thread thread;
    std::atomic<bool> stop{false};
    std::atomic<int> thread_error{0};
    uint64_t next_id = 1;
    // per-tick trace (environment variable MDN_SERVER_TRACE = output CSV path)
    std::string trace_path;
    std::vector<std::string> trace_rows;
    mdn_server_stats st{};
    std::chrono::steady_clock::time_point t0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    void run();
    int launch_tick(TickCtx& c);
};

static int build_tables(mdn_server* s, const mdn_bankset* sets, int nsets, Tables* tb) {
    std::memset(tb, 0, sizeof(*tb));
    float w[5];
    gauss5_weights(w);
    tb->w[0] = w[0]; tb->w[1] = w[1]; tb->w[2] = w[2];
    int nb = 0;
    for (int i = 0; i < nsets; ++i) {
        const mdn_bankset& bs = sets[i];
        if (bs.levels < 2 || bs.levels > MAX_LEVELS || !bs.banks || !bs.bparams)
            return fail(MDN_EINVAL, "server: bank set needs levels 2..8, banks and bparams");
        if (bs.color != MDN_YCBCR601 && bs.color != MDN_RGB) return fail(MDN_EINVAL, "server: bad colour space");
        mdn_server::Set st{};
        st.levels = bs.levels;
        s->max_levels = std::max(s->max_levels, bs.levels);
        for (int l = 0; l < bs.levels - 1; ++l) {
            if (nb >= MAX_BANKS) return fail(MDN_EINVAL, "server: more than 64 banks");
            if (!bs.banks[l]) return fail(MDN_EINVAL, "server: null bank");
            int rc = make_sel_params(&bs.bparams[l], &tb->sel[nb]);
            if (rc) return rc;
            tb->bank[nb] = (const __half*)bs.banks[l];
            tb->K[nb] = bs.bparams[l].n_angle * bs.bparams[l].n_strength * bs.bparams[l].n_coherence;
            if (tb->K[nb] > MDN_MAX_K) return fail(MDN_ESHAPE, "server: a bank set level has more than 4096 buckets");
            tb->color[nb] = bs.color;
            s->Kmax = std::max(s->Kmax, tb->K[nb]);
            st.bank_index[l] = nb++;
        }
        s->sets.push_back(st);
    }
    return MDN_OK;
}

// Work list of one tick: every request's whole chain, grouped by stage.
static void build_worklist(const mdn_server* s, std::vector<Request>& reqs, WorkList* wl) {
    const int TH = variant_tile_rows(s->variant);
    int np = 0, nl = 0;
    for (int l = 1; l < MAX_LEVELS; ++l) {   // pyramid stages: level l from l-1
        wl->pyr_begin[l] = np;
        int tiles = 0;
        for (auto& r : reqs) {
            if (l >= r.levels) continue;
            PyrItem& p = wl->pyr[np++];
            p.in = r.z[l - 1];
            p.out = r.z[l];
            p.H = r.hl[l - 1]; p.W = r.wl[l - 1]; p.Ho = r.hl[l]; p.Wo = r.wl[l];
            p.tiles_x = (p.Wo + pyr::PTX - 1) / pyr::PTX;
            p.tile_start = tiles;
            tiles += p.tiles_x * ((p.Ho + pyr::PTY - 1) / pyr::PTY);
        }
        wl->pyr_n[l] = np - wl->pyr_begin[l];
        wl->pyr_tiles[l] = tiles;
    }
    wl->pyr_begin[0] = wl->pyr_n[0] = wl->pyr_tiles[0] = 0;
    wl->n_up = wl->n_down = 0;
    for (auto& r : reqs) {
        const int64_t n16 = (int64_t)3 * r.h * r.w * 2 / 16;
        if (r.dev_in) wl->up[wl->n_up++] = CopyItem{(const uint4*)r.dev_in, (uint4*)r.z[0], n16};
        if (r.dev_out) wl->down[wl->n_down++] = CopyItem{(const uint4*)r.u[0], (uint4*)r.dev_out, n16};
    }
    for (int l = 0; l < MAX_LEVELS; ++l) {   // filter stages, items sorted by bank
        std::vector<LvlItem> items;
        for (auto& r : reqs) {
            if (l > r.levels - 2) continue;
            LvlItem it{};
            it.z = r.z[l];
            it.coarse = (l == r.levels - 2) ? r.z[r.levels - 1] : r.u[l + 1];
            it.out = r.u[l];
            it.H = r.hl[l]; it.W = r.wl[l]; it.Hc = r.hl[l + 1]; it.Wc = r.wl[l + 1];
            it.bank = s->sets[r.set].bank_index[l];
            items.push_back(it);
        }
        std::stable_sort(items.begin(), items.end(), [](const LvlItem& a, const LvlItem& b) { return a.bank < b.bank; });
        wl->lvl_begin[l] = nl;
        int tiles = 0;
        for (auto& it : items) {
            it.tiles_x = (it.W + 31) / 32;
            it.tile_start = tiles;
            tiles += it.tiles_x * ((it.H + TH - 1) / TH);
            wl->lvl[nl++] = it;
        }
        wl->lvl_n[l] = (int)items.size();
        wl->lvl_tiles[l] = tiles;
    }
}

int mdn_server::launch_tick(TickCtx& c) {
    NvtxRange nvtx_range("mdn_server tick");
    build_worklist(this, c.reqs, c.h_wl);
    cudaError_t e = cudaSuccess;
    const bool tr = !trace_path.empty();
    c.t_launch = now_ms();
    c.tick_id = st.ticks;
    c.pixels = 0;
    for (auto& r : c.reqs) c.pixels += (int64_t)r.h * r.w;
    if (tr) e = cudaEventRecord(c.ev_t0, c.s_up);
    // upload stream: the work list, then the inputs (overlapping other ticks' kernels)
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_wl, c.h_wl, sizeof(WorkList), cudaMemcpyHostToDevice, c.s_up);
    if (e == cudaSuccess && c.h_wl->n_up) {
        k_host_copy<<<COPY_BLOCKS, COPY_NT, 0, c.s_up>>>(c.d_wl, 0);
        e = cudaGetLastError();
    }
    for (auto& r : c.reqs) {   // copy-engine transfers: whole buffers, or the tails of the SM copies
        const size_t bytes = (size_t)3 * r.h * r.w * 2, done16 = r.dev_in ? bytes / 16 * 16 : 0;
        if (e == cudaSuccess && done16 < bytes)
            e = cudaMemcpyAsync((char*)r.z[0] + done16, (const char*)r.host_in + done16, bytes - done16,
                                cudaMemcpyHostToDevice, c.s_up);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_up, c.s_up);
    // compute stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s_comp, c.ev_up, 0);
    if (tr && e == cudaSuccess) e = cudaEventRecord(c.ev_cstart, c.s_comp);
    if (e == cudaSuccess) e = cudaGraphLaunch(c.gexec, c.s_comp);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_comp, c.s_comp);
    // download stream: outputs once this tick's kernels are done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.s_down, c.ev_comp, 0);
    if (tr && e == cudaSuccess) e = cudaEventRecord(c.ev_dstart, c.s_down);
    if (e == cudaSuccess && c.h_wl->n_down) {
        k_host_copy<<<COPY_BLOCKS, COPY_NT, 0, c.s_down>>>(c.d_wl, 1);
        e = cudaGetLastError();
    }
    for (auto& r : c.reqs) {
        const size_t bytes = (size_t)3 * r.h * r.w * 2, done16 = r.dev_out ? bytes / 16 * 16 : 0;
        if (e == cudaSuccess && done16 < bytes)
            e = cudaMemcpyAsync((char*)r.host_out + done16, (const char*)r.u[0] + done16, bytes - done16,
                                cudaMemcpyDeviceToHost, c.s_down);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_done, c.s_down);
    if (e != cudaSuccess) return cuda_fail(e, "server tick");
    return MDN_OK;
}

void mdn_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // retire finished ticks (their downloads completed)
        bool busy_any = false;
        for (auto& c : ctx) {
            if (c.busy) {
                const cudaError_t q = cudaEventQuery(c.ev_done);
                if (q == cudaErrorNotReady) {
                    busy_any = true;
                    continue;
                }
                if (q != cudaSuccess) {
                    thread_error = 1;
                    break;
                }
                const double t = now_ms();
                if (!trace_path.empty()) {
                    // host ms: launch, retire; device ms: upload, wait for compute, compute,
                    // wait for download, download; then the tick's request ids
                    float up = 0, qw = 0, cp = 0, dw = 0, dn = 0;
                    cudaEventElapsedTime(&up, c.ev_t0, c.ev_up);
                    cudaEventElapsedTime(&qw, c.ev_up, c.ev_cstart);
                    cudaEventElapsedTime(&cp, c.ev_cstart, c.ev_comp);
                    cudaEventElapsedTime(&dw, c.ev_comp, c.ev_dstart);
                    cudaEventElapsedTime(&dn, c.ev_dstart, c.ev_done);
                    char line[256];
                    snprintf(line, sizeof line, "%llu,%zu,%lld,%.3f,%.3f,%.3f,%.3f,%.3f,%.3f,%.3f,",
                             (unsigned long long)c.tick_id, c.reqs.size(), (long long)c.pixels, c.t_launch, t, up,
                             qw, cp, dw, dn);
                    std::string row(line);
                    for (size_t i = 0; i < c.reqs.size(); ++i) {
                        snprintf(line, sizeof line, "%s%llu", i ? ";" : "", (unsigned long long)c.reqs[i].id);
                        row += line;
                    }
                    trace_rows.push_back(row);
                }
                for (auto& r : c.reqs) {
                    arena.release(r.off, r.bytes);
                    done.push_back(mdn_result{r.id, MDN_OK, r.t_submit, r.t_admit, t});
                    st.completed++;
                }
                inflight -= (int)c.reqs.size();
                c.reqs.clear();
                c.busy = false;
                cv_done.notify_all();
            }
        }
        if (thread_error.load()) break;
        if (stop.load() && inflight == 0) break;
        // start a tick on a free context of each class with queued requests of that class
        bool launched = false;
        for (auto& c : ctx) {
            std::deque<Request>& q = queue[c.large ? 1 : 0];
            if (c.busy || q.empty() || stop.load()) continue;
            int64_t tick_pix = 0;
            while (!q.empty() && inflight < max_active && (int)c.reqs.size() < MAX_ITEMS) {
                Request& r = q.front();
                // a batch finishes as one: one large request per tick, small ones up to TICK_PIXELS
                if (!c.reqs.empty() && (c.large || tick_pix + (int64_t)r.h * r.w > TICK_PIXELS)) break;
                tick_pix += (int64_t)r.h * r.w;
                size_t off;
                if (!arena.alloc(r.bytes, &off)) break;
                r.off = off;
                char* p = arena.ptr(off);
                auto take = [&](size_t b) { char* q = p; p += align256(b); return (__half*)q; };
                r.z[0] = take((size_t)3 * r.h * r.w * 2);
                r.u[0] = take((size_t)3 * r.h * r.w * 2);
                for (int l = 1; l < r.levels; ++l) {
                    r.z[l] = take((size_t)3 * r.hl[l] * r.wl[l] * 2);
                    if (l <= r.levels - 2) r.u[l] = take((size_t)3 * r.hl[l] * r.wl[l] * 2);
                }
                r.t_admit = now_ms();
                c.reqs.push_back(r);
                q.pop_front();
                inflight++;
            }
            if (!c.reqs.empty()) {
                c.busy = true;
                st.ticks++;
                st.tick_items += c.reqs.size();
                if (c.large) st.ticks_large++;
                lk.unlock();
                const int rc = launch_tick(c);
                lk.lock();
                if (rc != MDN_OK) {
                    thread_error = 1;
                    break;
                }
                launched = true;
            }
        }
        if (thread_error.load()) break;
        if (launched) continue;   // look for more work at once
        // ticks in flight: poll their completion events every 20 us; idle:
        // sleep until a submission (or stop) arrives
        if (busy_any)
            cv.wait_for(lk, std::chrono::microseconds(20));
        else
            cv.wait_for(lk, std::chrono::milliseconds(100));
    }
    cv_done.notify_all();
}

static int autotune(mdn_server* s) {
    // one 1920x1080 request's filter level 0 with the first bank
    const int H = 1080, W = 1920;
    size_t need = 2 * align256((size_t)3 * H * W * 2) + align256((size_t)3 * 540 * 960 * 2);
    size_t off;
    if (!s->arena.alloc(need, &off)) return MDN_OK;   // arena too small to tune: keep the default
    TickCtx& c = s->ctx[0];
    __half* z = (__half*)s->arena.ptr(off);
    __half* uc = z + align256((size_t)3 * H * W * 2) / 2;
    __half* out = uc + align256((size_t)3 * 540 * 960 * 2) / 2;
    k_fill_pattern<<<(unsigned)((3 * H * W + 255) / 256), 256, 0, c.stream>>>(z, H, W);
    k_fill_pattern<<<(unsigned)((3 * 540 * 960 + 255) / 256), 256, 0, c.stream>>>(uc, 540, 960);
    int rc = MDN_OK;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int v = 0; v < NVAR && rc == MDN_OK; ++v) {
        if (v < 3 && !s->tile_ok) continue;   // tile kernels: 7x7 + 7x7 banks of at most 256 buckets
        s->variant = v;
        WorkList* wl = c.h_wl;
        std::memset(wl, 0, offsetof(WorkList, pyr));
        wl->lvl_n[0] = 1;
        LvlItem& it = wl->lvl[0];
        it = LvlItem{};
        it.z = z; it.coarse = uc; it.out = out; it.H = H; it.W = W; it.Hc = 540; it.Wc = 960; it.bank = 0;
        it.tiles_x = (W + 31) / 32;
        it.tile_start = 0;
        wl->lvl_tiles[0] = it.tiles_x * ((H + variant_rows(v) - 1) / variant_rows(v));
        cudaMemcpyAsync(c.d_wl, wl, sizeof(WorkList), cudaMemcpyHostToDevice, c.stream);
        rc = launch_variant(v, s->geom, c.d_wl, s->d_tb, s->Kmax, 0, c.stream);   // warm-up
        cudaEventRecord(a, c.stream);
        for (int rep = 0; rep < 3 && rc == MDN_OK; ++rep)
            rc = launch_variant(v, s->geom, c.d_wl, s->d_tb, s->Kmax, 0, c.stream);
        cudaEventRecord(b, c.stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        s->variant_ms[v] = ms / 3;
        if (ms < best) {
            best = ms;
            s->st.tile_variant = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    s->arena.release(off, need);
    s->variant = s->st.tile_variant;
    std::memset(c.h_wl, 0, sizeof(WorkList));
    cudaError_t e = cudaMemcpy(c.d_wl, c.h_wl, sizeof(WorkList), cudaMemcpyHostToDevice);
    if (rc == MDN_OK && e != cudaSuccess) rc = cuda_fail(e, "autotune: reset work list");
    return rc;
}

// Graph of one tick: pyramid stages 1 .. Lmax-1, then filter stages Lmax-2 .. 0.
static int capture_graph(mdn_server* s, TickCtx& c) {
    cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "server: begin capture");
    int rc = MDN_OK;
    for (int l = 1; l < s->max_levels; ++l) k_serve_pyr<<<compute_sms() * 4, pyr::PNT, 0, c.stream>>>(c.d_wl, l);
    for (int l = s->max_levels - 2; l >= 0 && rc == MDN_OK; --l)
        rc = launch_variant(s->variant, s->geom, c.d_wl, s->d_tb, s->Kmax, l, c.stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c.stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "server: end capture");
    c.graph = g;
    e = cudaGraphInstantiate(&c.gexec, g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "server: instantiate graph");
    return MDN_OK;
}

static void release_server(mdn_server* s) {
    for (auto& c : s->ctx) {
        if (c.ev_up) cudaEventDestroy(c.ev_up);
        if (c.ev_comp) cudaEventDestroy(c.ev_comp);
        if (c.ev_done) cudaEventDestroy(c.ev_done);
        for (cudaEvent_t ev : {c.ev_t0, c.ev_cstart, c.ev_dstart})
            if (ev) cudaEventDestroy(ev);
        if (c.gexec) cudaGraphExecDestroy(c.gexec);
        if (c.graph) cudaGraphDestroy(c.graph);
        if (c.d_wl) cudaFree(c.d_wl);
        if (c.h_wl) cudaFreeHost(c.h_wl);
        for (cudaStream_t st : {c.stream, c.s_up, c.s_comp, c.s_down})
            if (st) cudaStreamDestroy(st);
    }
    if (s->arena_mem) cudaFree(s->arena_mem);
    if (s->rows_mem) cudaFree(s->rows_mem);
    if (s->d_tb) cudaFree(s->d_tb);
    delete s;
}

extern "C" {

int mdn_server_create(const mdn_server_cfg* cfg, const mdn_bankset* sets, int32_t nsets, mdn_server** out) {
    if (!cfg || !sets || nsets < 1 || !out) return fail(MDN_EINVAL, "server_create: null argument");
    if (cfg->max_active < 1 || cfg->max_active > MAX_ITEMS) return fail(MDN_EINVAL, "server_create: max_active 1..256");
    if (cfg->hbm_budget_bytes < (size_t(1) << 20)) return fail(MDN_EBUDGET, "server_create: budget below 1 MiB");
    mdn_geometry geom = cfg->geom;
    if (geom.r_fine == 0) geom = mdn_geometry{3, 3, 0, MDN_YCBCR601};   // default: 7x7 + 7x7 per channel
    if (geom.r_fine != 3 || (geom.r_coarse != 3 && geom.r_coarse != 2) || geom.cross_channel != 0)
        return fail(MDN_ESHAPE, "server_create: geometry must be 7x7 + 7x7 or 7x7 + 5x5 per channel");
    mdn_server* s = new (std::nothrow) mdn_server();
    if (!s) return fail(MDN_ENOMEM, "server_create: host allocation");
    s->geom = geom;
    s->device = cfg->device;
    s->max_active = cfg->max_active;
    if (const char* tp = getenv("MDN_SERVER_TRACE")) s->trace_path = tp;
    if (const char* ce = getenv("MDN_SERVER_COPY_ENGINES")) s->copy_engines = ce[0] == '1';
    const unsigned evf = s->trace_path.empty() ? cudaEventDisableTiming : cudaEventDefault;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaSetDevice(cfg->device);
    int prio_low = 0, prio_high = 0;   // numerically: least >= greatest
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_mem, cfg->hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_tb, sizeof(Tables));
    for (int i = 0; i < NCTX && e == cudaSuccess; ++i) {
        TickCtx& c = s->ctx[i];
        c.large = i < NCTX_LARGE;
        e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.s_up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.s_down, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&c.s_comp, cudaStreamNonBlocking, c.large ? prio_low : prio_high);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_up, evf);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_comp, evf);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_done, evf);
        if (e == cudaSuccess && !s->trace_path.empty()) {
            e = cudaEventCreate(&c.ev_t0);
            if (e == cudaSuccess) e = cudaEventCreate(&c.ev_cstart);
            if (e == cudaSuccess) e = cudaEventCreate(&c.ev_dstart);
        }
        if (e == cudaSuccess) e = cudaMalloc(&c.d_wl, sizeof(WorkList));
        if (e == cudaSuccess) e = cudaMallocHost(&c.h_wl, sizeof(WorkList));
        if (e == cudaSuccess) {
            // the device work list starts empty: kernels launched with it do nothing
            std::memset(c.h_wl, 0, sizeof(WorkList));
            e = cudaMemcpy(c.d_wl, c.h_wl, sizeof(WorkList), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "server_create: device set-up");
        release_server(s);
        return rc;
    }
    s->arena.init(s->arena_mem, cfg->hbm_budget_bytes);
    Tables tb;
    int rc = build_tables(s, sets, nsets, &tb);
    int nbanks = 0;
    for (auto& st : s->sets) nbanks += st.levels - 1;
    // every bank once more as prepared row slots, which the fused kernel reads through L2
    size_t rows_total = 0;
    for (int b = 0; b < nbanks && rc == MDN_OK; ++b)
        rows_total += align256(mdn_bank_rows_bytes(&s->geom, tb.K[b], MDN_F16));
    if (rc == MDN_OK) {
        e = cudaMalloc(&s->rows_mem, rows_total);
        if (e != cudaSuccess) rc = cuda_fail(e, "server_create: prepared banks");
    }
    for (size_t b = 0, off = 0; (int)b < nbanks && rc == MDN_OK; ++b) {
        const size_t nbytes = mdn_bank_rows_bytes(&s->geom, tb.K[b], MDN_F16);
        rc = mdn_prepare_bank_rows(tb.bank[b], MDN_F16, &s->geom, tb.K[b], s->rows_mem + off, nbytes, nullptr);
        tb.rows[b] = s->rows_mem + off;
        off += align256(nbytes);
    }
    if (rc == MDN_OK) {
        e = cudaMemcpy(s->d_tb, &tb, sizeof(Tables), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "server_create: tables");
    }
    s->tile_ok = s->geom.r_coarse == RC && s->Kmax <= 256;
    int tv = cfg->tile_variant;
    if (tv < 0 || tv >= NVAR) {   // the autotune table's entry for this geometry and bank width, else the fused kernel
        tv = tune_server_lookup(s->geom, s->Kmax > 256);
        if (tv < 0) tv = 3;
    }
    s->st.tile_variant = s->tile_ok ? tv : 3;
    s->variant = s->st.tile_variant;
    if (rc == MDN_OK && cfg->autotune) {
        rc = autotune(s);
        if (rc == MDN_OK) tune_server_store(s->geom, s->Kmax > 256, s->variant, s->variant_ms[s->variant]);
    }
    for (int i = 0; i < NCTX && rc == MDN_OK; ++i) rc = capture_graph(s, s->ctx[i]);
    if (rc == MDN_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "server_create: set-up");
    }
    if (rc) {
        release_server(s);
        return rc;
    }
    s->thread = std::thread([s] { s->run(); });
    *out = s;
    return MDN_OK;
}

// The device address of a pinned (page-locked, mapped) host buffer if it is
// 16-byte aligned, else null: such buffers are copied by the SM copy kernel.
static const void* host_view(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error: the copy engines take this buffer
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || (uintptr_t)a.devicePointer % 16) return nullptr;
    return a.devicePointer;
}

int mdn_server_submit(mdn_server* s, const void* host_in, void* host_out, int64_t h, int64_t w, int32_t set,
                      uint64_t* id) {
    if (!s || !host_in || !host_out || !id) return fail(MDN_EINVAL, "server_submit: null argument");
    if (set < 0 || set >= (int)s->sets.size()) return fail(MDN_EINVAL, "server_submit: bad bank set");
    if (h < 1 || w < 1 || h > 16384 || w > 16384) return fail(MDN_ESHAPE, "server_submit: size out of range");
    if (s->thread_error.load()) return fail(MDN_ECUDA, "server_submit: the scheduler stopped on a CUDA error");
    Request r{};
    r.host_in = host_in;
    r.host_out = host_out;
    r.h = (int)h;
    r.w = (int)w;
    r.set = set;
    r.levels = s->sets[set].levels;
    r.hl[0] = r.h;
    r.wl[0] = r.w;
    for (int l = 1; l < r.levels; ++l) {
        r.hl[l] = (r.hl[l - 1] + 1) / 2;
        r.wl[l] = (r.wl[l - 1] + 1) / 2;
    }
    r.bytes = request_bytes(r.h, r.w, r.levels);
    if (!s->copy_engines) {
        r.dev_in = host_view(host_in);
        r.dev_out = const_cast<void*>(host_view(host_out));
    }
    if (r.bytes > s->arena.size()) return fail(MDN_EBUDGET, "server_submit: request exceeds the HBM budget");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop.load()) return fail(MDN_EINVAL, "server_submit: server is stopping");
        r.id = s->next_id++;
        r.t_submit = s->now_ms();
        s->queue[(int64_t)r.h * r.w >= LARGE_PIXELS ? 1 : 0].push_back(r);
        s->st.submitted++;
        *id = r.id;
    }
    s->cv.notify_all();
    return MDN_OK;
}

int mdn_server_cancel(mdn_server* s, uint64_t id) {
    if (!s) return fail(MDN_EINVAL, "server_cancel: null");
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& q : s->queue) {
        for (auto it = q.begin(); it != q.end(); ++it) {
            if (it->id == id) {
                s->done.push_back(mdn_result{id, MDN_ETIMEOUT, it->t_submit, -1.0, s->now_ms()});
                q.erase(it);
                s->st.cancelled++;
                s->cv_done.notify_all();
                return MDN_OK;
            }
        }
    }
    return fail(MDN_EINVAL, "server_cancel: request is not queued");
}

int mdn_server_poll(mdn_server* s, mdn_result* results, int32_t max, int32_t* n, int32_t timeout_ms) {
    if (!s || !results || !n || max < 1) return fail(MDN_EINVAL, "server_poll: bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                            [s] { return !s->done.empty() || s->thread_error.load(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        results[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    if (k == 0 && s->thread_error.load()) return fail(MDN_ECUDA, "server_poll: the scheduler stopped on a CUDA error");
    return MDN_OK;
}

int mdn_server_get_stats(mdn_server* s, mdn_server_stats* st) {
    if (!s || !st) return fail(MDN_EINVAL, "server_get_stats: null");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->active = s->inflight;
    st->queued = (int)(s->queue[0].size() + s->queue[1].size());
    st->arena_bytes = s->arena.size();
    st->arena_used = s->arena.used();
    st->arena_peak = s->arena.peak();
    for (int v = 0; v < NVAR; ++v) {
        st->variant_ms[v] = s->variant_ms[v];
        st->variant_threads[v] = variant_threads(v);
        st->variant_rows[v] = variant_rows(v);
    }
    return MDN_OK;
}

int mdn_server_destroy(mdn_server* s) {
    if (!s) return fail(MDN_EINVAL, "server_destroy: null");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue[0].clear();   // queued requests are dropped; admitted ticks finish
        s->queue[1].clear();
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->thread.joinable()) s->thread.join();
    cudaDeviceSynchronize();
    if (!s->trace_path.empty()) {
        if (FILE* f = fopen(s->trace_path.c_str(), "w")) {
            fprintf(f, "tick,requests,pixels,launch_ms,retire_ms,upload_ms,compute_wait_ms,compute_ms,"
                       "download_wait_ms,download_ms,ids\n");
            for (auto& l : s->trace_rows) fprintf(f, "%s\n", l.c_str());
            fclose(f);
        }
    }
    release_server(s);
    return MDN_OK;
}

}  // extern "C"
