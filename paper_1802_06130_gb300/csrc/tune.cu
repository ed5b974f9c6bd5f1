// tune.cu -- level-kernel autotuner: a process-wide table of the fastest
// level-kernel variant per (geometry, storage type, bank type and layout,
// bucket count, image-size class), filled by mdn_autotune_level (which times
// every applicable variant on synthetic frames of the requested size) and by
// the server's own tuning at create, persisted as a text file
// (mdn_autotune_save / mdn_autotune_load, or MDN_AUTOTUNE_TABLE=path, read
// on first use).  The level dispatch consults it before its static rule; the
// server reads its entry when created without tuning.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "internal.h"

namespace mdn {

thread_local int g_force_variant = -1;

namespace {

// (r_fine, r_coarse, cross, dtype, bank element type, prepared, K, size class)
using LevelKey = std::tuple<int, int, int, int, int, int, int, int>;
// (r_fine, r_coarse, wide banks)
using ServerKey = std::tuple<int, int, int>;
struct Entry {
    int variant;
    float ms;
};

std::mutex g_mu;
std::map<LevelKey, Entry> g_level;
std::map<ServerKey, Entry> g_server;
std::once_flag g_env_once;
std::atomic<int> g_entries{0};   // lets the dispatch skip the lock while the table is empty

int size_class(int64_t pixels) {
    int c = 0;
    while (c < 62 && (int64_t(1) << (c + 1)) <= pixels) ++c;
    return c;   // floor(log2(pixels)), 0 for a single pixel
}

LevelKey level_key(const mdn_geometry& g, int dtype, int bank_elem, bool rows, int K, int64_t pixels) {
    return LevelKey{g.r_fine, g.r_coarse, g.cross_channel != 0, dtype, bank_elem, rows ? 1 : 0, K,
                    size_class(pixels)};
}

int load_locked(const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return fail(MDN_EINVAL, "autotune_load: cannot open the table file");
    char line[256];
    int bad = 0;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int a[8], v;
        float ms;
        if (sscanf(line, "level %d %d %d %d %d %d %d %d %d %f", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6],
                   &a[7], &v, &ms) == 10 &&
            v >= 0 && v < LV_COUNT) {
            g_level[LevelKey{a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7]}] = Entry{v, ms};
        } else if (sscanf(line, "server %d %d %d %d %f", &a[0], &a[1], &a[2], &v, &ms) == 5 && v >= 0 && v < 4) {
            g_server[ServerKey{a[0], a[1], a[2]}] = Entry{v, ms};
        } else {
            ++bad;
        }
    }
    fclose(f);
    g_entries = (int)(g_level.size() + g_server.size());
    return bad ? fail(MDN_EINVAL, "autotune_load: malformed lines in the table file") : MDN_OK;
}

void env_load() {
    std::call_once(g_env_once, [] {
        if (const char* p = getenv("MDN_AUTOTUNE_TABLE")) {
            std::lock_guard<std::mutex> lk(g_mu);
            if (FILE* f = fopen(p, "r")) {
                fclose(f);
                load_locked(p);
            }
        }
    });
}

// synthetic frame: a smooth colour field with hashed noise, values in [0, 1]
template <typename T> __global__ void k_tune_fill(T* p, int64_t n, int64_t plane, int w, float amp) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % plane;
        const int c = (int)((i / plane) % 3);
        const int y = (int)(r / w), x = (int)(r % w);
        uint32_t hsh = (uint32_t)i * 2654435761u;
        hsh ^= hsh >> 13;
        hsh *= 0x5bd1e995u;
        hsh ^= hsh >> 15;
        const float noise = ((hsh & 0xffff) / 65535.f - 0.5f) * amp;
        const float v = fminf(fmaxf(0.5f + 0.3f * __sinf(0.031f * x + 0.047f * y + c) + noise, 0.f), 1.f);
        if constexpr (sizeof(T) == 2) p[i] = __float2half_rn(v); else p[i] = v;
    }
}
// synthetic bank: taps near 1/D with hashed variation
template <typename T> __global__ void k_tune_bank(T* b, int64_t n, int D) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t hsh = (uint32_t)i * 2246822519u;
        hsh ^= hsh >> 16;
        const float v = (1.f + ((hsh & 0xffff) / 65535.f - 0.5f)) / D;
        if constexpr (sizeof(T) == 2) b[i] = __float2half_rn(v); else b[i] = v;
    }
}

template <typename T> void fill(void* p, int64_t n, int64_t plane, int w, float amp, cudaStream_t s) {
    k_tune_fill<T><<<1024, 256, 0, s>>>((T*)p, n, plane, w, amp);
}

}  // namespace

int tune_lookup(const LevelArgs& a) {
    env_load();
    if (g_entries.load(std::memory_order_relaxed) == 0) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    const LevelKey k = level_key(a.geom, a.dtype, a.bank_dtype, a.bank_rows, a.K, a.n * a.h * a.w);
    auto it = g_level.find(k);
    if (it != g_level.end()) return it->second.variant;
    // nearest size class of the same configuration
    int best = -1, dist = 1 << 30;
    for (auto& e : g_level) {
        const LevelKey& q = e.first;
        if (std::get<0>(q) != std::get<0>(k) || std::get<1>(q) != std::get<1>(k) || std::get<2>(q) != std::get<2>(k) ||
            std::get<3>(q) != std::get<3>(k) || std::get<4>(q) != std::get<4>(k) || std::get<5>(q) != std::get<5>(k) ||
            std::get<6>(q) != std::get<6>(k))
            continue;
        const int d = std::abs(std::get<7>(q) - std::get<7>(k));
        if (d < dist) { dist = d; best = e.second.variant; }
    }
    return best;
}

int tune_server_lookup(const mdn_geometry& g, bool wide) {
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_server.find(ServerKey{g.r_fine, g.r_coarse, wide ? 1 : 0});
    return it == g_server.end() ? -1 : it->second.variant;
}

void tune_server_store(const mdn_geometry& g, bool wide, int variant, float ms) {
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    g_server[ServerKey{g.r_fine, g.r_coarse, wide ? 1 : 0}] = Entry{variant, ms};
    g_entries = (int)(g_level.size() + g_server.size());
}

}  // namespace mdn

using namespace mdn;

extern "C" {

int mdn_autotune_level(const mdn_geometry* geom, const mdn_bucket_params* bp, int32_t dtype, int32_t bank_dtype,
                       int64_t n, int64_t h, int64_t w, int32_t reps, int32_t* best, float* ms, void* stream) {
    NvtxRange nvtx_range("mdn_autotune_level");
    if (!geom || !bp || !best || !ms) return fail(MDN_EINVAL, "autotune_level: null argument");
    if (dtype != MDN_F32 && dtype != MDN_F16) return fail(MDN_EINVAL, "autotune_level: bad dtype");
    if (reps < 1 || reps > 100) return fail(MDN_EINVAL, "autotune_level: reps must be 1..100");
    if (!dims_ok(n, h, w) || n < 1 || h < 1 || w < 1 || n * h * w > (int64_t(1) << 28))
        return fail(MDN_ESHAPE, "autotune_level: sizes must be positive and at most 2^28 pixels");
    const bool rows = bank_dtype == MDN_F16_ROWS || bank_dtype == MDN_F32_ROWS;
    const int elem = (bank_dtype == MDN_F16 || bank_dtype == MDN_F16_ROWS) ? MDN_F16 : MDN_F32;
    if (bank_dtype < MDN_F32 || bank_dtype > MDN_F32_ROWS) return fail(MDN_EINVAL, "autotune_level: bad bank dtype");
    const int D = mdn_regressor_len(geom);
    const int K = bp->n_angle * bp->n_strength * bp->n_coherence;
    if (D <= 0 || mdn_bank_rows_bytes(geom, K < 1 ? 1 : K, MDN_F16) == 0)
        return fail(MDN_ESHAPE, "autotune_level: geometry not compiled");
    SelParams sp;
    if (int rc = make_sel_params(bp, &sp)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dtype == MDN_F16 ? 2 : 4, bes = elem == MDN_F16 ? 2 : 4;
    const int64_t hc = (h + 1) / 2, wc = (w + 1) / 2;
    const size_t zb = (size_t)n * 3 * h * w * es, cb = (size_t)n * 3 * hc * wc * es;
    const size_t bankb = (size_t)K * 3 * D * bes, rowsb = rows ? mdn_bank_rows_bytes(geom, K, elem) : 0;
    void *z = nullptr, *c = nullptr, *out = nullptr, *bank = nullptr, *rb = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&] {
        for (void* p : {z, c, out, bank, rb})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        g_force_variant = -1;
    };
    cudaError_t e = cudaMalloc(&z, zb);
    if (e == cudaSuccess && geom->r_coarse >= 0) e = cudaMalloc(&c, cb);
    if (e == cudaSuccess) e = cudaMalloc(&out, zb);
    if (e == cudaSuccess) e = cudaMalloc(&bank, bankb);
    if (e == cudaSuccess && rows) e = cudaMalloc(&rb, rowsb);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "autotune_level: scratch");
    }
    if (dtype == MDN_F16) {
        fill<__half>(z, (int64_t)n * 3 * h * w, h * w, (int)w, 0.2f, s);
        if (c) fill<__half>(c, (int64_t)n * 3 * hc * wc, hc * wc, (int)wc, 0.05f, s);
    } else {
        fill<float>(z, (int64_t)n * 3 * h * w, h * w, (int)w, 0.2f, s);
        if (c) fill<float>(c, (int64_t)n * 3 * hc * wc, hc * wc, (int)wc, 0.05f, s);
    }
    if (elem == MDN_F16) k_tune_bank<__half><<<256, 256, 0, s>>>((__half*)bank, (int64_t)K * 3 * D, D);
    else k_tune_bank<float><<<256, 256, 0, s>>>((float*)bank, (int64_t)K * 3 * D, D);
    int rc = check_launch("autotune_level: synthetic inputs");
    if (rc == MDN_OK && rows) rc = mdn_prepare_bank_rows(bank, elem, geom, K, rb, rowsb, stream);
    const void* use_bank = rows ? rb : bank;
    float best_ms = INFINITY;
    *best = -1;
    for (int v = 0; v < LV_COUNT && rc == MDN_OK; ++v) {
        ms[v] = -1.f;
        g_force_variant = v;
        int r = mdn_filter_level(z, c, dtype, n, h, w, use_bank, bank_dtype, geom, bp, out, nullptr, stream);
        if (r == MDN_ESHAPE) continue;   // this variant does not apply
        if (r != MDN_OK) { rc = r; break; }
        e = cudaEventRecord(e0, s);
        for (int i = 0; i < reps && rc == MDN_OK && e == cudaSuccess; ++i)
            rc = mdn_filter_level(z, c, dtype, n, h, w, use_bank, bank_dtype, geom, bp, out, nullptr, stream);
        if (rc == MDN_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (rc == MDN_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (rc == MDN_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (rc == MDN_OK && e != cudaSuccess) rc = cuda_fail(e, "autotune_level: timing");
        if (rc != MDN_OK) break;
        ms[v] = t / reps;
        if (ms[v] < best_ms) { best_ms = ms[v]; *best = v; }
    }
    cleanup();
    if (rc != MDN_OK) return rc;
    if (*best < 0) return fail(MDN_ESHAPE, "autotune_level: no level-kernel variant applies");
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    g_level[level_key(*geom, dtype, elem, rows, K, n * h * w)] = Entry{*best, best_ms};
    g_entries = (int)(g_level.size() + g_server.size());
    return MDN_OK;
}

int mdn_autotune_lookup(const mdn_geometry* geom, int32_t K, int32_t dtype, int32_t bank_dtype, int64_t n,
                        int64_t h, int64_t w) {
    if (!geom) return -1;
    LevelArgs a{};
    a.geom = *geom;
    a.K = K;
    a.dtype = dtype;
    a.bank_rows = bank_dtype == MDN_F16_ROWS || bank_dtype == MDN_F32_ROWS;
    a.bank_dtype = (bank_dtype == MDN_F16 || bank_dtype == MDN_F16_ROWS) ? MDN_F16 : MDN_F32;
    a.n = n;
    a.h = h;
    a.w = w;
    return tune_lookup(a);
}

int mdn_autotune_server_lookup(const mdn_geometry* geom, int32_t wide) {
    return geom ? tune_server_lookup(*geom, wide != 0) : -1;
}

int mdn_autotune_save(const char* path) {
    if (!path) return fail(MDN_EINVAL, "autotune_save: null path");
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    FILE* f = fopen(path, "w");
    if (!f) return fail(MDN_EINVAL, "autotune_save: cannot open the table file");
    fprintf(f, "# level r_fine r_coarse cross dtype bank_elem prepared K size_class variant ms\n"
               "# server r_fine r_coarse wide variant ms\n");
    for (auto& e : g_level) {
        const LevelKey& k = e.first;
        fprintf(f, "level %d %d %d %d %d %d %d %d %d %.5f\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), e.second.variant,
                e.second.ms);
    }
    for (auto& e : g_server)
        fprintf(f, "server %d %d %d %d %.5f\n", std::get<0>(e.first), std::get<1>(e.first), std::get<2>(e.first),
                e.second.variant, e.second.ms);
    const bool ok = fclose(f) == 0;
    return ok ? MDN_OK : fail(MDN_EINVAL, "autotune_save: write failed");
}

int mdn_autotune_load(const char* path) {
    if (!path) return fail(MDN_EINVAL, "autotune_load: null path");
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    return load_locked(path);
}

void mdn_autotune_clear(void) {
    env_load();
    std::lock_guard<std::mutex> lk(g_mu);
    g_level.clear();
    g_server.clear();
    g_entries = 0;
}

}  // extern "C"
