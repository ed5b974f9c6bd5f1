/*
 * mdn.h -- C ABI of libmdn: GB300 (sm_103a) trainable multiscale denoising
 * after Choi, Isidoro, Getreuer, Milanfar, "Fast, Trainable, Multiscale
 * Denoising" (arXiv 1802.06130).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are planar RGB, row-major: [n][3][h][w], values nominally in
 *   [0, 1], stored as FP32 (MDN_F32) or FP16 (MDN_F16).  Level l of a pyramid
 *   has size ceil(h / 2^l) x ceil(w / 2^l).  Sizes are limited to h, w <=
 *   2^20 and n * 3 * h * w < 2^31 elements (checked without overflow): larger
 *   images are rejected with MDN_ESHAPE, and the *_bytes size queries return
 *   SIZE_MAX for them.
 * - Every data pointer is a DEVICE pointer unless stated otherwise; the caller
 *   owns every buffer (images, banks, maps, Gram state, workspace).  The
 *   library never allocates or frees on these paths; the only state it keeps
 *   is per-device kernel configuration made on first use.  Pointers to the
 *   parameter structs are HOST pointers, read during the call only.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on that stream: the return status covers argument
 *   checks and launch errors only; device results are valid after the stream
 *   is synchronised.
 * - Status: MDN_OK (0) or one of the MDN_E* codes below; on error the message
 *   is kept per thread and returned by mdn_last_error().  No entry point
 *   aborts the process.
 * - Filter banks are [K][3][D] (bucket, output channel, regressor tap), FP32
 *   or FP16.  The regressor of output channel c at pixel i (Section 4, the
 *   multiscale filtering equation with h = [f; g]) is the coarse patch
 *   R_{floor(i/2)} u^{l+1} followed by the fine patch R_i z^l, each in
 *   (channel, dy, dx) row-major order, dy, dx in [-r, r]; per-channel
 *   geometry uses working channel c only, cross-channel geometry all three.
 *   Borders clamp to the edge.  Filtering runs in zero-offset BT.601 YCbCr
 *   (Section 3, footnote 1) unless color = MDN_RGB.
 */
#ifndef MDN_H
#define MDN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MDN_OK 0
#define MDN_EINVAL 1      /* null pointer, bad enum or parameter */
#define MDN_ESHAPE 2      /* inconsistent sizes or unsupported geometry */
#define MDN_EWORKSPACE 3  /* workspace too small (see the *_bytes queries) */
#define MDN_EBUDGET 4     /* serving: request exceeds the memory budget */
#define MDN_ETIMEOUT 5    /* a bounded wait expired */
#define MDN_ECUDA 6       /* CUDA error; message in mdn_last_error() */
#define MDN_ENOMEM 7      /* host allocation failed (serving set-up only) */

/* ---- element types ---- */
#define MDN_F32 0
#define MDN_F16 1
/* bank types only: a bank prepared by mdn_prepare_bank_rows (row slots) */
#define MDN_F16_ROWS 2
#define MDN_F32_ROWS 3

/* ---- colour spaces ---- */
#define MDN_YCBCR601 0
#define MDN_RGB 1

/* ---- Gram precisions for training ---- */
#define MDN_GRAM_FP32 0        /* CUDA-core FP32 products, FP64 reduction */
#define MDN_GRAM_TF32 1        /* tcgen05 kind::tf32, FP32 accumulate in TMEM */
#define MDN_GRAM_BF16 2        /* tcgen05 kind::f16 with BF16 operands */
#define MDN_GRAM_SPLIT_BF16 3  /* hi*hi + hi*lo + lo*hi BF16 products */

#define MDN_MAX_THR 16
#define MDN_MAX_K 4096

/* Filter footprint.  r_fine: radius of the fine patch R_i z^l (1..3);
 * r_coarse: radius of the coarse patch R_{i/2} u^{l+1} (0..3) or -1 for
 * single-scale filtering (Eq. 1); cross_channel: 0 = per-channel regressors
 * (D = P_c + P_f), 1 = all three channels (D = 3 (P_c + P_f)); color:
 * MDN_YCBCR601 or MDN_RGB. */
typedef struct {
    int32_t r_fine;
    int32_t r_coarse;
    int32_t cross_channel;
    int32_t color;
} mdn_geometry;

/* Filter selector s(i) (Section 3, "Filter selection").  Orientation (angle
 * of the minor eigenvector of the smoothed colour structure tensor, in
 * [0, pi)) is split into n_angle equal bins (n_angle even, <= 64); strength
 * sqrt(lambda1) and coherence (sqrt l1 - sqrt l2)/(sqrt l1 + sqrt l2) are
 * binned by the n_strength-1 and n_coherence-1 ascending thresholds
 * (lower-inclusive).  Coherence is 0 where sqrt l1 + sqrt l2 < coh_eps.
 * Bucket k = (a * n_strength + s) * n_coherence + c, K = product <= 4096
 * (n_strength, n_coherence <= MDN_MAX_THR + 1), e.g. the paper's own
 * 16 x 16 x 16 grid (Section 5).  Bucket maps hold one u8 per pixel when
 * K <= 256 and one u16 (native byte order) when K > 256. */
typedef struct {
    int32_t n_angle;
    int32_t n_strength;
    int32_t n_coherence;
    float strength_thr[MDN_MAX_THR];
    float coherence_thr[MDN_MAX_THR];
    float coh_eps;
} mdn_bucket_params;

/* Library version (major * 10000 + minor * 100 + patch). */
int mdn_version(void);

/* Message of the last failed call on this thread ("" if none).  The string
 * stays valid until the next call on the same thread. */
const char* mdn_last_error(void);

/* Regressor length D per output channel for a geometry, or -1 if invalid. */
int mdn_regressor_len(const mdn_geometry* geom);

/* Bytes per pixel of a bucket map for K buckets: 1 (u8) for K <= 256, 2 (u16)
 * for 256 < K <= MDN_MAX_K, 0 for K outside 1..MDN_MAX_K. */
int mdn_bucket_elem_bytes(int32_t K);

/* ------------------------------------------------------------------ */
/* Pyramid (Section 4, "Multiscale filtering": downsampling by two)    */
/* ------------------------------------------------------------------ */

/* Bytes of levels 1 .. levels-1 of an [n][3][h][w] image of element type
 * dtype (each level padded to 256 bytes). */
size_t mdn_pyramid_bytes(int64_t n, int64_t h, int64_t w, int32_t levels, int32_t dtype);

/* Builds levels 1 .. levels-1 of `img` by repeated 2x downsampling with the
 * separable 5-tap binomial kernel [1 4 6 4 1]/16 (clamped borders), computed
 * in FP32 (horizontal pass, then vertical) and rounded to `dtype`
 * (round-to-nearest-even for FP16).  out_levels: HOST array of levels-1
 * device pointers, out_levels[l-1] -> [n][3][h_l][w_l].  levels in 1..8. */
int mdn_build_pyramid(const void* img, int32_t dtype, int64_t n, int64_t h, int64_t w,
                      int32_t levels, void* const* out_levels, void* stream);

/* ------------------------------------------------------------------ */
/* Filter selection only (Section 3)                                   */
/* ------------------------------------------------------------------ */

/* Writes the bucket map s(i) ([n][h][w], u8 or u16 by K, see
 * mdn_bucket_elem_bytes) of image z ([n][3][h][w]). */
int mdn_select_buckets(const void* z, int32_t dtype, int64_t n, int64_t h, int64_t w,
                       const mdn_bucket_params* bp, void* buckets, void* stream);

/* ------------------------------------------------------------------ */
/* One level of filtering (Eq. 1; Section 4 multiscale equation)       */
/* ------------------------------------------------------------------ */

/* Fused selector + filter for one level: out = h^{s(i)} . [R_{i/2} coarse ;
 * R_i z] per output channel, converted back to RGB and rounded to dtype.
 * z, out: [n][3][h][w]; coarse: [n][3][ceil(h/2)][ceil(w/2)] or NULL when
 * geom->r_coarse < 0; bank: [K][3][D] of bank_dtype, K = bucket count of bp;
 * buckets_out: optional [n][h][w] copy of s(i) (u8 or u16 by K).  out must
 * not alias z or coarse.  Banks of up to ~145 KB in row-slot form (e.g. 216
 * buckets of 7x7 + 7x7 taps in FP16) are held in shared memory by the fused
 * kernel; larger plain banks (the paper's 4096-bucket grid, FP32 banks of
 * 7x7 + 7x7 taps) run a slower kernel that reads taps through L2, and larger
 * prepared banks (mdn_prepare_bank_rows) run the fused kernel reading row
 * slots through L2.  The kernel used can be tuned per configuration
 * (mdn_autotune_level). */
int mdn_filter_level(const void* z, const void* coarse, int32_t dtype, int64_t n, int64_t h,
                     int64_t w, const void* bank, int32_t bank_dtype, const mdn_geometry* geom,
                     const mdn_bucket_params* bp, void* out, void* buckets_out, void* stream);

/* Prepared banks.  mdn_prepare_bank_rows writes a bank [K][3][D] (bank_dtype
 * MDN_F32 or MDN_F16, device) into `rows` (device, 16-byte aligned, at least
 * mdn_bank_rows_bytes bytes) in the layout the fused level kernel reads: per
 * bucket, output channel, block (coarse patch of each input channel, then
 * fine patch of each) and filter row dy, one slot of 8 elements holding the
 * 2r+1 taps dx = -r..r of that row, zero padded.  Pass `rows` as the bank
 * with bank_dtype MDN_F16_ROWS / MDN_F32_ROWS to mdn_filter_level and the
 * mdn_denoise_multiscale family: a bank that fits in shared memory is copied
 * there whole; a larger one (the paper's 4096-bucket grid, FP32 banks of 216
 * buckets of 7x7 + 7x7 taps) is read from this layout through L2 with 16-byte
 * loads instead of tap by tap.  Results equal those of the plain bank where
 * both run the same kernel; geometries: 5x5, 7x7 + 7x7, 7x7 + 5x5, 5x5 + 3x3
 * per channel and 7x7x3 cross-channel.  mdn_bank_rows_bytes returns 0 for
 * another geometry or bad arguments.  The layout carries no header: a
 * prepared bank must be passed with the geometry and bucket count it was
 * prepared for (the caller's contract, like the size of any buffer; the
 * Python binding checks it).  Asynchronous on stream. */
size_t mdn_bank_rows_bytes(const mdn_geometry* geom, int32_t K, int32_t bank_dtype);
int mdn_prepare_bank_rows(const void* bank, int32_t bank_dtype, const mdn_geometry* geom, int32_t K, void* rows,
                          size_t rows_bytes, void* stream);

/* Level-kernel autotuner.  The paper fixes what a level computes, not how;
 * the library holds several kernels for it (variants, MDN_LV_*), and which
 * is fastest depends on the geometry, the storage and bank types, the bucket
 * count and the image size.  mdn_autotune_level times every variant that
 * applies to such a call on synthetic frames of that size (reps timed calls
 * each, after one warm-up; it allocates and frees its own device scratch,
 * so call it at set-up, not inside stream capture), writes the mean ms per
 * call of each variant to ms[MDN_LEVEL_VARIANTS] (-1 where one does not
 * apply) and the fastest to *best, and records it in a process-wide table.
 * mdn_filter_level and the mdn_denoise_multiscale family then use the
 * table's variant for calls with the same configuration (the entry of the
 * nearest image-size class when the size differs), and their static rule
 * otherwise.  Results differ between variants only by FP32 summation order.
 * mdn_autotune_save / _load write and merge the table as text (lines
 * "level r_fine r_coarse cross dtype bank_elem prepared K size_class variant
 * ms" and "server r_fine r_coarse wide variant ms"); the environment
 * variable MDN_AUTOTUNE_TABLE names a file loaded on first use.  The server
 * (mdn_server_create) stores its own tuning there and, created without
 * tuning and with tile_variant -1, uses the table's entry for its geometry
 * and bank width.  mdn_autotune_lookup / _server_lookup return the recorded
 * variant (-1: none); mdn_autotune_clear empties the table.  Thread-safe. */
#define MDN_LV_FUSED_SMEM 0     /* warp-specialised fused kernel, bank in shared memory */
#define MDN_LV_FUSED_L2 1       /* fused kernel, prepared bank read through L2 */
#define MDN_LV_STRIP 2          /* strip kernel, bank in shared memory */
#define MDN_LV_TILE_SMEM 3      /* one pixel per thread, bank in shared memory */
#define MDN_LV_TILE_L2 4        /* one pixel per thread, taps read through L2 */
#define MDN_LV_FUSED_CLUSTER 5  /* fused kernel on clusters of two CTAs, FP32 bank split between them */
#define MDN_LEVEL_VARIANTS 6
int mdn_autotune_level(const mdn_geometry* geom, const mdn_bucket_params* bp, int32_t dtype, int32_t bank_dtype,
                       int64_t n, int64_t h, int64_t w, int32_t reps, int32_t* best, float* ms, void* stream);
int mdn_autotune_lookup(const mdn_geometry* geom, int32_t K, int32_t dtype, int32_t bank_dtype, int64_t n,
                        int64_t h, int64_t w);
int mdn_autotune_server_lookup(const mdn_geometry* geom, int32_t wide);
int mdn_autotune_save(const char* path);
int mdn_autotune_load(const char* path);
void mdn_autotune_clear(void);

/* ------------------------------------------------------------------ */
/* Multiscale denoising (Section 4)                                    */
/* ------------------------------------------------------------------ */

/* Workspace bytes for mdn_denoise_multiscale: pyramid levels 1..L-1 plus
 * intermediate outputs u^1 .. u^{L-2}. */
size_t mdn_denoise_workspace_bytes(int64_t n, int64_t h, int64_t w, int32_t levels, int32_t dtype);

/* Multiscale inference: z^0 = noisy, z^{l+1} = downsample(z^l), base case
 * u^{L-1} = z^{L-1}, then for l = L-2 .. 0 u^l = filter_level(z^l, u^{l+1},
 * banks[l]); out = u^0.  levels = 1 is single-scale filtering (Eq. 1) with
 * banks[0] and geom->r_coarse = -1.  banks: HOST array of max(levels-1, 1)
 * device pointers; bparams: HOST array of the same length (level l uses
 * bparams[l]); bucket_maps: NULL or a HOST array of the same length of device
 * [n][h_l][w_l] pointers, u8 or u16 by the level's K (entries may be NULL).  ws: device workspace of
 * at least mdn_denoise_workspace_bytes(). */
int mdn_denoise_multiscale(const void* noisy, int32_t dtype, int64_t n, int64_t h, int64_t w,
                           int32_t levels, const void* const* banks, int32_t bank_dtype,
                           const mdn_geometry* geom, const mdn_bucket_params* bparams,
                           void* out, void* const* bucket_maps, void* ws, size_t ws_bytes,
                           void* stream);

/* mdn_denoise_multiscale for a batch held in HOST memory, with copies and
 * kernels overlapped (a deployment layer: the paper describes per-image
 * inference only).  The batch is cut into chunks of `chunk` images; chunk c
 * is copied host_noisy -> dev_in on the upload stream, denoised dev_in ->
 * dev_out on a compute stream with the same kernels and results as
 * mdn_denoise_multiscale, and copied dev_out -> host_out on the download
 * stream; each stage of a chunk waits for the previous stage of that chunk
 * only, so consecutive chunks' uploads, kernels and downloads overlap.
 * streams: HOST array of nstreams distinct cudaStream_t, either 3 (upload,
 * compute, download) or 4 (upload, compute A, compute B, download: chunks
 * alternate between the two compute streams, so one chunk's kernel start-up
 * and tail overlap the other's work).
 * host_noisy, host_out: HOST [n][3][h][w] buffers of dtype (page-locked
 * memory is needed for the copies to overlap); dev_in, dev_out: device
 * [n][3][h][w] buffers; ws: device workspace of at least one chunk's
 * mdn_denoise_workspace_bytes(min(chunk, n), h, w, levels, dtype) per compute
 * stream (with two, each slice rounded up to 256 bytes; chunks on one compute
 * stream share its slice).  The uploads, downloads and the second compute
 * stream start after the work already queued on streams[1]; the call is
 * asynchronous and host_out is complete once streams[1] is synchronised.
 * Allocates no device memory (it creates and releases five CUDA events per
 * call).  Bucket maps are not written.  MDN_EINVAL / MDN_ESHAPE /
 * MDN_EWORKSPACE as for mdn_denoise_multiscale, and MDN_EINVAL for chunk < 1,
 * nstreams other than 3 or 4, or equal streams. */
int mdn_denoise_multiscale_pipelined(const void* host_noisy, int32_t dtype, int64_t n, int64_t h, int64_t w,
                                     int32_t levels, const void* const* banks, int32_t bank_dtype,
                                     const mdn_geometry* geom, const mdn_bucket_params* bparams, void* host_out,
                                     int64_t chunk, void* dev_in, void* dev_out, void* ws, size_t ws_bytes,
                                     void* const* streams, int32_t nstreams);

/* Same as mdn_denoise_multiscale, for callers that cannot allocate device
 * memory: a plug-in inside a host application that owns every device
 * allocation, or a real-time pipeline where an allocation (which may
 * synchronise the device) is not allowed on the frame path.  The paper has
 * no counterpart; this is a deployment convenience.  The caller still owns
 * noisy, out, banks and bucket maps; the scratch (pyramid levels and
 * intermediate outputs) comes from one static device array of
 * MDN_STATIC_SCRATCH_BYTES (48 MiB) that every device loading the library
 * holds until the process exits.  No cudaMalloc/cudaFree or other allocating
 * call is made.  Images whose mdn_denoise_workspace_bytes() exceeds the array
 * are rejected with MDN_EWORKSPACE (e.g. one 12 MP FP16 frame at 3 levels
 * fits, eight do not).  The first call on a device, with that device
 * current, looks up the array's address and caches it per device ordinal:
 * make that first call before any stream capture, and do not call this entry
 * point again on a device after cudaDeviceReset (the cached address belongs
 * to the context that the reset ended).  All calls on a device share the array and it
 * keeps the previous call's contents (nothing needs clearing: each call
 * writes every scratch element before reading it), so calls whose GPU work
 * overlaps (different streams or host threads) race: serialise them. */
#define MDN_STATIC_SCRATCH_BYTES ((size_t)48 << 20)
int mdn_denoise_multiscale_static(const void* noisy, int32_t dtype, int64_t n, int64_t h, int64_t w,
                                  int32_t levels, const void* const* banks, int32_t bank_dtype,
                                  const mdn_geometry* geom, const mdn_bucket_params* bparams,
                                  void* out, void* const* bucket_maps, void* stream);

/* Tensor-descriptor forms.  The entry points above take plain pointers and
 * sizes; these take every array as an mdn_tensor and check it against the
 * shapes the operation implies before calling the pointer form, returning
 * MDN_ESHAPE (the argument named in mdn_last_error) for a wrong dtype, rank,
 * extent or stride, MDN_EINVAL for a null tensor or data pointer.  Strides
 * are in elements and must be the dense row-major ones (extents of 1 may
 * have any stride): the kernels read dense buffers, so a strided view must
 * be made contiguous by the caller.  Images are [N][3][H][W] MDN_F32 or
 * MDN_F16 (all of one call alike); coarse inputs [N][3][(H+1)/2][(W+1)/2];
 * banks [K][3][D] MDN_F32 / MDN_F16 (D = mdn_regressor_len, K from the
 * bucket parameters) or, prepared, a 1-D tensor of mdn_bank_rows_bytes
 * elements of dtype MDN_F16_ROWS / MDN_F32_ROWS; bucket maps [N][H][W]
 * MDN_U8 (K <= 256) or MDN_U16; the Gram state [K][G][Dp][Dp] MDN_F64 and
 * counts [K] MDN_I64 (see mdn_gram_state_bytes); bank_out [K][3][D] MDN_F32.
 * Arrays of tensors (pyramid levels, banks, bucket maps) are HOST arrays;
 * a bucket-map entry with null data is skipped.  Ownership, streams and
 * asynchrony as for the pointer forms. */
#define MDN_U8 8       /* tensor dtypes beyond MDN_F32 / MDN_F16 / the row-slot banks */
#define MDN_U16 9
#define MDN_F64 10
#define MDN_I64 11
typedef struct {
    int32_t dtype;
    int32_t ndim;          /* 1..4 */
    int64_t shape[4];
    int64_t strides[4];    /* elements */
    void* data;            /* device */
} mdn_tensor;
int mdn_t_build_pyramid(const mdn_tensor* img, int32_t levels, mdn_tensor* out, void* stream);
int mdn_t_filter_level(const mdn_tensor* z, const mdn_tensor* coarse, const mdn_tensor* bank,
                       const mdn_geometry* geom, const mdn_bucket_params* bp, mdn_tensor* out,
                       mdn_tensor* buckets_out, void* stream);
int mdn_t_denoise_multiscale(const mdn_tensor* noisy, int32_t levels, const mdn_tensor* banks,
                             const mdn_geometry* geom, const mdn_bucket_params* bparams, mdn_tensor* out,
                             mdn_tensor* bucket_maps, void* ws, size_t ws_bytes, void* stream);
int mdn_t_train_level_filters(const mdn_tensor* noisy_lvl, const mdn_tensor* coarse_out,
                              const mdn_tensor* clean_lvl, const mdn_geometry* geom, const mdn_bucket_params* bp,
                              int32_t gram_precision, int32_t accumulate, mdn_tensor* gram, mdn_tensor* counts,
                              double lambda, mdn_tensor* bank_out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Training (Eqs. 5-6: per-bucket least squares; Section 4 cascade)    */
/* ------------------------------------------------------------------ */

/* Gram state layout: gram[K][G][Dp][Dp] FP64 with G = 3, Dp = D + 1 for
 * per-channel geometry and G = 1, Dp = D + 3 for cross-channel geometry
 * (regressor taps first, then the target(s) in working colour space);
 * counts[K] int64 = pixels per bucket. */
size_t mdn_gram_state_bytes(const mdn_geometry* geom, int32_t K);

/* Workspace bytes for mdn_train_level_filters on n images of h x w. */
size_t mdn_train_workspace_bytes(int64_t n, int64_t h, int64_t w, const mdn_geometry* geom,
                                 int32_t K, int32_t gram_precision);

/* One level of training data: computes s(i) on noisy_lvl, sorts pixels by
 * bucket, and adds to gram/counts (cleared first unless `accumulate`) the
 * Gram matrix of [regressor ; target] over every pixel of each bucket, the
 * regressor as in mdn_filter_level with coarse = coarse_out (the trained
 * coarser level's output, NULL if geom->r_coarse < 0) and the target =
 * clean_lvl in working colour space.  gram_precision selects the product
 * arithmetic (MDN_GRAM_*); partial sums are reduced in FP64.  If bank_out
 * is not NULL, then solves the bank as mdn_solve_bank does. */
int mdn_train_level_filters(const void* noisy_lvl, const void* coarse_out, const void* clean_lvl,
                            int32_t dtype, int64_t n, int64_t h, int64_t w,
                            const mdn_geometry* geom, const mdn_bucket_params* bp,
                            int32_t gram_precision, int32_t accumulate, double* gram,
                            int64_t* counts, double lambda, float* bank_out, void* ws,
                            size_t ws_bytes, void* stream);

/* Bounds-checked debug build (the library built with -DMDN_CHECK, a
 * stand-in for a memory sanitizer): the kernels test their shared- and
 * global-memory indices against the buffers they address; the first
 * violation since the last call is reported here (synchronous) as the
 * check site (a number > 0 naming the access in the source) and the index,
 * and its access is skipped.  *site = 0: no violation; *site = -1: this
 * library is not the checked build.  Reading clears the record. */
int mdn_check_status(int32_t* site, int64_t* index);

/* Bound, in nanoseconds, of every wait inside the tensor-core Gram kernel
 * (mbarrier hand-offs between its warp roles) for launches made after the
 * call, on every device; 0 restores the default of 2 s.  A wait that runs
 * out makes the kernel stop its roles, wait (with the default bound) for
 * its issued tensor-core operations, free its tensor memory and return;
 * mdn_train_status then reports 1.  Always returns MDN_OK. */
int mdn_set_gram_wait_limit(uint64_t ns);

/* Failure-detection test without a GPU fault: when enable != 0, the next
 * tensor-core Gram launch (any precision but MDN_GRAM_FP32) starts with a
 * wait on a barrier phase that nothing completes, so the wait runs out after
 * the wait limit and the launch takes the abort path above (no tensor-core
 * operation issued, partial sums not written).  One-shot: cleared by that
 * launch.  Always returns MDN_OK. */
int mdn_gram_expire_next_wait(int32_t enable);

/* Reads and clears the device-side error flag of the tensor-core Gram
 * kernels (synchronous, host pointer): *flag = 1 if a bounded wait inside a
 * Gram kernel expired since the last call (its partial sums were not
 * written and the result must be discarded), else 0. */
int mdn_train_status(int32_t* flag);

/* Training-set augmentation by the 8 flips / 90-degree rotations of the
 * pairs (Section 5 of the paper), applied to accumulated Gram sums instead of
 * re-gathering 8x the patches.  Transform t = rot + 4 * flip (rotate the
 * image by 90 degrees rot times, then mirror the columns if flip) maps the
 * patch of every pixel to the same patch with its taps permuted, and moves the
 * pixel's orientation bin a to a + rot * n_angle / 2 (mod n_angle), then to
 * n_angle - 1 - a if flip (strength and coherence bins are invariant).  So
 *   gram_out[k'][g] = sum_t P_t gram_in[k_t][g] P_t^T,  counts_out[k'] = sum_t counts_in[k_t]
 * with k_t the bucket that t maps to k' and P_t the tap permutation (targets
 * and, cross-channel, the channel order are unchanged).  Equal to training on
 * the 8 transformed pairs except at pixels whose orientation lies on a bin
 * boundary or is undefined (a zero structure tensor).  Single-level
 * geometries only (geom->r_coarse < 0): the pyramid of a mirrored image is
 * not the mirrored pyramid when a level has even size.  gram_in, counts_in:
 * device, as filled by mdn_train_level_filters; gram_out, counts_out: device,
 * same sizes, overwritten, not aliasing the inputs.  bp->n_angle must be
 * even.  Asynchronous on stream.  MDN_EINVAL / MDN_ESHAPE on bad arguments. */
int mdn_augment_dihedral(const double* gram_in, const int64_t* counts_in, const mdn_geometry* geom,
                         const mdn_bucket_params* bp, double* gram_out, int64_t* counts_out, void* stream);

/* The image form of transform t (0..7) for multiscale training, whose
 * pyramids do not commute with the mirror: out = mirror_columns_if(t >= 4)(
 * rot90^(t mod 4)(in)) per channel, rot90 of an (h x w) plane being the
 * (w x h) plane r[i][j] = in[j][w - 1 - i].  in: device [n][3][h][w] F32 or
 * F16; out: device, [n][3][w][h] for odd t, else [n][3][h][w], not aliasing
 * in.  Asynchronous on stream. */
int mdn_dihedral_images(const void* in, int32_t dtype, int64_t n, int64_t h, int64_t w, int32_t t, void* out,
                        void* stream);

/* Noise-level estimate per image, to choose the bank set trained for the
 * nearest noise level (the paper assumes the level is known and points to
 * estimating it for selecting the filter set, Section 6).  Robust wavelet
 * estimate: the finest diagonal Haar detail d = (a - b - c + e) / 2 of every
 * 2x2 block [a b; c e] (rows and columns 2i, 2i+1; an odd last row or column
 * is left out) of every channel; sigma = median(|d|) / 0.6745, the median
 * taken from a 16384-bin histogram over [0, 0.5) with linear interpolation in
 * the median bin (within one bin, 3.05e-5, of the exact median of |d|).
 * img: device [n][3][h][w] F32 or F16, h, w >= 2; sigma_out: device float[n];
 * ws: device, mdn_noise_workspace_bytes(n).  Asynchronous on stream. */
size_t mdn_noise_workspace_bytes(int64_t n);
int mdn_estimate_noise(const void* img, int32_t dtype, int64_t n, int64_t h, int64_t w, float* sigma_out,
                       void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Pyramid depth (Section 5: enough levels that the coarsest level's   */
/* noise is below 2 on the 0-255 scale)                                */
/* ------------------------------------------------------------------ */

/* Standard deviation of white noise at pyramid level `level` (0..7) relative
 * to the input, for this library's pyramid (mdn_build_pyramid: the binomial
 * [1 4 6 4 1]/16 kernel; the paper's bicubic downsampling would give other
 * factors), away from the clamped borders: level l is the input filtered by
 * the composed kernel c_l (c_0 = delta, c_{l+1}[m] = sum_u b[u] c_l[m - 2^l u])
 * and subsampled, and the separable 2-D kernel gives the factor
 * sum_m c_l[m]^2: 1, 0.273, 0.123, 0.060, 0.030, ...  (after level 1 the
 * noise is correlated and falls by ~0.45-0.5 per level, not 0.5 squared).
 * Returns -1 for a level outside 0..7.  Host-only arithmetic. */
double mdn_pyramid_noise_factor(int32_t level);

/* Section 5's depth rule: the fewest levels L >= 1 whose coarsest level's
 * noise, sigma * mdn_pyramid_noise_factor(L - 1), is below coarsest_sigma
 * (2/255 in the paper, on [0, 1] images), then clamped to [min_levels,
 * max_levels] (max_levels <= 8).  The rule gives L = 1 (single-scale) when
 * sigma itself is below coarsest_sigma; a caller whose bank sets are all
 * multiscale passes min_levels = 2.  Returns -1 on bad arguments (sigma < 0,
 * coarsest_sigma <= 0, min_levels < 1, max_levels > 8, min > max).
 * Host-only arithmetic. */
int32_t mdn_levels_for_sigma(double sigma, double coarsest_sigma, int32_t min_levels, int32_t max_levels);

/* Ridge solve per bucket and group in FP64 on the GPU:
 * h = (G_xx / n_k + lambda I)^{-1} (G_xy / n_k) by Cholesky; buckets with
 * n_k = 0 take the pooled filter solved from sum_k G_k.  bank_out: FP32
 * [K][3][D].  ws: at least mdn_solve_workspace_bytes().  status_out: device
 * int32[1], set to the number of systems whose Cholesky pivot was not
 * positive (those filters are written as zeros). */
size_t mdn_solve_workspace_bytes(const mdn_geometry* geom, int32_t K);
int mdn_solve_bank(const double* gram, const int64_t* counts, const mdn_geometry* geom,
                   int32_t K, double lambda, float* bank_out, int32_t* status_out, void* ws,
                   size_t ws_bytes, void* stream);


/* ------------------------------------------------------------------ */
/* Serving: continuous batching of multiscale denoise requests         */
/* (a deployment layer; the paper describes per-image inference only)  */
/* ------------------------------------------------------------------ */

/* A registered bank set: the filters of one noise level for a `levels`-level
 * pyramid, in the server's geometry (mdn_server_cfg.geom: 7x7 fine + 7x7 or
 * 5x5 coarse taps per channel); banks are FP16 [K][3][D] device buffers,
 * K <= MDN_MAX_K (the paper's 4096-bucket grid included), owned by the
 * caller and read for the server's lifetime (the server also keeps a copy
 * of each in the prepared row-slot layout). */
typedef struct {
    int32_t levels;                     /* 2..8 */
    const void* const* banks;           /* HOST array of levels-1 device pointers */
    const mdn_bucket_params* bparams;   /* HOST array of levels-1 entries */
    int32_t color;                      /* MDN_YCBCR601 or MDN_RGB */
} mdn_bankset;

typedef struct {
    int32_t device;              /* CUDA device ordinal */
    size_t hbm_budget_bytes;     /* device memory for request buffers (one arena, allocated at create) */
    int32_t max_active;          /* requests on the device at once (1..256) */
    int32_t autotune;            /* 1: time the level-kernel variants at create and keep the fastest */
    int32_t tile_variant;        /* used when autotune = 0: 0, 1 or 2 (tile kernels, 7x7 + 7x7 banks of
                                    at most 256 buckets) or 3 (fused kernel, any bank); -1: the
                                    autotune table's entry, else 3 */
    mdn_geometry geom;           /* bank geometry: r_fine 3, r_coarse 3 or 2, cross_channel 0 (color is
                                    taken from each bank set); all zero = 7x7 + 7x7 */
} mdn_server_cfg;

typedef struct {
    uint64_t id;
    int32_t status;              /* MDN_OK, or MDN_ETIMEOUT when cancelled before admission */
    double submit_ms, admit_ms, done_ms;   /* server clock (ms since create) */
} mdn_result;

typedef struct {
    uint64_t submitted, completed, cancelled, ticks, tick_items;
    int32_t active, queued;
    size_t arena_bytes, arena_used, arena_peak;
    int32_t tile_variant;        /* chosen level-kernel variant */
    float variant_ms[4];         /* autotuner timings (ms, -1 = not measured or not applicable) */
    int32_t variant_threads[4], variant_rows[4];   /* threads per CTA, tile rows */
    uint64_t ticks_large;        /* ticks of the large-request class */
} mdn_server_stats;

typedef struct mdn_server mdn_server;

/* Creates a server on cfg->device: allocates the request arena
 * (hbm_budget_bytes) once, copies the bank-set tables to the device, runs the
 * tile-shape autotuner, captures the per-tick CUDA graph (batched pyramid
 * launch + batched level launch, both reading a device work list) and starts
 * the scheduler thread. */
int mdn_server_create(const mdn_server_cfg* cfg, const mdn_bankset* sets, int32_t nsets, mdn_server** out);

/* Queues one request: host_in and host_out are HOST buffers of [3][h][w]
 * FP16 RGB (pinned memory gives asynchronous copies) that must stay valid
 * until the request's result is polled.  Requests of at least 4 M pixels
 * (large) run one per tick on two large-class tick contexts; smaller ones
 * are batched, up to about 4 M pixels a tick, on four small-class contexts
 * whose compute streams have the highest priority.  Each context has its
 * own upload, compute and download streams, so small requests never wait in
 * a stream behind a large one.  Within a class requests are admitted in
 * FIFO order as arena space and slots free up; a tick runs its requests'
 * whole chains (upload, pyramid, filter levels, download) in one replay of
 * the context's graph.  Pinned (page-locked, mapped) host buffers at 16-byte
 * aligned addresses are read and written by an SM copy kernel on a few SMs
 * that the server's compute kernels leave free; other buffers go through the
 * copy engines.  On Grace hosts the copy engines slow down 10-30x on pinned
 * buffers the GPU has not used for a second or more, SM copies 2-4x.
 * Returns MDN_EBUDGET (nothing queued) if the request alone exceeds the
 * budget. */
int mdn_server_submit(mdn_server* srv, const void* host_in, void* host_out, int64_t h, int64_t w, int32_t set,
                      uint64_t* id);

/* Removes a request that has not been admitted yet; its result is reported
 * with status MDN_ETIMEOUT.  Returns MDN_EINVAL if the id is not queued. */
int mdn_server_cancel(mdn_server* srv, uint64_t id);

/* Waits up to timeout_ms for at least one finished request (0 = do not
 * wait) and returns up to max of them in results; *n = how many. */
int mdn_server_poll(mdn_server* srv, mdn_result* results, int32_t max, int32_t* n, int32_t timeout_ms);

int mdn_server_get_stats(mdn_server* srv, mdn_server_stats* st);

/* Stops the scheduler (queued requests are dropped, admitted ones finish
 * first), frees the arena and the graph.  With the environment variable
 * MDN_SERVER_TRACE set to a path when the server was created, writes there a
 * CSV line per tick: requests, pixels, host launch and retire times (ms since
 * creation), the device times of its upload, its wait for and run of the
 * compute stream, its wait for and run of the download stream, and the ids of
 * its requests.  With MDN_SERVER_COPY_ENGINES=1 at creation, all host
 * transfers use the copy engines (see mdn_server_submit). */
int mdn_server_destroy(mdn_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* MDN_H */
