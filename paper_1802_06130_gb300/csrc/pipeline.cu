// pipeline.cu -- mdn_denoise_multiscale_pipelined: multiscale denoising of a
// batch held in HOST memory, with the host-to-device copies, the kernels and
// the device-to-host copies of consecutive chunks overlapped.
//
// Chunk c of `chunk` images goes through
//   upload stream:     copy host_noisy[c] -> dev_in[c], record `up`
//   compute stream c%P: wait `up`, mdn_denoise_multiscale(dev_in[c] -> dev_out[c])
//                      on workspace slice c%P, record `done`
//   download stream:   wait `done`, copy dev_out[c] -> host_out[c]
// with P = 1 or 2 compute streams.  In steady state chunk c+1 uploads and
// chunk c-1 downloads while chunk c is filtered; with two compute streams the
// start-up and tail of one chunk's kernels also overlap the other chunk's.
// Every wait is enqueued right after the record it refers to (a stream waits
// on the event's state at the time of the call), so one event per role serves
// every chunk.  The events are created per call and released at its end (the
// driver frees them once their work completes); no device memory is
// allocated: dev_in, dev_out and the workspace are the caller's.
#include <string>

#include "internal.h"

namespace {

struct Events {
    cudaEvent_t start = nullptr, up = nullptr, done = nullptr, fin = nullptr, fin2 = nullptr;
    ~Events() {
        for (cudaEvent_t e : {start, up, done, fin, fin2})
            if (e) cudaEventDestroy(e);
    }
};

size_t esize(int dtype) { return dtype == MDN_F16 ? 2 : 4; }

}  // namespace

extern "C" int mdn_denoise_multiscale_pipelined(const void* host_noisy, int32_t dtype, int64_t n, int64_t h,
                                                int64_t w, int32_t levels, const void* const* banks,
                                                int32_t bank_dtype, const mdn_geometry* geom,
                                                const mdn_bucket_params* bparams, void* host_out, int64_t chunk,
                                                void* dev_in, void* dev_out, void* ws, size_t ws_bytes,
                                                void* const* streams, int32_t nstreams) {
    using namespace mdn;
    NvtxRange nvtx_range("mdn_denoise_multiscale_pipelined");
    int rc = check_img(host_noisy, dtype, n, h, w, "denoise_multiscale_pipelined");
    if (rc) return rc;
    if (!streams) return fail(MDN_EINVAL, "denoise_multiscale_pipelined: streams null");
    if (nstreams != 3 && nstreams != 4) return fail(MDN_EINVAL, "denoise_multiscale_pipelined: nstreams must be 3 or 4");
    if (chunk < 1) return fail(MDN_EINVAL, "denoise_multiscale_pipelined: chunk must be >= 1");
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "denoise_multiscale_pipelined: levels must be 1..8");
    if (n * h * w > 0 && (!host_out || !dev_in || !dev_out))
        return fail(MDN_EINVAL, "denoise_multiscale_pipelined: null buffer");
    const int P = nstreams - 2;   // compute streams
    const int64_t c = chunk < n ? chunk : n;
    const size_t slice = align256(mdn_denoise_workspace_bytes(c, h, w, levels, dtype));
    const size_t need = P == 1 ? mdn_denoise_workspace_bytes(c, h, w, levels, dtype) : 2 * slice;
    if (ws_bytes < need || (need && !ws))
        return fail(MDN_EWORKSPACE, "denoise_multiscale_pipelined: workspace too small (one chunk's "
                                    "mdn_denoise_workspace_bytes per compute stream, 256-byte aligned)");
    if (n == 0 || h == 0 || w == 0) return MDN_OK;
    cudaStream_t su = (cudaStream_t)streams[0], sd = (cudaStream_t)streams[nstreams - 1];
    cudaStream_t sc[2] = {(cudaStream_t)streams[1], (cudaStream_t)streams[P == 2 ? 2 : 1]};
    for (int i = 0; i < nstreams; ++i)
        for (int j = i + 1; j < nstreams; ++j)
            if (streams[i] == streams[j]) return fail(MDN_EINVAL, "denoise_multiscale_pipelined: the streams must differ");
    Events ev;
    cudaError_t e = cudaSuccess;
    for (cudaEvent_t* p : {&ev.start, &ev.up, &ev.done, &ev.fin, &ev.fin2})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "denoise_multiscale_pipelined: event create");
    // the copies and the second compute stream start after the work already
    // queued on the first compute stream
    if ((e = cudaEventRecord(ev.start, sc[0])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(su, ev.start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(sd, ev.start, 0)) != cudaSuccess ||
        (P == 2 && (e = cudaStreamWaitEvent(sc[1], ev.start, 0)) != cudaSuccess))
        return cuda_fail(e, "denoise_multiscale_pipelined: stream order");
    const size_t img_bytes = (size_t)3 * h * w * esize(dtype);
    int64_t idx = 0;
    for (int64_t i0 = 0; i0 < n; i0 += c, ++idx) {
        const int64_t m = n - i0 < c ? n - i0 : c;
        const int k = (int)(idx % P);
        const size_t off = (size_t)i0 * img_bytes, bytes = (size_t)m * img_bytes;
        char* din = (char*)dev_in + off;
        char* dout = (char*)dev_out + off;
        if ((e = cudaMemcpyAsync(din, (const char*)host_noisy + off, bytes, cudaMemcpyHostToDevice, su)) !=
                cudaSuccess ||
            (e = cudaEventRecord(ev.up, su)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(sc[k], ev.up, 0)) != cudaSuccess)
            return cuda_fail(e, "denoise_multiscale_pipelined: upload");
        void* wsk = P == 1 ? ws : (void*)((char*)ws + k * slice);
        const size_t wsb = P == 1 ? ws_bytes : slice;
        rc = mdn_denoise_multiscale(din, dtype, m, h, w, levels, banks, bank_dtype, geom, bparams, dout, nullptr, wsk,
                                    wsb, sc[k]);
        if (rc) return rc;
        if ((e = cudaEventRecord(ev.done, sc[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(sd, ev.done, 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync((char*)host_out + off, dout, bytes, cudaMemcpyDeviceToHost, sd)) != cudaSuccess)
            return cuda_fail(e, "denoise_multiscale_pipelined: download");
    }
    // completion is signalled on the first compute stream (after the last
    // download, and after the second compute stream's work)
    if ((e = cudaEventRecord(ev.fin, sd)) != cudaSuccess || (e = cudaStreamWaitEvent(sc[0], ev.fin, 0)) != cudaSuccess)
        return cuda_fail(e, "denoise_multiscale_pipelined: join");
    if (P == 2 && ((e = cudaEventRecord(ev.fin2, sc[1])) != cudaSuccess ||
                   (e = cudaStreamWaitEvent(sc[0], ev.fin2, 0)) != cudaSuccess))
        return cuda_fail(e, "denoise_multiscale_pipelined: join");
    return MDN_OK;
}
