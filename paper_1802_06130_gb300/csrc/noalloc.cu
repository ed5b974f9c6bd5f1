// noalloc.cu -- mdn_denoise_multiscale_static: multiscale denoising whose
// scratch memory (pyramid levels and intermediate level outputs) lives in a
// fixed, file-scope device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at all: a plug-in running
// inside a host application that owns every device allocation through its
// own pool, or a real-time camera pipeline where an allocation call (which
// may synchronise the device) is not allowed on the frame path.  They still
// own the input, the output and the banks; this entry point takes the
// workspace from g_scratch below and calls no cudaMalloc, cudaFree or any
// other allocating routine.
//
// Properties a caller must know (also stated in include/mdn.h):
//  * g_scratch is MDN_STATIC_SCRATCH_BYTES (48 MiB) on EVERY device that loads
//    the library, held until the process exits;
//  * the first call on a device, with that device current, looks up the
//    array's device address (cudaGetSymbolAddress) and caches it per device
//    ordinal; make that first call before any stream capture.  The cache is
//    not told about cudaDeviceReset: a process that resets a device (which
//    ends its context and every device address in it) must not call this
//    entry point on that device again;
//  * every call on a device shares the same array, which keeps the previous
//    call's contents: calls whose work overlaps on the GPU (other streams,
//    other host threads) race and corrupt each other's results.  Nothing in
//    the array needs clearing: every scratch element is written before it is
//    read within one call.
#include <mutex>

#include "internal.h"

namespace mdn {
namespace {

constexpr size_t kStaticScratchBytes = size_t(48) << 20;
static_assert(kStaticScratchBytes == MDN_STATIC_SCRATCH_BYTES, "header and implementation disagree");

__device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device (host code must not use
// the symbol itself: on the host it is only a stand-in).
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "denoise_multiscale_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(MDN_EINVAL, "denoise_multiscale_static: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "denoise_multiscale_static: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MDN_OK;
}

}  // namespace
}  // namespace mdn

extern "C" int mdn_denoise_multiscale_static(const void* noisy, int32_t dtype, int64_t n, int64_t h, int64_t w,
                                             int32_t levels, const void* const* banks, int32_t bank_dtype,
                                             const mdn_geometry* geom, const mdn_bucket_params* bparams,
                                             void* out, void* const* bucket_maps, void* stream) {
    using namespace mdn;
    if (levels < 1 || levels > 8) return fail(MDN_EINVAL, "denoise_multiscale_static: levels must be 1..8");
    // sizes first (bounded without overflow), then the workspace arithmetic
    int rc = check_img(noisy, dtype, n, h, w, "denoise_multiscale_static");
    if (rc) return rc;
    const size_t need = mdn_denoise_workspace_bytes(n, h, w, levels, dtype);
    if (need > kStaticScratchBytes)
        return fail(MDN_EWORKSPACE, "denoise_multiscale_static: this image needs " + std::to_string(need) +
                                        " bytes of scratch, more than the 48 MiB static array; use "
                                        "mdn_denoise_multiscale with a caller workspace");
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    return mdn_denoise_multiscale(noisy, dtype, n, h, w, levels, banks, bank_dtype, geom, bparams, out,
                                  bucket_maps, scratch, kStaticScratchBytes, stream);
}
