// bank_rows.cu -- mdn_prepare_bank_rows / mdn_bank_rows_bytes: a filter
// bank [K][3][D] laid out once in the row-slot form the fused level kernel
// reads (one 16-byte FP16 or 32-byte FP32 slot per bucket, output channel,
// block and filter row, with the 2r+1 taps of that row; see RowSlots and
// load_bank_rows in k_level.cuh).  Banks too large for shared memory (the
// 4096-bucket grid, FP32 banks of 216 buckets of 7x7 + 7x7 taps) are then
// read by the fused kernel straight from this layout through L2, with
// coalesced 16-byte loads; smaller ones are copied to shared memory whole.
#include "k_level.cuh"

namespace mdn {
namespace {

template <int RF, int RC, bool CROSS, typename TB>
__global__ void __launch_bounds__(256) k_prepare_rows(const TB* __restrict__ bank, int K, unsigned char* rows) {
    lvl::v3::load_bank_rows<RF, RC, CROSS, TB>(bank, K, rows, blockIdx.x * blockDim.x + threadIdx.x,
                                               gridDim.x * blockDim.x);
}

template <int RF, int RC, bool CROSS, typename TB>
int prepare(const void* bank, int K, void* rows, cudaStream_t s) {
    using SL = lvl::v3::RowSlots<RF, RC, CROSS>;
    const int64_t elems = (int64_t)K * SL::S * 8;
    const int grid = (int)((elems + 255) / 256 < 4096 ? (elems + 255) / 256 : 4096);
    k_prepare_rows<RF, RC, CROSS, TB><<<grid, 256, 0, s>>>((const TB*)bank, K, (unsigned char*)rows);
    return check_launch("k_prepare_rows");
}

// bytes per bucket of the row-slot layout, 0 for a geometry the kernels are not compiled for
int bucket_row_bytes(const mdn_geometry& g, int elem_dtype) {
    const int sb = elem_dtype == MDN_F16 ? 16 : 32;
#define MDN_GEO(RF_, RC_, CR_) \
    if (g.r_fine == RF_ && g.r_coarse == RC_ && (g.cross_channel != 0) == CR_) return lvl::v3::RowSlots<RF_, RC_, CR_>::S * sb;
    MDN_GEO(2, -1, false)
    MDN_GEO(3, 3, false)
    MDN_GEO(3, 2, false)
    MDN_GEO(3, -1, true)
    MDN_GEO(2, 1, false)
#undef MDN_GEO
    return 0;
}

}  // namespace
}  // namespace mdn

using namespace mdn;

extern "C" size_t mdn_bank_rows_bytes(const mdn_geometry* geom, int32_t K, int32_t bank_dtype) {
    if (!geom || K < 1 || K > MDN_MAX_K || (bank_dtype != MDN_F32 && bank_dtype != MDN_F16)) return 0;
    return (size_t)K * bucket_row_bytes(*geom, bank_dtype);
}

extern "C" int mdn_prepare_bank_rows(const void* bank, int32_t bank_dtype, const mdn_geometry* geom, int32_t K,
                                     void* rows, size_t rows_bytes, void* stream) {
    NvtxRange nvtx_range("mdn_prepare_bank_rows");
    if (!bank || !rows || !geom) return fail(MDN_EINVAL, "prepare_bank_rows: null pointer");
    if (bank_dtype != MDN_F32 && bank_dtype != MDN_F16)
        return fail(MDN_EINVAL, "prepare_bank_rows: bank dtype must be MDN_F32 or MDN_F16");
    if (K < 1 || K > MDN_MAX_K) return fail(MDN_EINVAL, "prepare_bank_rows: K must be 1..4096");
    const size_t need = mdn_bank_rows_bytes(geom, K, bank_dtype);
    if (need == 0) return fail(MDN_ESHAPE, "prepare_bank_rows: geometry not compiled");
    if (rows_bytes < need) return fail(MDN_EWORKSPACE, "prepare_bank_rows: output smaller than mdn_bank_rows_bytes");
    if ((uintptr_t)rows % 16 != 0) return fail(MDN_EINVAL, "prepare_bank_rows: output not 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const mdn_geometry& g = *geom;
#define MDN_GEO(RF_, RC_, CR_)                                                                              \
    if (g.r_fine == RF_ && g.r_coarse == RC_ && (g.cross_channel != 0) == CR_)                              \
        return bank_dtype == MDN_F16 ? prepare<RF_, RC_, CR_, __half>(bank, K, rows, s)                     \
                                     : prepare<RF_, RC_, CR_, float>(bank, K, rows, s);
    MDN_GEO(2, -1, false)
    MDN_GEO(3, 3, false)
    MDN_GEO(3, 2, false)
    MDN_GEO(3, -1, true)
    MDN_GEO(2, 1, false)
#undef MDN_GEO
    return fail(MDN_ESHAPE, "prepare_bank_rows: geometry not compiled");
}
