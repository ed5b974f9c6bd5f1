// common.cuh -- small device helpers shared by the kernel translation units.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace mdn {

// Bounds checks of the debug build (-DMDN_CHECK, stand-in for a memory
// sanitizer): mdn_in(i, n, site) is true when 0 <= i < n; otherwise the
// first violation of the process (site, index) is recorded in g_mdn_check
// (read and cleared by mdn_check_status) and the caller skips the access.
// In normal builds it is the constant true and costs nothing.
#ifdef MDN_CHECK
extern __device__ unsigned long long g_mdn_check;
__device__ __forceinline__ bool mdn_in(int64_t i, int64_t n, int site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_mdn_check, 0ull,
              (1ull << 63) | ((unsigned long long)(site & 0x7fff) << 48) | ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
#else
__device__ __forceinline__ constexpr bool mdn_in(int64_t, int64_t, int) { return true; }
#endif

template <typename T> __device__ __forceinline__ float ld_f(const T* p, int64_t i);
template <> __device__ __forceinline__ float ld_f<float>(const float* p, int64_t i) { return __ldg(p + i); }
template <> __device__ __forceinline__ float ld_f<__half>(const __half* p, int64_t i) {
    return __half2float(__ldg(p + i));
}

template <typename T> __device__ __forceinline__ void st_f(T* p, int64_t i, float v);
template <> __device__ __forceinline__ void st_f<float>(float* p, int64_t i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void st_f<__half>(__half* p, int64_t i, float v) {
    p[i] = __float2half_rn(v);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// four consecutive elements as floats (8-byte aligned FP16, 16-byte aligned FP32)
__device__ __forceinline__ void ld4(const __half* p, float* out) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float* out) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
}

}  // namespace mdn
