// common.cuh -- small device helpers shared by the kernel translation units.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace mdn {

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
