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

}  // namespace mdn
