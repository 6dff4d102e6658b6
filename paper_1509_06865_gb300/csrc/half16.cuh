// 16-bit storage types of the coarse links (bfloat16, IEEE half): conversion of
// one value from FP32 and of a packed pair to FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace mgeig {

template <typename H> struct H16;
template <> struct H16<__nv_bfloat16> {
    __device__ __forceinline__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    __device__ __forceinline__ static float2 pair(__nv_bfloat162 v) { return __bfloat1622float2(v); }
    using P = __nv_bfloat162;
};
template <> struct H16<__half> {
    __device__ __forceinline__ static __half from(float v) { return __float2half_rn(v); }
    __device__ __forceinline__ static float2 pair(__half2 v) { return __half22float2(v); }
    using P = __half2;
};

}  // namespace mgeig
