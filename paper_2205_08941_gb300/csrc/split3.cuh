// Three-term BF16 split of an FP64 value, x ~ b0 + b1 + b2, for the split-BF16 product.
// Host and device: the tile kernels' packing calls it on the device; a host build of the
// same function lets its arithmetic be checked without a GPU.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>

__host__ __device__ __forceinline__ uint64_t split3_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

__host__ __device__ __forceinline__ float split3_float(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
#endif
}

// Without FP64 instructions (the FP64 pipe is the scarce unit on this GPU): the double's
// bits give an FP32 head h (its significand cut to 24 bits) and an FP32 tail l (the 29 bits
// cut off, rounded to 24), x = h + l; then b0 = bf16(h), b1 = bf16(h - b0),
// b2 = bf16((h - b0 - b1) + l), the first two differences exact in FP32.
// |x - (b0 + b1 + b2)| is about 2^-27 |x| (at most 2^-25 |x|) for 2^-74 <= |x| < X_max,
// X_max = (2 - 2^-8) 2^127.  Below 2^-74 the tail's scale would be subnormal and is dropped
// (at most 2^-22 |x| down to 2^-109); below 2^-109 the later terms fall into BF16's
// subnormal range and lose bits (at most 2^-8 |x|, the first term's rounding); below the
// FP32 normal range (2^-126) all terms are zero.  From X_max on (where the first term
// rounds to infinity), and for infinities and NaNs, the terms are not finite and sum to
// NaN, so such values reach the product as NaN instead of vanishing.
__host__ __device__ __forceinline__ void split3(double x, __nv_bfloat16 &b0, __nv_bfloat16 &b1,
                                               __nv_bfloat16 &b2)
{
    const uint64_t u = split3_bits(x);
    const int e = (int)((u >> 52) & 0x7FF) - 1023 + 127;  // FP32 exponent field
    const uint64_t m = u & ((1ull << 52) - 1);
    const uint32_t sign = (uint32_t)(u >> 63) << 31;
    float h = 0.f, l = 0.f;
    if (e >= 1 && e <= 254) {
        h = split3_float(sign | ((uint32_t)e << 23) | (uint32_t)(m >> 29));
        if (e > 52) {  // the tail's scale 2^(exponent - 52) is a normal FP32 number
            l = (float)(uint32_t)(m & ((1u << 29) - 1)) * split3_float((uint32_t)(e - 52) << 23);
            if (sign) l = -l;
        }
    } else if (e > 254) {  // beyond the FP32 range, infinite or NaN
        h = split3_float(sign | 0x7FC00000u);
    }
    b0 = __float2bfloat16_rn(h);
    const float r1 = h - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r1);
    const float r2 = (r1 - __bfloat162float(b1)) + l;
    b2 = __float2bfloat16_rn(r2);
}
