// Eight signed 8-bit digits of an FP64 value against a power-of-two scale, for the
// emulated-FP64 tensor-core product (Ozaki-style slicing).  Host and device: the packing
// kernels call it on the device; a host build of the same functions lets the arithmetic be
// checked without a GPU.
//
// A group of values (one scalar row of an A panel, or one scalar column of a B panel, over
// sixteen atoms of K) shares an exponent E with |x| < 2^E for every x of the group.  Each
// x is rounded once to the fixed-point integer Y = round(x 2^(63 - E)), |Y| <= 2^63, and
// Y is cut into centred base-256 digits, Y = sum_{p=0..7} d_p 2^(8 (7 - p)) with
// |d_p| <= 128, so x = 2^(E - 7) sum_p d_p 2^(-8p) up to |x - that| <= 2^(E - 64).  Every
// d_p 2^(-8p) is exact in BF16 (an integer of at most 8 significant bits times a power of
// two inside BF16's exponent range), so the tensor cores multiply digits exactly and the
// product of planes p and q lands at its level's weight 2^(-8 (p + q)).
//
// Eight digits keep the representation error at 2^-64 of the group's largest magnitude, so a
// value up to 2^11 below that largest one is still carried to FP64's 2^-53 of itself.
// Only integer operations touch the double (its bits are taken apart), so packing stays
// off the FP64 pipe.  A group holding an infinity or a NaN gets the exponent EMU_POISON
// and NaN digits, so such values reach the product as NaN (as in FP64) instead of
// vanishing; a group of zeros gets EMU_NONE and zero digits.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>

constexpr int EMU_P = 8;              // digit planes
constexpr int EMU_NONE = -32768;      // exponent of a group with no nonzero value
constexpr int EMU_POISON = 32767;     // exponent of a group with an infinity or a NaN

__host__ __device__ __forceinline__ uint64_t emu_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

__host__ __device__ __forceinline__ float emu_float(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
#endif
}

__host__ __device__ __forceinline__ int emu_bitlen(uint64_t m)
{
#ifdef __CUDA_ARCH__
    return 64 - __clzll((long long)m);
#else
    int n = 0;
    while (m) {
        ++n;
        m >>= 1;
    }
    return n;
#endif
}

// Smallest E with |x| < 2^E (EMU_NONE for zero, EMU_POISON for infinities and NaNs).
__host__ __device__ __forceinline__ int emu_exponent(double x)
{
    const uint64_t u = emu_bits(x);
    const int ex = (int)((u >> 52) & 0x7FF);
    const uint64_t m = u & ((1ull << 52) - 1);
    if (ex == 0x7FF) return EMU_POISON;
    if (ex == 0) return m ? emu_bitlen(m) - 1074 : EMU_NONE;
    return ex - 1022;
}

// The eight digit planes of x in group exponent E (E >= emu_exponent(x)), as the BF16
// values d_p 2^(-8p).
__host__ __device__ __forceinline__ void emu_digits(double x, int E, __nv_bfloat16 (&out)[EMU_P])
{
    if (E == EMU_POISON) {
        out[0] = __float2bfloat16_rn(emu_float(0x7FC00000u));
        for (int p = 1; p < EMU_P; ++p) out[p] = __float2bfloat16_rn(0.0f);
        return;
    }
    const uint64_t u = emu_bits(x);
    int ex = (int)((u >> 52) & 0x7FF);
    uint64_t m = u & ((1ull << 52) - 1);
    if (ex) {
        m |= 1ull << 52;
    } else {
        ex = 1;  // subnormal: x = m 2^-1074
    }
    // |x| = m 2^(ex - 1075), so |Y| = |x| 2^(63 - E) = m 2^sh; |x| < 2^E keeps sh <= 10 for
    // normal x and |Y| below 2^63 (an unsigned 64-bit magnitude; the sign goes on the digits)
    const int sh = ex - 1012 - E;
    uint64_t Y = 0;
    if (E != EMU_NONE && m != 0) {
        if (sh >= 0)
            Y = m << sh;
        else if (sh > -64)
            Y = (m + (1ull << (-sh - 1))) >> (-sh);  // round half away from zero
    }
    int d[EMU_P];
    for (int p = EMU_P - 1; p > 0; --p) {
        d[p] = (int)((Y + 128) & 255) - 128;  // centred remainder, -128 <= d < 128
        Y = (Y - (uint64_t)(int64_t)d[p]) >> 8;  // exact: Y - d is a multiple of 256
    }
    d[0] = (int)Y;  // d_0 <= 128
    const float sgn = (u >> 63) ? -1.0f : 1.0f;
    float w = 1.0f;
    for (int p = 0; p < EMU_P; ++p) {
        out[p] = __float2bfloat16_rn(sgn * (float)d[p] * w);  // exact
        w *= 1.0f / 256.0f;
    }
}
