// FP64 -> FP32 round-to-nearest-even conversions built from the operand's
// IEEE 754 encoding with integer operations, and the double-single split
// v = hi + lo (hi = RN32(v), lo = RN32(v - hi)) that the mixed j images hold.
//
// On this part FP64 arithmetic and the f64 -> f32 conversion instruction share
// the narrow FP64 pipe (one warp instruction holds it for about as long as a
// DFMA), and packing an image record takes 10 conversions and 3 FP64
// subtractions. Built from the bits, the same results come from the integer
// pipes and one int -> float conversion per low word. The results are the
// conversion instructions' bit for bit: the bit construction covers the
// magnitudes where both words are normal floats (and zero); the rest (tiny,
// huge, non-finite) takes the conversion instructions in a separate function.
//
// The header also compiles as plain C++, so the host tests check the bit
// construction against the host's conversions.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define KIRIN_PACK_HD __host__ __device__ __forceinline__
#define KIRIN_PACK_COLD __host__ __device__ __noinline__
#else
#include <string.h>
#define KIRIN_PACK_HD inline
#define KIRIN_PACK_COLD __attribute__((noinline)) inline
#endif

namespace kirin {
namespace f32pack {
namespace {

KIRIN_PACK_HD uint64_t bits_of(double v)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    return b;
#endif
}

KIRIN_PACK_HD float float_of(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

KIRIN_PACK_HD float int_to_float(int32_t i)
{
#ifdef __CUDA_ARCH__
    return __int2float_rn(i);
#else
    return (float)i;
#endif
}

KIRIN_PACK_HD uint32_t exponent_field(uint64_t b) { return (uint32_t)(b >> 52) & 0x7ffu; }

// Finite (neither infinite nor NaN): the exponent field is not all ones.
KIRIN_PACK_HD bool finite(double v) { return exponent_field(bits_of(v)) != 0x7ffu; }

// The RN32 of v with exponent field e in [897, 1150] (2^-126 <= |v| < 2^128),
// as bits, and r = v - RN32(v) in units of v's last place 2^(e - 1075)
// (|r| <= 2^28, the sign taken against |v|). The 52-bit fraction keeps its top
// 23 bits; the 29 bits below decide the rounding, ties to the even word. A
// carry out of the fraction moves into the exponent, which is the rounded
// value (infinity above the largest float).
KIRIN_PACK_HD uint32_t rn32_bits(uint64_t b, int32_t &r)
{
    const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
    uint32_t f = ((exponent_field(b) - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
    const uint32_t rem = lw & 0x1fffffffu;
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (f & 1u));
    f += up ? 1u : 0u;
    r = up ? (int32_t)rem - 0x20000000 : (int32_t)rem;
    return (hw & 0x80000000u) | f;
}

KIRIN_PACK_COLD float to_f32_slow(double v)
{
#ifdef __CUDA_ARCH__
    return __double2float_rn(v);
#else
    return (float)v;
#endif
}

KIRIN_PACK_COLD void split_slow(double v, float &hi, float &lo)
{
#ifdef __CUDA_ARCH__
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
#else
    hi = (float)v;
    lo = (float)(v - (double)hi);
#endif
}

// RN32(v), as the conversion instruction gives it.
KIRIN_PACK_HD float to_f32(double v)
{
    const uint64_t b = bits_of(v);
    const uint32_t e = exponent_field(b);
    int32_t r;
    if (e - 897u <= 1150u - 897u)
        return float_of(rn32_bits(b, r));
    if ((b << 1) == 0)
        return float_of((uint32_t)(b >> 32) & 0x80000000u);  // +-0
    return to_f32_slow(v);
}

// hi = RN32(v), lo = RN32(v - hi). With the exponent field e of v in
// [949, 1149] (2^-74 <= |v| < 2^127), hi is finite and v - hi = r 2^(e - 1075)
// exactly, with 2^(e - 1075) a normal float, so lo is the RN32 of the integer r
// scaled by that power of two (exact). At zero both words are zero (hi keeps
// the sign, lo is +0 as v - hi is).
KIRIN_PACK_HD void split(double v, float &hi, float &lo)
{
    const uint64_t b = bits_of(v);
    const uint32_t e = exponent_field(b);
    if (e - 949u <= 1149u - 949u) {
        int32_t r;
        hi = float_of(rn32_bits(b, r));
        const int32_t rs = (b >> 63) ? -r : r;
        lo = int_to_float(rs) * float_of((e - 948u) << 23);
        return;
    }
    if ((b << 1) == 0) {
        hi = float_of((uint32_t)(b >> 32) & 0x80000000u);
        lo = 0.0f;
        return;
    }
    split_slow(v, hi, lo);
}

}  // namespace
}  // namespace f32pack
}  // namespace kirin
