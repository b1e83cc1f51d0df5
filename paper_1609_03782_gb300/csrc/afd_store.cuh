// Storage formats of a cube on the GPU (precision line).
//
// A 2-byte cube holds value / s in float16 or bfloat16, or round(value / s)
// as an int16 count of s = scale / 1024 (clamped to +-32767), with a
// power-of-two per-cube scale.  Kernels compute in storage units: because s
// is a power of two, filtering value / s with K / s is, operation for
// operation, the float32 filter of the dequantised cube divided by s (every
// product and quotient of the per-face arithmetic scales exactly), so a pass
// of a 2-byte kernel equals dequantise -> float32 iterations -> quantise, bit
// for bit.  Rounding into the 2-byte format is to nearest, ties to even.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace afd {

enum StoreKind : int { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2, STORE_I16 = 3 };

constexpr int kI16FracBits = 10;  // int16 step = scale / 2^10
constexpr int kI16Max = 32767;

template <int S>
struct Store;

template <>
struct Store<STORE_F32> {
    typedef float T;
    static constexpr int bytes = 4;
    __device__ __forceinline__ static float load(T v) { return v; }
    __device__ __forceinline__ static T store(float v) { return v; }
};

template <>
struct Store<STORE_F16> {
    typedef unsigned short T;
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float load(T v) { return __half2float(__ushort_as_half(v)); }
    __device__ __forceinline__ static T store(float v) { return __half_as_ushort(__float2half_rn(v)); }
};

template <>
struct Store<STORE_BF16> {
    typedef unsigned short T;
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float load(T v)
    {
        return __uint_as_float(static_cast<unsigned>(v) << 16);
    }
    __device__ __forceinline__ static T store(float v)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};

// int16 <-> float32 without the conversion unit (which the conductances'
// MUFU operations also use): the float 1.5 * 2^23 has an ulp of 1, so
//   load:  bits(1.5*2^23) + q, reinterpreted, minus 1.5*2^23 is exactly q;
//   store: v is first clamped to +-32767 (the same result as rounding then
//          clamping), then v + 1.5*2^23 rounds it to an integer (to nearest,
//          ties to even) and its bits minus bits(1.5*2^23) are that integer.
template <>
struct Store<STORE_I16> {
    typedef short T;
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float load(T v)
    {
        return __fsub_rn(__int_as_float(0x4B400000 + static_cast<int>(v)), 12582912.0f);
    }
    __device__ __forceinline__ static T store(float v)
    {
        const float c = fminf(fmaxf(v, -32767.0f), 32767.0f);
        return static_cast<short>(__float_as_int(__fadd_rn(c, 12582912.0f)) - 0x4B400000);
    }
};

// Two floats -> two storage elements packed in 32 bits (low = first).  The
// 2-byte float formats use the packed conversions (each lane rounds like the
// scalar one).
template <int S>
__device__ __forceinline__ unsigned store2(float lo, float hi)
{
    if constexpr (S == STORE_F16) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    } else if constexpr (S == STORE_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&h);
    } else {
        return static_cast<unsigned>(static_cast<unsigned short>(Store<S>::store(lo))) |
               (static_cast<unsigned>(static_cast<unsigned short>(Store<S>::store(hi))) << 16);
    }
}

// Size in bytes of one element of storage kind s.
inline int store_bytes(int s) { return s == STORE_F32 ? 4 : 2; }

// Storage units per unit of the cube's values: 1/scale (f16, bf16),
// 1024/scale (i16), 1 (f32).
inline double store_units_per_value(int s, double scale)
{
    if (s == STORE_F32)
        return 1.0;
    if (s == STORE_I16)
        return static_cast<double>(1 << kI16FracBits) / scale;
    return 1.0 / scale;
}

}  // namespace afd
