// dword.cuh -- double-word (FP32 pair) arithmetic for FP64-class steps of the MIXED32
// field solve, and FP64 <-> FP32 conversions by bit manipulation.
//
// GB300 retires about one FP64 operation per SM per cycle against 128 FP32 ones, so
// stencil arithmetic that needs more than FP32 precision (the refinement's residual
// r = b - A x, the right-hand side of Eq. (7), the field update) runs on pairs (h, l)
// of FP32 numbers, x = h + l with |l| <= ulp(h) / 2: 47 significant bits, about 7e-15
// relative. Building blocks: Knuth's TwoSum and Dekker's FastTwoSum (exact sums), the
// FMA-based exact product, and the "sloppy" pair sum and pair-times-pair product
// analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017): each result carries an
// absolute error of a few 2^-47 times its operands' magnitude, as long as the low words
// and error terms stay normal FP32 numbers: magnitudes above about 2^-75 (products above
// 2^-70; the fields, currents and residuals of the simulations here are many orders
// larger). Explicit
// round-to-nearest intrinsics keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace pic {

struct DW {  // h + l
    float h, l;
};

__device__ __forceinline__ DW two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DW fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DW dw_add(DW x, DW y) {
    const DW s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DW dw_neg(DW x) { return {-x.h, -x.l}; }
__device__ __forceinline__ DW dw_sub(DW x, DW y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ DW dw_add_f(DW x, float y) {
    const DW s = two_sum(x.h, y);
    return fast_two_sum(s.h, __fadd_rn(s.l, x.l));
}
__device__ __forceinline__ DW dw_mul(DW x, DW y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ DW dw_twice(DW x) { return {__fadd_rn(x.h, x.h), __fadd_rn(x.l, x.l)}; }  // exact

// FP64 -> pair: h = x truncated to 24 significant bits, l = the next 23 bits;
// magnitudes below 2^-126 (and l below 2^-126) flush to zero.
__device__ __forceinline__ DW dw_from(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    const unsigned int sgn = hw & 0x80000000u;
    const int E = (int)((hw >> 20) & 0x7ffu);
    const int fe = E - 896;  // float exponent field of h (1023 - 127 = 896)
    const float h = (fe > 0 && fe < 255)
                        ? __uint_as_float(sgn | ((unsigned int)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29))
                        : 0.f;
    // the next 23 mantissa bits m, worth m 2^(E - 1023 - 46): exactly (2^23 + m) - 2^23
    const float m = __fsub_rn(__uint_as_float(0x4b000000u | ((lw >> 6) & 0x7fffffu)), 8388608.f);
    const int se = E - 1023 - 46 + 127;
    const float l = (fe > 0 && fe < 255 && se > 0) ? __fmul_rn(m, __uint_as_float((unsigned int)se << 23)) : 0.f;
    return fast_two_sum(h, sgn ? -l : l);
}
// float -> double (exact; zero and subnormal inputs give zero)
__device__ __forceinline__ double f64_of(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
// pair -> FP64 (one FP64 add)
__device__ __forceinline__ double dw_join(DW x) { return f64_of(x.h) + f64_of(x.l); }
// double -> float rounded to nearest (ties to even), as (float)x does for values in the
// normal float range; magnitudes below 2^-126 give (signed) zero
__device__ __forceinline__ float f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    const unsigned int sgn = hw & 0x80000000u;
    const int fe = (int)((hw >> 20) & 0x7ffu) - 896;
    if (fe <= 0) return __uint_as_float(sgn);
    if (fe >= 255) return __uint_as_float(sgn | 0x7f800000u);
    const unsigned int mag = ((unsigned int)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned int rem = lw & 0x1fffffffu;  // the 29 bits below float precision
    const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (mag & 1u))) ? 1u : 0u;
    return __uint_as_float(sgn | (mag + up));  // a carry into the exponent is the correct rounding
}

// int64 -> pair by integer operations: h = the leading 24 bits, l = the next 23 (exact
// for |d| < 2^47; relative 2^-47 beyond)
__device__ __forceinline__ DW dw_from_i64(long long d) {
    if (d == 0) return {0.f, 0.f};
    const bool neg = d < 0;
    const unsigned long long a = neg ? 0ull - (unsigned long long)d : (unsigned long long)d;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;  // leading one at bit 63: a = n 2^-lz
    // h = (n >> 40) 2^(40 - lz): float exponent field 63 - lz + 127
    const unsigned int hb = ((unsigned int)(190 - lz) << 23) | ((unsigned int)(n >> 40) & 0x7fffffu);
    // the next 23 bits, worth (n >> 17 & 0x7fffff) 2^(17 - lz)
    const float m = __fsub_rn(__uint_as_float(0x4b000000u | ((unsigned int)(n >> 17) & 0x7fffffu)), 8388608.f);
    const float l = __fmul_rn(m, __uint_as_float((unsigned int)(144 - lz) << 23));  // 2^(17 - lz)
    const DW r = fast_two_sum(__uint_as_float(hb), l);
    return neg ? dw_neg(r) : r;
}

// Sum over a warp; every lane gets the same pair (the pair sum is symmetric in its
// operands).
__device__ __forceinline__ DW warp_sum_dw(DW v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DW w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = dw_add(v, w);
    }
    return v;
}

}  // namespace pic
