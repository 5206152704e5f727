// Float-float ("double-single") arithmetic for the float-float mode of FP64
// contexts: the demag passes and, for uniform material, the LLG stage.
//
// GB300 runs FP64 at about 2 FMA per SM per clock, against 128 FP32 lanes.
// A value is carried as the unevaluated sum h + l of two floats (about 48
// significant bits), and every operation is built from FP32 instructions:
//   add: Knuth's TwoSum of the high parts, the low parts added into the
//        error, then a renormalising fast two-sum (Dekker);
//   mul: the exact product error of the high parts from one FMA (TwoProd),
//        the cross terms added by FMA, then the fast two-sum.
// The add is the "sloppy" form: its error is bounded by a small multiple of
// 2^-48 (|a| + |b|), the same shape as an FP add's bound, which is what the
// FFT error analysis uses.  Spectra stored as ffc take 16 bytes, like double2.
//
// Conversions from double (d2ff) and to double (ff2d) are done with integer
// operations on the bit patterns plus at most one FP64 add, so the slow FP64
// pipe is touched once per output element.  Magnitudes must stay inside the
// normal float range (|x| < 2^128); values below 2^-126 become 0.
#pragma once

#include "mm_internal.cuh"

namespace mm {

struct ff {
    float h, l;
    ff() = default;
    __host__ __device__ constexpr ff(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ constexpr ff(int v) : h((float)v), l(0.f) {}
    __host__ __device__ constexpr ff(float v) : h(v), l(0.f) {}
    // rounding split of a double (d - h is exact in double); folded at
    // compile time for constants (runtime data goes through d2ff, which
    // needs no FP64 arithmetic)
    __host__ __device__ constexpr ff(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
};

struct ffc {
    ff x, y;
};
template <> struct cx<ff> { using type = ffc; };

// Every step uses an explicit round-to-nearest intrinsic: the compiler must
// not contract a product into a following add (the error-free
// transformations depend on each step being rounded on its own).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    const float s = __fadd_rn(a.h, b.h);
    const float v = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v)), __fadd_rn(a.l, b.l));
    return fast_two_sum(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.h, -a.l); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}
// a sign (+1 or -1) times a value: exact
__device__ __forceinline__ ff operator*(int s, ff a) { return s >= 0 ? a : -a; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }

// double -> ff without FP64 arithmetic: h keeps the leading 24 significant
// bits (truncated), l the next 29 bits rounded to a float
__device__ __forceinline__ ff d2ff(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned e = (hi >> 20) & 0x7ffu;             // biased exponent
    if (e <= 896u) return ff(0.f, 0.f);                  // below the float range (or zero)
    const unsigned sign = hi & 0x80000000u;
    const float h = __uint_as_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    float l = 0.f;
    if (e > 948u) {
        // remainder r * 2^(e - 1075), r < 2^29
        l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((e - 948u) << 23));
        if (sign) l = -l;
    }
    return ff(h, l);
}

// float -> double, exact, by bits (zero and subnormal floats give 0)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
__device__ __forceinline__ double ff2d(ff a) { return __dadd_rn(f2d_bits(a.h), f2d_bits(a.l)); }

// complex conversions used at the boundary of the FP64 passes
template <typename C> __device__ __forceinline__ C from_d2(double2 d);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 d) { return d; }
template <> __device__ __forceinline__ ffc from_d2<ffc>(double2 d) { return ffc{d2ff(d.x), d2ff(d.y)}; }
template <typename C> __device__ __forceinline__ C from_real(double d);
template <> __device__ __forceinline__ double from_real<double>(double d) { return d; }
template <> __device__ __forceinline__ ff from_real<ff>(double d) { return d2ff(d); }
__device__ __forceinline__ double to_d(double a) { return a; }
__device__ __forceinline__ double to_d(ff a) { return ff2d(a); }
__device__ __forceinline__ float to_d(float a) { return a; }

}  // namespace mm
