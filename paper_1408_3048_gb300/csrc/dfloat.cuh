// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits.  The FP64 refinement residual of
// the mixed solver runs its overlap-save FFT in this arithmetic on the FP32 pipe, which
// GB300 runs at 64 times its FP64 rate.
//
// The operations are the classical error-free transformations: Knuth's two-sum (the
// rounding error of a + b recovered exactly by six additions), Dekker's fast two-sum
// (three additions when |a| >= |b|) and the exact product error fma(a, b, -ab).  Sums
// follow Dekker's double-length addition (two-sum of the high parts, low parts added,
// renormalised): its error is a few units of 2^-48 relative to |a| + |b|, the norm-wise
// bound an FFT's error analysis uses.  The _rn intrinsics keep the compiler from
// contracting or reassociating the transformations.
#pragma once

#include <cuda_runtime.h>

namespace mm {

struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (hi = d rounded to FP32, lo = the rest rounded)
    __host__ __device__ explicit dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfl df_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return dfl(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_renorm(s, e);
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_renorm(p, e);
}

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) {
    a = a + b;
    return a;
}

struct dfl2 {
    dfl x, y;
};

// Conversions between double and double-float by bit operations.  FP64 instructions,
// conversions included, issue at 1/64 of the FP32 rate on this GPU, and the residual
// kernel converts every sample on the way in and every output on the way out.
// dfl_from_double: hi = d with its significand cut to 24 bits (exactly a float for the
// exponents kept here), lo = the remaining 29 bits rounded to a float, then renormalised;
// |d| below 2^-74 or above 2^127 and non-finite d take the FP64 route.  f64_from_f32 widens
// a normal float or a zero exactly (subnormal and non-finite floats take the FP64 route),
// so dfl_to_double equals (double)hi + (double)lo.
__device__ __forceinline__ dfl dfl_from_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);   // biased exponent
    if (e < 949 || e > 1150) return dfl(d);
    const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(s | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    const unsigned m = (unsigned)(b & 0x1fffffffu);   // lo = m 2^(e - 1075)
    float lo = 0.f;
    if (m != 0u) lo = __int_as_float(__float_as_int(__uint2float_rn(m)) + (e - 1075) * (1 << 23));
    return df_renorm(hi, __uint_as_float(__float_as_uint(lo) | s));
}

__device__ __forceinline__ double f64_from_f32(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned E = (u >> 23) & 0xffu;
    if (E == 0u || E == 255u) {
        if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
        return (double)f;
    }
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(E + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ double dfl_to_double(dfl v) { return f64_from_f32(v.hi) + f64_from_f32(v.lo); }

}  // namespace mm
