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

}  // namespace mm
