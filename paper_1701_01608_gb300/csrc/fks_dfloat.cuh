// fks_dfloat.cuh -- double-float numbers: the unevaluated sum hi + lo of two FP32 values
// (|lo| <= ulp(hi) / 2 after every operation), about 48 significant bits carried on the FP32
// pipes.  The arithmetic is built from error-free transformations: Knuth's two-sum (six
// roundings), Dekker's fast two-sum (|a| >= |b|, three roundings) and the product error by one
// fused multiply-add; the sum adds the lo parts before one renormalisation (error below
// 2^-44 (|a| + |b|), the normwise bound a transform needs).  Used as the arithmetic type of the
// collision kernel's last escalation tier: FP64 accuracy for the cells near equilibrium at a
// fraction of the cost of GB300's FP64 pipe.
//
// Host and device: the device uses round-to-nearest intrinsics (no contraction into FMAs, which
// would break the error-free transformations), the host plain IEEE float operations (compile it
// with contraction off).
#pragma once
#include <cmath>
#include <cuda_runtime.h>

#include "fks_fft.cuh"

#if defined(__CUDACC__)
#define FKS_DD_HD __host__ __device__ __forceinline__
#else
#define FKS_DD_HD inline
#endif

namespace fks {

#ifdef __CUDA_ARCH__
#define FKS_DADD(a, b) __fadd_rn(a, b)
#define FKS_DSUB(a, b) __fsub_rn(a, b)
#define FKS_DMUL(a, b) __fmul_rn(a, b)
#else
#define FKS_DADD(a, b) ((float)((a) + (b)))
#define FKS_DSUB(a, b) ((float)((a) - (b)))
#define FKS_DMUL(a, b) ((float)((a) * (b)))
#endif

// s + e = a + b exactly (any a, b)
FKS_DD_HD float2 dd_two_sum(float a, float b) {
    const float s = FKS_DADD(a, b);
    const float bb = FKS_DSUB(s, a);
    const float e = FKS_DADD(FKS_DSUB(a, FKS_DSUB(s, bb)), FKS_DSUB(b, bb));
    return make_float2(s, e);
}
// s + e = a + b exactly if |a| >= |b| (or a = 0)
FKS_DD_HD float2 dd_fast_two_sum(float a, float b) {
    const float s = FKS_DADD(a, b);
    const float e = FKS_DSUB(b, FKS_DSUB(s, a));
    return make_float2(s, e);
}

// The operations are hidden friends (found by argument-dependent lookup only), so that they do not
// hide the float and double overloads of fma and isfinite in the code that includes this header.
struct dfloat {
    float hi, lo;
    dfloat() = default;
    constexpr FKS_DD_HD dfloat(float h, float l) : hi(h), lo(l) {}
    constexpr FKS_DD_HD dfloat(float f) : hi(f), lo(0.0f) {}
    constexpr FKS_DD_HD dfloat(int i) : hi((float)i), lo(0.0f) {}
    // the nearest float and the rounding error of that conversion, rounded: 48 of the 53 bits
    constexpr FKS_DD_HD dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    explicit constexpr FKS_DD_HD operator double() const { return (double)hi + (double)lo; }
    explicit FKS_DD_HD operator float() const { return FKS_DADD(hi, lo); }

    friend FKS_DD_HD dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
    friend FKS_DD_HD dfloat operator+(dfloat a, dfloat b) {
        const float2 s = dd_two_sum(a.hi, b.hi);
        const float e = FKS_DADD(s.y, FKS_DADD(a.lo, b.lo));
        const float2 r = dd_fast_two_sum(s.x, e);
        return dfloat(r.x, r.y);
    }
    friend FKS_DD_HD dfloat operator-(dfloat a, dfloat b) { return a + dfloat(-b.hi, -b.lo); }
    friend FKS_DD_HD dfloat operator*(dfloat a, dfloat b) {
        const float p = FKS_DMUL(a.hi, b.hi);
        float e = fmaf(a.hi, b.hi, -p);   // exact: p + e = a.hi b.hi
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        const float2 r = dd_fast_two_sum(p, e);
        return dfloat(r.x, r.y);
    }
    // sum without the final renormalisation (|lo| up to ulp(hi) + |a.lo| + |b.lo|): for a sum whose
    // only use is another sum, which renormalises (the normwise error bound is unchanged in order)
    friend FKS_DD_HD dfloat add_lazy(dfloat a, dfloat b) {
        const float2 s = dd_two_sum(a.hi, b.hi);
        return dfloat(s.x, FKS_DADD(s.y, FKS_DADD(a.lo, b.lo)));
    }
    friend FKS_DD_HD dfloat sub_lazy(dfloat a, dfloat b) { return add_lazy(a, dfloat(-b.hi, -b.lo)); }
    friend FKS_DD_HD dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
    friend FKS_DD_HD dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
    friend FKS_DD_HD dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
    // a b + c (one product, one sum)
    friend FKS_DD_HD dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }
    friend FKS_DD_HD bool isfinite(dfloat a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }
};

// a b + c d with one renormalisation: the two high products and their exact errors, one two-sum of
// the products, the cross terms of the low parts by FMA (19 operations against 25 for two products
// and a sum; the dropped low-by-low terms are below 2^-46 of |a b| + |c d|)
FKS_DD_HD dfloat dd_dot2(dfloat a, dfloat b, dfloat c, dfloat d) {
    const float p1 = FKS_DMUL(a.hi, b.hi), p2 = FKS_DMUL(c.hi, d.hi);
    const float e1 = fmaf(a.hi, b.hi, -p1), e2 = fmaf(c.hi, d.hi, -p2);
    const float2 s = dd_two_sum(p1, p2);
    float t = FKS_DADD(s.y, FKS_DADD(e1, e2));
    t = fmaf(a.hi, b.lo, t);
    t = fmaf(a.lo, b.hi, t);
    t = fmaf(c.hi, d.lo, t);
    t = fmaf(c.lo, d.hi, t);
    const float2 r = dd_fast_two_sum(s.x, t);
    return dfloat(r.x, r.y);
}

// complex product of double-float pairs by two fused dot products (overload of cmul in fks_fft.cuh,
// found by argument-dependent lookup in the transforms)
FKS_DD_HD cpx<dfloat> cmul(cpx<dfloat> a, cpx<dfloat> b) {
    return {dd_dot2(a.x, b.x, -a.y, b.y), dd_dot2(a.x, b.y, a.y, b.x)};
}

template <> struct costly_mul<dfloat> { static constexpr bool value = true; };

#undef FKS_DADD
#undef FKS_DSUB
#undef FKS_DMUL

}  // namespace fks
