// fks_df.cuh -- double-float (hi, lo) helpers for compensated FP32 sums: add a float, add two
// pairs (two orders of the lo terms), multiply two pairs.  Error-free transformations (two-sum
// by six roundings, two-product by FMA); the lo parts are not renormalised beyond what the sums
// need.  Host and device: the device uses round-to-nearest intrinsics (no contraction), the
// host plain IEEE float operations (compile it with contraction off).
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace fks {

#ifdef __CUDA_ARCH__
#define FKS_FADD(a, b) __fadd_rn(a, b)
#define FKS_FSUB(a, b) __fsub_rn(a, b)
#define FKS_FMUL(a, b) __fmul_rn(a, b)
#else
#define FKS_FADD(a, b) ((float)((a) + (b)))
#define FKS_FSUB(a, b) ((float)((a) - (b)))
#define FKS_FMUL(a, b) ((float)((a) * (b)))
#endif

__host__ __device__ __forceinline__ float2 df_add1(float2 a, float b) {
    const float t = FKS_FADD(a.x, b);
    const float bb = FKS_FSUB(t, a.x);
    const float e = FKS_FADD(FKS_FSUB(a.x, FKS_FSUB(t, bb)), FKS_FSUB(b, bb));
    return make_float2(t, FKS_FADD(a.y, e));
}
__host__ __device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float2 s = df_add1(a, b.x);
    return make_float2(s.x, FKS_FADD(s.y, b.y));
}
// the same pair sum with the lo parts added before the rounding error of the hi parts
__host__ __device__ __forceinline__ float2 two_sum_add(float2 x, float2 y) {
    const float t = FKS_FADD(x.x, y.x);
    const float bb = FKS_FSUB(t, x.x);
    const float e = FKS_FADD(FKS_FSUB(x.x, FKS_FSUB(t, bb)), FKS_FSUB(y.x, bb));
    return make_float2(t, FKS_FADD(FKS_FADD(x.y, y.y), e));
}
__host__ __device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = FKS_FMUL(a.x, b.x);
    const float e = fmaf(a.x, b.x, -p);
    return make_float2(p, fmaf(a.x, b.y, fmaf(a.y, b.x, e)));
}

#undef FKS_FADD
#undef FKS_FSUB
#undef FKS_FMUL

}  // namespace fks
