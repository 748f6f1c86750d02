// Host harness of the compensated FP32 sums (csrc/fks_df.cuh) used by the collision epilogue,
// the moments, the single-read BGK and the variant-B truncation kernels.
#include "fks_df.cuh"

extern "C" {

// sum of x[i] as a (hi, lo) pair, then as a double
int fks_test_df_sum(const float* x, int n, double* out) {
    float2 s = make_float2(0.f, 0.f);
    for (int i = 0; i < n; ++i) s = fks::df_add1(s, x[i]);
    *out = (double)s.x + (double)s.y;
    return 0;
}

// sum of x[i] (wh[i] + wl[i]) with the exact products of the kernels
int fks_test_df_dot(const float* x, const float* wh, const float* wl, int n, double* out) {
    float2 s = make_float2(0.f, 0.f);
    for (int i = 0; i < n; ++i) {
        const float p = x[i] * wh[i];
        s = fks::df_add1(s, p);
        s.y += fmaf(x[i], wl[i], fmaf(x[i], wh[i], -p));
    }
    *out = (double)s.x + (double)s.y;
    return 0;
}

// pairwise (tree) reduction of n pairs by df_add, as the warp shuffles do
int fks_test_df_tree(const float* hi, const float* lo, int n, double* out) {
    float2 v[1024];
    if (n > 1024) return 1;
    for (int i = 0; i < n; ++i) v[i] = make_float2(hi[i], lo[i]);
    for (int w = 1; w < n; w *= 2)
        for (int i = 0; i + w < n; i += 2 * w) v[i] = fks::df_add(v[i], v[i + w]);
    *out = (double)v[0].x + (double)v[0].y;
    return 0;
}

// the same tree by two_sum_add (the single-read BGK kernel's order of the lo terms)
int fks_test_df_tree2(const float* hi, const float* lo, int n, double* out) {
    float2 v[1024];
    if (n > 1024) return 1;
    for (int i = 0; i < n; ++i) v[i] = make_float2(hi[i], lo[i]);
    for (int w = 1; w < n; w *= 2)
        for (int i = 0; i + w < n; i += 2 * w) v[i] = fks::two_sum_add(v[i], v[i + w]);
    *out = (double)v[0].x + (double)v[0].y;
    return 0;
}

// (ah + al)(bh + bl) by df_mul
int fks_test_df_mul(float ah, float al, float bh, float bl, double* out) {
    const float2 r = fks::df_mul(make_float2(ah, al), make_float2(bh, bl));
    *out = (double)r.x + (double)r.y;
    return 0;
}

}  // extern "C"
