// Host harness of the double-float arithmetic (csrc/fks_dfloat.cuh) of the collision kernel's
// last escalation tier: one sum or product of two pairs, or the fused a b + c d of four, returned as
// its (hi, lo) floats.
#include "fks_dfloat.cuh"

extern "C" {

int fks_test_dd_add(float ahi, float alo, float bhi, float blo, float* out) {
    const fks::dfloat r = fks::dfloat(ahi, alo) + fks::dfloat(bhi, blo);
    out[0] = r.hi;
    out[1] = r.lo;
    return 0;
}

int fks_test_dd_mul(float ahi, float alo, float bhi, float blo, float* out) {
    const fks::dfloat r = fks::dfloat(ahi, alo) * fks::dfloat(bhi, blo);
    out[0] = r.hi;
    out[1] = r.lo;
    return 0;
}

// a b + c d by the fused dot product (the real part of the complex product)
int fks_test_dd_dot2(const float* abcd, float* out) {
    const fks::dfloat r = fks::dd_dot2(fks::dfloat(abcd[0], abcd[1]), fks::dfloat(abcd[2], abcd[3]),
                                       fks::dfloat(abcd[4], abcd[5]), fks::dfloat(abcd[6], abcd[7]));
    out[0] = r.hi;
    out[1] = r.lo;
    return 0;
}

// (a + b) + (c - d) with the two inner sums left unnormalised (the first level of a radix-4 butterfly)
int fks_test_dd_lazy4(const float* abcd, float* out) {
    const fks::dfloat a(abcd[0], abcd[1]), b(abcd[2], abcd[3]), c(abcd[4], abcd[5]), d(abcd[6], abcd[7]);
    const fks::dfloat r = add_lazy(a, b) + sub_lazy(c, d);
    out[0] = r.hi;
    out[1] = r.lo;
    return 0;
}

int fks_test_dd_from_double(double d, float* out) {
    const fks::dfloat r(d);
    out[0] = r.hi;
    out[1] = r.lo;
    return 0;
}

}  // extern "C"
