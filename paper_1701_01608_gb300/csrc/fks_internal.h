// fks_internal.h -- declarations shared by the translation units of libfks.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "fks_collide.cuh"

namespace fks {

// One instantiation of collide_kernel<T, N, C>.
struct CollideVariant {
    const void* func;     // host stub of the kernel (cells of one problem)
    const void* func_batch;   // host stub of the batch kernel (one homogeneous problem per item)
    int N, C, NT;
    size_t smem;
    bool fp64;
};

// Look up an instantiation; returns false if (fp64, N, C) was not compiled.
bool find_collide_variant(bool fp64, int N, int C, CollideVariant* out);
bool find_collide_variant_f32(int N, int C, CollideVariant* out);
bool find_collide_variant_f64(int N, int C, CollideVariant* out);

// Arguments of the BGK relaxation kernel (fks_bgk.cu).
struct BgkArgs {
    const void* f;
    void* out;
    const signed char* delta;   // [3][n] shifts (transport) or nullptr
    int* flags;
    long ncells;
    int nc[3], bc[3];
    double L, inv_kn, dt;
    int mode;                   // 0 collide, 1 step
    double P[25];
};
cudaError_t launch_bgk(bool fp64, int n, const BgkArgs& a, cudaStream_t s);

// Default cluster size for (precision, N).
int default_cluster_size(bool fp64, int N);

}  // namespace fks
