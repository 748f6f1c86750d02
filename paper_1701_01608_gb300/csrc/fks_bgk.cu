// fks_bgk.cu -- BGK relaxation collision step (Sec. 2, BGK approximation,
// and the BGK variant of the FKS in Sec. 3) with the transport gather fused
// into its loads:
//   f*  = gather of f over the transport shifts (identity for collide)
//   U   = moments of f*, M = Maxwellian of U at the grid points
//   Q   = nu (M - f*), nu = rho / Kn, then the conservation projection
//   out = Q  or  f* + dt Q
// One CTA per cell (persistent over cells).  HBM bound: f is read from DRAM
// once, the two later passes over the cell hit L2, and out is written once.
#include <cuda_runtime.h>

#include "fks_internal.h"

namespace fks {

template <typename T, int N, int BS>
__global__ void __launch_bounds__(BS) bgk_kernel(BgkArgs a) {
    constexpr int N3 = N * N * N;
    constexpr int PER = (N3 + BS - 1) / BS;
    using Acc = T;   // per-thread partial sums (FP64 in FP64 mode); block sums in FP64
    __shared__ double red[BS / 32][5];
    __shared__ double cell5[8];
    __shared__ long src_x[N], src_y[N], src_z[N];   // element offsets of the source row pieces
    __shared__ T ex[N], ey[N], ez[N];               // separable Maxwellian factors
    __shared__ double vg[N];
    __shared__ signed char dsm[3 * N];

    const int tid = threadIdx.x;
    const T* __restrict__ fin = static_cast<const T*>(a.f);
    T* __restrict__ fout = static_cast<T*>(a.out);
    const bool transport = a.delta != nullptr;
    const double dv = 2.0 * a.L / N;
    for (int i = tid; i < N; i += BS) vg[i] = ((double)i + 0.5 - 0.5 * N) * dv;
    for (int i = tid; i < 3 * N; i += BS) dsm[i] = transport ? a.delta[i] : 0;
    const int ncx = a.nc[0], ncy = a.nc[1], ncz = a.nc[2];

    auto block_sum5 = [&](double (&s)[5]) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], off);
        if ((tid & 31) == 0)
            for (int i = 0; i < 5; ++i) red[tid >> 5][i] = s[i];
        __syncthreads();
        if (tid < 5) {
            double acc = 0.0;
            for (int w = 0; w < BS / 32; ++w) acc += red[w][tid];
            cell5[tid] = acc;
        }
        __syncthreads();
    };

    for (long cell = blockIdx.x; cell < a.ncells; cell += gridDim.x) {
        const int cx = (int)(cell / ((long)ncy * ncz));
        const int cy = (int)((cell / ncz) % ncy);
        const int cz = (int)(cell % ncz);
        __syncthreads();   // previous cell's readers of the row tables are done
        // source offsets along each axis: cell part * N^3 + velocity part
        for (int i = tid; i < 3 * N; i += BS) {
            const int ax = i / N, k = i % N;
            const int c0 = ax == 0 ? cx : (ax == 1 ? cy : cz);
            const int len = ax == 0 ? ncx : (ax == 1 ? ncy : ncz);
            int fl = 0;
            const int sc = transport ? fold_cell(c0 - dsm[i], len, a.bc[ax], fl) : c0;
            const int q = fl ? N - 1 - k : k;
            if (ax == 0) src_x[k] = (long)sc * ncy * ncz * N3 + (long)q * N * N;
            else if (ax == 1) src_y[k] = (long)sc * ncz * N3 + (long)q * N;
            else src_z[k] = (long)sc * N3 + q;
        }
        __syncthreads();
        auto load = [&](int e) -> T {
            const int x = e / (N * N), y = (e / N) % N, z = e % N;
            return fin[src_x[x] + src_y[y] + src_z[z]];
        };
        // pass 1: moments
        {
            Acc s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll 4
            for (int j = 0; j < PER; ++j) {
                const int e = tid + j * BS;
                if (e >= N3) break;
                const T fv = load(e);
                const int x = e / (N * N), y = (e / N) % N, z = e % N;
                const T vx = (T)vg[x], vy = (T)vg[y], vz = (T)vg[z];
                s0 += fv;
                s1 += fv * vx;
                s2 += fv * vy;
                s3 += fv * vz;
                s4 += fv * (T)0.5 * (vx * vx + vy * vy + vz * vz);
            }
            double s[5] = {(double)s0, (double)s1, (double)s2, (double)s3, (double)s4};
            block_sum5(s);
        }
        const double dv3 = dv * dv * dv;
        const double rho = cell5[0] * dv3;
        const double ux = cell5[1] * dv3 / rho, uy = cell5[2] * dv3 / rho, uz = cell5[3] * dv3 / rho;
        const double Tt = (cell5[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
        const double nu = rho * a.inv_kn;
        __syncthreads();
        for (int i = tid; i < 3 * N; i += BS) {
            const int ax = i / N, k = i % N;
            const double u = ax == 0 ? ux : (ax == 1 ? uy : uz);
            const double d = vg[k] - u;
            const double g = exp(-d * d / (2.0 * Tt));
            (ax == 0 ? ex : (ax == 1 ? ey : ez))[k] = (T)(ax == 0 ? rho * pow(2.0 * 3.14159265358979323846 * Tt, -1.5) * g : g);
        }
        __syncthreads();
        const T tnu = (T)nu;
        auto qval = [&](int e, T fv) -> T {
            const int x = e / (N * N), y = (e / N) % N, z = e % N;
            return tnu * (ex[x] * ey[y] * ez[z] - fv);
        };
        // pass 2: projection sums of Q
        {
            Acc s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll 4
            for (int j = 0; j < PER; ++j) {
                const int e = tid + j * BS;
                if (e >= N3) break;
                const T q = qval(e, load(e));
                const int x = e / (N * N), y = (e / N) % N, z = e % N;
                const T vx = (T)vg[x], vy = (T)vg[y], vz = (T)vg[z];
                s0 += q;
                s1 += q * vx;
                s2 += q * vy;
                s3 += q * vz;
                s4 += q * (T)0.5 * (vx * vx + vy * vy + vz * vz);
            }
            double s[5] = {(double)s0, (double)s1, (double)s2, (double)s3, (double)s4};
            block_sum5(s);
        }
        double mu[5];
        for (int i = 0; i < 5; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 5; ++j) acc += a.P[i * 5 + j] * cell5[j];
            mu[i] = acc;
        }
        // pass 3: corrected Q, output
        const T m0 = (T)mu[0], m1 = (T)mu[1], m2 = (T)mu[2], m3 = (T)mu[3], m4 = (T)mu[4];
        const T tdt = (T)a.dt;
        bool bad = false, neg = false;
#pragma unroll 4
        for (int j = 0; j < PER; ++j) {
            const int e = tid + j * BS;
            if (e >= N3) break;
            const T fv = load(e);
            const int x = e / (N * N), y = (e / N) % N, z = e % N;
            const T vx = (T)vg[x], vy = (T)vg[y], vz = (T)vg[z];
            const T q = qval(e, fv) - (m0 + m1 * vx + m2 * vy + m3 * vz + m4 * (T)0.5 * (vx * vx + vy * vy + vz * vz));
            const T o = a.mode == 1 ? fv + tdt * q : q;
            bad |= !isfinite(o);
            neg |= a.mode == 1 && o < T(0);
            fout[cell * N3 + e] = o;
        }
        if (bad) atomicOr(a.flags, 1);
        if (neg) atomicOr(a.flags, 2);
    }
}

template <typename T, int N>
static cudaError_t launch_n(const BgkArgs& a, cudaStream_t s) {
    constexpr int BS = 256;
    long grid = a.ncells < 152L * 8 ? a.ncells : 152L * 8;
    bgk_kernel<T, N, BS><<<(unsigned)grid, BS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bgk(bool fp64, int n, const BgkArgs& a, cudaStream_t s) {
    if (fp64) {
        switch (n) {
            case 8: return launch_n<double, 8>(a, s);
            case 16: return launch_n<double, 16>(a, s);
            case 24: return launch_n<double, 24>(a, s);
            case 32: return launch_n<double, 32>(a, s);
        }
    } else {
        switch (n) {
            case 8: return launch_n<float, 8>(a, s);
            case 16: return launch_n<float, 16>(a, s);
            case 24: return launch_n<float, 24>(a, s);
            case 32: return launch_n<float, 32>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace fks
