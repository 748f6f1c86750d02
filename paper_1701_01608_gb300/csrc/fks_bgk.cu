// fks_bgk.cu -- BGK relaxation collision step (Sec. 2, BGK approximation,
// and the BGK variant of the FKS in Sec. 3) with the transport gather fused
// into its loads:
//   f*  = gather of f over the transport shifts (identity for collide)
//   U   = moments of f*, M = Maxwellian of U at the grid points
//   Q   = nu (M - f*), nu = rho / Kn, then the conservation projection
//   out = Q  or  f* + dt Q
// One CTA per cell (persistent over cells).  HBM bound: f is read from DRAM
// once, the second pass over the cell hits L2, and out is written once.
#include <cuda_runtime.h>

#include "fks_internal.h"

namespace fks {

// One CTA of BS = 8N threads per cell: thread t owns velocity index z = t % N
// and the rows (x, y) = t / N + 8 j, so its z-part of the gather offset and of
// the velocity is fixed.  Two passes over the cell: moments, then output.  The
// projection sums of Q = nu (M - f) need no pass: M is a product of one-axis
// factors, so sum phi M follows from one-axis sums, and sum phi f is pass 1.
template <typename T, int N>
__global__ void __launch_bounds__(8 * N, 1024 / (8 * N)) bgk_kernel(BgkArgs a) {
    constexpr int BS = 8 * N;
    constexpr int N3 = N * N * N;
    constexpr int ROWS = N * N / 8;   // rows per thread
    __shared__ double red[(BS + 31) / 32][5];
    __shared__ double cell5[8];
    __shared__ double mu[8];
    __shared__ long src_x[N], src_y[N], src_z[N];   // element offsets of the source pieces
    __shared__ T gx[N], gy[N], gz[N];               // one-axis Maxwellian factors (gx carries rho (2 pi T)^-3/2)
    __shared__ T vgT[N];
    __shared__ double vg[N];
    __shared__ signed char dsm[3 * N];

    const int tid = threadIdx.x;
    const T* __restrict__ fin = static_cast<const T*>(a.f);
    T* __restrict__ fout = static_cast<T*>(a.out);
    const bool transport = a.delta != nullptr;
    const double dv = 2.0 * a.L / N;
    for (int i = tid; i < N; i += BS) {
        vg[i] = ((double)i + 0.5 - 0.5 * N) * dv;
        vgT[i] = (T)vg[i];
    }
    for (int i = tid; i < 3 * N; i += BS) dsm[i] = transport ? a.delta[i] : 0;
    const int ncx = a.nc[0], ncy = a.nc[1], ncz = a.nc[2];
    const int z = tid % N, r0 = tid / N;

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
            for (int w = 0; w < (BS + 31) / 32; ++w) acc += red[w][tid];
            cell5[tid] = acc;
        }
        __syncthreads();
    };

    for (long cell = blockIdx.x; cell < a.ncells; cell += gridDim.x) {
        const int cx = (int)(cell / ((long)ncy * ncz));
        const int cy = (int)((cell / ncz) % ncy);
        const int cz = (int)(cell % ncz);
        __syncthreads();   // the previous cell's readers of the shared tables are done
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
        const T* fz = fin + src_z[z];
        const T vz = vgT[z];
        // pass 1: moments (per-thread partials in T, block sums in FP64)
        {
            T s0 = 0, s1 = 0, s2 = 0, s4 = 0;
#pragma unroll 8
            for (int j = 0; j < ROWS; ++j) {
                const int r = r0 + 8 * j, x = r / N, y = r % N;
                const T fv = fz[src_x[x] + src_y[y]];
                const T vx = vgT[x], vy = vgT[y];
                s0 += fv;
                s1 += fv * vx;
                s2 += fv * vy;
                s4 += fv * (vx * vx + vy * vy);
            }
            double s[5] = {(double)s0, (double)s1, (double)s2, (double)vz * (double)s0,
                           0.5 * ((double)s4 + (double)vz * (double)vz * (double)s0)};
            block_sum5(s);
        }
        if (tid < N) {
            // cell moments, Maxwellian factors, projection coefficients
            const double dv3 = dv * dv * dv;
            const double rho = cell5[0] * dv3;
            const double ux = cell5[1] * dv3 / rho, uy = cell5[2] * dv3 / rho, uz = cell5[3] * dv3 / rho;
            const double Tt = (cell5[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
            const double A = rho * pow(2.0 * 3.14159265358979323846 * Tt, -1.5);
            const double dx = vg[tid] - ux, dy = vg[tid] - uy, dz = vg[tid] - uz;
            gx[tid] = (T)(A * exp(-dx * dx / (2.0 * Tt)));
            gy[tid] = (T)exp(-dy * dy / (2.0 * Tt));
            gz[tid] = (T)exp(-dz * dz / (2.0 * Tt));
        }
        __syncthreads();
        if (tid < 32) {
            // one-axis sums of g, v g, v^2 g (of the stored factors) by warp 0, then the
            // Maxwellian's moment sums, sum phi Q = nu (sum phi M - sum phi f) and mu = P sum phi Q
            double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = tid; i < N; i += 32) {
                const double v = vg[i];
                const double g0 = (double)gx[i], g1 = (double)gy[i], g2 = (double)gz[i];
                acc[0] += g0; acc[1] += v * g0; acc[2] += v * v * g0;
                acc[3] += g1; acc[4] += v * g1; acc[5] += v * v * g1;
                acc[6] += g2; acc[7] += v * g2; acc[8] += v * v * g2;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
            const double *X = acc, *Y = acc + 3, *Z = acc + 6;
            const double dv3 = dv * dv * dv;
            const double nu = cell5[0] * dv3 * a.inv_kn;
            const double sM[5] = {X[0] * Y[0] * Z[0], X[1] * Y[0] * Z[0], X[0] * Y[1] * Z[0], X[0] * Y[0] * Z[1],
                                  0.5 * (X[2] * Y[0] * Z[0] + X[0] * Y[2] * Z[0] + X[0] * Y[0] * Z[2])};
            if (tid < 5) {
                double m = 0.0;
                for (int j = 0; j < 5; ++j) m += a.P[tid * 5 + j] * nu * (sM[j] - cell5[j]);
                mu[tid] = m;
            }
            if (tid == 5) mu[5] = nu;
        }
        __syncthreads();
        // pass 2: corrected Q = nu (M - f) - phi.mu, output
        const T tnu = (T)mu[5];
        const T m0 = (T)mu[0], m1 = (T)mu[1], m2 = (T)mu[2], m4 = (T)mu[4];
        const T cz_ = (T)(mu[3] * (double)vz + 0.5 * mu[4] * (double)vz * (double)vz);
        const T gzz = gz[z];
        const T tdt = (T)a.dt;
        const bool stepm = a.mode == 1;
        T* oz = fout + cell * N3 + z;
        bool bad = false, neg = false;
#pragma unroll 8
        for (int j = 0; j < ROWS; ++j) {
            const int r = r0 + 8 * j, x = r / N, y = r % N;
            const T fv = fz[src_x[x] + src_y[y]];
            const T vx = vgT[x], vy = vgT[y];
            const T M = gx[x] * gy[y] * gzz;
            const T corr = m0 + m1 * vx + m2 * vy + (T)0.5 * m4 * (vx * vx + vy * vy) + cz_;
            const T q = tnu * (M - fv) - corr;
            const T o = stepm ? fv + tdt * q : q;
            bad |= !isfinite(o);
            neg |= stepm && o < T(0);
            oz[(long)r * N] = o;
        }
        if (bad) atomicOr(a.flags, 1);
        if (neg) atomicOr(a.flags, 2);
    }
}

template <typename T, int N>
static cudaError_t launch_n(const BgkArgs& a, cudaStream_t s) {
    long grid = a.ncells < 152L * 16 ? a.ncells : 152L * 16;
    bgk_kernel<T, N><<<(unsigned)grid, 8 * N, 0, s>>>(a);
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
