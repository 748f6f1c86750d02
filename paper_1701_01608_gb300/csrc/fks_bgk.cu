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

// One CTA of BS = 2N^2/V... threads per cell, organised as rows of N/V lanes:
// lane group t owns velocity indices z0 .. z0+V-1 (V = 16 bytes / sizeof T)
// and the rows (x, y) = t / (N/V) + RPI j.  Where the thread's V source
// elements are contiguous (the usual case) they move as one 16-byte access.
// Two passes over the cell: moments, then output; the projection sums of
// Q = nu (M - f) need no pass (M is a product of one-axis factors).  The
// second read and the output use evict-first hints, so that they do not push
// out of L2 the cells still waiting for their second pass.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
};
template <>
struct Vec<double> {
    using type = double2;
};

template <typename T, int N, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) bgk_kernel(BgkArgs a) {
    constexpr int V = 16 / (int)sizeof(T);          // elements per 16-byte access
    constexpr int LPR = N / V;                       // lanes per row
    constexpr int RPI = BS / LPR;                    // rows per iteration
    constexpr int ROWS = (N * N + RPI - 1) / RPI;    // iterations
    constexpr int N3 = N * N * N;
    using VT = typename Vec<T>::type;
    __shared__ double red[BS / 32][5];
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
    const bool lane_ok = tid < LPR * RPI;
    const int z0 = (tid % LPR) * V, r0 = tid / LPR;

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

    for (long cell = a.cell0 + blockIdx.x; cell < a.ncells; cell += gridDim.x) {
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
        // this thread's V source offsets along z, and whether they are one aligned run
        long zo[V];
        bool vec = true;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            zo[k] = src_z[z0 + k];
            vec &= zo[k] == zo[0] + k;
        }
        vec &= (zo[0] % V) == 0;
        T vz[V];
#pragma unroll
        for (int k = 0; k < V; ++k) vz[k] = vgT[z0 + k];
        auto row_base = [&](int r) -> long { return src_x[r / N] + src_y[r % N]; };
        auto load_run = [&](long rb, T (&v)[V], bool last) {
            if (vec) {
                const VT* pv = reinterpret_cast<const VT*>(fin + rb + zo[0]);
                const VT w = last ? __ldcs(pv) : *pv;
                const T* pw = reinterpret_cast<const T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = pw[k];
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = last ? __ldcs(fin + rb + zo[k]) : fin[rb + zo[k]];
            }
        };
        // pass 1: moments (per-thread partials in T, block sums in FP64)
        {
            T s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
            if (lane_ok) {
#pragma unroll 4
                for (int j = 0; j < ROWS; ++j) {
                    const int r = r0 + RPI * j;
                    if (r >= N * N) break;
                    T v[V];
                    load_run(row_base(r), v, false);
                    const T vx = vgT[r / N], vy = vgT[r % N];
                    T sr = 0, sz = 0, szz = 0;
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        sr += v[k];
                        sz += v[k] * vz[k];
                        szz += v[k] * vz[k] * vz[k];
                    }
                    s0 += sr;
                    s1 += sr * vx;
                    s2 += sr * vy;
                    s3 += sz;
                    s4 += sr * (vx * vx + vy * vy) + szz;
                }
            }
            double s[5] = {(double)s0, (double)s1, (double)s2, (double)s3, 0.5 * (double)s4};
            block_sum5(s);
        }
        if (tid < N) {
            // cell moments and the Maxwellian's one-axis factors (in T)
            const double dv3 = dv * dv * dv;
            const double rho = cell5[0] * dv3;
            const double ux = cell5[1] * dv3 / rho, uy = cell5[2] * dv3 / rho, uz = cell5[3] * dv3 / rho;
            const double Tt = (cell5[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
            const T A = (T)(rho / (2.0 * 3.14159265358979323846 * Tt * sqrt(2.0 * 3.14159265358979323846 * Tt)));
            const T i2T = (T)(0.5 / Tt);
            const T dx = vgT[tid] - (T)ux, dy = vgT[tid] - (T)uy, dz = vgT[tid] - (T)uz;
            gx[tid] = A * exp(-dx * dx * i2T);
            gy[tid] = exp(-dy * dy * i2T);
            gz[tid] = exp(-dz * dz * i2T);
        }
        __syncthreads();
        if (tid < 32) {
            // one-axis sums of g, v g, v^2 g (of the stored factors) by warp 0, then the
            // Maxwellian's moment sums, sum phi Q = nu (sum phi M - sum phi f) and mu = P sum phi Q
            T acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = tid; i < N; i += 32) {
                const T v = vgT[i];
                const T g0 = gx[i], g1 = gy[i], g2 = gz[i];
                acc[0] += g0; acc[1] += v * g0; acc[2] += v * v * g0;
                acc[3] += g1; acc[4] += v * g1; acc[5] += v * v * g1;
                acc[6] += g2; acc[7] += v * g2; acc[8] += v * v * g2;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
            if (tid < 6) {
                double X[3], Y[3], Z[3];
                for (int k = 0; k < 3; ++k) {
                    X[k] = (double)acc[k];
                    Y[k] = (double)acc[3 + k];
                    Z[k] = (double)acc[6 + k];
                }
                const double dv3 = dv * dv * dv;
                const double nu = cell5[0] * dv3 * a.inv_kn;
                const double sM[5] = {X[0] * Y[0] * Z[0], X[1] * Y[0] * Z[0], X[0] * Y[1] * Z[0], X[0] * Y[0] * Z[1],
                                      0.5 * (X[2] * Y[0] * Z[0] + X[0] * Y[2] * Z[0] + X[0] * Y[0] * Z[2])};
                if (tid < 5) {
                    double m = 0.0;
                    for (int j = 0; j < 5; ++j) m += a.P[tid * 5 + j] * nu * (sM[j] - cell5[j]);
                    mu[tid] = m;
                } else {
                    mu[5] = nu;
                }
            }
        }
        __syncthreads();
        // pass 2: corrected Q = nu (M - f) - phi.mu, output
        if (lane_ok) {
            const T tnu = (T)mu[5];
            const T m0 = (T)mu[0], m1 = (T)mu[1], m2 = (T)mu[2], m3 = (T)mu[3], m4 = (T)mu[4];
            T gzz[V], czz[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                gzz[k] = gz[z0 + k];
                czz[k] = m3 * vz[k] + (T)0.5 * m4 * vz[k] * vz[k];
            }
            const T tdt = (T)a.dt;
            const bool heun = a.mode == 3;
            const bool stepm = a.mode == 1 || heun;
            T* oc = fout + cell * N3 + z0;
            const T* bc = static_cast<const T*>(a.base) + cell * N3 + z0;   // Heun: base, read before the store
            bool bad = false, neg = false;
#pragma unroll 4
            for (int j = 0; j < ROWS; ++j) {
                const int r = r0 + RPI * j;
                if (r >= N * N) break;
                T v[V];
                load_run(row_base(r), v, true);
                const T vx = vgT[r / N], vy = vgT[r % N];
                const T gxy = gx[r / N] * gy[r % N];
                const T cxy = m0 + m1 * vx + m2 * vy + (T)0.5 * m4 * (vx * vx + vy * vy);
                T o[V], b[V];
                if (heun) {
                    const VT w = *reinterpret_cast<const VT*>(bc + (long)r * N);
                    const T* pw = reinterpret_cast<const T*>(&w);
#pragma unroll
                    for (int k = 0; k < V; ++k) b[k] = pw[k];
                }
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T q = tnu * (gxy * gzz[k] - v[k]) - (cxy + czz[k]);
                    o[k] = stepm ? v[k] + tdt * q : q;
                    if (heun) o[k] = (T)0.5 * (o[k] + b[k]);
                    bad |= !isfinite(o[k]);
                    neg |= stepm && o[k] < T(0);
                }
                VT w;
                T* pw = reinterpret_cast<T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) pw[k] = o[k];
                __stcs(reinterpret_cast<VT*>(oc + (long)r * N), w);
            }
            if (bad) atomicOr(a.flags, 1);
            if (neg) atomicOr(a.flags, 2);
        }
    }
}

template <typename T, int N>
static cudaError_t launch_n(const BgkArgs& a, cudaStream_t s) {
    // 128-thread CTAs, eight resident per SM (registers); two waves of them
    // (measured: 16 per SM 3.24 ms, 6 per SM 3.68 ms, 4 per SM 4.43 ms at 32^3 x 32^3)
    constexpr int BS = N >= 16 ? 128 : 256;
    const long cells = a.ncells - a.cell0;
    long grid = cells < 152L * 16 ? cells : 152L * 16;
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
