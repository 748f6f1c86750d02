// fks_bgk.cu -- BGK relaxation collision step (Sec. 2, BGK approximation,
// and the BGK variant of the FKS in Sec. 3) with the transport gather fused
// into its loads:
//   f*  = gather of f over the transport shifts (identity for collide)
//   U   = moments of f*, M = Maxwellian of U at the grid points
//   Q   = nu (M - f*), nu = rho / Kn, then the conservation projection
//   out = Q  or  f* + dt Q
// HBM bound.  FP32 n = 32: one cell per cluster of 4 CTAs holding the cell in
// registers (f* read once, out written once).  Other cases: one CTA per cell
// (persistent over cells), two passes whose second one mostly hits L2.
#include <cuda_runtime.h>

#include "fks_df.cuh"
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
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
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
            // cell moments and the Maxwellian's one-axis factors (in T); no Maxwellian exists
            // for rho <= 0 or T <= 0 (vacuum, degenerate cells): then M = 0 and nu = 0, Q = 0
            const double dv3 = dv * dv * dv;
            const double rho = cell5[0] * dv3;
            double ux = cell5[1] * dv3 / rho, uy = cell5[2] * dv3 / rho, uz = cell5[3] * dv3 / rho;
            double Tt = (cell5[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
            const bool ok = rho > 0.0 && Tt > 0.0;
            if (!ok) ux = uy = uz = 0.0, Tt = 1.0;
            const T A = ok ? (T)(rho / (2.0 * 3.14159265358979323846 * Tt * sqrt(2.0 * 3.14159265358979323846 * Tt)))
                           : T(0);
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
                const bool live = X[0] > 0.0;   // A > 0: the cell has a Maxwellian
                const double nu = live ? cell5[0] * dv3 * a.inv_kn : 0.0;
                const double sM[5] = {X[0] * Y[0] * Z[0], X[1] * Y[0] * Z[0], X[0] * Y[1] * Z[0], X[0] * Y[0] * Z[1],
                                      0.5 * (X[2] * Y[0] * Z[0] + X[0] * Y[2] * Z[0] + X[0] * Y[0] * Z[2])};
                if (tid < 5) {
                    double m = 0.0;
                    for (int j = 0; j < 5; ++j) m += a.P[tid * 5 + j] * nu * (sM[j] - cell5[j]);
                    mu[tid] = m;
                } else {
                    mu[5] = nu;
                    // mode 4: exponential step weight (1 - e^{-nu dt}) / nu (dt as nu -> 0)
                    if (a.mode == 4) mu[6] = nu > 0.0 ? -expm1(-nu * a.dt) / nu : a.dt;
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
            const T tdt = (T)(a.mode == 4 ? mu[6] : a.dt);
            const bool heun = a.mode == 3;
            const bool stepm = a.mode == 1 || heun || a.mode == 4;
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

// Single-read variant: one cell per cluster of CL CTAs, each
// CTA holding N/CL x-planes of f* in registers (E values per thread), so that
// f* is read from HBM once and written once.  The five moment sums of the
// cell are combined across the cluster through distributed shared memory
// (partials in FP64, added in rank order: every CTA gets the same totals),
// double-buffered by cell parity so one cluster barrier per cell suffices.
// Several clusters (cells) share an SM, so one cell's loads overlap another's
// reductions and stores.
template <typename T, int N, int CL>
struct BgkClusterCfg {
    static constexpr int NT = 256;                       // threads per CTA
    static constexpr int V = 16 / (int)sizeof(T);        // elements per 16-byte access
    static constexpr int PP = N / CL;                    // x-planes per CTA
    static constexpr int E = PP * N * N / NT;            // values per thread
    static constexpr int NV = E / V;                     // 16-byte runs per thread
    static_assert(N % CL == 0 && (PP * N * N) % (NT * V) == 0, "whole 16-byte runs per thread");
};

__device__ __forceinline__ float2 shfl_xor_f2(float2 v, int off) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
}

template <typename T, int N, int CL>
__global__ void __launch_bounds__(256, 3) bgk_cluster_kernel(BgkArgs a) {
    using Cfg = BgkClusterCfg<T, N, CL>;
    constexpr int NT = Cfg::NT, V = Cfg::V, PP = Cfg::PP, NV = Cfg::NV;
    constexpr int N3 = N * N * N;
    constexpr int LPR = N / V;                           // runs per row
    using VT = typename Vec<T>::type;
    __shared__ float2 red[2][8];                          // this CTA's partials (hi, lo), by cell parity
    __shared__ float2 redw[NT / 32][5];
    __shared__ double mu[8];
    __shared__ long src_x[PP], src_y[N], src_z[N];
    __shared__ T gx[N], gy[N], gz[N];
    __shared__ T vgT[N];
    __shared__ signed char dsm[3 * N];

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const long cluster_id = blockIdx.x / CL;
    const long nclusters = gridDim.x / CL;
    const T* __restrict__ fin = static_cast<const T*>(a.f);
    T* __restrict__ fout = static_cast<T*>(a.out);
    const bool transport = a.delta != nullptr;
    const double dv = 2.0 * a.L / N;
    for (int i = tid; i < N; i += NT) vgT[i] = (T)(((double)i + 0.5 - 0.5 * N) * dv);
    for (int i = tid; i < 3 * N; i += NT) dsm[i] = transport ? a.delta[i] : 0;
    const int ncx = a.nc[0], ncy = a.nc[1], ncz = a.nc[2];
    const bool heun = a.mode == 3;
    const bool stepm = a.mode == 1 || heun || a.mode == 4;
    // run j of this thread: row r = (xl, y) and z0 inside the CTA's planes
    auto run_row = [&](int j) { return (j * NT + tid) / LPR; };
    auto run_z0 = [&](int j) { return ((j * NT + tid) % LPR) * V; };
    int parity = 0;

    for (long cell = a.cell0 + cluster_id; cell < a.ncells; cell += nclusters, parity ^= 1) {
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
        __syncthreads();   // the previous cell's readers of the shared tables are done
        for (int i = tid; i < PP + 2 * N; i += NT) {
            const int ax = i < PP ? 0 : (i < PP + N ? 1 : 2);
            const int k = ax == 0 ? rank * PP + i : (ax == 1 ? i - PP : i - PP - N);
            const int c0 = ax == 0 ? cx : (ax == 1 ? cy : cz);
            const int len = ax == 0 ? ncx : (ax == 1 ? ncy : ncz);
            int fl = 0;
            const int sc = transport ? fold_cell(c0 - dsm[ax * N + k], len, a.bc[ax], fl) : c0;
            const int q = fl ? N - 1 - k : k;
            if (ax == 0) src_x[i] = (long)sc * ncy * ncz * N3 + (long)q * N * N;
            else if (ax == 1) src_y[k] = (long)sc * ncz * N3 + (long)q * N;
            else src_z[k] = (long)sc * N3 + q;
        }
        __syncthreads();
        // load the CTA's planes (all runs in flight), moment partials in T
        T v[NV][V];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int r = run_row(j), z0 = run_z0(j);
            const long rb = src_x[r / N] + src_y[r % N];
            const long zb = src_z[z0];
            bool vec = (zb % V) == 0;
#pragma unroll
            for (int k = 1; k < V; ++k) vec &= src_z[z0 + k] == zb + k;
            if (vec) {
                const VT w = __ldcs(reinterpret_cast<const VT*>(fin + rb + zb));
                const T* pw = reinterpret_cast<const T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) v[j][k] = pw[k];
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[j][k] = __ldcs(fin + rb + src_z[z0 + k]);
            }
        }
        {
            // moment partials in FP32
            float s[5] = {0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const int r = run_row(j), z0 = run_z0(j);
                const T vx = vgT[rank * PP + r / N], vy = vgT[r % N];
                T sr = 0, sz = 0, szz = 0;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T vz = vgT[z0 + k];
                    sr += v[j][k];
                    sz += v[j][k] * vz;
                    szz += v[j][k] * vz * vz;
                }
                s[0] += sr;
                s[1] += sr * vx;
                s[2] += sr * vy;
                s[3] += sz;
                s[4] += sr * (vx * vx + vy * vy) + szz;
            }
            // the FP64 pipe is slow on this part: the sums stay compensated FP32 pairs
            // (hi, lo) through the warp, block and cluster levels, and become FP64 once
            float2 p[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) p[i] = make_float2(s[i], 0.0f);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int i = 0; i < 5; ++i) p[i] = two_sum_add(p[i], shfl_xor_f2(p[i], off));
            if ((tid & 31) == 0)
                for (int i = 0; i < 5; ++i) redw[tid >> 5][i] = p[i];
            __syncthreads();
            if (tid < 32) {
                constexpr int NW = NT / 32;   // 8 warps: lanes 0..7 hold one each, the rest zero
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    float2 q = tid < NW ? redw[tid][i] : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int off = NW / 2; off > 0; off >>= 1) q = two_sum_add(q, shfl_xor_f2(q, off));
                    if (tid == 0) red[parity][i] = q;
                }
            }
        }
        cluster_sync_all();   // every CTA's partials of this cell are visible
        if (tid < 32) {
            // warp 0: cell moments, Maxwellian factors, their moment sums, mu
            const int lane = tid;
            double m[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                float2 q = lane < CL ? cluster.map_shared_rank(&red[parity][0], lane)[i] : make_float2(0.0f, 0.0f);
#pragma unroll
                for (int off = CL / 2; off > 0; off >>= 1) q = two_sum_add(q, shfl_xor_f2(q, off));
                q = make_float2(__shfl_sync(0xffffffffu, q.x, 0), __shfl_sync(0xffffffffu, q.y, 0));
                m[i] = (double)q.x + (double)q.y;
            }
            m[4] *= 0.5;
            // scalars of the Maxwellian: rho, u, T in FP64 (one division), A and 1/(2T) in FP32
            const double dv3 = dv * dv * dv;
            const double rho = m[0] * dv3, irho = 1.0 / rho;
            const double ux = m[1] * dv3 * irho, uy = m[2] * dv3 * irho, uz = m[3] * dv3 * irho;
            const double Tt = (m[4] * dv3 * irho - 0.5 * (ux * ux + uy * uy + uz * uz)) * (2.0 / 3.0);
            // no Maxwellian for rho <= 0 or T <= 0 (vacuum, degenerate cells): M = 0, nu = 0, Q = 0
            const bool ok = rho > 0.0 && Tt > 0.0;
            const float tf = ok ? (float)Tt : 1.0f, i2T = 0.5f / tf;
            const float A = ok ? (float)rho * rsqrtf(2.0f * 3.14159265358979f * tf) / (2.0f * 3.14159265358979f * tf)
                               : 0.0f;
            const T w = vgT[lane];
            const T dx = w - (ok ? (float)ux : 0.0f), dy = w - (ok ? (float)uy : 0.0f), dz = w - (ok ? (float)uz : 0.0f);
            const T g0 = A * exp(-dx * dx * i2T), g1 = exp(-dy * dy * i2T), g2 = exp(-dz * dz * i2T);
            gx[lane] = g0;
            gy[lane] = g1;
            gz[lane] = g2;
            T acc[9] = {g0, w * g0, w * w * g0, g1, w * g1, w * w * g1, g2, w * g2, w * w * g2};
#pragma unroll
            for (int k = 0; k < 9; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
            if (lane < 6) {
                const double X[3] = {(double)acc[0], (double)acc[1], (double)acc[2]};
                const double Y[3] = {(double)acc[3], (double)acc[4], (double)acc[5]};
                const double Z[3] = {(double)acc[6], (double)acc[7], (double)acc[8]};
                const double nu = ok ? rho * a.inv_kn : 0.0;
                const double sM[5] = {X[0] * Y[0] * Z[0], X[1] * Y[0] * Z[0], X[0] * Y[1] * Z[0], X[0] * Y[0] * Z[1],
                                      0.5 * (X[2] * Y[0] * Z[0] + X[0] * Y[2] * Z[0] + X[0] * Y[0] * Z[2])};
                if (lane < 5) {
                    double mm = 0.0;
                    for (int jj = 0; jj < 5; ++jj) mm += a.P[lane * 5 + jj] * (sM[jj] - m[jj]);
                    mu[lane] = nu * mm;
                } else {
                    mu[5] = nu;
                    // mode 4: exponential step weight (1 - e^{-nu dt}) / nu (dt as nu -> 0)
                    if (a.mode == 4) mu[6] = nu > 0.0 ? -expm1(-nu * a.dt) / nu : a.dt;
                }
            }
        }
        __syncthreads();
        // output from registers: Q = nu (M - f) - phi.mu, out = Q, f* + dt Q or the Heun average
        {
            const T tnu = (T)mu[5];
            const T m0 = (T)mu[0], m1 = (T)mu[1], m2 = (T)mu[2], m3 = (T)mu[3], m4 = (T)mu[4];
            const T tdt = (T)(a.mode == 4 ? mu[6] : a.dt);
            T* oc = fout + cell * N3 + (long)rank * PP * N * N;
            const T* bc = static_cast<const T*>(a.base) + cell * N3 + (long)rank * PP * N * N;
            bool bad = false, neg = false;
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const int r = run_row(j), z0 = run_z0(j);
                const T vx = vgT[rank * PP + r / N], vy = vgT[r % N];
                const T gxy = gx[rank * PP + r / N] * gy[r % N];
                const T cxy = m0 + m1 * vx + m2 * vy + (T)0.5 * m4 * (vx * vx + vy * vy);
                T b[V];
                if (heun) {
                    const VT w = *reinterpret_cast<const VT*>(bc + (long)r * N + z0);
                    const T* pw = reinterpret_cast<const T*>(&w);
#pragma unroll
                    for (int k = 0; k < V; ++k) b[k] = pw[k];
                }
                VT w;
                T* pw = reinterpret_cast<T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T vz = vgT[z0 + k];
                    const T q = tnu * (gxy * gz[z0 + k] - v[j][k]) - (cxy + m3 * vz + (T)0.5 * m4 * vz * vz);
                    T o = stepm ? v[j][k] + tdt * q : q;
                    if (heun) o = (T)0.5 * (o + b[k]);
                    bad |= !isfinite(o);
                    neg |= stepm && o < T(0);
                    pw[k] = o;
                }
                __stcs(reinterpret_cast<VT*>(oc + (long)r * N + z0), w);
            }
            if (bad) atomicOr(a.flags, 1);
            if (neg) atomicOr(a.flags, 2);
        }
    }
    cluster_sync_all();   // no CTA leaves while a peer may still read its partials
}

// resident clusters of the single-read kernel (0: not resident)
template <typename T, int N, int CL>
static int bgk_cluster_capacity() {
    static int cap = -1;
    if (cap < 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CL, 1, 1);
        cfg.blockDim = dim3(BgkClusterCfg<T, N, CL>::NT, 1, 1);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        cap = cudaOccupancyMaxActiveClusters(&n, bgk_cluster_kernel<T, N, CL>, &cfg) == cudaSuccess ? n : 0;
    }
    return cap;
}

template <typename T, int N, int CL>
static cudaError_t launch_cluster(const BgkArgs& a, cudaStream_t s) {
    const long cells = a.ncells - a.cell0;
    const int cap = bgk_cluster_capacity<T, N, CL>();
    if (cap <= 0) return cudaErrorInvalidConfiguration;
    const long nclus = cells < cap ? cells : cap;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nclus * CL), 1, 1);
    cfg.blockDim = dim3(BgkClusterCfg<T, N, CL>::NT, 1, 1);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BgkArgs args = a;
    void* kargs[] = {&args};
    return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&bgk_cluster_kernel<T, N, CL>), kargs);
}

template <typename T, int N>
static cudaError_t launch_n(const BgkArgs& a, cudaStream_t s) {
    // 128-thread CTAs, eight resident per SM (registers); two waves of them
    // (measured: 16 per SM 3.24 ms, 6 per SM 3.68 ms, 4 per SM 4.43 ms at 32^3 x 32^3)
    constexpr int BS = N >= 16 ? 128 : 256;
    const long cells = a.ncells - a.cell0;
    if (cells <= 0) return cudaSuccess;
    // the single-read cluster kernel for FP32 n = 32 (4 CTAs of 8 planes, 32 values per thread);
    // FP64 would need twice the registers per value and keeps the two-pass kernel
    if constexpr (N == 32 && sizeof(T) == 4) return launch_cluster<T, N, 4>(a, s);
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
