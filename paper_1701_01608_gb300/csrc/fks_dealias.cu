// fks_dealias.cu -- variant B of the fast operator: Eq. CF1 with l + m = k over
// the modes l, m in [-n/2, n/2]^3 (not reduced mod n), evaluated with
// transforms of size 2n as in Sec. 5.  The coefficient of a Nyquist component
// is split equally between +n/2 and -n/2; the result keeps the modes
// |k| <= n/2 and folds +-n/2 back onto the Nyquist index.
//
// Per chunk of cells:
//   pad_kernel   f* (n^3, gathered by the transport shifts in step mode)
//                -> f2 = P x P x P f* on the 2n grid (trigonometric interpolant)
//   collision    the cluster kernel of the 2n grid, without projection
//                (mode 2), on f2 -> Q2 = (G2 - L2) / Kn
//   trunc_kernel Q = T x T x T Q2 on the n grid, FP64 conservation projection,
//                out = Q or f* + dt Q
// P (2n x n) and T (n x 2n) are the one-axis operators, built on the host from
// the DFT definitions.  T P = I.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "fks_collide.cuh"
#include "fks_internal.h"

namespace fks {
namespace dealias {

constexpr int BS = 256;

struct Args {
    const void* f;              // coarse cells (n^3 each)
    void* f2;                   // [chunk][(2n)^3]
    const void* q2;             // [chunk][(2n)^3]
    void* out;                  // coarse cells
    const void* P;              // [2n][n]
    const void* T;              // [n][2n]
    const signed char* delta;   // [3][n] transport shifts (step mode) or nullptr
    int* flags;
    long c0, k;                 // cells c0 .. c0 + k - 1
    int nc[3], bc[3];
    double L, dt;
    int mode;                   // 0 collide, 1 step
    double Pm[25];              // projection coefficients of the n grid
};

// f* at (x, y, z) of cell `cell` (transport gather when delta is set)
template <typename T, int N>
__device__ __forceinline__ T fstar(const Args& a, const int* dsm, long cell, int x, int y, int z) {
    constexpr long N3 = (long)N * N * N;
    const T* f = static_cast<const T*>(a.f);
    if (!a.delta) return f[cell * N3 + ((long)x * N + y) * N + z];
    const int ncy = a.nc[1], ncz = a.nc[2];
    int cx, cy, cz;
    cell_coords(cell, ncy, ncz, cx, cy, cz);
    int fx, fy, fz;
    const int sx = fold_cell(cx - dsm[x], a.nc[0], a.bc[0], fx);
    const int sy = fold_cell(cy - dsm[N + y], ncy, a.bc[1], fy);
    const int sz = fold_cell(cz - dsm[2 * N + z], ncz, a.bc[2], fz);
    const int qx = fx ? N - 1 - x : x, qy = fy ? N - 1 - y : y, qz = fz ? N - 1 - z : z;
    return f[(((long)sx * ncy + sy) * ncz + sz) * N3 + ((long)qx * N + qy) * N + qz];
}

// one CTA per cell: f2[x2][y2][z2] = sum P[x2][x] P[y2][y] P[z2][z] f*[x][y][z],
// one axis at a time in shared memory
template <typename T, int N>
__global__ void __launch_bounds__(BS) pad_kernel(const Args a) {
    constexpr int M2 = 2 * N;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* Pm = reinterpret_cast<T*>(sm_raw);   // [M2][N]
    T* B = Pm + M2 * N;                     // [N][N][M2]
    T* AC = B + N * N * M2;                 // A [N][N][N], then C [N][M2][M2]
    __shared__ int dsm[3 * N];
    const int tid = threadIdx.x;
    for (int i = tid; i < M2 * N; i += BS) Pm[i] = static_cast<const T*>(a.P)[i];
    for (int i = tid; i < 3 * N; i += BS) dsm[i] = a.delta ? (int)a.delta[i] : 0;
    __syncthreads();
    for (long cell = a.c0 + blockIdx.x; cell < a.c0 + a.k; cell += gridDim.x) {
        for (int e = tid; e < N * N * N; e += BS)
            AC[e] = fstar<T, N>(a, dsm, cell, e / (N * N), (e / N) % N, e % N);
        __syncthreads();
        for (int e = tid; e < N * N * M2; e += BS) {   // along z
            const int xy = e / M2, z2 = e % M2;
            T acc = 0;
#pragma unroll
            for (int z = 0; z < N; ++z) acc += AC[xy * N + z] * Pm[z2 * N + z];
            B[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < N * M2 * M2; e += BS) {   // along y (C overwrites A)
            const int x = e / (M2 * M2), y2 = (e / M2) % M2, z2 = e % M2;
            T acc = 0;
#pragma unroll
            for (int y = 0; y < N; ++y) acc += B[(x * N + y) * M2 + z2] * Pm[y2 * N + y];
            AC[e] = acc;
        }
        __syncthreads();
        T* dst = static_cast<T*>(a.f2) + (cell - a.c0) * (long)M2 * M2 * M2;
        for (int e = tid; e < M2 * M2; e += BS) {   // along x, straight to global (coalesced in z2)
            T col[N];
#pragma unroll
            for (int x = 0; x < N; ++x) col[x] = AC[x * M2 * M2 + e];
            for (int x2 = 0; x2 < M2; ++x2) {
                T acc = 0;
#pragma unroll
                for (int x = 0; x < N; ++x) acc += col[x] * Pm[x2 * N + x];
                dst[(long)x2 * M2 * M2 + e] = acc;
            }
        }
        __syncthreads();   // B and AC are rewritten by the next cell
    }
}

// one CTA per cell: Q = T x T x T Q2, FP64 moment sums, projection, output
template <typename T, int N>
__global__ void __launch_bounds__(BS) trunc_kernel(const Args a) {
    constexpr int M2 = 2 * N;
    constexpr long N3 = (long)N * N * N;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* Tm = reinterpret_cast<T*>(sm_raw);   // [N][M2]
    T* Cp = Tm + N * M2;                    // [N][M2][M2], then Q [N][N][N]
    T* Bp = Cp + N * M2 * M2;               // [N][N][M2]
    __shared__ int dsm[3 * N];
    __shared__ double vg[N];
    __shared__ float vgf[N], vgl[N], vg2f[N], vg2l[N];   // v and v^2/2 as FP32 pairs hi + lo
    __shared__ double red[BS / 32][5];
    __shared__ double mu[5];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < N * M2; i += BS) Tm[i] = static_cast<const T*>(a.T)[i];
    for (int i = tid; i < 3 * N; i += BS) dsm[i] = a.delta ? (int)a.delta[i] : 0;
    const double dv = 2.0 * a.L / N;
    if (tid < N) {
        vg[tid] = ((double)tid + 0.5 - 0.5 * N) * dv;
        const double h = 0.5 * vg[tid] * vg[tid];
        vgf[tid] = (float)vg[tid];
        vgl[tid] = (float)(vg[tid] - (double)vgf[tid]);
        vg2f[tid] = (float)h;
        vg2l[tid] = (float)(h - (double)vg2f[tid]);
    }
    __syncthreads();
    for (long cell = a.c0 + blockIdx.x; cell < a.c0 + a.k; cell += gridDim.x) {
        const T* src = static_cast<const T*>(a.q2) + (cell - a.c0) * (long)M2 * M2 * M2;
        for (int e = tid; e < M2 * M2; e += BS) {   // along x, from global (coalesced in z2)
            T acc[N];
#pragma unroll
            for (int x = 0; x < N; ++x) acc[x] = 0;
            for (int x2 = 0; x2 < M2; ++x2) {
                const T q = src[(long)x2 * M2 * M2 + e];
#pragma unroll
                for (int x = 0; x < N; ++x) acc[x] += Tm[x * M2 + x2] * q;
            }
#pragma unroll
            for (int x = 0; x < N; ++x) Cp[x * M2 * M2 + e] = acc[x];
        }
        __syncthreads();
        for (int e = tid; e < N * N * M2; e += BS) {   // along y
            const int x = e / (N * M2), y = (e / M2) % N, z2 = e % M2;
            T acc = 0;
            for (int y2 = 0; y2 < M2; ++y2) acc += Tm[y * M2 + y2] * Cp[(x * M2 + y2) * M2 + z2];
            Bp[e] = acc;
        }
        __syncthreads();
        T* Q = Cp;   // the x-pass result is no longer needed
        double s[5] = {0, 0, 0, 0, 0};
        if constexpr (sizeof(T) == 4) {
            // FP32: compensated FP32 moment sums (hi, lo pairs, exact products by FMA), FP64
            // from the warp totals on (per-element FP64 work is slow on this part)
            float2 sf[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) sf[i] = make_float2(0.f, 0.f);
            for (int e = tid; e < N * N * N; e += BS) {   // along z, and the moment sums
                const int xy = e / N, z = e % N;
                T acc = 0;
                for (int z2 = 0; z2 < M2; ++z2) acc += Tm[z * M2 + z2] * Bp[xy * M2 + z2];
                Q[e] = acc;
                const int x = xy / N, y = xy % N;
                const float q = acc;
                sf[0] = df_add1(sf[0], q);
                sf[1] = df_add(sf[1], df_mul(make_float2(q, 0.f), make_float2(vgf[x], vgl[x])));
                sf[2] = df_add(sf[2], df_mul(make_float2(q, 0.f), make_float2(vgf[y], vgl[y])));
                sf[3] = df_add(sf[3], df_mul(make_float2(q, 0.f), make_float2(vgf[z], vgl[z])));
                const float2 w = df_add(df_add(make_float2(vg2f[x], vg2l[x]), make_float2(vg2f[y], vg2l[y])),
                                        make_float2(vg2f[z], vg2l[z]));
                sf[4] = df_add(sf[4], df_mul(make_float2(q, 0.f), w));
            }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sf[i] = df_add(sf[i], df_shfl_xor(sf[i], off));
#pragma unroll
            for (int i = 0; i < 5; ++i) s[i] = (double)sf[i].x + (double)sf[i].y;
            if (lane == 0)
                for (int i = 0; i < 5; ++i) red[warp][i] = s[i];
        } else {
            for (int e = tid; e < N * N * N; e += BS) {   // along z, and the moment sums (FP64)
                const int xy = e / N, z = e % N;
                T acc = 0;
                for (int z2 = 0; z2 < M2; ++z2) acc += Tm[z * M2 + z2] * Bp[xy * M2 + z2];
                Q[e] = acc;
                const double q = (double)acc, vx = vg[xy / N], vy = vg[xy % N], vz = vg[z];
                s[0] += q;
                s[1] = fma(q, vx, s[1]);
                s[2] = fma(q, vy, s[2]);
                s[3] = fma(q, vz, s[3]);
                s[4] = fma(q, 0.5 * (vx * vx + vy * vy + vz * vz), s[4]);
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                double v = s[i];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) red[warp][i] = v;
            }
        }
        __syncthreads();
        if (tid < 5) {
            double tot[5] = {0, 0, 0, 0, 0};
            for (int w = 0; w < BS / 32; ++w)
                for (int j = 0; j < 5; ++j) tot[j] += red[w][j];
            double acc = 0.0;
            for (int j = 0; j < 5; ++j) acc += a.Pm[tid * 5 + j] * tot[j];
            mu[tid] = acc;
        }
        __syncthreads();
        T* out = static_cast<T*>(a.out);
        bool bad = false, neg = false;
        const float muf[5] = {(float)mu[0], (float)mu[1], (float)mu[2], (float)mu[3], (float)mu[4]};
        for (int e = tid; e < N * N * N; e += BS) {
            const int x = e / (N * N), y = (e / N) % N, z = e % N;
            T q;
            if constexpr (sizeof(T) == 4) {
                // the correction in FP32 (a small term next to Q)
                const float corr = muf[0] + muf[1] * vgf[x] + muf[2] * vgf[y] + muf[3] * vgf[z] +
                                   muf[4] * (vg2f[x] + vg2f[y] + vg2f[z]);
                q = Q[e] - corr;
            } else {
                const double vx = vg[x], vy = vg[y], vz = vg[z];
                const double corr =
                    mu[0] + mu[1] * vx + mu[2] * vy + mu[3] * vz + mu[4] * 0.5 * (vx * vx + vy * vy + vz * vz);
                q = (T)((double)Q[e] - corr);
            }
            const T o = a.mode == 1 ? fstar<T, N>(a, dsm, cell, x, y, z) + (T)a.dt * q : q;
            bad |= !isfinite(o);
            neg |= a.mode == 1 && o < T(0);
            out[cell * N3 + e] = o;
        }
        if (bad) atomicOr(a.flags, 1);
        if (neg) atomicOr(a.flags, 2);
        __syncthreads();   // Cp, Bp, red and mu are rewritten by the next cell
    }
}

template <typename T, int N>
size_t pad_smem() { return sizeof(T) * (2 * N * N + N * N * 2 * N + (size_t)N * 2 * N * 2 * N); }
template <typename T, int N>
size_t trunc_smem() { return sizeof(T) * (N * 2 * N + (size_t)N * 2 * N * 2 * N + N * N * 2 * N); }

template <typename T, int N>
cudaError_t launch(const Args& a, bool pad, cudaStream_t s) {
    const size_t smem = pad ? pad_smem<T, N>() : trunc_smem<T, N>();
    auto k = pad ? pad_kernel<T, N> : trunc_kernel<T, N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long grid = a.k < 2L * 152 ? a.k : 2L * 152;
    k<<<(unsigned)grid, BS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_any(bool fp64, int n, const Args& a, bool pad, cudaStream_t s) {
    if (fp64) {
        if (n == 8) return launch<double, 8>(a, pad, s);
        if (n == 16) return launch<double, 16>(a, pad, s);
    } else {
        if (n == 8) return launch<float, 8>(a, pad, s);
        if (n == 16) return launch<float, 16>(a, pad, s);
    }
    return cudaErrorInvalidValue;
}

// One-axis operators from the DFT definitions, applied to unit vectors:
//   P (2n x n): coefficients c_k = (1/n) sum_j x_j e^{-2 pi i k j / n}, k in
//   [-n/2, n/2), the Nyquist coefficient split between +-n/2, evaluated at the
//   2n points: x2_j2 = sum_k c_k e^{2 pi i k j2 / (2n)}.
//   T (n x 2n): coefficients (1/2n) sum_j2 y_j2 e^{-2 pi i k j2 / (2n)}, k in
//   [-n, n), kept for |k| <= n/2, +-n/2 folded, evaluated at the n points.
void matrices(int n, std::vector<double>& P, std::vector<double>& T) {
    const int m = 2 * n;
    const double pi = 3.14159265358979323846;
    using cd = std::complex<double>;
    P.assign((size_t)m * n, 0.0);
    T.assign((size_t)n * m, 0.0);
    for (int j = 0; j < n; ++j)
        for (int j2 = 0; j2 < m; ++j2) {
            cd acc = 0.0;
            for (int k = -n / 2; k < n / 2; ++k) {
                const cd c = std::exp(cd(0.0, -2.0 * pi * k * j / n)) / (double)n;
                if (2 * k == -n) {   // Nyquist: half at -n/2, half at +n/2
                    acc += 0.5 * c * std::exp(cd(0.0, 2.0 * pi * (-n / 2) * j2 / m));
                    acc += 0.5 * c * std::exp(cd(0.0, 2.0 * pi * (n / 2) * j2 / m));
                } else {
                    acc += c * std::exp(cd(0.0, 2.0 * pi * k * j2 / m));
                }
            }
            P[(size_t)j2 * n + j] = acc.real();
        }
    for (int j2 = 0; j2 < m; ++j2)
        for (int j = 0; j < n; ++j) {
            cd acc = 0.0;
            for (int k = -n; k < n; ++k) {
                if (2 * std::abs(k) > n) continue;
                const cd c = std::exp(cd(0.0, -2.0 * pi * k * j2 / m)) / (double)m;
                acc += c * std::exp(cd(0.0, 2.0 * pi * k * j / n));   // +-n/2 land on the same n-grid mode
            }
            T[(size_t)j * m + j2] = acc.real();
        }
}

}  // namespace dealias
}  // namespace fks

using namespace fks;

// Variant B for cells [0, ncells): chunks of c->dchunk cells through the pad,
// the inner 2n collision (no projection) and the truncation with projection.
fks_status launch_dealias(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                          cudaStream_t s) {
    dealias::Args a;
    std::memset(&a, 0, sizeof(a));
    a.f = f;
    a.f2 = c->d2f;
    a.q2 = c->d2q;
    a.out = out;
    a.P = c->dPm;
    a.T = c->dTm;
    a.delta = delta;
    a.flags = c->d_flags;
    a.nc[0] = c->grid.nx;
    a.nc[1] = c->grid.ny;
    a.nc[2] = c->grid.nz;
    for (int i = 0; i < 3; ++i) a.bc[i] = c->grid.bc[i];
    a.L = c->vbox.L;
    a.dt = dt;
    a.mode = mode;
    std::memcpy(a.Pm, c->P, sizeof(a.Pm));
    for (long c0 = 0; c0 < c->ncells; c0 += c->dchunk) {
        a.c0 = c0;
        a.k = c->ncells - c0 < c->dchunk ? c->ncells - c0 : c->dchunk;
        cudaError_t e = dealias::launch_any(c->fp64, c->n, a, true, s);
        if (e != cudaSuccess) return fks_internal_fail(c, FKS_ERR_CUDA, std::string("pad kernel: ") + cudaGetErrorString(e));
        c->inner->ncells = a.k;
        c->inner->grid.nx = (int)a.k;
        fks_status st = fks_internal_collide(c->inner, c->d2f, c->d2q, 2, s);
        if (st != FKS_OK) return fks_internal_fail(c, st, std::string("2n collision: ") + fks_last_error(c->inner));
        e = dealias::launch_any(c->fp64, c->n, a, false, s);
        if (e != cudaSuccess)
            return fks_internal_fail(c, FKS_ERR_CUDA, std::string("truncation kernel: ") + cudaGetErrorString(e));
        c->launches += 3;
    }
    return FKS_OK;
}

extern "C" fks_status fks_set_dealias(fks_ctx* c, int on) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!on) {
        fks_destroy(c->inner);
        cudaFree(c->d2f);
        cudaFree(c->d2q);
        cudaFree(c->dPm);
        cudaFree(c->dTm);
        c->inner = nullptr;
        c->d2f = c->d2q = c->dPm = c->dTm = nullptr;
        c->dealias = false;
        return FKS_OK;
    }
    if (c->dealias) return FKS_OK;
    if (c->bgk || c->tc || (c->n != 8 && c->n != 16))
        return fks_internal_fail(c, FKS_ERR_UNSUPPORTED, "variant B needs a spectral FP32/FP64 context with n = 8 or 16");
    // inner context: the 2n grid of the same box, kernel and directions
    c->dchunk = c->ncells < 2048 ? (c->ncells > 0 ? c->ncells : 1) : 2048;
    fks_grid g = c->grid;
    g.nx = (int)c->dchunk;
    g.ny = g.nz = 1;
    for (int i = 0; i < 3; ++i) g.bc[i] = FKS_BC_PERIODIC;
    fks_vbox vb = c->vbox;
    vb.n = 2 * c->n;
    fks_ctx* in = nullptr;
    fks_status st = fks_init(&g, &vb, &c->kern, &c->dirs, c->fp64 ? FKS_FP64 : FKS_FP32, &in);
    if (st != FKS_OK) return fks_internal_fail(c, st, "inner 2n context");
    // the inner grid's unprojected operator keeps its own arithmetic (the escalation bound is
    // stated for the projected n-grid result)
    if (!c->fp64) fks_set_escalation(in, 0.0);
    const size_t esz = c->fp64 ? 8 : 4;
    const size_t m3 = (size_t)8 * c->n * c->n * c->n;
    std::vector<double> P, T;
    dealias::matrices(c->n, P, T);
    std::vector<float> Pf(P.begin(), P.end()), Tf(T.begin(), T.end());
    bool ok = cudaMalloc(&c->d2f, esz * m3 * c->dchunk) == cudaSuccess &&
              cudaMalloc(&c->d2q, esz * m3 * c->dchunk) == cudaSuccess &&
              cudaMalloc(&c->dPm, esz * P.size()) == cudaSuccess && cudaMalloc(&c->dTm, esz * T.size()) == cudaSuccess;
    if (ok)
        ok = cudaMemcpy(c->dPm, c->fp64 ? (const void*)P.data() : (const void*)Pf.data(), esz * P.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(c->dTm, c->fp64 ? (const void*)T.data() : (const void*)Tf.data(), esz * T.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    c->inner = in;
    c->dealias = true;
    if (!ok) {
        const fks_status st = alloc_failure();
        fks_set_dealias(c, 0);
        return fks_internal_fail(c, st, "variant B buffers");
    }
    return FKS_OK;
}
