// fks_capi.cu -- C ABI of libfks: context, spectral tables, transport,
// moments and the launch of the fused collision kernel.
//
// Method: arXiv 1701.01608 (Fast Kinetic Scheme), Sec. 2.1 (transport and
// explicit Euler collision step, Eq. disc_relax), Sec. 3 (generic-cell
// particles, moments), Appendix A (fast spectral Boltzmann operator).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "fks_internal.h"

namespace fks {

// ------------------------------------------------------------------ tables
//
// Carleman form with a separable kernel B~ = a(|x|) b(|y|) (Appendix A):
//   alpha_p(k)  = phi(xi_k . e_p),   phi(s) = int_{-R}^{R} |r| a(|r|) e^{i r s} dr
//   alphap_p(k) = psi(|xi_k - (xi_k . e_p) e_p|),
//                 psi(s) = int_0^pi phi_b(s cos t) dt  (disc integral in the plane
//                 orthogonal to e_p, written in polar form)
// with xi_k = (pi/L) kappa(k), cut-off R = lam L, lam = 2/(3+sqrt 2).
// Hard spheres: a = b = sqrt(4C); pseudo-Maxwell: a = b = sqrt(4C) r^-1/2.

constexpr int kGL = 64;

struct TableParams {
    int n, M, ktype, HF;
    double L, R, c4;               // c4 = sqrt(4C)
    const double* e;               // [M][3]
    const double* w;               // [M]
    const double* glt_x;           // Gauss-Legendre on [0, pi/2]: nodes
    const double* glt_w;           //                               weights
    const double* glu_x;           // Gauss-Legendre on [0, sqrt(R)]: nodes
    const double* glu_w;           //                                  weights
    // variable hard spheres (ktype 3): table pair p is term p % vS of direction p / vS
    int vS, vQ;
    const double* vr;              // [vQ] radial nodes
    const double* vca;             // [vS][vQ] phi_s coefficients
    const double* vcb;             // [vS][vQ] psi_s coefficients
};

// phi for hard spheres in closed form: 2 c4 [R sin(Rs)/s + (cos(Rs) - 1)/s^2]
__host__ __device__ inline double phi_hs(double c4, double R, double s) {
    s = fabs(s);
    const double x = R * s;
    if (x < 1e-3) {
        const double x2 = x * x;
        return c4 * R * R * (1.0 - x2 * (1.0 / 4.0) + x2 * x2 * (1.0 / 72.0) - x2 * x2 * x2 * (1.0 / 2880.0));
    }
    const double sh = sin(0.5 * x);
    return c4 * 2.0 * (R * sin(x) / s - 2.0 * sh * sh / (s * s));
}

// phi for the pseudo-Maxwell kernel: 2 c4 int_0^R sqrt(r) cos(r s) dr,
// r = u^2:  4 c4 int_0^sqrt(R) u^2 cos(u^2 s) du, Gauss-Legendre in u
__host__ __device__ inline double phi_pm(double c4, double s, const double* gx, const double* gw) {
    double acc = 0.0;
    for (int i = 0; i < kGL; ++i) acc += gw[i] * gx[i] * gx[i] * cos(gx[i] * gx[i] * s);
    return 4.0 * c4 * acc;
}

__host__ __device__ inline double phi_any(const TableParams& tp, double s) {
    return tp.ktype == 0 ? phi_hs(tp.c4, tp.R, s) : phi_pm(tp.c4, s, tp.glu_x, tp.glu_w);
}

// psi(s) = 2 int_0^{pi/2} phi(s cos t) dt  (phi is even), Gauss-Legendre in t
__host__ __device__ inline double psi_any(const TableParams& tp, double s) {
    double acc = 0.0;
    for (int i = 0; i < kGL; ++i) acc += tp.glt_w[i] * phi_any(tp, s * cos(tp.glt_x[i]));
    return 2.0 * acc;
}

__host__ __device__ inline int signed_freq(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// alpha and alphap of mode (kx, ky, kz) for direction p, averaged over the
// sign choices of Nyquist components (each stands for +-n/2 with half weight)
__host__ __device__ inline void mode_tables(const TableParams& tp, int p, int kx, int ky, int kz,
                                            double* a_out, double* b_out) {
    const int n = tp.n;
    const int kk[3] = {kx, ky, kz};
    const double h = 3.14159265358979323846 / tp.L;
    int nyq_axes[3], nnyq = 0;
    for (int a = 0; a < 3; ++a)
        if ((n % 2 == 0) && kk[a] == n / 2) nyq_axes[nnyq++] = a;
    const double ex = tp.e[3 * p], ey = tp.e[3 * p + 1], ez = tp.e[3 * p + 2];
    double sa = 0.0, sb = 0.0;
    const int ncomb = 1 << nnyq;
    for (int c = 0; c < ncomb; ++c) {
        double xi[3];
        for (int a = 0; a < 3; ++a) xi[a] = h * signed_freq(kk[a], n);
        for (int b = 0; b < nnyq; ++b)
            if (c & (1 << b)) xi[nyq_axes[b]] = -xi[nyq_axes[b]];
        const double d = xi[0] * ex + xi[1] * ey + xi[2] * ez;
        const double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] - d * d;
        const double u = sqrt(q2 > 0.0 ? q2 : 0.0);
        if (tp.ktype == 3) {
            const int term = p % tp.vS;
            sa += vhs_phi(tp.vca + (long)term * tp.vQ, tp.vr, tp.vQ, d);
            sb += vhs_psi(tp.vcb + (long)term * tp.vQ, tp.vr, tp.vQ, u);
        } else {
            sa += phi_any(tp, d);
            sb += psi_any(tp, u);
        }
    }
    *a_out = sa / ncomb;
    *b_out = sb / ncomb;
}

// FP64 tables on the half spectrum kz in [0, n/2]: A, B = [M][n][n][HF]
__global__ void tables_kernel(TableParams tp, double* A, double* B) {
    const long total = (long)tp.M * tp.n * tp.n * tp.HF;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(i % tp.HF);
        const int ky = (int)((i / tp.HF) % tp.n);
        const int kx = (int)((i / ((long)tp.HF * tp.n)) % tp.n);
        const int p = (int)(i / ((long)tp.HF * tp.n * tp.n));
        double a, b;
        mode_tables(tp, p, kx, ky, kz, &a, &b);
        A[i] = a;
        B[i] = b;
    }
}

// Pack into the collision kernel's layout: for every direction p (slot M =
// loss) and cluster rank r one contiguous slab [tab][kx][kyl][kz = 0..n/2];
// table 0 = alpha N^-3, table 1 = w_p alphap N^-3; slot M: betaL N^-3
// (betaL = sum_p w_p alpha_p alphap_p) and zeros.
template <typename T>
__global__ void pack_tables_kernel(int n, int M, int C, int HF, const double* A, const double* B,
                                   const double* w, T* out) {
    const int NS = n / C;
    const double s3 = 1.0 / ((double)n * n * n);
    const long per = (long)n * NS * HF;
    const long total = (long)(M + 1) * C * 2 * per;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(i % HF);
        const int kyl = (int)((i / HF) % NS);
        const int kx = (int)((i / ((long)HF * NS)) % n);
        const int tab = (int)((i / per) % 2);
        const int r = (int)((i / (per * 2)) % C);
        const int p = (int)(i / (per * 2 * C));
        const int ky = r * NS + kyl;
        const long src = ((long)kx * n + ky) * HF + kz;
        const long plane = (long)n * n * HF;
        double v;
        if (p < M) {
            v = tab == 0 ? A[p * plane + src] * s3 : w[p] * B[p * plane + src] * s3;
        } else if (tab == 0) {
            double acc = 0.0;
            for (int q = 0; q < M; ++q) acc += w[q] * A[q * plane + src] * B[q * plane + src];
            v = acc * s3;
        } else {
            v = 0.0;
        }
        out[i] = (T)v;
    }
}

// Full-spectrum tables of the tensor-core path: [M+1][kx][ky][kz] pairs
// (alpha N^-3, w_p alphap N^-3), slot M (betaL N^-3, 0).  A mode with
// kz > n/2 takes the value of its mirror -k, which lies in the half spectrum
// (the tables are even in k).
__global__ void pack_tables_full_kernel(int n, int M, int HF, const double* A, const double* B, const double* w,
                                        float2* out) {
    const double s3 = 1.0 / ((double)n * n * n);
    const long n3 = (long)n * n * n;
    const long total = (long)(M + 1) * n3;
    const long plane = (long)n * n * HF;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        int kz = (int)(i % n), ky = (int)((i / n) % n), kx = (int)((i / ((long)n * n)) % n);
        const int p = (int)(i / n3);
        if (kz > n / 2) {
            kz = n - kz;
            ky = (n - ky) % n;
            kx = (n - kx) % n;
        }
        const long src = ((long)kx * n + ky) * HF + kz;
        double va, vb;
        if (p < M) {
            va = A[p * plane + src] * s3;
            vb = w[p] * B[p * plane + src] * s3;
        } else {
            double acc = 0.0;
            for (int q = 0; q < M; ++q) acc += w[q] * A[q * plane + src] * B[q * plane + src];
            va = acc * s3;
            vb = 0.0;
        }
        out[i] = make_float2((float)va, (float)vb);
    }
}

// ------------------------------------------------------------------ offsets
// Generic-cell particle offsets (Sec. 3), one axis per blockIdx.y:
//   s <- s + v dt;  delta = floor((s + dx/2)/dx);  s <- s - delta dx
// computed for v > 0 and mirrored for -v.  Explicit roundings (no
// contraction) keep the result identical to a plain IEEE evaluation.
__global__ void offsets_kernel(int n, double L, double3 dx3, double dt, double* s, signed char* delta, int* flags) {
    const int a = blockIdx.y;
    const int i = n / 2 + threadIdx.x;
    if (i >= n) return;
    const double dx = a == 0 ? dx3.x : (a == 1 ? dx3.y : dx3.z);
    const double dv = __ddiv_rn(2.0 * L, (double)n);
    const double v = __dmul_rn((double)i + 0.5 - 0.5 * n, dv);
    const double sn = __dadd_rn(s[a * n + i], __dmul_rn(v, dt));
    const double d = floor(__ddiv_rn(__dadd_rn(sn, __dmul_rn(0.5, dx)), dx));
    const double snew = __dsub_rn(sn, __dmul_rn(d, dx));
    const int im = n - 1 - i;
    s[a * n + i] = snew;
    s[a * n + im] = -snew;
    if (fabs(d) > 120.0) atomicOr(flags, 4);
    const int di = (int)d;
    delta[a * n + i] = (signed char)di;
    delta[a * n + im] = (signed char)(-di);
}

// ------------------------------------------------------------------ transport
// f_out[j][k] = f[j - delta_k][k'] : one thread per output element
// One CTA per cell (persistent over cells), rows of N/V lanes: lane group t
// owns velocity indices z0 .. z0+V-1 (V = 16 bytes / sizeof T) of the rows
// (x, y) = t / (N/V) + RPI j.  The source offsets of the transported cell are
// tabulated per axis in shared memory; where the thread's V source elements
// are one aligned run they move as one 16-byte access.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

// transport gather f*[j][k] = f[j - delta_k][k'] (Sec. 2.1, exact shift)
template <typename T, int N>
__global__ void __launch_bounds__(256) transport_kernel(int ncx, int ncy, int ncz, int bcx, int bcy, int bcz,
                                                        const signed char* __restrict__ delta, const T* __restrict__ f,
                                                        T* __restrict__ out, long ncells) {
    constexpr int BS = 256, V = 16 / (int)sizeof(T), LPR = N / V, RPI = BS / LPR;
    constexpr int ROWS = (N * N + RPI - 1) / RPI;
    constexpr long N3 = (long)N * N * N;
    using VT = typename Vec16<T>::type;
    __shared__ long src_x[N], src_y[N], src_z[N];
    const int tid = threadIdx.x;
    const bool lane_ok = tid < LPR * RPI;
    const int z0 = (tid % LPR) * V, r0 = tid / LPR;
    for (long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
        __syncthreads();   // the previous cell's readers of the tables are done
        for (int i = tid; i < 3 * N; i += BS) {
            const int ax = i / N, k = i % N;
            const int c0 = ax == 0 ? cx : (ax == 1 ? cy : cz);
            const int len = ax == 0 ? ncx : (ax == 1 ? ncy : ncz);
            const int bc = ax == 0 ? bcx : (ax == 1 ? bcy : bcz);
            int fl = 0;
            const int sc = fold_cell(c0 - delta[i], len, bc, fl);
            const int q = fl ? N - 1 - k : k;
            if (ax == 0) src_x[k] = (long)sc * ncy * ncz * N3 + (long)q * N * N;
            else if (ax == 1) src_y[k] = (long)sc * ncz * N3 + (long)q * N;
            else src_z[k] = (long)sc * N3 + q;
        }
        __syncthreads();
        if (!lane_ok) continue;
        long zo[V];
        bool vec = true;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            zo[k] = src_z[z0 + k];
            vec &= zo[k] == zo[0] + k;
        }
        vec &= (zo[0] % V) == 0;
        T* oc = out + cell * N3 + z0;
#pragma unroll 4
        for (int j = 0; j < ROWS; ++j) {
            const int r = r0 + RPI * j;
            if (r >= N * N) break;
            const long rb = src_x[r / N] + src_y[r % N];
            VT w;
            if (vec) {
                w = __ldcs(reinterpret_cast<const VT*>(f + rb + zo[0]));
            } else {
                T* pw = reinterpret_cast<T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) pw[k] = __ldcs(f + rb + zo[k]);
            }
            __stcs(reinterpret_cast<VT*>(oc + (long)r * N), w);
        }
    }
}

// ------------------------------------------------------------------ moments
// U = dv^3 sum phi(v) f, phi = (1, v, |v|^2/2): along a 16-byte run the sums of
// f, f v_z and f v_z^2/2, then per row the factors v_x, v_y.  FP64 input: FP64
// sums.  FP32 input: compensated FP32 sums (FP64-equivalent accuracy; GB300's
// FP64 pipe made the FP64 version FP64-bound at 3 operations per element).
template <typename T, int N>
__global__ void __launch_bounds__(256) moments_kernel(double L, long ncells, const T* __restrict__ f,
                                                      double* __restrict__ U) {
    constexpr int BS = 256, V = 16 / (int)sizeof(T), LPR = N / V, RPI = BS / LPR;
    constexpr int ROWS = (N * N + RPI - 1) / RPI;
    constexpr long N3 = (long)N * N * N;
    using VT = typename Vec16<T>::type;
    __shared__ double red[BS / 32][5];
    __shared__ double vg[N];
    const int tid = threadIdx.x;
    const double dv = 2.0 * L / N;
    if (tid < N) vg[tid] = ((double)tid + 0.5 - 0.5 * N) * dv;
    __syncthreads();
    const bool lane_ok = tid < LPR * RPI;
    const int z0 = (tid % LPR) * V, r0 = tid / LPR;
    double vz[V], vz2[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        vz[k] = vg[(z0 + k) % N];
        vz2[k] = 0.5 * vz[k] * vz[k];
    }
    if constexpr (sizeof(T) == 4) {
        // FP32 input: compensated FP32 sums (hi, lo) with exact products by FMA, as accurate
        // as FP64 accumulation, off GB300's slow FP64 pipe (FP64 from the block totals on)
        __shared__ float vgf[2][N], vg2f[2][N];   // v and v^2/2 as FP32 pairs hi + lo
        if (tid < N) {
            const double w = vg[tid], w2 = 0.5 * w * w;
            vgf[0][tid] = (float)w;
            vgf[1][tid] = (float)(w - (double)(float)w);
            vg2f[0][tid] = (float)w2;
            vg2f[1][tid] = (float)(w2 - (double)(float)w2);
        }
        __syncthreads();
        float vzh[V], vzl[V], vz2h[V], vz2l[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int z = (z0 + k) % N;
            vzh[k] = vgf[0][z];
            vzl[k] = vgf[1][z];
            vz2h[k] = vg2f[0][z];
            vz2l[k] = vg2f[1][z];
        }
        __shared__ float2 redf[BS / 32][5];
        for (long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
            float2 sm[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) sm[i] = make_float2(0.f, 0.f);
            if (lane_ok) {
                const T* fc = f + cell * N3 + z0;
#pragma unroll 4
                for (int j = 0; j < ROWS; ++j) {
                    const int r = r0 + RPI * j;
                    if (r >= N * N) break;
                    const VT w = __ldcs(reinterpret_cast<const VT*>(fc + (long)r * N));
                    const float* pw = reinterpret_cast<const float*>(&w);
                    float2 t0 = make_float2(0.f, 0.f), tz = t0, tzz = t0;
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        const float m = pw[k];
                        t0 = df_add1(t0, m);
                        const float p = m * vzh[k];
                        tz = df_add1(tz, p);
                        tz.y += fmaf(m, vzl[k], fmaf(m, vzh[k], -p));
                        const float q = m * vz2h[k];
                        tzz = df_add1(tzz, q);
                        tzz.y += fmaf(m, vz2l[k], fmaf(m, vz2h[k], -q));
                    }
                    const int ix = r / N, iy = r % N;
                    const float2 vx = make_float2(vgf[0][ix], vgf[1][ix]), vy = make_float2(vgf[0][iy], vgf[1][iy]);
                    const float2 v2 = df_add(make_float2(vg2f[0][ix], vg2f[1][ix]), make_float2(vg2f[0][iy], vg2f[1][iy]));
                    sm[0] = df_add(sm[0], t0);
                    sm[1] = df_add(sm[1], df_mul(t0, vx));
                    sm[2] = df_add(sm[2], df_mul(t0, vy));
                    sm[3] = df_add(sm[3], tz);
                    sm[4] = df_add(sm[4], df_add(df_mul(t0, v2), tzz));
                }
            }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sm[i] = df_add(sm[i], df_shfl_xor(sm[i], off));
            const int warp = tid >> 5;
            if ((tid & 31) == 0)
                for (int i = 0; i < 5; ++i) redf[warp][i] = sm[i];
            __syncthreads();
            if (tid < 5) {
                float2 acc = make_float2(0.f, 0.f);
                for (int w2 = 0; w2 < BS / 32; ++w2) acc = df_add(acc, redf[w2][tid]);
                U[cell * 5 + tid] = ((double)acc.x + (double)acc.y) * dv * dv * dv;
            }
            __syncthreads();
        }
        return;
    }
    for (long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
        double s[5] = {0, 0, 0, 0, 0};
        if (lane_ok) {
            const T* fc = f + cell * N3 + z0;
#pragma unroll 4
            for (int j = 0; j < ROWS; ++j) {
                const int r = r0 + RPI * j;
                if (r >= N * N) break;
                const VT w = __ldcs(reinterpret_cast<const VT*>(fc + (long)r * N));
                const T* pw = reinterpret_cast<const T*>(&w);
                double t0 = 0.0, tz = 0.0, tzz = 0.0;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const double m = (double)pw[k];
                    t0 += m;
                    tz = fma(m, vz[k], tz);
                    tzz = fma(m, vz2[k], tzz);
                }
                const double vx = vg[r / N], vy = vg[r % N];
                s[0] += t0;
                s[1] = fma(t0, vx, s[1]);
                s[2] = fma(t0, vy, s[2]);
                s[3] += tz;
                s[4] = fma(t0, 0.5 * (vx * vx + vy * vy), s[4]) + tzz;
            }
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], off);
        const int warp = tid >> 5;
        if ((tid & 31) == 0)
            for (int i = 0; i < 5; ++i) red[warp][i] = s[i];
        __syncthreads();
        if (tid < 5) {
            double acc = 0.0;
            for (int w = 0; w < BS / 32; ++w) acc += red[w][tid];
            U[cell * 5 + tid] = acc * dv * dv * dv;
        }
        __syncthreads();
    }
}

// the same gather for any n and any alignment, one element per thread
template <typename T>
__global__ void transport_any_kernel(int n, int ncx, int ncy, int ncz, int bcx, int bcy, int bcz,
                                     const signed char* __restrict__ delta, const T* __restrict__ f,
                                     T* __restrict__ out, long total) {
    const long n3 = (long)n * n * n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long cell = i / n3;
        const int k = (int)(i - cell * n3);
        const int kz = k % n, ky = (k / n) % n, kx = k / (n * n);
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
        int fx, fy, fz;
        const int sx = fold_cell(cx - delta[kx], ncx, bcx, fx);
        const int sy = fold_cell(cy - delta[n + ky], ncy, bcy, fy);
        const int sz = fold_cell(cz - delta[2 * n + kz], ncz, bcz, fz);
        const int qx = fx ? n - 1 - kx : kx;
        const int qy = fy ? n - 1 - ky : ky;
        const int qz = fz ? n - 1 - kz : kz;
        out[i] = f[(((long)sx * ncy + sy) * ncz + sz) * n3 + ((long)qx * n + qy) * n + qz];
    }
}

// transport of ncells cells: the run kernel for n = 8, 16, 24, 32 and 16-byte
// aligned arrays, the element kernel otherwise
template <typename T>
static cudaError_t launch_transport(int n, const fks_grid& g, const signed char* delta, const void* f, void* out,
                                    cudaStream_t s) {
    const long ncells = (long)g.nx * g.ny * g.nz;
    const bool al = ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    const long grid = ncells < 152L * 8 ? ncells : 152L * 8;
    const T* fi = static_cast<const T*>(f);
    T* fo = static_cast<T*>(out);
#define FKS_TRANSPORT_RUN(NN)                                                                                   \
    case NN:                                                                                                    \
        transport_kernel<T, NN><<<(unsigned)grid, 256, 0, s>>>(g.nx, g.ny, g.nz, g.bc[0], g.bc[1], g.bc[2], delta, \
                                                               fi, fo, ncells);                                 \
        return cudaGetLastError();
    if (al) {
        switch (n) {
            FKS_TRANSPORT_RUN(8)
            FKS_TRANSPORT_RUN(16)
            FKS_TRANSPORT_RUN(24)
            FKS_TRANSPORT_RUN(32)
        }
    }
#undef FKS_TRANSPORT_RUN
    const long total = ncells * n * n * n;
    long blocks = (total + 255) / 256;
    if (blocks > 152L * 64) blocks = 152L * 64;
    if (blocks < 1) blocks = 1;
    transport_any_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(n, g.nx, g.ny, g.nz, g.bc[0], g.bc[1], g.bc[2], delta, fi,
                                                             fo, total);
    return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t launch_moments_n(const fks_ctx* c, const void* f, double* U, cudaStream_t s) {
    const long grid = c->ncells < 152L * 8 ? c->ncells : 152L * 8;
    moments_kernel<T, N><<<(unsigned)grid, 256, 0, s>>>(c->vbox.L, c->ncells, static_cast<const T*>(f), U);
    return cudaGetLastError();
}
template <typename T>
static cudaError_t launch_moments_t(const fks_ctx* c, const void* f, double* U, cudaStream_t s) {
    switch (c->n) {
        case 8: return launch_moments_n<T, 8>(c, f, U, s);
        case 16: return launch_moments_n<T, 16>(c, f, U, s);
        case 24: return launch_moments_n<T, 24>(c, f, U, s);
        case 32: return launch_moments_n<T, 32>(c, f, U, s);
    }
    return cudaErrorInvalidValue;
}

// FMA-chain throughput: eight independent chains per thread keep the FMA (or
// FP64) pipe full; the sum is stored only if it hits an impossible value, so
// the chains stay live.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T b, T c, int iters, T* sink) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += a[k];
    if (sum == (T)-12345.0) sink[0] = sum;
}

int default_cluster_size(bool fp64, int N) {
    // FP32 n = 32: C = 8 measured 176.9 ms against 178.4 ms for C = 4 (32^3 x 32^3 step)
    if (!fp64) return N == 32 ? 8 : (N == 24 ? 2 : 1);
    return N == 32 ? 8 : (N == 24 ? 4 : (N == 16 ? 2 : 1));
}

bool find_collide_variant(bool fp64, int N, int C, CollideVariant* out, int radix) {
    if (radix != 0) return !fp64 && find_collide_variant_f32_radix(N, C, radix, out);
    const bool ok = fp64 ? find_collide_variant_f64(N, C, out) : find_collide_variant_f32(N, C, out);
    if (ok) out->radix = 0;
    return ok;
}

// Gauss-Legendre rule on [a, b] by Newton iteration on the Legendre recurrence
static void gl_rule(int m, double a, double b, double* x, double* w) {
    for (int i = 0; i < m; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (m + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (b - a) * z + 0.5 * (b + a);
        w[i] = (b - a) / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace fks

using namespace fks;

static fks_status fail(fks_ctx* c, fks_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

static fks_status cuda_fail(fks_ctx* c, cudaError_t e, const char* where) {
    return fail(c, FKS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FKS_CUDA(call)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

// (declared in fks_internal.h)
cudaError_t fks::query_variant(bool fp64, int n, int C, CollideVariant* v, int* max_clusters, bool* found, int radix) {
    *found = find_collide_variant(fp64, n, C, v, radix);
    if (!*found) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(v->func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(v->func_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem);
    if (e == cudaSuccess && C > 8) {   // clusters of 16 are an opt-in size
        e = cudaFuncSetAttribute(v->func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(v->func_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(v->NT, 1, 1);
    cfg.dynamicSmemBytes = v->smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    *max_clusters = 0;
    return cudaOccupancyMaxActiveClusters(max_clusters, v->func, &cfg);
}

static fks_status configure_variant(fks_ctx* c, int C, int radix = 0) {
    CollideVariant v;
    int nclus = 0;
    bool found = false;
    FKS_CUDA(query_variant(c->fp64, c->n, C, &v, &nclus, &found, radix));
    if (!found) return fail(c, FKS_ERR_UNSUPPORTED, "no collision kernel for this (precision, n, cluster size)");
    if (nclus <= 0) return fail(c, FKS_ERR_UNSUPPORTED, "collision kernel cannot be resident on this device");
    c->var = v;
    c->C = C;
    c->max_clusters = nclus;
    return FKS_OK;
}

// (declared in fks_internal.h)
fks_status fks::build_tables_raw(int n, const fks_dirs& dirs, double L, int ktype, double Ck, int C, bool fp64,
                                 void** out, std::string* err, bool full, const VhsExpansion* vx, bool dfl) {
    const int S = (ktype == FKS_VHS && vx) ? vx->S : 1;
    const int M = dirs.A1 * dirs.A2 * S, HF = n / 2 + 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> e(3 * M), w(M);
    for (int p = 0; p < dirs.A1; ++p) {
        const double t = (dirs.rule == 0 ? (p + 0.5) : (double)p) * pi / dirs.A1;
        for (int q = 0; q < dirs.A2; ++q) {
            const double fi = q * pi / dirs.A2;
            for (int term = 0; term < S; ++term) {
                const int m = (p * dirs.A2 + q) * S + term;
                e[3 * m] = std::sin(t) * std::cos(fi);
                e[3 * m + 1] = std::sin(t) * std::sin(fi);
                e[3 * m + 2] = std::cos(t);
                w[m] = pi * pi / ((double)dirs.A1 * dirs.A2) * std::sin(t);
            }
        }
    }
    if (ktype == FKS_VHS && (!vx || vx->S < 1)) {
        *err = "VHS tables need the separable expansion";
        return FKS_ERR_INVALID_ARG;
    }
    const size_t nv = ktype == FKS_VHS ? vx->r.size() + vx->ca.size() + vx->cb.size() : 0;
    const double R = 2.0 / (3.0 + std::sqrt(2.0)) * L;
    std::vector<double> gl(4 * kGL);
    gl_rule(kGL, 0.0, 0.5 * pi, gl.data(), gl.data() + kGL);
    gl_rule(kGL, 0.0, std::sqrt(R), gl.data() + 2 * kGL, gl.data() + 3 * kGL);

    double *d_e = nullptr, *d_gl = nullptr, *d_A = nullptr, *d_B = nullptr, *d_w = nullptr;
    const long half = (long)M * n * n * HF;
    const long packed = full ? (long)(M + 1) * 2 * n * n * n : (long)(M + 1) * C * 2 * n * (n / C) * HF;
    const size_t esz = fp64 ? 8 : 4;
    fks_status st = FKS_OK;
    *out = nullptr;
    cudaError_t e1 = cudaMalloc(&d_e, sizeof(double) * (3 * M + M + nv));
    cudaError_t e2 = cudaMalloc(&d_gl, sizeof(double) * 4 * kGL);
    cudaError_t e3 = cudaMalloc(&d_A, sizeof(double) * half);
    cudaError_t e4 = cudaMalloc(&d_B, sizeof(double) * half);
    cudaError_t e5 = cudaMalloc(out, esz * packed);
    if (e1 || e2 || e3 || e4 || e5) {
        *err = "cudaMalloc of spectral tables failed";
        st = alloc_failure();
    } else {
        d_w = d_e + 3 * M;
        double* d_v = d_w + M;
        cudaMemcpy(d_e, e.data(), sizeof(double) * 3 * M, cudaMemcpyHostToDevice);
        cudaMemcpy(d_w, w.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
        if (nv) {
            cudaMemcpy(d_v, vx->r.data(), sizeof(double) * vx->r.size(), cudaMemcpyHostToDevice);
            cudaMemcpy(d_v + vx->r.size(), vx->ca.data(), sizeof(double) * vx->ca.size(), cudaMemcpyHostToDevice);
            cudaMemcpy(d_v + vx->r.size() + vx->ca.size(), vx->cb.data(), sizeof(double) * vx->cb.size(),
                       cudaMemcpyHostToDevice);
        }
        cudaMemcpy(d_gl, gl.data(), sizeof(double) * 4 * kGL, cudaMemcpyHostToDevice);
        TableParams tp;
        tp.n = n;
        tp.M = M;
        tp.ktype = ktype;
        tp.HF = HF;
        tp.L = L;
        tp.R = R;
        tp.c4 = std::sqrt(4.0 * Ck);
        tp.e = d_e;
        tp.w = d_w;
        tp.glt_x = d_gl;
        tp.glt_w = d_gl + kGL;
        tp.glu_x = d_gl + 2 * kGL;
        tp.glu_w = d_gl + 3 * kGL;
        tp.vS = S;
        tp.vQ = nv ? (int)vx->r.size() : 0;
        tp.vr = d_v;
        tp.vca = d_v + tp.vQ;
        tp.vcb = d_v + tp.vQ + (nv ? vx->ca.size() : 0);
        tables_kernel<<<1024, 128>>>(tp, d_A, d_B);
        if (full)
            pack_tables_full_kernel<<<1024, 256>>>(n, M, HF, d_A, d_B, d_w, (float2*)*out);
        else if (dfl)
            pack_tables_kernel<dfloat><<<1024, 256>>>(n, M, C, HF, d_A, d_B, d_w, (dfloat*)*out);
        else if (fp64)
            pack_tables_kernel<double><<<1024, 256>>>(n, M, C, HF, d_A, d_B, d_w, (double*)*out);
        else
            pack_tables_kernel<float><<<1024, 256>>>(n, M, C, HF, d_A, d_B, d_w, (float*)*out);
        cudaError_t es = cudaDeviceSynchronize();
        if (es != cudaSuccess) {
            *err = std::string("table construction: ") + cudaGetErrorString(es);
            st = FKS_ERR_CUDA;
        }
    }
    cudaFree(d_e);
    cudaFree(d_gl);
    cudaFree(d_A);
    cudaFree(d_B);
    if (st != FKS_OK && *out) {
        cudaFree(*out);
        *out = nullptr;
    }
    return st;
}

static fks_status build_tables(fks_ctx* c) {
    std::string err;
    fks_status st = build_tables_raw(c->n, c->dirs, c->vbox.L, c->kern.type, c->kern.C, c->C, c->fp64, &c->tables, &err,
                                     c->tc, &c->vhs);
    c->launches += 2;
    if (st != FKS_OK) return fail(c, st, err);
    return FKS_OK;
}

// Precision escalation of an FP32 or split-BF16 context: the tiers that recompute the cells whose
// error bound exceeds the tolerance (FP32 context: FP64 arithmetic; split-BF16 context: FP32, then
// FP64), each with its own tables, and the device lists that connect them.  Kernels without tiers
// (BGK, the separable VHS expansion, variant B's inner grid) keep their own arithmetic.
static fks_status setup_escalation(fks_ctx* c) {
    if (c->fp64 || c->bgk || c->kern.type == FKS_VHS) return FKS_OK;
    int k = 0;
    auto add_tier = [&](bool fp64) -> fks_status {
        EscTier& t = c->esc[k];
        if (t.tables) cudaFree(t.tables);
        t = EscTier{};
        t.fp64 = fp64;
        t.dfl = fp64 && c->esc_arith == FKS_FP32X2;
        t.C = default_cluster_size(fp64, c->n);
        const bool found = !fp64 ? find_collide_variant_f32(c->n, t.C, &t.var)
                                 : (t.dfl ? find_collide_variant_dfloat(c->n, t.C, &t.var)
                                          : find_collide_variant_mixed(c->n, t.C, &t.var));
        if (!found) return fail(c, FKS_ERR_UNSUPPORTED, "no escalation kernel for this n");
        cudaError_t e = cudaFuncSetAttribute(t.var.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.var.smem);
        if (e == cudaSuccess && t.C > 8) e = cudaFuncSetAttribute(t.var.func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cuda_fail(c, e, "escalation kernel attributes");
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = t.C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(t.C, 1, 1);
        cfg.blockDim = dim3(t.var.NT, 1, 1);
        cfg.dynamicSmemBytes = t.var.smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&t.max_clusters, t.var.func, &cfg);
        if (e != cudaSuccess) return cuda_fail(c, e, "escalation kernel occupancy");
        if (t.max_clusters <= 0) return fail(c, FKS_ERR_UNSUPPORTED, "escalation kernel cannot be resident");
        std::string err;
        const fks_status st = build_tables_raw(c->n, c->dirs, c->vbox.L, c->kern.type, c->kern.C, t.C, fp64, &t.tables,
                                               &err, false, nullptr, t.dfl);
        if (st != FKS_OK) return fail(c, st, err);
        ++k;
        return FKS_OK;
    };
    fks_status st = FKS_OK;
    if (c->tc) st = add_tier(false);
    if (st == FKS_OK) st = add_tier(true);
    if (st != FKS_OK) return st;
    const long nl = c->ncells > 0 ? c->ncells : 1;
    if (!c->esc_lists) {
        if (cudaMalloc(&c->esc_lists, sizeof(int) * 2 * nl) != cudaSuccess ||
            cudaMalloc(&c->esc_counts, sizeof(int) * 2) != cudaSuccess)
            return fail(c, alloc_failure(), "escalation lists");
        if (cudaMemset(c->esc_counts, 0, sizeof(int) * 2) != cudaSuccess)
            return fail(c, FKS_ERR_CUDA, "escalation lists");
        c->esc_tol = c->tc ? 1e-3 : 1e-5;   // the stated relative L2 bounds of Q (split BF16, FP32)
    }
    c->esc_ntier = k;
    return FKS_OK;
}

// P = (sum_k phi(v_k) phi(v_k)^T)^-1, phi = (1, v, |v|^2/2): the projection
// Q -= C^T (C C^T)^-1 C Q with C = dv^3 phi^T becomes Q -= phi^T P (phi^T Q)
void fks::projection_matrix(int n, double L, double* P) {
    const double dv = 2.0 * L / n;
    double A[5][10];
    std::memset(A, 0, sizeof(A));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                const double vx = (i + 0.5 - 0.5 * n) * dv, vy = (j + 0.5 - 0.5 * n) * dv, vz = (k + 0.5 - 0.5 * n) * dv;
                const double ph[5] = {1.0, vx, vy, vz, 0.5 * (vx * vx + vy * vy + vz * vz)};
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) A[a][b] += ph[a] * ph[b];
            }
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) A[a][5 + b] = (a == b) ? 1.0 : 0.0;
    for (int col = 0; col < 5; ++col) {   // Gauss-Jordan with partial pivoting
        int piv = col;
        for (int r = col + 1; r < 5; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int t = 0; t < 10; ++t) std::swap(A[col][t], A[piv][t]);
        const double d = A[col][col];
        for (int t = 0; t < 10; ++t) A[col][t] /= d;
        for (int r = 0; r < 5; ++r) {
            if (r == col) continue;
            const double fct = A[r][col];
            for (int t = 0; t < 10; ++t) A[r][t] -= fct * A[col][t];
        }
    }
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) P[a * 5 + b] = A[a][5 + b];
}

// DFT matrices and per-CTA scratch of the tensor-core path (one CTA per SM)
static fks_status setup_tc(fks_ctx* c) {
    std::vector<uint16_t> h;
    tc_dft_matrices(c->n, h);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->tc_grid = sms > 0 ? sms : 1;
    const size_t scratch = (size_t)c->tc_grid * tc_scratch_per_cta(c->n);
    if (cudaMalloc(&c->tc_dft, h.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&c->tc_scratch, scratch) != cudaSuccess)
        return fail(c, alloc_failure(), "tensor-core scratch");
    if (cudaMemcpy(c->tc_dft, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(c, FKS_ERR_CUDA, "DFT matrix upload");
    return FKS_OK;
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing
// arrives at, with the helper every kernel uses, and records the timeout bit.
__global__ void selftest_wait_kernel(long polls, int* flags) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_wait_bounded(&bar, 0, flags, polls);
}

extern "C" {

const char* fks_status_string(fks_status s) {
    switch (s) {
        case FKS_OK: return "ok";
        case FKS_ERR_INVALID_ARG: return "invalid argument";
        case FKS_ERR_UNSUPPORTED: return "unsupported configuration";
        case FKS_ERR_OOM: return "out of device memory";
        case FKS_ERR_CUDA: return "CUDA error";
        case FKS_ERR_NUMERIC: return "numerical health check failed";
        case FKS_ERR_TIMEOUT: return "timeout";
    }
    return "unknown";
}

fks_status fks_init(const fks_grid* grid, const fks_vbox* vbox, const fks_kernel* kernel, const fks_dirs* dirs,
                    int precision, fks_ctx** out) {
    if (out) *out = nullptr;
    if (!grid || !vbox || !kernel || !dirs || !out) return FKS_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return FKS_ERR_INVALID_ARG;
    if ((long)grid->nx * grid->ny * grid->nz >= (1L << 31)) return FKS_ERR_INVALID_ARG;   // 32-bit cell indices
    for (int a = 0; a < 3; ++a) {
        if (!(grid->x1[a] > grid->x0[a])) return FKS_ERR_INVALID_ARG;
        if (grid->bc[a] != FKS_BC_PERIODIC && grid->bc[a] != FKS_BC_SPECULAR) return FKS_ERR_INVALID_ARG;
    }
    if (!(vbox->L > 0.0) || !std::isfinite(vbox->L)) return FKS_ERR_INVALID_ARG;
    if (vbox->n != 8 && vbox->n != 16 && vbox->n != 24 && vbox->n != 32) return FKS_ERR_UNSUPPORTED;
    if (kernel->type != FKS_HARD_SPHERE && kernel->type != FKS_MAXWELL && kernel->type != FKS_BGK &&
        kernel->type != FKS_VHS)
        return FKS_ERR_INVALID_ARG;
    if (kernel->type == FKS_VHS &&
        (!(kernel->alpha >= -1.0 && kernel->alpha <= 1.0) || kernel->terms < 0 || kernel->terms > kVhsMaxTerms))
        return FKS_ERR_INVALID_ARG;
    if (!(kernel->C > 0.0) || !(kernel->knudsen > 0.0)) return FKS_ERR_INVALID_ARG;
    if (dirs->A1 < 1 || dirs->A2 < 1 || dirs->A1 * dirs->A2 > 4096 || (dirs->rule != 0 && dirs->rule != 1))
        return FKS_ERR_INVALID_ARG;
    if (precision != FKS_FP64 && precision != FKS_FP32 && precision != FKS_BF16X3) return FKS_ERR_UNSUPPORTED;
    if (precision == FKS_BF16X3 && (kernel->type == FKS_BGK || (vbox->n != 16 && vbox->n != 32)))
        return FKS_ERR_UNSUPPORTED;

    fks_ctx* c = new (std::nothrow) fks_ctx();
    if (!c) return FKS_ERR_OOM;
    c->grid = *grid;
    c->vbox = *vbox;
    c->kern = *kernel;
    c->dirs = *dirs;
    c->fp64 = precision == FKS_FP64;
    c->n = vbox->n;
    c->M = dirs->A1 * dirs->A2;
    c->ncells = (long)grid->nx * grid->ny * grid->nz;
    const int nca[3] = {grid->nx, grid->ny, grid->nz};
    for (int a = 0; a < 3; ++a) c->dx[a] = (grid->x1[a] - grid->x0[a]) / nca[a];
    cudaGetDevice(&c->device);
    c->bgk = kernel->type == FKS_BGK;
    c->tc = precision == FKS_BF16X3;
    fks_status st = FKS_OK;
    if (kernel->type == FKS_VHS) {
        // the separable terms, each one more table pair per direction
        st = vhs_expand(kernel->alpha, kernel->C, vbox->L, vbox->n, vhs_tolerance(precision), kernel->terms, &c->vhs,
                        &c->err);
        if (st == FKS_OK && (long)c->M * c->vhs.S > 4096) st = fail(c, FKS_ERR_UNSUPPORTED, "A1 A2 x VHS terms > 4096");
        if (st == FKS_OK) c->M *= c->vhs.S;
    }
    if (st != FKS_OK) {
        std::fprintf(stderr, "fks_init: %s\n", c->err.c_str());
        fks_destroy(c);
        return st;
    }
    if (c->tc) {
        c->C = 1;
        st = build_tables(c);
        if (st == FKS_OK) st = setup_tc(c);
    } else if (!c->bgk) {
        st = configure_variant(c, default_cluster_size(c->fp64, c->n));
        if (st == FKS_OK) st = build_tables(c);
    } else {
        c->C = 1;
    }
    if (st == FKS_OK) st = setup_escalation(c);
    if (st == FKS_OK) {
        if (cudaMalloc(&c->d_s, sizeof(double) * 3 * c->n) != cudaSuccess ||
            cudaMalloc(&c->d_delta, 3 * c->n) != cudaSuccess || cudaMalloc(&c->d_flags, sizeof(int)) != cudaSuccess)
            st = alloc_failure();
        else if (cudaMemset(c->d_s, 0, sizeof(double) * 3 * c->n) != cudaSuccess ||
                 cudaMemset(c->d_delta, 0, 3 * c->n) != cudaSuccess || cudaMemset(c->d_flags, 0, sizeof(int)) != cudaSuccess)
            st = FKS_ERR_CUDA;
    }
    if (st != FKS_OK) {
        std::fprintf(stderr, "fks_init: %s\n", c->err.c_str());
        fks_destroy(c);
        return st;
    }
    projection_matrix(c->n, c->vbox.L, c->P);
    if (cudaMalloc(&c->d_P, sizeof(c->P)) != cudaSuccess ||
        cudaMemcpy(c->d_P, c->P, sizeof(c->P), cudaMemcpyHostToDevice) != cudaSuccess) {
        const fks_status st2 = alloc_failure();
        fks_destroy(c);
        return st2;
    }
    *out = c;
    return FKS_OK;
}

void fks_destroy(fks_ctx* c) {
    if (!c) return;
    if (c->dealias) fks_set_dealias(c, 0);
    if (c->h_in) {
        cudaDeviceSynchronize();
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 64; ++i)
                if (c->h_ev[k][i]) cudaEventDestroy(c->h_ev[k][i]);
        if (c->h_up) cudaStreamDestroy(c->h_up);
        if (c->h_down) cudaStreamDestroy(c->h_down);
        cudaFree(c->h_in);
        cudaFree(c->h_out);
    }
    cudaFree(c->tables);
    cudaFree(c->tc_dft);
    cudaFree(c->tc_scratch);
    cudaFree(c->d_s);
    cudaFree(c->d_delta);
    cudaFree(c->d_flags);
    cudaFree(c->d_P);
    cudaFree(c->s_rho);
    cudaFree(c->s_dist);
    cudaFree(c->s_ind);
    cudaFree(c->s_cells);
    cudaFree(c->s_cand);
    cudaFree(c->s_count);
    for (int i = 0; i < 2; ++i) cudaFree(c->esc[i].tables);
    for (int k = 0; k < 3; ++k)
        for (cudaEvent_t e : c->prof_ev[k]) cudaEventDestroy(e);
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    cudaFree(c->esc_lists);
    cudaFree(c->esc_counts);
    delete c;
}

const char* fks_last_error(const fks_ctx* c) { return c ? c->err.c_str() : "null context"; }
long fks_ncells(const fks_ctx* c) { return c ? c->ncells : -1; }
int fks_nv(const fks_ctx* c) { return c ? c->n * c->n * c->n : -1; }
int fks_cluster_size(const fks_ctx* c) { return c ? c->C : -1; }
long fks_launch_count(const fks_ctx* c) { return c ? c->launches : -1; }

fks_status fks_set_schedule(fks_ctx* c, int C, int radix) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (c->bgk) return fail(c, FKS_ERR_UNSUPPORTED, "the BGK kernel has no cluster size");
    if (c->tc) return fail(c, FKS_ERR_UNSUPPORTED, "the tensor-core kernel has no cluster size");
    if (c->dealias) return fks_set_schedule(c->inner, C, radix);   // the 2n kernel does the transforms
    if (C == c->C && radix == c->var.radix) return FKS_OK;
    CollideVariant v;
    if (!find_collide_variant(c->fp64, c->n, C, &v, radix))
        return fail(c, FKS_ERR_UNSUPPORTED, "no kernel for this cluster size and radix schedule");
    cudaDeviceSynchronize();
    const bool retable = C != c->C;   // tables are laid out per cluster rank
    fks_status st = configure_variant(c, C, radix);
    if (st == FKS_OK && retable) {
        cudaFree(c->tables);
        c->tables = nullptr;
        st = build_tables(c);
    }
    return st;
}

fks_status fks_set_cluster_size(fks_ctx* c, int C) { return fks_set_schedule(c, C, 0); }

int fks_radix(const fks_ctx* c) { return c ? c->var.radix : -1; }


static fks_status launch_bgk_ctx(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                                 cudaStream_t s, long cell0 = 0, long cell1 = -1, const void* base = nullptr) {
    BgkArgs a;
    a.base = base;
    a.f = f;
    a.out = out;
    a.delta = delta;
    a.flags = c->d_flags;
    a.ncells = cell1 >= 0 ? cell1 : c->ncells;
    a.cell0 = cell0;
    a.nc[0] = c->grid.nx;
    a.nc[1] = c->grid.ny;
    a.nc[2] = c->grid.nz;
    for (int i = 0; i < 3; ++i) a.bc[i] = c->grid.bc[i];
    a.L = c->vbox.L;
    a.inv_kn = 1.0 / c->kern.knudsen;
    a.dt = dt;
    a.mode = mode;
    std::memcpy(a.P, c->P, sizeof(a.P));
    cudaError_t e = launch_bgk(c->fp64, c->n, a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "BGK kernel launch");
    c->launches += 1;
    return FKS_OK;
}

static bool esc_on(const fks_ctx* c) { return c->esc_tol > 0.0 && c->esc_ntier > 0; }

// stage timing: an event before and after a launch of stage `stage` on stream s
static cudaEvent_t prof_event(fks_ctx* c) {
    cudaEvent_t e = nullptr;
    if (!c->prof_pool.empty()) {
        e = c->prof_pool.back();
        c->prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}
static void prof_mark(fks_ctx* c, int stage, cudaStream_t s) {
    if (!c->prof) return;
    cudaEvent_t e = prof_event(c);
    if (e && cudaEventRecord(e, s) == cudaSuccess) c->prof_ev[stage].push_back(e);
}

static fks_status launch_tc_ctx(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                                cudaStream_t s, const int* cells = nullptr, long ncells = -1,
                                const int* cells_count = nullptr) {
    TcLaunch l;
    l.cells_count = cells_count;
    if (esc_on(c)) {
        l.esc_list = c->esc_lists;
        l.esc_count = c->esc_counts;
        l.esc_c2 = kEscBf16 * kEscBf16;
        l.esc_tol2 = c->esc_tol * c->esc_tol;
        // A cell whose FP32 bound must exceed the tolerance is listed for the last tier at once: with
        // |q_b - q| <= c_b l and |q_32 - q| <= c_32 l (q = ||Q_proj||, l = ||L|| / Kn; b: this kernel,
        // 32: the FP32 tier), c_32 l > tol q_32 holds whenever (c_32 - tol (c_b + c_32)) l > tol q_b;
        // 0.9 of that constant covers the tiers' different estimates of ||L||.  The last tier
        // recomputes from f*, so the results are those of the route through the FP32 tier.
        const double cd = 0.9 * (kEscFp32 - c->esc_tol * (kEscBf16 + kEscFp32));
        if (c->esc_direct && c->esc_ntier == 2 && cd > 0.0) {
            l.esc_last_list = c->esc_lists + c->ncells;
            l.esc_last_count = c->esc_counts + 1;
            l.esc_last_c2 = cd * cd;
        }
    }
    l.f = f;
    l.out = out;
    l.tables = c->tables;
    l.dft = c->tc_dft;
    l.scratch = c->tc_scratch;
    l.delta = delta;
    l.flags = c->d_flags;
    l.ncells = ncells >= 0 ? ncells : c->ncells;
    l.cells = cells;
    l.nc[0] = c->grid.nx;
    l.nc[1] = c->grid.ny;
    l.nc[2] = c->grid.nz;
    for (int i = 0; i < 3; ++i) l.bc[i] = c->grid.bc[i];
    l.M = c->M;
    l.L = c->vbox.L;
    l.inv_kn = 1.0 / c->kern.knudsen;
    l.dt = dt;
    l.mode = mode;
    std::memcpy(l.P, c->P, sizeof(l.P));
    l.grid = c->tc_grid;
    cudaError_t e = launch_collide_tc(c->n, l, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core collision kernel launch");
    c->launches += 1;
    return FKS_OK;
}

// arguments of the cluster kernel for a context (tables: the context's own or an escalation tier's)
static CollideArgs cluster_args(const fks_ctx* c, const void* tables, const void* f, void* out, const signed char* delta,
                                double dt, int mode, long cell0, long cell1, const void* base) {
    CollideArgs a;
    std::memset(&a, 0, sizeof(a));
    a.base = base;
    a.f = f;
    a.out = out;
    a.tables = tables;
    a.delta = delta;
    a.flags = c->d_flags;
    a.ncells = cell1;
    a.cell0 = cell0;
    a.nc[0] = c->grid.nx;
    a.nc[1] = c->grid.ny;
    a.nc[2] = c->grid.nz;
    for (int i = 0; i < 3; ++i) a.bc[i] = c->grid.bc[i];
    a.M = c->M;
    a.L = c->vbox.L;
    a.inv_kn = 1.0 / c->kern.knudsen;
    a.dt = dt;
    a.mode = mode;
    std::memcpy(a.P, c->P, sizeof(a.P));
    a.items = nullptr;
    return a;
}

// persistent launch of one cluster-kernel instantiation over `work` cells (at most max_clusters clusters)
static cudaError_t launch_cluster(const CollideVariant& var, int C, int max_clusters, const CollideArgs& a, long work,
                                  cudaStream_t s) {
    const long nclus = work < max_clusters ? work : max_clusters;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nclus * C), 1, 1);
    cfg.blockDim = dim3(var.NT, 1, 1);
    cfg.dynamicSmemBytes = var.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CollideArgs arg = a;
    void* args[] = {&arg};
    return cudaLaunchKernelExC(&cfg, var.func, args);
}

// the escalation tiers after a launch of the context's own kernel: tier i recomputes the cells the
// launch before it listed (device count: no host synchronisation) and lists its own failures
static fks_status launch_esc_tiers(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                                   cudaStream_t s, const void* base) {
    for (int i = 0; i < c->esc_ntier; ++i) {
        const EscTier& t = c->esc[i];
        CollideArgs a = cluster_args(c, t.tables, f, out, delta, dt, mode, 0, c->ncells, base);
        a.list = c->esc_lists + (long)i * c->ncells;
        a.list_count = c->esc_counts + i;
        if (i + 1 < c->esc_ntier) {
            a.esc_list = c->esc_lists + (long)(i + 1) * c->ncells;
            a.esc_count = c->esc_counts + i + 1;
            a.esc_c2 = kEscFp32 * kEscFp32;
            a.esc_tol2 = c->esc_tol * c->esc_tol;
        }
        prof_mark(c, 1 + i, s);
        const cudaError_t e = launch_cluster(t.var, t.C, t.max_clusters, a, c->ncells, s);
        prof_mark(c, 1 + i, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "escalation kernel launch");
        c->launches += 1;
    }
    return FKS_OK;
}

static fks_status reset_esc(fks_ctx* c, cudaStream_t s) {
    if (cudaMemsetAsync(c->esc_counts, 0, sizeof(int) * 2, s) != cudaSuccess)
        return fail(c, FKS_ERR_CUDA, "escalation counts");
    return FKS_OK;
}

// collision of the cells [cell0, cell1) (cell1 < 0: all); ranges other than
// all cells are for the cluster and BGK kernels
static fks_status launch_collide(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                                 cudaStream_t s, long cell0 = 0, long cell1 = -1, const void* base = nullptr) {
    if (c->bgk) return launch_bgk_ctx(c, f, out, delta, dt, mode, s, cell0, cell1, base);
    if (c->dealias) return launch_dealias(c, f, out, delta, dt, mode, s);
    const bool esc = esc_on(c);
    if (esc) {
        const fks_status st = reset_esc(c, s);
        if (st != FKS_OK) return st;
    }
    if (c->tc) {
        prof_mark(c, 0, s);
        const fks_status st = launch_tc_ctx(c, f, out, delta, dt, mode, s);
        prof_mark(c, 0, s);
        if (st != FKS_OK || !esc) return st;
        return launch_esc_tiers(c, f, out, delta, dt, mode, s, base);
    }
    if (cell1 < 0) cell1 = c->ncells;
    if (cell1 <= cell0) return FKS_OK;
    CollideArgs a = cluster_args(c, c->tables, f, out, delta, dt, mode, cell0, cell1, base);
    if (esc) {
        a.esc_list = c->esc_lists;
        a.esc_count = c->esc_counts;
        a.esc_c2 = kEscFp32 * kEscFp32;
        a.esc_tol2 = c->esc_tol * c->esc_tol;
    }
    prof_mark(c, 0, s);
    const cudaError_t e = launch_cluster(c->var, c->C, c->max_clusters, a, cell1 - cell0, s);
    prof_mark(c, 0, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "collision kernel launch");
    c->launches += 1;
    if (!esc) return FKS_OK;
    return launch_esc_tiers(c, f, out, delta, dt, mode, s, base);
}

fks_status fks_internal_fail(fks_ctx* c, fks_status st, const std::string& msg) { return fail(c, st, msg); }
fks_status fks_internal_last_tier_route(fks_ctx* c, cudaStream_t s, int** list, int** count, double* d_max,
                                        int** mid_list, int** mid_count, double* d_mid) {
    *list = nullptr;
    *count = nullptr;
    *d_max = 0.0;
    *mid_list = nullptr;
    *mid_count = nullptr;
    *d_mid = 0.0;
    if (!esc_on(c)) return FKS_OK;
    const fks_status st = reset_esc(c, s);
    if (st != FKS_OK) return st;
    const int last = c->esc_ntier - 1;
    *list = c->esc_lists + (long)last * c->ncells;
    *count = c->esc_counts + last;
    if (!c->esc_direct) return FKS_OK;
    // the last tier: the FP32 bound is the binding one (the split-BF16 bound is 30x looser)
    *d_max = kKappaDist * kEscFp32 / c->esc_tol;
    if (c->tc && c->esc_ntier == 2) {
        // the FP32 tier (first of two): cells the split-BF16 bound must fail
        *mid_list = c->esc_lists;
        *mid_count = c->esc_counts;
        *d_mid = kKappaDist * kEscBf16 / c->esc_tol;
    }
    return FKS_OK;
}

fks_status fks_internal_collide_list(fks_ctx* c, const void* f, void* out, const int* cells, const int* count,
                                     int mode, double dt, cudaStream_t s, int keep_counts) {
    if (c->bgk || c->dealias) return fail(c, FKS_ERR_UNSUPPORTED, "cell lists need a spectral context (variant A)");
    const bool esc = esc_on(c);
    if (esc && !keep_counts) {
        const fks_status st = reset_esc(c, s);
        if (st != FKS_OK) return st;
    }
    if (c->tc) {
        prof_mark(c, 0, s);
        const fks_status st = launch_tc_ctx(c, f, out, nullptr, dt, mode, s, cells, c->ncells, count);
        prof_mark(c, 0, s);
        if (st != FKS_OK) return st;
    } else {
        CollideArgs a = cluster_args(c, c->tables, f, out, nullptr, dt, mode, 0, c->ncells, nullptr);
        a.list = cells;
        a.list_count = count;
        if (esc) {
            a.esc_list = c->esc_lists;
            a.esc_count = c->esc_counts;
            a.esc_c2 = kEscFp32 * kEscFp32;
            a.esc_tol2 = c->esc_tol * c->esc_tol;
        }
        prof_mark(c, 0, s);
        const cudaError_t e = launch_cluster(c->var, c->C, c->max_clusters, a, c->ncells, s);
        prof_mark(c, 0, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "collision kernel launch");
        c->launches += 1;
    }
    return esc ? launch_esc_tiers(c, f, out, nullptr, dt, mode, s, nullptr) : FKS_OK;
}
fks_status fks_internal_collide(fks_ctx* c, const void* f, void* out, int mode, cudaStream_t s) {
    return launch_collide(c, f, out, nullptr, 0.0, mode, s);
}

static fks_status launch_offsets(fks_ctx* c, double dt, cudaStream_t s) {
    if (!std::isfinite(dt)) return fail(c, FKS_ERR_INVALID_ARG, "dt must be finite");
    const double vmax = c->vbox.L;
    for (int a = 0; a < 3; ++a)
        if (std::fabs(vmax * dt) > 100.0 * c->dx[a]) return fail(c, FKS_ERR_INVALID_ARG, "dt moves particles more than 100 cells");
    offsets_kernel<<<dim3(1, 3), c->n / 2, 0, s>>>(c->n, c->vbox.L, make_double3(c->dx[0], c->dx[1], c->dx[2]), dt, c->d_s,
                                                 c->d_delta, c->d_flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "offsets kernel launch");
    c->launches += 1;
    return FKS_OK;
}

fks_status fks_collide(fks_ctx* c, const void* f, void* Q, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !Q || !aligned16(f) || !aligned16(Q)) return fail(c, FKS_ERR_INVALID_ARG, "f and Q must be 16-byte aligned device pointers");
    if (f == Q) return fail(c, FKS_ERR_INVALID_ARG, "f and Q must not alias");
    if (c->ncells == 0) return FKS_OK;
    return launch_collide(c, f, Q, nullptr, 0.0, 0, (cudaStream_t)stream);
}

// offsets over dt, then the transport gather f -> f_out
static fks_status transport_ctx(fks_ctx* c, const void* f, void* f_out, double dt, cudaStream_t s) {
    fks_status st = launch_offsets(c, dt, s);
    if (st != FKS_OK) return st;
    if (c->ncells == 0) return FKS_OK;
    const cudaError_t e0 = c->fp64 ? launch_transport<double>(c->n, c->grid, c->d_delta, f, f_out, s)
                                   : launch_transport<float>(c->n, c->grid, c->d_delta, f, f_out, s);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "transport kernel launch");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "transport kernel launch");
    c->launches += 1;
    return FKS_OK;
}

fks_status fks_transport(fks_ctx* c, const void* f, void* f_out, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !f_out || f == f_out) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must be distinct device pointers");
    return transport_ctx(c, f, f_out, dt, (cudaStream_t)stream);
}

// Second-order step: Strang splitting T(dt/2) C(dt) T(dt/2) with the collision
// sub-step by Heun's method (the second-order explicit Runge-Kutta analogue of
// Eq. disc_relax):  a = T(dt/2) f,  b = a + dt Q(a),  c = (a + b + dt Q(b)) / 2,
// f_out = T(dt/2) c.  work holds a and then c (the second stage writes over its
// own base element by element).
fks_status fks_step_strang(fks_ctx* c, const void* f, void* f_out, void* work, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !f_out || !work || !aligned16(f) || !aligned16(f_out) || !aligned16(work))
        return fail(c, FKS_ERR_INVALID_ARG, "f, f_out and work must be 16-byte aligned device pointers");
    if (f == f_out || f == work || f_out == work) return fail(c, FKS_ERR_INVALID_ARG, "f, f_out and work must be distinct");
    if (c->tc || c->dealias)
        return fail(c, FKS_ERR_UNSUPPORTED, "the Strang step runs on the FP64/FP32 spectral and BGK kernels");
    if (!std::isfinite(dt)) return fail(c, FKS_ERR_INVALID_ARG, "dt must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = transport_ctx(c, f, work, 0.5 * dt, s);
    if (st == FKS_OK && c->ncells > 0) st = launch_collide(c, work, f_out, nullptr, dt, 1, s);
    if (st == FKS_OK && c->ncells > 0) st = launch_collide(c, f_out, work, nullptr, dt, 3, s, 0, -1, work);
    if (st == FKS_OK) st = transport_ctx(c, work, f_out, 0.5 * dt, s);
    return st;
}

// Exponential steps.  BGK: the relaxation df/dt = Q(f) = nu (M[f] - f) - phi.mu keeps M[f], nu and
// the projection term fixed over the step (collision invariants), so its exact solution from f* is
// f* + (1 - e^{-nu dt}) / nu Q(f*): stable for any nu dt, and it reaches M[f*] as Kn -> 0.
// Spectral operator: the gain-loss split df/dt = G(f) - nu(f) f (nu the loss frequency) with G and nu
// frozen at f* is solved exactly per velocity point, f* + dt phi(nu dt) (G - nu f*), phi(x) =
// (1 - e^-x) / x, and the increment projected; bounded for any nu dt (f* + (G - nu f*) / nu = G / nu
// in the stiff limit), first order in dt like the Euler step it reduces to as nu dt -> 0.
fks_status fks_step_exp(fks_ctx* c, const void* f, void* f_out, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !f_out || !aligned16(f) || !aligned16(f_out)) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must be 16-byte aligned device pointers");
    if (f == f_out) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must not alias");
    if (c->tc || c->dealias)
        return fail(c, FKS_ERR_UNSUPPORTED, "the exponential step runs on the BGK and the FP64/FP32 spectral kernels");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(c, FKS_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = launch_offsets(c, dt, s);
    if (st != FKS_OK) return st;
    if (c->ncells == 0) return FKS_OK;
    return launch_collide(c, f, f_out, c->d_delta, dt, 4, s);
}

// The collision sub-step alone (space-homogeneous cells): f_out = f + dt Q(f), mode 1 without shifts.
fks_status fks_relax(fks_ctx* c, const void* f, void* f_out, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !f_out || !aligned16(f) || !aligned16(f_out)) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must be 16-byte aligned device pointers");
    if (f == f_out) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must not alias");
    if (!std::isfinite(dt)) return fail(c, FKS_ERR_INVALID_ARG, "dt must be finite");
    if (c->ncells == 0) return FKS_OK;
    return launch_collide(c, f, f_out, nullptr, dt, 1, (cudaStream_t)stream);
}

fks_status fks_step(fks_ctx* c, const void* f, void* f_out, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !f_out || !aligned16(f) || !aligned16(f_out)) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must be 16-byte aligned device pointers");
    if (f == f_out) return fail(c, FKS_ERR_INVALID_ARG, "f and f_out must not alias");
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = launch_offsets(c, dt, s);
    if (st != FKS_OK) return st;
    if (c->ncells == 0) return FKS_OK;
    return launch_collide(c, f, f_out, c->d_delta, dt, 1, s);
}

// One step with host arrays, pipelined over chunks of x-slabs: upload (stream
// h_up), step of a chunk once every slab its transport can reach has landed
// (the caller's stream), download (stream h_down) as soon as it is done.
fks_status fks_step_host(fks_ctx* c, const void* host_f, void* host_out, double dt, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!host_f || !host_out || host_f == host_out) return fail(c, FKS_ERR_INVALID_ARG, "host arrays must be distinct");
    if (c->ncells == 0) return FKS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t esz = c->fp64 ? 8 : 4;
    const long n3 = (long)c->n * c->n * c->n;
    const size_t bytes = esz * (size_t)c->ncells * n3;
    if (!c->h_in) {
        if (cudaMalloc(&c->h_in, bytes) != cudaSuccess || cudaMalloc(&c->h_out, bytes) != cudaSuccess)
            return fail(c, alloc_failure(), "device copies of the state");
        if (cudaStreamCreateWithFlags(&c->h_up, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->h_down, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, FKS_ERR_CUDA, "copy streams");
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 64; ++i)
                if (cudaEventCreateWithFlags(&c->h_ev[k][i], cudaEventDisableTiming) != cudaSuccess)
                    return fail(c, FKS_ERR_CUDA, "events");
    }
    fks_status st = launch_offsets(c, dt, s);
    if (st != FKS_OK) return st;
    // chunks of whole x-slabs (the cluster and BGK kernels take cell ranges; the others one chunk)
    const int nx = c->grid.nx;
    const long slab = (long)c->grid.ny * c->grid.nz;
    const int nchunk = (c->tc || c->dealias) ? 1 : (nx < 8 ? nx : 8);
    auto chunk_of = [&](int x) { return (int)((long)x * nchunk / nx); };
    auto first_slab = [&](int k) { return (int)(((long)k * nx + nchunk - 1) / nchunk); };
    // shifts along x reach at most floor(L |dt| / dx) + 1 cells (|offset| < dx/2, |v| < L)
    const int reach = (int)std::floor(c->vbox.L * std::fabs(dt) / c->dx[0]) + 1;
    const char* hf = static_cast<const char*>(host_f);
    char* ho = static_cast<char*>(host_out);
    char* din = static_cast<char*>(c->h_in);
    char* dout = static_cast<char*>(c->h_out);
    cudaEvent_t* up = c->h_ev[0];
    cudaEvent_t* done = c->h_ev[1];
    cudaEvent_t* down = c->h_ev[2];
    // the copy streams start after the caller's earlier work (ordering of the host arrays)
    if (cudaEventRecord(down[63], s) != cudaSuccess || cudaStreamWaitEvent(c->h_up, down[63], 0) != cudaSuccess ||
        cudaStreamWaitEvent(c->h_down, down[63], 0) != cudaSuccess)
        return fail(c, FKS_ERR_CUDA, "stream order");
    for (int k = 0; k < nchunk; ++k) {
        const long c0 = (long)first_slab(k) * slab, c1 = (long)first_slab(k + 1) * slab;
        if (cudaMemcpyAsync(din + c0 * n3 * esz, hf + c0 * n3 * esz, (c1 - c0) * n3 * esz, cudaMemcpyHostToDevice,
                            c->h_up) != cudaSuccess ||
            cudaEventRecord(up[k], c->h_up) != cudaSuccess)
            return fail(c, FKS_ERR_CUDA, "upload");
    }
    for (int k = 0; k < nchunk; ++k) {
        const int a = first_slab(k), b = first_slab(k + 1);
        // every upload chunk a slab of [a - reach, b - 1 + reach] folds into
        bool need[64] = {};
        for (int x = a - reach; x <= b - 1 + reach; ++x) {
            int xf = x;
            if (c->grid.bc[0] == FKS_BC_PERIODIC) {
                xf = ((x % nx) + nx) % nx;
            } else {
                const int per = 2 * nx;
                int r = ((x % per) + per) % per;
                xf = r >= nx ? per - 1 - r : r;
            }
            need[chunk_of(xf)] = true;
            if (nchunk == 1) break;
        }
        for (int j = 0; j < nchunk; ++j)
            if (need[j] && cudaStreamWaitEvent(s, up[j], 0) != cudaSuccess) return fail(c, FKS_ERR_CUDA, "wait upload");
        st = nchunk == 1 ? launch_collide(c, din, dout, c->d_delta, dt, 1, s)
                         : launch_collide(c, din, dout, c->d_delta, dt, 1, s, (long)a * slab, (long)b * slab);
        if (st != FKS_OK) return st;
        if (cudaEventRecord(done[k], s) != cudaSuccess || cudaStreamWaitEvent(c->h_down, done[k], 0) != cudaSuccess)
            return fail(c, FKS_ERR_CUDA, "step event");
        const long c0 = (long)a * slab, c1 = (long)b * slab;
        if (cudaMemcpyAsync(ho + c0 * n3 * esz, dout + c0 * n3 * esz, (c1 - c0) * n3 * esz, cudaMemcpyDeviceToHost,
                            c->h_down) != cudaSuccess ||
            cudaEventRecord(down[k], c->h_down) != cudaSuccess)
            return fail(c, FKS_ERR_CUDA, "download");
    }
    // the caller's stream completes after the last download
    for (int k = 0; k < nchunk; ++k)
        if (cudaStreamWaitEvent(s, down[k], 0) != cudaSuccess) return fail(c, FKS_ERR_CUDA, "join");
    return FKS_OK;
}

fks_status fks_moments(fks_ctx* c, const void* f, double* U, void* stream) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!f || !U) return fail(c, FKS_ERR_INVALID_ARG, "null pointer");
    if (c->ncells == 0) return FKS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e0 = c->fp64 ? launch_moments_t<double>(c, f, U, s) : launch_moments_t<float>(c, f, U, s);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "moments kernel launch");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel launch");
    c->launches += 1;
    return FKS_OK;
}

fks_status fks_check(fks_ctx* c, void* stream, int* bits) {
    if (!c) return FKS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    e = cudaMemcpy(&h, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "flag read");
    e = cudaMemset(c->d_flags, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(c, e, "flag reset");
    if (bits) *bits = h;
    if (h & 1) return fail(c, FKS_ERR_NUMERIC, "non-finite value written");
    if (h & 4) return fail(c, FKS_ERR_NUMERIC, "cell shift out of range");
    if (h & 8) return fail(c, FKS_ERR_TIMEOUT, "a bulk copy did not complete in time");
    return FKS_OK;
}

fks_status fks_selftest_wait(long polls, void* stream) {
    if (polls < 1 || polls > (1L << 26)) return FKS_ERR_INVALID_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return alloc_failure();
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        selftest_wait_kernel<<<1, 32, 0, s>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return FKS_ERR_CUDA;
    return (h & 8) ? FKS_ERR_TIMEOUT : FKS_OK;
}

fks_status fks_alu_peak(int precision, double* tflops, void* stream) {
    if (!tflops || (precision != FKS_FP64 && precision != FKS_FP32)) return FKS_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FKS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 16) != cudaSuccess) return alloc_failure();
    const bool fp64 = precision == FKS_FP64;
    const int iters = fp64 ? 1024 : 32768;
    const dim3 grid((unsigned)(sms * 8)), block(256);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = cudaEventRecord(e0, s);
        if (fp64) fma_peak_kernel<double><<<grid, block, 0, s>>>(0.999999, 1e-7, iters, (double*)sink);
        else fma_peak_kernel<float><<<grid, block, 0, s>>>(0.999999f, 1e-7f, iters, (float*)sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.f)) return FKS_ERR_CUDA;
    *tflops = 2.0 * 8.0 * iters * (double)grid.x * block.x / (ms * 1e-3) / 1e12;
    return FKS_OK;
}

fks_status fks_set_escalation(fks_ctx* c, double tol) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, FKS_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (tol > 0.0 && c->esc_ntier == 0)
        return fail(c, FKS_ERR_UNSUPPORTED, "this context has no escalation tiers (FP64, BGK, VHS)");
    cudaDeviceSynchronize();   // launches in flight keep the tolerance they were issued with
    c->esc_tol = tol;
    return FKS_OK;
}

fks_status fks_set_escalation_arith(fks_ctx* c, int arith) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (arith != FKS_FP64 && arith != FKS_FP32X2) return fail(c, FKS_ERR_INVALID_ARG, "arith: FKS_FP64 or FKS_FP32X2");
    if (c->esc_ntier == 0) return fail(c, FKS_ERR_UNSUPPORTED, "this context has no escalation tiers");
    if (arith == c->esc_arith) return FKS_OK;
    cudaDeviceSynchronize();
    c->esc_arith = arith;
    return setup_escalation(c);   // rebuilds the tiers (the last one in the new arithmetic)
}

fks_status fks_set_escalation_direct(fks_ctx* c, int on) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (c->esc_ntier < 1) return fail(c, FKS_ERR_UNSUPPORTED, "direct routing needs a context with escalation tiers");
    c->esc_direct = on != 0;
    return FKS_OK;
}

fks_status fks_get_escalation(const fks_ctx* c, double* tol, long* counts) {
    if (!c) return FKS_ERR_INVALID_ARG;
    if (tol) *tol = c->esc_tol;
    if (counts) {
        int h[2] = {0, 0};
        if (c->esc_counts && cudaMemcpy(h, c->esc_counts, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
            return FKS_ERR_CUDA;
        counts[0] = h[0];
        counts[1] = h[1];
    }
    return FKS_OK;
}

fks_status fks_set_profiling(fks_ctx* c, int on) {
    if (!c) return FKS_ERR_INVALID_ARG;
    c->prof = on != 0;
    return FKS_OK;
}

fks_status fks_get_profile(fks_ctx* c, double* ms, long* launches) {
    if (!c || !ms) return FKS_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(c, FKS_ERR_CUDA, "profile synchronisation");
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        auto& v = c->prof_ev[k];
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, v[i], v[i + 1]) == cudaSuccess) acc += t;
        }
        ms[k] = acc;
        if (launches) launches[k] = (long)(v.size() / 2);
        for (cudaEvent_t e : v) c->prof_pool.push_back(e);
        v.clear();
    }
    return FKS_OK;
}

fks_status fks_get_offsets(fks_ctx* c, double* s) {
    if (!c || !s) return FKS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(s, c->d_s, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "offset read");
    return FKS_OK;
}

fks_status fks_set_offsets(fks_ctx* c, const double* s) {
    if (!c || !s) return FKS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(c->d_s, s, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "offset write");
    return FKS_OK;
}

// Host evaluation of the kernel transforms phi_R(s), psi_R(s) with the same
// code the table kernel runs on the device (a diagnostic: no GPU needed).
fks_status fks_kernel_transform(int ktype, double C, double L, double s, double* phi, double* psi) {
    if (!phi || !psi || (ktype != 0 && ktype != 1) || !(C > 0) || !(L > 0)) return FKS_ERR_INVALID_ARG;
    const double R = 2.0 / (3.0 + std::sqrt(2.0)) * L;
    std::vector<double> gl(4 * kGL);
    gl_rule(kGL, 0.0, 0.5 * 3.14159265358979323846, gl.data(), gl.data() + kGL);
    gl_rule(kGL, 0.0, std::sqrt(R), gl.data() + 2 * kGL, gl.data() + 3 * kGL);
    TableParams tp;
    tp.n = 0;
    tp.M = 0;
    tp.ktype = ktype;
    tp.HF = 0;
    tp.L = L;
    tp.R = R;
    tp.c4 = std::sqrt(4.0 * C);
    tp.e = nullptr;
    tp.w = nullptr;
    tp.glt_x = gl.data();
    tp.glt_w = gl.data() + kGL;
    tp.glu_x = gl.data() + 2 * kGL;
    tp.glu_w = gl.data() + 3 * kGL;
    *phi = phi_any(tp, s);
    *psi = psi_any(tp, s);
    return FKS_OK;
}

}  // extern "C"


// ------------------------------------------------------------------ no-allocation transport
//
// fks_transport_noalloc: the transport of fks_transport for callers that
// cannot allocate device memory.  Its only scratch (the per-call table of
// cell shifts and a flag word) lives in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
namespace {

constexpr int kNoAllocMaxN = 32;            // largest velocity grid n it accepts
constexpr int kNoAllocFlagOffset = 128;     // byte offset of the flag word
static __device__ __align__(256) unsigned char g_noalloc_scratch[256];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side name is only a stand-in, not a device address).
fks_status noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return FKS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FKS_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FKS_OK;
}

}  // namespace

extern "C" fks_status fks_transport_noalloc(const fks_grid* grid, const fks_vbox* vbox, int precision, double* s,
                                            double dt, const void* f, void* f_out, void* stream) {
    if (!grid || !vbox || !s || !f || !f_out || f == f_out) return FKS_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return FKS_ERR_INVALID_ARG;
    if ((long)grid->nx * grid->ny * grid->nz >= (1L << 31)) return FKS_ERR_INVALID_ARG;   // 32-bit cell indices
    for (int a = 0; a < 3; ++a) {
        if (!(grid->x1[a] > grid->x0[a])) return FKS_ERR_INVALID_ARG;
        if (grid->bc[a] != FKS_BC_PERIODIC && grid->bc[a] != FKS_BC_SPECULAR) return FKS_ERR_INVALID_ARG;
    }
    if (!(vbox->L > 0.0) || !std::isfinite(vbox->L) || !std::isfinite(dt)) return FKS_ERR_INVALID_ARG;
    if (vbox->n < 2 || vbox->n % 2 != 0) return FKS_ERR_INVALID_ARG;
    if (vbox->n > kNoAllocMaxN) return FKS_ERR_UNSUPPORTED;   // beyond the static scratch
    if (precision != FKS_FP64 && precision != FKS_FP32) return FKS_ERR_UNSUPPORTED;
    const int n = vbox->n;
    const int nca[3] = {grid->nx, grid->ny, grid->nz};
    double dx[3];
    for (int a = 0; a < 3; ++a) {
        dx[a] = (grid->x1[a] - grid->x0[a]) / nca[a];
        if (std::fabs(vbox->L * dt) > 100.0 * dx[a]) return FKS_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    fks_status st = noalloc_scratch(&base);
    if (st != FKS_OK) return st;
    signed char* d_delta = static_cast<signed char*>(base);
    int* d_flags = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kNoAllocFlagOffset);
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_flags, 0, sizeof(int), cs) != cudaSuccess) return FKS_ERR_CUDA;
    offsets_kernel<<<dim3(1, 3), n / 2, 0, cs>>>(n, vbox->L, make_double3(dx[0], dx[1], dx[2]), dt, s, d_delta, d_flags);
    const cudaError_t e0 = precision == FKS_FP64 ? launch_transport<double>(n, *grid, d_delta, f, f_out, cs)
                                                 : launch_transport<float>(n, *grid, d_delta, f, f_out, cs);
    if (e0 != cudaSuccess || cudaGetLastError() != cudaSuccess) return FKS_ERR_CUDA;
    // the flag word: bit 2 = a cell shift beyond the range of the shift table.  The host check on
    // |L dt| keeps it clear for offsets in [-dx/2, dx/2); offsets outside (a corrupted s) set it.
    int bits = 0;
    if (cudaMemcpyAsync(&bits, d_flags, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
        return FKS_ERR_CUDA;
    return (bits & 4) ? FKS_ERR_NUMERIC : FKS_OK;
}
