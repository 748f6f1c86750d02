// fks_surrogate.cu -- inference path of the learned collision surrogate:
//   inputs  : per cell, rho, u, T of f (FP64 sums), x = (f / rho, M[f] / rho),
//             and the distance from equilibrium d = ||f - M|| / ||M||
//   network : fks_net inference (tcgen05 tensor cores, BF16 weights and
//             activations, FP32 accumulation; CUDA-core FP32 path for n = 8, 24)
//   output  : Q = rho^2 y out_scale / Kn, conservation projection (FP64 sums),
//             indicator = ind_scale / d + defect, defect = relative size of the
//             raw output's moments: the network's error is roughly a fixed
//             fraction of the output scale, while ||Q|| shrinks with the
//             distance d from equilibrium, so its relative error grows as 1/d
//   routing : the d part of the indicator is known before inference: cells with
//             ind_scale / d over the threshold skip the network; the others are
//             inferred (compacted into chunks) and routed if the full indicator
//             exceeds the threshold.  Routed cells are recomputed by the
//             context's spectral kernel over a device list (with the context's
//             precision escalation).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/fks.h"
#include "fks_internal.h"

namespace fks {
namespace surr {

constexpr int BS = 512;

// block-wide FP64 sums of k values (k <= 8), fixed order: deterministic
__device__ __forceinline__ void block_sum(double* v, int k, double* red) {
    const int tid = threadIdx.x;
    for (int i = 0; i < k; ++i) {
        double s = v[i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        v[i] = s;
    }
    __syncthreads();
    if ((tid & 31) == 0)
        for (int i = 0; i < k; ++i) red[(tid >> 5) * 8 + i] = v[i];
    __syncthreads();
    for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int w = 0; w < BS / 32; ++w) s += red[w * 8 + i];
        v[i] = s;
    }
    __syncthreads();
}

// Both kernels sweep a cell as float4 runs along v_z (n % 4 == 0): run q holds
// elements 4q .. 4q+3 of row r = q / (n/4), i.e. ix = r / n, iy = r % n.

// one CTA per cell: moments (FP32 partials, FP64 block sums), the Maxwellian
// as a product of three one-axis tables, network input x = (f / rho, M / rho)
// and the distance from equilibrium
//   list: the cells are list[c0 .. c0 + ncells) (x packed by list position), else c0 .. c0 + ncells;
//   x = nullptr: only rho and dist (the classification before inference)
__global__ void __launch_bounds__(BS) inputs_kernel(int n, double L, long c0, long ncells, const float* __restrict__ f,
                                                    float* __restrict__ x, double* __restrict__ rho_out,
                                                    float* __restrict__ dist, const int* __restrict__ list = nullptr) {
    __shared__ double red[(BS / 32) * 8];
    __shared__ float vg[64], ex[3][64];
    const long n3 = (long)n * n * n;
    const int q4 = n / 4;
    const long runs = n3 / 4;
    const double dv = 2.0 * L / n;
    for (int i = threadIdx.x; i < n; i += BS) vg[i] = (float)(((double)i + 0.5 - 0.5 * n) * dv);
    __syncthreads();
    for (long ci = c0 + blockIdx.x; ci < c0 + ncells; ci += gridDim.x) {
        const long c = list ? (long)list[ci] : ci;
        const float4* fc = reinterpret_cast<const float4*>(f + c * n3);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
        for (long q = threadIdx.x; q < runs; q += BS) {
            const float4 m = fc[q];
            const int r = (int)(q / q4), iz = 4 * (int)(q % q4);
            const float vx = vg[r / n], vy = vg[r % n];
            const float z0 = vg[iz], z1 = vg[iz + 1], z2 = vg[iz + 2], z3 = vg[iz + 3];
            const float s = (m.x + m.y) + (m.z + m.w);
            a0 += s;
            a1 = fmaf(s, vx, a1);
            a2 = fmaf(s, vy, a2);
            a3 += m.x * z0 + m.y * z1 + m.z * z2 + m.w * z3;
            a4 += s * (vx * vx + vy * vy) + (m.x * z0 * z0 + m.y * z1 * z1 + m.z * z2 * z2 + m.w * z3 * z3);
        }
        double sm[5] = {a0, a1, a2, a3, 0.5 * (double)a4};
        block_sum(sm, 5, red);
        const double dv3 = dv * dv * dv;
        const double rho = sm[0] * dv3;
        const double ux = sm[1] * dv3 / rho, uy = sm[2] * dv3 / rho, uz = sm[3] * dv3 / rho;
        const double T = (sm[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
        const double pre = 1.0 / (2.0 * 3.14159265358979323846 * T * sqrt(2.0 * 3.14159265358979323846 * T));
        // M / rho = pre * ex[0][ix] * ex[1][iy] * ex[2][iz]
        const double u3[3] = {ux, uy, uz};
        for (int i = threadIdx.x; i < 3 * n; i += BS) {
            const int ax = i / n, k = i % n;
            const double d = ((double)k + 0.5 - 0.5 * n) * dv - u3[ax];
            ex[ax][k] = (float)(exp(-d * d / (2.0 * T)) * (ax == 0 ? pre : 1.0));
        }
        __syncthreads();
        const float inv_rho = (float)(1.0 / rho);
        float4* xg = x ? reinterpret_cast<float4*>(x + (ci - c0) * 2 * n3) : nullptr;
        float4* xm = x ? reinterpret_cast<float4*>(x + (ci - c0) * 2 * n3 + n3) : nullptr;
        float d0 = 0.f, d1 = 0.f;
        for (long q = threadIdx.x; q < runs; q += BS) {
            const float4 m = fc[q];
            const int r = (int)(q / q4), iz = 4 * (int)(q % q4);
            const float exy = ex[0][r / n] * ex[1][r % n];
            const float4 g = make_float4(m.x * inv_rho, m.y * inv_rho, m.z * inv_rho, m.w * inv_rho);
            const float4 M = make_float4(exy * ex[2][iz], exy * ex[2][iz + 1], exy * ex[2][iz + 2], exy * ex[2][iz + 3]);
            if (x) {
                xg[q] = g;
                xm[q] = M;
            }
            d0 += (g.x - M.x) * (g.x - M.x) + (g.y - M.y) * (g.y - M.y) + (g.z - M.z) * (g.z - M.z) +
                  (g.w - M.w) * (g.w - M.w);
            d1 += M.x * M.x + M.y * M.y + M.z * M.z + M.w * M.w;
        }
        double d2[2] = {d0, d1};
        block_sum(d2, 2, red);
        if (threadIdx.x == 0) {
            rho_out[c] = rho;
            dist[c] = (float)sqrt(d2[0] / d2[1]);
        }
    }
}

// one CTA per cell: q = rho^2 y s / Kn (FP32), the five moments of q as FP64
// sums of the FP32 values, conservation projection Q = q - C^T mu, indicator
//   list: y row i belongs to cell list[c0 + i]; step: out = f* + dt Q (fs = f*), else out = Q; cells whose
//   indicator exceeds the threshold (or is not finite) are appended to route (count *nroute)
__global__ void __launch_bounds__(BS) output_kernel(int n, double L, long c0, long ncells, const float* __restrict__ y,
                                                    const double* __restrict__ rho, const float* __restrict__ dist,
                                                    const double* __restrict__ P, double scale, double ind_scale,
                                                    float* __restrict__ Q, float* __restrict__ ind,
                                                    const int* __restrict__ list, const float* __restrict__ fs,
                                                    float dt, float threshold, int* __restrict__ route,
                                                    int* __restrict__ nroute) {
    __shared__ double red[(BS / 32) * 8];
    __shared__ double vd[64];
    __shared__ float vg[64];
    __shared__ double mu[5];
    const long n3 = (long)n * n * n;
    const int q4 = n / 4;
    const long runs = n3 / 4;
    const double dv = 2.0 * L / n;
    for (int i = threadIdx.x; i < n; i += BS) {
        vd[i] = ((double)i + 0.5 - 0.5 * n) * dv;
        vg[i] = (float)vd[i];
    }
    __syncthreads();
    for (long ci = c0 + blockIdx.x; ci < c0 + ncells; ci += gridDim.x) {
        const long c = list ? (long)list[ci] : ci;
        const float4* yc = reinterpret_cast<const float4*>(y + (ci - c0) * n3);
        const float a = (float)(rho[c] * rho[c] * scale);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        float sa = 0.f;   // sum |phi| |q| (indicator scale only)
        for (long q = threadIdx.x; q < runs; q += BS) {
            const float4 v = yc[q];
            const int r = (int)(q / q4), iz = 4 * (int)(q % q4);
            const float e4[4] = {a * v.x, a * v.y, a * v.z, a * v.w};
            double t0 = 0.0, tz = 0.0, tzz = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double qk = (double)e4[k], z = vd[iz + k];
                t0 += qk;
                tz = fma(qk, z, tz);
                tzz = fma(qk, 0.5 * z * z, tzz);
            }
            const double vx = vd[r / n], vy = vd[r % n];
            s0 += t0;
            s1 = fma(t0, vx, s1);
            s2 = fma(t0, vy, s2);
            s3 += tz;
            s4 = fma(t0, 0.5 * (vx * vx + vy * vy), s4) + tzz;
            const float ax = fabsf(vg[r / n]) + fabsf(vg[r % n]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float z = vg[iz + k];
                sa += fabsf(e4[k]) * (1.f + ax + fabsf(z) + 0.5f * (vg[r / n] * vg[r / n] + vg[r % n] * vg[r % n] + z * z));
            }
        }
        double sm[6] = {s0, s1, s2, s3, s4, (double)sa};
        block_sum(sm, 6, red);
        if (threadIdx.x < 5) {
            double acc = 0.0;
            for (int j = 0; j < 5; ++j) acc += P[threadIdx.x * 5 + j] * sm[j];
            mu[threadIdx.x] = acc;
        }
        __syncthreads();
        const float m0 = (float)mu[0], m1 = (float)mu[1], m2 = (float)mu[2], m3 = (float)mu[3], m4 = (float)mu[4];
        float4* Qc = reinterpret_cast<float4*>(Q + c * n3);
        const float4* fsc = fs ? reinterpret_cast<const float4*>(fs + c * n3) : nullptr;
        for (long q = threadIdx.x; q < runs; q += BS) {
            const float4 v = yc[q];
            const int r = (int)(q / q4), iz = 4 * (int)(q % q4);
            const float vx = vg[r / n], vy = vg[r % n];
            const float cxy = m0 + m1 * vx + m2 * vy + 0.5f * m4 * (vx * vx + vy * vy);
            float4 o;
            o.x = a * v.x - (cxy + m3 * vg[iz] + 0.5f * m4 * vg[iz] * vg[iz]);
            o.y = a * v.y - (cxy + m3 * vg[iz + 1] + 0.5f * m4 * vg[iz + 1] * vg[iz + 1]);
            o.z = a * v.z - (cxy + m3 * vg[iz + 2] + 0.5f * m4 * vg[iz + 2] * vg[iz + 2]);
            o.w = a * v.w - (cxy + m3 * vg[iz + 3] + 0.5f * m4 * vg[iz + 3] * vg[iz + 3]);
            if (fsc) {
                const float4 b = fsc[q];
                o = make_float4(fmaf(dt, o.x, b.x), fmaf(dt, o.y, b.y), fmaf(dt, o.z, b.z), fmaf(dt, o.w, b.w));
            }
            Qc[q] = o;
        }
        if (threadIdx.x == 0) {
            const double defect =
                (fabs(sm[0]) + fabs(sm[1]) + fabs(sm[2]) + fabs(sm[3]) + fabs(sm[4])) / (sm[5] > 0 ? sm[5] : 1.0);
            const double d = (double)dist[c];
            const float v = (float)(ind_scale / (d > 1e-30 ? d : 1e-30) + defect);
            ind[c] = v;
            if (route && !(v <= threshold)) route[atomicAdd(nroute, 1)] = (int)c;
        }
        __syncthreads();   // mu and red are rewritten by the next cell
    }
}

// split the cells by the indicator's lower bound ind_scale / d (known before inference): over the
// threshold (or not finite) -> route list (their indicator is that bound), else -> candidate list
//   d < d_last: straight to the last escalation tier's list (last, count *nlast); else d < d_mid: straight
//   to the middle tier's list (mid, count *nmid); *ndirect counts both
__global__ void classify_kernel(long ncells, const float* __restrict__ dist, double ind_scale, float threshold,
                                float* __restrict__ ind, int* __restrict__ route, int* __restrict__ nroute,
                                int* __restrict__ cand, int* __restrict__ ncand, double d_last,
                                int* __restrict__ last, int* __restrict__ nlast, double d_mid, int* __restrict__ mid,
                                int* __restrict__ nmid, int* __restrict__ ndirect) {
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncells; c += (long)gridDim.x * blockDim.x) {
        const double d = (double)dist[c];
        const float lb = (float)(ind_scale / (d > 1e-30 ? d : 1e-30));
        if (d < d_last) {
            ind[c] = lb;
            last[atomicAdd(nlast, 1)] = (int)c;
            atomicAdd(ndirect, 1);
        } else if (d < d_mid) {
            ind[c] = lb;
            mid[atomicAdd(nmid, 1)] = (int)c;
            atomicAdd(ndirect, 1);
        } else if (!(lb <= threshold)) {
            ind[c] = lb;
            route[atomicAdd(nroute, 1)] = (int)c;
        } else {
            cand[atomicAdd(ncand, 1)] = (int)c;
        }
    }
}

}  // namespace surr
}  // namespace fks

using namespace fks;

extern "C" {

fks_status fks_surrogate_inputs(int n, double L, long ncells, const float* f, float* x, double* rho, float* dist,
                                void* stream) {
    if (!f || !x || !rho || !dist || ncells < 0 || n < 4 || n % 4 != 0 || n > 64 || !(L > 0) ||
        ((uintptr_t)f & 15) || ((uintptr_t)x & 15))
        return FKS_ERR_INVALID_ARG;
    if (ncells == 0) return FKS_OK;
    const long grid = ncells < 152L * 8 ? ncells : 152L * 8;
    surr::inputs_kernel<<<(unsigned)grid, surr::BS, 0, (cudaStream_t)stream>>>(n, L, 0, ncells, f, x, rho, dist);
    return cudaGetLastError() == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

}  // extern "C"

// The surrogate over fs (f* of every cell): out = Q (mode 0) or fs + dt Q (mode 1, fs already transported).
static fks_status surrogate_run(fks_ctx* c, fks_net* net, const float* fs, float* out, double dt, int mode,
                                double out_scale, double ind_scale, double threshold, long* nrouted, cudaStream_t s) {
    const int n = c->n;
    const long nc = c->ncells;
    // per-context surrogate workspace: rho, distance, indicator, routed and candidate lists, two counts
    if (!c->s_rho) {
        if (cudaMalloc(&c->s_rho, sizeof(double) * nc) != cudaSuccess || cudaMalloc(&c->s_dist, sizeof(float) * nc) ||
            cudaMalloc(&c->s_ind, sizeof(float) * nc) || cudaMalloc(&c->s_count, 3 * sizeof(int)) ||
            cudaMalloc(&c->s_cells, sizeof(int) * (nc > 0 ? nc : 1)) ||
            cudaMalloc(&c->s_cand, sizeof(int) * (nc > 0 ? nc : 1))) {
            c->err = "surrogate workspace";
            return alloc_failure();
        }
    }
    const int B = fks_net_infer_capacity(net);
    float* xbuf = fks_net_input_buffer(net);
    if (B < 1 || !xbuf) {
        c->err = "surrogate inference workspace";
        return FKS_ERR_OOM;
    }
    if (cudaMemsetAsync(c->s_count, 0, 3 * sizeof(int), s) != cudaSuccess) return FKS_ERR_CUDA;
    // the escalation lists start here: cells that certainly fail every earlier tier (d below the
    // route's bound) go straight to the last tier
    int *last = nullptr, *nlast = nullptr, *mid = nullptr, *nmid = nullptr;
    double d_last = 0.0, d_mid = 0.0;
    fks_status st0 = fks_internal_last_tier_route(c, s, &last, &nlast, &d_last, &mid, &nmid, &d_mid);
    if (st0 != FKS_OK) return st0;
    // 1. rho and d of every cell; the cells whose bound ind_scale / d already exceeds the threshold
    //    are routed without inference
    const long gridc = nc < 152L * 8 ? nc : 152L * 8;
    surr::inputs_kernel<<<(unsigned)gridc, surr::BS, 0, s>>>(n, c->vbox.L, 0, nc, fs, nullptr, c->s_rho, c->s_dist);
    surr::classify_kernel<<<256, 256, 0, s>>>(nc, c->s_dist, ind_scale, (float)threshold, c->s_ind, c->s_cells,
                                             c->s_count, c->s_cand, c->s_count + 1, last ? d_last : 0.0, last, nlast,
                                             mid ? d_mid : 0.0, mid, nmid, c->s_count + 2);
    c->launches += 2;
    // 2. the candidates in chunks of B (their count read back: one synchronisation)
    int ncand = 0;
    if (cudaMemcpyAsync(&ncand, c->s_count + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FKS_ERR_CUDA;
    for (long c0 = 0; c0 < ncand; c0 += B) {
        const long k = ncand - c0 < B ? ncand - c0 : B;
        const long grid = k < 152L * 8 ? k : 152L * 8;
        surr::inputs_kernel<<<(unsigned)grid, surr::BS, 0, s>>>(n, c->vbox.L, c0, k, fs, xbuf, c->s_rho, c->s_dist,
                                                             c->s_cand);
        fks_status st = FKS_OK;
        const float* y = fks_net_infer_internal(net, (int)k, xbuf, s, &st);
        if (st != FKS_OK) return st;
        surr::output_kernel<<<(unsigned)grid, surr::BS, 0, s>>>(
            n, c->vbox.L, c0, k, y, c->s_rho, c->s_dist, c->d_P, out_scale / c->kern.knudsen, ind_scale, out, c->s_ind,
            c->s_cand, mode == 1 ? fs : nullptr, (float)dt, (float)threshold, c->s_cells, c->s_count);
        c->launches += 2;
    }
    // 3. the context's spectral operator (projected, with its precision escalation) on the routed
    //    cells; the kernels read the routed count on the device
    const fks_status st = fks_internal_collide_list(c, fs, out, c->s_cells, c->s_count, mode, dt, s, last != nullptr);
    if (st != FKS_OK) return st;
    if (nrouted) {
        int count[3] = {0, 0, 0};
        if (cudaMemcpyAsync(count, c->s_count, sizeof(count), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FKS_ERR_CUDA;
        *nrouted = count[0] + count[2];   // to the spectral operator, directly or through its first kernel
    }
    return cudaGetLastError() == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

static fks_status surrogate_check(fks_ctx* c, fks_net* net) {
    if (c->fp64 || c->bgk || c->dealias || fks_net_grid(net) != c->n) {
        c->err = "the surrogate needs an FP32 or split-BF16 spectral context (variant A) with the network's grid";
        return FKS_ERR_UNSUPPORTED;
    }
    return FKS_OK;
}

extern "C" {

fks_status fks_surrogate_collide(fks_ctx* c, fks_net* net, const void* f, void* Q, double out_scale,
                                 double ind_scale, double threshold, long* nrouted, void* stream) {
    if (!c || !net || !f || !Q || f == Q) return FKS_ERR_INVALID_ARG;
    const fks_status st = surrogate_check(c, net);
    if (st != FKS_OK) return st;
    if (((uintptr_t)f & 15) || ((uintptr_t)Q & 15)) return FKS_ERR_INVALID_ARG;
    return surrogate_run(c, net, static_cast<const float*>(f), static_cast<float*>(Q), 0.0, 0, out_scale, ind_scale,
                         threshold, nrouted, (cudaStream_t)stream);
}

fks_status fks_surrogate_step(fks_ctx* c, fks_net* net, const void* f, void* f_out, void* work, double dt,
                              double out_scale, double ind_scale, double threshold, long* nrouted, void* stream) {
    if (!c || !net || !f || !f_out || !work) return FKS_ERR_INVALID_ARG;
    if (f == f_out || f == work || f_out == work) return fks_internal_fail(c, FKS_ERR_INVALID_ARG, "f, f_out and work must be distinct");
    if (((uintptr_t)f & 15) || ((uintptr_t)f_out & 15) || ((uintptr_t)work & 15)) return FKS_ERR_INVALID_ARG;
    fks_status st = surrogate_check(c, net);
    if (st != FKS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = fks_transport(c, f, work, dt, stream);   // offsets over dt, f* -> work
    if (st != FKS_OK) return st;
    return surrogate_run(c, net, static_cast<const float*>(work), static_cast<float*>(f_out), dt, 1, out_scale,
                         ind_scale, threshold, nrouted, s);
}

fks_status fks_surrogate_indicator(const fks_ctx* c, float* host, long count) {
    if (!c || !host || count != c->ncells || !c->s_ind) return FKS_ERR_INVALID_ARG;
    return cudaMemcpy(host, c->s_ind, sizeof(float) * count, cudaMemcpyDeviceToHost) == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

}  // extern "C"
