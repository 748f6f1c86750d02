// fks_surrogate.cu -- inference path of the learned collision surrogate:
//   inputs  : per cell, rho, u, T of f (FP64 sums), x = (f / rho, M[f] / rho),
//             and the distance from equilibrium d = ||f - M|| / ||M||
//   network : fks_net inference (tcgen05 tensor cores, BF16 weights and
//             activations, FP32 accumulation; CUDA-core FP32 path for n = 8, 24)
//   output  : Q = rho^2 y out_scale / Kn, conservation projection (FP64 sums),
//             indicator = ind_scale (d + defect), defect = relative size of the
//             raw output's moments
//   routing : cells whose indicator exceeds the threshold are recomputed by
//             the spectral kernel (batch mode over the routed cells).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/fks.h"
#include "fks_internal.h"

namespace fks {
namespace surr {

constexpr int BS = 256;

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

// one CTA per cell: moments, Maxwellian, network input, distance from equilibrium
__global__ void __launch_bounds__(BS) inputs_kernel(int n, double L, long c0, long ncells, const float* __restrict__ f,
                                                    float* __restrict__ x, double* __restrict__ rho_out,
                                                    float* __restrict__ dist) {
    __shared__ double red[(BS / 32) * 8];
    const long n3 = (long)n * n * n;
    const double dv = 2.0 * L / n;
    for (long c = c0 + blockIdx.x; c < c0 + ncells; c += gridDim.x) {
        const float* fc = f + c * n3;
        double s[5] = {0, 0, 0, 0, 0};
        for (long k = threadIdx.x; k < n3; k += BS) {
            const double vx = ((double)(k / (n * n)) + 0.5 - 0.5 * n) * dv;
            const double vy = ((double)((k / n) % n) + 0.5 - 0.5 * n) * dv;
            const double vz = ((double)(k % n) + 0.5 - 0.5 * n) * dv;
            const double m = fc[k];
            s[0] += m;
            s[1] += m * vx;
            s[2] += m * vy;
            s[3] += m * vz;
            s[4] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        }
        block_sum(s, 5, red);
        const double dv3 = dv * dv * dv;
        const double rho = s[0] * dv3;
        const double ux = s[1] * dv3 / rho, uy = s[2] * dv3 / rho, uz = s[3] * dv3 / rho;
        const double T = (s[4] * dv3 - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / (1.5 * rho);
        const double pre = 1.0 / (2.0 * 3.14159265358979323846 * T * sqrt(2.0 * 3.14159265358979323846 * T));
        float* xc = x + (c - c0) * 2 * n3;
        double d2[2] = {0.0, 0.0};
        for (long k = threadIdx.x; k < n3; k += BS) {
            const double vx = ((double)(k / (n * n)) + 0.5 - 0.5 * n) * dv - ux;
            const double vy = ((double)((k / n) % n) + 0.5 - 0.5 * n) * dv - uy;
            const double vz = ((double)(k % n) + 0.5 - 0.5 * n) * dv - uz;
            const double Mg = pre * exp(-(vx * vx + vy * vy + vz * vz) / (2.0 * T));   // M / rho
            const double g = fc[k] / rho;
            xc[k] = (float)g;
            xc[n3 + k] = (float)Mg;
            d2[0] += (g - Mg) * (g - Mg);
            d2[1] += Mg * Mg;
        }
        block_sum(d2, 2, red);
        if (threadIdx.x == 0) {
            rho_out[c] = rho;
            dist[c] = (float)sqrt(d2[0] / d2[1]);
        }
    }
}

// one CTA per cell: Q = rho^2 y s / Kn, conservation projection, indicator
__global__ void __launch_bounds__(BS) output_kernel(int n, double L, long c0, long ncells, const float* __restrict__ y,
                                                    const double* __restrict__ rho, const float* __restrict__ dist,
                                                    const double* __restrict__ P, double scale, double ind_scale,
                                                    float* __restrict__ Q, float* __restrict__ ind) {
    __shared__ double red[(BS / 32) * 8];
    const long n3 = (long)n * n * n;
    const double dv = 2.0 * L / n;
    for (long c = c0 + blockIdx.x; c < c0 + ncells; c += gridDim.x) {
        const float* yc = y + (c - c0) * n3;
        const double a = rho[c] * rho[c] * scale;
        double s[6] = {0, 0, 0, 0, 0, 0};   // sum phi Q, sum |phi| |Q|
        for (long k = threadIdx.x; k < n3; k += BS) {
            const double vx = ((double)(k / (n * n)) + 0.5 - 0.5 * n) * dv;
            const double vy = ((double)((k / n) % n) + 0.5 - 0.5 * n) * dv;
            const double vz = ((double)(k % n) + 0.5 - 0.5 * n) * dv;
            const double q = a * yc[k];
            const double e = 0.5 * (vx * vx + vy * vy + vz * vz);
            s[0] += q;
            s[1] += q * vx;
            s[2] += q * vy;
            s[3] += q * vz;
            s[4] += q * e;
            s[5] += fabs(q) * (1.0 + fabs(vx) + fabs(vy) + fabs(vz) + e);
        }
        block_sum(s, 6, red);
        double mu[5];
        for (int i = 0; i < 5; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 5; ++j) acc += P[i * 5 + j] * s[j];
            mu[i] = acc;
        }
        const double defect = (fabs(s[0]) + fabs(s[1]) + fabs(s[2]) + fabs(s[3]) + fabs(s[4])) / (s[5] > 0 ? s[5] : 1.0);
        float* Qc = Q + c * n3;
        for (long k = threadIdx.x; k < n3; k += BS) {
            const double vx = ((double)(k / (n * n)) + 0.5 - 0.5 * n) * dv;
            const double vy = ((double)((k / n) % n) + 0.5 - 0.5 * n) * dv;
            const double vz = ((double)(k % n) + 0.5 - 0.5 * n) * dv;
            const double corr = mu[0] + mu[1] * vx + mu[2] * vy + mu[3] * vz + mu[4] * 0.5 * (vx * vx + vy * vy + vz * vz);
            Qc[k] = (float)(a * yc[k] - corr);
        }
        if (threadIdx.x == 0) ind[c] = (float)(ind_scale * ((double)dist[c] + defect));
    }
}

// descriptors of the cells whose indicator exceeds the threshold
__global__ void route_kernel(long ncells, const float* __restrict__ ind, float threshold, int n, const float* f,
                             float* Q, const void* tables, const double* P, double inv_kn, double L,
                             BatchItem* __restrict__ items, int* __restrict__ count) {
    const long n3 = (long)n * n * n;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncells; c += (long)gridDim.x * blockDim.x) {
        if (!(ind[c] <= threshold)) {   // NaN indicators are routed too
            const int slot = atomicAdd(count, 1);
            BatchItem it;
            it.f = f + c * n3;
            it.out = Q + c * n3;
            it.tables = tables;
            it.P = P;
            it.inv_kn = inv_kn;
            it.dt = 0.0;
            it.L = L;
            it.pad_ = 0.0;
            items[slot] = it;
        }
    }
}

}  // namespace surr
}  // namespace fks

using namespace fks;

extern "C" {

fks_status fks_surrogate_inputs(int n, double L, long ncells, const float* f, float* x, double* rho, float* dist,
                                void* stream) {
    if (!f || !x || !rho || !dist || ncells < 0 || n < 2 || !(L > 0)) return FKS_ERR_INVALID_ARG;
    if (ncells == 0) return FKS_OK;
    const long grid = ncells < 152L * 8 ? ncells : 152L * 8;
    surr::inputs_kernel<<<(unsigned)grid, surr::BS, 0, (cudaStream_t)stream>>>(n, L, 0, ncells, f, x, rho, dist);
    return cudaGetLastError() == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

fks_status fks_surrogate_collide(fks_ctx* c, fks_net* net, const void* f, void* Q, double out_scale,
                                 double ind_scale, double threshold, long* nrouted, void* stream) {
    if (!c || !net || !f || !Q || f == Q) return FKS_ERR_INVALID_ARG;
    if (c->fp64 || c->bgk || fks_net_grid(net) != c->n) {
        c->err = "the surrogate needs an FP32 spectral context with the network's grid";
        return FKS_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = c->n;
    const long n3 = (long)n * n * n;
    const long nc = c->ncells;
    // per-context surrogate workspace (rho, distance, indicator, routed descriptors, count)
    if (!c->s_rho) {
        if (cudaMalloc(&c->s_rho, sizeof(double) * nc) != cudaSuccess || cudaMalloc(&c->s_dist, sizeof(float) * nc) ||
            cudaMalloc(&c->s_ind, sizeof(float) * nc) || cudaMalloc(&c->s_items, sizeof(BatchItem) * nc) ||
            cudaMalloc(&c->s_count, sizeof(int))) {
            c->err = "surrogate workspace";
            return FKS_ERR_OOM;
        }
    }
    const float* fin = static_cast<const float*>(f);
    float* Qo = static_cast<float*>(Q);
    const int B = fks_net_max_batch(net);
    float* xbuf = fks_net_input_buffer(net);
    for (long c0 = 0; c0 < nc; c0 += B) {
        const long k = nc - c0 < B ? nc - c0 : B;
        const long grid = k < 152L * 8 ? k : 152L * 8;
        surr::inputs_kernel<<<(unsigned)grid, surr::BS, 0, s>>>(n, c->vbox.L, c0, k, fin, xbuf, c->s_rho, c->s_dist);
        fks_status st = FKS_OK;
        const float* y = fks_net_infer_internal(net, (int)k, xbuf, s, &st);
        if (st != FKS_OK) return st;
        surr::output_kernel<<<(unsigned)grid, surr::BS, 0, s>>>(n, c->vbox.L, c0, k, y, c->s_rho, c->s_dist, c->d_P,
                                                             out_scale / c->kern.knudsen, ind_scale, Qo, c->s_ind);
        c->launches += 2;
    }
    if (cudaMemsetAsync(c->s_count, 0, sizeof(int), s) != cudaSuccess) return FKS_ERR_CUDA;
    surr::route_kernel<<<256, 256, 0, s>>>(nc, c->s_ind, (float)threshold, n, fin, Qo, c->tables, c->d_P,
                                          1.0 / c->kern.knudsen, c->vbox.L, c->s_items, c->s_count);
    c->launches += 1;
    int count = 0;
    if (cudaMemcpyAsync(&count, c->s_count, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FKS_ERR_CUDA;
    if (nrouted) *nrouted = count;
    if (count > 0) {
        // spectral operator (projected) on the routed cells, in batch mode
        CollideArgs a;
        std::memset(&a, 0, sizeof(a));
        a.items = c->s_items;
        a.ncells = count;
        a.nc[0] = a.nc[1] = a.nc[2] = 1;
        a.M = c->M;
        a.L = c->vbox.L;
        a.mode = 0;
        a.flags = c->d_flags;
        const long nclus = count < c->max_clusters ? count : c->max_clusters;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c->C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(nclus * c->C), 1, 1);
        cfg.blockDim = dim3(c->var.NT, 1, 1);
        cfg.dynamicSmemBytes = c->var.smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {&a};
        cudaError_t e = cudaLaunchKernelExC(&cfg, c->var.func_batch, args);
        if (e != cudaSuccess) {
            c->err = std::string("routed spectral launch: ") + cudaGetErrorString(e);
            return FKS_ERR_CUDA;
        }
        c->launches += 1;
    }
    return cudaGetLastError() == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

fks_status fks_surrogate_indicator(const fks_ctx* c, float* host, long count) {
    if (!c || !host || count != c->ncells || !c->s_ind) return FKS_ERR_INVALID_ARG;
    return cudaMemcpy(host, c->s_ind, sizeof(float) * count, cudaMemcpyDeviceToHost) == cudaSuccess ? FKS_OK : FKS_ERR_CUDA;
}

}  // extern "C"
