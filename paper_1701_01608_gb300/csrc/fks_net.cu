// fks_net.cu -- learned collision surrogate: a stack of 3x3x3 convolutions
// over the velocity grid (channels 2, 32, 32, 32, 32, 32, 1; ReLU between
// layers; zero padding), BF16 weights with FP32 accumulation, trained by the
// library's own forward / backward / Adam kernels.
//
// Input channels of a cell: g = f / rho and m = M[f] / rho (the cell's
// Maxwellian); output y ~ Q Kn / rho^2 / out_scale (the operator is quadratic,
// Q(rho g) = rho^2 Q(g)).  The surrogate's Q is then projected onto the
// conservation constraints like the spectral one, and an indicator routes
// cells whose predicted error exceeds a threshold back to the spectral kernel.
//
// Weight layout of layer l: W[co][ci][27], tap t = (dx+1)*9 + (dy+1)*3 + (dz+1),
// then bias[co]; the layers are packed in one flat FP32 master vector.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "fks_internal.h"

namespace fks {
namespace net {

constexpr int NL = 6;
constexpr int CH[NL + 1] = {2, 32, 32, 32, 32, 32, 1};
constexpr int TILE = 8;            // output voxels per tile edge
constexpr int HALO = TILE + 2;
constexpr int NTH = 256;           // threads per CTA (2 voxels each)

constexpr long layer_w(int l) { return (long)CH[l + 1] * CH[l] * 27; }
constexpr long layer_off(int l) {
    long o = 0;
    for (int i = 0; i < l; ++i) o += layer_w(i) + CH[i + 1];
    return o;
}
constexpr long NPARAM = layer_off(NL);

// ---------------------------------------------------------------- convolution
// y[b][co][p] = act(sum_{ci,t} W[co][ci][t] x[b][ci][p + d_t] + bias[co]),
// weights given as BF16 in [COUT][CIN][27].  One CTA = one 8^3 tile of one
// sample, all COUT channels; thread (tx, ty, tz) owns voxels z = tz, tz + 4.
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(NTH) conv_fwd_kernel(int n, const float* __restrict__ x,
                                                       const __nv_bfloat16* __restrict__ W,
                                                       const float* __restrict__ bias, float* __restrict__ y) {
    constexpr int CC = CIN < 4 ? CIN : 4;   // input channels per chunk
    __shared__ float s_in[CC][HALO][HALO][HALO];
    __shared__ __align__(16) float s_w[CC][27][COUT];
    const int tiles = n / TILE;
    const int tile = blockIdx.x % (tiles * tiles * tiles);
    const int b = blockIdx.x / (tiles * tiles * tiles);
    const int x0 = (tile / (tiles * tiles)) * TILE, y0 = ((tile / tiles) % tiles) * TILE, z0 = (tile % tiles) * TILE;
    const int tid = threadIdx.x;
    const int tx = tid / 32, ty = (tid / 4) % 8, tz = tid % 4;
    const long n3 = (long)n * n * n;
    float acc0[COUT], acc1[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc0[c] = acc1[c] = 0.f;
    for (int c0 = 0; c0 < CIN; c0 += CC) {
        __syncthreads();
        for (int i = tid; i < CC * HALO * HALO * HALO; i += NTH) {
            const int cc = i / (HALO * HALO * HALO), r = i % (HALO * HALO * HALO);
            const int hx = r / (HALO * HALO), hy = (r / HALO) % HALO, hz = r % HALO;
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            float v = 0.f;
            if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
                v = x[((long)b * CIN + c0 + cc) * n3 + ((long)gx * n + gy) * n + gz];
            s_in[cc][hx][hy][hz] = v;
        }
        for (int i = tid; i < CC * 27 * COUT; i += NTH) {
            const int co = i % COUT, t = (i / COUT) % 27, cc = i / (COUT * 27);
            s_w[cc][t][co] = __bfloat162float(W[((long)co * CIN + c0 + cc) * 27 + t]);
        }
        __syncthreads();
#pragma unroll 1
        for (int cc = 0; cc < CC; ++cc) {
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dx = t / 9, dy = (t / 3) % 3, dz = t % 3;
                const float a0 = s_in[cc][tx + dx][ty + dy][tz + dz];
                const float a1 = s_in[cc][tx + dx][ty + dy][tz + 4 + dz];
                const float* w = s_w[cc][t];
                if constexpr (COUT % 4 == 0) {
#pragma unroll
                    for (int co = 0; co < COUT; co += 4) {
                        const float4 w4 = *reinterpret_cast<const float4*>(w + co);
                        acc0[co] = fmaf(w4.x, a0, acc0[co]);
                        acc0[co + 1] = fmaf(w4.y, a0, acc0[co + 1]);
                        acc0[co + 2] = fmaf(w4.z, a0, acc0[co + 2]);
                        acc0[co + 3] = fmaf(w4.w, a0, acc0[co + 3]);
                        acc1[co] = fmaf(w4.x, a1, acc1[co]);
                        acc1[co + 1] = fmaf(w4.y, a1, acc1[co + 1]);
                        acc1[co + 2] = fmaf(w4.z, a1, acc1[co + 2]);
                        acc1[co + 3] = fmaf(w4.w, a1, acc1[co + 3]);
                    }
                } else {
#pragma unroll
                    for (int co = 0; co < COUT; ++co) {
                        acc0[co] = fmaf(w[co], a0, acc0[co]);
                        acc1[co] = fmaf(w[co], a1, acc1[co]);
                    }
                }
            }
        }
    }
    const long p0 = ((long)(x0 + tx) * n + (y0 + ty)) * n + (z0 + tz);
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        float v0 = acc0[co] + (bias ? bias[co] : 0.f), v1 = acc1[co] + (bias ? bias[co] : 0.f);
        if (RELU) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
        }
        y[((long)b * COUT + co) * n3 + p0] = v0;
        y[((long)b * COUT + co) * n3 + p0 + 4] = v1;
    }
}

// weight gradient: gW[co][ci][t] += sum_{b,p} g[b][co][p] x[b][ci][p + d_t];
// gb[co] += sum_{b,p} g[b][co][p].  One CTA = one tile of one sample; the
// (co, ci) plane is walked in chunks of 8 x 4 with the tile's g and x halo in
// shared memory; partial sums go to global memory with atomics.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NTH) conv_wgrad_kernel(int n, const float* __restrict__ x,
                                                         const float* __restrict__ g, float* __restrict__ gW,
                                                         float* __restrict__ gb) {
    constexpr int CC = CIN < 4 ? CIN : 4;
    constexpr int OC = COUT < 8 ? COUT : 8;
    __shared__ float s_in[CC][HALO][HALO][HALO];
    __shared__ float s_g[OC][TILE * TILE * TILE];
    const int tiles = n / TILE;
    const int tile = blockIdx.x % (tiles * tiles * tiles);
    const int b = blockIdx.x / (tiles * tiles * tiles);
    const int x0 = (tile / (tiles * tiles)) * TILE, y0 = ((tile / tiles) % tiles) * TILE, z0 = (tile % tiles) * TILE;
    const int tid = threadIdx.x;
    const long n3 = (long)n * n * n;
    for (int o0 = 0; o0 < COUT; o0 += OC) {
        __syncthreads();
        for (int i = tid; i < OC * 512; i += NTH) {
            const int oc = i / 512, v = i % 512;
            const int vx = v / 64, vy = (v / 8) % 8, vz = v % 8;
            s_g[oc][v] = g[((long)b * COUT + o0 + oc) * n3 + ((long)(x0 + vx) * n + (y0 + vy)) * n + (z0 + vz)];
        }
        __syncthreads();
        if (gb && tid < OC) {
            float s = 0.f;
            for (int v = 0; v < 512; ++v) s += s_g[tid][v];
            atomicAdd(gb + o0 + tid, s);
        }
        for (int c0 = 0; c0 < CIN; c0 += CC) {
            __syncthreads();
            for (int i = tid; i < CC * HALO * HALO * HALO; i += NTH) {
                const int cc = i / (HALO * HALO * HALO), r = i % (HALO * HALO * HALO);
                const int hx = r / (HALO * HALO), hy = (r / HALO) % HALO, hz = r % HALO;
                const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
                float v = 0.f;
                if (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
                    v = x[((long)b * CIN + c0 + cc) * n3 + ((long)gx * n + gy) * n + gz];
                s_in[cc][hx][hy][hz] = v;
            }
            __syncthreads();
            for (int e = tid; e < OC * CC * 27; e += NTH) {
                const int t = e % 27, cc = (e / 27) % CC, oc = e / (27 * CC);
                const int dx = t / 9, dy = (t / 3) % 3, dz = t % 3;
                float s = 0.f;
                for (int v = 0; v < 512; ++v) {
                    const int vx = v / 64, vy = (v / 8) % 8, vz = v % 8;
                    s = fmaf(s_g[oc][v], s_in[cc][vx + dx][vy + dy][vz + dz], s);
                }
                atomicAdd(gW + ((long)(o0 + oc) * CIN + c0 + cc) * 27 + t, s);
            }
        }
    }
}

// g <- g * (a > 0) (ReLU derivative through the stored activation a)
__global__ void relu_mask_kernel(long count, const float* __restrict__ a, float* __restrict__ g) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) g[i] = 0.f;
}

// backward-data weights: Wt[ci][co][t] = W[co][ci][26 - t] (transpose, flipped taps)
__global__ void transpose_flip_kernel(int cin, int cout, const __nv_bfloat16* __restrict__ W,
                                      __nv_bfloat16* __restrict__ Wt) {
    const long total = (long)cin * cout * 27;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int t = (int)(i % 27), co = (int)((i / 27) % cout), ci = (int)(i / (27L * cout));
        Wt[i] = W[((long)co * cin + ci) * 27 + (26 - t)];
    }
}

// FP32 master -> BF16 compute copy (weights only; biases stay FP32 in the master)
__global__ void to_bf16_kernel(long count, const float* __restrict__ w, __nv_bfloat16* __restrict__ o) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        o[i] = __float2bfloat16_rn(w[i]);
}

// MSE loss gradient dy = 2 (y - t) / count, loss accumulated into *loss
__global__ void mse_kernel(long count, const float* __restrict__ y, const float* __restrict__ t,
                           float* __restrict__ dy, float* __restrict__ loss) {
    float s = 0.f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)count;
        s += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, s / (float)count);
}

// Adam on the FP32 master parameters
__global__ void adam_kernel(long count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

template <int CIN, int COUT, bool RELU>
static void conv_fwd(int n, int batch, const float* x, const __nv_bfloat16* W, const float* bias, float* y,
                     cudaStream_t s) {
    const int tiles = n / TILE;
    conv_fwd_kernel<CIN, COUT, RELU><<<batch * tiles * tiles * tiles, NTH, 0, s>>>(n, x, W, bias, y);
}

template <int CIN, int COUT>
static void conv_wgrad(int n, int batch, const float* x, const float* g, float* gW, float* gb, cudaStream_t s) {
    const int tiles = n / TILE;
    conv_wgrad_kernel<CIN, COUT><<<batch * tiles * tiles * tiles, NTH, 0, s>>>(n, x, g, gW, gb);
}

// layer dispatch (the channel pattern is fixed)
static void layer_fwd(int l, int n, int batch, const float* x, const __nv_bfloat16* W, const float* b, float* y,
                      cudaStream_t s) {
    if (l == 0) conv_fwd<2, 32, true>(n, batch, x, W, b, y, s);
    else if (l < NL - 1) conv_fwd<32, 32, true>(n, batch, x, W, b, y, s);
    else conv_fwd<32, 1, false>(n, batch, x, W, b, y, s);
}

// input gradient of layer l: a convolution of g (COUT channels) with the
// transposed, flipped weights (CIN outputs), no bias
static void layer_dgrad(int l, int n, int batch, const float* g, const __nv_bfloat16* Wt, float* gin, cudaStream_t s) {
    if (l == NL - 1) conv_fwd<1, 32, false>(n, batch, g, Wt, nullptr, gin, s);
    else if (l > 0) conv_fwd<32, 32, false>(n, batch, g, Wt, nullptr, gin, s);
    // layer 0: the input gradient is not needed
}

static void layer_wgrad(int l, int n, int batch, const float* x, const float* g, float* gW, float* gb, cudaStream_t s) {
    if (l == 0) conv_wgrad<2, 32>(n, batch, x, g, gW, gb, s);
    else if (l < NL - 1) conv_wgrad<32, 32>(n, batch, x, g, gW, gb, s);
    else conv_wgrad<32, 1>(n, batch, x, g, gW, gb, s);
}

}  // namespace net
}  // namespace fks

using namespace fks;
using namespace fks::net;

struct fks_net {
    int n = 0, max_batch = 0;
    float* master = nullptr;          // FP32 parameters
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wbf = nullptr;     // BF16 weights per layer (packed like the master, biases unused)
    __nv_bfloat16* wt = nullptr;      // transposed-flipped BF16 weights (scratch for one layer)
    float* act[NL + 1] = {};          // activations: act[0] = input copy slot unused, act[l+1] = layer l output
    float* gbuf[2] = {};              // gradient ping-pong
    float* dy = nullptr;
    float* xbuf = nullptr;            // [max_batch][2][n^3] input workspace of the routing path
    long step = 0;
    long launches = 0;
    std::string err;
};

static fks_status nfail(fks_net* m, fks_status s, const std::string& e) {
    if (m) m->err = e;
    return s;
}

// counter-based normal draws (SplitMix64 + Box-Muller) for He initialisation
static double splitmix_uniform(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static fks_status refresh_bf16(fks_net* m, cudaStream_t s) {
    to_bf16_kernel<<<256, 256, 0, s>>>(NPARAM, m->master, m->wbf);
    m->launches += 1;
    return cudaGetLastError() == cudaSuccess ? FKS_OK : nfail(m, FKS_ERR_CUDA, "bf16 conversion");
}

static const float* bias_ptr(const fks_net* m, int l) { return m->master + layer_off(l) + layer_w(l); }
static const __nv_bfloat16* wbf_ptr(const fks_net* m, int l) { return m->wbf + layer_off(l); }

static fks_status run_forward(fks_net* m, int batch, const float* x, cudaStream_t s) {
    const float* in = x;
    for (int l = 0; l < NL; ++l) {
        layer_fwd(l, m->n, batch, in, wbf_ptr(m, l), bias_ptr(m, l), m->act[l + 1], s);
        in = m->act[l + 1];
        m->launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FKS_OK : nfail(m, FKS_ERR_CUDA, std::string("net forward: ") + cudaGetErrorString(e));
}

// gradient of sum(gy * y) with respect to the master parameters into m->grad
static fks_status run_backward(fks_net* m, int batch, const float* x, const float* gy, cudaStream_t s) {
    const long n3 = (long)m->n * m->n * m->n;
    if (cudaMemsetAsync(m->grad, 0, sizeof(float) * NPARAM, s) != cudaSuccess) return nfail(m, FKS_ERR_CUDA, "grad reset");
    const float* g = gy;
    int cur = 0;
    for (int l = NL - 1; l >= 0; --l) {
        const float* xin = l == 0 ? x : m->act[l];
        float* gW = m->grad + layer_off(l);
        float* gb = gW + layer_w(l);
        layer_wgrad(l, m->n, batch, xin, g, gW, gb, s);
        m->launches += 1;
        if (l > 0) {
            const int cin = CH[l], cout = CH[l + 1];
            transpose_flip_kernel<<<256, 256, 0, s>>>(cin, cout, wbf_ptr(m, l), m->wt);
            float* gin = m->gbuf[cur];
            layer_dgrad(l, m->n, batch, g, m->wt, gin, s);
            relu_mask_kernel<<<1024, 256, 0, s>>>((long)batch * cin * n3, m->act[l], gin);
            m->launches += 3;
            g = gin;
            cur ^= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FKS_OK : nfail(m, FKS_ERR_CUDA, std::string("net backward: ") + cudaGetErrorString(e));
}

const float* fks_net_forward_internal(fks_net* m, int batch, const float* x, cudaStream_t s, fks_status* st) {
    *st = run_forward(m, batch, x, s);
    return m->act[NL];
}
float* fks_net_input_buffer(fks_net* m) { return m->xbuf; }
int fks_net_grid(const fks_net* m) { return m->n; }
int fks_net_max_batch(const fks_net* m) { return m->max_batch; }

extern "C" {

fks_status fks_net_init(int n, int max_batch, unsigned long long seed, fks_net** out) {
    if (out) *out = nullptr;
    if (!out || n < TILE || n % TILE != 0 || n > 64 || max_batch < 1) return FKS_ERR_INVALID_ARG;
    fks_net* m = new (std::nothrow) fks_net();
    if (!m) return FKS_ERR_OOM;
    m->n = n;
    m->max_batch = max_batch;
    const long n3 = (long)n * n * n;
    bool ok = cudaMalloc(&m->master, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->grad, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->adam_m, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->adam_v, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->wbf, sizeof(__nv_bfloat16) * NPARAM) == cudaSuccess &&
              cudaMalloc(&m->wt, sizeof(__nv_bfloat16) * 32 * 32 * 27) == cudaSuccess &&
              cudaMalloc(&m->dy, sizeof(float) * max_batch * n3) == cudaSuccess &&
              cudaMalloc(&m->xbuf, sizeof(float) * max_batch * 2 * n3) == cudaSuccess;
    for (int l = 1; l <= NL && ok; ++l) ok = cudaMalloc(&m->act[l], sizeof(float) * max_batch * CH[l] * n3) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&m->gbuf[i], sizeof(float) * max_batch * 32 * n3) == cudaSuccess;
    if (!ok) {
        fks_net_destroy(m);
        return FKS_ERR_OOM;
    }
    // He initialisation (normal, std sqrt(2 / fan_in)), zero biases
    std::vector<float> h(NPARAM, 0.f);
    uint64_t st = seed;
    for (int l = 0; l < NL; ++l) {
        const double sd = std::sqrt(2.0 / (CH[l] * 27.0)) * (l == NL - 1 ? 0.1 : 1.0);
        for (long i = 0; i < layer_w(l); ++i) {
            const double u1 = splitmix_uniform(st), u2 = splitmix_uniform(st);
            h[layer_off(l) + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    cudaMemcpy(m->master, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    cudaMemset(m->adam_m, 0, sizeof(float) * NPARAM);
    cudaMemset(m->adam_v, 0, sizeof(float) * NPARAM);
    if (refresh_bf16(m, nullptr) != FKS_OK || cudaDeviceSynchronize() != cudaSuccess) {
        fks_net_destroy(m);
        return FKS_ERR_CUDA;
    }
    *out = m;
    return FKS_OK;
}

void fks_net_destroy(fks_net* m) {
    if (!m) return;
    cudaFree(m->master);
    cudaFree(m->grad);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->wbf);
    cudaFree(m->wt);
    cudaFree(m->dy);
    cudaFree(m->xbuf);
    for (int l = 1; l <= NL; ++l) cudaFree(m->act[l]);
    for (int i = 0; i < 2; ++i) cudaFree(m->gbuf[i]);
    delete m;
}

long fks_net_num_params(const fks_net* m) { return m ? NPARAM : -1; }
long fks_net_launch_count(const fks_net* m) { return m ? m->launches : -1; }
const char* fks_net_last_error(const fks_net* m) { return m ? m->err.c_str() : "null net"; }

fks_status fks_net_set_params(fks_net* m, const float* host, long count) {
    if (!m || !host || count != NPARAM) return FKS_ERR_INVALID_ARG;
    if (cudaMemcpy(m->master, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
        return nfail(m, FKS_ERR_CUDA, "parameter upload");
    fks_status st = refresh_bf16(m, nullptr);
    if (st == FKS_OK && cudaDeviceSynchronize() != cudaSuccess) st = nfail(m, FKS_ERR_CUDA, "sync");
    return st;
}

fks_status fks_net_get_params(fks_net* m, float* host, long count) {
    if (!m || !host || count != NPARAM) return FKS_ERR_INVALID_ARG;
    if (cudaMemcpy(host, m->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return nfail(m, FKS_ERR_CUDA, "parameter download");
    return FKS_OK;
}

fks_status fks_net_forward(fks_net* m, int batch, const float* x, float* y, void* stream) {
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return FKS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = run_forward(m, batch, x, s);
    if (st != FKS_OK) return st;
    const long n3 = (long)m->n * m->n * m->n;
    if (cudaMemcpyAsync(y, m->act[NL], sizeof(float) * batch * n3, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return nfail(m, FKS_ERR_CUDA, "output copy");
    return FKS_OK;
}

fks_status fks_net_gradient(fks_net* m, int batch, const float* x, const float* gy, float* grad, void* stream) {
    if (!m || !x || !gy || !grad || batch < 1 || batch > m->max_batch) return FKS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = run_forward(m, batch, x, s);
    if (st == FKS_OK) st = run_backward(m, batch, x, gy, s);
    if (st != FKS_OK) return st;
    if (cudaMemcpyAsync(grad, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return nfail(m, FKS_ERR_CUDA, "gradient copy");
    return FKS_OK;
}

fks_status fks_net_train_step(fks_net* m, int batch, const float* x, const float* target, float lr, float* loss,
                              void* stream) {
    if (!m || !x || !target || batch < 1 || batch > m->max_batch || !(lr > 0.f)) return FKS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long n3 = (long)m->n * m->n * m->n;
    fks_status st = run_forward(m, batch, x, s);
    if (st != FKS_OK) return st;
    mse_kernel<<<256, 256, 0, s>>>((long)batch * n3, m->act[NL], target, m->dy, loss);
    st = run_backward(m, batch, x, m->dy, s);
    if (st != FKS_OK) return st;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(b1, (double)m->step), c2 = 1.f - (float)std::pow(b2, (double)m->step);
    adam_kernel<<<256, 256, 0, s>>>(NPARAM, m->master, m->grad, m->adam_m, m->adam_v, lr, b1, b2, 1e-8f, c1, c2);
    m->launches += 2;
    return refresh_bf16(m, s);
}

}  // extern "C"
