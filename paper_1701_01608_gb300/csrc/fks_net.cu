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
#include <cuda.h>
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


// ---------------------------------------------------------------- tensor-core inference
//
// Implicit-GEMM convolution on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulation in tensor memory), used for inference.
// Activations are BF16 in chunks of 8 channels: [b][chunk][voxel][8] (2 or 4
// chunks), so that the halo of one chunk is a TMA box of contiguous voxels.
// A tile is 1 x 16 x 8 output voxels (x, y, z) = 128 rows of D; D[m][co] =
// sum_t sum_ci A_t[m][ci] B_t[ci][co] over the 27 taps t.  The tile's input
// halo (3 x 18 x 10 voxels) is stored as [k-chunk j][halo row r][8 channels]
// (16 bytes per row and chunk), so the A operand of every tap is a plain
// no-swizzle K-major descriptor into the halo: start row r0(t), 16-byte rows
// inside an 8-row core matrix (consecutive z), SBO = 10 rows (next y), LBO =
// one k-chunk plane.  No im2col copy.  Weights are pre-arranged per tap as
// [j][co][8 ci] and stay in shared memory for the CTA's lifetime.
namespace tc {

constexpr int TY = 16, TZ = 8;                  // tile: 1 x 16 x 8 voxels
constexpr int HX = 3, HY = TY + 2, HZ = TZ + 2;
constexpr int NTHR = 160;                       // warps 0-3: epilogue (TMEM lanes 0..127); warp 4: TMA + MMA

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major
template <int M, int N>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void fence_async_shared_cta() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(saddr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

constexpr uint32_t HPLANE = 8704;             // 128-aligned k-chunk plane of a halo tile (540 x 16 B = 8640)

// bounded wait; on a timeout record bit 3 and set *abort, after which no wait
// is taken again (the kernel runs to its end without waiting)
__device__ __forceinline__ void wait_bounded(uint64_t* bar, uint32_t parity, int* flags, volatile int* abort) {
    if (*abort) return;
    bool ok = false;
    for (long it = 0; it < (1L << 26) && !ok; ++it) ok = mbar_try(bar, parity);
    if (!ok) {
        atomicOr(flags, 8);
        *abort = 1;
    }
}

// Implicit-GEMM 3^3 convolution on the tensor cores, one tile of 1 x 16 x 8
// voxels (M = 128) per MMA group.  Activations are BF16 in chunks of 8
// channels, [cell][chunk][x][y][z][8].  The halo of a tile (3 x 18 x 10
// voxels, zero outside the grid) arrives by TMA as KC boxes (one per chunk,
// contiguous 16-byte voxels), one 16-byte row per voxel, so that tap t's A operand is
// the plane of k-chunk j shifted by the tap's row offset: a K-major descriptor
// with LBO = the plane stride and SBO = 10 rows (next y).  B: the tap's
// [KC][NP][16 B] weight block.  Warp-specialised pipeline per CTA: warp 4
// loads the halos (TMA, double-buffered) and issues the MMAs into two TMEM
// accumulators; warps 0-3 read an accumulator, release it (an mbarrier of 128
// arrivals) and store the tile, while the next tile's MMAs run.
template <int KC, int NP, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(NTHR, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap xmap, int n, int batch,
                                                          const __nv_bfloat16* __restrict__ wpk,
                                                          const float* __restrict__ bias, void* __restrict__ y,
                                                          int cout, int* flags) {
    constexpr uint32_t HALO_BYTES = KC * HPLANE;
    constexpr uint32_t W_BYTES = 27 * KC * NP * 16;
    constexpr uint32_t IDESC = instr_desc<128, NP>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations on 128-byte boundaries (the launch adds 128 bytes of slack)
    unsigned char* smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
    unsigned char* halo = smem;                          // [2][KC][HPLANE]
    unsigned char* wsm = smem + 2 * HALO_BYTES;          // [27][KC][NP][16 B]
    __shared__ uint64_t bar_ld[2], bar_mma[2], bar_free[2];   // halo landed, MMAs done, accumulator read
    __shared__ uint32_t tmem_base;
    __shared__ float sbias[32];
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (uint32_t i = tid; i < W_BYTES / 16; i += NTHR)
        reinterpret_cast<uint4*>(wsm)[i] = reinterpret_cast<const uint4*>(wpk)[i];
    if (tid < 32) sbias[tid] = tid < cout ? bias[tid] : 0.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(saddr(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init1(&bar_ld[i]);
            mbar_init1(&bar_mma[i]);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(saddr(&bar_free[i])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    fence_async_shared_cta();   // the weights (generic stores) before the tensor core reads them
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    const int ny = n / TY, nz = n / TZ;
    const long tiles = (long)batch * n * ny * nz;
    const long mine = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // tiles of this CTA
    const long n3 = (long)n * n * n;
    auto coords = [&](long i, int& b, int& x0, int& y0, int& z0) {
        const long tile = blockIdx.x + i * gridDim.x;
        z0 = (int)(tile % nz) * TZ;
        y0 = (int)((tile / nz) % ny) * TY;
        x0 = (int)((tile / ((long)nz * ny)) % n);
        b = (int)(tile / ((long)nz * ny * n));
    };
    auto load = [&](long i) {   // thread 0: the halo of tile i into buffer i & 1 (zero fill outside the grid)
        int b, x0, y0, z0;
        coords(i, b, x0, y0, z0);
        uint64_t* bar = &bar_ld[i & 1];
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(KC * 8640u)
                     : "memory");
        for (int j = 0; j < KC; ++j) {
            const uint32_t dst = saddr(halo + (i & 1) * HALO_BYTES + j * HPLANE);
            asm volatile(
                "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5, %6}], [%7];\n" ::"r"(dst),
                "l"(reinterpret_cast<uint64_t>(&xmap)), "r"(0), "r"(z0 - 1), "r"(y0 - 1), "r"(x0 - 1), "r"(b * KC + j),
                "r"(saddr(bar))
                : "memory");
        }
    };
    auto wait_halo = [&](long i) {   // thread 0: the halo of tile i has landed
        wait_bounded(&bar_ld[i & 1], (uint32_t)((i >> 1) & 1), flags, &s_abort);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    };
    auto mma = [&](long i) {   // thread 0: 27 taps x KC/2 k-steps of tile i into TMEM (i & 1) * 32
        // descriptors of base + off are the base descriptors + off / 16 (addresses < 2^18 bytes:
        // no carry out of the start-address field); every offset is a compile-time constant
        const uint64_t a0 = smem_desc(saddr(halo + (i & 1) * HALO_BYTES), HPLANE, HZ * 16u);
        const uint64_t b0 = smem_desc(saddr(wsm), NP * 16u, 128u);
        const uint32_t d = tmem + (uint32_t)(i & 1) * 32u;
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const uint32_t r0 = (uint32_t)(((t / 9) * HY + (t / 3) % 3) * HZ + t % 3);
#pragma unroll
            for (int s2 = 0; s2 < KC / 2; ++s2) {
                const uint64_t ad = a0 + ((2u * s2 * HPLANE + r0 * 16u) >> 4);
                const uint64_t bd = b0 + ((uint32_t)((t * KC + 2 * s2) * NP) * 16u >> 4);
                const uint32_t acc = (t > 0 || s2 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                    : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         saddr(&bar_mma[i & 1]))
                     : "memory");
    };
    if (warp == 4) {
        // producer: lane 0 loads halos and issues MMAs; the MMAs of tile i queue behind
        // those of tile i-1, whose completion frees the halo buffer for tile i+1
        if (lane == 0 && mine > 0) {
            load(0);
            if (mine > 1) load(1);
#pragma unroll 1
            for (long i = 0; i < mine; ++i) {
                wait_halo(i);
                if (i >= 2)   // the epilogue of tile i-2 has read accumulator i & 1
                    wait_bounded(&bar_free[i & 1], (uint32_t)(((i - 2) >> 1) & 1), flags, &s_abort);
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                mma(i);
                if (i >= 1) {
                    wait_bounded(&bar_mma[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), flags, &s_abort);
                    if (i + 1 < mine) load(i + 1);   // into the buffer of tile i-1
                }
            }
        }
    } else {
#pragma unroll 1
    for (long i = 0; i < mine; ++i) {
        wait_bounded(&bar_mma[i & 1], (uint32_t)((i >> 1) & 1), flags, &s_abort);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // epilogue: warp w reads D rows 32w .. 32w+31 (one voxel per thread)
        int b, x0, y0, z0;
        coords(i, b, x0, y0, z0);
        float v[NP];
        {
            const uint32_t taddr = tmem + (uint32_t)(i & 1) * 32u + ((uint32_t)(32 * warp) << 16);
            uint32_t r[NP];
            if constexpr (NP == 32) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
            } else {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int c = 0; c < NP; ++c) v[c] = __uint_as_float(r[c]);
        }
        // this thread's reads of accumulator i & 1 are done: release it to the producer
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(&bar_free[i & 1])) : "memory");
        const int m = 32 * warp + lane;
        const long vloc = ((long)x0 * n + (y0 + m / TZ)) * n + (z0 + m % TZ);   // voxel within the cell
        if constexpr (OUT_F32) {
            static_cast<float*>(y)[(long)b * n3 + vloc] = v[0] + sbias[0];
        } else {
            // chunk c of 8 channels at [cell][c][voxel][8]: consecutive voxels are 16 bytes apart
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float a = (8 * c + e < NP) ? v[8 * c + e] + sbias[8 * c + e] : 0.f;
                    if (RELU) a = fmaxf(a, 0.f);
                    h[e] = __float2bfloat16_rn(a);
                }
                __nv_bfloat16* yo = static_cast<__nv_bfloat16*>(y) + (((long)b * 4 + c) * n3 + vloc) * 8;
                *reinterpret_cast<uint4*>(yo) = *reinterpret_cast<const uint4*>(h);
            }
        }
    }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // every MMA has completed and been read
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem) : "memory");
}

// FP32 master weights of one layer -> [27][KC][NP][8] BF16 (zero padding)
__global__ void pack_weights_kernel(int cin, int cout, int KC, int NP, const float* __restrict__ W,
                                    __nv_bfloat16* __restrict__ out) {
    const long total = 27L * KC * NP * 8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int e = (int)(i % 8), co = (int)((i / 8) % NP), j = (int)((i / (8L * NP)) % KC), t = (int)(i / (8L * NP * KC));
        const int ci = 8 * j + e;
        out[i] = __float2bfloat16_rn(co < cout && ci < cin ? W[((long)co * cin + ci) * 27 + t] : 0.f);
    }
}

// FP32 [b][2][n^3] -> BF16 [b][2 chunks][n^3][8] (channels 2..15 zero)
__global__ void input_pack_kernel(long nvox, long n3, const float* __restrict__ x, __nv_bfloat16* __restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nvox; i += (long)gridDim.x * blockDim.x) {
        const long b = i / n3, p = i % n3;
        __align__(16) __nv_bfloat16 h[8];
        for (int c = 0; c < 8; ++c) h[c] = __float2bfloat16_rn(c < 2 ? x[(b * 2 + c) * n3 + p] : 0.f);
        reinterpret_cast<uint4*>(out)[(b * 2) * n3 + p] = *reinterpret_cast<const uint4*>(h);
        reinterpret_cast<uint4*>(out)[(b * 2 + 1) * n3 + p] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// tensor map of a BF16 activation in chunks of 8 channels, [batch][KC][n][n][n][8]
// (the chunk index folded into the last dimension), with a halo box of
// 8 channels x 10 (z) x 18 (y) x 3 (x) x 1 chunk: contiguous 16-byte voxels
static bool halo_map(CUtensorMap* m, const __nv_bfloat16* x, int n, int batch, int KC) {
    EncodeTiled enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[5] = {8, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)batch * KC};
    const cuuint64_t strides[4] = {16, 16ull * n, 16ull * n * n, 16ull * n * n * n};
    const cuuint32_t box[5] = {8, HZ, HY, HX, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(x), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KC, int NP, bool RELU, bool OUT_F32>
static cudaError_t launch_tc(int n, int batch, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias,
                             void* y, int cout, int* flags, cudaStream_t s) {
    alignas(64) CUtensorMap xmap;
    if (!halo_map(&xmap, x, n, batch, KC)) return cudaErrorInvalidValue;
    // two halo buffers and the weights; one CTA per SM (64 TMEM columns)
    const size_t smem = (size_t)2 * KC * HPLANE + (size_t)27 * KC * NP * 16 + 128;
    auto k = conv_tc_kernel<KC, NP, RELU, OUT_F32>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long tiles = (long)batch * n * (n / TY) * (n / TZ);
    const long grid = tiles < 152 ? tiles : 152;
    k<<<(unsigned)grid, NTHR, smem, s>>>(xmap, n, batch, w, bias, y, cout, flags);
    return cudaGetLastError();
}

}  // namespace tc

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
    // inference workspace (allocated on first use): ib cells per call
    int ib = 0;
    float* xbuf = nullptr;            // [ib][2][n^3] input workspace of the routing path
    float* yinf = nullptr;            // [ib][n^3] network output
    // tensor-core inference: packed BF16 weights per layer, BF16 activations in 8-channel chunks
    __nv_bfloat16* wpk[NL] = {};
    __nv_bfloat16* tact[2] = {};
    int* tflags = nullptr;
    long wver = 0, wpk_ver = -1;      // master-weight version, version packed in wpk
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
    m->wver += 1;
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

// cells per inference call of the routing path: enough CTAs to fill the GPU
// in the per-cell kernels around the network
constexpr int kInferChunk = 2 * 152;

static bool use_tc(const fks_net* m) { return m->n % tc::TY == 0; }

// inference workspace: the tensor-core path takes kInferChunk cells per call,
// the CUDA-core path (training activations) max_batch
static fks_status ensure_infer(fks_net* m) {
    if (m->ib > 0) return FKS_OK;
    const long n3 = (long)m->n * m->n * m->n;
    const int ib = use_tc(m) ? (m->max_batch > kInferChunk ? m->max_batch : kInferChunk) : m->max_batch;
    bool ok = cudaMalloc(&m->xbuf, sizeof(float) * ib * 2 * n3) == cudaSuccess &&
              cudaMalloc(&m->yinf, sizeof(float) * ib * n3) == cudaSuccess;
    if (ok && use_tc(m)) {
        ok = cudaMalloc(&m->tflags, sizeof(int)) == cudaSuccess && cudaMemset(m->tflags, 0, sizeof(int)) == cudaSuccess;
        for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&m->tact[i], sizeof(__nv_bfloat16) * ib * n3 * 32) == cudaSuccess;
        for (int l = 0; l < NL && ok; ++l) {
            const int KC = l == 0 ? 2 : 4, NP = l == NL - 1 ? 16 : 32;
            ok = cudaMalloc(&m->wpk[l], sizeof(__nv_bfloat16) * 27 * KC * NP * 8) == cudaSuccess;
        }
    }
    if (!ok) return nfail(m, alloc_failure(), "inference workspace");
    m->ib = ib;
    return FKS_OK;
}

// tensor-core inference (n a multiple of 16): output y[b][n^3] (FP32) in m->yinf
static fks_status run_infer_tc(fks_net* m, int batch, const float* x, cudaStream_t s) {
    const int n = m->n;
    const long n3 = (long)n * n * n;
    if (!use_tc(m)) return nfail(m, FKS_ERR_UNSUPPORTED, "tensor-core inference needs n % 16 == 0");
    fks_status st = ensure_infer(m);
    if (st != FKS_OK) return st;
    if (batch < 1 || batch > m->ib) return nfail(m, FKS_ERR_INVALID_ARG, "inference batch above the workspace");
    if (m->wpk_ver != m->wver) {   // weights changed since they were packed
        for (int l = 0; l < NL; ++l) {
            const int KC = l == 0 ? 2 : 4, NP = l == NL - 1 ? 16 : 32;
            tc::pack_weights_kernel<<<128, 256, 0, s>>>(CH[l], CH[l + 1], KC, NP, m->master + layer_off(l), m->wpk[l]);
        }
        m->launches += NL;
        m->wpk_ver = m->wver;
    }
    tc::input_pack_kernel<<<1024, 256, 0, s>>>((long)batch * n3, n3, x, m->tact[0]);
    m->launches += 1;
    cudaError_t e = cudaSuccess;
    int cur = 0;
    for (int l = 0; l < NL && e == cudaSuccess; ++l) {
        const float* bias = bias_ptr(m, l);
        if (l == 0)
            e = tc::launch_tc<2, 32, true, false>(n, batch, m->tact[0], m->wpk[0], bias, m->tact[1], 32, m->tflags, s);
        else if (l < NL - 1)
            e = tc::launch_tc<4, 32, true, false>(n, batch, m->tact[cur], m->wpk[l], bias, m->tact[cur ^ 1], 32,
                                                  m->tflags, s);
        else
            e = tc::launch_tc<4, 16, false, true>(n, batch, m->tact[cur], m->wpk[l], bias, m->yinf, 1, m->tflags, s);
        if (l > 0) cur ^= 1;
        else cur = 1;
        m->launches += 1;
    }
    return e == cudaSuccess ? FKS_OK : nfail(m, FKS_ERR_CUDA, std::string("tensor-core inference: ") + cudaGetErrorString(e));
}

const float* fks_net_infer_internal(fks_net* m, int batch, const float* x, cudaStream_t s, fks_status* st) {
    if (use_tc(m)) {
        *st = run_infer_tc(m, batch, x, s);
        return m->yinf;
    }
    *st = run_forward(m, batch, x, s);
    return m->act[NL];
}

const float* fks_net_forward_internal(fks_net* m, int batch, const float* x, cudaStream_t s, fks_status* st) {
    *st = run_forward(m, batch, x, s);
    return m->act[NL];
}
int fks_net_infer_capacity(fks_net* m) { return ensure_infer(m) == FKS_OK ? m->ib : 0; }
float* fks_net_input_buffer(fks_net* m) { return ensure_infer(m) == FKS_OK ? m->xbuf : nullptr; }
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
              cudaMalloc(&m->dy, sizeof(float) * max_batch * n3) == cudaSuccess;
    for (int l = 1; l <= NL && ok; ++l) ok = cudaMalloc(&m->act[l], sizeof(float) * max_batch * CH[l] * n3) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&m->gbuf[i], sizeof(float) * max_batch * 32 * n3) == cudaSuccess;
    if (!ok) {
        const fks_status st = alloc_failure();
        fks_net_destroy(m);
        return st;
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
    cudaFree(m->yinf);
    for (int l = 0; l < NL; ++l) cudaFree(m->wpk[l]);
    for (int i = 0; i < 2; ++i) cudaFree(m->tact[i]);
    cudaFree(m->tflags);
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

fks_status fks_net_infer(fks_net* m, int batch, const float* x, float* y, void* stream) {
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return FKS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    fks_status st = run_infer_tc(m, batch, x, s);
    if (st != FKS_OK) return st;
    const long n3 = (long)m->n * m->n * m->n;
    if (cudaMemcpyAsync(y, m->yinf, sizeof(float) * batch * n3, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return nfail(m, FKS_ERR_CUDA, "output copy");
    return FKS_OK;
}

fks_status fks_net_check(fks_net* m, void* stream) {
    if (!m) return FKS_ERR_INVALID_ARG;
    int h = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return nfail(m, FKS_ERR_CUDA, "sync");
    if (m->tflags) {
        if (cudaMemcpy(&h, m->tflags, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FKS_ERR_CUDA;
        cudaMemset(m->tflags, 0, sizeof(int));
    }
    return (h & 8) ? nfail(m, FKS_ERR_TIMEOUT, "tensor-core MMA completion wait timed out") : FKS_OK;
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
