// fks_collide_tc.cu -- the fast spectral collision operator with every
// discrete Fourier transform on the tensor cores (tcgen05), in split BF16.
//
// The operator is the one of the cluster kernel (Appendix A: Fourier
// coefficients of f*, gain = sum over the M half-sphere directions of
// IDFT(alpha_p F) IDFT(w_p alphap_p F), loss f* IDFT(betaL F), Q = (G - L)/Kn,
// FP64 conservation projection, Euler step of Eq. disc_relax); only the
// arithmetic of the transforms differs.  A 3-D transform is three passes of
// one-axis DFTs, and one pass over the N^2 lines of a cell is a dense real
// product [lines x 2N] (re | im) times the 2N x 2N real form of the N-point
// DFT matrix.  Both factors are split into BF16 pairs x = hi + lo
// (hi = bf16(x), lo = bf16(x - hi)) and the product is hi*hi + lo*hi + hi*lo,
// accumulated in FP32 in tensor memory (the dropped lo*lo term is ~2^-18 of
// the product).  Everything between the passes (table products, the splits,
// the gain update, the loss, the projection) is FP32 on the CUDA cores with
// FP64 moment sums.
//
// Since alpha_p F and w_p alphap_p F are Hermitian (real, even tables times
// the transform of a real f), one complex inverse transform of
// (alpha_p + i w_p alphap_p) F gives a_p + i b_p: 1 + M + 1 complex 3-D
// transforms per cell.
//
// Work split: one CTA of 512 threads per cell (persistent over cells); warp w
// reads TMEM lanes 32 (w % 4) .. +31 and a quarter (w / 4) of the columns.  Passes 1 (along z) and 2 (along y) run for a group of
// 8 x-planes at a time entirely on chip: each pass's epilogue reads its
// accumulators from TMEM and writes the next operand, transposed, into shared
// memory.  Pass 3 (along x) needs every plane, so the second epilogue writes
// its operand through a per-CTA scratch in global memory (L2 resident) with
// bulk copies, and pass 3 reads it back tile by tile.  The gain accumulates in
// TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "fks_collide.cuh"
#include "fks_internal.h"

namespace fks {
namespace tcd {

template <int N>
struct Cfg {
    static constexpr int K = 2 * N;                    // real width of a complex line (re | im)
    static constexpr int KCH = K / 8;                  // 16-byte k-chunks of an operand row
    static constexpr int KSTEPS = K / 16;              // MMA k-steps (K = 16 per instruction)
    static constexpr long N3 = (long)N * N * N;
    static constexpr int TILES = N * N / 128;          // 128-line tiles of one pass
    static constexpr int GX = 8;                       // x-planes per group (passes 1, 2)
    static constexpr int GROUPS = N / GX;
    static constexpr int GROWS = GX * N;               // operand rows of a group
    static constexpr int GT = GROWS / 128;             // tiles of a group
    // group operands: [split][k-chunk][GROWS rows][16 B]; the plane is padded
    // by 32 bytes so that the transposing stores of a warp hit distinct banks
    static constexpr uint32_t GPLANE = GROWS * 16 + 32;
    static constexpr uint32_t GSPLIT = KCH * GPLANE;
    static constexpr uint32_t GBUF = 2 * GSPLIT;
    // DFT matrices: [dir][split][k-chunk][K output rows][16 B]
    static constexpr uint32_t BPLANE = K * 16;
    static constexpr uint32_t BMAT = KCH * BPLANE;
    // pass-3 tiles: [split][k-chunk][128 rows][16 B]
    static constexpr uint32_t TPLANE = 128 * 16;
    static constexpr uint32_t TSPLIT = KCH * TPLANE;
    static constexpr long A3_CELL = 2L * TILES * TSPLIT;     // pass-3 operands of one cell (bytes)
    // shared memory: the DFT matrices of the current direction (hi, lo), group
    // buffers A1 and A2, the staging of the second epilogue; pass 3
    // double-buffers its tiles over A1|A2
    static constexpr uint32_t SM_B = 0;
    static constexpr uint32_t SM_A1 = SM_B + 2 * BMAT;
    static constexpr uint32_t SM_A2 = SM_A1 + GBUF;
    static constexpr uint32_t STAGE = 4 * TILES * TPLANE;
    static constexpr uint32_t SM_ST = SM_A2 + GBUF;
    static constexpr uint32_t SMEM = SM_ST + STAGE;
    static_assert(4 * TSPLIT <= 2 * GBUF, "two pass-3 tiles fit in A1|A2");
    // tensor memory columns
    static constexpr int ACC1 = 0;                     // pass-1 accumulators (GT x K)
    static constexpr int ACC2 = GT * K;                // pass-2 accumulators (GT x K)
    static constexpr int GCOL = 2 * GT * K;            // gain, then Q: TILES x N
    static constexpr int USED = GCOL + TILES * N;
    static constexpr int TCOLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    static_assert(USED <= 512, "tensor memory");
    static_assert(2 * K <= GCOL, "pass-3 accumulators below the gain");
};

// ---------------------------------------------------------------- tcgen05

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int Nn) {
    // D FP32, A and B BF16, both K-major, N >> 3, M >> 4
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Nn >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// shared-memory matrix descriptor, no swizzle, K-major: rows of 16 bytes,
// 8-row core matrices SBO apart along M/N, k-chunks LBO apart along K
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// bulk copy shared -> global (async proxy), completion by bulk groups
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// operand lists of the 32x32b TMEM loads and stores (4, 8 and 16 columns); a
// wait ties the loaded registers so that no use is scheduled before it
__device__ __forceinline__ void tld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void twait4(uint32_t (&r)[4]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])::"memory");
}
__device__ __forceinline__ void tst4(uint32_t taddr, const uint32_t (&r)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
                 : "memory");
}
__device__ __forceinline__ void tld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void twait8(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])::"memory");
}
__device__ __forceinline__ void tst8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void twait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])::"memory");
}
__device__ __forceinline__ void tst16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}

// X consecutive TMEM columns of this thread's lane <-> registers
template <int X>
struct TCols;
#define FKS_TCOLS(X)                                                                   \
    template <>                                                                        \
    struct TCols<X> {                                                                  \
        /* two X-column groups (re and im of a D slice) with one wait */               \
        static __device__ __forceinline__ void load2(uint32_t t0, uint32_t t1, float* u, float* v) { \
            uint32_t r[X], q[X];                                                       \
            tld##X(t0, r);                                                             \
            tld##X(t1, q);                                                             \
            twait##X(r);                                                               \
            twait##X(q);                                                               \
            _Pragma("unroll") for (int i = 0; i < X; ++i) {                            \
                u[i] = __uint_as_float(r[i]);                                          \
                v[i] = __uint_as_float(q[i]);                                          \
            }                                                                          \
        }                                                                              \
        static __device__ __forceinline__ void load(uint32_t t, float* u) {            \
            uint32_t r[X];                                                             \
            tld##X(t, r);                                                              \
            twait##X(r);                                                               \
            _Pragma("unroll") for (int i = 0; i < X; ++i) u[i] = __uint_as_float(r[i]); \
        }                                                                              \
        static __device__ __forceinline__ void store(uint32_t t, const float* u) {     \
            uint32_t r[X];                                                             \
            _Pragma("unroll") for (int i = 0; i < X; ++i) r[i] = __float_as_uint(u[i]); \
            tst##X(t, r);                                                              \
        }                                                                              \
    };
FKS_TCOLS(4)
FKS_TCOLS(8)
FKS_TCOLS(16)
#undef FKS_TCOLS

// BF16 split of an FP32 value: x = hi + lo + O(2^-18 |x|)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

struct Args {
    const float* f;
    float* out;
    const float2* tab;          // [M+1][N][N][N]: (alpha N^-3, w alphap N^-3); slot M (betaL N^-3, 0)
    const uint4* dft;           // [dir][split][k-chunk][K][16 B] BF16 DFT matrices, dir 0 forward
    float2* fh;                 // [gridDim.x][N^3] Fourier coefficients of the CTA's current cell
    unsigned char* a3;          // [gridDim.x][A3_CELL] pass-3 operands of the CTA's current cell
    const signed char* delta;   // [3][N] cell shifts of the transport (step mode) or nullptr
    int* flags;                 // health bits
    long ncells;                // cells to process (entries of `cells`, if given)
    const int* cells;           // optional list of cell indices (routed cells), else 0 .. ncells-1
    const int* cells_count;     // optional device count of `cells` (replaces ncells)
    int* esc_list;              // precision escalation (as in the cluster kernel): cells whose bound
    int* esc_count;             //   esc_c ||L|| / Kn exceeds esc_tol ||Q|| are listed here, not written
    double esc_c2, esc_tol2;
    int* esc_last_list;         //   cells beyond the next tier's reach (bound with esc_last_c2) go to
    int* esc_last_count;        //   the last tier's list instead (nullptr: all to esc_list)
    double esc_last_c2;
    int nc[3], bc[3];
    int M;
    double L, inv_kn, dt;
    int mode;                   // 0 collide, 1 step
    double P[25];
};

constexpr int NTH = 512;   // 16 warps: warp w owns TMEM lanes 32 (w % 4) .. +31, column slice w / 4
constexpr int BULK = 32;   // the thread (warp 1) that issues and completes the bulk stores

template <int N>
__global__ void __launch_bounds__(NTH, 1) collide_tc_kernel(const __grid_constant__ Args a) {
    using C = Cfg<N>;
    constexpr int K = C::K, KCH = C::KCH, TILES = C::TILES, GT = C::GT, GROWS = C::GROWS;
    constexpr int ZS = N / 4;          // columns of one slice (of re, and of im)
    constexpr long N3 = C::N3;
    constexpr uint32_t ID = idesc_bf16(128, K);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar1, bar2, bar3[2], bar_ld;   // pass-1, pass-2, pass-3 MMAs; pass-3 loads
    __shared__ uint32_t tmem_base;
    __shared__ long zoff[N];
    __shared__ int dsm[3 * N];
    __shared__ float vg[N];
    __shared__ double vgd[N];
    __shared__ double red[NTH / 32][7];
    __shared__ double mu[5];
    __shared__ int s_abort, s_esc;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cs = warp >> 2;
    const uint32_t sbase = smem_addr(smem);
    const bool transport = a.delta != nullptr;
    for (int i = tid; i < 3 * N; i += NTH) dsm[i] = transport ? (int)a.delta[i] : 0;
    const double dv = 2.0 * a.L / N;
    if (tid < N) {
        vgd[tid] = ((double)tid + 0.5 - 0.5 * N) * dv;
        vg[tid] = (float)vgd[tid];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                     "r"(C::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar1, 1);
        mbar_init(&bar2, 1);
        mbar_init(&bar3[0], 1);
        mbar_init(&bar3[1], 1);
        mbar_init(&bar_ld, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = tmem + ((uint32_t)(32 * quad) << 16);   // this warp's TMEM lanes
    // mbarrier phases; every barrier has at most one commit or load outstanding
    uint32_t ph1 = 0, ph2 = 0, ph3a = 0, ph3b = 0, ph_ld = 0;
    float2* fh = a.fh + (long)blockIdx.x * N3;
    unsigned char* a3 = a.a3 + (long)blockIdx.x * C::A3_CELL;
    const int ncx = a.nc[0], ncy = a.nc[1], ncz = a.nc[2];

    // bounded waits: a timeout records bit 3; after it no wait is taken again
    // and the kernel ends after the current cell
    auto wait_bar = [&](uint64_t* bar, uint32_t& ph) {
        if (s_abort) {
            ph ^= 1u;
            return;
        }
        bool ok = false;
        for (long it = 0; it < (1L << 26) && !ok; ++it) ok = mbar_try_wait(bar, ph);
        ph ^= 1u;
        if (!ok) {
            atomicOr(a.flags, 8);
            s_abort = 1;
        }
    };
    // MMAs of one pass over ntile 128-row tiles of an operand in shared memory.
    // The start-address field of a descriptor is the address >> 4 in its low
    // bits, so a descriptor of base + off is the base descriptor + off / 16
    // (every address here is below 2^18 bytes: no carry out of the field).
    auto issue = [&](uint32_t abase, uint32_t aplane, uint32_t asplit, int ntile, uint32_t bbase, uint32_t dcol,
                     uint64_t* bar) {
        const uint64_t a0 = sdesc(abase, aplane, 128), b0 = sdesc(bbase, C::BPLANE, 128);
        for (int tt = 0; tt < ntile; ++tt) {
#pragma unroll
            for (int s = 0; s < C::KSTEPS; ++s) {
                const uint64_t ah = a0 + ((2u * s * aplane + (uint32_t)tt * 2048u) >> 4);
                const uint64_t al = ah + (asplit >> 4);
                const uint64_t bh = b0 + ((2u * s * C::BPLANE) >> 4);
                const uint64_t bl = bh + (C::BMAT >> 4);
                const uint32_t d = tmem + dcol + (uint32_t)tt * K;
                mma(d, ah, bh, ID, s > 0 ? 1u : 0u);
                mma(d, al, bh, ID, 1u);
                mma(d, ah, bl, ID, 1u);
            }
        }
        commit(bar);
    };

    const long nitems = a.cells_count ? (long)*a.cells_count : a.ncells;
    for (long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const long cell = a.cells ? (long)a.cells[item] : item;
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
        if (tid < N) {
            if (!transport) {
                zoff[tid] = cell * N3 + tid;
            } else {
                int fz;
                const int sz = fold_cell(cz - dsm[2 * N + tid], ncz, a.bc[2], fz);
                zoff[tid] = (long)sz * N3 + (fz ? N - 1 - tid : tid);
            }
        }
        __syncthreads();
        if (s_abort) break;
        // f* row (x, y, :) of the transported cell: element z at frow[zoff[z]]
        auto frow = [&](int x, int y) -> const float* {
            if (!transport) return a.f + ((long)x * N + y) * N;
            int fx, fy;
            const int sx = fold_cell(cx - dsm[x], ncx, a.bc[0], fx);
            const int sy = fold_cell(cy - dsm[N + y], ncy, a.bc[1], fy);
            const int qx = fx ? N - 1 - x : x, qy = fy ? N - 1 - y : y;
            return a.f + ((long)sx * ncy + sy) * ncz * N3 + ((long)qx * N + qy) * N;
        };
        double s5[5] = {0, 0, 0, 0, 0};
        float e_ll = 0.f, e_qq = 0.f;   // escalation bound: sum (f* l)^2, sum q^2

        // transform t: -1 forward (f* -> fh), 0..M-1 gain directions, M loss
        for (int t = -1; t <= a.M; ++t) {
            const bool fwd = t < 0;
            const uint32_t bdir = sbase + C::SM_B;
            if (t <= 0) {
                // DFT matrices of this direction (the previous transform's MMAs have completed)
                const uint4* src = a.dft + (fwd ? 0 : 2 * C::BMAT / 16);
                for (uint32_t i = tid; i < 2 * C::BMAT / 16; i += NTH) reinterpret_cast<uint4*>(smem + C::SM_B)[i] = src[i];
            }

            // pass-1 operand of group g into A1: rows m = xl N + y, line (x, y, :) along z.
            // Unit e = (row, z pair): consecutive threads take consecutive pairs of a row,
            // so the loads of a warp are contiguous; each thread writes its 4-byte piece
            // (two BF16) of the 16-byte chunks of re and im, hi and lo.
            auto build = [&](int g) {
                constexpr int PAIRS = N / 2;
                constexpr int EPT = GROWS * PAIRS / NTH;   // units per thread (8 at n = 32, 2 at n = 16)
                static_assert(GROWS * PAIRS % NTH == 0, "whole units per thread");
                float r0[EPT], i0[EPT], r1[EPT], i1[EPT];
                if (fwd) {
#pragma unroll
                    for (int u = 0; u < EPT; ++u) {
                        const int e = tid + u * NTH, m = e / PAIRS, z2 = e % PAIRS;
                        const float* fr = frow(C::GX * g + m / N, m % N);
                        r0[u] = fr[zoff[2 * z2]];
                        r1[u] = fr[zoff[2 * z2 + 1]];
                        i0[u] = i1[u] = 0.f;
                    }
                } else {
                    // all loads of the thread first: EPT coefficient and EPT table vectors in flight
                    float4 fv[EPT], tv[EPT];
                    const float4* F4 = reinterpret_cast<const float4*>(fh + (long)C::GX * g * N * N);
                    const float4* T4 = reinterpret_cast<const float4*>(a.tab + ((long)t * N + C::GX * g) * N * N);
#pragma unroll
                    for (int u = 0; u < EPT; ++u) {
                        fv[u] = F4[tid + u * NTH];
                        tv[u] = __ldg(T4 + tid + u * NTH);
                    }
#pragma unroll
                    for (int u = 0; u < EPT; ++u) {
                        r0[u] = fv[u].x * tv[u].x - fv[u].y * tv[u].y;
                        i0[u] = fv[u].x * tv[u].y + fv[u].y * tv[u].x;
                        r1[u] = fv[u].z * tv[u].z - fv[u].w * tv[u].w;
                        i1[u] = fv[u].z * tv[u].w + fv[u].w * tv[u].z;
                    }
                }
#pragma unroll
                for (int u = 0; u < EPT; ++u) {
                    const int e = tid + u * NTH, m = e / PAIRS, z2 = e % PAIRS;
                    const __nv_bfloat162 hr = __floats2bfloat162_rn(r0[u], r1[u]);
                    const __nv_bfloat162 hi = __floats2bfloat162_rn(i0[u], i1[u]);
                    const float2 fr2 = __bfloat1622float2(hr), fi2 = __bfloat1622float2(hi);
                    const __nv_bfloat162 lr = __floats2bfloat162_rn(r0[u] - fr2.x, r1[u] - fr2.y);
                    const __nv_bfloat162 li = __floats2bfloat162_rn(i0[u] - fi2.x, i1[u] - fi2.y);
                    const int c = z2 / 4;   // chunk of z = 2 z2 (8 z per chunk)
                    unsigned char* dre = smem + C::SM_A1 + c * C::GPLANE + m * 16 + (z2 % 4) * 4;
                    unsigned char* dim = dre + (N / 8) * C::GPLANE;
                    *reinterpret_cast<__nv_bfloat162*>(dre) = hr;
                    *reinterpret_cast<__nv_bfloat162*>(dre + C::GSPLIT) = lr;
                    *reinterpret_cast<__nv_bfloat162*>(dim) = hi;
                    *reinterpret_cast<__nv_bfloat162*>(dim + C::GSPLIT) = li;
                }
                fence_async_smem();
                fence_before();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    issue(sbase + C::SM_A1, C::GPLANE, C::GSPLIT, GT, bdir, C::ACC1, &bar1);
                }
            };

            // Group pipeline: build(g+1) runs beside the pass-2 MMAs of g, and the
            // second epilogue of g beside the pass-1 MMAs of g+1; the bulk stores of
            // g's staging drain while group g+1 runs its first epilogue.
            build(0);
            for (int g = 0; g < C::GROUPS; ++g) {
                wait_bar(&bar1, ph1);   // A2 and ACC2 were released when pass 2 of g-1 completed
                fence_after();
                // ---- epilogue 1: line (xl, y) -> pass-2 operand rows m2 = z' 8 + xl, k = y (re), N + y (im)
#pragma unroll 1
                for (int tt = 0; tt < GT; ++tt) {
                    const int m = 128 * tt + 32 * quad + lane;
                    const int xl = m / N, y = m % N;
                    float dr[ZS], di[ZS];
                    const uint32_t tc = tlane + C::ACC1 + tt * K + ZS * cs;
                    TCols<ZS>::load2(tc, tc + N, dr, di);
                    unsigned char* base =
                        smem + C::SM_A2 + (y / 8) * C::GPLANE + xl * 16 + (y % 8) * 2 + ZS * cs * 128;
                    unsigned char* bim = base + (N / 8) * C::GPLANE;
#pragma unroll
                    for (int z = 0; z < ZS; ++z) {
                        __nv_bfloat16 h, l;
                        split_bf16(dr[z], h, l);
                        *reinterpret_cast<__nv_bfloat16*>(base + z * 128) = h;
                        *reinterpret_cast<__nv_bfloat16*>(base + z * 128 + C::GSPLIT) = l;
                        split_bf16(di[z], h, l);
                        *reinterpret_cast<__nv_bfloat16*>(bim + z * 128) = h;
                        *reinterpret_cast<__nv_bfloat16*>(bim + z * 128 + C::GSPLIT) = l;
                    }
                }
                if (tid == BULK) bulk_wait_read();   // the staging of g-1 has been read out
                fence_async_smem();
                fence_before();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    issue(sbase + C::SM_A2, C::GPLANE, C::GSPLIT, GT, bdir, C::ACC2, &bar2);
                }
                if (g + 1 < C::GROUPS) build(g + 1);   // A1 and ACC1 are free
                wait_bar(&bar2, ph2);
                fence_after();
                // ---- epilogue 2: line (z', xl) along y -> staging of the pass-3 operand:
                // row r = y' N + z' of tile r / 128, k = x (re) or N + x (im); blocks
                // [split][part][tile][128 rows][16 B]
#pragma unroll 1
                for (int tt = 0; tt < GT; ++tt) {
                    const int m2 = 128 * tt + 32 * quad + lane;
                    const int z = m2 / 8, xl = m2 % 8;
                    float dr[ZS], di[ZS];
                    const uint32_t tc = tlane + C::ACC2 + tt * K + ZS * cs;
                    TCols<ZS>::load2(tc, tc + N, dr, di);
#pragma unroll
                    for (int j = 0; j < ZS; ++j) {
                        const int r = (ZS * cs + j) * N + z;
                        unsigned char* b0 = smem + C::SM_ST + (r / 128) * C::TPLANE + (r % 128) * 16 + xl * 2;
                        __nv_bfloat16 h, l;
                        split_bf16(dr[j], h, l);   // re: part 0
                        *reinterpret_cast<__nv_bfloat16*>(b0) = h;
                        *reinterpret_cast<__nv_bfloat16*>(b0 + 2 * TILES * C::TPLANE) = l;
                        split_bf16(di[j], h, l);   // im: part 1
                        *reinterpret_cast<__nv_bfloat16*>(b0 + TILES * C::TPLANE) = h;
                        *reinterpret_cast<__nv_bfloat16*>(b0 + 3 * TILES * C::TPLANE) = l;
                    }
                }
                fence_async_smem();
                fence_before();
                __syncthreads();
                if (tid == BULK) {
                    // block (split, part, tile) -> global k-chunk part * KCH/2 + g of that tile
                    for (int sp = 0; sp < 2; ++sp)
                        for (int part = 0; part < 2; ++part)
                            for (int T = 0; T < TILES; ++T) {
                                unsigned char* dst =
                                    a3 + ((long)(sp * TILES + T) * KCH + part * (KCH / 2) + g) * C::TPLANE;
                                const uint32_t src = sbase + C::SM_ST + ((sp * 2 + part) * TILES + T) * C::TPLANE;
                                bulk_s2g(dst, src, C::TPLANE);
                            }
                    bulk_commit();
                }
            }
            // every pass-3 operand of this transform is in global memory
            if (tid == BULK) bulk_wait_all();
            __syncthreads();

            // ---- pass 3 (along x): tiles double-buffered in A1|A2 and in TMEM; the MMAs
            // of tile T+1 run beside the epilogue of tile T
            auto load_tile = [&](int T) {
                const uint32_t buf = C::SM_A1 + (uint32_t)(T & 1) * 2u * C::TSPLIT;
                mbar_expect_tx(&bar_ld, 2 * C::TSPLIT);
                for (int sp = 0; sp < 2; ++sp)
                    bulk_g2s(smem + buf + sp * C::TSPLIT, a3 + (long)(sp * TILES + T) * KCH * C::TPLANE, C::TSPLIT,
                             &bar_ld);
            };
            auto mma_tile = [&](int T) {   // thread 0: tile T has landed -> MMAs into accumulator T & 1
                wait_bar(&bar_ld, ph_ld);
                fence_after();
                issue(sbase + C::SM_A1 + (uint32_t)(T & 1) * 2u * C::TSPLIT, C::TPLANE, C::TSPLIT, 1, bdir,
                      (uint32_t)(T & 1) * K, &bar3[T & 1]);
            };
            if (tid == 0) {
                load_tile(0);
                mma_tile(0);
                if (TILES > 1) load_tile(1);
            }
#pragma unroll 1
            for (int T = 0; T < TILES; ++T) {
                if (tid == 0 && T + 1 < TILES) mma_tile(T + 1);   // accumulator (T+1) & 1 was read by tile T-1
                wait_bar(&bar3[T & 1], (T & 1) ? ph3b : ph3a);
                fence_after();
                if (tid == 0 && T + 2 < TILES) load_tile(T + 2);   // buffer T & 1: the MMAs of tile T are done
                // epilogue 3: line (y', z') along x, outputs x' of this warp's slice
                const int r = 128 * T + 32 * quad + lane, yy = r / N, zz = r % N;
                const int x0 = ZS * cs;
                float dr[ZS], di[ZS];
                const uint32_t tc = tlane + (uint32_t)(T & 1) * K + x0;
                TCols<ZS>::load2(tc, tc + N, dr, di);
                const uint32_t gaddr = tlane + C::GCOL + (uint32_t)T * N + x0;
                if (fwd) {
#pragma unroll
                    for (int j = 0; j < ZS; ++j) fh[((long)(x0 + j) * N + yy) * N + zz] = make_float2(dr[j], di[j]);
                } else if (t < a.M) {
                    float gv[ZS];
                    if (t == 0) {
#pragma unroll
                        for (int j = 0; j < ZS; ++j) gv[j] = dr[j] * di[j];
                    } else {
                        TCols<ZS>::load(gaddr, gv);
#pragma unroll
                        for (int j = 0; j < ZS; ++j) gv[j] = fmaf(dr[j], di[j], gv[j]);
                    }
                    TCols<ZS>::store(gaddr, gv);
                    wait_st();
                } else {
                    // loss: r = G - f* l (one rounding), q = r / Kn; FP64 moment sums
                    float gv[ZS];
                    TCols<ZS>::load(gaddr, gv);
                    const float kn = (float)a.inv_kn;
                    double sr = 0.0, sx = 0.0, sxx = 0.0;
#pragma unroll
                    for (int j = 0; j < ZS; ++j) {
                        const float fv = frow(x0 + j, yy)[zoff[zz]];
                        const float q = fmaf(-fv, dr[j], gv[j]) * kn;
                        const float lz = fv * dr[j];
                        e_ll = fmaf(lz, lz, e_ll);
                        e_qq = fmaf(q, q, e_qq);
                        gv[j] = q;
                        const double qd = (double)q, vx = vgd[x0 + j];
                        sr += qd;
                        sx = fma(qd, vx, sx);
                        sxx = fma(qd, 0.5 * vx * vx, sxx);
                    }
                    TCols<ZS>::store(gaddr, gv);
                    wait_st();
                    const double vy = vgd[yy], vz = vgd[zz];
                    s5[0] += sr;
                    s5[1] += sx;
                    s5[2] = fma(sr, vy, s5[2]);
                    s5[3] = fma(sr, vz, s5[3]);
                    s5[4] += sxx + sr * 0.5 * (vy * vy + vz * vz);
                }
                fence_before();
                __syncthreads();
            }
        }
        if (s_abort) break;

        // ---- projection: mu = P sum phi Q (FP64), Q -= phi . mu; output
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            double v = s5[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][i] = v;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            e_ll += __shfl_xor_sync(0xffffffffu, e_ll, off);
            e_qq += __shfl_xor_sync(0xffffffffu, e_qq, off);
        }
        if (lane == 0) {
            red[warp][5] = (double)e_ll;
            red[warp][6] = (double)e_qq;
        }
        __syncthreads();
        if (tid < 5) {
            double tot[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int w = 0; w < NTH / 32; ++w)
                for (int j = 0; j < 7; ++j) tot[j] += red[w][j];
            double m[5];
            for (int i = 0; i < 5; ++i) {
                double acc = 0.0;
                for (int j = 0; j < 5; ++j) acc += a.P[i * 5 + j] * tot[j];
                m[i] = acc;
            }
            mu[tid] = m[tid];
            if (tid == 0) {
                // ||Q_proj||^2 = ||Q||^2 - mu . s (s = the moment sums of Q)
                bool esc = false, last = false;
                if (a.esc_list) {
                    double ms = 0.0;
                    for (int i = 0; i < 5; ++i) ms += m[i] * tot[i];
                    const double qp = tot[6] - ms, k2 = a.inv_kn * a.inv_kn;
                    const double rhs = a.esc_tol2 * (qp > 0.0 ? qp : 0.0);
                    esc = a.esc_c2 * k2 * tot[5] > rhs;
                    last = esc && a.esc_last_list && a.esc_last_c2 * k2 * tot[5] > rhs;
                }
                s_esc = esc ? 1 : 0;
                if (last) a.esc_last_list[atomicAdd(a.esc_last_count, 1)] = (int)cell;
                else if (esc) a.esc_list[atomicAdd(a.esc_count, 1)] = (int)cell;
            }
        }
        __syncthreads();
        fence_after();
        // an escalated cell is left to the next tier
        const bool escalated = s_esc != 0;
        const float m0 = (float)mu[0], m1 = (float)mu[1], m2 = (float)mu[2], m3 = (float)mu[3], m4 = (float)mu[4];
        const bool stepm = a.mode == 1;
        const float dt = (float)a.dt;
        bool bad = false, neg = false;
#pragma unroll 1
        for (int T = 0; T < (escalated ? 0 : TILES); ++T) {
            const int r = 128 * T + 32 * quad + lane, yy = r / N, zz = r % N;
            const int x0 = ZS * cs;
            float gv[ZS];
            TCols<ZS>::load(tlane + C::GCOL + (uint32_t)T * N + x0, gv);
            const float vy = vg[yy], vz = vg[zz];
            const float cyz = m0 + m2 * vy + m3 * vz + 0.5f * m4 * (vy * vy + vz * vz);
            float* dst = a.out + cell * N3 + (long)yy * N + zz;
#pragma unroll
            for (int j = 0; j < ZS; ++j) {
                const int x = x0 + j;
                const float vx = vg[x];
                const float q = gv[j] - (cyz + m1 * vx + 0.5f * m4 * vx * vx);
                const float o = stepm ? fmaf(dt, q, frow(x, yy)[zoff[zz]]) : q;
                bad |= !isfinite(o);
                neg |= stepm && (o < 0.f);
                dst[(long)x * N * N] = o;
            }
        }
        if (bad) atomicOr(a.flags, 1);
        if (neg) atomicOr(a.flags, 2);
        fence_before();
        __syncthreads();   // TMEM gain columns and zoff are reused by the next cell
    }
    // leave no asynchronous work behind
    if (tid == BULK) bulk_wait_all();
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::TCOLS) : "memory");
}

// ---------------------------------------------------------------- host side

// BF16 of a float by round-to-nearest-even of its bit pattern (finite values)
static uint16_t host_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float host_bf16_float(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace tcd

// sizes of the tensor-core path for n (0 if n is not supported)
long tc_scratch_per_cta(int n) {
    if (n == 16) return tcd::Cfg<16>::N3 * 8 + tcd::Cfg<16>::A3_CELL;
    if (n == 32) return tcd::Cfg<32>::N3 * 8 + tcd::Cfg<32>::A3_CELL;
    return 0;
}

// DFT matrices for n: [dir 0 forward (e^-i), 1 inverse (e^+i)][split hi, lo]
// [k-chunk][2n output rows][8 BF16 of input k].  Output row j < n is Re Y_j,
// n + j is Im Y_j; input k < n is Re X_k, n + k is Im X_k.
void tc_dft_matrices(int n, std::vector<uint16_t>& out) {
    const int K = 2 * n, KCH = K / 8;
    out.assign((size_t)4 * KCH * K * 8, 0);
    const double pi = 3.14159265358979323846;
    for (int dir = 0; dir < 2; ++dir) {
        const double sg = dir == 0 ? -1.0 : 1.0;
        for (int row = 0; row < K; ++row)
            for (int k = 0; k < K; ++k) {
                const int j = row % n, l = k % n;
                const double th = sg * 2.0 * pi * (double)((j * l) % n) / n;
                const double c = std::cos(th), s = std::sin(th);
                const bool oim = row >= n, iim = k >= n;
                // Re Y = sum Re X c - Im X s;  Im Y = sum Re X s + Im X c
                const double v = !oim ? (!iim ? c : -s) : (!iim ? s : c);
                const uint16_t hi = tcd::host_bf16((float)v);
                const uint16_t lo = tcd::host_bf16((float)(v - (double)tcd::host_bf16_float(hi)));
                for (int sp = 0; sp < 2; ++sp) {
                    const size_t idx = ((((size_t)(dir * 2 + sp) * KCH + k / 8) * K + row) * 8) + k % 8;
                    out[idx] = sp == 0 ? hi : lo;
                }
            }
    }
}

template <int N>
static cudaError_t launch_n(const tcd::Args& a, int grid, cudaStream_t s) {
    using C = tcd::Cfg<N>;
    auto k = tcd::collide_tc_kernel<N>;
    // one CTA per SM: the kernel holds TCOLS tensor-memory columns for its lifetime
    const int smem = C::SMEM > 117 * 1024 ? (int)C::SMEM : 117 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, tcd::NTH, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_collide_tc(int n, const TcLaunch& l, cudaStream_t s) {
    tcd::Args a;
    a.f = static_cast<const float*>(l.f);
    a.out = static_cast<float*>(l.out);
    a.tab = static_cast<const float2*>(l.tables);
    a.dft = static_cast<const uint4*>(l.dft);
    a.fh = static_cast<float2*>(l.scratch);
    a.a3 = static_cast<unsigned char*>(l.scratch) + (long)l.grid * n * n * n * 8;
    a.delta = l.delta;
    a.flags = l.flags;
    a.ncells = l.ncells;
    a.cells = l.cells;
    a.cells_count = l.cells_count;
    a.esc_list = l.esc_list;
    a.esc_count = l.esc_count;
    a.esc_c2 = l.esc_c2;
    a.esc_tol2 = l.esc_tol2;
    a.esc_last_list = l.esc_last_list;
    a.esc_last_count = l.esc_last_count;
    a.esc_last_c2 = l.esc_last_c2;
    for (int i = 0; i < 3; ++i) {
        a.nc[i] = l.nc[i];
        a.bc[i] = l.bc[i];
    }
    a.M = l.M;
    a.L = l.L;
    a.inv_kn = l.inv_kn;
    a.dt = l.dt;
    a.mode = l.mode;
    std::memcpy(a.P, l.P, sizeof(a.P));
    const int grid = (int)(l.ncells < l.grid ? l.ncells : l.grid);
    if (n == 16) return launch_n<16>(a, grid, s);
    if (n == 32) return launch_n<32>(a, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace fks
