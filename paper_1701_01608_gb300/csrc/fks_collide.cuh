// fks_collide.cuh -- per-cell fast spectral collision operator (Appendix A of
// arXiv 1701.01608) with the FKS transport gather and the explicit Euler step
// (Eq. disc_relax) fused around it.
//
// One cell is processed by one thread-block cluster of C CTAs.  The
// half-spectrum f^ (kz' = 0..N/2) is distributed over the cluster by ky slab;
// each inverse transform runs x-pass (local) -> DSMEM exchange -> y-pass ->
// z-pass (C2R, local), so the whole per-cell working set stays on chip and f^
// is read from shared memory 2M+1 times instead of from HBM.
//
// Per cell:
//   f*  = gather of f over the transport shifts delta_k (identity for collide)
//   F   = DFT(f*)                                   forward R2C, 3 passes
//   for p < M:  a = IDFT(alpha_p F) / N^3,  b = IDFT(w_p alphap_p F) / N^3,
//               G += a b                            (gain, Appendix A)
//   l   = IDFT(betaL F) / N^3,  L = f* l             (loss: the B_F(m,m) term)
//   Q   = (G - L) / Kn                               (G - f* l by one FMA: one rounding)
//   Q  -= C^T (C C^T)^-1 C Q                         (conservation projection: moment sums in FP64,
//                                                     or in compensated FP32 pairs for FP32 data;
//                                                     the coefficients in FP64)
//   out = Q, f* + dt Q, or the second Heun stage (base + f* + dt Q) / 2
//
// Inverse-pass packing: the kz' = 0 and kz' = N/2 planes of a real field are
// each 2-D Hermitian, so they travel together as one complex plane
// (plane 0 = P_0 + i P_{N/2}); every pass then has exactly N/2 planes.
//
// Plane layouts: f^, the table slab and the exchange buffer W store the planes
// of one (kx or x, ky) row contiguously with an odd stride (N/2+1), and the
// x-pass tasks are assigned to lanes so that the lanes of one shared-memory
// phase hit distinct banks (see xpass_task_map).
//
// Exchange between the x and y passes: each CTA writes its x-pass output for
// itself into W[own block] and for every peer into a local staging block; one
// thread per peer then moves that peer's staged block with a bulk copy (TMA,
// shared::cta -> shared::cluster) that completes on the receiving CTA's
// mbarrier (issued by one thread in sequence they cost 5 % of the kernel).
// The double-float instantiations (pencils split over lane pairs) store their
// x-pass outputs straight into block `rank` of every owner's W instead, with W
// double-buffered by direction parity, so one cluster barrier per direction
// orders both the stores and the reuse of the buffer (no staging, no copies).
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <type_traits>

#include "fks_df.cuh"
#include "fks_dfloat.cuh"
#include "fks_fft.cuh"

namespace cg = cooperative_groups;

namespace fks {

// One independent space-homogeneous problem of a batch (one cell, no transport).
struct BatchItem {
    const void* f;          // n^3 input values
    void* out;              // n^3 output values
    const void* tables;     // this problem's table slabs (kernel type, L)
    const double* P;        // 25 projection coefficients for (n, L)
    double inv_kn;
    double dt;
    double L;
    double pad_;
};

struct CollideArgs {
    const void* f;          // input distribution, ncells * N^3 (element type T)
    void* out;              // Q or f^{n+1}
    const void* tables;     // [M+1][C] slabs: [2][N kx][NS kyl][H-1] planes 1..H-1, then [2][N][NS][2] planes 0, H
    const signed char* delta;  // [3][N] cell shifts for this step (transport) or nullptr
    int* flags;             // health bits (atomicOr)
    long ncells;            // end (exclusive) of the cells (items) this launch processes
    long cell0;             // first cell of this launch (0 in batch mode)
    int nc[3];              // spatial cells per axis
    int bc[3];              // 0 periodic, 1 specular
    int M;                  // number of directions
    double L;               // velocity box half width
    double inv_kn;
    double dt;              // Euler step (step mode)
    int mode;               // 0 collide (out = Q), 1 step (out = f* + dt Q), 2 collide without projection,
                            // 3 second Heun stage (out = (base + f* + dt Q) / 2; no transport, not batch),
                            // 4 exponential step: out = f* + dt P[phi(nu dt) (G - nu f*)], nu = l / Kn the
                            //   loss frequency, phi(x) = (1 - e^-x) / x, P the projection
    double P[25];           // dv^6 (C C^T)^-1 over the rows phi = (1, v, |v|^2/2)
    const BatchItem* items; // batch mode: ncells items, each a homogeneous problem
    const void* base;       // mode 3: the first stage's input, same layout as out (may be out itself)
    // list mode: the cells (batch: items) processed are list[cell0 .. *list_count) instead of cell0 .. ncells
    const int* list;
    const int* list_count;
    // precision escalation: a cell whose error bound esc_c * ||L|| / Kn exceeds esc_tol * ||Q|| (Q
    // projected) is appended to esc_list (count esc_count) and not written; nullptr: every cell is written
    int* esc_list;
    int* esc_count;
    double esc_c2;          // esc_c^2
    double esc_tol2;        // esc_tol^2
};

// Error constants of the escalation bound ||dQ|| <= c ||L|| / Kn (L = f* l, the loss term): the
// transforms' rounding in each arithmetic measured against the FP64 operator, with a margin
// (FP32 ~2.4e-7, split BF16 ~5e-6 of ||L|| on near-equilibrium and two-stream cells).
constexpr double kEscFp32 = 5e-7;
constexpr double kEscBf16 = 1.5e-5;
// Near equilibrium, d = ||f - M|| / ||M|| (M the Maxwellian of f's moments): Q ~ L_M (f - M) + Q(M), so
// ||Q|| <~ d ||L|| / k_d + ||Q(M)|| with ||L_M h|| of the order of the loss frequency times ||h|| (k_d
// of order one: 0.75 .. 2.6 measured over shock-tube cells and perturbations of several shapes) and the
// operator's residual Q(M) below 1e-5 ||L|| (||L|| / ||Q|| > 1e5 at exact discrete Maxwellians).  With
// k_d taken as kKappaDist (a margin of 7 or more) a cell with d < kKappaDist c / tol fails the bound
// c ||L|| / Kn <= tol ||Q|| of a tier with constant c.
constexpr double kKappaDist = 0.1;

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
// arrive without release: only orders this CTA's earlier reads (whose values
// are already consumed) before peers overwrite the buffer they read
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    cluster_arrive();
    cluster_wait();
}

// 32-bit shared-window addresses and stores into a peer CTA's shared memory
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, cpx<float> v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, cpx<double> v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};\n" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, cpx<dfloat> v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(v.x.hi), "f"(v.x.lo),
                 "f"(v.y.hi), "f"(v.y.lo)
                 : "memory");
}

// mbarrier and bulk-copy (TMA) helpers for the per-direction table slab
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: a bulk copy of valid memory always completes; if it has not
// after `polls` polls (default ~2^26) the kernel records FKS timeout (bit 3)
// and goes on.  Returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* flags, long polls = 1L << 26) {
    for (long it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(flags, 8);
    return false;
}

// bulk prefetch of a global range into L2 (16-byte aligned address, size a multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// double-float helpers (df_add1, df_add, df_mul) for the compensated FP32 sums: fks_df.cuh
__device__ __forceinline__ float2 df_shfl_xor(float2 v, int off) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
}

// ---- transforms split over G = 2 or 4 consecutive lanes of a warp -------------------------
// The double-float instantiations split every length-N transform of a pencil over G threads: 1/G of
// the registers and about 1/G of the transform code per thread and G times the warps per SM (with
// one thread per pencil the double-float kernel is bound by instruction fetch, one warp per
// scheduler).
__device__ __forceinline__ float lane_xchg(float v, unsigned mask, int d) { return __shfl_xor_sync(mask, v, d); }
__device__ __forceinline__ double lane_xchg(double v, unsigned mask, int d) { return __shfl_xor_sync(mask, v, d); }
__device__ __forceinline__ dfloat lane_xchg(dfloat v, unsigned mask, int d) {
    return dfloat(lane_xchg(v.hi, mask, d), lane_xchg(v.lo, mask, d));
}
template <typename T>
__device__ __forceinline__ cpx<T> lane_xchg(cpx<T> v, unsigned mask, int d) {
    return {lane_xchg(v.x, mask, d), lane_xchg(v.y, mask, d)};
}

// element index held in local slot m after fft_split by thread g = sum_b g_b 2^b of G: G = 1, m
// itself; otherwise the outputs k and k + N/2 of the last radix-2 combination, with
// k = (m mod N/2G) + (N/2G) (g_{r-1} + 2 g_{r-2} + ... + 2^{r-1} g_0), G = 2^r (bit-reversed part)
template <int N, int G>
__device__ __forceinline__ int split_out(int m, int g) {
    if constexpr (G == 1) {
        return m;
    } else {
        constexpr int Q = N / (2 * G);
        int rev = 0;
#pragma unroll
        for (int b = 1; b < G; b <<= 1) rev = (rev << 1) | ((g & b) ? 1 : 0);
        return m % Q + rev * Q + (m / Q) * (N / 2);
    }
}

namespace detail {
// output pair k = kb(M) of the last radix-2 combination X_k = E_k + W^k O_k, X_{k+N/2} = E_k - W^k O_k
// (W = exp(SIGN 2 pi i / N); E, O the half-length transforms of the even and odd samples): the
// lane with bit D clear holds E, its partner (lane ^ D) holds O at the same indices; each keeps one
// half of the M slots and sends the partner the other half.  Slot M < L/2 of the E lane and slot
// M + L/2 of the O lane combine; the index of slot M is M + base, base = Q (bit-reversed higher part)
// with the O lane's extra N/4 (W^{N/4} = SIGN i) and the higher parts' extra N/8 (an eighth turn).
template <typename T, int SIGN, int N, int L, int M>
__device__ __forceinline__ void split_combine(cpx<T> (&a)[L], bool odd, bool eighth, unsigned mask, int d) {
    constexpr int H2 = L / 2;
    const cpx<T> recv = lane_xchg(odd ? a[M] : a[M + H2], mask, d);
    const cpx<T> u = odd ? recv : a[M];
    cpx<T> v = mul_tw<T, SIGN, M, N>(odd ? a[M + H2] : recv);
    if constexpr (N % 8 == 0 && L * 2 < N) {
        const cpx<T> ve = mul_tw<T, SIGN, N / 8, N>(v);   // the part's eighth turn (G = 4)
        v = eighth ? ve : v;
    }
    const cpx<T> vq = mul_si<T, SIGN>(v);   // W^{N/4} = SIGN i for the odd lane's slots
    v = odd ? vq : v;
    a[M] = cadd(u, v);
    a[M + H2] = csub(u, v);
}
template <typename T, int SIGN, int N, int L, int... M>
__device__ __forceinline__ void split_combine_all(cpx<T> (&a)[L], bool odd, bool eighth, unsigned mask, int d,
                                                  std::integer_sequence<int, M...>) {
    (split_combine<T, SIGN, N, L, M>(a, odd, eighth, mask, d), ...);
}
}  // namespace detail

// fft<N, SIGN> of a pencil spread over G consecutive lanes: thread g holds a[j] = x_{jG+g} (j < N/G)
// and ends with a[m] = X_{split_out<N, G>(m, g)}; mask names the pencil's lanes (they call it
// together).  G = 2: both halves transform their samples (decimation in time) and combine; G = 4:
// the even lanes (bit 0 clear) transform the even samples as a 2-lane split over lane bit 1, the odd
// lanes the odd samples, then one combination across lane bit 0.
template <int N, int SIGN, int G, int R0, typename T>
__device__ __forceinline__ void fft_split(cpx<T> (&a)[N / G], int g, unsigned mask) {
    if constexpr (G == 1) {
        fft<N, SIGN, R0>(a);
    } else if constexpr (G == 2) {
        static_assert(N % 4 == 0, "a pencil split over two lanes");
        fft<N / 2, SIGN>(a);
        detail::split_combine_all<T, SIGN, N, N / 2>(a, g != 0, false, mask, 1,
                                                      std::make_integer_sequence<int, N / 4>{});
    } else {
        static_assert(G == 4 && N % 8 == 0, "a pencil split over two or four lanes");
        // half-length transform of this lane's parity class over lane bit 1 (partner lane ^ 2)
        fft<N / 4, SIGN>(a);
        detail::split_combine_all<T, SIGN, N / 2, N / 4>(a, (g & 2) != 0, false, mask, 2,
                                                          std::make_integer_sequence<int, N / 8>{});
        // across lane bit 0 (partner lane ^ 1): slot indices k = M + (N/8) g1 (+ N/4 for the odd lane)
        detail::split_combine_all<T, SIGN, N, N / 4>(a, (g & 1) != 0, (g & 2) != 0, mask, 1,
                                                      std::make_integer_sequence<int, N / 8>{});
    }
}

// cell index -> (cx, cy, cz) in 32-bit unsigned arithmetic (a context holds fewer
// than 2^31 cells; 64-bit division is a long emulated sequence, run by every thread)
__device__ __forceinline__ void cell_coords(long cell, int ncy, int ncz, int& cx, int& cy, int& cz) {
    const unsigned c = (unsigned)cell, nyz = (unsigned)ncy * (unsigned)ncz;
    const unsigned r = c % nyz;
    cx = (int)(c / nyz);
    cy = (int)(r / (unsigned)ncz);
    cz = (int)(r % (unsigned)ncz);
}

// fold a source cell coordinate: periodic wrap or specular reflection
__device__ __forceinline__ int fold_cell(int u, int len, int specular, int& flip) {
    if (!specular) {
        int r = u % len;
        if (r < 0) r += len;
        flip = 0;
        return r;
    }
    int per = 2 * len;
    int r = u % per;
    if (r < 0) r += per;
    if (r >= len) { flip = 1; return per - 1 - r; }
    flip = 0;
    return r;
}

// Padding (in cpx elements) between the W source blocks: the z-pass lanes of a
// shared-memory phase read column y = src*NS + kyl at
// src*(BLK+pad) + kyl*(H-1) (+ k); pick the pad (a multiple of 16 bytes) that
// minimises the worst bank multiplicity of one phase.
template <int ESZ>   // bytes per complex element (8 or 16)
constexpr int best_block_pad(int N, int NS, int HM, long BLK) {
    const int lanes = ESZ == 8 ? 16 : 8;          // lanes per shared-memory phase
    const int words = ESZ / 4;
    const int step = ESZ == 8 ? 2 : 1;            // pads keep 16-byte alignment
    int best_pad = 0, best_m = 1 << 30;
    for (int pad = 0; pad < 32; pad += step) {
        int worst = 0;
        for (int ph = 0; ph + lanes <= N; ph += lanes) {
            int cnt[32] = {};
            for (int l = 0; l < lanes; ++l) {
                const int y = ph + l;
                const long e = (long)(y / NS) * (BLK + pad) + (long)(y % NS) * HM;
                for (int w = 0; w < words; ++w) ++cnt[(int)((e * words + w) % 32)];
            }
            for (int b = 0; b < 32; ++b) worst = cnt[b] > worst ? cnt[b] : worst;
        }
        if (worst < best_m) { best_m = worst; best_pad = pad; }
    }
    return best_pad;
}

template <typename T, int N, int C>
struct CollideCfg {
    static constexpr int NS = N / C;          // slab width (ky for f^, x for W)
    static constexpr int H = N / 2;           // packed planes per inverse transform
    static constexpr int HF = H + 1;          // kz' planes of f^ (odd row stride)
    static constexpr int HP = H + 1;          // row stride of W (odd)
    static constexpr int NTASK = N * N / C;   // pencils / columns per pass per CTA
    // threads per pencil: double-float transforms are split over consecutive lanes (fft_split)
    static constexpr int G = std::is_same<T, dfloat>::value ? 2 : 1;
    static constexpr int NE = N / G;          // pencil elements per thread
    static constexpr int NT = (NTASK * G + 31) / 32 * 32;   // threads per CTA (whole warps)
    static constexpr bool G_REG = sizeof(T) == 4;       // FP32: gain accumulator in registers
    static constexpr long FH_ELEMS = (long)N * NS * HF;  // f^ slab [N kx][NS kyl][HF]
    // W: C source blocks, each [2 tab][NS xl][NS kyl][HP]   (cpx<T>)
    static constexpr long BLK = 2L * NS * NS * HP;
    static constexpr long BLK_STRIDE = BLK + best_block_pad<(int)sizeof(cpx<T>)>(N, NS, HP, BLK);
    // split pencils (double-float): the x-pass stores its outputs straight into the owner CTAs' W (DSMEM),
    // W double-buffered by direction parity, one cluster barrier per direction, no staging blocks;
    // otherwise W single, the peers' blocks staged in S and moved by bulk copies
    static constexpr bool XDIRECT = G > 1;
    static constexpr long W_ONE = (long)C * BLK_STRIDE;                 // one W buffer
    static constexpr long W_ELEMS = (XDIRECT ? 2 : 1) * W_ONE;
    static constexpr long S_ELEMS = XDIRECT ? 0 : (long)(C - 1) * BLK_STRIDE;   // staging for the peers' blocks
    static constexpr unsigned BLK_BYTES = (unsigned)(sizeof(cpx<T>) * BLK);
    // forward-transform staging [NS xl][N y][HF] reuses W
    static constexpr long STG_ELEMS = (long)NS * N * HF;
    // table slab of one direction: [2 tab][N kx][NS kyl][HF]   (T)
    static constexpr long TAB_ELEMS = 2L * N * NS * HF;
    static constexpr unsigned TAB_BYTES = (unsigned)(sizeof(T) * TAB_ELEMS);
    // gain accumulator [N z][GSTR] (FP64, double-float): split pencils pad the row by one element so
    // that the lanes of a pencil, N/(2G) rows apart, fall on different banks
    static constexpr int GSTR = NTASK + (G > 1 ? 1 : 0);
    static constexpr long G_ELEMS = G_REG ? 0 : (long)GSTR * N;
    static constexpr size_t SMEM_BASE = sizeof(cpx<T>) * (FH_ELEMS + W_ELEMS + S_ELEMS) + sizeof(T) * G_ELEMS +
                                        sizeof(double) * (8 + (NT / 32) * 7 + 8 + 2 * N) + sizeof(float) * (4 * N + 8) +
                                        sizeof(T) * N + sizeof(long) * N + 2 * sizeof(uint64_t) + 3 * N + 4 * NT + 64;
    // the table slab is staged in shared memory (bulk-copy prefetch) when it fits
    static constexpr bool TAB_SMEM = SMEM_BASE + sizeof(T) * TAB_ELEMS <= 227u * 1024u;
    static constexpr long TB_ELEMS = TAB_SMEM ? TAB_ELEMS : 0;
    static constexpr size_t SMEM_BYTES = sizeof(cpx<T>) * (FH_ELEMS + W_ELEMS + S_ELEMS) +
                                         sizeof(T) * (TB_ELEMS + G_ELEMS) +
                                         sizeof(double) * (8 + (NT / 32) * 7 + 8 + 2 * N) +
                                         sizeof(float) * (4 * N + 8) + sizeof(T) * N + sizeof(long) * N +
                                         2 * sizeof(uint64_t) + 3 * N + 4 * NT + 64;
    static_assert(N % C == 0, "cluster size must divide N");
    static_assert(G == 1 || NTASK % 8 == 0, "split pencils permute their tasks in groups of 8");
    static_assert(TAB_BYTES % 16 == 0 && BLK_BYTES % 16 == 0, "bulk copies move whole 16-byte units");
    static_assert(STG_ELEMS <= W_ONE, "forward staging fits in W");
};

// Lane assignment of the x-pass tasks (tab, kyl, plane).  Tasks of the packed
// plane 0 take the first 2*NS lanes (their longer code path diverges in the
// first warp only).  The others are placed group by group (a group = the
// lanes of one shared-memory phase, 16 for 8-byte and 8 for 16-byte elements)
// so that (kyl + plane) differs modulo the group size inside a group: the
// row stride of f^, W and the tables is odd, so their addresses then fall on
// distinct banks.  Written by one thread into map[NT] as tab<<16|kyl<<8|plane.
template <int N, int C, int ESZ>
__device__ void xpass_task_map(unsigned* map, unsigned char* used) {
    constexpr int NS = N / C, H = N / 2, NTASK = N * N / C;
    constexpr int G = ESZ == 8 ? 16 : 8;
    constexpr int NTK = 2 * NS * (H - 1);           // non-packed tasks
    for (int i = 0; i < NTK; ++i) used[i] = 0;
    for (int t = 0; t < 2 * NS; ++t) map[t] = ((unsigned)(t / NS) << 16) | ((unsigned)(t % NS) << 8);
    int slot = 2 * NS;
    while (slot < NTASK) {
        const int gend = (slot / G + 1) * G < NTASK ? (slot / G + 1) * G : NTASK;
        bool taken[G] = {};
        // residues already used by packed tasks sharing this group
        for (int s = (slot / G) * G; s < slot; ++s) taken[(((map[s] >> 8) & 255u) + (map[s] & 255u)) % G] = true;
        for (int pass = 0; pass < 2 && slot < gend; ++pass) {
            for (int i = 0; i < NTK && slot < gend; ++i) {
                if (used[i]) continue;
                const int tab = i / (NS * (H - 1));
                const int kyl = (i / (H - 1)) % NS;
                const int pp = 1 + i % (H - 1);
                const int res = (kyl + pp) % G;
                if (pass == 0 && taken[res]) continue;   // second pass: fill what is left
                taken[res] = true;
                used[i] = 1;
                map[slot++] = ((unsigned)tab << 16) | ((unsigned)kyl << 8) | (unsigned)pp;
            }
        }
    }
}

// phi(x) = (1 - e^-x) / x of the exponential step for x > 0, 1 otherwise (the explicit update where
// the discrete loss frequency is not positive).  Not inlined: the unrolled epilogue calls it per
// element and an inlined copy of expm1 per call site makes the kernels large.
static __device__ __noinline__ float exp_step_factor(float x) { return x > 0.0f ? -expm1f(-x) / x : 1.0f; }
static __device__ __noinline__ double exp_step_factor(double x) { return x > 0.0 ? -expm1(-x) / x : 1.0; }

// T: arithmetic of the transforms (float, double, or dfloat: double-float pairs on the FP32 pipes);
// ST: element type of f, out and base in global memory (ST = float with T = double or dfloat: the
// last escalation tier of an FP32 state)
// R0: top radix of the length-N transforms (0: the default schedule; see fft in fks_fft.cuh)
template <typename T, int N, int C, bool BATCH = false, typename ST = T, int R0 = 0>
__global__ void __launch_bounds__(CollideCfg<T, N, C>::NT, 1)
collide_kernel(CollideArgs args) {
    using Cfg = CollideCfg<T, N, C>;
    constexpr int NS = Cfg::NS, H = Cfg::H, HF = Cfg::HF, HP = Cfg::HP, NT = Cfg::NT, NTASK = Cfg::NTASK;
    constexpr long N3 = (long)N * N * N;
    constexpr long BLK = Cfg::BLK_STRIDE;   // block stride in W (padded)

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const long cluster_id = blockIdx.x / C;
    const long nclusters = gridDim.x / C;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<T>* Fh = reinterpret_cast<cpx<T>*>(smem_raw);                 // f^ slab [N kx][NS kyl][HF]
    cpx<T>* W = Fh + Cfg::FH_ELEMS;                                    // [C src][block]
    cpx<T>* S = W + Cfg::W_ELEMS;                                      // [C-1][block] staging
    T* Tb = reinterpret_cast<T*>(S + Cfg::S_ELEMS);                   // table slab
    T* Gs = Tb + Cfg::TB_ELEMS;                                        // FP64 gain [N z][GSTR]
    double* red = reinterpret_cast<double*>(Gs + Cfg::G_ELEMS);       // [8] own partials
    double* redw = red + 8;                                            // [NT/32][7]
    double* mu = redw + (NT / 32) * 7;                                 // [8] correction coefficients, [7] escalation
    double* vzt = mu + 8;                                              // [N] v_z
    double* vz2t = vzt + N;                                            // [N] v_z^2 / 2
    float* vzf = reinterpret_cast<float*>(vz2t + N);                  // [4][N] v_z, v_z^2/2 as FP32 (hi, lo)
    float* muf = vzf + 4 * N;                                          // [8] mu in FP32
    T* czt = reinterpret_cast<T*>(muf + 8);                           // [N] projection correction along z
    long* zoff = reinterpret_cast<long*>(czt + N + (N & 1));          // [N] gather offsets along z
    uint64_t* tbar = reinterpret_cast<uint64_t*>(zoff + N);           // table-slab mbarrier
    uint64_t* xbar = tbar + 1;                                         // exchange mbarrier
    unsigned* xmap = reinterpret_cast<unsigned*>(xbar + 1);           // [NT] x-pass task map
    signed char* dsm = reinterpret_cast<signed char*>(xmap + NT);     // [3][N] shifts

    // shared::cluster addresses of Fh (forward exchange) in every CTA
    uint32_t Frank[C];
#pragma unroll
    for (int r = 0; r < C; ++r) Frank[r] = map_rank(smem_addr(Fh), r);
    // store v at element idx of the f^ slab of CTA dst
    auto putF = [&](int dst, long idx, cpx<T> v) {
        if constexpr (C == 1) Fh[idx] = v;
        else if constexpr (Cfg::G == 1) st_cluster(Frank[dst] + (uint32_t)(idx * (long)sizeof(cpx<T>)), v);
        else st_cluster(map_rank(smem_addr(Fh), dst) + (uint32_t)(idx * (long)sizeof(cpx<T>)), v);   // dst per lane
    };

    // per-item data: the cells of one problem, or (batch) one problem per item
    auto item_tables = [&](long it) -> const T* {
        if constexpr (BATCH) return static_cast<const T*>(args.items[it].tables);
        else return static_cast<const T*>(args.tables);
    };
    const bool transport = !BATCH && args.delta != nullptr;
    for (int i = tid; i < 3 * N; i += NT) dsm[i] = transport ? args.delta[i] : 0;
    double dv = 2.0 * args.L / N;
    // velocity of grid index i: (i + 1/2 - N/2) dv
    auto vel = [&dv](int i) { return ((double)i + 0.5 - 0.5 * N) * dv; };
    // v_z and v_z^2/2 as FP32 pairs hi + lo (the compensated FP32 moment sums)
    auto set_vel = [&](int i) {
        vzt[i] = vel(i);
        vz2t[i] = 0.5 * vel(i) * vel(i);
        const float h1 = (float)vzt[i], h2 = (float)vz2t[i];
        vzf[i] = h1;
        vzf[N + i] = (float)(vzt[i] - (double)h1);
        vzf[2 * N + i] = h2;
        vzf[3 * N + i] = (float)(vz2t[i] - (double)h2);
    };
    for (int i = tid; i < N; i += NT) set_vel(i);
    if (tid == 0) {
        mbar_init(tbar, 1);
        mbar_init(xbar, 1);
        fence_mbar_init();
        // scratch for the task-map construction: the (not yet used) W buffer
        xpass_task_map<N, C, (int)sizeof(cpx<T>)>(xmap, reinterpret_cast<unsigned char*>(W));
    }
    // every CTA of the cluster is running before any distributed-shared access
    cluster_sync_all();
    unsigned tphase = 0, xphase = 0;
    // after a wait has run out (bit 3 recorded), this thread's further waits poll once: the launch
    // then finishes its cells quickly; every CTA of a cluster keeps the same barrier sequence, so
    // none leaves while a peer may still address its shared memory
    bool tmo = false;
    // table slab of direction p (p = M: loss) for this CTA, fetched by one thread
    auto fetch_tables = [&](const T* tab, int p) {
        if (Cfg::TAB_SMEM && tid == 0) {
            mbar_expect_tx(tbar, Cfg::TAB_BYTES);
            bulk_g2s(Tb, tab + ((long)p * C + rank) * Cfg::TAB_ELEMS, Cfg::TAB_BYTES, tbar);
        }
    };
    // list mode: the count was written by an earlier launch on the stream
    const long end = args.list ? (long)*args.list_count : args.ncells;
    auto item_at = [&](long it) -> long { return args.list ? (long)args.list[it] : it; };
    if (args.cell0 + cluster_id < end) fetch_tables(item_tables(item_at(args.cell0 + cluster_id)), 0);
    const int ncx = args.nc[0], ncy = args.nc[1], ncz = args.nc[2];

    // the double-float instantiations (instruction-fetch bound: every inlined transform is long) share
    // one call site of each transform between the passes of a direction
    constexpr bool kCompact = std::is_same<T, dfloat>::value;

    // pencil task of this thread and its part g of the pencil (G threads per pencil: lanes
    // Gt .. Gt + G - 1; element j of a pencil is loaded by part j mod G, outputs are at split_out)
    constexpr int G = Cfg::G, NE = Cfg::NE;
    const int task = G == 1 ? tid : tid / G;
    const int g = G == 1 ? 0 : tid % G;
    const unsigned pmask = G == 1 ? 0xffffffffu : ((1u << G) - 1u) << (tid & (32 - G));   // the pencil's lanes
    auto zz = [g](int m) { return split_out<N, G>(m, g); };   // element of output slot m

    // split pencils: the y- and z-pass tasks are permuted within groups of 8 (even members first), so
    // that the four pencils of a shared-memory phase take every other plane (column) and the pair's
    // lanes, one element apart, fall on different banks
    auto perm8 = [](int t) { const int q = t & 7; return (t & ~7) | (q < 4 ? 2 * q : 2 * q - 7); };
    const int ztask = G == 2 ? perm8(task) : task;
    constexpr int GSTR = Cfg::GSTR;

    // z-pass ownership: column (xl, y), x = rank*NS + xl (tasks >= NTASK idle)
    const bool has_col = task < NTASK;
    const int zl_x = has_col ? ztask / N : 0, zl_y = ztask % N;
    const int zx = rank * NS + zl_x;
    const int z_src = zl_y / NS, z_kyl = zl_y % NS;   // where column y sits in W
    T* Gcol = Gs + task;   // FP64: element z at Gcol[z * GSTR]

    // y-pass task (tab, xl, plane), plane fastest
    const int t_tab = ztask / (NS * H);
    const int t_rem = ztask % (NS * H);
    const int t_xl = t_rem / H;
    const int t_pp = t_rem % H;
    // x-pass task (tab, kyl, plane) from the lane map (built before the first cluster barrier)
    const unsigned xm = task < NTASK ? xmap[task] : 0u;
    const int x_tab = task < NTASK ? (int)(xm >> 16) : 2;
    const int x_kyl = (int)((xm >> 8) & 255u);
    const int x_pp = (int)(xm & 255u);
    // offset of (tab, xl, kyl, plane) inside a W block
    auto widx = [](int tb, int xl, int kyl, int pp) -> long { return (((long)tb * NS + xl) * NS + kyl) * HP + pp; };
    // y-pass lane addressing: element (src, kyl) at ybase + src*BLK + kyl*HP
    const long ybase = widx(t_tab, t_xl, 0, t_pp);

    for (long it = args.cell0 + cluster_id; it < end; it += nclusters) {
        const long item = item_at(it);
        const bool has_next = it + nclusters < end;
        // batch: item = one homogeneous problem (cell 0 of its own arrays)
        const long cell = BATCH ? 0 : item;
        if constexpr (!BATCH) {
            // the x-planes of this cluster's next cell towards L2 while this one is processed
            // (its forward pass then starts on L2 hits; with transport most sources are the cell itself)
            if (tid == 0 && has_next)
                prefetch_l2(static_cast<const ST*>(args.f) + item_at(it + nclusters) * N3 + (long)rank * NS * N * N,
                            (unsigned)(sizeof(ST) * NS * N * N));
        }
        const ST* __restrict__ fin;
        ST* __restrict__ fout;
        const T* __restrict__ tab = item_tables(item);
        const double* Pm;
        double inv_kn, dt_step;
        if constexpr (BATCH) {
            const BatchItem& bi = args.items[item];
            fin = static_cast<const ST*>(bi.f);
            fout = static_cast<ST*>(bi.out);
            Pm = bi.P;
            inv_kn = bi.inv_kn;
            dt_step = bi.dt;
            // velocity tables of this problem's box (read after the barrier below;
            // the previous item's last reads precede its final cluster barrier)
            dv = 2.0 * bi.L / N;
            if (tid < N) set_vel(tid);
        } else {
            fin = static_cast<const ST*>(args.f);
            fout = static_cast<ST*>(args.out);
            Pm = args.P;
            inv_kn = args.inv_kn;
            dt_step = args.dt;
        }
        int cx, cy, cz;
        cell_coords(cell, ncy, ncz, cx, cy, cz);
        // gather offsets along z for this cell (relative to the (x, y) source row)
        if (tid < N) {
            if (!transport) {
                zoff[tid] = cell * N3 + tid;
            } else {
                int fz;
                const int sz = fold_cell(cz - dsm[2 * N + tid], ncz, args.bc[2], fz);
                zoff[tid] = (long)sz * N3 + (fz ? N - 1 - tid : tid);
            }
        }
        __syncthreads();
        // base of the f* column (x, y, :) of the transported cell
        const ST* colbase;
        if (!transport) {
            colbase = fin + ((long)zx * N + zl_y) * N;
        } else {
            int fx, fy;
            const int sx = fold_cell(cx - dsm[zx], ncx, args.bc[0], fx);
            const int sy = fold_cell(cy - dsm[N + zl_y], ncy, args.bc[1], fy);
            const int qx = fx ? N - 1 - zx : zx;
            const int qy = fy ? N - 1 - zl_y : zl_y;
            colbase = fin + ((long)sx * ncy + sy) * ncz * N3 + ((long)qx * N + qy) * N;
        }

        // ---------------- forward transform -----------------------------
        // F1: z-R2C of this CTA's columns; staging = W as [xl][y][HF]
        if (has_col) {
            cpx<T> a[NE];
#pragma unroll
            for (int j = 0; j < NE; ++j) a[j] = {T(colbase[zoff[j * G + g]]), T(0)};
            fft_split<N, -1, G, R0>(a, g, pmask);
            cpx<T>* stg = W + ((long)zl_x * N + zl_y) * HF;
#pragma unroll
            for (int m = 0; m < NE; ++m) {
                const int k = zz(m);
                if (G == 1 ? m < HF : k < HF) stg[k] = a[m];
            }
            if constexpr (!Cfg::G_REG) {
#pragma unroll
                for (int m = 0; m < NE; ++m) Gcol[(long)zz(m) * GSTR] = T(0);
            }
        }
        T Greg[Cfg::G_REG ? N : 1];
        if constexpr (Cfg::G_REG) {
#pragma unroll
            for (int z = 0; z < N; ++z) Greg[z] = T(0);
        }
        __syncthreads();
        // F2 + F3: y-FFT of (xl, kz') pencils, scatter to the ky owner (pre-x-FFT, x in place of kx)
        if (task < NS * HF) {
            const int xl = task / HF, kz = task % HF;
            cpx<T> a[NE];
#pragma unroll
            for (int j = 0; j < NE; ++j) a[j] = W[((long)xl * N + (j * G + g)) * HF + kz];
            fft_split<N, -1, G, R0>(a, g, pmask);
            const int x = rank * NS + xl;
#pragma unroll
            for (int m = 0; m < NE; ++m) {
                const int ky = zz(m);
                putF(ky / NS, ((long)x * NS + ky % NS) * HF + kz, a[m]);
            }
        }
        cluster_sync_all();
        // F4: x-FFT of (kyl, kz') pencils in place
        if (task < NS * HF) {
            const int kyl = task / HF, kz = task % HF;
            cpx<T> a[NE];
#pragma unroll
            for (int j = 0; j < NE; ++j) a[j] = Fh[((long)(j * G + g) * NS + kyl) * HF + kz];
            fft_split<N, -1, G, R0>(a, g, pmask);
#pragma unroll
            for (int m = 0; m < NE; ++m) Fh[((long)zz(m) * NS + kyl) * HF + kz] = a[m];
        }
        __syncthreads();

        // ---------------- gain and loss ---------------------------------
        // staged exchange: matches the wait before the first x-pass exchange (W staging reads done); the
        // direct stores need none (the forward transform's cluster barrier freed W)
        if constexpr (!Cfg::XDIRECT) cluster_arrive();
        for (int p = 0; p <= args.M; ++p) {
            const bool loss = (p == args.M);
            // this direction's W (direct stores: the buffer of its parity, last read by direction p - 2)
            cpx<T>* const Wp = W + (Cfg::XDIRECT ? (long)(p & 1) * Cfg::W_ONE : 0L);
            // ---- x-pass: table product, pack kz'=0 with kz'=N/2, inverse FFT along kx
            const bool active = has_col && (!loss || x_tab == 0);
            const bool active_y = has_col && (!loss || t_tab == 0);
            // the exchange after the x-pass stores (the same steps as the inline sequence below)
            auto exchange = [&]() {
                if constexpr (C > 1) {
                    if (tid == 0) mbar_expect_tx(xbar, (C - 1) * Cfg::BLK_BYTES);
                }
                __syncthreads();
                if constexpr (C > 1) {
                    if (tid < C && tid != rank) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        const int dst = tid;
                        const cpx<T>* src = S + (long)(dst < rank ? dst : dst - 1) * BLK;
                        const uint32_t d =
                            map_rank(smem_addr(W), dst) + (uint32_t)((long)rank * BLK * (long)sizeof(cpx<T>));
                        const uint32_t bar = map_rank(smem_addr(xbar), dst);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
                            "r"(smem_addr(src)), "r"(Cfg::BLK_BYTES), "r"(bar)
                            : "memory");
                    }
                }
                if (tid == 0) {
                    if (!loss) fetch_tables(tab, p + 1);
                    else if (has_next) fetch_tables(item_tables(item_at(it + nclusters)), 0);
                }
                if constexpr (C > 1) {
                    tmo |= !mbar_wait_bounded(xbar, xphase, args.flags, tmo ? 1L : (1L << 26));
                    xphase ^= 1u;
                }
            };
            cpx<T> a[NE];
            T av[NE];   // loss direction: the loss frequency l at the elements zz(m) of this thread's column
            if constexpr (kCompact) {
                // z-pass input of the two tables' columns packed as one complex sequence: Z_k = X_k + i Y_k
                // (X, Y the Hermitian spectra of table 0 and 1, stored as X_0 + i X_{N/2}, X_1 .. X_{N/2-1});
                // its transform holds the two real C2R results as real and imaginary parts.  The loss
                // direction transforms table 0 alone (Y = 0).
                auto load_z = [&](bool two) {
                    const cpx<T>* c0 = Wp + (long)z_src * BLK + widx(0, zl_x, z_kyl, 0);
                    const cpx<T>* c1 = Wp + (long)z_src * BLK + widx(1, zl_x, z_kyl, 0);
#pragma unroll
                    for (int j = 0; j < NE; ++j) {
                        const int k = j * G + g;
                        const int kk = k <= H ? k : N - k;
                        const int e = kk == H ? 0 : kk;
                        const cpx<T> x0 = c0[e];
                        const cpx<T> x1 = two ? c1[e] : cpx<T>{T(0), T(0)};
                        cpx<T> X, Y;
                        if (kk == 0) {
                            X = {x0.x, T(0)};
                            Y = {x1.x, T(0)};
                        } else if (kk == H) {
                            X = {x0.y, T(0)};
                            Y = {x1.y, T(0)};
                        } else if (k < H) {
                            X = x0;
                            Y = x1;
                        } else {
                            X = {x0.x, -x0.y};
                            Y = {x1.x, -x1.y};
                        }
                        a[j] = {X.x - Y.y, X.y + Y.x};
                    }
                };
                // one call site of the length-N transform serves the x-, y- and z-passes (ps = 0, 1, 2):
                // the double-float kernel is bound by instruction fetch, and each inlined transform is
                // thousands of instructions
#pragma unroll 1
                for (int ps = 0; ps < (loss ? 2 : 3); ++ps) {
                    const bool act = ps == 0 ? active : (ps == 1 ? active_y : has_col);
                    if (ps == 0) {
                        if constexpr (Cfg::TAB_SMEM) {
                            tmo |= !mbar_wait_bounded(tbar, tphase, args.flags, tmo ? 1L : (1L << 26));
                            tphase ^= 1u;
                        }
                    } else if (ps == 2) {
                        __syncthreads();   // the y-pass results are in W
                    }
                    if (act) {
                        if (ps == 0) {
                            const cpx<T>* fb = Fh + (long)x_kyl * HF;
                            const T* tslab = Cfg::TAB_SMEM ? Tb : tab + ((long)p * C + rank) * Cfg::TAB_ELEMS;
                            const T* tb = tslab + (long)x_tab * N * NS * HF + (long)x_kyl * HF;
                            if (x_pp == 0) {
#pragma unroll
                                for (int j = 0; j < NE; ++j) {
                                    const long o = (long)(j * G + g) * NS * HF;
                                    const cpx<T> fv = fb[o], fn = fb[o + H];
                                    const T tv = tb[o], tn = tb[o + H];
                                    a[j] = {tv * fv.x - tn * fn.y, tv * fv.y + tn * fn.x};
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < NE; ++j) {
                                    const long o = (long)(j * G + g) * NS * HF + x_pp;
                                    const cpx<T> fv = fb[o];
                                    const T tv = tb[o];
                                    a[j] = {tv * fv.x, tv * fv.y};
                                }
                            }
                        } else if (ps == 1) {
#pragma unroll
                            for (int j = 0; j < NE; ++j) {
                                const int y = j * G + g;
                                a[j] = Wp[ybase + (long)(y / NS) * BLK + (long)(y % NS) * HP];
                            }
                        } else {
                            load_z(true);
                        }
                        fft_split<N, +1, G, R0>(a, g, pmask);
                    }
                    if (ps == 0) {
                        if constexpr (Cfg::XDIRECT) {
                            // straight into block `rank` of the owner's W (this direction's buffer), then
                            // one cluster barrier: every CTA's outputs are in place
                            if (act) {
                                const uint32_t wsrc = smem_addr(Wp + (long)rank * BLK);
#pragma unroll
                                for (int m = 0; m < NE; ++m) {
                                    const int x = zz(m);
                                    const long o = widx(x_tab, x % NS, x_kyl, x_pp);
                                    st_cluster(map_rank(wsrc + (uint32_t)(o * (long)sizeof(cpx<T>)), x / NS), a[m]);
                                }
                            }
                            cluster_arrive();
                            cluster_wait();
                            // the table slab has been read by every thread: the next one (staged tables)
                            if (tid == 0) {
                                if (!loss) fetch_tables(tab, p + 1);
                                else if (has_next) fetch_tables(item_tables(item_at(it + nclusters)), 0);
                            }
                        } else {
                            cluster_wait();   // every CTA has finished reading its W (previous z-pass)
                            if (act) {
#pragma unroll
                                for (int m = 0; m < NE; ++m) {
                                    const int x = zz(m);
                                    const int dst = x / NS;
                                    const long o = widx(x_tab, x % NS, x_kyl, x_pp);
                                    if (dst == rank) W[(long)rank * BLK + o] = a[m];
                                    else S[(long)(dst < rank ? dst : dst - 1) * BLK + o] = a[m];
                                }
                            }
                            exchange();
                        }
                    } else if (ps == 1) {
                        if (act) {
#pragma unroll
                            for (int m = 0; m < NE; ++m) {
                                const int y = zz(m);
                                Wp[ybase + (long)(y / NS) * BLK + (long)(y % NS) * HP] = a[m];
                            }
                        }
                    } else {
                        if (act) {
#pragma unroll
                            for (int m = 0; m < NE; ++m) Gcol[(long)zz(m) * GSTR] += a[m].x * a[m].y;
                        }
                        // staged exchange: this CTA has finished with W (its accesses ordered before peers' copies)
                        if constexpr (!Cfg::XDIRECT) cluster_arrive();
                    }
                }
                if (loss) {
                    __syncthreads();
                    if (has_col) {
                        load_z(false);
                        fft_split<N, +1, G, R0>(a, g, pmask);
#pragma unroll
                        for (int m = 0; m < NE; ++m) av[m] = a[m].x;
                    }
                }
            } else {
                if constexpr (Cfg::TAB_SMEM) {
                    tmo |= !mbar_wait_bounded(tbar, tphase, args.flags, tmo ? 1L : (1L << 26));   // table slab of direction p has landed
                    tphase ^= 1u;
                }
                if (active) {
                    const cpx<T>* fb = Fh + (long)x_kyl * HF;
                    const T* tslab = Cfg::TAB_SMEM ? Tb : tab + ((long)p * C + rank) * Cfg::TAB_ELEMS;
                    const T* tb = tslab + (long)x_tab * N * NS * HF + (long)x_kyl * HF;
                    if (x_pp == 0) {
    #pragma unroll
                        for (int kx = 0; kx < N; ++kx) {
                            const long o = (long)kx * NS * HF;
                            const cpx<T> fv = fb[o], fn = fb[o + H];
                            const T tv = tb[o], tn = tb[o + H];
                            a[kx] = {tv * fv.x - tn * fn.y, tv * fv.y + tn * fn.x};   // tv fv + i tn fn
                        }
                    } else {
    #pragma unroll
                        for (int kx = 0; kx < N; ++kx) {
                            const long o = (long)kx * NS * HF + x_pp;
                            const cpx<T> fv = fb[o];
                            const T tv = tb[o];
                            a[kx] = {tv * fv.x, tv * fv.y};
                        }
                    }
                    fft<N, +1, R0>(a);
                }
                cluster_wait();   // every CTA has finished reading its W (previous z-pass)
                if (active) {
                    // own block directly into W[rank], peers' blocks into staging
    #pragma unroll
                    for (int x = 0; x < N; ++x) {
                        const int dst = x / NS;
                        const long o = widx(x_tab, x % NS, x_kyl, x_pp);
                        if (dst == rank) W[(long)rank * BLK + o] = a[x];
                        else S[(long)(dst < rank ? dst : dst - 1) * BLK + o] = a[x];
                    }
                }
                if constexpr (C > 1) {
                    if (tid == 0) mbar_expect_tx(xbar, (C - 1) * Cfg::BLK_BYTES);
                }
                __syncthreads();   // this CTA's x-pass is complete: staging written, slab free
                if constexpr (C > 1) {
                    // one thread per peer issues that peer's bulk copy (the copies start together)
                    if (tid < C && tid != rank) {
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        const int dst = tid;
                        const cpx<T>* src = S + (long)(dst < rank ? dst : dst - 1) * BLK;
                        const uint32_t d = map_rank(smem_addr(W), dst) + (uint32_t)((long)rank * BLK * (long)sizeof(cpx<T>));
                        const uint32_t bar = map_rank(smem_addr(xbar), dst);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
                            "r"(smem_addr(src)), "r"(Cfg::BLK_BYTES), "r"(bar)
                            : "memory");
                    }
                }
                if (tid == 0) {
                    if (!loss) fetch_tables(tab, p + 1);
                    else if (has_next) fetch_tables(item_tables(item_at(it + nclusters)), 0);
                }
                if constexpr (C > 1) {
                    tmo |= !mbar_wait_bounded(xbar, xphase, args.flags, tmo ? 1L : (1L << 26));   // every peer's block has landed
                    xphase ^= 1u;
                }
                // ---- y-pass in place
                if (active_y) {
    #pragma unroll
                    for (int y = 0; y < N; ++y) a[y] = W[ybase + (long)(y / NS) * BLK + (long)(y % NS) * HP];
                    fft<N, +1, R0>(a);
    #pragma unroll
                    for (int y = 0; y < N; ++y) W[ybase + (long)(y / NS) * BLK + (long)(y % NS) * HP] = a[y];
                }
                __syncthreads();
                // ---- z-pass: C2R along z, products
                if (has_col) {
                    const cpx<T>* c0 = W + (long)z_src * BLK + widx(0, zl_x, z_kyl, 0);
                    cpx<T> h[H];
#pragma unroll
                    for (int k = 0; k < H; ++k) h[k] = c0[k];
                    c2r<N>(h, av);
                }
                if (!loss) {
                    if (has_col) {
                        const cpx<T>* c1 = W + (long)z_src * BLK + widx(1, zl_x, z_kyl, 0);
                        cpx<T> h[H];
#pragma unroll
                        for (int k = 0; k < H; ++k) h[k] = c1[k];
                        T bv[N];
                        c2r<N>(h, bv);
#pragma unroll
                        for (int z = 0; z < N; ++z) {
                            if constexpr (Cfg::G_REG) Greg[z] = fma(av[z], bv[z], Greg[z]);
                            else Gcol[(long)z * GSTR] += av[z] * bv[z];
                        }
                    }
                    cluster_arrive();   // this CTA has finished with W (its accesses ordered before peers' copies)
                }
            }
            if (!loss) {
            } else {
                // loss: r = G - f* l by one fused multiply-add (the product is exact,
                // one rounding of the difference: relative to r itself), Q = r / Kn;
                // the five moments of Q from three sums per column
                const double vx = vel(zx), vy = vel(zl_y);
                const double v2xy = 0.5 * (vx * vx + vy * vy);
                T col[NE];   // f* at the elements zz(m) of this thread's column
                if (has_col) {
#pragma unroll
                    for (int m = 0; m < NE; ++m) col[m] = T(colbase[zoff[zz(m)]]);
                }
                // mode 4, the exponential (integrating-factor) step of the gain-loss split
                // df/dt = G - nu f with nu = l / Kn and G frozen at f*: the increment is
                // dt phi(nu dt) (G - nu f*), phi(x) = (1 - e^-x) / x, then projected like Q (the
                // factor is computed in FP32 except in FP64 contexts; phi -> 1 as nu dt -> 0).  Where the
                // discrete loss frequency is not positive (ringing of the truncated spectrum in the far
                // tails) the term stays explicit: phi(max(x, 0)) = 1.
                const bool expm = args.mode == 4;
                const double kdt = inv_kn * dt_step;
                // slot m of this thread's column (element zz(m))
                auto phi = [&](int m) -> T {
                    if constexpr (sizeof(T) == 8 && !std::is_same<T, dfloat>::value)
                        return exp_step_factor((double)av[m] * kdt);
                    else
                        return T(exp_step_factor((float)av[m] * (float)kdt));
                };
                auto rval = [&](int m) -> T {
                    T gz;
                    if constexpr (Cfg::G_REG) gz = Greg[m];
                    else gz = Gcol[(long)zz(m) * GSTR];
                    const T r = fma(-col[m], av[m], gz);
                    return expm ? r * phi(m) : r;
                };
                const int warp = tid >> 5, lane = tid & 31;
                // escalation bound inputs: sum r^2 (r = G - f* l) and sum (f* l)^2 over the cell (FP32: an
                // estimate of the norms is all the bound needs)
                float e_qq = 0.f, e_ll = 0.f;
                if constexpr (sizeof(T) == 4) {
                    // FP32: compensated sums (hi, lo) with exact products (FMA), carried as pairs
                    // through the warp and block reductions, FP64 from the block totals on (the
                    // FP64 pipe of this part is slow: per-element FP64 sums dominated the epilogue)
                    float2 m5[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) m5[i] = make_float2(0.f, 0.f);
                    if (has_col) {
                        float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
#pragma unroll
                        for (int m = 0; m < NE; ++m) {
                            const int z = zz(m);
                            const float r = rval(m);
                            const float lz = expm ? col[m] * av[m] * phi(m) : col[m] * av[m];
                            e_qq = fmaf(r, r, e_qq);
                            e_ll = fmaf(lz, lz, e_ll);
                            a0 = df_add1(a0, r);
                            const float p = r * vzf[z];
                            const float pe = fmaf(r, vzf[N + z], fmaf(r, vzf[z], -p));
                            a1 = df_add1(a1, p);
                            a1.y += pe;
                            const float q = r * vzf[2 * N + z];
                            const float qe = fmaf(r, vzf[3 * N + z], fmaf(r, vzf[2 * N + z], -q));
                            a2 = df_add1(a2, q);
                            a2.y += qe;
                        }
                        const float2 v2 = df_add(make_float2(vzf[2 * N + zx], vzf[3 * N + zx]),
                                                 make_float2(vzf[2 * N + zl_y], vzf[3 * N + zl_y]));
                        m5[0] = a0;
                        m5[1] = df_mul(a0, make_float2(vzf[zx], vzf[N + zx]));
                        m5[2] = df_mul(a0, make_float2(vzf[zl_y], vzf[N + zl_y]));
                        m5[3] = a1;
                        m5[4] = df_add(df_mul(a0, v2), a2);
                    }
#pragma unroll
                    for (int i = 0; i < 5; ++i)
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) m5[i] = df_add(m5[i], df_shfl_xor(m5[i], off));
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        e_qq += __shfl_xor_sync(0xffffffffu, e_qq, off);
                        e_ll += __shfl_xor_sync(0xffffffffu, e_ll, off);
                    }
                    float2* redw2 = reinterpret_cast<float2*>(redw);
                    if (lane == 0) {
#pragma unroll
                        for (int i = 0; i < 5; ++i) redw2[warp * 7 + i] = m5[i];
                        redw[warp * 7 + 5] = (double)e_ll;
                        redw[warp * 7 + 6] = (double)e_qq;
                    }
                    __syncthreads();
                    if (tid < 5) {
                        float2 acc = make_float2(0.f, 0.f);
                        for (int w = 0; w < NT / 32; ++w) acc = df_add(acc, redw2[w * 7 + tid]);
                        red[tid] = ((double)acc.x + (double)acc.y) * inv_kn;
                    } else if (tid < 7) {
                        double acc = 0.0;
                        for (int w = 0; w < NT / 32; ++w) acc += redw[w * 7 + tid];
                        red[tid] = acc;
                    }
                } else {
                    double s5[5] = {0, 0, 0, 0, 0};
                    if (has_col) {
                        double s0 = 0.0, sz = 0.0, szz = 0.0;
#pragma unroll
                        for (int m = 0; m < NE; ++m) {
                            const int z = zz(m);
                            const double r = (double)rval(m);
                            s0 += r;
                            sz = fma(r, vzt[z], sz);
                            szz = fma(r, vz2t[z], szz);
                        }
                        const double k = inv_kn;
                        s5[0] = s0 * k;
                        s5[1] = vx * s0 * k;
                        s5[2] = vy * s0 * k;
                        s5[3] = sz * k;
                        s5[4] = (v2xy * s0 + szz) * k;
                    }
                    // block reduction of the five moments (fixed order: deterministic)
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        double v = s5[i];
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                        s5[i] = v;
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int i = 0; i < 5; ++i) redw[warp * 7 + i] = s5[i];
                    }
                    __syncthreads();
                    if (tid < 5) {
                        double acc = 0.0;
                        for (int w = 0; w < NT / 32; ++w) acc += redw[w * 7 + tid];
                        red[tid] = acc;
                    } else if (tid < 7) {
                        red[tid] = 0.0;   // the FP64 arithmetic is the last escalation tier
                    }
                }
                cluster_sync_all();
                if (tid < 32) {
                    // warp 0: cluster totals (lane i: moment i over the ranks, in rank order),
                    // mu = P tot, the z part of the correction
                    double tot = 0.0;
                    if (lane < 7)
                        for (int r = 0; r < C; ++r) tot += cluster.map_shared_rank(red, r)[lane];
                    double t5[5];
#pragma unroll
                    for (int i = 0; i < 5; ++i) t5[i] = __shfl_sync(0xffffffffu, tot, i);
                    double mval = 0.0;
                    if (lane < 5) {
                        double acc = 0.0;
                        for (int j = 0; j < 5; ++j) acc += Pm[lane * 5 + j] * t5[j];
                        acc = args.mode == 2 ? 0.0 : acc;   // mode 2: the caller projects
                        mu[lane] = acc;
                        muf[lane] = (float)acc;
                        mval = acc;
                    }
                    // escalation: ||Q_proj||^2 = ||Q||^2 - mu . s (s = the moment sums of Q, mu = P s)
                    double ms = lane < 5 ? mval * tot : 0.0;
#pragma unroll
                    for (int off = 4; off > 0; off >>= 1) ms += __shfl_xor_sync(0xffffffffu, ms, off);
                    const double e_l2 = __shfl_sync(0xffffffffu, tot, 5), e_q2 = __shfl_sync(0xffffffffu, tot, 6);
                    if (lane == 0) {
                        bool esc = false;
                        if (args.esc_list) {
                            const double k2 = inv_kn * inv_kn, qp = k2 * e_q2 - ms;
                            esc = args.esc_c2 * k2 * e_l2 > args.esc_tol2 * (qp > 0.0 ? qp : 0.0);
                        }
                        mu[7] = esc ? 1.0 : 0.0;
                    }
                    __syncwarp();
                    // correction phi(v).mu = mu0 + mu1 vx + mu2 vy + mu4 (vx^2+vy^2)/2 + [mu3 vz + mu4 vz^2/2]
                    for (int z = lane; z < N; z += 32) czt[z] = (T)(mu[3] * vzt[z] + mu[4] * vz2t[z]);
                }
                cluster_sync_all();   // every CTA has read the partials; mu, czt and the decision are visible
                // an escalated cell is left to the next tier (which reads f, and base in mode 3, again)
                const bool escalated = mu[7] != 0.0;
                if (escalated && rank == 0 && tid == 0)
                    args.esc_list[atomicAdd(args.esc_count, 1)] = (int)(BATCH ? item : cell);
                if (has_col && !escalated) {
                    // corrected Q = r / Kn - phi(v).mu, then out = Q or f* + dt Q
                    T cxy;
                    if constexpr (sizeof(T) == 4)
                        cxy = muf[0] + muf[1] * vzf[zx] + muf[2] * vzf[zl_y] +
                              muf[4] * (vzf[2 * N + zx] + vzf[2 * N + zl_y]);
                    else
                        cxy = (T)(mu[0] + mu[1] * vx + mu[2] * vy + mu[4] * v2xy);
                    const T kn = (T)inv_kn, dt = (T)dt_step;
                    const bool heun = !BATCH && args.mode == 3;
                    const bool stepm = args.mode == 1 || heun || expm;
                    ST* dst = fout + cell * N3 + ((long)zx * N + zl_y) * N;
                    // Heun: base row of this column (read before this thread's own store to it)
                    const ST* brow = static_cast<const ST*>(args.base) + cell * N3 + ((long)zx * N + zl_y) * N;
                    bool bad = false, neg = false;
                    // 16-byte vectors of the row where this thread's elements run in whole vectors
                    // (split pencils: runs of N / 2G consecutive elements), single elements otherwise
                    constexpr int VW = 16 / sizeof(ST);
                    constexpr int V = (G == 1 || (N / (2 * G)) % VW == 0) ? VW : 1;
                    static_assert((N * sizeof(ST)) % 16 == 0, "rows are whole 16-byte vectors");
#pragma unroll
                    for (int m0 = 0; m0 < NE; m0 += V) {
                        const int z0 = zz(m0);
                        ST res[V];
                        T bv[V];
                        if (heun) {
                            if constexpr (V == 1) {
                                bv[0] = T(brow[z0]);
                            } else if constexpr (sizeof(ST) == 4) {
                                const float4 w = *reinterpret_cast<const float4*>(brow + z0);
                                bv[0] = T(w.x); bv[1] = T(w.y); bv[2] = T(w.z); bv[3] = T(w.w);
                            } else {
                                const double2 w = *reinterpret_cast<const double2*>(brow + z0);
                                bv[0] = T(w.x); bv[1] = T(w.y);
                            }
                        }
#pragma unroll
                        for (int j = 0; j < V; ++j) {
                            const int z = z0 + j;
                            const T q = fma(rval(m0 + j), kn, -(cxy + czt[z]));
                            T o = stepm ? fma(dt, q, col[m0 + j]) : q;
                            if (heun) o = T(0.5) * (o + bv[j]);
                            res[j] = ST(o);
                            bad |= !isfinite(res[j]);
                            neg |= stepm && (res[j] < ST(0));
                        }
                        if constexpr (V == 1)
                            dst[z0] = res[0];
                        else if constexpr (sizeof(ST) == 4)
                            *reinterpret_cast<float4*>(dst + z0) = make_float4(res[0], res[1], res[2], res[3]);
                        else
                            *reinterpret_cast<double2*>(dst + z0) = make_double2(res[0], res[1]);
                    }
                    if (bad) atomicOr(args.flags, 1);
                    if (neg) atomicOr(args.flags, 2);
                }
            }
        }
        // the loss pass ended with a full cluster sync: W, Fh, S and red are free
    }
}

}  // namespace fks
