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
//   Q   = (G - L) / Kn                               (difference in FP64)
//   Q  -= C^T (C C^T)^-1 C Q                         (FP64 conservation projection)
//   out = Q  or  f* + dt Q
//
// Inverse-pass packing: the kz' = 0 and kz' = N/2 planes of a real field are
// each 2-D Hermitian, so they travel together as one complex plane
// (plane 0 = P_0 + i P_{N/2}); every pass then has exactly N/2 planes.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>

#include "fks_fft.cuh"

namespace cg = cooperative_groups;

namespace fks {

struct CollideArgs {
    const void* f;          // input distribution, ncells * N^3 (element type T)
    void* out;              // Q or f^{n+1}
    const void* tables;     // [M+1][C][2][N kx][NS kyl][H+1 kz'] of T
    const signed char* delta;  // [3][N] cell shifts for this step (transport) or nullptr
    int* flags;             // health bits (atomicOr)
    long ncells;
    int nc[3];              // spatial cells per axis
    int bc[3];              // 0 periodic, 1 specular
    int M;                  // number of directions
    double L;               // velocity box half width
    double inv_kn;
    double dt;              // Euler step (step mode)
    int mode;               // 0 collide (out = Q), 1 step (out = f* + dt Q)
    double P[25];           // dv^6 (C C^T)^-1 over the rows phi = (1, v, |v|^2/2)
};

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
// after ~2^26 polls the kernel records FKS timeout (bit 3) and goes on.
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, unsigned parity, int* flags) {
    for (long it = 0; it < (1L << 26); ++it)
        if (mbar_try_wait(bar, parity)) return;
    atomicOr(flags, 8);
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

template <typename T, int N, int C>
struct CollideCfg {
    static constexpr int NS = N / C;          // slab width (ky for f^, x for W)
    static constexpr int H = N / 2;           // packed planes per inverse transform
    static constexpr int HF = H + 1;          // kz' planes of f^
    static constexpr int HP = H + 1;          // padded plane stride of W
    static constexpr int NTASK = N * N / C;   // pencils / columns per pass per CTA
    static constexpr int NT = (NTASK + 31) / 32 * 32;   // threads per CTA (whole warps)
    // shared memory: Fh, W (cpx<T>); G, f* (T, one column of N per task)
    static constexpr long FH_ELEMS = (long)N * NS * HF;
    static constexpr long W_ELEMS = 2L * NS * N * HP;
    static constexpr long COL_ELEMS = (long)NS * N * N;
    static constexpr long TAB_ELEMS = 2L * N * NS * HF;               // one direction's slab (T)
    static constexpr unsigned TAB_BYTES = (unsigned)(sizeof(T) * TAB_ELEMS);
    static constexpr bool G_REG = sizeof(T) == 4;   // FP32: gain accumulator in registers
    static constexpr size_t SMEM_BYTES = sizeof(cpx<T>) * (FH_ELEMS + W_ELEMS) + sizeof(T) * (2 * COL_ELEMS + TAB_ELEMS) +
                                         sizeof(double) * (8 + (NT / 32) * 5 + 8 + 2 * N + N) + 8 + 3 * N + 16;
    static_assert(TAB_BYTES % 16 == 0, "bulk copies move whole 16-byte units");
    static_assert(N % C == 0, "cluster size must divide N");
};

template <typename T, int N, int C>
__global__ void __launch_bounds__(CollideCfg<T, N, C>::NT, 1)
collide_kernel(CollideArgs args) {
    using Cfg = CollideCfg<T, N, C>;
    constexpr int NS = Cfg::NS, H = Cfg::H, HF = Cfg::HF, HP = Cfg::HP, NT = Cfg::NT, NTASK = Cfg::NTASK;
    constexpr long N3 = (long)N * N * N;

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const long cluster_id = blockIdx.x / C;
    const long nclusters = gridDim.x / C;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* Fh = reinterpret_cast<cpx<T>*>(smem_raw);                 // [N kx][NS kyl][HF]
    cpx<T>* W = Fh + Cfg::FH_ELEMS;                                    // [2][NS xl][N ky][HP]
    T* Tb = reinterpret_cast<T*>(W + Cfg::W_ELEMS);                   // [2][N kx][NS kyl][HF] table slab
    T* Gs = Tb + Cfg::TAB_ELEMS;                                       // [N z][NTASK] gain
    T* Fs = Gs + Cfg::COL_ELEMS;                                       // [N z][NTASK] f*
    double* red = reinterpret_cast<double*>(Fs + Cfg::COL_ELEMS);     // [8] own partials
    double* redw = red + 8;                                            // [NT/32][5]
    double* mu = redw + (NT / 32) * 5;                                 // [8] correction coefficients
    double* vzt = mu + 8;                                              // [N] v_z
    double* vz2t = vzt + N;                                            // [N] v_z^2 / 2
    T* czt = reinterpret_cast<T*>(vz2t + N);                          // [N] projection correction along z
    uint64_t* tbar = reinterpret_cast<uint64_t*>(vz2t + 2 * N);       // table-slab mbarrier
    signed char* dsm = reinterpret_cast<signed char*>(tbar + 1);      // [3][N] shifts

    // shared::cluster addresses of W and Fh in every CTA of the cluster: the
    // window of a CTA is contiguous, so element addresses are base + offset
    uint32_t Wrank[C], Frank[C];
#pragma unroll
    for (int r = 0; r < C; ++r) {
        Wrank[r] = map_rank(smem_addr(W), r);
        Frank[r] = map_rank(smem_addr(Fh), r);
    }
    // store v at element `idx` of W (or Fh) in CTA `dst`
    auto putW = [&](int dst, long idx, cpx<T> v) {
        if constexpr (C == 1) W[idx] = v;
        else st_cluster(Wrank[dst] + (uint32_t)(idx * (long)sizeof(cpx<T>)), v);
    };
    auto putF = [&](int dst, long idx, cpx<T> v) {
        if constexpr (C == 1) Fh[idx] = v;
        else st_cluster(Frank[dst] + (uint32_t)(idx * (long)sizeof(cpx<T>)), v);
    };

    const T* __restrict__ fin = static_cast<const T*>(args.f);
    T* __restrict__ fout = static_cast<T*>(args.out);
    const T* __restrict__ tab = static_cast<const T*>(args.tables);
    const bool transport = args.delta != nullptr;
    for (int i = tid; i < 3 * N; i += NT) dsm[i] = transport ? args.delta[i] : 0;
    const double dv = 2.0 * args.L / N;
    // velocity of grid index i: (i + 1/2 - N/2) dv
    auto vel = [dv](int i) { return ((double)i + 0.5 - 0.5 * N) * dv; };
    for (int i = tid; i < N; i += NT) {
        vzt[i] = vel(i);
        vz2t[i] = 0.5 * vel(i) * vel(i);
    }
    if (tid == 0) {
        mbar_init(tbar, 1);
        fence_mbar_init();
    }
    // every CTA of the cluster is running before any distributed-shared access
    cluster_sync_all();
    unsigned tphase = 0;
    // table slab of direction p (p = M: loss) for this CTA, fetched by one thread
    auto fetch_tables = [&](int p) {
        if (tid == 0) {
            mbar_expect_tx(tbar, Cfg::TAB_BYTES);
            bulk_g2s(Tb, tab + ((long)p * C + rank) * Cfg::TAB_ELEMS, Cfg::TAB_BYTES, tbar);
        }
    };
    if (cluster_id < args.ncells) fetch_tables(0);
    const int ncx = args.nc[0], ncy = args.nc[1], ncz = args.nc[2];

    // z-pass ownership: column (xl, y), x = rank*NS + xl (threads >= NTASK idle)
    const bool has_col = tid < NTASK;
    const int zl_x = has_col ? tid / N : 0, zl_y = tid % N;
    const int zx = rank * NS + zl_x;
    T* Gcol = Gs + tid;   // element z at Gcol[z * NTASK]
    T* Fcol = Fs + tid;

    // y-pass task (tab, xl, plane): plane fastest
    const int t_tab = tid / (NS * H);
    const int t_rem = tid % (NS * H);
    const int t_a = t_rem / H;     // xl
    const int t_pp = t_rem % H;
    // x-pass task (tab, kyl, plane): the 2*NS tasks of the packed plane 0 come
    // first, so that their longer code path diverges inside the first warp only
    int x_tab, x_kyl, x_pp;
    if (tid < 2 * NS) {
        x_pp = 0;
        x_tab = tid / NS;
        x_kyl = tid % NS;
    } else {
        const int u = tid - 2 * NS;
        x_pp = 1 + u % (H - 1);
        x_kyl = (u / (H - 1)) % NS;
        x_tab = u / ((H - 1) * NS);
    }

    for (long cell = cluster_id; cell < args.ncells; cell += nclusters) {
        const int cx = (int)(cell / ((long)ncy * ncz));
        const int cy = (int)((cell / ncz) % ncy);
        const int cz = (int)(cell % ncz);

        // ---------------- forward transform -----------------------------
        // F1: gather the f* column (x, y, :) of the transported cell into
        // shared memory, z-R2C; staging S = W[0] as [xl][y][HP]
        if (has_col) {
            if (!transport) {
                const T* src = fin + cell * N3 + ((long)zx * N + zl_y) * N;
#pragma unroll 4
                for (int z = 0; z < N; ++z) Fcol[(long)z * NTASK] = src[z];
            } else {
                int fx, fy;
                const int sx = fold_cell(cx - dsm[zx], ncx, args.bc[0], fx);
                const int sy = fold_cell(cy - dsm[N + zl_y], ncy, args.bc[1], fy);
                const int qx = fx ? N - 1 - zx : zx;
                const int qy = fy ? N - 1 - zl_y : zl_y;
                const T* base_xy = fin + ((long)sx * ncy + sy) * ncz * N3 + ((long)qx * N + qy) * N;
#pragma unroll 4
                for (int z = 0; z < N; ++z) {
                    int fz;
                    const int sz = fold_cell(cz - dsm[2 * N + z], ncz, args.bc[2], fz);
                    const int qz = fz ? N - 1 - z : z;
                    Fcol[(long)z * NTASK] = base_xy[(long)sz * N3 + qz];
                }
            }
            cpx<T> a[N];
#pragma unroll
            for (int z = 0; z < N; ++z) a[z] = {Fcol[(long)z * NTASK], T(0)};
            fft<N, -1>(a);
            cpx<T>* S = W + ((long)zl_x * N + zl_y) * HP;
#pragma unroll
            for (int k = 0; k < HF; ++k) S[k] = a[k];
            if constexpr (!Cfg::G_REG) {
#pragma unroll
                for (int z = 0; z < N; ++z) Gcol[(long)z * NTASK] = T(0);
            }
        }
        T Greg[Cfg::G_REG ? N : 1];
        if constexpr (Cfg::G_REG) {
#pragma unroll
            for (int z = 0; z < N; ++z) Greg[z] = T(0);
        }
        __syncthreads();
        // F2 + F3: y-FFT of (xl, kz') pencils, scatter to the ky owner as Fh[x][kyl][kz']
        if (tid < NS * HF) {
            const int xl = tid / HF, kz = tid % HF;
            cpx<T> a[N];
#pragma unroll
            for (int y = 0; y < N; ++y) a[y] = W[((long)xl * N + y) * HP + kz];
            fft<N, -1>(a);
            const int x = rank * NS + xl;
#pragma unroll
            for (int ky = 0; ky < N; ++ky) putF(ky / NS, ((long)x * NS + ky % NS) * HF + kz, a[ky]);
        }
        cluster_sync_all();
        // F4: x-FFT of (kyl, kz') pencils in place
        if (tid < NS * HF) {
            const int kyl = tid / HF, kz = tid % HF;
            cpx<T> a[N];
#pragma unroll
            for (int x = 0; x < N; ++x) a[x] = Fh[((long)x * NS + kyl) * HF + kz];
            fft<N, -1>(a);
#pragma unroll
            for (int kx = 0; kx < N; ++kx) Fh[((long)kx * NS + kyl) * HF + kz] = a[kx];
        }
        __syncthreads();

        // ---------------- gain and loss ---------------------------------
        cluster_arrive_relaxed();   // matches the wait before the first x-pass scatter
        for (int p = 0; p <= args.M; ++p) {
            const bool loss = (p == args.M);
            // ---- x-pass: table product, pack kz'=0 with kz'=N/2, inverse FFT along kx
            const bool active = has_col && (!loss || x_tab == 0);
            const bool active_y = has_col && (!loss || t_tab == 0);
            cpx<T> a[N];
            mbar_wait_bounded(tbar, tphase, args.flags);   // table slab of direction p has landed
            tphase ^= 1u;
            if (active) {
                const T* tb = Tb + (long)x_tab * N * NS * HF + (long)x_kyl * HF;
                const cpx<T>* fb = Fh + (long)x_kyl * HF;
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
                fft<N, +1>(a);
            }
            cluster_wait();   // every CTA has finished reading its W (previous z-pass)
            if (active) {
                const int ky = rank * NS + x_kyl;
#pragma unroll
                for (int x = 0; x < N; ++x)
                    putW(x / NS, (((long)x_tab * NS + x % NS) * N + ky) * HP + x_pp, a[x]);
            }
            cluster_sync_all();
            // every thread of this CTA is past its x-pass: the slab buffer is free
            if (!loss) fetch_tables(p + 1);
            else if (cell + nclusters < args.ncells) fetch_tables(0);
            // ---- y-pass in place
            if (active_y) {
                cpx<T>* base = W + ((long)t_tab * NS + t_a) * N * HP + t_pp;
#pragma unroll
                for (int y = 0; y < N; ++y) a[y] = base[(long)y * HP];
                fft<N, +1>(a);
#pragma unroll
                for (int y = 0; y < N; ++y) base[(long)y * HP] = a[y];
            }
            __syncthreads();
            // ---- z-pass: C2R along z, products
            T av[N];
            if (has_col) {
                const cpx<T>* c0 = W + ((long)zl_x * N + zl_y) * HP;          // table 0
                cpx<T> h[H];
#pragma unroll
                for (int k = 0; k < H; ++k) h[k] = c0[k];
                c2r<N>(h, av);
            }
            if (!loss) {
                if (has_col) {
                    const cpx<T>* c1 = W + ((long)(NS + zl_x) * N + zl_y) * HP;   // table 1
                    cpx<T> h[H];
#pragma unroll
                    for (int k = 0; k < H; ++k) h[k] = c1[k];
                    T bv[N];
                    c2r<N>(h, bv);
#pragma unroll
                    for (int z = 0; z < N; ++z) {
                        if constexpr (Cfg::G_REG) Greg[z] = fma(av[z], bv[z], Greg[z]);
                        else Gcol[(long)z * NTASK] += av[z] * bv[z];
                    }
                }
                cluster_arrive_relaxed();   // this CTA has finished reading W
            } else {
                // loss: r = G - f* l by one fused multiply-add (the product is exact,
                // one rounding of the difference: FP32 relative to r itself), Q = r / Kn;
                // the five moments of Q from three FP64 sums per column
                double s5[5] = {0, 0, 0, 0, 0};
                const double vx = vel(zx), vy = vel(zl_y);
                const double v2xy = 0.5 * (vx * vx + vy * vy);
                auto gval = [&](int z) -> T {
                    if constexpr (Cfg::G_REG) return Greg[z];
                    else return Gcol[(long)z * NTASK];
                };
                auto rval = [&](int z) -> T { return fma(-Fcol[(long)z * NTASK], av[z], gval(z)); };
                if (has_col) {
                    double s0 = 0.0, sz = 0.0, szz = 0.0;
#pragma unroll
                    for (int z = 0; z < N; ++z) {
                        const double r = (double)rval(z);
                        s0 += r;
                        sz = fma(r, vzt[z], sz);
                        szz = fma(r, vz2t[z], szz);
                    }
                    const double k = args.inv_kn;
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
                const int warp = tid >> 5, lane = tid & 31;
                if (lane == 0) {
#pragma unroll
                    for (int i = 0; i < 5; ++i) redw[warp * 5 + i] = s5[i];
                }
                __syncthreads();
                if (tid == 0) {
                    for (int i = 0; i < 5; ++i) {
                        double acc = 0.0;
                        for (int w = 0; w < NT / 32; ++w) acc += redw[w * 5 + i];
                        red[i] = acc;
                    }
                }
                cluster_sync_all();
                if (tid == 0) {
                    double tot[5] = {0, 0, 0, 0, 0};
                    for (int r = 0; r < C; ++r) {
                        const double* rr = cluster.map_shared_rank(red, r);
                        for (int i = 0; i < 5; ++i) tot[i] += rr[i];
                    }
                    for (int i = 0; i < 5; ++i) {
                        double acc = 0.0;
                        for (int j = 0; j < 5; ++j) acc += args.P[i * 5 + j] * tot[j];
                        mu[i] = acc;
                    }
                    // correction phi(v) . mu = mu0 + mu1 vx + mu2 vy + [mu3 vz + mu4 vz^2/2] + mu4 (vx^2+vy^2)/2
                    for (int z = 0; z < N; ++z) czt[z] = (T)(mu[3] * vzt[z] + mu[4] * vz2t[z]);
                }
                cluster_sync_all();   // every CTA has read the partials; mu and czt are visible
                if (has_col) {
                    // corrected Q = r / Kn - phi(v).mu, then out = Q or f* + dt Q
                    const T cxy = (T)(mu[0] + mu[1] * vx + mu[2] * vy + mu[4] * v2xy);
                    const T kn = (T)args.inv_kn, dt = (T)args.dt;
                    const bool stepm = args.mode == 1;
                    T* dst = fout + cell * N3 + ((long)zx * N + zl_y) * N;
                    bool bad = false, neg = false;
                    constexpr int V = 16 / sizeof(T);
                    static_assert((N * sizeof(T)) % 16 == 0, "rows are whole 16-byte vectors");
#pragma unroll
                    for (int z0 = 0; z0 < N; z0 += V) {
                        T res[V];
#pragma unroll
                        for (int j = 0; j < V; ++j) {
                            const int z = z0 + j;
                            const T q = fma(rval(z), kn, -(cxy + czt[z]));
                            const T o = stepm ? fma(dt, q, Fcol[(long)z * NTASK]) : q;
                            bad |= !isfinite(o);
                            neg |= stepm && (o < T(0));
                            res[j] = o;
                        }
                        if constexpr (sizeof(T) == 4)
                            *reinterpret_cast<float4*>(dst + z0) = make_float4(res[0], res[1], res[2], res[3]);
                        else
                            *reinterpret_cast<double2*>(dst + z0) = make_double2(res[0], res[1]);
                    }
                    if (bad) atomicOr(args.flags, 1);
                    if (neg) atomicOr(args.flags, 2);
                }
            }
        }
        // the loss pass ended with a full cluster sync: W, Fh and red are free
    }
}

}  // namespace fks
