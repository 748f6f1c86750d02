// fks_internal.h -- declarations shared by the translation units of libfks.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "fks_collide.cuh"

namespace fks {

// One instantiation of collide_kernel<T, N, C>.
struct CollideVariant {
    const void* func;     // host stub of the kernel (cells of one problem)
    const void* func_batch;   // host stub of the batch kernel (one homogeneous problem per item)
    int N, C, NT;
    size_t smem;
    bool fp64;
    int radix = 0;            // top radix of the length-N transforms (0: the default schedule)
};

// Look up an instantiation; returns false if (fp64, N, C, radix) was not compiled (radix 0: the
// default schedule; other radixes: FP32 only).
bool find_collide_variant(bool fp64, int N, int C, CollideVariant* out, int radix = 0);
bool find_collide_variant_f32_radix(int N, int C, int R0, CollideVariant* out);
bool find_collide_variant_f32(int N, int C, CollideVariant* out);
bool find_collide_variant_f64(int N, int C, CollideVariant* out);
// FP64 arithmetic over an FP32 state (the last tier of the precision escalation), and the same
// with double-float arithmetic on the FP32 pipes
bool find_collide_variant_mixed(int N, int C, CollideVariant* out);
bool find_collide_variant_dfloat(int N, int C, CollideVariant* out);
// the double-float instantiation of each n at its cluster size (fks_collide_df*.cu)
bool find_collide_variant_dfloat_8(CollideVariant* out);
bool find_collide_variant_dfloat_16(CollideVariant* out);
bool find_collide_variant_dfloat_24(CollideVariant* out);
bool find_collide_variant_dfloat_32(CollideVariant* out);

// fill *out with the instantiation collide_kernel<T, N, C, *, ST, R0> (both the cell and the batch kernel)
template <typename T, int N, int C, typename ST = T, int R0 = 0>
inline bool collide_variant(CollideVariant* out) {
    using Cfg = CollideCfg<T, N, C>;
    out->func = reinterpret_cast<const void*>(&collide_kernel<T, N, C, false, ST, R0>);
    out->func_batch = reinterpret_cast<const void*>(&collide_kernel<T, N, C, true, ST, R0>);
    out->N = N;
    out->C = C;
    out->NT = Cfg::NT;
    out->smem = Cfg::SMEM_BYTES;
    out->fp64 = sizeof(T) == 8;
    out->radix = R0;
    return true;
}

// One tier of the precision escalation: the cluster kernel that recomputes the listed cells of the
// tier before it (FP32 arithmetic, or FP64 arithmetic over the FP32 state) with its own tables.
struct EscTier {
    bool fp64 = false;          // FP64-accurate arithmetic (FP64 or double-float)
    bool dfl = false;           // double-float pairs on the FP32 pipes
    CollideVariant var{};
    int C = 0;
    int max_clusters = 0;
    void* tables = nullptr;
};

// Arguments of the BGK relaxation kernel (fks_bgk.cu).
struct BgkArgs {
    const void* f;
    void* out;
    const signed char* delta;   // [3][n] shifts (transport) or nullptr
    int* flags;
    long ncells;                // end (exclusive) of the cells this launch processes
    long cell0;                 // first cell
    int nc[3], bc[3];
    double L, inv_kn, dt;
    int mode;                   // 0 collide, 1 step, 3 second Heun stage (out = (base + f* + dt Q) / 2),
                                // 4 exponential step (out = f* + (1 - e^{-nu dt}) / nu Q)
    double P[25];
    const void* base = nullptr; // mode 3: the first stage's input (may be out itself)
};
cudaError_t launch_bgk(bool fp64, int n, const BgkArgs& a, cudaStream_t s);

// Default cluster size for (precision, N).
int default_cluster_size(bool fp64, int N);

// Tensor-core (split BF16) collision kernel (fks_collide_tc.cu), n = 16 or 32.
struct TcLaunch {
    const void* f;
    void* out;
    const void* tables;         // [M+1][n][n][n] float2
    const void* dft;            // BF16 DFT matrices (tc_dft_matrices)
    void* scratch;              // grid x tc_scratch_per_cta(n) bytes
    const signed char* delta;   // transport shifts (step) or nullptr
    int* flags;
    long ncells;
    const int* cells = nullptr; // optional device list of cell indices (the cells to process)
    const int* cells_count = nullptr;   // optional device count of `cells` (ncells then only sizes the grid)
    int* esc_list = nullptr;    // precision escalation output (see CollideArgs)
    int* esc_count = nullptr;
    double esc_c2 = 0.0, esc_tol2 = 0.0;
    // cells whose bound with esc_last_c2 exceeds the tolerance go straight to the last tier's list
    // (the FP32 tier would list them again); nullptr: every escalated cell goes to esc_list
    int* esc_last_list = nullptr;
    int* esc_last_count = nullptr;
    double esc_last_c2 = 0.0;
    int nc[3], bc[3];
    int M;
    double L, inv_kn, dt;
    int mode;
    double P[25];
    int grid;                   // CTAs the scratch is sized for
};
cudaError_t launch_collide_tc(int n, const TcLaunch& l, cudaStream_t s);
long tc_scratch_per_cta(int n);
void tc_dft_matrices(int n, std::vector<uint16_t>& out);

// Separable expansion of the variable-hard-sphere kernel (fks_vhs.cu):
// H(t, u) ~ sum_{s<S} phi_s(t) psi_s(u), phi_s(t) = sum_i ca[s][i] cos(r_i t),
// psi_s(u) = sum_i cb[s][i] J0(r_i u) over Q radial nodes r_i.
constexpr int kVhsMaxTerms = 64;
struct VhsExpansion {
    int S = 0, Q = 0;
    double err = 0.0;               // max |H_S - H| / max |H| on the check grid
    std::vector<double> r, ca, cb;  // [Q], [S][Q], [S][Q]
    std::vector<double> lambda;     // [S] eigenvalues kept
};
// truncation target of the automatic term count: the rounding scale of the precision
inline double vhs_tolerance(int precision) { return precision == FKS_FP64 ? 1e-12 : 1e-7; }
__host__ __device__ inline double vhs_phi(const double* ca, const double* r, int Q, double t) {
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) acc += ca[i] * cos(r[i] * t);
    return acc;
}
__host__ __device__ inline double vhs_psi(const double* cb, const double* r, int Q, double u) {
    double acc = 0.0;
    for (int i = 0; i < Q; ++i) acc += cb[i] * j0(r[i] * u);
    return acc;
}
// terms = 0: the smallest S meeting tol on the frequencies of the n^3 grid
fks_status vhs_expand(double alpha, double C, double L, int n, double tol, int terms, VhsExpansion* out,
                      std::string* err);

// Status after a failed device allocation (or the copy that follows it): FKS_ERR_OOM when the
// device ran out of memory, FKS_ERR_CUDA for any other CUDA error (no device, driver).  Reads and
// clears the runtime's last error, so that a later launch check does not report it again.
inline fks_status alloc_failure() {
    return cudaGetLastError() == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
}

// Helpers of the context API (fks_capi.cu) that the uneven batches (fks_batch.cu) share.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// Look up the (precision, n, C) instantiation, raise its shared-memory limit and count how many
// clusters can be resident at once (*found = false: no such instantiation).
cudaError_t query_variant(bool fp64, int n, int C, CollideVariant* v, int* max_clusters, bool* found, int radix = 0);
// Spectral tables of one (n, L, kernel, directions) in the collision kernel's layout for cluster
// size C (full: the unsplit layout of the split-BF16 kernel), built on the device in FP64 and
// stored in the working precision; *out is a new device allocation.  vx (FKS_VHS only): the
// separable terms, table pair p * S + s being term s of direction p.
// dfl: the cluster layout with double-float (hi, lo) elements (fp64 must be true: 8 bytes each)
fks_status build_tables_raw(int n, const fks_dirs& dirs, double L, int ktype, double Ck, int C, bool fp64,
                            void** out, std::string* err, bool full = false, const VhsExpansion* vx = nullptr,
                            bool dfl = false);
// P = (sum_k phi(v_k) phi(v_k)^T)^-1 over the n^3 grid on [-L, L)^3, phi = (1, v, |v|^2/2)
void projection_matrix(int n, double L, double* P);

}  // namespace fks

// Context state (fks_capi.cu); visible to the other translation units.
struct fks_ctx {
    bool bgk = false;           // BGK relaxation instead of the spectral operator
    bool tc = false;            // split-BF16 tensor-core transforms (FKS_BF16X3)
    void* tc_dft = nullptr;     // BF16 DFT matrices
    void* tc_scratch = nullptr; // per-CTA spectrum and pass-3 operand scratch
    int tc_grid = 0;
    // fks_step_host: device copies of the state, copy streams, per-chunk events
    void* h_in = nullptr;
    void* h_out = nullptr;
    cudaStream_t h_up = nullptr, h_down = nullptr;
    cudaEvent_t h_ev[3][64] = {};
    // variant B (fks_set_dealias): inner context of the 2n grid, chunk buffers, P and T
    bool dealias = false;
    fks_ctx* inner = nullptr;
    void* d2f = nullptr;
    void* d2q = nullptr;
    void* dPm = nullptr;
    void* dTm = nullptr;
    long dchunk = 0;
    fks_grid grid;
    fks_vbox vbox;
    fks_kernel kern;
    fks::VhsExpansion vhs;      // FKS_VHS: the separable terms (M = A1 A2 S table pairs)
    fks_dirs dirs;
    bool fp64;
    int n, M, C;
    long ncells;
    double dx[3];
    void* tables = nullptr;     // collision-kernel layout, element T
    double* d_s = nullptr;      // [3][n] offsets
    signed char* d_delta = nullptr;
    int* d_flags = nullptr;
    double P[25];
    fks::CollideVariant var;
    int max_clusters = 0;
    long launches = 0;
    std::string err;
    int device = 0;
    double* d_P = nullptr;      // device copy of P (batch-mode descriptors)
    // surrogate routing workspace (allocated on first use)
    double* s_rho = nullptr;
    float* s_dist = nullptr;
    float* s_ind = nullptr;
    int* s_cells = nullptr;     // routed cell indices
    int* s_cand = nullptr;      // cells the network infers
    int* s_count = nullptr;     // [2]: routed, candidates
    // precision escalation (FP32 and split-BF16 contexts): cells whose error bound exceeds esc_tol are
    // listed by the context's kernel and recomputed by esc[0] (whose own failures go to esc[1])
    double esc_tol = 0.0;       // 0: off
    int esc_ntier = 0;
    int esc_arith = FKS_FP32X2; // arithmetic of the last tier: FKS_FP32X2 or FKS_FP64
    bool esc_direct = true;     // split BF16: cells beyond the FP32 tier's reach go straight to the last tier
    fks::EscTier esc[2];
    int* esc_lists = nullptr;   // [2][ncells]
    int* esc_counts = nullptr;  // [2]
    // stage timing (fks_set_profiling): CUDA-event pairs around each collision launch, by stage
    // (0 the context's kernel, 1 and 2 the escalation tiers), summed by fks_get_profile
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev[3];   // start, end, start, end, ...
    std::vector<cudaEvent_t> prof_pool;
};


// Context helpers shared by the translation units (fks_capi.cu): record an
// error message and return the status; launch a context's collision kernel
// (mode 0 collide, 1 step without transport, 2 collide without projection).
// (C linkage: they are defined beside the C ABI.)
extern "C" fks_status fks_internal_fail(fks_ctx* c, fks_status st, const std::string& msg);
extern "C" fks_status fks_internal_collide(fks_ctx* c, const void* f, void* out, int mode, cudaStream_t s);
// collide (projected, with the context's escalation) only the cells cells[0 .. *count) (a device count):
// mode 0 out = Q, mode 1 out = f + dt Q (no transport)
// keep_counts: the escalation counts were reset by fks_internal_last_tier_route before a classification
// that listed cells for the last tier (the tiers then add to that list)
extern "C" fks_status fks_internal_collide_list(fks_ctx* c, const void* f, void* out, const int* cells, const int* count,
                                                int mode, double dt, cudaStream_t s, int keep_counts);
// Before a classification of the cells (surrogate step): resets the escalation counts on s and returns
// the last tier's device list and count and the distance from equilibrium d = ||f - M|| / ||M|| below
// which a cell certainly fails every earlier tier (d_max = 0: no such route; list = nullptr: no tiers),
// and for split-BF16 contexts the FP32 tier's list, count and the distance below which a cell fails the
// split-BF16 bound (d_mid = 0: none).  See kKappaDist.
extern "C" fks_status fks_internal_last_tier_route(fks_ctx* c, cudaStream_t s, int** list, int** count, double* d_max,
                                                   int** mid_list, int** mid_count, double* d_mid);
// variant B (fks_dealias.cu)
fks_status launch_dealias(fks_ctx* c, const void* f, void* out, const signed char* delta, double dt, int mode,
                          cudaStream_t s);

// Surrogate network internals (fks_net.cu) used by the routing path.
const float* fks_net_forward_internal(fks_net* m, int batch, const float* x, cudaStream_t s, fks_status* st);
const float* fks_net_infer_internal(fks_net* m, int batch, const float* x, cudaStream_t s, fks_status* st);
// inference chunk of the routing path: cells per fks_net_infer_internal call
// (allocates the inference workspace on first use; 0 if that fails) and its
// [capacity][2][n^3] FP32 input buffer
int fks_net_infer_capacity(fks_net* m);
float* fks_net_input_buffer(fks_net* m);
int fks_net_grid(const fks_net* m);
int fks_net_max_batch(const fks_net* m);
