/*
 * fks.h -- C ABI of the GB300 Fast Kinetic Scheme library (libfks.so).
 *
 * Method: J. Narski, "Fast Kinetic Scheme: efficient MPI parallelization
 * strategy for 3D Boltzmann equation", arXiv 1701.01608.
 *   - phase space: N_s spatial cells x N_v = n^3 discrete velocities (Sec. 2.1,
 *     "Let us start by truncating a velocity space"), velocity grid cell-centred
 *     on [-L, L]^3: v_i = (i + 1/2 - n/2) * 2L/n;
 *   - transport: exact shift of the generic-cell particles (Sec. 2.1
 *     "Transport step", Sec. 3);
 *   - collision: explicit Euler f = f* + dt Q(f*) (Eq. disc_relax) with the
 *     fast spectral Boltzmann operator Q (Appendix A);
 *   - moments U = (rho, rho u, E) = sum_k phi(v_k) f_k dv^3 (Sec. 3).
 *
 * Data layout of every distribution array: f[cell][ix][iy][iz] (iz fastest),
 * cell = (cx*ny + cy)*nz + cz, element type double for FKS_FP64 and float
 * for FKS_FP32.  All distribution / moment pointers are DEVICE pointers owned
 * by the caller, 16-byte aligned, and must not alias unless stated.  The
 * library owns its tables, offsets and flags.  `stream` is a cudaStream_t
 * (NULL = legacy default stream); every call only enqueues work on it.
 *
 * Errors: every call returns an fks_status; nothing throws across the ABI.
 * Invalid arguments are rejected before any work is enqueued.  Kernel health
 * bits (non-finite result, negative f after a step) are read by fks_check.
 * fks_last_error() gives a message for the last failing call on a context.
 * One context per stream: calls on one context are not thread-safe.
 */
#ifndef FKS_H
#define FKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fks_ctx fks_ctx;

typedef enum {
    FKS_OK = 0,
    FKS_ERR_INVALID_ARG = 1,
    FKS_ERR_UNSUPPORTED = 2,
    FKS_ERR_OOM = 3,        /* a device allocation failed for lack of memory */
    FKS_ERR_CUDA = 4,       /* any other CUDA error (no device, driver, launch, copy) */
    FKS_ERR_NUMERIC = 5,
    FKS_ERR_TIMEOUT = 6
} fks_status;

enum { FKS_BC_PERIODIC = 0, FKS_BC_SPECULAR = 1 };
/* FKS_BF16X3: FP32 storage and FP32 work between the transforms, every DFT on
 * the tensor cores as a split-BF16 product (x = hi + lo for both factors,
 * hi*hi + lo*hi + hi*lo accumulated in FP32); n = 16 or 32, spectral kernels
 * only (not BGK, not batches). */
/* FKS_FP32X2: double-float arithmetic (an unevaluated sum of two FP32 values,
 * about 48 significant bits, on the FP32 pipes); the arithmetic of the last
 * precision-escalation tier (fks_set_escalation_arith), not a context
 * precision. */
enum { FKS_FP64 = 0, FKS_FP32 = 1, FKS_BF16X3 = 2, FKS_FP32X2 = 3 };
enum { FKS_HARD_SPHERE = 0, FKS_MAXWELL = 1, FKS_BGK = 2, FKS_VHS = 3 };

/* Spatial grid: nx*ny*nz cells (fewer than 2^31) on the box [x0, x1]; bc[a]
 * applies to both walls of axis a.  nx = ny = nz = 1 is the space-homogeneous
 * problem. */
typedef struct {
    int nx, ny, nz;
    double x0[3], x1[3];
    int bc[3];
} fks_grid;

/* Velocity box: n^3 points on [-L, L]^3; n in {8, 16, 24, 32}. */
typedef struct {
    int n;
    double L;
} fks_vbox;

/* Collision kernel (Appendix A, Eq. Btilde_pl):
 *   FKS_HARD_SPHERE: B~(|x|,|y|) = 4C             (C = 1/4 gives B~ = 1)
 *   FKS_MAXWELL:     B~(|x|,|y|) = 4C (|x||y|)^-1/2, a separable kernel whose
 *                    collision kernel B = C (sin(theta)/2)^-1/2 does not
 *                    depend on |g| (Maxwell type).
 *   FKS_VHS:         variable hard spheres B = C |g|^alpha, -1 <= alpha <= 1
 *                    (alpha = 0: Maxwell molecules, alpha = 1: hard spheres):
 *                    B~(|x|,|y|) = 4C (|x|^2 + |y|^2)^((alpha-1)/2), which is
 *                    not a product a(|x|) b(|y|) for alpha != 1.  The library
 *                    expands the radial factor of B_F(l, m) into `terms`
 *                    separable terms (eigen-decomposition of the kernel on a
 *                    radial quadrature; terms = 0 picks the smallest count whose
 *                    error on the grid's frequencies is below 1e-7 (FP32,
 *                    BF16X3) or 1e-12 (FP64) of the factor), each term one more
 *                    pair of tables per direction: the cost grows with the
 *                    count.  Not available in batches.
 * The operator returned is Q / knudsen.
 *   FKS_BGK:         the BGK relaxation nu (M[f] - f) of Sec. 2 with the
 *                    cell's Maxwellian M[f] and nu = rho / knudsen (C unused),
 *                    followed by the same conservation projection; not
 *                    available in batches.
 * alpha and terms are read for FKS_VHS only (terms <= 64). */
typedef struct {
    int type;
    double C;
    double knudsen;
    double alpha;
    int terms;
} fks_kernel;

/* Collision directions (Appendix A): M = A1*A2 half-sphere directions
 * e = (sin t cos f, sin t sin f, cos t), f_q = q pi/A2, weight
 * pi^2/(A1 A2) sin t_p;  rule 0: t_p = (p + 1/2) pi/A1, rule 1: t_p = p pi/A1. */
typedef struct {
    int A1, A2;
    int rule;
} fks_dirs;

/* Create a context: validates the arguments, builds the spectral tables on
 * the current device (FP64 arithmetic, stored in the working precision),
 * and allocates the per-context state (sub-cell offsets, shift table,
 * flags).  precision: FKS_FP64, FKS_FP32 or FKS_BF16X3 (element type float
 * for the last two).  On failure *out is NULL. */
fks_status fks_init(const fks_grid *grid, const fks_vbox *vbox, const fks_kernel *kernel,
                    const fks_dirs *dirs, int precision, fks_ctx **out);

/* Q[cell] = Q(f[cell]) / Kn for every cell (Appendix A), followed by the
 * conservation projection Q <- Q - C^T (C C^T)^-1 C Q onto the space
 * orthogonal to the collision invariants (1, v, |v|^2/2): FP64 coefficients
 * from moment sums in FP64 (FP64 states) or in compensated FP32 pairs (FP32
 * states), so the stored Q conserves to the rounding of its own values.
 * f, Q: device arrays of ncells * n^3 elements; f and Q must not overlap. */
fks_status fks_collide(fks_ctx *ctx, const void *f, void *Q, void *stream);

/* Precision escalation of FKS_FP32 and FKS_BF16X3 contexts (the FP64 kept for
 * the gain-loss subtraction near equilibrium).  Near equilibrium the gain G
 * and the loss L = f* IDFT(betaL F) of Appendix A cancel to a few digits, and
 * the rounding of the transforms (not of the subtraction itself) bounds the
 * error of Q at about c ||L|| / Kn: c ~ 2.4e-7 in FP32, ~5e-6 for the split-BF16
 * tensor cores.  After its projection, each cell whose bound
 * c ||L|| / Kn exceeds tol ||Q|| (c: 5e-7 FP32, 1.5e-5 split BF16, with a margin)
 * is not written by the context's kernel but listed on the device and
 * recomputed by the next tier: FKS_FP32 contexts -> FP64 arithmetic over the
 * FP32 state; FKS_BF16X3 -> FP32 (with the same test) -> FP64.  Every cell of
 * fks_collide, fks_step, fks_step_strang and fks_surrogate_collide then meets
 * relative L2 <= tol of Q against the FP64 operator, with no host
 * synchronisation (the tiers read the device counts).  Default tol: 1e-5
 * (FP32), 1e-3 (BF16X3); tol = 0 switches it off (the raw FP32 / split-BF16
 * result).  FKS_ERR_UNSUPPORTED for a positive tol on FP64, BGK and FKS_VHS
 * contexts (no tiers).  Synchronises the device. */
fks_status fks_set_escalation(fks_ctx *ctx, double tol);
/* Arithmetic of the last escalation tier: FKS_FP32X2 (default; double-float
 * pairs on the FP32 pipes, relative error ~1e-14 of the loss term, enough for
 * tol down to ~1e-6 at ||L|| / ||Q|| = 1e7) or FKS_FP64 (GB300's FP64 pipe,
 * 1/64 of the FP32 rate).  Rebuilds that tier's tables; synchronises the
 * device.  FKS_ERR_UNSUPPORTED on contexts without tiers. */
fks_status fks_set_escalation_arith(fks_ctx *ctx, int arith);
/* Direct routes to the last escalation tier of the bound above (the loss term
 * L of the gain-loss split of Appendix A against ||Q||), on by default
 * (on != 0) for contexts with tiers (FKS_ERR_UNSUPPORTED otherwise,
 * FKS_ERR_INVALID_ARG for a NULL ctx; takes effect from the next call):
 *  - FKS_BF16X3: a cell whose FP32 bound must also exceed tol (the split-BF16
 *    kernel's own estimates of ||Q|| and ||L|| show c_32 ||L|| / Kn > tol ||Q||
 *    whatever the FP32 tier computes, c_32 = 5e-7, the split-BF16 error
 *    allowed for) is listed for the last tier at once instead of passing
 *    through the FP32 tier.  The last tier recomputes from f*, so the results
 *    are identical either way; only the FP32 tier's work changes.
 *  - fks_surrogate_step / fks_surrogate_collide: the classification before
 *    inference sends a cell whose distance from its local Maxwellian
 *    d = ||f* - M|| / ||M|| is below 0.1 c_32 / tol straight to the last tier
 *    (near equilibrium ||Q|| <~ d ||L|| / k_d + ||Q(M)||, k_d = 0.75 .. 2.6
 *    measured, the residual Q(M) below 1e-5 ||L||: such a cell fails the
 *    earlier tiers' bound), skipping the context's own kernel; results are
 *    identical wherever that holds, and a cell where it did not would get the
 *    last tier's (more accurate) result.  In FKS_BF16X3 contexts a cell with
 *    d below 0.1 c_b / tol (c_b = 1.5e-5, the split-BF16 constant) goes
 *    straight to the FP32 tier in the same way.
 * Off: every escalated cell passes through every tier. */
fks_status fks_set_escalation_direct(fks_ctx *ctx, int on);
/* The tolerance in force and, if counts != NULL, the cells sent to each tier
 * (counts[0]: first tier, counts[1]: second, including the cells a split-BF16
 * kernel listed for it directly) by the last collision or step call
 * (synchronous device read). */
fks_status fks_get_escalation(const fks_ctx *ctx, double *tol, long *counts);

/* Exact shift transport over time dt (Sec. 2.1): advances the generic-cell
 * particle offsets (FP64, s <- s + v dt, cell shift delta = floor((s + dx/2)/dx))
 * and writes f_out[j][k] = f[j - delta_k][k'] (k' = k mirrored along an axis
 * whose specular wall was crossed).  A permutation of the values: bit-exact.
 * f and f_out must not overlap. */
fks_status fks_transport(fks_ctx *ctx, const void *f, void *f_out, double dt, void *stream);

/* One FKS step (Sec. 2.1, Eq. disc_relax): transport over dt, then the
 * collision step f_out = f* + dt Q(f*) with the projected Q, fused in one
 * kernel per cell (f* never goes to memory).  f and f_out must not overlap. */
fks_status fks_step(fks_ctx *ctx, const void *f, void *f_out, double dt, void *stream);

/* The collision sub-step of Eq. disc_relax alone: f_out = f + dt Q(f) per
 * cell with the projected Q, no transport and no change to the offsets -- the
 * explicit Euler step of the space-homogeneous Boltzmann equation, cell by
 * cell (every cell an independent homogeneous problem).  Same kernels,
 * precisions and escalation as fks_step.  f and f_out must not overlap. */
fks_status fks_relax(fks_ctx *ctx, const void *f, void *f_out, double dt, void *stream);

/* A stiff step (Sec. 2.1 asks for care in the stiff limit): transport over
 * dt, then
 *  - BGK contexts: the exact solution of the BGK relaxation
 *    df/dt = nu (M[f*] - f) - phi.mu from f*, whose Maxwellian, rate nu = rho/Kn
 *    and projection term stay fixed over the step (the relaxation conserves
 *    rho, rho u, E):  f_out = f* + (1 - e^{-nu dt}) / nu * Q(f*);  equal to M[f*]
 *    (plus the projection correction) as Kn -> 0;
 *  - FP64 and FP32 spectral contexts: the integrating-factor (exponential Euler)
 *    step of the gain-loss split df/dt = G(f) - nu(v) f with the loss
 *    frequency nu = IDFT(betaL F) / Kn and G frozen at f*, solved per velocity
 *    point:  f_out = f* + dt P[phi(nu dt) (G - nu f*)], phi(x) = (1 - e^-x)/x, P the
 *    conservation projection of the increment; bounded for any nu dt (tends to
 *    G / nu in the stiff limit), with the FP32 context's escalation.
 * Both tend to fks_step as nu dt -> 0 (first order in dt).  dt >= 0.
 * FKS_ERR_UNSUPPORTED for split-BF16 and variant-B contexts.  f and f_out must
 * not overlap. */
fks_status fks_step_exp(fks_ctx *ctx, const void *f, void *f_out, double dt, void *stream);

/* A second-order step (the higher-order splitting the paper allows in Sec. 2.1):
 * Strang splitting T(dt/2) C(dt) T(dt/2) of transport T and collision C, the
 * collision sub-step integrated by Heun's method, the second-order explicit
 * Runge-Kutta counterpart of Eq. disc_relax:
 *   a = T(dt/2) f,  b = a + dt Q(a),  c = (a + b + dt Q(b)) / 2,  f_out = T(dt/2) c,
 * Q projected as in fks_collide.  Advances the offsets by dt (two half steps).
 * work: a caller-owned device array of the size of f (scratch; overwritten).
 * f, f_out and work must be distinct.  FKS_FP64 and FKS_FP32 spectral
 * contexts and BGK contexts; FKS_ERR_UNSUPPORTED for FKS_BF16X3 and
 * variant-B contexts. */
fks_status fks_step_strang(fks_ctx *ctx, const void *f, void *f_out, void *work, double dt, void *stream);

/* U[cell][0..4] = sum_k (1, vx, vy, vz, |v|^2/2) f[cell][k] dv^3 (Sec. 3),
 * accumulated in FP64 (FP64 states) or in compensated FP32 pairs with exact
 * products (FP32 states; as accurate as FP64 accumulation), returned in FP64.
 * U: device array of ncells * 5 doubles. */
fks_status fks_moments(fks_ctx *ctx, const void *f, double *U, void *stream);

/* Synchronises `stream`, reads and clears the health bits of the kernels
 * launched so far: bit 0 = non-finite value written, bit 1 = negative f
 * after a step, bit 2 = cell shift out of range, bit 3 = a bulk copy into
 * shared memory did not complete within its bounded wait.  Returns
 * FKS_ERR_NUMERIC for bits 0 and 2, FKS_ERR_TIMEOUT for bit 3, and stores the
 * bits in *bits if bits != NULL. */
fks_status fks_check(fks_ctx *ctx, void *stream, int *bits);

/* Stage timing for measurement: with on != 0 every collision launch of the
 * context is bracketed by two CUDA events on its stream, by stage (0 the
 * context's own kernel, 1 and 2 the escalation tiers).  fks_get_profile
 * synchronises the device and returns, per stage, the summed event time in
 * ms[3] and the number of launches in launches[3] (may be NULL), then clears
 * the record. */
fks_status fks_set_profiling(fks_ctx *ctx, int on);
fks_status fks_get_profile(fks_ctx *ctx, double *ms, long *launches);

/* Host copies of the per-axis sub-cell offsets s[3][n] (FP64).  get
 * synchronises the device; set is synchronous too. */
fks_status fks_get_offsets(fks_ctx *ctx, double *s);
fks_status fks_set_offsets(fks_ctx *ctx, const double *s);

/* Number of cells, velocity points per cell, and the thread-block cluster
 * size the collision kernel runs with. */
long fks_ncells(const fks_ctx *ctx);
int fks_nv(const fks_ctx *ctx);
int fks_cluster_size(const fks_ctx *ctx);

/* Override the cluster size (a divisor of n for which a kernel exists);
 * used by the autotuner.  Returns FKS_ERR_UNSUPPORTED if there is none. */
fks_status fks_set_cluster_size(fks_ctx *ctx, int C);
/* Cluster size and radix schedule together: radix = the top radix of the
 * length-n transforms (0 the default schedule 32 = 4 x 8, 24 = 3 x 8,
 * 16 = 4 x 4; FP32 kernels are also compiled with 2 and 8 at n = 32 and 16 and
 * with 2, 4, 8 at n = 24, at the default cluster size).  The result is the same
 * transform to rounding.  FKS_ERR_UNSUPPORTED for a combination not compiled. */
fks_status fks_set_schedule(fks_ctx *ctx, int C, int radix);
/* The radix schedule in use (0: default), -1 for a NULL context. */
int fks_radix(const fks_ctx *ctx);

/* Kernel launches enqueued by this context since creation (for accounting). */
long fks_launch_count(const fks_ctx *ctx);

/* Diagnostic: the kernel transforms phi_R(s) and psi_R(s) of Appendix A
 * (R = 2L/(3+sqrt 2)) evaluated on the host by the same code the table
 * kernel runs on the device.  Needs no GPU. */
fks_status fks_kernel_transform(int ktype, double C, double L, double s, double *phi, double *psi);

/* Diagnostic: the radial factor H(t, u) of one direction of the FKS_VHS kernel
 * (alpha, C, box [-L, L]^3 with n^3 points) as the library's expansion gives
 * it: sum over the separable terms of phi_s(t) psi_s(u), where the exact factor is
 *   H(t, u) = int_0^R int_0^R 2r cos(rt) B~(r, r') 2 pi r' J0(r'u) dr dr',
 * R = 2L/(3 + sqrt 2) (Appendix A).  Returns the term count in *S and the
 * truncation error estimate (max over the check grid, relative) in *trunc_err
 * (either may be NULL).  precision selects the automatic tolerance; terms as in
 * fks_kernel.  Runs on the host; needs no GPU. */
fks_status fks_vhs_factor(double alpha, double C, double L, int n, int precision, int terms, double t, double u,
                          double *H, int *S, double *trunc_err);

/* ---------------------------------------------------------------- batches
 * Independent space-homogeneous problems (one cell each, no transport) of
 * uneven size: problem i has n[i]^3 velocities on [-L[i], L[i]]^3, kernel
 * ktype[i] with constant C[i], Knudsen number knudsen[i]; all share the
 * direction set.  Problems of one n form a class run by one persistent
 * launch over per-problem descriptors (the spectral operator of Appendix A,
 * the FP64 projection and, for steps, the Euler update of Eq. disc_relax);
 * the classes run concurrently.  Arrays of problem pointers are HOST arrays
 * of nprob DEVICE pointers (n[i]^3 elements each, distinct, 16-byte
 * aligned).  Descriptors are cached per pointer set (the first call with a
 * new set uploads them synchronously). */
typedef struct fks_batch fks_batch;

fks_status fks_batch_init(int nprob, const int *n, const double *L, const int *ktype, const double *C,
                          const double *knudsen, const fks_dirs *dirs, int precision, fks_batch **out);

/* Q[i] = projected Q(f[i]) / Kn_i for every problem. */
fks_status fks_batch_collide(fks_batch *b, const void *const *f, void *const *Q, void *stream);

/* f_out[i] = f[i] + dt[i] Q(f[i]) for every problem (dt: host array). */
fks_status fks_batch_step(fks_batch *b, const void *const *f, void *const *f_out, const double *dt, void *stream);

/* nsteps steps alternating fa -> fb -> fa ...: captured once per (fa, fb,
 * dt, nsteps) into a CUDA graph and replayed on `stream`.  The result is in
 * fb if nsteps is odd, else in fa. */
fks_status fks_batch_run(fks_batch *b, void *const *fa, void *const *fb, const double *dt, int nsteps, void *stream);

/* As fks_check, for the batch kernels. */
fks_status fks_batch_check(fks_batch *b, void *stream, int *bits);

/* Precision escalation of FP32 batches, as fks_set_escalation: a problem whose
 * error bound 5e-7 ||L|| / Kn exceeds tol ||Q|| is recomputed in double-float
 * arithmetic over its FP32 arrays by a second persistent launch of its class
 * (device-side list and count: graph-capturable).  Default tol 1e-5; 0: off.
 * FKS_ERR_UNSUPPORTED for a positive tol on FP64 batches.  Drops the captured
 * graphs; synchronises the device. */
fks_status fks_batch_set_escalation(fks_batch *b, double tol);
/* The tolerance and, if count != NULL, the problems escalated by the last
 * launch (synchronous device read). */
fks_status fks_batch_get_escalation(const fks_batch *b, double *tol, long *count);

/* Cluster size used for the class of velocity grid n (-1 if none); the
 * setter rebuilds that class's tables (used by the autotuner). */
int fks_batch_cluster_size(const fks_batch *b, int n);
fks_status fks_batch_set_cluster_size(fks_batch *b, int n, int C);
/* cluster size and radix schedule of class n together (as fks_set_schedule); the radix in use */
fks_status fks_batch_set_schedule(fks_batch *b, int n, int C, int radix);
int fks_batch_radix(const fks_batch *b, int n);
long fks_batch_launch_count(const fks_batch *b);
void fks_batch_destroy(fks_batch *b);
const char *fks_batch_last_error(const fks_batch *b);

/* ---------------------------------------------------------------- learned surrogate
 * A convolutional surrogate of the collision operator for cells near
 * equilibrium (an extension, not in the paper): six 3x3x3 convolutions over
 * the n^3 velocity grid, channels 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU
 * between layers, zero padding, BF16 weights and FP32 accumulation.  Inputs
 * per cell: f / rho and M[f] / rho; output y ~ Q Kn / (rho^2 out_scale).  The
 * parameters are one flat FP32 master vector: per layer W[co][ci][27] (tap
 * (dx+1)*9 + (dy+1)*3 + (dz+1)) then bias[co].  n must be a multiple of 8.
 * The network owns its activations for batches of up to max_batch cells. */
typedef struct fks_net fks_net;

fks_status fks_net_init(int n, int max_batch, unsigned long long seed, fks_net **out);
long fks_net_num_params(const fks_net *net);
/* host copies of the FP32 master parameters (count = fks_net_num_params) */
fks_status fks_net_set_params(fks_net *net, const float *host, long count);
fks_status fks_net_get_params(fks_net *net, float *host, long count);
/* y[b][n^3] = net(x[b][2][n^3]) for b < batch (device arrays) */
fks_status fks_net_forward(fks_net *net, int batch, const float *x, float *y, void *stream);
/* inference on the tensor cores (n a multiple of 16): the same network with
 * BF16 activations between layers (inputs rounded to BF16), BF16 weights and
 * FP32 accumulation in tensor memory; y FP32.  Used by fks_surrogate_collide,
 * which calls it on chunks of up to max(max_batch, 304) cells (its own
 * workspace, allocated on first use); here batch <= max_batch. */
fks_status fks_net_infer(fks_net *net, int batch, const float *x, float *y, void *stream);
/* synchronises `stream`; FKS_ERR_TIMEOUT if a tensor-core completion wait of
 * an inference kernel ran out (bounded wait), FKS_OK otherwise */
fks_status fks_net_check(fks_net *net, void *stream);
/* grad (device, num_params floats) = d(sum gy * y)/d params, through the BF16
 * weights (the rounding is treated as the identity) */
fks_status fks_net_gradient(fks_net *net, int batch, const float *x, const float *gy, float *grad, void *stream);
/* one Adam step on the mean squared error against target; *loss (device
 * float) is incremented by the batch's loss */
fks_status fks_net_train_step(fks_net *net, int batch, const float *x, const float *target, float lr, float *loss,
                              void *stream);
long fks_net_launch_count(const fks_net *net);
const char *fks_net_last_error(const fks_net *net);
void fks_net_destroy(fks_net *net);

/* Network inputs of ncells FP32 cells: x[c] = (f/rho, M[f]/rho), rho[c]
 * (FP64) and dist[c] = ||f/rho - M/rho|| / ||M/rho|| (device arrays; f and x
 * 16-byte aligned).  n a multiple of 4, at most 64, else FKS_ERR_INVALID_ARG.
 * The moments behind rho, u, T are FP32 partial sums added in FP64. */
fks_status fks_surrogate_inputs(int n, double L, long ncells, const float *f, float *x, double *rho, float *dist,
                                void *stream);

/* Q for every cell of an FP32 or split-BF16 (FKS_BF16X3) spectral context
 * (variant A) by the surrogate: Q = rho^2 y out_scale / Kn, projected onto
 * the conservation constraints; indicator = ind_scale / dist + the relative
 * moment defect of the raw output (the network's error is about a fixed
 * fraction of its output scale while ||Q|| shrinks with dist, so its
 * relative error grows as 1 / dist).  Cells whose bound ind_scale / dist
 * already exceeds `threshold` skip the network; the others are inferred in
 * compacted chunks.  Cells whose indicator exceeds `threshold` (or is not
 * finite) are recomputed with the context's spectral operator (the FP32
 * cluster kernel or the split-BF16 tensor-core kernel over a device list of
 * the routed cells, each with the context's precision escalation).
 * Synchronises `stream` once to read the candidate count, and once more if
 * nrouted != NULL (the routed count).  f and Q 16-byte aligned.  The moments of the raw
 * output are FP64 sums of its FP32 values; the correction is applied in FP32. */
fks_status fks_surrogate_collide(fks_ctx *ctx, fks_net *net, const void *f, void *Q, double out_scale,
                                 double ind_scale, double threshold, long *nrouted, void *stream);
/* One FKS step with the surrogate: transport over dt into `work` (a device
 * array of the size of f, overwritten: f*), then f_out = f* + dt Q with Q as in
 * fks_surrogate_collide (the routed cells by the spectral step without
 * transport).  f, f_out and work distinct and 16-byte aligned. */
fks_status fks_surrogate_step(fks_ctx *ctx, fks_net *net, const void *f, void *f_out, void *work, double dt,
                              double out_scale, double ind_scale, double threshold, long *nrouted, void *stream);
/* host copy of the last indicators (count = number of cells) */
fks_status fks_surrogate_indicator(const fks_ctx *ctx, float *host, long count);

/* fks_step with HOST arrays (f -> f_out, ncells * n^3 elements each, distinct):
 * the state is copied to device buffers owned by the context, stepped and
 * copied back, pipelined over chunks of x-slabs: the host-to-device copies of
 * later chunks, the step of a chunk (once every slab its transport shift can
 * reach, at most floor(L |dt| / dx) + 1 slabs away, has landed) and the
 * device-to-host copies of earlier chunks overlap on internal copy streams.
 * Spectral FP32/FP64 and BGK contexts use up to 8 chunks; split-BF16 and
 * variant-B contexts one.  Same values as fks_step on device copies.  Returns
 * after queueing; the output is complete when `stream` is.  The host arrays
 * should be page-locked for the copies to overlap; they must not be touched
 * before `stream` completes.  Allocates two device copies of the state on
 * first use. */
fks_status fks_step_host(fks_ctx *ctx, const void *host_f, void *host_out, double dt, void *stream);

/* Variant B (de-aliased operator), Appendix A Eq. CF1 with l + m = k over the
 * modes l, m in [-n/2, n/2]^3, not reduced mod n, evaluated with transforms of
 * size 2n as in Sec. 5 (2n^3 transforms for n^3 modes).  on != 0: from then on
 * fks_collide and fks_step of this context interpolate f* (the trigonometric
 * interpolant; a Nyquist coefficient split between +-n/2) onto the 2n grid
 * of the same box, run the operator there without projection, keep the modes
 * |k| <= n/2 (+-n/2 folded back onto the Nyquist index) on the n grid and
 * project.  Needs a spectral FP32 or FP64 context with n = 8 or 16, else
 * FKS_ERR_UNSUPPORTED.  Allocates an inner context of the 2n grid and two
 * chunk buffers of up to 2048 cells x (2n)^3 values.  on = 0 releases them. */
fks_status fks_set_dealias(fks_ctx *ctx, int on);

/* Self-test of the failure detection of the kernels' waits (no GPU fault):
 * one thread waits, with the bounded-wait helper of the collision kernels
 * (bulk-copy and tensor-core completions), on an mbarrier that nothing
 * arrives at; after `polls` polls (1 .. 2^26) it records the timeout bit and
 * returns.  Synchronises `stream`.  Returns FKS_ERR_TIMEOUT (the expected
 * result), FKS_ERR_INVALID_ARG for polls out of range, FKS_ERR_CUDA or
 * FKS_ERR_OOM on a CUDA failure.  The device stays usable. */
fks_status fks_selftest_wait(long polls, void *stream);

/* Measurement helper: the device's FMA throughput in TFLOP/s (2 flop per FMA)
 * for precision FKS_FP32 (the FP32 pipe) or FKS_FP64 (the FP64 pipe), from a
 * kernel of independent FMA chains (8 per thread, 8 CTAs of 256 threads per
 * SM), timed with CUDA events after one warm-up launch.  Synchronises
 * `stream`.  The roofline denominator of the CUDA-core collision kernels. */
fks_status fks_alu_peak(int precision, double *tflops, void *stream);

/* fks_transport_noalloc -- the transport of fks_transport for callers that
 * cannot allocate device memory.  It is an addition of this library; the
 * paper has no counterpart.
 *
 * Some callers must not call cudaMalloc: applications whose device memory
 * is owned entirely by their own pool allocator, plugins that may not grow
 * the device footprint of the host program, and loops where the implicit
 * device synchronisation of cudaMalloc would stall an asynchronous pipeline.
 * fks_init allocates (tables, offsets, flags), so such callers cannot use a
 * context; this entry point needs none and allocates nothing.
 *
 * It advances the particle offsets s (a DEVICE array of 3*n doubles owned by
 * the caller, read and updated in place; start from zeros) by dt and writes
 * f_out[j][k] = f[j - delta_k][k'] exactly as fks_transport does (same
 * kernels, bit-identical results).  f, f_out: device arrays of
 * nx*ny*nz*n^3 elements (double for FKS_FP64, float for FKS_FP32), distinct.
 *
 * Scratch: the per-call table of cell shifts and a flag word live in one
 * file-scope __device__ array of 256 bytes, which every GPU that loads this
 * library holds until the process exits.  Limit: n <= 32 (larger n returns
 * FKS_ERR_UNSUPPORTED before any work); n must be even.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.
 * Every call shares the array and overwrites it (the flag word is cleared at
 * the start of each call), so calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race: serialise them.
 * The call synchronises `stream` at its end to read the flag word: it returns
 * FKS_ERR_NUMERIC if a cell shift left the range of the shift table
 * (|delta| > 120), which the check |L dt| <= 100 dx rules out for offsets in
 * [-dx/2, dx/2) and so signals a corrupted s (f_out then holds an in-range
 * but wrong permutation).  Returns FKS_ERR_INVALID_ARG for bad arguments,
 * FKS_ERR_CUDA if a CUDA call fails.  It calls no cudaMalloc, cudaFree or
 * allocating routine. */
fks_status fks_transport_noalloc(const fks_grid *grid, const fks_vbox *vbox, int precision, double *s,
                                 double dt, const void *f, void *f_out, void *stream);

void fks_destroy(fks_ctx *ctx);
const char *fks_last_error(const fks_ctx *ctx);
const char *fks_status_string(fks_status s);

#ifdef __cplusplus
}
#endif

#endif /* FKS_H */
