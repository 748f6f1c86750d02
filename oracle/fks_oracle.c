/*
 * fks_oracle.c -- plain, slow FP64 CPU reference of the Fast Kinetic Scheme
 * hot path (Narski, "Fast Kinetic Scheme: efficient MPI parallelization
 * strategy for 3D Boltzmann equation", arXiv 1701.01608).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * it exists so that the CUDA library can be checked against an independent
 * statement of the method.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every routine follows the paper's formulas in the order the paper states
 * them, with no blocking, fusion or reordering:
 *   - velocity moments U = sum_k phi(v_k) m_k dv^3                (Sec. 3, moments sum)
 *   - exact shift transport of the generic-cell particles          (Sec. 2.1 "Transport step", Sec. 3)
 *   - explicit Euler collision step  f = f* + dt Q(f*)             (Eq. disc_relax)
 *   - fast spectral operator: Fourier coefficients, Carleman form,
 *     separable kernel, quadrature over half-sphere directions     (Appendix A)
 *   - the O(N_v^2) Galerkin sum  Q^_k = sum_{l+m=k} beta_F(l,m) f^_l f^_m
 *     used as a brute-force check of the fast algorithm           (Appendix A, Eq. CF1)
 *
 * Readings of the paper (where it is garbled or silent) are listed in the
 * repository's design notes; the ones that change arithmetic are restated at
 * the routine that uses them.
 *
 * Parity status of every exported function: pinned by tests/test_oracle_*.py
 * (FFT against numpy.fft, kernel transforms against scipy quadrature and
 * scipy.special.j1, Galerkin identity, conservation, Q(M)=0, closed-form
 * loss frequency of a Maxwellian, BKW shape, transport permutation; the
 * variable-hard-sphere operator against scipy's double quadrature, the hard-
 * sphere operator at alpha = 1, the closed-form loss frequency of a
 * Maxwellian for every alpha and BKW for Maxwell molecules).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double OR_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* velocity grid: n cell-centred points on [-L, L]                     */
/* ------------------------------------------------------------------ */

/* v_i = (i + 1/2 - n/2) * dv, dv = 2L/n.  Written as a half-integer times dv
 * so that v_{n-1-i} = -v_i holds exactly in floating point. */
void or_vgrid(int n, double L, double *v)
{
    double dv = 2.0 * L / n;
    for (int i = 0; i < n; ++i)
        v[i] = ((double)i + 0.5 - 0.5 * n) * dv;
}

/* ------------------------------------------------------------------ */
/* FFT (own implementation)                                             */
/* ------------------------------------------------------------------ */

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place 1-D DFT  X_k = sum_j x_j exp(sign * 2 pi i j k / n), unnormalised.
 * Power-of-two n: iterative radix-2 decimation in time.  Other n: the direct
 * O(n^2) sum. */
void or_fft1d(cplx *x, int n, int sign)
{
    if (n <= 1) return;
    if (!is_pow2(n)) {
        cplx *y = (cplx *)malloc(sizeof(cplx) * n);
        for (int k = 0; k < n; ++k) {
            cplx s = 0;
            for (int j = 0; j < n; ++j) {
                long jk = ((long)j * k) % n;
                double ang = sign * 2.0 * OR_PI * (double)jk / n;
                s += x[j] * (cos(ang) + I * sin(ang));
            }
            y[k] = s;
        }
        memcpy(x, y, sizeof(cplx) * n);
        free(y);
        return;
    }
    /* bit reversal */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < len / 2; ++k) {
                double ang = sign * 2.0 * OR_PI * k / len;
                cplx w = cos(ang) + I * sin(ang);
                cplx u = x[i + k];
                cplx t = w * x[i + k + len / 2];
                x[i + k] = u + t;
                x[i + k + len / 2] = u - t;
            }
        }
    }
}

/* In-place 3-D DFT of a[(i*n + j)*n + k], one axis after the other. */
void or_fft3d(cplx *a, int n, int sign)
{
    cplx *p = (cplx *)malloc(sizeof(cplx) * n);
    for (int axis = 0; axis < 3; ++axis) {
        long stride = axis == 0 ? (long)n * n : (axis == 1 ? n : 1);
        for (int u = 0; u < n; ++u)
            for (int w = 0; w < n; ++w) {
                long base;
                if (axis == 0) base = (long)u * n + w;
                else if (axis == 1) base = (long)u * n * n + w;
                else base = ((long)u * n + w) * n;
                for (int t = 0; t < n; ++t) p[t] = a[base + t * stride];
                or_fft1d(p, n, sign);
                for (int t = 0; t < n; ++t) a[base + t * stride] = p[t];
            }
    }
    free(p);
}

/* Python-friendly wrapper: interleaved (re, im) doubles. */
void or_fft3d_ri(double *ri, int n, int sign)
{
    or_fft3d((cplx *)ri, n, sign);
}

void or_fft1d_ri(double *ri, int n, int sign)
{
    or_fft1d((cplx *)ri, n, sign);
}

/* ------------------------------------------------------------------ */
/* collision directions and weights (Appendix A, quadrature over e)     */
/* ------------------------------------------------------------------ */

/* Half-sphere directions e_{pq} = (sin t cos f, sin t sin f, cos t),
 * f_q = q pi / A2 (q = 0..A2-1), with
 *   rule 0: t_p = (p + 1/2) pi / A1   (midpoint rule, every weight > 0)
 *   rule 1: t_p = p pi / A1           (angles as printed)
 * and weight w_pq = pi^2 / (A1 A2) * sin t_p, the surface element of the
 * half sphere.  Returns M = A1*A2.  Order: p major, q minor. */
int or_directions(int A1, int A2, int rule, double *e, double *w)
{
    int M = 0;
    for (int p = 0; p < A1; ++p) {
        double t = (rule == 0 ? (p + 0.5) : (double)p) * OR_PI / A1;
        for (int q = 0; q < A2; ++q) {
            double f = q * OR_PI / A2;
            e[3 * M + 0] = sin(t) * cos(f);
            e[3 * M + 1] = sin(t) * sin(f);
            e[3 * M + 2] = cos(t);
            w[M] = OR_PI * OR_PI / ((double)A1 * A2) * sin(t);
            ++M;
        }
    }
    return M;
}

/* ------------------------------------------------------------------ */
/* kernel transforms phi_R and psi_R (Appendix A)                       */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on the
 * three-term recurrence of P_m. */
static void gauss_legendre(int m, double *x, double *w)
{
    for (int i = 0; i < m; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            /* p1 = P_m(z), p0 = P_{m-1}(z) */
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* 64-point rule, computed once (or_tables fills it before its parallel loop) */
enum { NGL = 64 };
static double GLX[NGL], GLW[NGL];
static int gl_ready = 0;
static void gl_init(void)
{
    if (!gl_ready) { gauss_legendre(NGL, GLX, GLW); gl_ready = 1; }
}

/* Bessel function J_nu(x), integer nu, from Bessel's integral
 *   J_nu(x) = (1/pi) int_0^pi cos(nu t - x sin t) dt,
 * by the trapezoidal rule, which is spectrally accurate for this periodic
 * integrand.  For nu = 0 the integrand is symmetric about pi/2 and the rule
 * is taken on [0, pi/2]. */
static double bessel_j(int nu, double x)
{
    int K = 40 + (int)fabs(x);
    if (nu == 0) {
        double s = 0.5 * (1.0 + cos(x));
        for (int j = 1; j < K; ++j) s += cos(x * sin(0.5 * OR_PI * j / K));
        return s / K;
    }
    K *= 2;
    double s = 0.5 * (cos(0.0) + cos(nu * OR_PI - x * sin(OR_PI)));
    for (int j = 1; j < K; ++j) {
        double t = j * OR_PI / K;
        s += cos(nu * t - x * sin(t));
    }
    return s / K;
}

double or_bessel_j(int nu, double x) { return bessel_j(nu, x); }

/* Kernel type 0 (hard spheres): B~ = 4C, i.e. a(r) = b(r) = sqrt(4C).
 * Kernel type 1 (pseudo-Maxwell): B~ = 4C (|x||y|)^{-1/2},
 *                                 a(r) = b(r) = sqrt(4C) r^{-1/2}.
 *
 * phi_R(s) = int_{-R}^{R} |rho| a(|rho|) exp(i rho s) d rho
 *          = 2 int_0^R rho a(rho) cos(rho s) d rho.
 * (The printed integrand "rho" is read as |rho|: it comes from dx = rho^2
 *  d rho de together with delta(rho e.y) = delta(e.y)/|rho|.) */
double or_phi(int ktype, double C, double R, double s)
{
    double c = sqrt(4.0 * C);
    s = fabs(s);
    if (ktype == 0) {
        if (s * R < 1e-4) {
            double x2 = (R * s) * (R * s);
            return c * R * R * (1.0 - x2 / 4.0 + x2 * x2 / 72.0);
        }
        double sh = sin(0.5 * R * s);
        return c * 2.0 * (R * sin(R * s) / s - 2.0 * sh * sh / (s * s));
    }
    /* pseudo-Maxwell: rho = u^2, d rho = 2u du,
     * 2 int_0^R sqrt(rho) cos(rho s) d rho = 4 int_0^sqrt(R) u^2 cos(u^2 s) du */
    gl_init();
    double U = sqrt(R), acc = 0.0;
    for (int i = 0; i < NGL; ++i) {
        double u = 0.5 * U * (GLX[i] + 1.0);
        acc += 0.5 * U * GLW[i] * u * u * cos(u * u * s);
    }
    return c * 4.0 * acc;
}

/* psi_R(s) = int over the disc |y| <= R in a plane, of b(|y|) exp(i s y_1) dy
 *          = 2 pi int_0^R r b(r) J_0(r s) dr.
 * Hard spheres: 2 pi R J_1(R s) / s (J_1 from Bessel's integral).
 * Pseudo-Maxwell: r = u^2, 2 pi sqrt(4C) * 2 int_0^sqrt(R) u^2 J_0(u^2 s) du. */
double or_psi(int ktype, double C, double R, double s)
{
    double c = sqrt(4.0 * C);
    s = fabs(s);
    if (ktype == 0) {
        double x = R * s;
        if (x < 1e-3) {
            double x2 = x * x;
            return c * OR_PI * R * R * (1.0 - x2 / 8.0 + x2 * x2 / 192.0);
        }
        return c * 2.0 * OR_PI * R * bessel_j(1, x) / s;
    }
    gl_init();
    double U = sqrt(R), acc = 0.0;
    for (int i = 0; i < NGL; ++i) {
        double u = 0.5 * U * (GLX[i] + 1.0);
        acc += 0.5 * U * GLW[i] * u * u * bessel_j(0, u * u * s);
    }
    return c * 2.0 * OR_PI * 2.0 * acc;
}

/* ------------------------------------------------------------------ */
/* spectral tables                                                      */
/* ------------------------------------------------------------------ */

/* signed frequency of DFT index k: k for k < n/2, k - n otherwise */
static int kappa(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

/* Tables on the standard DFT index grid k = (kx*n + ky)*n + kz:
 *   alpha [p][k] = phi_R( xi_k . e_p )
 *   alphap[p][k] = psi_R( |xi_k - (xi_k . e_p) e_p| )
 *   betaL [k]    = sum_p w_p alpha[p][k] alphap[p][k]       (the B_F(m,m) term)
 * with xi_k = (pi/L) kappa(k) and cut-off R = lam L, lam = 2/(3+sqrt 2)
 * (Appendix A: T = pi, R = lam pi, rescaled to the box [-L, L]).
 *
 * Reading of the inclusive sum k = -N/2..N/2: for even n a Nyquist component
 * (kappa = -n/2) stands for both +n/2 and -n/2 with half weight each, so
 * every table value is the mean over the sign choices of its Nyquist
 * components.  This makes the tables Hermitian-even, the gain factors real
 * and the discrete mass exactly conserved.
 *
 * Returns M. */
int or_tables(int n, double L, int ktype, double C, int A1, int A2, int rule,
              double *alpha, double *alphap, double *betaL, double *w)
{
    int M = A1 * A2;
    double *e = (double *)malloc(sizeof(double) * 3 * M);
    or_directions(A1, A2, rule, e, w);
    double lam = 2.0 / (3.0 + sqrt(2.0));
    double R = lam * L;
    double h = OR_PI / L;
    long n3 = (long)n * n * n;
    int nyq = (n % 2 == 0) ? n / 2 : -1;
    gl_init();

#pragma omp parallel for schedule(dynamic)
    for (long idx = 0; idx < (long)M * n3; ++idx) {
        int p = (int)(idx / n3);
        long k = idx % n3;
        int kk[3] = {(int)(k / ((long)n * n)), (int)((k / n) % n), (int)(k % n)};
        int nflip = 0, fl[3];
        for (int a = 0; a < 3; ++a) if (kk[a] == nyq) fl[nflip++] = a;
        double sa = 0.0, sb = 0.0;
        int ncomb = 1 << nflip;
        for (int c = 0; c < ncomb; ++c) {
            double xi[3];
            for (int a = 0; a < 3; ++a) xi[a] = h * kappa(kk[a], n);
            for (int b = 0; b < nflip; ++b)
                if (c & (1 << b)) xi[fl[b]] = -xi[fl[b]];
            double de = xi[0] * e[3 * p] + xi[1] * e[3 * p + 1] + xi[2] * e[3 * p + 2];
            double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] - de * de;
            double sp = sqrt(q2 > 0 ? q2 : 0.0);
            sa += or_phi(ktype, C, R, de);
            sb += or_psi(ktype, C, R, sp);
        }
        alpha[(long)p * n3 + k] = sa / ncomb;
        alphap[(long)p * n3 + k] = sb / ncomb;
    }
    for (long k = 0; k < n3; ++k) {
        double s = 0.0;
        for (int p = 0; p < M; ++p) s += w[p] * alpha[(long)p * n3 + k] * alphap[(long)p * n3 + k];
        betaL[k] = s;
    }
    free(e);
    return M;
}

/* ------------------------------------------------------------------ */
/* conservation projection                                              */
/* ------------------------------------------------------------------ */

/* Q <- Q - C^T (C C^T)^{-1} C Q, rows of C: dv^3 phi_i(v_k),
 * phi = (1, vx, vy, vz, |v|^2/2).  Gaussian elimination with partial
 * pivoting on the 5x5 Gram system. */
void or_project(int n, double L, double *Q)
{
    double v[64], dv = 2.0 * L / n, dv3 = dv * dv * dv;
    or_vgrid(n, L, v);
    double A[5][6];
    memset(A, 0, sizeof(A));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double ph[5] = {1.0, v[i], v[j], v[k], 0.5 * (v[i] * v[i] + v[j] * v[j] + v[k] * v[k])};
                double q = Q[((long)i * n + j) * n + k];
                for (int a = 0; a < 5; ++a) {
                    for (int b = 0; b < 5; ++b) A[a][b] += dv3 * ph[a] * dv3 * ph[b];
                    A[a][5] += dv3 * ph[a] * q;
                }
            }
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c) for (int t = 0; t < 6; ++t) { double x = A[c][t]; A[c][t] = A[piv][t]; A[piv][t] = x; }
        for (int r = 0; r < 5; ++r) {
            if (r == c) continue;
            double fct = A[r][c] / A[c][c];
            for (int t = c; t < 6; ++t) A[r][t] -= fct * A[c][t];
        }
    }
    double lam[5];
    for (int a = 0; a < 5; ++a) lam[a] = A[a][5] / A[a][a];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double ph[5] = {1.0, v[i], v[j], v[k], 0.5 * (v[i] * v[i] + v[j] * v[j] + v[k] * v[k])};
                double corr = 0.0;
                for (int a = 0; a < 5; ++a) corr += lam[a] * dv3 * ph[a];
                Q[((long)i * n + j) * n + k] -= corr;
            }
}

/* ------------------------------------------------------------------ */
/* fast spectral collision operator, one cell at a time (Appendix A)    */
/* ------------------------------------------------------------------ */

/* For each cell:
 *   F = DFT(f)
 *   G = sum_p w_p * a_p * b_p,  a_p = IDFT(alpha_p F)/n^3, b_p = IDFT(alphap_p F)/n^3
 *   L = f * IDFT(betaL F)/n^3
 *   Q = (G - L) * inv_kn, then the conservation projection if project != 0.
 * f, Q: ncells * n^3, cell-major, velocity index (ix*n + iy)*n + iz. */
void or_collide(int n, double L, int M, const double *alpha, const double *alphap,
                const double *w, const double *betaL, double inv_kn, int project,
                long ncells, const double *f, double *Q)
{
    long n3 = (long)n * n * n;
#pragma omp parallel
    {
        cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
        cplx *A = (cplx *)malloc(sizeof(cplx) * n3);
        cplx *B = (cplx *)malloc(sizeof(cplx) * n3);
        double *G = (double *)malloc(sizeof(double) * n3);
#pragma omp for schedule(dynamic)
        for (long c = 0; c < ncells; ++c) {
            const double *fc = f + c * n3;
            double *Qc = Q + c * n3;
            for (long k = 0; k < n3; ++k) F[k] = fc[k];
            or_fft3d(F, n, -1);
            for (long k = 0; k < n3; ++k) G[k] = 0.0;
            for (int p = 0; p < M; ++p) {
                for (long k = 0; k < n3; ++k) {
                    A[k] = alpha[p * n3 + k] * F[k];
                    B[k] = alphap[p * n3 + k] * F[k];
                }
                or_fft3d(A, n, +1);
                or_fft3d(B, n, +1);
                for (long k = 0; k < n3; ++k)
                    G[k] += w[p] * (creal(A[k]) / n3) * (creal(B[k]) / n3);
            }
            for (long k = 0; k < n3; ++k) A[k] = betaL[k] * F[k];
            or_fft3d(A, n, +1);
            for (long k = 0; k < n3; ++k)
                Qc[k] = (G[k] - fc[k] * creal(A[k]) / n3) * inv_kn;
            if (project) or_project(n, L, Qc);
        }
        free(F); free(A); free(B); free(G);
    }
}

/* Gain and loss separately (no projection, no 1/Kn), for diagnostics. */
void or_gain_loss(int n, int M, const double *alpha, const double *alphap,
                  const double *w, const double *betaL, const double *f,
                  double *G, double *Lo)
{
    long n3 = (long)n * n * n;
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
    cplx *A = (cplx *)malloc(sizeof(cplx) * n3);
    cplx *B = (cplx *)malloc(sizeof(cplx) * n3);
    for (long k = 0; k < n3; ++k) F[k] = f[k];
    or_fft3d(F, n, -1);
    for (long k = 0; k < n3; ++k) G[k] = 0.0;
    for (int p = 0; p < M; ++p) {
        for (long k = 0; k < n3; ++k) {
            A[k] = alpha[p * n3 + k] * F[k];
            B[k] = alphap[p * n3 + k] * F[k];
        }
        or_fft3d(A, n, +1);
        or_fft3d(B, n, +1);
        for (long k = 0; k < n3; ++k) G[k] += w[p] * (creal(A[k]) / n3) * (creal(B[k]) / n3);
    }
    for (long k = 0; k < n3; ++k) A[k] = betaL[k] * F[k];
    or_fft3d(A, n, +1);
    for (long k = 0; k < n3; ++k) Lo[k] = f[k] * creal(A[k]) / n3;
    free(F); free(A); free(B);
}

/* ------------------------------------------------------------------ */
/* brute-force Galerkin sum (Appendix A, Eq. CF1)                        */
/* ------------------------------------------------------------------ */

/* Q^_k = n^-3 sum_{l+m = k (mod n)} [beta(l,m) - beta(m,m)] F_l F_m,
 * beta(l,m) = sum_p w_p alpha_p(l) alphap_p(m), F = DFT(f) by the direct
 * O(n^6) sum, Q = IDFT(Q^)/n^3 by the direct sum, times inv_kn.
 * Cost O(n^6 (M + 1)): for n <= 8 only. */
void or_galerkin(int n, int M, const double *alpha, const double *alphap,
                 const double *w, const double *f, double inv_kn, double *Q)
{
    long n3 = (long)n * n * n;
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
    cplx *Qh = (cplx *)malloc(sizeof(cplx) * n3);
    for (long k = 0; k < n3; ++k) {
        int kx = (int)(k / (n * n)), ky = (int)((k / n) % n), kz = (int)(k % n);
        cplx s = 0;
        for (long j = 0; j < n3; ++j) {
            int jx = (int)(j / (n * n)), jy = (int)((j / n) % n), jz = (int)(j % n);
            double ang = -2.0 * OR_PI * (double)(kx * jx + ky * jy + kz * jz) / n;
            s += f[j] * (cos(ang) + I * sin(ang));
        }
        F[k] = s;
        Qh[k] = 0;
    }
    for (long l = 0; l < n3; ++l) {
        int lx = (int)(l / (n * n)), ly = (int)((l / n) % n), lz = (int)(l % n);
        for (long m = 0; m < n3; ++m) {
            int mx = (int)(m / (n * n)), my = (int)((m / n) % n), mz = (int)(m % n);
            double bl = 0.0, bm = 0.0;
            for (int p = 0; p < M; ++p) {
                bl += w[p] * alpha[p * n3 + l] * alphap[p * n3 + m];
                bm += w[p] * alpha[p * n3 + m] * alphap[p * n3 + m];
            }
            long k = (((long)((lx + mx) % n) * n) + (ly + my) % n) * n + (lz + mz) % n;
            Qh[k] += (bl - bm) * F[l] * F[m];
        }
    }
    for (long j = 0; j < n3; ++j) {
        int jx = (int)(j / (n * n)), jy = (int)((j / n) % n), jz = (int)(j % n);
        cplx s = 0;
        for (long k = 0; k < n3; ++k) {
            int kx = (int)(k / (n * n)), ky = (int)((k / n) % n), kz = (int)(k % n);
            double ang = 2.0 * OR_PI * (double)(kx * jx + ky * jy + kz * jz) / n;
            s += Qh[k] * (cos(ang) + I * sin(ang));
        }
        Q[j] = creal(s) / ((double)n3 * n3) * inv_kn;
    }
    free(F); free(Qh);
}

/* ------------------------------------------------------------------ */
/* moments (Sec. 3)                                                     */
/* ------------------------------------------------------------------ */

/* U[c] = sum_k phi(v_k) f[c][k] dv^3, phi = (1, vx, vy, vz, |v|^2/2). */
void or_moments(int n, double L, long ncells, const double *f, double *U)
{
    double v[64], dv = 2.0 * L / n, dv3 = dv * dv * dv;
    or_vgrid(n, L, v);
    long n3 = (long)n * n * n;
    for (long c = 0; c < ncells; ++c) {
        double u[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double m = f[c * n3 + ((long)i * n + j) * n + k] * dv3;
                    u[0] += m;
                    u[1] += m * v[i];
                    u[2] += m * v[j];
                    u[3] += m * v[k];
                    u[4] += m * 0.5 * (v[i] * v[i] + v[j] * v[j] + v[k] * v[k]);
                }
        for (int a = 0; a < 5; ++a) U[5 * c + a] = u[a];
    }
}

/* ------------------------------------------------------------------ */
/* transport (Sec. 2.1 "Transport step", Sec. 3 particle interpretation) */
/* ------------------------------------------------------------------ */

/* Advance the generic-cell particle offsets along one axis and return the
 * integer cell shifts.  Offsets s are measured from the cell centre, cell
 * membership is the half-open interval [-dx/2, dx/2):
 *   s <- s + v dt;  delta = floor((s + dx/2)/dx);  s <- s - delta dx.
 * The offset of -v is kept the exact mirror of the offset of +v (it is
 * computed from +v and negated), so that the specular wall rule below stays
 * a bijection even at ties. */
void or_offsets(int n, double L, double dx, double dt, double *s, int *delta)
{
    double v[64];
    or_vgrid(n, L, v);
    for (int i = n / 2; i < n; ++i) {
        double sn = s[i] + v[i] * dt;
        double d = floor((sn + 0.5 * dx) / dx);
        s[i] = sn - d * dx;
        delta[i] = (int)d;
        int im = n - 1 - i;
        s[im] = -s[i];
        delta[im] = -(int)d;
    }
}

/* Fold a source coordinate into [0, len): periodic wrap, or reflection at
 * specular walls (each reflection mirrors the velocity along that axis). */
static int fold(int u, int len, int specular, int *flip)
{
    if (!specular) {
        int r = u % len;
        if (r < 0) r += len;
        *flip = 0;
        return r;
    }
    int per = 2 * len;
    int r = u % per;
    if (r < 0) r += per;
    if (r >= len) { *flip = 1; return per - 1 - r; }
    *flip = 0;
    return r;
}

/* f*[cell j][k] = f[cell j - delta_k][k'] : the piecewise-constant profile
 * of velocity k shifted by delta_k cells (the sister particle that enters
 * cell j comes from cell j - delta_k).  k' = k, or k mirrored along an axis
 * whose specular wall the particle crossed.
 * nc = (nx, ny, nz), bc[a] = 0 periodic / 1 specular, delta = [3][n]. */
void or_transport(const int *nc, const int *bc, int n, const int *delta,
                  const double *f, double *fout)
{
    long n3 = (long)n * n * n;
    for (int cx = 0; cx < nc[0]; ++cx)
        for (int cy = 0; cy < nc[1]; ++cy)
            for (int cz = 0; cz < nc[2]; ++cz) {
                long dst = ((long)cx * nc[1] + cy) * nc[2] + cz;
                for (int kx = 0; kx < n; ++kx)
                    for (int ky = 0; ky < n; ++ky)
                        for (int kz = 0; kz < n; ++kz) {
                            int fx, fy, fz;
                            int sx = fold(cx - delta[0 * n + kx], nc[0], bc[0], &fx);
                            int sy = fold(cy - delta[1 * n + ky], nc[1], bc[1], &fy);
                            int sz = fold(cz - delta[2 * n + kz], nc[2], bc[2], &fz);
                            int qx = fx ? n - 1 - kx : kx;
                            int qy = fy ? n - 1 - ky : ky;
                            int qz = fz ? n - 1 - kz : kz;
                            long src = ((long)sx * nc[1] + sy) * nc[2] + sz;
                            fout[dst * n3 + ((long)kx * n + ky) * n + kz] =
                                f[src * n3 + ((long)qx * n + qy) * n + qz];
                        }
            }
}

/* ------------------------------------------------------------------ */
/* BGK relaxation operator (Sec. 2, BGK approximation; Sec. 2.3)         */
/* ------------------------------------------------------------------ */

/* Q = nu (M[f] - f) for every cell, with M[f] the Maxwellian of the cell's
 * moments rho, u, T (3/2 rho T = E - rho |u|^2 / 2) evaluated at the grid
 * points, collision frequency nu = rho / Kn (the paper leaves nu(x, t) free),
 * followed by the conservation projection if project != 0 (the discrete
 * Maxwellian does not carry the discrete moments of f exactly). */
void or_bgk(int n, double L, double inv_kn, int project, long ncells, const double *f, double *Q)
{
    double v[64];
    or_vgrid(n, L, v);
    long n3 = (long)n * n * n;
    for (long c = 0; c < ncells; ++c) {
        double U[5];
        or_moments(n, L, 1, f + c * n3, U);
        double rho = U[0];
        double u[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
        double T = (U[4] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2])) / (1.5 * rho);
        if (!(rho > 0.0) || !(T > 0.0)) {
            /* no Maxwellian exists (vacuum or a degenerate cell): the cell does not relax */
            for (long k = 0; k < n3; ++k) Q[c * n3 + k] = 0.0;
            continue;
        }
        double nu = rho * inv_kn;
        double pre = rho * pow(2.0 * OR_PI * T, -1.5);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double dx = v[i] - u[0], dy = v[j] - u[1], dz = v[k] - u[2];
                    double M = pre * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * T));
                    long id = c * n3 + ((long)i * n + j) * n + k;
                    Q[id] = nu * (M - f[id]);
                }
        if (project) or_project(n, L, Q + c * n3);
    }
}

/* ------------------------------------------------------------------ */
/* variant B: the de-aliased operator of Eq. CF1 (l + m = k over the    */
/* modes l, m in [-n/2, n/2]^3, not reduced mod n), evaluated with      */
/* transforms of size 2n as in Sec. 5 (2n^3 transforms for n^3 modes).  */
/* Reading of the inclusive mode range: the coefficient of a Nyquist    */
/* component is split equally between +n/2 and -n/2; the result keeps   */
/* the modes |k| <= n/2 and folds +-n/2 back onto the Nyquist index.    */
/* ------------------------------------------------------------------ */

/* f2 = the trigonometric interpolant of f on the 2n grid of the same box
 * (points v_0 + j dv/2): FFT_n, Nyquist split, placement on the 2n index
 * grid, inverse FFT_2n.  f2 at even indices equals f. */
void or_pad(int n, const double *f, double *f2)
{
    int m = 2 * n;
    long n3 = (long)n * n * n, m3 = (long)m * m * m;
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
    cplx *G = (cplx *)calloc(m3, sizeof(cplx));
    for (long k = 0; k < n3; ++k) F[k] = f[k];
    or_fft3d(F, n, -1);
    for (long k = 0; k < n3; ++k) {
        int kk[3] = {(int)(k / ((long)n * n)), (int)((k / n) % n), (int)(k % n)};
        int fl[3], nf = 0, s0[3];
        for (int a = 0; a < 3; ++a) {
            s0[a] = kappa(kk[a], n);
            if (2 * kk[a] == n) fl[nf++] = a;
        }
        cplx val = F[k] / (double)n3 / (double)(1 << nf);
        for (int c = 0; c < (1 << nf); ++c) {
            int s[3] = {s0[0], s0[1], s0[2]};
            for (int b = 0; b < nf; ++b)
                if (c & (1 << b)) s[fl[b]] = -s[fl[b]];
            long t = ((long)((s[0] + m) % m) * m + (s[1] + m) % m) * m + (s[2] + m) % m;
            G[t] += val;
        }
    }
    or_fft3d(G, m, +1);
    for (long k = 0; k < m3; ++k) f2[k] = creal(G[k]);
    free(F); free(G);
}

/* Q = the modes |k| <= n/2 of Q2 (2n grid), +-n/2 folded onto the Nyquist
 * index, evaluated on the n grid: FFT_2n, selection, inverse FFT_n. */
void or_truncate(int n, const double *Q2, double *Q)
{
    int m = 2 * n;
    long n3 = (long)n * n * n, m3 = (long)m * m * m;
    cplx *A = (cplx *)malloc(sizeof(cplx) * m3);
    cplx *C = (cplx *)calloc(n3, sizeof(cplx));
    for (long k = 0; k < m3; ++k) A[k] = Q2[k];
    or_fft3d(A, m, -1);
    for (long k = 0; k < m3; ++k) {
        int kk[3] = {(int)(k / ((long)m * m)), (int)((k / m) % m), (int)(k % m)};
        int s[3], keep = 1;
        for (int a = 0; a < 3; ++a) {
            s[a] = kappa(kk[a], m);
            if (2 * abs(s[a]) > n) keep = 0;
        }
        if (!keep) continue;
        long t = ((long)((s[0] + n) % n) * n + (s[1] + n) % n) * n + (s[2] + n) % n;
        C[t] += A[k] / (double)m3;
    }
    or_fft3d(C, n, +1);
    for (long k = 0; k < n3; ++k) Q[k] = creal(C[k]);
    free(A); free(C);
}

/* Variant B for every cell: f2 = pad(f); gain and loss on the 2n grid with
 * the tables of the 2n grid (alpha2, alphap2, betaL2 of or_tables(2n, L, ...));
 * Q = truncate((G2 - L2) inv_kn), then the projection on the n grid. */
void or_collide_b(int n, double L, int M, const double *alpha2, const double *alphap2, const double *w,
                  const double *betaL2, double inv_kn, int project, long ncells, const double *f, double *Q)
{
    long n3 = (long)n * n * n, m3 = 8 * n3;
#pragma omp parallel
    {
        double *f2 = (double *)malloc(sizeof(double) * m3);
        double *G2 = (double *)malloc(sizeof(double) * m3);
        double *L2 = (double *)malloc(sizeof(double) * m3);
#pragma omp for schedule(dynamic)
        for (long c = 0; c < ncells; ++c) {
            or_pad(n, f + c * n3, f2);
            or_gain_loss(2 * n, M, alpha2, alphap2, w, betaL2, f2, G2, L2);
            for (long k = 0; k < m3; ++k) G2[k] = (G2[k] - L2[k]) * inv_kn;
            or_truncate(n, G2, Q + c * n3);
            if (project) or_project(n, L, Q + c * n3);
        }
        free(f2); free(G2); free(L2);
    }
}

/* Brute-force Eq. CF1 without reduction mod n (unprojected): coefficients
 * g_l of f on l in [-n/2, n/2]^3 (Nyquist split), beta(l, m) = sum_p w_p
 * [alpha_p(l) alphap_p(m) - alpha_p(m) alphap_p(m)] with alpha_p(l) =
 * phi(xi_l . e_p), alphap_p(l) = psi(|xi_l x e_p|) at the exact frequency
 * xi_l = (pi/L) l, Qhat_k = sum_{l + m = k} beta(l, m) g_l g_m for |k| <= n/2,
 * folded onto the n index grid and summed back: Q_j = sum_k Qhat_k e^{i xi_k v_j}.
 * Cost O((n+1)^6 M): for n <= 8. */
void or_galerkin_b(int n, double L, int ktype, double C, int A1, int A2, int rule, double inv_kn,
                   const double *f, double *Q)
{
    int M = A1 * A2, ne = n + 1, h = n / 2;
    long n3 = (long)n * n * n, e3 = (long)ne * ne * ne;
    double *e = (double *)malloc(sizeof(double) * 3 * M), *w = (double *)malloc(sizeof(double) * M);
    or_directions(A1, A2, rule, e, w);
    double R = 2.0 / (3.0 + sqrt(2.0)) * L, hx = OR_PI / L;
    gl_init();
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
    for (long k = 0; k < n3; ++k) F[k] = f[k];
    or_fft3d(F, n, -1);
    /* extended coefficients and tables, index (l + h) per axis */
    cplx *g = (cplx *)malloc(sizeof(cplx) * e3);
    double *a = (double *)malloc(sizeof(double) * M * e3), *b = (double *)malloc(sizeof(double) * M * e3);
    for (long i = 0; i < e3; ++i) {
        int l[3] = {(int)(i / ((long)ne * ne)) - h, (int)((i / ne) % ne) - h, (int)(i % ne) - h};
        int nf = 0;
        long src = 0;
        for (int x = 0; x < 3; ++x) {
            if (abs(l[x]) == h) ++nf;
            src = src * n + (l[x] + n) % n;
        }
        g[i] = F[src] / (double)n3 / (double)(1 << nf);
        double xi[3] = {hx * l[0], hx * l[1], hx * l[2]};
        for (int p = 0; p < M; ++p) {
            double de = xi[0] * e[3 * p] + xi[1] * e[3 * p + 1] + xi[2] * e[3 * p + 2];
            double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] - de * de;
            a[(long)p * e3 + i] = or_phi(ktype, C, R, de);
            b[(long)p * e3 + i] = or_psi(ktype, C, R, sqrt(q2 > 0 ? q2 : 0.0));
        }
    }
    cplx *Qc = (cplx *)calloc(n3, sizeof(cplx));
#pragma omp parallel for schedule(dynamic)
    for (long ik = 0; ik < e3; ++ik) {
        int k[3] = {(int)(ik / ((long)ne * ne)) - h, (int)((ik / ne) % ne) - h, (int)(ik % ne) - h};
        cplx acc = 0;
        for (long il = 0; il < e3; ++il) {
            int l[3] = {(int)(il / ((long)ne * ne)) - h, (int)((il / ne) % ne) - h, (int)(il % ne) - h};
            int mm[3] = {k[0] - l[0], k[1] - l[1], k[2] - l[2]};
            if (abs(mm[0]) > h || abs(mm[1]) > h || abs(mm[2]) > h) continue;
            long im = ((long)(mm[0] + h) * ne + (mm[1] + h)) * ne + (mm[2] + h);
            double beta = 0.0;
            for (int p = 0; p < M; ++p)
                beta += w[p] * (a[(long)p * e3 + il] - a[(long)p * e3 + im]) * b[(long)p * e3 + im];
            acc += beta * g[il] * g[im];
        }
        long t = ((long)((k[0] + n) % n) * n + (k[1] + n) % n) * n + (k[2] + n) % n;
#pragma omp critical
        Qc[t] += acc;
    }
    or_fft3d(Qc, n, +1);
    for (long j = 0; j < n3; ++j) Q[j] = creal(Qc[j]) * inv_kn;
    free(e); free(w); free(F); free(g); free(a); free(b); free(Qc);
}

/* ------------------------------------------------------------------ */
/* variable hard spheres: the non-separable kernel of Eq. Btilde_pl     */
/* ------------------------------------------------------------------ */

/* For the collision kernel B = C |g|^alpha the Carleman kernel is
 *   B~(r, r') = 4C (r^2 + r'^2)^((alpha - 1)/2),   r = |x|, r' = |y|
 * (Appendix A, Eq. Btilde_pl).  Only alpha = 1 makes it a product a(r) b(r');
 * for any other alpha the direction-p factor of B_F(l, m) stays the double
 * radial integral
 *   H(t, u) = int_0^R int_0^R [2 r cos(r t)] B~(r, r') [2 pi r' J_0(r' u)] dr dr'
 * (the phi and psi integrals of the separable case, here with B~ inside), and
 *   B_F(l, m) = sum_p w_p H(xi_l . e_p, |xi_m - (xi_m . e_p) e_p|).
 * The oracle evaluates H by a product quadrature in (r, r') on a composite
 * Gauss-Legendre rule: 20 nodes on each of [R/3, 2R/3] and [2R/3, R], and
 * 12 nodes on each of 16 panels of [0, R/3] that halve towards 0 (the last
 * one reaching 0), which resolves the corner r = r' = 0 where B~ is singular
 * for alpha < 1. */
enum { VHS_TOP = 20, VHS_LOW = 12, VHS_LEVELS = 16, VHS_NQ = 2 * VHS_TOP + VHS_LEVELS * VHS_LOW };

static void vhs_rule(double R, double *r, double *wr)
{
    double xt[VHS_TOP], wt[VHS_TOP], xl[VHS_LOW], wl[VHS_LOW];
    gauss_legendre(VHS_TOP, xt, wt);
    gauss_legendre(VHS_LOW, xl, wl);
    int q = 0;
    for (int j = 1; j <= 2; ++j) {
        double a = j * R / 3.0, b = (j + 1) * R / 3.0;
        for (int i = 0; i < VHS_TOP; ++i, ++q) {
            r[q] = a + 0.5 * (b - a) * (xt[i] + 1.0);
            wr[q] = 0.5 * (b - a) * wt[i];
        }
    }
    double b = R / 3.0;
    for (int lev = 0; lev < VHS_LEVELS; ++lev) {
        double a = lev < VHS_LEVELS - 1 ? 0.5 * b : 0.0;
        for (int i = 0; i < VHS_LOW; ++i, ++q) {
            r[q] = a + 0.5 * (b - a) * (xl[i] + 1.0);
            wr[q] = 0.5 * (b - a) * wl[i];
        }
        b = a;
    }
}

/* B~ on the node pairs: Bt[i * NQ + j] = 4C (r_i^2 + r_j^2)^((alpha-1)/2) */
static void vhs_kernel_matrix(double alpha, double C, const double *r, double *Bt)
{
    for (int i = 0; i < VHS_NQ; ++i)
        for (int j = 0; j < VHS_NQ; ++j)
            Bt[i * VHS_NQ + j] = 4.0 * C * pow(r[i] * r[i] + r[j] * r[j], 0.5 * (alpha - 1.0));
}

double or_vhs_h(double alpha, double C, double R, double t, double u)
{
    double r[VHS_NQ], wr[VHS_NQ], c[VHS_NQ], d[VHS_NQ];
    vhs_rule(R, r, wr);
    for (int i = 0; i < VHS_NQ; ++i) {
        c[i] = 2.0 * wr[i] * r[i] * cos(r[i] * t);
        d[i] = 2.0 * OR_PI * wr[i] * r[i] * bessel_j(0, r[i] * u);
    }
    double s = 0.0;
    for (int i = 0; i < VHS_NQ; ++i)
        for (int j = 0; j < VHS_NQ; ++j)
            s += c[i] * 4.0 * C * pow(r[i] * r[i] + r[j] * r[j], 0.5 * (alpha - 1.0)) * d[j];
    return s;
}

/* Radial factors of direction p on the DFT index grid, each the mean over
 * the sign choices of the Nyquist components (as in or_tables):
 *   c[i][k] = 2 w_i r_i cos(r_i xi_k . e_p)
 *   D[i][k] = sum_j B~(r_i, r_j) 2 pi w_j r_j J_0(r_j |xi_k - (xi_k . e_p) e_p|)
 * so that sum_i c[i][l] D[i][m] = H(xi_l . e_p, |xi_m x e_p|). */
static void vhs_direction_factors(int n, double L, const double *ep, const double *r, const double *wr,
                                  const double *Bt, double *c, double *D)
{
    long n3 = (long)n * n * n;
    double h = OR_PI / L;
    int nyq = (n % 2 == 0) ? n / 2 : -1;
#pragma omp parallel
    {
        double *ca = (double *)malloc(sizeof(double) * VHS_NQ);
        double *da = (double *)malloc(sizeof(double) * VHS_NQ);
#pragma omp for schedule(dynamic)
        for (long k = 0; k < n3; ++k) {
            int kk[3] = {(int)(k / ((long)n * n)), (int)((k / n) % n), (int)(k % n)};
            int nflip = 0, fl[3];
            for (int a = 0; a < 3; ++a) if (kk[a] == nyq) fl[nflip++] = a;
            int ncomb = 1 << nflip;
            for (int i = 0; i < VHS_NQ; ++i) ca[i] = da[i] = 0.0;
            for (int cmb = 0; cmb < ncomb; ++cmb) {
                double xi[3];
                for (int a = 0; a < 3; ++a) xi[a] = h * kappa(kk[a], n);
                for (int b = 0; b < nflip; ++b)
                    if (cmb & (1 << b)) xi[fl[b]] = -xi[fl[b]];
                double de = xi[0] * ep[0] + xi[1] * ep[1] + xi[2] * ep[2];
                double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] - de * de;
                double sp = sqrt(q2 > 0 ? q2 : 0.0);
                for (int i = 0; i < VHS_NQ; ++i) {
                    ca[i] += 2.0 * wr[i] * r[i] * cos(r[i] * de);
                    da[i] += 2.0 * OR_PI * wr[i] * r[i] * bessel_j(0, r[i] * sp);
                }
            }
            for (int i = 0; i < VHS_NQ; ++i) {
                double s = 0.0;
                for (int j = 0; j < VHS_NQ; ++j) s += Bt[i * VHS_NQ + j] * da[j];
                c[(long)i * n3 + k] = ca[i] / ncomb;
                D[(long)i * n3 + k] = s / ncomb;
            }
        }
        free(ca); free(da);
    }
}

/* Gain and loss of the VHS operator for every cell (no projection, no 1/Kn):
 *   G = sum_p w_p sum_i IDFT(c_{p,i} F) IDFT(D_{p,i} F) / n^6
 *   L = f IDFT(betaL F) / n^3,  betaL(k) = sum_p w_p sum_i c_{p,i}(k) D_{p,i}(k)
 * i.e. the Galerkin sum of Eq. CF1 with B_F(l, m) = sum_p w_p H_p(l, m),
 * written as a sum of products because H_p is a finite sum over quadrature
 * nodes of functions of l times functions of m. */
void or_vhs_gain_loss(int n, double L, double alpha, double C, int A1, int A2, int rule,
                      long ncells, const double *f, double *G, double *Lo)
{
    int M = A1 * A2;
    long n3 = (long)n * n * n;
    double *e = (double *)malloc(sizeof(double) * 3 * M), *w = (double *)malloc(sizeof(double) * M);
    or_directions(A1, A2, rule, e, w);
    double R = 2.0 / (3.0 + sqrt(2.0)) * L;
    double r[VHS_NQ], wr[VHS_NQ];
    vhs_rule(R, r, wr);
    double *Bt = (double *)malloc(sizeof(double) * VHS_NQ * VHS_NQ);
    vhs_kernel_matrix(alpha, C, r, Bt);
    double *c = (double *)malloc(sizeof(double) * VHS_NQ * n3);
    double *D = (double *)malloc(sizeof(double) * VHS_NQ * n3);
    double *betaL = (double *)calloc(n3, sizeof(double));
    double *P = (double *)malloc(sizeof(double) * VHS_NQ * n3);
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3 * ncells);
    for (long cl = 0; cl < ncells; ++cl) {
        for (long k = 0; k < n3; ++k) F[cl * n3 + k] = f[cl * n3 + k];
        or_fft3d(F + cl * n3, n, -1);
    }
    for (long k = 0; k < n3 * ncells; ++k) G[k] = 0.0;
    for (int p = 0; p < M; ++p) {
        vhs_direction_factors(n, L, e + 3 * p, r, wr, Bt, c, D);
        for (long k = 0; k < n3; ++k) {
            double s = 0.0;
            for (int i = 0; i < VHS_NQ; ++i) s += c[(long)i * n3 + k] * D[(long)i * n3 + k];
            betaL[k] += w[p] * s;
        }
        for (long cl = 0; cl < ncells; ++cl) {
            const cplx *Fc = F + cl * n3;
#pragma omp parallel
            {
                cplx *A = (cplx *)malloc(sizeof(cplx) * n3);
                cplx *B = (cplx *)malloc(sizeof(cplx) * n3);
#pragma omp for schedule(dynamic)
                for (int i = 0; i < VHS_NQ; ++i) {
                    for (long k = 0; k < n3; ++k) {
                        A[k] = c[(long)i * n3 + k] * Fc[k];
                        B[k] = D[(long)i * n3 + k] * Fc[k];
                    }
                    or_fft3d(A, n, +1);
                    or_fft3d(B, n, +1);
                    for (long k = 0; k < n3; ++k) P[(long)i * n3 + k] = (creal(A[k]) / n3) * (creal(B[k]) / n3);
                }
                free(A); free(B);
            }
            /* sum over the nodes in a fixed order (deterministic) */
            double *Gc = G + cl * n3;
#pragma omp parallel for
            for (long k = 0; k < n3; ++k) {
                double s = 0.0;
                for (int i = 0; i < VHS_NQ; ++i) s += P[(long)i * n3 + k];
                Gc[k] += w[p] * s;
            }
        }
    }
    cplx *A = (cplx *)malloc(sizeof(cplx) * n3);
    for (long cl = 0; cl < ncells; ++cl) {
        for (long k = 0; k < n3; ++k) A[k] = betaL[k] * F[cl * n3 + k];
        or_fft3d(A, n, +1);
        for (long k = 0; k < n3; ++k) Lo[cl * n3 + k] = f[cl * n3 + k] * creal(A[k]) / n3;
    }
    free(A); free(P); free(e); free(w); free(Bt); free(c); free(D); free(betaL); free(F);
}

/* Brute-force Eq. CF1 for the VHS kernel (one cell, unprojected):
 * Q^_k = n^-3 sum_{l+m=k mod n} [B_F(l,m) - B_F(m,m)] F_l F_m with
 * B_F(l,m) = sum_p w_p sum_i c_{p,i}(l) D_{p,i}(m), F by the direct DFT sum,
 * Q = IDFT(Q^)/n^3 by the direct sum, times inv_kn.  O(n^6 M NQ): n <= 8. */
void or_vhs_galerkin(int n, double L, double alpha, double C, int A1, int A2, int rule, double inv_kn,
                     const double *f, double *Q)
{
    int M = A1 * A2;
    long n3 = (long)n * n * n;
    double *e = (double *)malloc(sizeof(double) * 3 * M), *w = (double *)malloc(sizeof(double) * M);
    or_directions(A1, A2, rule, e, w);
    double R = 2.0 / (3.0 + sqrt(2.0)) * L;
    double r[VHS_NQ], wr[VHS_NQ];
    vhs_rule(R, r, wr);
    double *Bt = (double *)malloc(sizeof(double) * VHS_NQ * VHS_NQ);
    vhs_kernel_matrix(alpha, C, r, Bt);
    double *c = (double *)malloc(sizeof(double) * (long)M * VHS_NQ * n3);
    double *D = (double *)malloc(sizeof(double) * (long)M * VHS_NQ * n3);
    /* node factors of every direction, stored [p][k][i] (node index fastest) */
    double *tc = (double *)malloc(sizeof(double) * VHS_NQ * n3), *tD = (double *)malloc(sizeof(double) * VHS_NQ * n3);
    for (int p = 0; p < M; ++p) {
        vhs_direction_factors(n, L, e + 3 * p, r, wr, Bt, tc, tD);
        for (long k = 0; k < n3; ++k)
            for (int i = 0; i < VHS_NQ; ++i) {
                c[((long)p * n3 + k) * VHS_NQ + i] = tc[(long)i * n3 + k];
                D[((long)p * n3 + k) * VHS_NQ + i] = tD[(long)i * n3 + k];
            }
    }
    free(tc); free(tD);
    cplx *F = (cplx *)malloc(sizeof(cplx) * n3);
    cplx *Qh = (cplx *)calloc(n3, sizeof(cplx));
    for (long k = 0; k < n3; ++k) {
        int kx = (int)(k / (n * n)), ky = (int)((k / n) % n), kz = (int)(k % n);
        cplx s = 0;
        for (long j = 0; j < n3; ++j) {
            int jx = (int)(j / (n * n)), jy = (int)((j / n) % n), jz = (int)(j % n);
            double ang = -2.0 * OR_PI * (double)(kx * jx + ky * jy + kz * jz) / n;
            s += f[j] * (cos(ang) + I * sin(ang));
        }
        F[k] = s;
    }
#pragma omp parallel for schedule(dynamic)
    for (long k = 0; k < n3; ++k) {
        int kx = (int)(k / (n * n)), ky = (int)((k / n) % n), kz = (int)(k % n);
        cplx acc = 0;
        for (long l = 0; l < n3; ++l) {
            int lx = (int)(l / (n * n)), ly = (int)((l / n) % n), lz = (int)(l % n);
            long m = (((long)((kx - lx + n) % n) * n) + (ky - ly + n) % n) * n + (kz - lz + n) % n;
            double beta = 0.0;
            for (int p = 0; p < M; ++p) {
                const double *cl = c + ((long)p * n3 + l) * VHS_NQ, *cm = c + ((long)p * n3 + m) * VHS_NQ;
                const double *Dm = D + ((long)p * n3 + m) * VHS_NQ;
                double s = 0.0;
                for (int i = 0; i < VHS_NQ; ++i) s += (cl[i] - cm[i]) * Dm[i];
                beta += w[p] * s;
            }
            acc += beta * F[l] * F[m];
        }
        Qh[k] = acc;
    }
    for (long j = 0; j < n3; ++j) {
        int jx = (int)(j / (n * n)), jy = (int)((j / n) % n), jz = (int)(j % n);
        cplx s = 0;
        for (long k = 0; k < n3; ++k) {
            int kx = (int)(k / (n * n)), ky = (int)((k / n) % n), kz = (int)(k % n);
            double ang = 2.0 * OR_PI * (double)(kx * jx + ky * jy + kz * jz) / n;
            s += Qh[k] * (cos(ang) + I * sin(ang));
        }
        Q[j] = creal(s) / ((double)n3 * n3) * inv_kn;
    }
    free(e); free(w); free(Bt); free(c); free(D); free(F); free(Qh);
}
