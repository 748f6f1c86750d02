// fks_fft.cuh -- register-resident 1-D FFTs for the per-cell spectral passes.
//
// Sizes are compile-time: N = 2^a or 3 * 2^a (4, 8, 12, 16, 24, 32 are the
// ones the collision kernel uses).  Every index is a compile-time constant
// after unrolling, so the arrays live in registers.  Twiddle factors are
// computed at compile time from the Taylor series of sin/cos (own code, with
// octant reduction), never from a device math call.
//
//   fft<N, SIGN>(a)  :  a_k <- sum_j a_j exp(SIGN * 2 pi i j k / N), unnormalised
//   fft<N, SIGN, R0> :  the same with the top radix R0 in {2, 3, 4, 8} (the radix schedule:
//                       N = R0 x P, the sub-transforms of size P by the default schedule)
//   c2r<N>(h, x)     :  real x_j = sum_{k=0}^{N-1} X_k exp(+2 pi i j k / N) for a
//                       Hermitian X given as h[0] = (X_0, X_{N/2}) (both real)
//                       and h[k] = X_k, 1 <= k < N/2; costs one N/2-point FFT.
#pragma once
#include <utility>

#if defined(__CUDACC__)
#define FKS_HD __host__ __device__ __forceinline__
#else
#define FKS_HD inline
#endif

namespace fks {

template <typename T> struct cpx { T x, y; };

// Arithmetic types whose products cost several sums (double-float pairs): an eighth-turn twiddle
// is then taken as one sum scaled by 1/sqrt 2 instead of four products.
template <typename T> struct costly_mul { static constexpr bool value = false; };

template <typename T> FKS_HD cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> FKS_HD cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> FKS_HD cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> FKS_HD cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
// sums that feed only further sums: a type may leave them unnormalised (double-float pairs skip the
// final renormalisation, see fks_dfloat.cuh); plain sums otherwise
template <typename T> FKS_HD T add_lazy(T a, T b) { return a + b; }
template <typename T> FKS_HD T sub_lazy(T a, T b) { return a - b; }
template <typename T> FKS_HD cpx<T> cadd_lazy(cpx<T> a, cpx<T> b) { return {add_lazy(a.x, b.x), add_lazy(a.y, b.y)}; }
template <typename T> FKS_HD cpx<T> csub_lazy(cpx<T> a, cpx<T> b) { return {sub_lazy(a.x, b.x), sub_lazy(a.y, b.y)}; }

// ---------------------------------------------------------------- constexpr trig
namespace detail {
constexpr double kPi = 3.141592653589793238462643383279502884;
// sin and cos of |x| <= pi/4 by their Taylor series (18 terms: far below 1 ulp)
constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i < 18; ++i) { term *= -x2 / ((2.0 * i) * (2.0 * i + 1.0)); sum += term; }
    return sum;
}
constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i < 18; ++i) { term *= -x2 / ((2.0 * i - 1.0) * (2.0 * i)); sum += term; }
    return sum;
}
// cos / sin of 2 pi k / n with exact octant reduction on the integer fraction
struct SC { double s, c; };
constexpr SC sincos_frac(long k, long n) {
    k %= n;
    if (k < 0) k += n;
    // angle = 2 pi k / n = (pi/4) * (8k / n); octant o, remainder r in [0, n)
    long m = 8 * k;
    long o = m / n;
    long r = m - o * n;             // angle = (pi/4) * (o + r / n)
    double t = (kPi / 4.0) * double(r) / double(n);   // in [0, pi/4)
    double s0 = taylor_sin(t), c0 = taylor_cos(t);
    double ts = (kPi / 4.0) - t;                      // complementary angle for odd octants
    double s1 = taylor_sin(ts), c1 = taylor_cos(ts);
    switch (o) {
        case 0: return {s0, c0};          // t
        case 1: return {c1, s1};          // pi/2 - ts
        case 2: return {c0, -s0};         // pi/2 + t
        case 3: return {s1, -c1};         // pi - ts
        case 4: return {-s0, -c0};        // pi + t
        case 5: return {-c1, -s1};        // 3pi/2 - ts
        case 6: return {-c0, s0};         // 3pi/2 + t
        default: return {-s1, c1};        // 2pi - ts
    }
}
}  // namespace detail

// W = exp(SIGN * 2 pi i K / LEN) as a compile-time constant
template <typename T, int SIGN, long K, long LEN>
FKS_HD cpx<T> twiddle() {
    constexpr detail::SC sc = detail::sincos_frac(K, LEN);
    return {T(sc.c), T(SIGN * sc.s)};
}

template <typename T, int SIGN, long K, long LEN>
FKS_HD cpx<T> mul_tw(cpx<T> a) {
    if constexpr (K % LEN == 0) return a;
    else if constexpr ((4 * K) % LEN == 0) {
        constexpr long q = ((4 * K) / LEN) % 4;   // multiple of a quarter turn
        if constexpr (q == 2) return {-a.x, -a.y};
        else if constexpr ((q == 1) == (SIGN > 0)) return {-a.y, a.x};   // * i
        else return {a.y, -a.x};                                           // * -i
    } else if constexpr ((8 * K) % LEN == 0) {
        // odd multiple of an eighth turn: (+-1 +- i)/sqrt 2
        constexpr detail::SC sc = detail::sincos_frac(K, LEN);
        const T h = T(0.707106781186547524400844362104849039);
        if constexpr (costly_mul<T>::value) {
            // (sr + i si) h a with sr, si = +-1: the sums first, then two products
            constexpr bool pr = sc.c > 0, pi = (SIGN * sc.s) > 0;
            const T re = pr ? (pi ? sub_lazy(a.x, a.y) : add_lazy(a.x, a.y)) : (pi ? -add_lazy(a.x, a.y) : sub_lazy(a.y, a.x));
            const T im = pr ? (pi ? add_lazy(a.y, a.x) : sub_lazy(a.y, a.x)) : (pi ? sub_lazy(a.x, a.y) : -add_lazy(a.x, a.y));
            return {h * re, h * im};
        } else {
            const T cr = sc.c > 0 ? h : -h;
            const T ci = (SIGN * sc.s) > 0 ? h : -h;
            return {cr * a.x - ci * a.y, cr * a.y + ci * a.x};
        }
    } else {
        return cmul(a, twiddle<T, SIGN, K, LEN>());
    }
}

// ---------------------------------------------------------------- FFT kernels
//
// Mixed-radix decimation in time: N = R * P with R in {3, 4} at the top (or the
// requested R0 in {2, 3, 4, 8}) and the sub-transforms of size P recursive;
// sizes 2, 3, 4 and 8 are direct butterflies.  Default schedules: 32 = 4 x 8,
// 16 = 4 x 4, 24 = 3 x 8, 12 = 3 x 4; alternatives e.g. 32 = 8 x 4 or 2 x 16.
namespace detail {

template <int N> constexpr bool is_pow2() { return N > 0 && (N & (N - 1)) == 0; }

template <typename T, int SIGN>
FKS_HD void dft2(cpx<T>& a0, cpx<T>& a1) {
    const cpx<T> s = cadd_lazy(a0, a1), d = csub_lazy(a0, a1);
    a0 = s;
    a1 = d;
}

// a * (SIGN i)
template <typename T, int SIGN>
FKS_HD cpx<T> mul_si(cpx<T> a) {
    if constexpr (SIGN > 0) return {-a.y, a.x};
    else return {a.y, -a.x};
}

template <typename T, int SIGN>
FKS_HD void dft4(cpx<T>& a0, cpx<T>& a1, cpx<T>& a2, cpx<T>& a3) {
    // every butterfly sum may stay unnormalised: its uses are sums and products (which take an
    // unnormalised operand); the caller renormalises the transform's outputs where it needs them
    const cpx<T> s02 = cadd_lazy(a0, a2), d02 = csub_lazy(a0, a2);
    const cpx<T> s13 = cadd_lazy(a1, a3), d13 = mul_si<T, SIGN>(csub_lazy(a1, a3));
    a0 = cadd_lazy(s02, s13);
    a2 = csub_lazy(s02, s13);
    a1 = cadd_lazy(d02, d13);
    a3 = csub_lazy(d02, d13);
}

template <typename T, int SIGN>
FKS_HD void dft3(cpx<T>& a0, cpx<T>& a1, cpx<T>& a2) {
    const T c = T(-0.5);
    const T s = T(SIGN) * T(0.866025403784438646763723170752936183);   // sin(2 pi / 3)
    const cpx<T> sum = cadd_lazy(a1, a2), dif = csub_lazy(a1, a2);
    const cpx<T> m = {a0.x + c * sum.x, a0.y + c * sum.y};
    const cpx<T> r = {-s * dif.y, s * dif.x};
    a0 = cadd_lazy(a0, sum);
    a1 = cadd_lazy(m, r);
    a2 = csub_lazy(m, r);
}

template <typename T, int SIGN>
FKS_HD void dft8(cpx<T> (&a)[8]) {
    cpx<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    cpx<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<T, SIGN>(e0, e1, e2, e3);
    dft4<T, SIGN>(o0, o1, o2, o3);
    o1 = mul_tw<T, SIGN, 1, 8>(o1);
    o2 = mul_tw<T, SIGN, 2, 8>(o2);
    o3 = mul_tw<T, SIGN, 3, 8>(o3);
    a[0] = cadd_lazy(e0, o0); a[4] = csub_lazy(e0, o0);
    a[1] = cadd_lazy(e1, o1); a[5] = csub_lazy(e1, o1);
    a[2] = cadd_lazy(e2, o2); a[6] = csub_lazy(e2, o2);
    a[3] = cadd_lazy(e3, o3); a[7] = csub_lazy(e3, o3);
}

template <int N, int R0> constexpr int top_radix() {
    if constexpr (R0 != 0) return R0;
    else if constexpr (N % 3 == 0) return 3;
    else return 4;
}

// t[q] <- sub[q][K] W^{qK} for q < R (W = exp(SIGN 2 pi i / N)), compile-time q
template <typename T, int SIGN, int N, int R, int P, int K, int... Q>
FKS_HD void twiddle_column(cpx<T> (&t)[R], const cpx<T> (&sub)[R][P], std::integer_sequence<int, Q...>) {
    ((t[Q] = mul_tw<T, SIGN, (long)Q * K, N>(sub[Q][K])), ...);
}

template <typename T, int SIGN, int N, int R, int P, int K>
FKS_HD void combine_column(cpx<T> (&a)[N], const cpx<T> (&sub)[R][P]) {
    cpx<T> t[R];
    twiddle_column<T, SIGN, N, R, P, K>(t, sub, std::make_integer_sequence<int, R>{});
    if constexpr (R == 2) {
        dft2<T, SIGN>(t[0], t[1]);
    } else if constexpr (R == 3) {
        dft3<T, SIGN>(t[0], t[1], t[2]);
    } else if constexpr (R == 4) {
        dft4<T, SIGN>(t[0], t[1], t[2], t[3]);
    } else {
        static_assert(R == 8, "top radix 2, 3, 4 or 8");
        dft8<T, SIGN>(t);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) a[K + P * q] = t[q];
}

template <typename T, int SIGN, int N, int R, int P, int... K>
FKS_HD void combine_all(cpx<T> (&a)[N], const cpx<T> (&sub)[R][P], std::integer_sequence<int, K...>) {
    (combine_column<T, SIGN, N, R, P, K>(a, sub), ...);
}

}  // namespace detail

template <int N, int SIGN, int R0 = 0, typename T>
FKS_HD void fft(cpx<T> (&a)[N]) {
    if constexpr (N == 1) {
        return;
    } else if constexpr (N == 2) {
        detail::dft2<T, SIGN>(a[0], a[1]);
    } else if constexpr (N == 3) {
        detail::dft3<T, SIGN>(a[0], a[1], a[2]);
    } else if constexpr (N == 4 && R0 == 0) {
        detail::dft4<T, SIGN>(a[0], a[1], a[2], a[3]);
    } else if constexpr (N == 8 && R0 == 0) {
        detail::dft8<T, SIGN>(a);
    } else {
        constexpr int R = detail::top_radix<N, R0>();
        constexpr int P = N / R;
        static_assert(P * R == N, "FFT size must be 2^a or 3*2^a");
        cpx<T> sub[R][P];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < P; ++m) sub[r][m] = a[R * m + r];
#pragma unroll
        for (int r = 0; r < R; ++r) fft<P, SIGN>(sub[r]);
        detail::combine_all<T, SIGN, N, R, P>(a, sub, std::make_integer_sequence<int, P>{});
    }
}

// ---------------------------------------------------------------- C2R
namespace detail {
template <typename T, int N, int K>
FKS_HD void c2r_pre(const cpx<T> (&h)[N / 2], cpx<T> (&z)[N / 2]) {
    // E_k = X_k + conj(X_{N/2-k}),  O_k = (X_k - conj(X_{N/2-k})) e^{+2 pi i k / N},  Z_k = E_k + i O_k
    if constexpr (K == 0) {
        T x0 = h[0].x, xn = h[0].y;
        z[0] = {x0 + xn, x0 - xn};   // E_0 = X0 + X_{N/2} (real), O_0 = X0 - X_{N/2} (real)
    } else {
        cpx<T> a = h[K];
        cpx<T> b = {h[N / 2 - K].x, -h[N / 2 - K].y};
        cpx<T> e = cadd(a, b);
        cpx<T> o = mul_tw<T, +1, K, N>(csub(a, b));
        z[K] = {e.x - o.y, e.y + o.x};
    }
}
template <typename T, int N, int... K>
FKS_HD void c2r_pre_all(const cpx<T> (&h)[N / 2], cpx<T> (&z)[N / 2],
                                            std::integer_sequence<int, K...>) {
    (c2r_pre<T, N, K>(h, z), ...);
}
}  // namespace detail

// h: N/2 packed Hermitian coefficients (see header); x: N real outputs.
template <int N, typename T>
FKS_HD void c2r(const cpx<T> (&h)[N / 2], T (&x)[N]) {
    cpx<T> z[N / 2];
    detail::c2r_pre_all<T, N>(h, z, std::make_integer_sequence<int, N / 2>{});
    fft<N / 2, +1>(z);
#pragma unroll
    for (int m = 0; m < N / 2; ++m) { x[2 * m] = z[m].x; x[2 * m + 1] = z[m].y; }
}

}  // namespace fks
