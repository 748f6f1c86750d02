// fks_fft.cuh -- register-resident 1-D FFTs for the per-cell spectral passes.
//
// Sizes are compile-time: N = 2^a or 3 * 2^a (4, 8, 12, 16, 24, 32 are the
// ones the collision kernel uses).  Every index is a compile-time constant
// after unrolling, so the arrays live in registers.  Twiddle factors are
// computed at compile time from the Taylor series of sin/cos (own code, with
// octant reduction), never from a device math call.
//
//   fft<N, SIGN>(a)  :  a_k <- sum_j a_j exp(SIGN * 2 pi i j k / N), unnormalised
//   c2r<N>(h, x)     :  real x_j = sum_{k=0}^{N-1} X_k exp(+2 pi i j k / N) for a
//                       Hermitian X given as h[0] = (X_0, X_{N/2}) (both real)
//                       and h[k] = X_k, 1 <= k < N/2; costs one N/2-point FFT.
#pragma once
#include <utility>

namespace fks {

template <typename T> struct cpx { T x, y; };

template <typename T> __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }

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
__device__ __forceinline__ cpx<T> twiddle() {
    constexpr detail::SC sc = detail::sincos_frac(K, LEN);
    return {T(sc.c), T(SIGN * sc.s)};
}

template <typename T, int SIGN, long K, long LEN>
__device__ __forceinline__ cpx<T> mul_tw(cpx<T> a) {
    if constexpr (K % LEN == 0) return a;
    else if constexpr ((4 * K) % LEN == 0) {
        constexpr long q = ((4 * K) / LEN) % 4;   // multiple of a quarter turn
        if constexpr (q == 2) return {-a.x, -a.y};
        else if constexpr ((q == 1) == (SIGN > 0)) return {-a.y, a.x};   // * i
        else return {a.y, -a.x};                                           // * -i
    } else {
        return cmul(a, twiddle<T, SIGN, K, LEN>());
    }
}

// ---------------------------------------------------------------- FFT kernels
namespace detail {

template <int N> constexpr bool is_pow2() { return N > 0 && (N & (N - 1)) == 0; }

constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

// one radix-2 DIT butterfly column k (compile-time) for stage LEN
template <typename T, int SIGN, int N, int LEN, int K>
__device__ __forceinline__ void r2_column(cpx<T> (&a)[N]) {
#pragma unroll
    for (int i = 0; i < N; i += LEN) {
        cpx<T> u = a[i + K];
        cpx<T> t = mul_tw<T, SIGN, K, LEN>(a[i + K + LEN / 2]);
        a[i + K] = cadd(u, t);
        a[i + K + LEN / 2] = csub(u, t);
    }
}

template <typename T, int SIGN, int N, int LEN, int... K>
__device__ __forceinline__ void r2_stage(cpx<T> (&a)[N], std::integer_sequence<int, K...>) {
    (r2_column<T, SIGN, N, LEN, K>(a), ...);
}

template <typename T, int SIGN, int N, int LEN>
__device__ __forceinline__ void r2_stages(cpx<T> (&a)[N]) {
    r2_stage<T, SIGN, N, LEN>(a, std::make_integer_sequence<int, LEN / 2>{});
    if constexpr (LEN < N) r2_stages<T, SIGN, N, LEN * 2>(a);
}

template <typename T, int SIGN, int N>
__device__ __forceinline__ void fft_pow2(cpx<T> (&a)[N]) {
    if constexpr (N == 1) return;
    else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int j = bitrev(i, N);
            if (i < j) { cpx<T> t = a[i]; a[i] = a[j]; a[j] = t; }
        }
        r2_stages<T, SIGN, N, 2>(a);
    }
}

// radix-3 combine for output column k of an N = 3P transform
template <typename T, int SIGN, int N, int P, int K>
__device__ __forceinline__ void r3_column(cpx<T> (&a)[N], const cpx<T> (&b0)[P], const cpx<T> (&b1)[P],
                                          const cpx<T> (&b2)[P]) {
    cpx<T> t0 = b0[K];
    cpx<T> t1 = mul_tw<T, SIGN, K, N>(b1[K]);
    cpx<T> t2 = mul_tw<T, SIGN, 2 * K, N>(b2[K]);
    // X[k + qP] = t0 + w3^q t1 + w3^{2q} t2, w3 = exp(SIGN 2 pi i / 3)
    const T c = T(-0.5);
    const T s = T(SIGN) * T(0.866025403784438646763723170752936183);   // sin(2 pi / 3)
    cpx<T> sum = cadd(t1, t2);
    cpx<T> dif = csub(t1, t2);
    cpx<T> m = {t0.x + c * sum.x, t0.y + c * sum.y};
    cpx<T> r = {-s * dif.y, s * dif.x};   // i * s * (t1 - t2)
    a[K] = cadd(t0, sum);
    a[K + P] = cadd(m, r);
    a[K + 2 * P] = csub(m, r);
}

template <typename T, int SIGN, int N, int P, int... K>
__device__ __forceinline__ void r3_all(cpx<T> (&a)[N], const cpx<T> (&b0)[P], const cpx<T> (&b1)[P],
                                       const cpx<T> (&b2)[P], std::integer_sequence<int, K...>) {
    (r3_column<T, SIGN, N, P, K>(a, b0, b1, b2), ...);
}

}  // namespace detail

template <int N, int SIGN, typename T>
__device__ __forceinline__ void fft(cpx<T> (&a)[N]) {
    if constexpr (detail::is_pow2<N>()) {
        detail::fft_pow2<T, SIGN, N>(a);
    } else {
        static_assert(N % 3 == 0 && detail::is_pow2<N / 3>(), "FFT size must be 2^a or 3*2^a");
        constexpr int P = N / 3;
        cpx<T> b0[P], b1[P], b2[P];
#pragma unroll
        for (int m = 0; m < P; ++m) { b0[m] = a[3 * m]; b1[m] = a[3 * m + 1]; b2[m] = a[3 * m + 2]; }
        fft<P, SIGN>(b0);
        fft<P, SIGN>(b1);
        fft<P, SIGN>(b2);
        detail::r3_all<T, SIGN, N, P>(a, b0, b1, b2, std::make_integer_sequence<int, P>{});
    }
}

// ---------------------------------------------------------------- C2R
namespace detail {
template <typename T, int N, int K>
__device__ __forceinline__ void c2r_pre(const cpx<T> (&h)[N / 2], cpx<T> (&z)[N / 2]) {
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
__device__ __forceinline__ void c2r_pre_all(const cpx<T> (&h)[N / 2], cpx<T> (&z)[N / 2],
                                            std::integer_sequence<int, K...>) {
    (c2r_pre<T, N, K>(h, z), ...);
}
}  // namespace detail

// h: N/2 packed Hermitian coefficients (see header); x: N real outputs.
template <int N, typename T>
__device__ __forceinline__ void c2r(const cpx<T> (&h)[N / 2], T (&x)[N]) {
    cpx<T> z[N / 2];
    detail::c2r_pre_all<T, N>(h, z, std::make_integer_sequence<int, N / 2>{});
    fft<N / 2, +1>(z);
#pragma unroll
    for (int m = 0; m < N / 2; ++m) { x[2 * m] = z[m].x; x[2 * m + 1] = z[m].y; }
}

}  // namespace fks
