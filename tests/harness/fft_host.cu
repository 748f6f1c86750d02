// Host build of the library's register FFTs (csrc/fks_fft.cuh) for CPU tests:
// fks_test_fft(n, sign, prec, in, out) transforms one complex vector of length n
// (interleaved doubles), fks_test_c2r(n, in, out) runs the packed C2R; prec 0 float,
// 1 double, 2 double-float (csrc/fks_dfloat.cuh).
#include <cstring>

#include "fks_dfloat.cuh"
#include "fks_fft.cuh"

template <int N, typename T>
static void run_fft(int sign, const double* in, double* out) {
    fks::cpx<T> a[N];
    for (int i = 0; i < N; ++i) a[i] = {T(in[2 * i]), T(in[2 * i + 1])};
    if (sign < 0) fks::fft<N, -1>(a);
    else fks::fft<N, +1>(a);
    for (int i = 0; i < N; ++i) { out[2 * i] = double(a[i].x); out[2 * i + 1] = double(a[i].y); }
}

template <int N, typename T>
static void run_c2r(const double* in, double* out) {
    fks::cpx<T> h[N / 2];
    for (int i = 0; i < N / 2; ++i) h[i] = {T(in[2 * i]), T(in[2 * i + 1])};
    T x[N];
    fks::c2r<N>(h, x);
    for (int i = 0; i < N; ++i) out[i] = double(x[i]);
}

template <typename T>
static int dispatch_fft(int n, int sign, const double* in, double* out) {
    switch (n) {
        case 2: run_fft<2, T>(sign, in, out); return 0;
        case 3: run_fft<3, T>(sign, in, out); return 0;
        case 4: run_fft<4, T>(sign, in, out); return 0;
        case 8: run_fft<8, T>(sign, in, out); return 0;
        case 12: run_fft<12, T>(sign, in, out); return 0;
        case 16: run_fft<16, T>(sign, in, out); return 0;
        case 24: run_fft<24, T>(sign, in, out); return 0;
        case 32: run_fft<32, T>(sign, in, out); return 0;
    }
    return 1;
}

template <typename T>
static int dispatch_c2r(int n, const double* in, double* out) {
    switch (n) {
        case 8: run_c2r<8, T>(in, out); return 0;
        case 16: run_c2r<16, T>(in, out); return 0;
        case 24: run_c2r<24, T>(in, out); return 0;
        case 32: run_c2r<32, T>(in, out); return 0;
    }
    return 1;
}

template <int N, int R0, typename T>
static void run_fft_r(int sign, const double* in, double* out) {
    fks::cpx<T> a[N];
    for (int i = 0; i < N; ++i) a[i] = {T(in[2 * i]), T(in[2 * i + 1])};
    if (sign < 0) fks::fft<N, -1, R0>(a);
    else fks::fft<N, +1, R0>(a);
    for (int i = 0; i < N; ++i) { out[2 * i] = double(a[i].x); out[2 * i + 1] = double(a[i].y); }
}

// the radix schedules the collision kernels instantiate (top radix r0 of an n-point transform)
template <typename T>
static int dispatch_fft_r(int n, int r0, int sign, const double* in, double* out) {
    switch (n * 16 + r0) {
        case 8 * 16 + 2: run_fft_r<8, 2, T>(sign, in, out); return 0;
        case 8 * 16 + 4: run_fft_r<8, 4, T>(sign, in, out); return 0;
        case 16 * 16 + 2: run_fft_r<16, 2, T>(sign, in, out); return 0;
        case 16 * 16 + 8: run_fft_r<16, 8, T>(sign, in, out); return 0;
        case 24 * 16 + 2: run_fft_r<24, 2, T>(sign, in, out); return 0;
        case 24 * 16 + 4: run_fft_r<24, 4, T>(sign, in, out); return 0;
        case 24 * 16 + 8: run_fft_r<24, 8, T>(sign, in, out); return 0;
        case 32 * 16 + 2: run_fft_r<32, 2, T>(sign, in, out); return 0;
        case 32 * 16 + 8: run_fft_r<32, 8, T>(sign, in, out); return 0;
    }
    return 1;
}

extern "C" int fks_test_fft_radix(int n, int r0, int sign, int prec, const double* in, double* out) {
    if (prec == 2) return dispatch_fft_r<fks::dfloat>(n, r0, sign, in, out);
    return prec ? dispatch_fft_r<double>(n, r0, sign, in, out) : dispatch_fft_r<float>(n, r0, sign, in, out);
}

extern "C" int fks_test_fft(int n, int sign, int prec, const double* in, double* out) {
    if (prec == 2) return dispatch_fft<fks::dfloat>(n, sign, in, out);
    return prec ? dispatch_fft<double>(n, sign, in, out) : dispatch_fft<float>(n, sign, in, out);
}

extern "C" int fks_test_c2r(int n, int prec, const double* in, double* out) {
    if (prec == 2) return dispatch_c2r<fks::dfloat>(n, in, out);
    return prec ? dispatch_c2r<double>(n, in, out) : dispatch_c2r<float>(n, in, out);
}
