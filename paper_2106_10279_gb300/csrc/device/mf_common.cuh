// Common device definitions for the run-time-compiled process kernels.
// Compiled by NVRTC (no standard headers): fixed-width integer types and a
// small complex type are defined here.
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned long long uint64_t;
typedef long long int64_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned short uint16_t;
typedef signed char int8_t;
typedef unsigned char uint8_t;
#else
#include <cstdint>
#endif

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define MF_DEV __device__ __forceinline__
#else
// host compilation of the arithmetic headers, used only by the unit tests of
// the routines (tests/adjoint_check.cpp)
#include <cmath>
#define MF_DEV inline
#endif

namespace mf {

template <typename R>
struct cx {
    R re, im;
};

template <typename R> MF_DEV cx<R> C(R a, R b) { return cx<R>{a, b}; }
template <typename R> MF_DEV cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> MF_DEV cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> MF_DEV cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R> MF_DEV cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> MF_DEV cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> MF_DEV cx<R> operator*(cx<R> a, R s) { return {s * a.re, s * a.im}; }
template <typename R> MF_DEV cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// i * a and -i * a
template <typename R> MF_DEV cx<R> mul_i(cx<R> a) { return {-a.im, a.re}; }
template <typename R> MF_DEV cx<R> mul_mi(cx<R> a) { return {a.im, -a.re}; }
// a + b * c (complex fused form)
template <typename R> MF_DEV cx<R> cfma(cx<R> b, cx<R> c, cx<R> a) {
    return {a.re + b.re * c.re - b.im * c.im, a.im + b.re * c.im + b.im * c.re};
}

// Product with a factor whose phase class is known when the program is
// generated: PH 1 a real factor (f.im == 0), PH 2 an imaginary one
// (f.re == 0), PH 0 a general complex factor.  The couplings of the vertex
// routines are real or imaginary in QCD (i g_s, g_s, -i g_s^2), which turns
// their complex products into real-times-complex ones.
template <int PH, typename R> MF_DEV cx<R> pmul(cx<R> f, cx<R> a) {
    if constexpr (PH == 1) return {f.re * a.re, f.re * a.im};
    else if constexpr (PH == 2) return {-(f.im * a.im), f.im * a.re};
    else return f * a;
}
// the phase class of i f (or -i f) from that of f
constexpr int rotate_phase(int ph) { return ph == 1 ? 2 : ph == 2 ? 1 : 0; }

// Wavefunction: four complex components.  Its momentum (flowing into the
// diagram through the legs it contains) is a signed sum of external momenta
// known when the program is generated, and is formed where a routine needs it.
template <typename R>
struct W {
    cx<R> c[4];
};

// Minkowski product of two complex 4-vectors, no conjugation.
template <typename R> MF_DEV cx<R> mdot(const cx<R> *a, const cx<R> *b) {
    cx<R> r = a[0] * b[0];
    r = r - a[1] * b[1];
    r = r - a[2] * b[2];
    r = r - a[3] * b[3];
    return r;
}
// Minkowski product of a real and a complex 4-vector.
template <typename R> MF_DEV cx<R> mdot(const R *k, const cx<R> *b) {
    return {k[0] * b[0].re - k[1] * b[1].re - k[2] * b[2].re - k[3] * b[3].re,
            k[0] * b[0].im - k[1] * b[1].im - k[2] * b[2].im - k[3] * b[3].im};
}

}  // namespace mf
