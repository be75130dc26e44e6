// Forward-mode tangents (dual numbers with K directions) for the per-event
// kinematics of the gradient kernel: a value and its derivatives with respect
// to K seeded inputs, propagated through +, -, *, / and the elementary
// functions by the chain rule.  Comparisons look at the value only.
#pragma once
#include "mf_common.cuh"

namespace mf {

// keep the double-precision math functions visible next to the overloads
using ::atan2;
using ::cos;
using ::exp;
using ::expm1;
using ::fabs;
using ::floor;
using ::fmax;
using ::log;
using ::log1p;
using ::pow;
using ::sin;
using ::sincos;
using ::sqrt;

template <int K>
struct Dual {
    double v;
    double d[K];
    MF_DEV Dual() {}
    MF_DEV Dual(double x) : v(x) {
#pragma unroll
        for (int i = 0; i < K; ++i) d[i] = 0.0;
    }
    MF_DEV static Dual seed(double x, int j) {
        Dual r(x);
        r.d[j] = 1.0;
        return r;
    }
};

template <int K> MF_DEV Dual<K> operator+(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r; r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int K> MF_DEV Dual<K> operator-(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r; r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int K> MF_DEV Dual<K> operator-(const Dual<K> &a) {
    Dual<K> r; r.v = -a.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int K> MF_DEV Dual<K> operator*(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r; r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int K> MF_DEV Dual<K> operator/(const Dual<K> &a, const Dual<K> &b) {
    Dual<K> r; r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int K> MF_DEV Dual<K> operator+(const Dual<K> &a, double b) { return a + Dual<K>(b); }
template <int K> MF_DEV Dual<K> operator+(double a, const Dual<K> &b) { return Dual<K>(a) + b; }
template <int K> MF_DEV Dual<K> operator-(const Dual<K> &a, double b) { return a - Dual<K>(b); }
template <int K> MF_DEV Dual<K> operator-(double a, const Dual<K> &b) { return Dual<K>(a) - b; }
template <int K> MF_DEV Dual<K> operator*(const Dual<K> &a, double b) {
    Dual<K> r; r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <int K> MF_DEV Dual<K> operator*(double a, const Dual<K> &b) { return b * a; }
template <int K> MF_DEV Dual<K> operator/(const Dual<K> &a, double b) { return a * (1.0 / b); }
template <int K> MF_DEV Dual<K> operator/(double a, const Dual<K> &b) { return Dual<K>(a) / b; }
template <int K> MF_DEV Dual<K> &operator+=(Dual<K> &a, const Dual<K> &b) { a = a + b; return a; }
template <int K> MF_DEV Dual<K> &operator-=(Dual<K> &a, const Dual<K> &b) { a = a - b; return a; }
template <int K> MF_DEV Dual<K> &operator*=(Dual<K> &a, const Dual<K> &b) { a = a * b; return a; }

template <int K> MF_DEV bool operator<(const Dual<K> &a, const Dual<K> &b) { return a.v < b.v; }
template <int K> MF_DEV bool operator>(const Dual<K> &a, const Dual<K> &b) { return a.v > b.v; }
template <int K> MF_DEV bool operator<=(const Dual<K> &a, const Dual<K> &b) { return a.v <= b.v; }
template <int K> MF_DEV bool operator>=(const Dual<K> &a, const Dual<K> &b) { return a.v >= b.v; }
template <int K> MF_DEV bool operator<(const Dual<K> &a, double b) { return a.v < b; }
template <int K> MF_DEV bool operator>(const Dual<K> &a, double b) { return a.v > b; }
template <int K> MF_DEV bool operator<=(const Dual<K> &a, double b) { return a.v <= b; }
template <int K> MF_DEV bool operator>=(const Dual<K> &a, double b) { return a.v >= b; }
template <int K> MF_DEV bool operator==(const Dual<K> &a, double b) { return a.v == b; }
template <int K> MF_DEV bool operator!=(const Dual<K> &a, double b) { return a.v != b; }

// f(a) with f'(a) = df
template <int K> MF_DEV Dual<K> chain(const Dual<K> &a, double f, double df) {
    Dual<K> r; r.v = f;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = df * a.d[i];
    return r;
}
template <int K> MF_DEV Dual<K> sqrt(const Dual<K> &a) { double s = ::sqrt(a.v); return chain(a, s, s > 0.0 ? 0.5 / s : 0.0); }
template <int K> MF_DEV Dual<K> exp(const Dual<K> &a) { double e = ::exp(a.v); return chain(a, e, e); }
template <int K> MF_DEV Dual<K> log(const Dual<K> &a) { return chain(a, ::log(a.v), 1.0 / a.v); }
template <int K> MF_DEV Dual<K> log1p(const Dual<K> &a) { return chain(a, ::log1p(a.v), 1.0 / (1.0 + a.v)); }
template <int K> MF_DEV Dual<K> expm1(const Dual<K> &a) { return chain(a, ::expm1(a.v), ::exp(a.v)); }
template <int K> MF_DEV Dual<K> sin(const Dual<K> &a) { return chain(a, ::sin(a.v), ::cos(a.v)); }
template <int K> MF_DEV Dual<K> cos(const Dual<K> &a) { return chain(a, ::cos(a.v), -::sin(a.v)); }
template <int K> MF_DEV void sincos(const Dual<K> &a, Dual<K> *s, Dual<K> *c) {
    double sv, cv;
    ::sincos(a.v, &sv, &cv);
    *s = chain(a, sv, cv);
    *c = chain(a, cv, -sv);
}
template <int K> MF_DEV Dual<K> fabs(const Dual<K> &a) { return a.v < 0.0 ? -a : a; }
template <int K> MF_DEV Dual<K> fmax(const Dual<K> &a, double b) { return a.v >= b ? a : Dual<K>(b); }
template <int K> MF_DEV Dual<K> atan2(const Dual<K> &y, const Dual<K> &x) {
    double r2 = x.v * x.v + y.v * y.v;
    Dual<K> r; r.v = ::atan2(y.v, x.v);
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / r2;
    return r;
}

// value of a scalar (double or Dual)
MF_DEV double value(double a) { return a; }
template <int K> MF_DEV double value(const Dual<K> &a) { return a.v; }

}  // namespace mf
