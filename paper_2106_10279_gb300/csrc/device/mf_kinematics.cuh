// Double-precision per-event kinematics: counter-based random numbers, the
// Vegas map, the x1/x2 map, flat phase space with the RAMBO massive
// rescaling (Sec. 2.4), cuts and the PDF interpolation (Sec. 1, Fig. 1).
#pragma once
#include "mf_common.cuh"
#include "mf_dual.cuh"

namespace mf {

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of the 4x64 Philox bijection.
MF_DEV void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}
// odd multiples of 2^-53: strictly inside (0, 1), exact
MF_DEV double unit_from_bits(uint64_t r) { return (double)((r >> 11) | 1ull) * 0x1p-53; }

// ---------------------------------------------------------------- Vegas map
// y -> x through per-dimension edges; returns the Jacobian factor, bin index.
MF_DEV double vegas_map1(const double *edges, int nb, double y, double &x, int &bin) {
    double ynb = y * nb;
    int i = (int)floor(ynb);
    if (i > nb - 1) i = nb - 1;
    if (i < 0) i = 0;
    double lo = edges[i], w = edges[i + 1] - lo;
    x = lo + (ynb - i) * w;
    bin = i;
    return nb * w;
}

// ---------------------------------------------------------------- x1, x2 map
// tau = tau_min^y0, x1 = tau^y1, x2 = tau / x1, J = tau ln(1/tau_min) ln(1/tau).
// T is double, or a dual number carrying derivatives (gradient kernel).
template <typename T>
struct XMap {
    T x1, x2, tau, ln_x1, ln_x2, jac;
};
template <typename T>
MF_DEV XMap<T> xmap(const T &y0, const T &y1, const T &ln_tau_min) {
    XMap<T> m;
    T ln_tau = y0 * ln_tau_min;
    m.tau = exp(ln_tau);
    m.ln_x1 = y1 * ln_tau;
    m.x1 = exp(m.ln_x1);
    m.x2 = m.tau / m.x1;
    // ln x2 = (1 - y1) ln tau: no cancellation when x2 -> 1
    m.ln_x2 = (1.0 - y1) * ln_tau;
    m.jac = m.tau * (-ln_tau_min) * (-ln_tau);
    return m;
}

// ---------------------------------------------------------------- phase space
// Boost p (given in the rest frame of Q, mass M) into the frame of Q.
template <typename T>
MF_DEV void boost_from_rest(const T *p, const T *Q, const T &M, T *out) {
    T e = (Q[0] * p[0] + Q[1] * p[1] + Q[2] * p[2] + Q[3] * p[3]) / M;
    T c = (p[0] + e) / (Q[0] + M);
    out[0] = e;
    out[1] = p[1] + c * Q[1];
    out[2] = p[2] + c * Q[2];
    out[3] = p[3] + c * Q[3];
}

#define MF_MAX_MASS_RATIO_M 8   // daughter systems of up to 8 massless particles

// Safeguarded Newton solve of an increasing G on [0, 1] for G(z) = t, with
// G and G' from g(z, &dG).
template <typename Gf>
MF_DEV double increasing_root(Gf g, double t, double z) {
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        double dG;
        double f = g(z, dG) - t;
        if (f < 0.0) lo = z; else hi = z;
        double nz = (dG > 0.0) ? z - f / dG : 0.5 * (lo + hi);
        if (!(nz > lo && nz < hi)) nz = 0.5 * (lo + hi);
        if (fabs(nz - z) <= 4e-16 * z || hi - lo <= 4e-16 * hi) return nz;
        z = nz;
    }
    return z;
}

// Squared-mass ratio x of a daughter system of m massless particles: solves
// F(x) = m x^(m-1) - (m-1) x^m = r on [0, 1], and returns x with its
// complement d = 1 - x, both to full relative precision.  For r > 1/2 the
// root is near 1, where F is flat and x as a double fixes 1 - x only to
// ~sqrt(eps); there d solves the complementary equation
// G(d) = 1 - F(1 - d) = sum_{k>=2} c_k (-d)^k = 1 - r with the exact integer
// coefficients c_k = (m-1) C(m, k) - m C(m-1, k) (1 - r is exact).
MF_DEV double mass_ratio(int m, double r, double &d) {
    if (m == 2) {
        // 2x - x^2 = r  ->  d = sqrt(1 - r), x = r / (1 + d)
        d = sqrt(1.0 - r);
        return r / (1.0 + d);
    }
    if (m == 3) {
        // 3x^2 - 2x^3 = r is symmetric under (x, r) -> (1-x, 1-r): solve the
        // half with x <= 1/2 by Newton from sqrt(t/3), which is then monotone.
        bool upper = r > 0.5;
        double t = upper ? 1.0 - r : r;
        double s = sqrt(t / 3.0);
        for (int it = 0; it < 60; ++it) {
            double f = s * s * (3.0 - 2.0 * s) - t;
            double dd = 6.0 * s * (1.0 - s);
            if (dd <= 0.0) break;
            double ns = s - f / dd;
            if (ns < 0.0) ns = 0.5 * s;
            if (ns > 0.5) ns = 0.5 * (s + 0.5);
            double step = fabs(ns - s);
            s = ns;
            if (step <= 1e-17 + 4e-16 * s) break;
        }
        d = upper ? s : 1.0 - s;
        return upper ? 1.0 - s : s;
    }
    if (r <= 0.5) {
        double x = increasing_root([m](double z, double &dG) {
            double zm2 = pow(z, m - 2);
            dG = m * (m - 1) * zm2 * (1.0 - z);
            return m * zm2 * z - (m - 1) * zm2 * z * z;
        }, r, pow(r, 1.0 / (m - 1)));
        d = 1.0 - x;
        return x;
    }
    d = increasing_root([m](double z, double &dG) {
        // Horner in -z over k = m .. 2 of c_k, then times z^2
        double acc = 0.0, cm = 1.0, cm1 = 1.0;     // C(m, k), C(m-1, k) from k = 0 upwards
        double c[MF_MAX_MASS_RATIO_M + 1];
        for (int k = 0; k <= m; ++k) {
            c[k] = (m - 1) * cm - m * (k <= m - 1 ? cm1 : 0.0);
            cm = cm * (m - k) / (k + 1);
            cm1 = cm1 * (m - 1 - k) / (k + 1);
        }
        for (int k = m; k >= 2; --k) acc = acc * (-z) + c[k];
        dG = m * (m - 1) * pow(1.0 - z, m - 2) * z;
        return acc * z * z;
    }, 1.0 - r, sqrt((1.0 - r) / (0.5 * m * (m - 1))));
    return 1.0 - d;
}
// With derivatives: the root's value from the double solver, its tangent from
// the implicit function theorem, dx = -dd = dr / F'(x), F' = m(m-1) x^(m-2) (1-x).
template <int K>
MF_DEV Dual<K> mass_ratio(int m, const Dual<K> &r, Dual<K> &d) {
    double dv;
    double x = mass_ratio(m, r.v, dv);
    double xm2 = 1.0;
    for (int i = 0; i < m - 2; ++i) xm2 *= x;
    double dF = m * (m - 1) * xm2 * dv;
    double inv = dF > 0.0 ? 1.0 / dF : 0.0;
    d = chain(r, dv, -inv);
    return chain(r, x, inv);
}

// Flat massless n-body momenta in the centre-of-mass frame of energy rs from
// 3n-4 unit numbers u (per decay step: cos-theta, phi[, mass ratio]).
template <int N, typename T>
MF_DEV void massless_diet(const T *u, const T &rs, T p[N][4]) {
    T Q[4] = {rs, T(0.0), T(0.0), T(0.0)};
    T M = rs;
    int col = 0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
        T cth = 2.0 * u[col] - 1.0;
        T phi = 6.283185307179586 * u[col + 1];
        col += 2;
        int md = N - k - 1;
        T Mn = T(0.0), d = T(1.0);
        if (md >= 2) {
            T x = mass_ratio(md, u[col], d);
            col += 1;
            Mn = M * sqrt(x);
        }
        // daughter energy in the rest frame of Q: (M^2 - Mn^2) / (2M) = M (1 - x) / 2
        T e = 0.5 * M * d;
        T s2 = (1.0 - cth) * (1.0 + cth);
        T sth = value(s2) > 0.0 ? sqrt(s2) : T(0.0);
        T sp, cp;
        sincos(phi, &sp, &cp);
        T q[4] = {e, e * sth * cp, e * sth * sp, e * cth};
        T rest[4] = {M - e, -q[1], -q[2], -q[3]};
        T Qn[4];
        boost_from_rest(q, Q, M, p[k]);
        boost_from_rest(rest, Q, M, Qn);
        if (k == N - 2) {
            p[N - 1][0] = Qn[0]; p[N - 1][1] = Qn[1]; p[N - 1][2] = Qn[2]; p[N - 1][3] = Qn[3];
        }
        Q[0] = Qn[0]; Q[1] = Qn[1]; Q[2] = Qn[2]; Q[3] = Qn[3];
        M = Mn;
    }
}

// Newton solution of sum_i sqrt(m_i^2 + xi^2 E_i^2) = rs for xi (values only)
template <int N>
MF_DEV double rescale_factor(const double *E, const double *m, double rs) {
    double msum = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) msum += m[i];
    double r = msum / rs;
    double xi = sqrt((1.0 - r) * (1.0 + r));
    for (int it = 0; it < 50; ++it) {
        double f = -rs, d = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double e = sqrt(m[i] * m[i] + xi * xi * E[i] * E[i]);
            f += e;
            d += xi * E[i] * E[i] / e;
        }
        double step = f / d;
        xi -= step;
        if (fabs(step) <= 1e-15 * xi) break;
    }
    return xi;
}
MF_DEV double rescale_solve(const double *, const double *, double, double xi0, int) { return xi0; }
// with derivatives: one Newton step from the converged value carries the
// implicit-function tangent d xi = -dF / F'
template <int K>
MF_DEV Dual<K> rescale_solve(const Dual<K> *E, const Dual<K> *m, const Dual<K> &rs, double xi0, int n) {
    Dual<K> F = -rs;
    double dF = 0.0;
    for (int i = 0; i < n; ++i) {
        Dual<K> e = sqrt(m[i] * m[i] + xi0 * xi0 * E[i] * E[i]);
        F += e;
        dF += xi0 * E[i].v * E[i].v / e.v;
    }
    Dual<K> xi(xi0);
    return xi - F * (1.0 / dF);
}

// RAMBO massive rescaling (Kleiss, Stirling, Ellis, CPC 40 (1986) 359): scale
// the 3-momenta by xi with sum_i sqrt(m_i^2 + xi^2 E_i^2) = rs (Newton), and
// return the weight factor relative to the massless weight, or 0 below
// threshold.  p is replaced by the massive momenta.
template <int N, typename T>
MF_DEV T massive_rescale(T p[N][4], const T *m, const T &rs) {
    double msum = 0.0;
    bool any = false;
#pragma unroll
    for (int i = 0; i < N; ++i) { msum += value(m[i]); any |= (value(m[i]) != 0.0); }
    if (!(value(rs) > msum)) return T(0.0);
    if (!any) return T(1.0);
    double Ev[N], mv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) { Ev[i] = value(p[i][0]); mv[i] = value(m[i]); }
    const double xi0 = rescale_factor<N>(Ev, mv, value(rs));
    T E[N];
#pragma unroll
    for (int i = 0; i < N; ++i) E[i] = p[i][0];
    T xi = rescale_solve(E, m, rs, xi0, N);
    T sk = T(0.0), prod = T(1.0), sk2 = T(0.0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T kabs = xi * p[i][0];
        T k0 = sqrt(m[i] * m[i] + kabs * kabs);
        p[i][0] = k0;
        p[i][1] = p[i][1] * xi; p[i][2] = p[i][2] * xi; p[i][3] = p[i][3] * xi;
        sk += kabs;
        prod *= kabs / k0;
        sk2 += kabs * kabs / k0;
    }
    T a = sk / rs, pw = T(1.0);
#pragma unroll
    for (int i = 0; i < 2 * N - 3; ++i) pw *= a;
    return pw * prod * rs / sk2;
}

// ---------------------------------------------------------------- cuts
// pT^2 of a momentum
MF_DEV double pt2(const double *p) { return p[1] * p[1] + p[2] * p[2]; }
// Delta R^2 = Delta y^2 + Delta phi^2 between two momenta (phi in [0, pi])
MF_DEV double delta_r2(const double *a, const double *b) {
    // E - pz without cancellation for pz > 0: (m^2 + pT^2)/(E + pz)
    double apl = a[0] + fabs(a[3]), bpl = b[0] + fabs(b[3]);
    double am2 = fmax(0.0, (a[0] - a[3]) * (a[0] + a[3]) - pt2(a));
    double bm2 = fmax(0.0, (b[0] - b[3]) * (b[0] + b[3]) - pt2(b));
    double amin = (am2 + pt2(a)) / apl, bmin = (bm2 + pt2(b)) / bpl;
    double ap = a[3] >= 0 ? apl : amin, am = a[3] >= 0 ? amin : apl;   // E + pz, E - pz
    double bp = b[3] >= 0 ? bpl : bmin, bm = b[3] >= 0 ? bmin : bpl;
    double dy = 0.5 * log((ap * bm) / (am * bp));
    double cr = a[1] * b[2] - a[2] * b[1];
    double dt = a[1] * b[1] + a[2] * b[2];
    double dphi = atan2(fabs(cr), dt);
    return dy * dy + dphi * dphi;
}

// ---------------------------------------------------------------- PDF
// One beam's density at fixed mu_F^2, collapsed on the host to a single row of
// x f values over ln x knots (the ln Q^2 Hermite weights folded in) together
// with that row's knot slopes.  Cubic Hermite in ln x; returns f = (x f) / x.
template <typename T>
MF_DEV T pdf_eval(const double *row, const double *slope, int nx, double a0, double h, const T &ln_x, const T &x) {
    T s = (ln_x - a0) / h;
    int i = (int)floor(value(s));
    if (i < 0) i = 0;
    if (i > nx - 2) i = nx - 2;
    T t = s - (double)i;
    T t2 = t * t, t3 = t2 * t;
    T v = (2.0 * t3 - 3.0 * t2 + 1.0) * row[i] + (t3 - 2.0 * t2 + t) * (h * slope[i])
        + (-2.0 * t3 + 3.0 * t2) * row[i + 1] + (t3 - t2) * (h * slope[i + 1]);
    return v / x;
}

}  // namespace mf
