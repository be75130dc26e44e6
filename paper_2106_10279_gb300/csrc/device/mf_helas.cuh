// Helicity wavefunctions and vertex routines of the diagram program (Sec. 2.3:
// "ALOHA waveforms and vertices"), written from the Feynman rules in the chiral
// representation: gamma^0 = [[0,1],[1,0]], gamma^k = [[0,s^k],[-s^k,0]], so that
// for a 4-vector V,  V-slash = [[0, A],[B, 0]] with
//   A = V^0 - V.sigma = [[V0-V3, -(V1 - iV2)], [-(V1 + iV2), V0+V3]],
//   B = V^0 + V.sigma = [[V0+V3,  (V1 - iV2)], [ (V1 + iV2), V0-V3]].
// External states follow the HELAS helicity conventions (KEK-91-11):
//   u(p,l) = (sqrt(E - lP) chi_l, sqrt(E + lP) chi_l),
//   v(p,l) = (-l sqrt(E + lP) chi_-l, l sqrt(E - lP) chi_-l),
//   chi_+ = (P+pz, px+ipy)/sqrt(2P(P+pz)), chi_- = (-px+ipy, P+pz)/sqrt(2P(P+pz)),
//   eps(k,l) = (-l e1 - i e2)/sqrt2, e1 = (0, ct cp, ct sp, -st), e2 = (0, -sp, cp, 0).
// Branch-free where the branch depends on the helicity (lanes of a warp may
// carry different helicities of the same event).
#pragma once
#include "mf_common.cuh"

namespace mf {

// two-component helicity eigenvectors chi_l of sigma.p-hat
template <typename R>
MF_DEV void chi(const R *p, int l, cx<R> &c0, cx<R> &c1) {
    R px = p[1], py = p[2], pz = p[3];
    R pt2 = px * px + py * py;
    R P = sqrt(pt2 + pz * pz);
    R ppz = (pz >= R(0)) ? P + pz : pt2 / (P - pz);     // P + pz without cancellation
    if (ppz > R(0)) {
        R inv = R(1) / sqrt(R(2) * P * ppz);
        if (l > 0) { c0 = C<R>(ppz * inv, R(0)); c1 = C<R>(px * inv, py * inv); }
        else       { c0 = C<R>(-px * inv, py * inv); c1 = C<R>(ppz * inv, R(0)); }
    } else if (P > R(0)) {   // along -z
        if (l > 0) { c0 = C<R>(R(0), R(0)); c1 = C<R>(R(1), R(0)); }
        else       { c0 = C<R>(R(-1), R(0)); c1 = C<R>(R(0), R(0)); }
    } else {                 // at rest: quantise along +z
        if (l > 0) { c0 = C<R>(R(1), R(0)); c1 = C<R>(R(0), R(0)); }
        else       { c0 = C<R>(R(0), R(0)); c1 = C<R>(R(1), R(0)); }
    }
}

// sqrt(E - P) and sqrt(E + P) without cancellation: E - P = m^2 / (E + P)
template <typename R>
MF_DEV void omegas(const R *p, R m, R &wm, R &wp) {
    R P = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    R s = sqrt(p[0] + P);
    wp = s;
    wm = (m > R(0)) ? m / s : R(0);
}

// Column spinor (flow-in): u of an incoming particle (anti=0) or v of an
// outgoing antiparticle (anti=1).
template <typename R>
MF_DEV W<R> ixx(const R *p, R m, int l, int anti) {
    W<R> w;
    R wm, wp;
    omegas(p, m, wm, wp);
    cx<R> c0, c1;
    if (!anti) {
        chi(p, l, c0, c1);
        R a = (l > 0) ? wm : wp, b = (l > 0) ? wp : wm;        // sqrt(E - lP), sqrt(E + lP)
        w.c[0] = a * c0; w.c[1] = a * c1; w.c[2] = b * c0; w.c[3] = b * c1;
    } else {
        chi(p, -l, c0, c1);
        R c = (l > 0) ? -wp : wm, d = (l > 0) ? wm : -wp;      // -l sqrt(E + lP), l sqrt(E - lP)
        w.c[0] = c * c0; w.c[1] = c * c1; w.c[2] = d * c0; w.c[3] = d * c1;
    }
    return w;
}

// Row spinor (flow-out): u-bar of an outgoing particle (anti=0) or v-bar of an
// incoming antiparticle (anti=1).  psi-bar = psi^dagger gamma^0.
template <typename R>
MF_DEV W<R> oxx(const R *p, R m, int l, int anti) {
    W<R> col = ixx(p, m, l, anti);
    W<R> w;
    w.c[0] = conj(col.c[2]); w.c[1] = conj(col.c[3]);
    w.c[2] = conj(col.c[0]); w.c[3] = conj(col.c[1]);
    return w;
}

// Massless vector: eps(k, l) for incoming, eps*(k, l) for outgoing.
template <typename R>
MF_DEV W<R> vxx(const R *k, int l, int incoming) {
    W<R> w;
    R kx = k[1], ky = k[2], kz = k[3];
    R kt = sqrt(kx * kx + ky * ky);
    R K = sqrt(kt * kt + kz * kz);
    R st, ct, sp, cp;
    if (kt > R(0)) { st = kt / K; ct = kz / K; cp = kx / kt; sp = ky / kt; }
    else { st = R(0); ct = (kz >= R(0)) ? R(1) : R(-1); cp = R(1); sp = R(0); }
    const R rs2 = R(0.70710678118654752440);
    R lr = R(-l) * rs2;                // -l/sqrt2 times e1
    R im_sign = incoming ? R(-1) : R(1);    // -i e2 (incoming), +i e2 (conjugated)
    w.c[0] = C<R>(R(0), R(0));
    w.c[1] = C<R>(lr * ct * cp, im_sign * rs2 * (-sp));
    w.c[2] = C<R>(lr * ct * sp, im_sign * rs2 * cp);
    w.c[3] = C<R>(lr * (-st), R(0));
    return w;
}

// ---------------------------------------------------------------- Dirac algebra
// (V-slash) psi for a column psi
template <typename R>
MF_DEV void vslash_col(const cx<R> *V, const cx<R> *s, cx<R> *o) {
    cx<R> vm = V[1] - mul_i(V[2]);   // V1 - i V2
    cx<R> vp = V[1] + mul_i(V[2]);   // V1 + i V2
    cx<R> a = V[0] - V[3], b = V[0] + V[3];
    o[0] = a * s[2] - vm * s[3];
    o[1] = b * s[3] - vp * s[2];
    o[2] = b * s[0] + vm * s[1];
    o[3] = vp * s[0] + a * s[1];
}
// psi-bar (V-slash) for a row psi-bar
template <typename R>
MF_DEV void vslash_row(const cx<R> *r, const cx<R> *V, cx<R> *o) {
    cx<R> vm = V[1] - mul_i(V[2]);
    cx<R> vp = V[1] + mul_i(V[2]);
    cx<R> a = V[0] - V[3], b = V[0] + V[3];
    o[0] = r[2] * b + r[3] * vp;
    o[1] = r[2] * vm + r[3] * a;
    o[2] = r[0] * a - r[1] * vp;
    o[3] = r[1] * b - r[0] * vm;
}
// (q-slash + M) psi for real q
template <typename R>
MF_DEV void qslash_col(const R *q, R M, const cx<R> *s, cx<R> *o) {
    cx<R> qm = C<R>(q[1], -q[2]), qp = C<R>(q[1], q[2]);
    R a = q[0] - q[3], b = q[0] + q[3];
    o[0] = a * s[2] - qm * s[3] + M * s[0];
    o[1] = b * s[3] - qp * s[2] + M * s[1];
    o[2] = b * s[0] + qm * s[1] + M * s[2];
    o[3] = qp * s[0] + a * s[1] + M * s[3];
}
template <typename R>
MF_DEV void qslash_row(const cx<R> *r, const R *q, R M, cx<R> *o) {
    cx<R> qm = C<R>(q[1], -q[2]), qp = C<R>(q[1], q[2]);
    R a = q[0] - q[3], b = q[0] + q[3];
    o[0] = b * r[2] + qp * r[3] + M * r[0];
    o[1] = qm * r[2] + a * r[3] + M * r[1];
    o[2] = a * r[0] - qp * r[1] + M * r[2];
    o[3] = b * r[1] - qm * r[0] + M * r[3];
}

// ---------------------------------------------------------------- vertices
// PH: the phase class of the coupling g (pmul); 0 keeps every product general.
template <typename R, int PH = 0>
MF_DEV cx<R> FFV_AMP(const W<R> &row, const W<R> &col, const W<R> &V, cx<R> g) {
    cx<R> t[4];
    vslash_col(V.c, col.c, t);
    cx<R> s = row.c[0] * t[0];
    s = cfma(row.c[1], t[1], s);
    s = cfma(row.c[2], t[2], s);
    s = cfma(row.c[3], t[3], s);
    return pmul<PH>(g, s);
}

// Two amplitudes of a helicity pair that share everything but one external
// spinor: row_a and row_b (the row spinor differs) share (V-slash) col, and
// col_a and col_b (the column spinor differs) share row (V-slash).
template <typename R>
struct A2 {
    cx<R> a, b;
};

template <typename R, int PH = 0>
MF_DEV A2<R> FFV_AMP_R2(const W<R> &row_a, const W<R> &row_b, const W<R> &col, const W<R> &V, cx<R> g) {
    cx<R> t[4];
    vslash_col(V.c, col.c, t);
    cx<R> sa = row_a.c[0] * t[0], sb = row_b.c[0] * t[0];
    for (int k = 1; k < 4; ++k) {
        sa = cfma(row_a.c[k], t[k], sa);
        sb = cfma(row_b.c[k], t[k], sb);
    }
    return A2<R>{pmul<PH>(g, sa), pmul<PH>(g, sb)};
}

template <typename R, int PH = 0>
MF_DEV A2<R> FFV_AMP_C2(const W<R> &row, const W<R> &col_a, const W<R> &col_b, const W<R> &V, cx<R> g) {
    cx<R> t[4];
    vslash_row(row.c, V.c, t);
    cx<R> sa = t[0] * col_a.c[0], sb = t[0] * col_b.c[0];
    for (int k = 1; k < 4; ++k) {
        sa = cfma(t[k], col_a.c[k], sa);
        sb = cfma(t[k], col_b.c[k], sb);
    }
    return A2<R>{pmul<PH>(g, sa), pmul<PH>(g, sb)};
}

// P: momentum of the new current (into the diagram through its legs)
template <typename R, int PH = 0>
MF_DEV W<R> FFV_FIN(const W<R> &col, const W<R> &V, cx<R> g, R M, R inv_den, const R *P) {
    W<R> w;
    cx<R> t[4], u[4];
    vslash_col(V.c, col.c, t);
    qslash_col(P, M, t, u);
    cx<R> f = mul_i(g) * inv_den;
    for (int k = 0; k < 4; ++k) w.c[k] = pmul<rotate_phase(PH)>(f, u[k]);
    return w;
}

template <typename R, int PH = 0>
MF_DEV W<R> FFV_FOUT(const W<R> &row, const W<R> &V, cx<R> g, R M, R inv_den, const R *P) {
    W<R> w;
    R q[4] = {-P[0], -P[1], -P[2], -P[3]};
    cx<R> t[4], u[4];
    vslash_row(row.c, V.c, t);
    qslash_row(t, q, M, u);
    cx<R> f = mul_i(g) * inv_den;
    for (int k = 0; k < 4; ++k) w.c[k] = pmul<rotate_phase(PH)>(f, u[k]);
    return w;
}

template <typename R, int PH = 0>
MF_DEV W<R> FFV_VEC(const W<R> &row, const W<R> &col, cx<R> g, R inv_den) {
    W<R> w;
    const cx<R> *a = row.c, *s = col.c;
    cx<R> j0 = a[0] * s[2] + a[1] * s[3] + a[2] * s[0] + a[3] * s[1];
    cx<R> j1 = a[0] * s[3] + a[1] * s[2] - a[2] * s[1] - a[3] * s[0];
    cx<R> j2 = mul_i(a[1] * s[2] - a[0] * s[3] + a[2] * s[1] - a[3] * s[0]);
    cx<R> j3 = a[0] * s[2] - a[1] * s[3] - a[2] * s[0] + a[3] * s[1];
    cx<R> f = mul_mi(g) * inv_den;
    constexpr int F = rotate_phase(PH);
    w.c[0] = pmul<F>(f, j0); w.c[1] = pmul<F>(f, j1); w.c[2] = pmul<F>(f, j2); w.c[3] = pmul<F>(f, j3);
    return w;
}

// kA, kB, kC: momenta into the vertex along A, B, C
template <typename R, int PH = 0>
MF_DEV cx<R> VVV_AMP(const W<R> &A, const W<R> &B, const W<R> &Cv, const R *kA, const R *kB, const R *kC,
                     cx<R> g) {
    R d12[4], d23[4], d31[4];
    for (int k = 0; k < 4; ++k) {
        d12[k] = kA[k] - kB[k];
        d23[k] = kB[k] - kC[k];
        d31[k] = kC[k] - kA[k];
    }
    cx<R> r = mdot(A.c, B.c) * mdot(d12, Cv.c);
    r = cfma(mdot(B.c, Cv.c), mdot(d23, A.c), r);
    r = cfma(mdot(Cv.c, A.c), mdot(d31, B.c), r);
    return pmul<PH>(g, r);
}

template <typename R, int PH = 0>
MF_DEV W<R> VVV_VEC(const W<R> &A, const W<R> &B, const R *kA, const R *kB, cx<R> g, R inv_den) {
    W<R> w;
    R d12[4], d23[4], d31[4];
    for (int k = 0; k < 4; ++k) {
        // k3 = -(kA + kB):  kB - k3 = kA + 2 kB,  k3 - kA = -2 kA - kB
        d12[k] = kA[k] - kB[k];
        d23[k] = kA[k] + R(2) * kB[k];
        d31[k] = -R(2) * kA[k] - kB[k];
    }
    cx<R> ab = mdot(A.c, B.c);
    cx<R> fb = mdot(d23, A.c);
    cx<R> fa = mdot(d31, B.c);
    cx<R> f = mul_mi(g) * inv_den;
    for (int k = 0; k < 4; ++k) {
        cx<R> v = ab * d12[k];
        v = cfma(B.c[k], fb, v);
        v = cfma(A.c[k], fa, v);
        w.c[k] = pmul<rotate_phase(PH)>(f, v);
    }
    return w;
}

template <typename R, int S, int PH = 0>
MF_DEV cx<R> VVVV_AMP(const W<R> &A, const W<R> &B, const W<R> &Cv, const W<R> &D, cx<R> g) {
    cx<R> r;
    if (S == 1) r = mdot(A.c, Cv.c) * mdot(B.c, D.c) - mdot(A.c, D.c) * mdot(B.c, Cv.c);
    else if (S == 2) r = mdot(A.c, B.c) * mdot(Cv.c, D.c) - mdot(A.c, D.c) * mdot(B.c, Cv.c);
    else r = mdot(A.c, B.c) * mdot(Cv.c, D.c) - mdot(A.c, Cv.c) * mdot(B.c, D.c);
    return pmul<PH>(g, r);
}

template <typename R, int S, int PH = 0>
MF_DEV W<R> VVVV_VEC(const W<R> &A, const W<R> &B, const W<R> &Cv, cx<R> g, R inv_den) {
    W<R> w;
    cx<R> f = mul_mi(g) * inv_den;
    cx<R> x, y;
    const W<R> *X, *Y;
    if (S == 1) { x = mdot(A.c, Cv.c); X = &B; y = mdot(B.c, Cv.c); Y = &A; }
    else if (S == 2) { x = mdot(A.c, B.c); X = &Cv; y = mdot(B.c, Cv.c); Y = &A; }
    else { x = mdot(A.c, B.c); X = &Cv; y = mdot(A.c, Cv.c); Y = &B; }
    for (int k = 0; k < 4; ++k) w.c[k] = pmul<rotate_phase(PH)>(f, x * X->c[k] - y * Y->c[k]);
    return w;
}


// The vertex routines as non-inlined functions taking everything by value
// (momenta as four scalars): a program made of calls to these holds one copy
// of each routine's code.
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define MF_NOINL __device__ __noinline__
#else
#define MF_NOINL inline
#endif
template <typename R, int PH = 0>
MF_NOINL W<R> nFFV_FIN(W<R> col, W<R> V, cx<R> g, R M, R inv_den, R p0, R p1, R p2, R p3) {
    const R P[4] = {p0, p1, p2, p3};
    return FFV_FIN<R, PH>(col, V, g, M, inv_den, P);
}
template <typename R, int PH = 0>
MF_NOINL W<R> nFFV_FOUT(W<R> row, W<R> V, cx<R> g, R M, R inv_den, R p0, R p1, R p2, R p3) {
    const R P[4] = {p0, p1, p2, p3};
    return FFV_FOUT<R, PH>(row, V, g, M, inv_den, P);
}
template <typename R, int PH = 0>
MF_NOINL W<R> nFFV_VEC(W<R> row, W<R> col, cx<R> g, R inv_den) { return FFV_VEC<R, PH>(row, col, g, inv_den); }
template <typename R, int PH = 0>
MF_NOINL W<R> nVVV_VEC(W<R> A, W<R> B, R a0, R a1, R a2, R a3, R b0, R b1, R b2, R b3, cx<R> g, R inv_den) {
    const R kA[4] = {a0, a1, a2, a3}, kB[4] = {b0, b1, b2, b3};
    return VVV_VEC<R, PH>(A, B, kA, kB, g, inv_den);
}
template <typename R, int S, int PH = 0>
MF_NOINL W<R> nVVVV_VEC(W<R> A, W<R> B, W<R> Cv, cx<R> g, R inv_den) {
    return VVVV_VEC<R, S, PH>(A, B, Cv, g, inv_den);
}
template <typename R, int PH = 0>
MF_NOINL cx<R> nFFV_AMP(W<R> row, W<R> col, W<R> V, cx<R> g) { return FFV_AMP<R, PH>(row, col, V, g); }
template <typename R, int PH = 0>
MF_NOINL A2<R> nFFV_AMP_R2(W<R> row_a, W<R> row_b, W<R> col, W<R> V, cx<R> g) {
    return FFV_AMP_R2<R, PH>(row_a, row_b, col, V, g);
}
template <typename R, int PH = 0>
MF_NOINL A2<R> nFFV_AMP_C2(W<R> row, W<R> col_a, W<R> col_b, W<R> V, cx<R> g) {
    return FFV_AMP_C2<R, PH>(row, col_a, col_b, V, g);
}
template <typename R, int PH = 0>
MF_NOINL cx<R> nVVV_AMP(W<R> A, W<R> B, W<R> Cv, R a0, R a1, R a2, R a3, R b0, R b1, R b2, R b3, R c0, R c1, R c2,
                        R c3, cx<R> g) {
    const R kA[4] = {a0, a1, a2, a3}, kB[4] = {b0, b1, b2, b3}, kC[4] = {c0, c1, c2, c3};
    return VVV_AMP<R, PH>(A, B, Cv, kA, kB, kC, g);
}
template <typename R, int S, int PH = 0>
MF_NOINL cx<R> nVVVV_AMP(W<R> A, W<R> B, W<R> Cv, W<R> D, cx<R> g) { return VVVV_AMP<R, S, PH>(A, B, Cv, D, g); }
#undef MF_NOINL

}  // namespace mf
