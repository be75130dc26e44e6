// Adjoints (reverse-mode derivatives) of the vertex routines in mf_helas.cuh,
// for the gradient kernel.  Convention: for a real objective L and a complex
// quantity z = x + i y the adjoint is zb = dL/dx + i dL/dy; then
//   z = u + v   ->  ub += zb,            vb += zb
//   z = u v     ->  ub += zb conj(v),    vb += zb conj(u)
//   z = c u     ->  ub += zb conj(c)     (c a constant)
//   z = s u     ->  sb += Re(zb conj(u)) (s real)
// Every routine recomputes the intermediate values it needs from its inputs
// (nothing is stored by the forward sweep beyond the wavefunctions), and ADDS
// into the adjoint arrays it is given.
#pragma once
#include "mf_dual.cuh"
#include "mf_helas.cuh"

namespace mf {

template <typename R> MF_DEV R re(const cx<R> &a) { return a.re; }
template <typename R> MF_DEV cx<R> &operator+=(cx<R> &a, const cx<R> &b) { a = a + b; return a; }
template <typename R> MF_DEV cx<R> &operator-=(cx<R> &a, const cx<R> &b) { a = a - b; return a; }

// --------------------------------------------------------------- primitives
// o = (V-slash) s
template <typename R>
MF_DEV void vslash_col_adj(const cx<R> *V, const cx<R> *s, const cx<R> *ob, cx<R> *Vb, cx<R> *sb) {
    cx<R> vm = V[1] - mul_i(V[2]), vp = V[1] + mul_i(V[2]);
    cx<R> a = V[0] - V[3], b = V[0] + V[3];
    // o0 = a s2 - vm s3; o1 = b s3 - vp s2; o2 = b s0 + vm s1; o3 = vp s0 + a s1
    cx<R> ab = ob[0] * conj(s[2]) + ob[3] * conj(s[1]);
    cx<R> bb = ob[1] * conj(s[3]) + ob[2] * conj(s[0]);
    cx<R> vmb = ob[2] * conj(s[1]) - ob[0] * conj(s[3]);
    cx<R> vpb = ob[3] * conj(s[0]) - ob[1] * conj(s[2]);
    sb[0] += ob[2] * conj(b) + ob[3] * conj(vp);
    sb[1] += ob[2] * conj(vm) + ob[3] * conj(a);
    sb[2] += ob[0] * conj(a) - ob[1] * conj(vp);
    sb[3] += ob[1] * conj(b) - ob[0] * conj(vm);
    // a = V0 - V3, b = V0 + V3, vm = V1 - i V2, vp = V1 + i V2
    Vb[0] += ab + bb;
    Vb[3] += bb - ab;
    Vb[1] += vmb + vpb;
    Vb[2] += mul_i(vmb) - mul_i(vpb);
}

// o = r (V-slash)
template <typename R>
MF_DEV void vslash_row_adj(const cx<R> *r, const cx<R> *V, const cx<R> *ob, cx<R> *rb, cx<R> *Vb) {
    cx<R> vm = V[1] - mul_i(V[2]), vp = V[1] + mul_i(V[2]);
    cx<R> a = V[0] - V[3], b = V[0] + V[3];
    // o0 = r2 b + r3 vp; o1 = r2 vm + r3 a; o2 = r0 a - r1 vp; o3 = r1 b - r0 vm
    rb[0] += ob[2] * conj(a) - ob[3] * conj(vm);
    rb[1] += ob[3] * conj(b) - ob[2] * conj(vp);
    rb[2] += ob[0] * conj(b) + ob[1] * conj(vm);
    rb[3] += ob[0] * conj(vp) + ob[1] * conj(a);
    cx<R> ab = ob[1] * conj(r[3]) + ob[2] * conj(r[0]);
    cx<R> bb = ob[0] * conj(r[2]) + ob[3] * conj(r[1]);
    cx<R> vmb = ob[1] * conj(r[2]) - ob[3] * conj(r[0]);
    cx<R> vpb = ob[0] * conj(r[3]) - ob[2] * conj(r[1]);
    Vb[0] += ab + bb;
    Vb[3] += bb - ab;
    Vb[1] += vmb + vpb;
    Vb[2] += mul_i(vmb) - mul_i(vpb);
}

// o = (q-slash + M) s, q real
template <typename R>
MF_DEV void qslash_col_adj(const R *q, R M, const cx<R> *s, const cx<R> *ob, R *qb, R &Mb, cx<R> *sb) {
    cx<R> qm = C<R>(q[1], -q[2]), qp = C<R>(q[1], q[2]);
    R a = q[0] - q[3], b = q[0] + q[3];
    // o0 = a s2 - qm s3 + M s0; o1 = b s3 - qp s2 + M s1
    // o2 = b s0 + qm s1 + M s2; o3 = qp s0 + a s1 + M s3
    sb[0] += ob[0] * M + ob[2] * b + ob[3] * conj(qp);
    sb[1] += ob[1] * M + ob[2] * conj(qm) + ob[3] * a;
    sb[2] += ob[0] * a - ob[1] * conj(qp) + ob[2] * M;
    sb[3] += ob[1] * b - ob[0] * conj(qm) + ob[3] * M;
    R ab = re(ob[0] * conj(s[2])) + re(ob[3] * conj(s[1]));
    R bb = re(ob[1] * conj(s[3])) + re(ob[2] * conj(s[0]));
    cx<R> qmb = ob[2] * conj(s[1]) - ob[0] * conj(s[3]);
    cx<R> qpb = ob[3] * conj(s[0]) - ob[1] * conj(s[2]);
    Mb += re(ob[0] * conj(s[0])) + re(ob[1] * conj(s[1])) + re(ob[2] * conj(s[2])) + re(ob[3] * conj(s[3]));
    qb[0] += ab + bb;
    qb[3] += bb - ab;
    // qm = q1 - i q2, qp = q1 + i q2
    qb[1] += qmb.re + qpb.re;
    qb[2] += qpb.im - qmb.im;
}

// o = r (q-slash + M), q real
template <typename R>
MF_DEV void qslash_row_adj(const cx<R> *r, const R *q, R M, const cx<R> *ob, cx<R> *rb, R *qb, R &Mb) {
    cx<R> qm = C<R>(q[1], -q[2]), qp = C<R>(q[1], q[2]);
    R a = q[0] - q[3], b = q[0] + q[3];
    // o0 = b r2 + qp r3 + M r0; o1 = qm r2 + a r3 + M r1
    // o2 = a r0 - qp r1 + M r2; o3 = b r1 - qm r0 + M r3
    rb[0] += ob[0] * M + ob[2] * a - ob[3] * conj(qm);
    rb[1] += ob[1] * M - ob[2] * conj(qp) + ob[3] * b;
    rb[2] += ob[0] * b + ob[1] * conj(qm) + ob[2] * M;
    rb[3] += ob[0] * conj(qp) + ob[1] * a + ob[3] * M;
    R ab = re(ob[1] * conj(r[3])) + re(ob[2] * conj(r[0]));
    R bb = re(ob[0] * conj(r[2])) + re(ob[3] * conj(r[1]));
    cx<R> qmb = ob[1] * conj(r[2]) - ob[3] * conj(r[0]);
    cx<R> qpb = ob[0] * conj(r[3]) - ob[2] * conj(r[1]);
    Mb += re(ob[0] * conj(r[0])) + re(ob[1] * conj(r[1])) + re(ob[2] * conj(r[2])) + re(ob[3] * conj(r[3]));
    qb[0] += ab + bb;
    qb[3] += bb - ab;
    qb[1] += qmb.re + qpb.re;
    qb[2] += qpb.im - qmb.im;
}

// r = a.b (Minkowski, no conjugation)
template <typename R>
MF_DEV void mdot_adj(const cx<R> *a, const cx<R> *b, cx<R> rb, cx<R> *abar, cx<R> *bbar) {
    abar[0] += rb * conj(b[0]); bbar[0] += rb * conj(a[0]);
    for (int k = 1; k < 4; ++k) { abar[k] -= rb * conj(b[k]); bbar[k] -= rb * conj(a[k]); }
}
// r = k.b with k real
template <typename R>
MF_DEV void mdot_adj(const R *k, const cx<R> *b, cx<R> rb, R *kbar, cx<R> *bbar) {
    kbar[0] += re(rb * conj(b[0])); bbar[0] += rb * k[0];
    for (int q = 1; q < 4; ++q) { kbar[q] -= re(rb * conj(b[q])); bbar[q] -= rb * k[q]; }
}

// --------------------------------------------------------------- routines
template <typename R>
MF_DEV void FFV_AMP_adj(const W<R> &row, const W<R> &col, const W<R> &V, cx<R> g, cx<R> ab, W<R> &rowb,
                        W<R> &colb, W<R> &Vb) {
    cx<R> t[4], tb[4];
    vslash_col(V.c, col.c, t);
    cx<R> sb = ab * conj(g);
    for (int k = 0; k < 4; ++k) {
        rowb.c[k] += sb * conj(t[k]);
        tb[k] = sb * conj(row.c[k]);
    }
    vslash_col_adj(V.c, col.c, tb, Vb.c, colb.c);
}

template <typename R>
MF_DEV void FFV_FIN_adj(const W<R> &col, const W<R> &V, cx<R> g, R M, R inv_den, const R *P, const W<R> &wb,
                        W<R> &colb, W<R> &Vb, R &invb, R *Pb, R &Mb) {
    cx<R> t[4], u[4], ub[4], tb[4] = {};
    vslash_col(V.c, col.c, t);
    qslash_col(P, M, t, u);
    cx<R> f = mul_i(g) * inv_den;
    cx<R> fb = C<R>(R(0), R(0));
    for (int k = 0; k < 4; ++k) {
        ub[k] = wb.c[k] * conj(f);
        fb += wb.c[k] * conj(u[k]);
    }
    invb += re(fb * conj(mul_i(g)));
    qslash_col_adj(P, M, t, ub, Pb, Mb, tb);
    vslash_col_adj(V.c, col.c, tb, Vb.c, colb.c);
}

template <typename R>
MF_DEV void FFV_FOUT_adj(const W<R> &row, const W<R> &V, cx<R> g, R M, R inv_den, const R *P, const W<R> &wb,
                         W<R> &rowb, W<R> &Vb, R &invb, R *Pb, R &Mb) {
    R q[4] = {-P[0], -P[1], -P[2], -P[3]};
    cx<R> t[4], u[4], ub[4], tb[4] = {};
    vslash_row(row.c, V.c, t);
    qslash_row(t, q, M, u);
    cx<R> f = mul_i(g) * inv_den;
    cx<R> fb = C<R>(R(0), R(0));
    for (int k = 0; k < 4; ++k) {
        ub[k] = wb.c[k] * conj(f);
        fb += wb.c[k] * conj(u[k]);
    }
    invb += re(fb * conj(mul_i(g)));
    R qb[4] = {R(0), R(0), R(0), R(0)};
    qslash_row_adj(t, q, M, ub, tb, qb, Mb);
    for (int k = 0; k < 4; ++k) Pb[k] -= qb[k];
    vslash_row_adj(row.c, V.c, tb, rowb.c, Vb.c);
}

template <typename R>
MF_DEV void FFV_VEC_adj(const W<R> &row, const W<R> &col, cx<R> g, R inv_den, const W<R> &wb, W<R> &rowb,
                        W<R> &colb, R &invb) {
    const cx<R> *a = row.c, *s = col.c;
    cx<R> j[4];
    j[0] = a[0] * s[2] + a[1] * s[3] + a[2] * s[0] + a[3] * s[1];
    j[1] = a[0] * s[3] + a[1] * s[2] - a[2] * s[1] - a[3] * s[0];
    j[2] = mul_i(a[1] * s[2] - a[0] * s[3] + a[2] * s[1] - a[3] * s[0]);
    j[3] = a[0] * s[2] - a[1] * s[3] - a[2] * s[0] + a[3] * s[1];
    cx<R> f = mul_mi(g) * inv_den;
    cx<R> jb[4], fb = C<R>(R(0), R(0));
    for (int k = 0; k < 4; ++k) {
        jb[k] = wb.c[k] * conj(f);
        fb += wb.c[k] * conj(j[k]);
    }
    invb += re(fb * conj(mul_mi(g)));
    cx<R> Xb = mul_mi(jb[2]);   // j2 = i X
    cx<R> *ab = rowb.c, *sb = colb.c;
    ab[0] += jb[0] * conj(s[2]) + jb[1] * conj(s[3]) - Xb * conj(s[3]) + jb[3] * conj(s[2]);
    ab[1] += jb[0] * conj(s[3]) + jb[1] * conj(s[2]) + Xb * conj(s[2]) - jb[3] * conj(s[3]);
    ab[2] += jb[0] * conj(s[0]) - jb[1] * conj(s[1]) + Xb * conj(s[1]) - jb[3] * conj(s[0]);
    ab[3] += jb[0] * conj(s[1]) - jb[1] * conj(s[0]) - Xb * conj(s[0]) + jb[3] * conj(s[1]);
    sb[0] += jb[0] * conj(a[2]) - jb[1] * conj(a[3]) - Xb * conj(a[3]) - jb[3] * conj(a[2]);
    sb[1] += jb[0] * conj(a[3]) - jb[1] * conj(a[2]) + Xb * conj(a[2]) + jb[3] * conj(a[3]);
    sb[2] += jb[0] * conj(a[0]) + jb[1] * conj(a[1]) + Xb * conj(a[1]) + jb[3] * conj(a[0]);
    sb[3] += jb[0] * conj(a[1]) + jb[1] * conj(a[0]) - Xb * conj(a[0]) - jb[3] * conj(a[1]);
}

template <typename R>
MF_DEV void VVV_AMP_adj(const W<R> &A, const W<R> &B, const W<R> &Cv, const R *kA, const R *kB, const R *kC,
                        cx<R> g, cx<R> ab, W<R> &Ab, W<R> &Bb, W<R> &Cb, R *kAb, R *kBb, R *kCb) {
    R d12[4], d23[4], d31[4];
    for (int k = 0; k < 4; ++k) {
        d12[k] = kA[k] - kB[k];
        d23[k] = kB[k] - kC[k];
        d31[k] = kC[k] - kA[k];
    }
    cx<R> AB = mdot(A.c, B.c), BC = mdot(B.c, Cv.c), CA = mdot(Cv.c, A.c);
    cx<R> x12 = mdot(d12, Cv.c), x23 = mdot(d23, A.c), x31 = mdot(d31, B.c);
    cx<R> rb = ab * conj(g);
    R d12b[4] = {}, d23b[4] = {}, d31b[4] = {};
    mdot_adj(A.c, B.c, rb * conj(x12), Ab.c, Bb.c);
    mdot_adj(d12, Cv.c, rb * conj(AB), d12b, Cb.c);
    mdot_adj(B.c, Cv.c, rb * conj(x23), Bb.c, Cb.c);
    mdot_adj(d23, A.c, rb * conj(BC), d23b, Ab.c);
    mdot_adj(Cv.c, A.c, rb * conj(x31), Cb.c, Ab.c);
    mdot_adj(d31, B.c, rb * conj(CA), d31b, Bb.c);
    for (int k = 0; k < 4; ++k) {
        kAb[k] += d12b[k] - d31b[k];
        kBb[k] += d23b[k] - d12b[k];
        kCb[k] += d31b[k] - d23b[k];
    }
}

template <typename R>
MF_DEV void VVV_VEC_adj(const W<R> &A, const W<R> &B, const R *kA, const R *kB, cx<R> g, R inv_den,
                        const W<R> &wb, W<R> &Ab, W<R> &Bb, R &invb, R *kAb, R *kBb) {
    R d12[4], d23[4], d31[4];
    for (int k = 0; k < 4; ++k) {
        d12[k] = kA[k] - kB[k];
        d23[k] = kA[k] + R(2) * kB[k];
        d31[k] = -R(2) * kA[k] - kB[k];
    }
    cx<R> abv = mdot(A.c, B.c), fbv = mdot(d23, A.c), fav = mdot(d31, B.c);
    cx<R> f = mul_mi(g) * inv_den;
    cx<R> vb[4], fb = C<R>(R(0), R(0));
    for (int k = 0; k < 4; ++k) {
        cx<R> v = abv * d12[k];
        v = cfma(B.c[k], fbv, v);
        v = cfma(A.c[k], fav, v);
        vb[k] = wb.c[k] * conj(f);
        fb += wb.c[k] * conj(v);
    }
    invb += re(fb * conj(mul_mi(g)));
    cx<R> abb = C<R>(R(0), R(0)), fbb = C<R>(R(0), R(0)), fab = C<R>(R(0), R(0));
    R d12b[4], d23b[4] = {}, d31b[4] = {};
    for (int k = 0; k < 4; ++k) {
        abb += vb[k] * d12[k];
        d12b[k] = re(vb[k] * conj(abv));
        Bb.c[k] += vb[k] * conj(fbv);
        fbb += vb[k] * conj(B.c[k]);
        Ab.c[k] += vb[k] * conj(fav);
        fab += vb[k] * conj(A.c[k]);
    }
    mdot_adj(A.c, B.c, abb, Ab.c, Bb.c);
    mdot_adj(d23, A.c, fbb, d23b, Ab.c);
    mdot_adj(d31, B.c, fab, d31b, Bb.c);
    for (int k = 0; k < 4; ++k) {
        kAb[k] += d12b[k] + d23b[k] - R(2) * d31b[k];
        kBb[k] += -d12b[k] + R(2) * d23b[k] - d31b[k];
    }
}

template <typename R, int S>
MF_DEV void VVVV_AMP_adj(const W<R> &A, const W<R> &B, const W<R> &Cv, const W<R> &D, cx<R> g, cx<R> ab,
                         W<R> &Ab, W<R> &Bb, W<R> &Cb, W<R> &Db) {
    cx<R> rb = ab * conj(g);
    // r = x1 y1 - x2 y2 for the structure's pairs
    const W<R> *x1a, *x1b, *y1a, *y1b, *x2a, *x2b, *y2a, *y2b;
    W<R> *x1ab, *x1bb, *y1ab, *y1bb, *x2ab, *x2bb, *y2ab, *y2bb;
    if (S == 1) {        // (A.C)(B.D) - (A.D)(B.C)
        x1a = &A; x1b = &Cv; y1a = &B; y1b = &D; x2a = &A; x2b = &D; y2a = &B; y2b = &Cv;
        x1ab = &Ab; x1bb = &Cb; y1ab = &Bb; y1bb = &Db; x2ab = &Ab; x2bb = &Db; y2ab = &Bb; y2bb = &Cb;
    } else if (S == 2) { // (A.B)(C.D) - (A.D)(B.C)
        x1a = &A; x1b = &B; y1a = &Cv; y1b = &D; x2a = &A; x2b = &D; y2a = &B; y2b = &Cv;
        x1ab = &Ab; x1bb = &Bb; y1ab = &Cb; y1bb = &Db; x2ab = &Ab; x2bb = &Db; y2ab = &Bb; y2bb = &Cb;
    } else {             // (A.B)(C.D) - (A.C)(B.D)
        x1a = &A; x1b = &B; y1a = &Cv; y1b = &D; x2a = &A; x2b = &Cv; y2a = &B; y2b = &D;
        x1ab = &Ab; x1bb = &Bb; y1ab = &Cb; y1bb = &Db; x2ab = &Ab; x2bb = &Cb; y2ab = &Bb; y2bb = &Db;
    }
    cx<R> x1 = mdot(x1a->c, x1b->c), y1 = mdot(y1a->c, y1b->c);
    cx<R> x2 = mdot(x2a->c, x2b->c), y2 = mdot(y2a->c, y2b->c);
    mdot_adj(x1a->c, x1b->c, rb * conj(y1), x1ab->c, x1bb->c);
    mdot_adj(y1a->c, y1b->c, rb * conj(x1), y1ab->c, y1bb->c);
    mdot_adj(x2a->c, x2b->c, -(rb * conj(y2)), x2ab->c, x2bb->c);
    mdot_adj(y2a->c, y2b->c, -(rb * conj(x2)), y2ab->c, y2bb->c);
}

template <typename R, int S>
MF_DEV void VVVV_VEC_adj(const W<R> &A, const W<R> &B, const W<R> &Cv, cx<R> g, R inv_den, const W<R> &wb,
                         W<R> &Ab, W<R> &Bb, W<R> &Cb, R &invb) {
    // w = f (x X - y Y)
    const W<R> *xa, *xb, *X, *ya, *yb, *Y;
    W<R> *xab, *xbb, *Xb, *yab, *ybb, *Yb;
    if (S == 1) { xa = &A; xb = &Cv; X = &B; ya = &B; yb = &Cv; Y = &A;
                  xab = &Ab; xbb = &Cb; Xb = &Bb; yab = &Bb; ybb = &Cb; Yb = &Ab; }
    else if (S == 2) { xa = &A; xb = &B; X = &Cv; ya = &B; yb = &Cv; Y = &A;
                       xab = &Ab; xbb = &Bb; Xb = &Cb; yab = &Bb; ybb = &Cb; Yb = &Ab; }
    else { xa = &A; xb = &B; X = &Cv; ya = &A; yb = &Cv; Y = &B;
           xab = &Ab; xbb = &Bb; Xb = &Cb; yab = &Ab; ybb = &Cb; Yb = &Bb; }
    cx<R> x = mdot(xa->c, xb->c), y = mdot(ya->c, yb->c);
    cx<R> f = mul_mi(g) * inv_den;
    cx<R> fb = C<R>(R(0), R(0)), xbar = C<R>(R(0), R(0)), ybar = C<R>(R(0), R(0));
    for (int k = 0; k < 4; ++k) {
        cx<R> v = x * X->c[k] - y * Y->c[k];
        cx<R> vb = wb.c[k] * conj(f);
        fb += wb.c[k] * conj(v);
        xbar += vb * conj(X->c[k]);
        Xb->c[k] += vb * conj(x);
        ybar -= vb * conj(Y->c[k]);
        Yb->c[k] -= vb * conj(y);
    }
    invb += re(fb * conj(mul_mi(g)));
    mdot_adj(xa->c, xb->c, xbar, xab->c, xbb->c);
    mdot_adj(ya->c, yb->c, ybar, yab->c, ybb->c);
}

// --------------------------------------------------------------- external legs
// Derivatives of an external wavefunction with respect to its momentum (4) and
// mass (1) by forward tangents, contracted with the wavefunction's adjoint:
// pb[mu] += Re(conj(wb) dw/dp_mu), mb += Re(conj(wb) dw/dm).
template <typename F>
MF_DEV void external_adj(F make, const double *p, double m, const W<double> &wb, double *pb, double &mb) {
    typedef Dual<5> D;
    D pd[4];
    for (int q = 0; q < 4; ++q) pd[q] = D::seed(p[q], q);
    D md = D::seed(m, 4);
    W<D> w = make(pd, md);
    for (int t = 0; t < 5; ++t) {
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += wb.c[c].re * w.c[c].re.d[t] + wb.c[c].im * w.c[c].im.d[t];
        if (t < 4) pb[t] += acc; else mb += acc;
    }
}

}  // namespace mf
