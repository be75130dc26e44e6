// Topology-aware multichannel phase space (the paper's outlook, Sec. 4, and
// the "Scope" caveat of Sec. 2.6 on the flat RAMBO phase space of Sec. 2.4;
// multichannel weights after Kleiss & Pittau, the paper's ref. for it).
//
// A channel is taken from a tree diagram: its t-channel propagators (on the
// path between the incoming legs a and b) order the final state into
// clusters c_1..c_k along that path; its s-channel propagators form a binary
// tree inside each cluster.  The channel maps 3n-4 unit numbers to massive
// final-state momenta in the partonic centre-of-mass frame:
//   (i)   the masses of the clusters c_j with two or more legs, in spine
//         order, each on [m(c_j)^2, (sqrt(s-hat) - sum_{i<j} sqrt(s_ci)
//         - sum_{i>j} m(c_i))^2] with the density of its propagator;
//   (ii)  the masses of the remainders R_j = c_{j+1} + .. + c_k, j = 1..k-2,
//         flat on [(sum_{i>j} sqrt(s_ci))^2, (sqrt(s_R{j-1}) - sqrt(s_cj))^2];
//   (iii) the splits R_{j-1} -> c_j + R_j: in the rest frame of R_{j-1} the
//         polar angle of c_j about q_{j-1} = p_a - c_1 - .. - c_{j-1} with
//         the density of the t-channel propagator, 1 / (M^2 + t0 - t) in
//         t = (q_{j-1} - c_j)^2, and a flat azimuth about that axis;
//   (iv)  each cluster's nodes X -> (L, R) in pre-order: s_L on
//         [m(L)^2, (sqrt(s_X) - m(R))^2], s_R on [m(R)^2, (sqrt(s_X) -
//         sqrt(s_L))^2] (clusters only), L's direction isotropic in X's frame.
// An s-channel mass takes the density 1 / (s - M^2 + s0) of its propagator
// on its range (flat where that is not positive at the lower end).  The
// channel's density g relative to dPhi_n = prod ds/(2 pi) prod dPhi_2,
// dPhi_2 = lambda^(1/2) / (32 pi^2 s) dOmega, is returned as 1/g.
//
// The integrand is shared out among the channels by a_i = P_i / sum_j P_j,
// P_i the product over channel i's propagators of 1 / (|x - M^2| + r)^2
// (x = the propagator's s or t, r = s0 or t0); a point of channel i weighs
// a_i / g_i.
//
// Table (int32, device memory), written by the host library:
//   [0] K channels, [1] E distinct propagators, [2] final particles,
//   [3..16) unused;
//   propagators at 16: E records of 4: type (0 s-channel, 1 t-channel),
//       mask of final legs (t: those on the side of leg a), mass id, 0;
//   channels at 16 + 4 E: K records of MF_CH_STRIDE (offsets below).
#pragma once
#include "mf_common.cuh"
#include "mf_dual.cuh"

#define MF_CH_MAX_FINAL 6
#define MF_CH_MAX_EDGES 128
#define MF_CH_HDR 16
#define MF_CH_EDGE 4
#define MF_CH_STRIDE 64
// offsets inside a channel record
#define MF_CH_K 0          // clusters along the spine
#define MF_CH_NNODE 1      // s-channel nodes (pre-order, clusters in spine order)
#define MF_CH_NEDGE 2      // propagators of the channel
#define MF_CH_CMASK 4      // [6] final-leg mask of c_j
#define MF_CH_CNODE 10     // [6] node of c_j, -1 for a single leg
#define MF_CH_TMASS 16     // [6] mass id of the t-channel propagator after c_j
#define MF_CH_EDGES 22     // [10] propagator indices
#define MF_CH_NODES 32     // [5][6] mask, mass id, left, right, 0, 0 (child < 0: leg -1-child)
#define MF_CH_NODE_W 6

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define MF_CH_FN __device__ __noinline__
#else
#define MF_CH_FN inline
#endif

namespace mf {

// T is double, or a dual number carrying derivatives (the gradient kernel).
template <typename T>
MF_DEV T ch_sqrt_lambda(const T &s, const T &s1, const T &s2) {
    const T m1 = sqrt(s1), m2 = sqrt(s2);
    T a = s - (m1 + m2) * (m1 + m2), b = s - (m1 - m2) * (m1 - m2);
    a = a > 0.0 ? a : T(0.0);
    b = b > 0.0 ? b : T(0.0);
    return sqrt(a * b);
}

// p (given in the frame where Q = (Q0, Q)) -> rest frame of Q (mass M)
template <typename T>
MF_DEV void ch_boost_to_rest(const T *p, const T *Q, const T &M, T *out) {
    const T e = (Q[0] * p[0] - Q[1] * p[1] - Q[2] * p[2] - Q[3] * p[3]) / M;
    const T c = (p[0] + e) / (Q[0] + M);
    out[0] = e;
    out[1] = p[1] - c * Q[1];
    out[2] = p[2] - c * Q[2];
    out[3] = p[3] - c * Q[3];
}

// p (given in the rest frame of Q, mass M) -> frame of Q
template <typename T>
MF_DEV void ch_boost_from_rest(const T *p, const T *Q, const T &M, T *out) {
    const T e = (Q[0] * p[0] + Q[1] * p[1] + Q[2] * p[2] + Q[3] * p[3]) / M;
    const T c = (p[0] + e) / (Q[0] + M);
    out[0] = e;
    out[1] = p[1] + c * Q[1];
    out[2] = p[2] + c * Q[2];
    out[3] = p[3] + c * Q[3];
}

// s on [lo, hi] with density 1 / (s - M2 + reg) (flat where lo - M2 + reg
// <= 0); inv = 1 / density
template <typename T>
MF_DEV T ch_mass_sample(const T &u, const T &lo, const T &hi, const T &M2, double reg, T &inv) {
    const T a = lo - M2 + reg;
    if (a > 0.0) {
        const T L = log1p((hi - lo) / a);
        const T s = lo + a * expm1(u * L);
        inv = (a * exp(u * L)) * L;
        return s;
    }
    inv = hi - lo;
    return lo + u * (hi - lo);
}

// daughters of X (mass^2 sX) with masses^2 sL, sR, L along the unit vector n
// in X's rest frame; momenta in X's frame; returns lambda^(1/2)(sX, sL, sR)
template <typename T>
MF_DEV T ch_two_body(const T *X, const T &sX, const T &sL, const T &sR, const T *n, T *L, T *R) {
    const T M = sqrt(sX);
    const T lam = ch_sqrt_lambda(sX, sL, sR);
    const T p = lam / (2.0 * M);
    const T l[4] = {(sX + sL - sR) / (2.0 * M), p * n[0], p * n[1], p * n[2]};
    const T r[4] = {(sX + sR - sL) / (2.0 * M), -(p * n[0]), -(p * n[1]), -(p * n[2])};
    ch_boost_from_rest(l, X, M, L);
    ch_boost_from_rest(r, X, M, R);
    return lam;
}

template <typename T>
MF_DEV void ch_direction(const T &c, const T &phi, T *n) {
    T s2 = (1.0 - c) * (1.0 + c);
    const T st = s2 > 0.0 ? sqrt(s2) : T(0.0);
    T sp, cp;
    sincos(phi, &sp, &cp);
    n[0] = st * cp;
    n[1] = st * sp;
    n[2] = c;
}

MF_DEV const int32_t *ch_record(const int32_t *tab, int ch) {
    return tab + MF_CH_HDR + MF_CH_EDGE * tab[1] + MF_CH_STRIDE * ch;
}

template <int NOUT, typename T>
MF_DEV T ch_mmin(int mask, const T *fm) {
    T m = T(0.0);
#pragma unroll
    for (int i = 0; i < NOUT; ++i)
        if ((mask >> i) & 1) m = m + fm[i];
    return m;
}

template <typename T>
MF_DEV T ch_m2(int id, const T *masses) { return id < 0 ? T(0.0) : masses[id] * masses[id]; }

MF_DEV int ch_lowest(int mask) {
    int i = 0;
    while (i < 31 && !((mask >> i) & 1)) ++i;
    return i;
}

// Momenta p (partonic CM frame) and 1/g of channel ch from the unit numbers
// u[0 .. 3 NOUT - 4); fm: final masses, masses: the process's mass table.
// Returns false where a sampled range came out empty (the point then has
// weight zero).
template <int NOUT, typename T = double>
MF_CH_FN bool channel_generate(const int32_t *tab, int ch, const T *u, T rs, const T *fm, const T *masses, double s0,
                               double t0, T (*p)[4], T &inv_g) {
    const double two_pi = 6.283185307179586;
    const double pi = 3.141592653589793;
    const double pi2_32 = 32.0 * (pi * pi);
    const int32_t *c = ch_record(tab, ch);
    const int k = c[MF_CH_K];
    const T s_hat = rs * rs;
    int col = 0;
    bool ok = true;
    T ig = T(1.0);
    T sc[NOUT], sR[NOUT], mom[NOUT][4];
    // (i) masses of the clusters on the spine
    for (int j = 0; j < k; ++j) {
        const int node = c[MF_CH_CNODE + j];
        if (node < 0) {
            const T m = fm[ch_lowest(c[MF_CH_CMASK + j])];
            sc[j] = m * m;
            continue;
        }
        if (k == 1) {
            sc[j] = s_hat;
            continue;
        }
        T before = T(0.0), after = T(0.0);
        for (int i = 0; i < j; ++i) before = before + sqrt(sc[i]);
        for (int i = j + 1; i < k; ++i) after = after + ch_mmin<NOUT>(c[MF_CH_CMASK + i], fm);
        T top = rs - before - after;
        top = top > 0.0 ? top : T(0.0);
        const T m0 = ch_mmin<NOUT>(c[MF_CH_CMASK + j], fm);
        const T lo = m0 * m0;
        T hi = top * top;
        ok = ok && hi >= lo;
        hi = hi > lo ? hi : lo;
        T inv;
        sc[j] = ch_mass_sample(u[col++], lo, hi, ch_m2(c[MF_CH_NODES + MF_CH_NODE_W * node + 1], masses), s0, inv);
        ig = ig * (inv / two_pi);
    }
    // (ii) the remainders of the chain
    sR[0] = s_hat;
    if (k >= 2) sR[k - 1] = sc[k - 1];
    for (int j = 1; j < k - 1; ++j) {
        T lo = T(0.0);
        for (int i = j; i < k; ++i) lo = lo + sqrt(sc[i]);
        lo = lo * lo;
        T hi = sqrt(sR[j - 1]) - sqrt(sc[j - 1]);
        hi = hi > 0.0 ? hi * hi : T(0.0);
        ok = ok && hi >= lo;
        hi = hi > lo ? hi : lo;
        sR[j] = lo + u[col++] * (hi - lo);
        ig = ig * ((hi - lo) / two_pi);
    }
    // (iii) the chain R_{j-1} -> c_j + R_j
    T R[4] = {rs, T(0.0), T(0.0), T(0.0)};
    T q[4] = {0.5 * rs, T(0.0), T(0.0), 0.5 * rs};
    for (int j = 1; j < k; ++j) {
        const T sRp = sR[j - 1], scj = sc[j - 1], sRj = sR[j];
        const T Mr = sqrt(sRp);
        T qs[4];
        ch_boost_to_rest(q, R, Mr, qs);
        const T qabs = sqrt(qs[1] * qs[1] + qs[2] * qs[2] + qs[3] * qs[3]);
        const T q2 = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
        const T Ec = (sRp + scj - sRj) / (2.0 * Mr);
        const T pc = ch_sqrt_lambda(sRp, scj, sRj) / (2.0 * Mr);
        const T A = ch_m2(c[MF_CH_TMASS + j - 1], masses) + t0 - q2 - scj + 2.0 * qs[0] * Ec;
        const T B = 2.0 * qabs * pc;
        const T uc = u[col++];
        T cth, inv_h;
        if (B > 0.0 && A - B > 0.0) {
            const T L = log1p(2.0 * B / (A - B));
            cth = -1.0 - (A + B) * expm1(-(uc * L)) / B;
            cth = cth < -1.0 ? T(-1.0) : (cth > 1.0 ? T(1.0) : cth);
            inv_h = (A - B * cth) * L / B;
        } else {
            cth = 2.0 * uc - 1.0;
            cth = cth < -1.0 ? T(-1.0) : (cth > 1.0 ? T(1.0) : cth);
            inv_h = T(2.0);
        }
        const T phi = two_pi * u[col++];
        // axis frame R_z(phi_q) R_y(theta_q) of the direction of q
        T hx = T(0.0), hy = T(0.0), hz = T(1.0);
        if (qabs > 0.0) {
            hx = qs[1] / qabs;
            hy = qs[2] / qabs;
            hz = qs[3] / qabs;
        }
        const T rho = sqrt(hx * hx + hy * hy);
        T cq = T(1.0), sq = T(0.0);
        if (rho > 0.0) {
            cq = hx / rho;
            sq = hy / rho;
        }
        T nl[3], n[3];
        ch_direction(cth, phi, nl);
        const T vx = hz * nl[0] + rho * nl[2];
        const T vy = nl[1];
        const T vz = hz * nl[2] - rho * nl[0];
        n[0] = cq * vx - sq * vy;
        n[1] = sq * vx + cq * vy;
        n[2] = vz;
        T Rn[4];
        const T lam = ch_two_body(R, sRp, scj, sRj, n, mom[j - 1], Rn);
        ig = ig * (lam / (pi2_32 * sRp) * two_pi * inv_h);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            q[a] = q[a] - mom[j - 1][a];
            R[a] = Rn[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) mom[k - 1][a] = R[a];
    // (iv) inside the clusters, nodes in pre-order
    const int nn = c[MF_CH_NNODE];
    T ns[NOUT], nmom[NOUT][4];
    for (int j = 0; j < k; ++j) {
        const int node = c[MF_CH_CNODE + j];
        if (node < 0) {
            const int leg = ch_lowest(c[MF_CH_CMASK + j]);
#pragma unroll
            for (int a = 0; a < 4; ++a) p[leg][a] = mom[j][a];
        } else {
            ns[node] = sc[j];
#pragma unroll
            for (int a = 0; a < 4; ++a) nmom[node][a] = mom[j][a];
        }
    }
    for (int i = 0; i < nn; ++i) {
        const int32_t *nd = c + MF_CH_NODES + MF_CH_NODE_W * i;
        const int left = nd[2], right = nd[3];
        const int lmask = left >= 0 ? c[MF_CH_NODES + MF_CH_NODE_W * left] : (1 << (-1 - left));
        const int rmask = right >= 0 ? c[MF_CH_NODES + MF_CH_NODE_W * right] : (1 << (-1 - right));
        const T sX = ns[i];
        T sL, sRr;
        if (left >= 0) {
            const T m0 = ch_mmin<NOUT>(lmask, fm);
            const T lo = m0 * m0;
            T hi = sqrt(sX) - ch_mmin<NOUT>(rmask, fm);
            hi = hi > 0.0 ? hi * hi : T(0.0);
            ok = ok && hi >= lo;
            hi = hi > lo ? hi : lo;
            T inv;
            sL = ch_mass_sample(u[col++], lo, hi, ch_m2(c[MF_CH_NODES + MF_CH_NODE_W * left + 1], masses), s0, inv);
            ig = ig * (inv / two_pi);
        } else {
            const T m = fm[-1 - left];
            sL = m * m;
        }
        if (right >= 0) {
            const T m0 = ch_mmin<NOUT>(rmask, fm);
            const T lo = m0 * m0;
            T hi = sqrt(sX) - sqrt(sL);
            hi = hi > 0.0 ? hi * hi : T(0.0);
            ok = ok && hi >= lo;
            hi = hi > lo ? hi : lo;
            T inv;
            sRr = ch_mass_sample(u[col++], lo, hi, ch_m2(c[MF_CH_NODES + MF_CH_NODE_W * right + 1], masses), s0, inv);
            ig = ig * (inv / two_pi);
        } else {
            const T m = fm[-1 - right];
            sRr = m * m;
        }
        const T cth = 2.0 * u[col] - 1.0;
        const T phi = two_pi * u[col + 1];
        col += 2;
        T n[3], PL[4], PR[4];
        ch_direction(cth, phi, n);
        const T lam = ch_two_body(nmom[i], sX, sL, sRr, n, PL, PR);
        ig = ig * (lam / (pi2_32 * sX) * (2.0 * two_pi));
        if (left >= 0) {
            ns[left] = sL;
#pragma unroll
            for (int a = 0; a < 4; ++a) nmom[left][a] = PL[a];
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) p[-1 - left][a] = PL[a];
        }
        if (right >= 0) {
            ns[right] = sRr;
#pragma unroll
            for (int a = 0; a < 4; ++a) nmom[right][a] = PR[a];
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) p[-1 - right][a] = PR[a];
        }
    }
    inv_g = ig;
    return ok;
}

// Channel ch's share a_ch = P_ch / sum_j P_j of the partition at final
// momenta p (partonic CM frame, beam a along +z with energy rs/2).
template <int NOUT, typename T = double>
MF_CH_FN T channel_share(const int32_t *tab, int ch, T rs, const T (*p)[4], const T *masses, double s0, double t0) {
    const int K = tab[0], E = tab[1];
    T fac[MF_CH_MAX_EDGES];
    const T pa[4] = {0.5 * rs, T(0.0), T(0.0), 0.5 * rs};
    for (int e = 0; e < E; ++e) {
        const int32_t *ed = tab + MF_CH_HDR + MF_CH_EDGE * e;
        const int mask = ed[1];
        T Q[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
#pragma unroll
        for (int i = 0; i < NOUT; ++i)
            if ((mask >> i) & 1) {
#pragma unroll
                for (int a = 0; a < 4; ++a) Q[a] = Q[a] + p[i][a];
            }
        if (ed[0] == 1) {
#pragma unroll
            for (int a = 0; a < 4; ++a) Q[a] = pa[a] - Q[a];
        }
        const T x = Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3];
        const T d = fabs(x - ch_m2(ed[2], masses)) + (ed[0] == 1 ? t0 : s0);
        fac[e] = 1.0 / (d * d);
    }
    T tot = T(0.0), own = T(0.0);
    for (int i = 0; i < K; ++i) {
        const int32_t *c = ch_record(tab, i);
        T P = T(1.0);
        const int ne = c[MF_CH_NEDGE];
        for (int a = 0; a < ne; ++a) P = P * fac[c[MF_CH_EDGES + a]];
        tot = tot + P;
        if (i == ch) own = P;
    }
    return own / tot;
}

}  // namespace mf
