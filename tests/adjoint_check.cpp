// Unit test of the hand-written adjoints in csrc/device/mf_helas_adj.cuh:
// for each vertex routine, L = Re sum_k conj(r_k) out_k with random complex
// weights r (so dL/d out = r), the adjoint routine's derivatives of L with
// respect to every real input component (wavefunction re/im parts, momenta,
// masses, inverse denominators) are compared with central finite
// differences.  Compiled on the host with g++ from the same headers the
// kernels use; prints the worst relative error per routine.
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <random>
#include <vector>

#include "mf_helas_adj.cuh"

using namespace mf;
typedef double R;
typedef cx<R> Cx;
typedef W<R> Wf;

static std::mt19937_64 rng(42);
static double uni() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); }
static Wf rwf() { Wf w; for (int k = 0; k < 4; ++k) w.c[k] = C<R>(uni(), uni()); return w; }
static Wf zwf() { Wf w; for (int k = 0; k < 4; ++k) w.c[k] = C<R>(0.0, 0.0); return w; }

// real parameters of a routine call, flattened: wavefunctions (8 each), momenta (4 each), scalars
struct Case {
    std::vector<double> x;                                    // inputs
    std::function<void(const std::vector<double> &, Cx *, int &)> fwd;   // outputs (complex), count
    std::function<void(const std::vector<double> &, const Cx *, std::vector<double> &)> adj;  // grad
};

static double check(const char *name, Case c) {
    Cx out[4];
    int nout = 0;
    c.fwd(c.x, out, nout);
    Cx r[4];
    for (int k = 0; k < nout; ++k) r[k] = C<R>(uni(), uni());
    auto L = [&](const std::vector<double> &x) {
        Cx o[4]; int n = 0; c.fwd(x, o, n);
        double s = 0; for (int k = 0; k < n; ++k) s += r[k].re * o[k].re + r[k].im * o[k].im; return s;
    };
    std::vector<double> g(c.x.size(), 0.0);
    c.adj(c.x, r, g);
    double worst = 0.0;
    for (size_t i = 0; i < c.x.size(); ++i) {
        std::vector<double> a = c.x, b = c.x;
        double h = 1e-6 * (1.0 + std::fabs(c.x[i]));
        a[i] += h; b[i] -= h;
        double fd = (L(a) - L(b)) / (2 * h);
        double err = std::fabs(fd - g[i]) / (1e-8 + std::fabs(fd) + std::fabs(g[i]));
        if (err > worst) worst = err;
    }
    std::printf("%-14s %.3e\n", name, worst);
    return worst;
}

static Wf getw(const std::vector<double> &x, int off) {
    Wf w; for (int k = 0; k < 4; ++k) w.c[k] = C<R>(x[off + 2 * k], x[off + 2 * k + 1]); return w;
}
static void putw(std::vector<double> &g, int off, const Wf &w) {
    for (int k = 0; k < 4; ++k) { g[off + 2 * k] += w.c[k].re; g[off + 2 * k + 1] += w.c[k].im; }
}
static std::vector<double> rnd(int n) { std::vector<double> v(n); for (auto &e : v) e = uni(); return v; }

int main() {
    double worst = 0.0;
    Cx g = C<R>(0.3, -1.1);
    // FFV_AMP(row, col, V): x = row(8) col(8) V(8)
    {
        Case c; c.x = rnd(24);
        c.fwd = [&](const std::vector<double> &x, Cx *o, int &n) { o[0] = FFV_AMP<R>(getw(x, 0), getw(x, 8), getw(x, 16), g); n = 1; };
        c.adj = [&](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf a = zwf(), b = zwf(), v = zwf();
            FFV_AMP_adj<R>(getw(x, 0), getw(x, 8), getw(x, 16), g, r[0], a, b, v);
            putw(G, 0, a); putw(G, 8, b); putw(G, 16, v); };
        worst = std::max(worst, check("FFV_AMP", c));
    }
    // FFV_FIN / FFV_FOUT(psi, V, M, inv, P): x = psi(8) V(8) M inv P(4)
    for (int fout = 0; fout < 2; ++fout) {
        Case c; c.x = rnd(22); c.x[16] = 0.7; c.x[17] = 0.4;
        auto call = [fout, g](const std::vector<double> &x) {
            double P[4] = {x[18], x[19], x[20], x[21]};
            return fout ? FFV_FOUT<R>(getw(x, 0), getw(x, 8), g, x[16], x[17], P)
                        : FFV_FIN<R>(getw(x, 0), getw(x, 8), g, x[16], x[17], P); };
        c.fwd = [call](const std::vector<double> &x, Cx *o, int &n) { Wf w = call(x); for (int k = 0; k < 4; ++k) o[k] = w.c[k]; n = 4; };
        c.adj = [fout, g](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf wb; for (int k = 0; k < 4; ++k) wb.c[k] = r[k];
            Wf a = zwf(), v = zwf(); double invb = 0, Mb = 0, Pb[4] = {0, 0, 0, 0};
            double P[4] = {x[18], x[19], x[20], x[21]};
            if (fout) FFV_FOUT_adj<R>(getw(x, 0), getw(x, 8), g, x[16], x[17], P, wb, a, v, invb, Pb, Mb);
            else FFV_FIN_adj<R>(getw(x, 0), getw(x, 8), g, x[16], x[17], P, wb, a, v, invb, Pb, Mb);
            putw(G, 0, a); putw(G, 8, v); G[16] += Mb; G[17] += invb; for (int q = 0; q < 4; ++q) G[18 + q] += Pb[q]; };
        worst = std::max(worst, check(fout ? "FFV_FOUT" : "FFV_FIN", c));
    }
    // FFV_VEC(row, col, inv): x = row(8) col(8) inv
    {
        Case c; c.x = rnd(17);
        c.fwd = [g](const std::vector<double> &x, Cx *o, int &n) { Wf w = FFV_VEC<R>(getw(x, 0), getw(x, 8), g, x[16]); for (int k = 0; k < 4; ++k) o[k] = w.c[k]; n = 4; };
        c.adj = [g](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf wb; for (int k = 0; k < 4; ++k) wb.c[k] = r[k];
            Wf a = zwf(), b = zwf(); double invb = 0;
            FFV_VEC_adj<R>(getw(x, 0), getw(x, 8), g, x[16], wb, a, b, invb);
            putw(G, 0, a); putw(G, 8, b); G[16] += invb; };
        worst = std::max(worst, check("FFV_VEC", c));
    }
    // VVV_AMP(A, B, C, kA, kB, kC): x = A B C (24) kA kB kC (12)
    {
        Case c; c.x = rnd(36);
        auto k = [](const std::vector<double> &x, int i) { return &x[24 + 4 * i]; };
        c.fwd = [g, k](const std::vector<double> &x, Cx *o, int &n) { o[0] = VVV_AMP<R>(getw(x, 0), getw(x, 8), getw(x, 16), k(x, 0), k(x, 1), k(x, 2), g); n = 1; };
        c.adj = [g, k](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf a = zwf(), b = zwf(), cc = zwf(); double ka[4] = {}, kb[4] = {}, kc[4] = {};
            VVV_AMP_adj<R>(getw(x, 0), getw(x, 8), getw(x, 16), k(x, 0), k(x, 1), k(x, 2), g, r[0], a, b, cc, ka, kb, kc);
            putw(G, 0, a); putw(G, 8, b); putw(G, 16, cc);
            for (int q = 0; q < 4; ++q) { G[24 + q] += ka[q]; G[28 + q] += kb[q]; G[32 + q] += kc[q]; } };
        worst = std::max(worst, check("VVV_AMP", c));
    }
    // VVV_VEC(A, B, kA, kB, inv): x = A B (16) kA kB (8) inv
    {
        Case c; c.x = rnd(25);
        c.fwd = [g](const std::vector<double> &x, Cx *o, int &n) { Wf w = VVV_VEC<R>(getw(x, 0), getw(x, 8), &x[16], &x[20], g, x[24]); for (int k = 0; k < 4; ++k) o[k] = w.c[k]; n = 4; };
        c.adj = [g](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf wb; for (int k = 0; k < 4; ++k) wb.c[k] = r[k];
            Wf a = zwf(), b = zwf(); double invb = 0, ka[4] = {}, kb[4] = {};
            VVV_VEC_adj<R>(getw(x, 0), getw(x, 8), &x[16], &x[20], g, x[24], wb, a, b, invb, ka, kb);
            putw(G, 0, a); putw(G, 8, b); G[24] += invb; for (int q = 0; q < 4; ++q) { G[16 + q] += ka[q]; G[20 + q] += kb[q]; } };
        worst = std::max(worst, check("VVV_VEC", c));
    }
    // VVVV_AMP<S>(A, B, C, D) and VVVV_VEC<S>(A, B, C, inv)
    const char *an[3] = {"VVVV1_AMP", "VVVV2_AMP", "VVVV3_AMP"}, *vn[3] = {"VVVV1_VEC", "VVVV2_VEC", "VVVV3_VEC"};
    for (int S = 1; S <= 3; ++S) {
        Case c; c.x = rnd(32);
        c.fwd = [g, S](const std::vector<double> &x, Cx *o, int &n) {
            Wf A = getw(x, 0), B = getw(x, 8), Cw = getw(x, 16), D = getw(x, 24);
            o[0] = S == 1 ? VVVV_AMP<R, 1>(A, B, Cw, D, g) : S == 2 ? VVVV_AMP<R, 2>(A, B, Cw, D, g) : VVVV_AMP<R, 3>(A, B, Cw, D, g); n = 1; };
        c.adj = [g, S](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf A = getw(x, 0), B = getw(x, 8), Cw = getw(x, 16), D = getw(x, 24), a = zwf(), b = zwf(), cc = zwf(), d = zwf();
            if (S == 1) VVVV_AMP_adj<R, 1>(A, B, Cw, D, g, r[0], a, b, cc, d);
            else if (S == 2) VVVV_AMP_adj<R, 2>(A, B, Cw, D, g, r[0], a, b, cc, d);
            else VVVV_AMP_adj<R, 3>(A, B, Cw, D, g, r[0], a, b, cc, d);
            putw(G, 0, a); putw(G, 8, b); putw(G, 16, cc); putw(G, 24, d); };
        worst = std::max(worst, check(an[S - 1], c));
        Case v; v.x = rnd(25);
        v.fwd = [g, S](const std::vector<double> &x, Cx *o, int &n) {
            Wf A = getw(x, 0), B = getw(x, 8), Cw = getw(x, 16), w;
            w = S == 1 ? VVVV_VEC<R, 1>(A, B, Cw, g, x[24]) : S == 2 ? VVVV_VEC<R, 2>(A, B, Cw, g, x[24]) : VVVV_VEC<R, 3>(A, B, Cw, g, x[24]);
            for (int k = 0; k < 4; ++k) o[k] = w.c[k]; n = 4; };
        v.adj = [g, S](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf wb; for (int k = 0; k < 4; ++k) wb.c[k] = r[k];
            Wf A = getw(x, 0), B = getw(x, 8), Cw = getw(x, 16), a = zwf(), b = zwf(), cc = zwf(); double invb = 0;
            if (S == 1) VVVV_VEC_adj<R, 1>(A, B, Cw, g, x[24], wb, a, b, cc, invb);
            else if (S == 2) VVVV_VEC_adj<R, 2>(A, B, Cw, g, x[24], wb, a, b, cc, invb);
            else VVVV_VEC_adj<R, 3>(A, B, Cw, g, x[24], wb, a, b, cc, invb);
            putw(G, 0, a); putw(G, 8, b); putw(G, 16, cc); G[24] += invb; };
        worst = std::max(worst, check(vn[S - 1], v));
    }
    // external wavefunctions: momentum and mass tangents contracted with an adjoint
    for (int kind = 0; kind < 4; ++kind) {
        Case c; c.x = {0, 0, 0, 0, 0};
        double px = 0.3 * uni() * 100, py = 0.3 * uni() * 100, pz = uni() * 100, m = kind < 3 ? 17.3 : 0.0;
        c.x = {std::sqrt(px * px + py * py + pz * pz + m * m) * 1.3, px, py, pz, m};
        auto make = [kind](const double *p, double m) -> Wf {
            if (kind == 0) return ixx<R>(p, m, 1, 0);
            if (kind == 1) return oxx<R>(p, m, -1, 1);
            if (kind == 2) return ixx<R>(p, m, -1, 1);
            return vxx<R>(p, 1, 0); };
        c.fwd = [make](const std::vector<double> &x, Cx *o, int &n) { Wf w = make(&x[0], x[4]); for (int k = 0; k < 4; ++k) o[k] = w.c[k]; n = 4; };
        c.adj = [kind](const std::vector<double> &x, const Cx *r, std::vector<double> &G) {
            Wf wb; for (int k = 0; k < 4; ++k) wb.c[k] = r[k];
            double pb[4] = {0, 0, 0, 0}, mb = 0;
            auto mk = [kind](const Dual<5> *pd, const Dual<5> &md) -> W<Dual<5>> {
                if (kind == 0) return ixx<Dual<5>>(pd, md, 1, 0);
                if (kind == 1) return oxx<Dual<5>>(pd, md, -1, 1);
                if (kind == 2) return ixx<Dual<5>>(pd, md, -1, 1);
                return vxx<Dual<5>>(pd, 1, 0); };
            external_adj(mk, &x[0], x[4], wb, pb, mb);
            for (int q = 0; q < 4; ++q) G[q] += pb[q];
            G[4] += mb; };
        const char *names[4] = {"ixx(u)", "oxx(vbar)", "ixx(v)", "vxx(eps*)"};
        worst = std::max(worst, check(names[kind], c));
    }
    std::printf("WORST %.3e\n", worst);
    return worst < 1e-6 ? 0 : 1;
}
