// Gradient kernel (mf_grad): per event, f(x) together with df/dx_j, df/dm_t
// and df/dalpha_s.
//   * the helicity-independent kinematics (phase A) run once per event with
//     forward tangents (dual numbers) in the directions x_0 .. x_{d-1}, m_t;
//   * for every helicity the diagram program runs forward (double), and its
//     hand-written adjoint runs backwards from dL/dJ = 2 C J / den, giving the
//     derivatives of |M_h|^2 with respect to the external momenta, the
//     inverse propagator denominators and the masses; wavefunctions are
//     recomputed per helicity in registers / thread-local memory, nothing is
//     stored across helicities or written to global memory;
//   * the two are chained per event: dM/dtheta = sum pbar . dp/dtheta +
//     sum idnbar . d(1/den)/dtheta (+ mbar for m_t), and df = dpref M + pref dM;
//   * |M|^2 ~ alpha_s^k exactly, so df/dalpha_s = k f / alpha_s.
// One thread per event; the helicity sum is sequential.
#pragma once
#include "mf_kernel.cuh"
#include "mf_helas_adj.cuh"

namespace mf {

template <int K>
MF_DEV void grad_body(const KParams &kp) {
    using namespace proc;
    typedef Dual<K> D;
    constexpr int NDEN1 = NDEN > 0 ? NDEN : 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kp.n; e += (int64_t)gridDim.x * blockDim.x) {
        D y[NDIM];
#pragma unroll
        for (int j = 0; j < NDIM; ++j) y[j] = D::seed(kp.x[(int64_t)j * kp.n + e], j);
        D masses[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) masses[i] = D(kp.masses[i]);
        masses[0] = D::seed(kp.masses[0], NDIM);          // m_t
        D ln_tau_min = D(0.0);
        if (HADRONIC) {
            D msum = D(0.0);
#pragma unroll
            for (int i = 2; i < NLEG; ++i)
                if (LEG_MASS_ID[i] >= 0) msum = msum + masses[LEG_MASS_ID[i]];
            ln_tau_min = 2.0 * log(msum) - ::log(kp.S);
        }
        EventKin<D> ev;
        const bool ok = phase_a<D>(kp, y, masses, ln_tau_min, ev, kp.channel);
        double f = 0.0, df[K];
#pragma unroll
        for (int k = 0; k < K; ++k) df[k] = 0.0;
        if (ok) {
            double ms[NLEG * 4], idn[NDEN1], pbar[NLEG * 4], idnbar[NDEN1], mbar[8], mass[8];
            cx<double> cpl[8];
#pragma unroll
            for (int i = 0; i < NLEG; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) { ms[4 * i + q] = ev.p[i][q].v; pbar[4 * i + q] = 0.0; }
#pragma unroll
            for (int s = 0; s < NDEN1; ++s) { idn[s] = NDEN > 0 ? 1.0 / ev.den[s].v : 0.0; idnbar[s] = 0.0; }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                mbar[i] = 0.0;
                mass[i] = kp.masses[i];
                cpl[i] = C<double>(kp.couplings[2 * i], kp.couplings[2 * i + 1]);
            }
            double M = 0.0;
            for (int h = 0; h < kp.nhel; ++h) M += helicity_grad<double>(ms, idn, kp.hel[h], cpl, mass, pbar, idnbar, mbar);
            f = ev.pref.v * M;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double dM = 0.0;
#pragma unroll
                for (int i = 0; i < NLEG; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) dM += pbar[4 * i + q] * ev.p[i][q].d[k];
#pragma unroll
                for (int s = 0; s < NDEN; ++s) dM -= idnbar[s] * idn[s] * idn[s] * ev.den[s].d[k];
                if (k == NDIM) dM += mbar[0];
                df[k] = ev.pref.d[k] * M + ev.pref.v * dM;
            }
        }
        kp.f[e] = f;
        kp.g_dparam[e] = df[NDIM];
        kp.g_dparam[kp.n + e] = kp.alpha_s > 0.0 ? kp.alpha_s_power * f / kp.alpha_s : 0.0;
        if (kp.g_dx) {
#pragma unroll
            for (int j = 0; j < NDIM; ++j) kp.g_dx[(int64_t)j * kp.n + e] = df[j];
        }
    }
}

}  // namespace mf
