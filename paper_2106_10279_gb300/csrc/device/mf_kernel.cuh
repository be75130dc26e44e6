// Kernel body of the fused per-event integrand (Fig. 1: L(x1,x2) x sigma-hat),
// included by the run-time generated source after it has defined namespace
// `proc` (the process's diagram program and constants).
//
// One CUDA block works on tiles of BLOCK events:
//   phase A  one thread per event, double precision: unit numbers (given x, or
//            Philox + Vegas map), x1/x2 map, phase space + massive rescaling,
//            cuts, PDFs, weight prefactor, invariants and propagator
//            denominators -> shared memory; events that pass are compacted;
//   phase B  HT threads per passing event, each running the diagram program
//            for its share of the helicities in precision R (float or double)
//            and the colour sum J^dagger C J; the per-helicity |M|^2 are summed
//            in a fixed pairwise tree (independent of HT) across the HT lanes;
//   phase C  one thread per event writes f (integrand) or w = f J_V and the
//            bin indices (Vegas).
#pragma once
#include "mf_common.cuh"
#include "mf_kinematics.cuh"
#include "mf_helas.cuh"
#include "mf_kparams.h"

namespace mf {

typedef mf_kparams KParams;

// fixed pairwise summation over a power-of-two count, as a binary counter:
// after adding item k (0-based), merge levels while bit j of k+1 is zero
struct PairSum {
    double lvl[9];          // enough for 256 items per lane
    int count;
    MF_DEV void init() { count = 0; }
    MF_DEV void add(double v) {
        int c = count;
        double s = v;
        int j = 0;
        while ((c >> j) & 1) { s = lvl[j] + s; ++j; }
        lvl[j] = s;
        count = c + 1;
    }
    // total of a power-of-two count
    MF_DEV double total() const {
        int j = 0;
        while ((1 << (j + 1)) <= count) ++j;
        return count ? lvl[j] : 0.0;
    }
};

// Per-event work that does not depend on helicity (phase A), for one point y
// of the unit hypercube (after the Vegas map).  T is double in the integrand
// kernel and a dual number (derivatives with respect to y and m_t) in the
// gradient kernel.  Returns false if the point fails the threshold or the
// cuts (the outputs are then unspecified).
template <typename T>
struct EventKin {
    T pref;                    // f = pref * sum_h |M_h|^2
    T p[proc::NLEG][4];        // momenta: incoming along +z / -z, outgoing from phase space
    T den[proc::NDEN > 0 ? proc::NDEN : 1];   // propagator denominators P^2 - M^2
};

template <typename T>
MF_DEV bool phase_a(const KParams &kp, const T *y, const T *masses, const T &ln_tau_min, EventKin<T> &ev) {
    using namespace proc;
    T s_hat = T(kp.S), jx = T(1.0), lum = T(1.0);
    XMap<T> xm;
    const T *u = y;
    if (HADRONIC) {
        xm = xmap(y[0], y[1], ln_tau_min);
        s_hat = xm.tau * kp.S;
        jx = xm.jac;
        u = y + 2;
    }
    T rs = sqrt(s_hat);
    T (*p)[4] = ev.p;
    p[0][0] = 0.5 * rs; p[0][1] = T(0.0); p[0][2] = T(0.0); p[0][3] = 0.5 * rs;
    p[1][0] = 0.5 * rs; p[1][1] = T(0.0); p[1][2] = T(0.0); p[1][3] = -0.5 * rs;
    T (*pout)[4] = reinterpret_cast<T (*)[4]>(&p[2][0]);
    massless_diet<NOUT>(u, rs, pout);
    T mout[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) mout[i] = LEG_MASS_ID[2 + i] >= 0 ? masses[LEG_MASS_ID[2 + i]] : T(0.0);
    T wfac = massive_rescale<NOUT>(pout, mout, rs);
    bool ok = value(wfac) > 0.0;
    // cuts on the flagged legs (decided on values)
    if (ok && NCUT > 0) {
        double pv[NLEG][4];
#pragma unroll
        for (int i = 0; i < NLEG; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) pv[i][q] = value(p[i][q]);
#pragma unroll
        for (int a = 0; a < NCUT; ++a) ok &= pt2(pv[CUT_LEGS[a]]) > kp.pt_min2;
        if (kp.dr_min2 > 0.0) {
#pragma unroll
            for (int a = 0; a < NCUT; ++a)
#pragma unroll
                for (int b = a + 1; b < NCUT; ++b) ok &= delta_r2(pv[CUT_LEGS[a]], pv[CUT_LEGS[b]]) > kp.dr_min2;
        }
    }
    if (!ok) return false;
    T wps = kp.w0_const * wfac;
#pragma unroll
    for (int i = 0; i < NOUT - 2; ++i) wps = wps * s_hat;
    if (HADRONIC) {
        const double *r = kp.pdf_rows;
        const int nx = kp.pdf_nx;
        T f1 = pdf_eval(r, r + nx, nx, kp.pdf_a0, kp.pdf_h, xm.ln_x1, xm.x1);
        T f2 = pdf_eval(r + 2 * nx, r + 3 * nx, nx, kp.pdf_a0, kp.pdf_h, xm.ln_x2, xm.x2);
        lum = f1 * f2;
    }
    ev.pref = jx * wps * lum * kp.pref_const / s_hat;
    denominators(p, masses, ev.den);
    return true;
}

template <typename R, int BLOCK, int HT>
MF_DEV void kernel_body(const KParams &kp) {
    using namespace proc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s_mom = reinterpret_cast<R *>(smem_raw);                                   // [BLOCK][NLEG][4]
    R *s_den = s_mom + BLOCK * NLEG * 4;                                           // [BLOCK][NDEN1]
    constexpr int NDEN1 = NDEN > 0 ? NDEN : 1;
    double *s_pref = reinterpret_cast<double *>(
        reinterpret_cast<unsigned char *>(s_den + BLOCK * NDEN1) +
        ((16 - ((BLOCK * NDEN1 * sizeof(R)) % 16)) % 16));
    double *s_msq = s_pref + BLOCK;
    int *s_list = reinterpret_cast<int *>(s_msq + BLOCK);
    int *s_warp = s_list + BLOCK;                                                  // [BLOCK/32 + 1]
    __shared__ double s_grid[NDIM * 65];

    const int tid = threadIdx.x;
    const int lane32 = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (kp.n + BLOCK - 1) / BLOCK;

    if (kp.mode == 1) {
        for (int i = tid; i < NDIM * (kp.nb + 1); i += BLOCK) s_grid[i] = kp.grid[i];
    }

    // couplings and masses in the matrix-element precision, in shared memory
    __shared__ cx<R> cpl[8];
    __shared__ R mass_r[8];
    if (tid < 8) {
        mass_r[tid] = (R)kp.masses[tid];
        cpl[tid] = C<R>((R)kp.couplings[2 * tid], (R)kp.couplings[2 * tid + 1]);
    }
    __syncthreads();

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e = tile * BLOCK + tid;
        bool ok = false;
        double pref = 0.0, jv = 1.0;
        uint8_t bins[NDIM];
        if (e < kp.n) {
            // ---------------- phase A: kinematics in double precision
            double y[NDIM];
            if (kp.mode != 1) {
#pragma unroll
                for (int j = 0; j < NDIM; ++j) y[j] = kp.x[(int64_t)j * kp.n + e];
            } else {
#pragma unroll
                for (int b = 0; b < (NDIM + 3) / 4; ++b) {
                    uint64_t c[4] = {(uint64_t)(e + kp.ev0), kp.iteration, kp.subprocess, (uint64_t)b};
                    philox4x64_10(c, kp.seed, 0ull);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (4 * b + q < NDIM) y[4 * b + q] = unit_from_bits(c[q]);
                }
#pragma unroll
                for (int j = 0; j < NDIM; ++j) {
                    double xj;
                    int bj;
                    jv *= vegas_map1(s_grid + j * (kp.nb + 1), kp.nb, y[j], xj, bj);
                    y[j] = xj;
                    bins[j] = (uint8_t)bj;
                }
            }
            EventKin<double> ev;
            ok = phase_a<double>(kp, y, kp.masses, kp.ln_tau_min, ev);
            if (ok) {
                pref = ev.pref;
                R *sd = s_den + tid * NDEN1;
#pragma unroll
                for (int k = 0; k < NDEN; ++k) sd[k] = (R)(1.0 / ev.den[k]);
                R *sm = s_mom + tid * NLEG * 4;
#pragma unroll
                for (int i = 0; i < NLEG; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) sm[4 * i + q] = (R)ev.p[i][q];
            }
        }
        s_pref[tid] = pref;
        // ---------------- compaction of passing events
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane32 == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < BLOCK / 32; ++w) { int c = s_warp[w]; s_warp[w] = acc; acc += c; }
            s_warp[BLOCK / 32] = acc;
        }
        __syncthreads();
        if (ok) s_list[s_warp[warp] + __popc(bal & ((1u << lane32) - 1u))] = tid;
        const int npass = s_warp[BLOCK / 32];
        __syncthreads();
        // ---------------- phase B: helicity amplitudes, HT lanes per event
        {
            constexpr int EPR = BLOCK / HT;     // events per round
            const int sub = tid % HT;
            const int nhp = kp.nhel_pow2;       // padded helicity count (power of two)
            const int per = nhp >= HT ? nhp / HT : 1;   // contiguous helicities per lane
            // every thread runs the program the same number of times (lanes
            // without an event or a helicity compute on a valid stand-in and
            // discard it), so that the program may contain block barriers
            for (int base = 0; base < npass; base += EPR) {
                const int slot = base + tid / HT;
                const bool valid = slot < npass;
                PairSum ps;
                ps.init();
                const int ev = s_list[valid ? slot : 0];
                const R *ms = s_mom + ev * NLEG * 4;
                const R *idn = s_den + ev * NDEN1;
                for (int k = 0; k < per; ++k) {
                    const int h = sub * per + k;
                    const bool hv = h < kp.nhel;
                    double v = (double)helicity_msq<R>(ms, idn, kp.hel[hv ? h : 0], cpl, mass_r);
                    if (!(hv && valid)) v = 0.0;
                    if (kp.mode == 2 && hv && valid) kp.f[(int64_t)h * kp.n + tile * BLOCK + ev] = v;
                    ps.add(v);
                }
                double part = ps.total();
#pragma unroll
                for (int off = 1; off < HT; off <<= 1) {
                    double o = __shfl_xor_sync(0xffffffffu, part, off);
                    // lanes combine (lower block) + (upper block) in that order
                    part = (sub & off) ? (o + part) : (part + o);
                }
                if (sub == 0 && slot < npass) s_msq[s_list[slot]] = part;
            }
        }
        __syncthreads();
        // ---------------- phase C: outputs
        if (e < kp.n) {
            double fval = ok ? s_pref[tid] * s_msq[tid] : 0.0;
            if (kp.mode == 0) {
                kp.f[e] = fval;
            } else if (kp.mode == 1) {
                kp.w_out[e] = fval * jv;
#pragma unroll
                for (int j = 0; j < NDIM; ++j) kp.bins_out[(int64_t)j * kp.n + e] = bins[j];
            }
        }
        __syncthreads();
    }
}

}  // namespace mf
