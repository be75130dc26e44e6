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
//
// The process-independent part below is included once.  The process-dependent
// part (EventKin, phase_a, tile_body, kernel_body) may be included several
// times in one translation unit, once per process of a batched kernel: the
// includer names the process namespace in MF_PROC and the namespace that
// receives these definitions in MF_BODY (defaults: proc and mf).
#ifndef MF_KERNEL_COMMON_DEFINED
#define MF_KERNEL_COMMON_DEFINED
#include "mf_common.cuh"
#include "mf_kinematics.cuh"
#include "mf_helas.cuh"
#include "mf_kparams.h"
#include "mf_tc.cuh"
#include "mf_channels.cuh"

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

}  // namespace mf
#endif  // MF_KERNEL_COMMON_DEFINED

#ifndef MF_PROC
#define MF_PROC proc
#define MF_BODY mf
#endif

namespace MF_BODY {
using namespace ::mf;

// Per-event work that does not depend on helicity (phase A), for one point y
// of the unit hypercube (after the Vegas map).  T is double in the integrand
// kernel and a dual number (derivatives with respect to y and m_t) in the
// gradient kernel.  Returns false if the point fails the threshold or the
// cuts (the outputs are then unspecified).
template <typename T>
struct EventKin {
    T pref;                    // f = pref * sum_h |M_h|^2
    T x1, x2, yb;              // momentum fractions and the rapidity of the partonic frame
    T p[MF_PROC::NLEG][4];     // momenta: incoming along +z / -z, outgoing from phase space
    T den[MF_PROC::NDEN > 0 ? MF_PROC::NDEN : 1];   // propagator denominators P^2 - M^2
};

template <typename T>
MF_DEV bool phase_a(const KParams &kp, const T *y, const T *masses, const T &ln_tau_min, EventKin<T> &ev,
                    int channel = -1) {
    using namespace MF_PROC;
    T s_hat = T(kp.S), jx = T(1.0), lum = T(1.0);
    XMap<T> xm;
    const T *u = y;
    ev.x1 = T(1.0);
    ev.x2 = T(1.0);
    ev.yb = T(0.0);
    if (HADRONIC) {
        xm = xmap(y[0], y[1], ln_tau_min);
        s_hat = xm.tau * kp.S;
        jx = xm.jac;
        u = y + 2;
        ev.x1 = xm.x1;
        ev.x2 = xm.x2;
        ev.yb = 0.5 * (xm.ln_x1 - xm.ln_x2);
    }
    T rs = sqrt(s_hat);
    T (*p)[4] = ev.p;
    p[0][0] = 0.5 * rs; p[0][1] = T(0.0); p[0][2] = T(0.0); p[0][3] = 0.5 * rs;
    p[1][0] = 0.5 * rs; p[1][1] = T(0.0); p[1][2] = T(0.0); p[1][3] = -0.5 * rs;
    T (*pout)[4] = reinterpret_cast<T (*)[4]>(&p[2][0]);
    T mout[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) mout[i] = LEG_MASS_ID[2 + i] >= 0 ? masses[LEG_MASS_ID[2 + i]] : T(0.0);
    T wfac;
    bool ok;
    // a multichannel point: the channel's momenta and 1/g (in the gradient
    // kernel with their derivatives)
    const bool chan = channel >= 0;
    if (chan) {
        ok = channel_generate<NOUT, T>(kp.chan, channel, u, rs, mout, masses, kp.ch_s0, kp.ch_t0, pout, wfac);
    } else {
        massless_diet<NOUT>(u, rs, pout);
        wfac = massive_rescale<NOUT>(pout, mout, rs);
        ok = value(wfac) > 0.0;
    }
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
    T wps;
    if (chan) {
        wps = wfac * channel_share<NOUT, T>(kp.chan, channel, rs, pout, masses, kp.ch_s0, kp.ch_t0);
    } else {
        wps = kp.w0_const * wfac;
#pragma unroll
        for (int i = 0; i < NOUT - 2; ++i) wps = wps * s_hat;
    }
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

// Shared-memory bytes of tile_body's dynamic buffers.
template <typename R, int BLOCK>
constexpr size_t tile_smem_bytes() {
    constexpr int NDEN1 = MF_PROC::NDEN > 0 ? MF_PROC::NDEN : 1;
    return (size_t)BLOCK * MF_PROC::NLEG * 4 * sizeof(R) + (size_t)BLOCK * NDEN1 * sizeof(R) +
           (16 - ((BLOCK * NDEN1 * sizeof(R)) % 16)) % 16 + (size_t)BLOCK * 8 * 2 + (size_t)BLOCK * 4 +
           (BLOCK / 32 + 1) * 4;
}

// Per-block constants of a process: the Vegas grid (the modes that map
// Philox points through it: 1, 3, 4 and 5) and the couplings and masses in
// the matrix-element precision.
template <typename R, int BLOCK>
MF_DEV void load_block_constants(const KParams &kp, double *s_grid, cx<R> *cpl, R *mass_r, bool copy_grid = true) {
    using namespace MF_PROC;
    const int tid = threadIdx.x;
    if (copy_grid && ((kp.mode == 1 && !kp.ch_off) || kp.mode == 3 || kp.mode == 4 || kp.mode == 5)) {
        for (int i = tid; i < NDIM * (kp.nb + 1); i += BLOCK) s_grid[i] = kp.grid[i];
    }
    if (tid < 8) {
        mass_r[tid] = (R)kp.masses[tid];
        cpl[tid] = C<R>((R)kp.couplings[2 * tid], (R)kp.couplings[2 * tid + 1]);
    }
}

// The channel of point e of a launch over every channel (mode 1 with
// ch_off): the k with ch_off[k] <= e < ch_off[k+1].
MF_DEV int point_channel(const KParams &kp, int64_t e) {
    int lo = 0, hi = kp.ch_count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (kp.ch_off[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Colour sampling: the unbiased estimate of a helicity's colour sum from
// one colour flow k of the NJAMP, drawn uniformly per point:
// NJAMP Re(conj(J_k) sum_l C_kl J_l) / den (with the leading-colour
// approximation, NJAMP C_kk |J_k|^2 / den).
template <typename R>
MF_DEV double sampled_colour_value(const cx<R> *J, int k) {
    using namespace MF_PROC;
    double v;
    if constexpr (LEADING_COLOUR) {
        cx<R> jk = C<R>(R(0), R(0));
#pragma unroll
        for (int l = 0; l < NJAMP; ++l)
            if (l == k) jk = J[l];
        v = (double)COLOUR_NUM[k * NJAMP + k] * ((double)jk.re * (double)jk.re + (double)jk.im * (double)jk.im);
    } else {
        v = (double)colour_row<R>(J, k);
    }
    return v * (double)NJAMP * INV_COLOUR_DEN;
}

// The colour flow a colour-sampled kernel uses for point e of a launch: the
// first unit number of Philox counter (point, iteration, subprocess, 12)
// (given points: (e, 0, 0, 12) with the process's sampling key).
MF_DEV int sampled_colour_flow(const KParams &kp, int64_t e, uint64_t iteration) {
    const bool given = kp.mode == 0 || kp.mode == 2;
    uint64_t gi = given ? (uint64_t)e : ((kp.mode == 3 || kp.mode == 5) ? (uint64_t)kp.idx[e] : (uint64_t)(e + kp.ev0));
    uint64_t sub = given ? 0ull : kp.subprocess;
    if (kp.mode == 1 && kp.ch_off) {
        const int k = point_channel(kp, e);
        gi = (uint64_t)(e - kp.ch_off[k]);
        sub = (uint64_t)k;
    }
    uint64_t c[4] = {gi, given ? 0ull : iteration, sub, 12ull};
    philox4x64_10(c, kp.seed, 0ull);
    int k = (int)(unit_from_bits(c[0]) * MF_PROC::NJAMP);
    return k < MF_PROC::NJAMP ? k : MF_PROC::NJAMP - 1;
}

// Colour-summed |M|^2 of one helicity: the colour flows of the program, then
// the full colour sum (FMA units, or the tensor cores with TC) or, for a
// process generated with the leading-colour approximation, only the diagonal
// of the colour matrix; with CS, the colour-sampled estimate of flow krow.
// With TC every thread of the block must call it the same number of times.
template <typename R, bool TC, bool CS = false>
MF_DEV double helicity_value(const KParams &kp, const R *ms, const R *idn, const int8_t *hel, const cx<R> *cpl,
                             const R *mass_r, tc::State *tcs, int krow = -1) {
    using namespace MF_PROC;
    if constexpr (CS) {
        cx<R> J[NJAMP];
        helicity_jamp<R>(ms, idn, hel, cpl, mass_r, J);
        return sampled_colour_value<R>(J, krow);
    } else if constexpr (LEADING_COLOUR || TC) {
        cx<R> J[NJAMP];
        helicity_jamp<R>(ms, idn, hel, cpl, mass_r, J);
        if constexpr (LEADING_COLOUR) return (double)colour_sum_lc<R>(J);
        else return (double)(tc::colour_sum<NJAMP>(*tcs, J) * (float)INV_COLOUR_DEN);
    } else {
        return (double)helicity_msq<R>(ms, idn, hel, cpl, mass_r);
    }
}

// Both members' values of a helicity pair: their colour sums, or with CS
// their colour-sampled estimates from flow krow.
template <typename R, bool CS>
MF_DEV void pair_values(const R *ms, const R *idn, const int8_t *hel, const cx<R> *cpl, const R *mass_r, int krow,
                        double &va, double &vb) {
    if constexpr (CS) {
        cx<R> J[MF_PROC::NJAMP], Jb[MF_PROC::NJAMP];
        MF_PROC::helicity_pair_jamp<R>(ms, idn, hel, cpl, mass_r, J, Jb);
        va = sampled_colour_value<R>(J, krow);
        vb = sampled_colour_value<R>(Jb, krow);
    } else {
        R a, b;
        MF_PROC::helicity_pair_msq<R>(ms, idn, hel, cpl, mass_r, a, b);
        va = (double)a;
        vb = (double)b;
    }
}

// Whether helicity sampling draws pairs (mode 2, a process with pairs, not
// the tensor-core kernel, which evaluates single helicities).
template <bool TC>
MF_DEV bool sample_pairs(const KParams &kp) {
    return MF_PROC::PAIR_LEG >= 0 && !TC && kp.hel_sample == 2 && kp.npairs > 0;
}

// One tile of BLOCK events: phases A, B and C.  Ends with a block barrier.
// With TC the colour sum of phase B runs on the tensor cores (R = float,
// BLOCK = 128, tcs set up by the caller).  VARIANT 1 (the flow kernel)
// replaces phase B by the leading-colour flow draw of mode 5; VARIANT 2
// (the colour-sampled kernel) replaces each colour sum by the estimate from
// one colour flow per point.  Each variant is a kernel of its own, so that
// the integrand kernel carries none of their code.
template <typename R, int BLOCK, int HT, bool TC = false, int VARIANT = 0>
MF_DEV void tile_body(const KParams &kp, const int64_t tile, unsigned char *smem_raw, const double *s_grid,
                      const cx<R> *cpl, const R *mass_r, tc::State *tcs = nullptr) {
    using namespace MF_PROC;
    R *s_mom = reinterpret_cast<R *>(smem_raw);                                   // [BLOCK][NLEG][4]
    R *s_den = s_mom + BLOCK * NLEG * 4;                                           // [BLOCK][NDEN1]
    constexpr int NDEN1 = NDEN > 0 ? NDEN : 1;
    double *s_pref = reinterpret_cast<double *>(
        reinterpret_cast<unsigned char *>(s_den + BLOCK * NDEN1) +
        ((16 - ((BLOCK * NDEN1 * sizeof(R)) % 16)) % 16));
    double *s_msq = s_pref + BLOCK;
    int *s_list = reinterpret_cast<int *>(s_msq + BLOCK);
    int *s_warp = s_list + BLOCK;                                                  // [BLOCK/32 + 1]
    const int tid = threadIdx.x;
    const int lane32 = tid & 31, warp = tid >> 5;
    const uint64_t iteration = kp.iter_dev ? (uint64_t)*kp.iter_dev : kp.iteration;
    {
        const int64_t e = tile * BLOCK + tid;
        bool ok = false, finite_in = true;
        double pref = 0.0, jv = 1.0;
        uint8_t bins[NDIM];
        int chn = kp.channel;                       // phase-space channel of the point (-1: flat)
        int64_t bin_base = e, bin_stride = kp.n;    // where the point's bin indices go (mode 1)
        if (e < kp.n) {
            // ---------------- phase A: kinematics in double precision
            double y[NDIM];
            if (kp.mode != 1 && kp.mode != 3 && kp.mode != 4 && kp.mode != 5) {
#pragma unroll
                for (int j = 0; j < NDIM; ++j) {
                    y[j] = kp.x[(int64_t)j * kp.n + e];
                    finite_in &= isfinite(y[j]);
                }
            } else {
                uint64_t gi = (kp.mode == 3 || kp.mode == 5) ? (uint64_t)kp.idx[e] : (uint64_t)(e + kp.ev0);
                uint64_t sub = kp.subprocess;
                const double *grid = s_grid;
                if (kp.mode == 1 && kp.ch_off) {
                    // one launch over every channel: point e is point gi of channel chn
                    chn = point_channel(kp, e);
                    const int64_t off = kp.ch_off[chn];
                    gi = (uint64_t)(e - off);
                    sub = (uint64_t)chn;
                    grid = kp.ch_grids[chn];
                    bin_base = off * NDIM + (e - off);
                    bin_stride = kp.ch_off[chn + 1] - off;
                }
#pragma unroll
                for (int b = 0; b < (NDIM + 3) / 4; ++b) {
                    uint64_t c[4] = {gi, iteration, sub, (uint64_t)b};
                    philox4x64_10(c, kp.seed, 0ull);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (4 * b + q < NDIM) y[4 * b + q] = unit_from_bits(c[q]);
                }
#pragma unroll
                for (int j = 0; j < NDIM; ++j) {
                    double xj;
                    int bj;
                    jv *= vegas_map1(grid + j * (kp.nb + 1), kp.nb, y[j], xj, bj);
                    y[j] = xj;
                    bins[j] = (uint8_t)bj;
                }
            }
            EventKin<double> ev;
            ok = phase_a<double>(kp, y, kp.masses, kp.ln_tau_min, ev, chn) && finite_in;
            if (kp.mode == 3) {
                // event record: x1, x2 and the momenta boosted along z from the
                // partonic centre-of-mass frame to the collider frame
                double *rec = kp.f + e * (2 + 4 * NLEG);
                const double ch = cosh(ev.yb), sh = sinh(ev.yb);
                rec[0] = ok ? ev.x1 : 0.0;
                rec[1] = ok ? ev.x2 : 0.0;
#pragma unroll
                for (int i = 0; i < NLEG; ++i) {
                    rec[2 + 4 * i] = ok ? ch * ev.p[i][0] + sh * ev.p[i][3] : 0.0;
                    rec[3 + 4 * i] = ok ? ev.p[i][1] : 0.0;
                    rec[4 + 4 * i] = ok ? ev.p[i][2] : 0.0;
                    rec[5 + 4 * i] = ok ? sh * ev.p[i][0] + ch * ev.p[i][3] : 0.0;
                }
                ok = false;            // no helicity work for records
            }
            if (kp.mode == 4) {
                // observables of the point in the collider frame (boost along
                // z by the rapidity of the parton pair); points failing the
                // threshold or the cuts are not binned
                const double ch = cosh(ev.yb), sh = sinh(ev.yb);
                for (int k = 0; k < kp.n_obs; ++k) {
                    uint16_t b = 0xFFFFu;
                    if (ok) {
                        const double *q = ev.p[kp.obs_leg[k]];
                        const double E = ch * q[0] + sh * q[3], pz = sh * q[0] + ch * q[3];
                        const double pt = sqrt(q[1] * q[1] + q[2] * q[2]);
                        const int kind = kp.obs_kind[k];
                        const double v = kind == 0 ? pt : kind == 1 ? 0.5 * log((E + pz) / (E - pz)) : asinh(pz / pt);
                        const double t = (v - kp.obs_lo[k]) * kp.obs_scale[k];
                        if (t >= 0.0 && t < (double)kp.obs_nbins[k]) b = (uint16_t)t;
                    }
                    kp.obs_out[(int64_t)k * kp.n + e] = b;
                }
                ok = false;            // no helicity work for observables
            }
            if (ok && kp.hel_sample) {
                // helicity sampling: one helicity (or, in mode 2, one helicity
                // pair) per point, uniform over the non-vanishing ones, from
                // Philox block 14 of the point's counter
                const bool per_channel = kp.mode == 1 && kp.ch_off;
                uint64_t c[4] = {kp.mode == 0 ? (uint64_t)e
                                 : (kp.mode == 3 ? (uint64_t)kp.idx[e]
                                                 : (per_channel ? (uint64_t)(e - kp.ch_off[chn]) : (uint64_t)(e + kp.ev0))),
                                 kp.mode == 0 ? 0ull : iteration,
                                 kp.mode == 0 ? 0ull : (per_channel ? (uint64_t)chn : kp.subprocess), 14ull};
                philox4x64_10(c, kp.seed, 0ull);
                const int nchoice = sample_pairs<TC>(kp) ? kp.npairs : kp.nhel;
                int h = (int)(unit_from_bits(c[0]) * nchoice);
                if (h >= nchoice) h = nchoice - 1;
                s_msq[tid] = (double)h;
            }
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
        // ---------------- phase B': the leading-colour flow of an event
        // (mode 5): per flow k the helicity sum of C_kk |J_k|^2 (the lanes'
        // helicities, then a butterfly over the HT lanes), and a flow drawn
        // with probability proportional to it by the first unit number of
        // Philox counter (point, iteration, subprocess, 13)
        if constexpr (VARIANT == 1) {
            const int EPR = BLOCK / HT, sub = tid % HT;
            const int nhp = kp.nhel_pow2;
            const int per = nhp >= HT ? nhp / HT : 1;
            for (int base = 0; base < npass; base += EPR) {
                const int slot = base + tid / HT;
                const bool valid = slot < npass;
                const int ev = s_list[valid ? slot : 0];
                const R *ms = s_mom + ev * NLEG * 4;
                const R *idn = s_den + ev * NDEN1;
                double wk[NJAMP];
#pragma unroll
                for (int k = 0; k < NJAMP; ++k) wk[k] = 0.0;
                for (int q = 0; q < per; ++q) {
                    const int h = sub * per + q;
                    const bool hv = h < kp.nhel;
                    cx<R> J[NJAMP];
                    helicity_jamp<R>(ms, idn, kp.hel[hv ? h : 0], cpl, mass_r, J);
                    if (hv && valid) {
#pragma unroll
                        for (int k = 0; k < NJAMP; ++k)
                            wk[k] += (double)COLOUR_NUM[k * NJAMP + k] *
                                     ((double)J[k].re * (double)J[k].re + (double)J[k].im * (double)J[k].im);
                    }
                }
#pragma unroll
                for (int k = 0; k < NJAMP; ++k)
#pragma unroll
                    for (int off = 1; off < HT; off <<= 1) {
                        const double o = __shfl_xor_sync(0xffffffffu, wk[k], off);
                        wk[k] = (sub & off) ? (o + wk[k]) : (wk[k] + o);
                    }
                if (sub == 0 && valid) {
                    const int64_t pe = tile * BLOCK + ev;
                    uint64_t c[4] = {(uint64_t)kp.idx[pe], iteration, kp.subprocess, 13ull};
                    philox4x64_10(c, kp.seed, 0ull);
                    double tot = 0.0;
#pragma unroll
                    for (int k = 0; k < NJAMP; ++k) tot += wk[k];
                    const double target = unit_from_bits(c[0]) * tot;
                    int pick = -1;
                    double cum = 0.0;
#pragma unroll
                    for (int k = 0; k < NJAMP; ++k) {
                        cum += wk[k];
                        if (pick < 0 && wk[k] > 0.0 && target < cum) pick = k;
                    }
                    if (pick < 0 && tot > 0.0) {     // target rounded onto the total
                        for (int k = NJAMP - 1; k >= 0 && pick < 0; --k)
                            if (wk[k] > 0.0) pick = k;
                    }
                    kp.flow_out[pe] = pick;
                }
            }
        }
        // ---------------- phase B: helicity amplitudes, HT lanes per event
        if constexpr (VARIANT != 1) {
            // HT lanes per point, each running the program for a contiguous
            // block of helicities; with helicity sampling one lane per point
            // and its sampled helicity (one call site of the program either way)
            const bool samp = kp.hel_sample != 0;
            // helicity pairs (summed helicities of modes 0 and 1): each lane
            // evaluates whole pairs, whose two |M|^2 are consecutive leaves
            // of the summation tree
            const bool pairs = PAIR_LEG >= 0 && !TC && !samp && kp.mode <= 1 && kp.npairs > 0;
            const bool samp_pair = samp && sample_pairs<TC>(kp);
            const int EPR = samp ? BLOCK : BLOCK / HT;  // points per round
            const int sub = samp ? 0 : tid % HT;
            const int nhp = pairs ? kp.npairs_pow2 : kp.nhel_pow2;   // padded units (power of two)
            const int per = samp ? 1 : (nhp >= HT ? nhp / HT : 1);   // units per lane
            // every thread runs the program the same number of times (lanes
            // without an event or a helicity compute on a valid stand-in and
            // discard it), so that the program may contain block barriers
            for (int base = 0; base < npass; base += EPR) {
                const int slot = base + (samp ? tid : tid / HT);
                const bool valid = slot < npass;
                PairSum ps;
                ps.init();
                const int ev = s_list[valid ? slot : 0];
                const int hs = (samp && valid) ? (int)s_msq[ev] : 0;
                const R *ms = s_mom + ev * NLEG * 4;
                const R *idn = s_den + ev * NDEN1;
                int krow = -1;
                if constexpr (VARIANT == 2) krow = sampled_colour_flow(kp, tile * BLOCK + ev, iteration);
                if constexpr (PAIR_LEG >= 0 && !TC) {
                    if (samp_pair) {
                        // the sampled pair: its present members' |M|^2
                        const uint8_t ia = kp.pairs[hs][0], ib = kp.pairs[hs][1];
                        double va, vb;
                        pair_values<R, VARIANT == 2>(ms, idn, kp.hel[ia != 0xFF ? ia : ib], cpl, mass_r, krow, va, vb);
                        ps.add((valid && ia != 0xFF) ? va : 0.0);
                        ps.add((valid && ib != 0xFF) ? vb : 0.0);
                    }
                    if (pairs) {
                        for (int k = 0; k < per; ++k) {
                            const int u = sub * per + k;
                            const bool uv = u < kp.npairs;
                            const uint8_t ia = kp.pairs[uv ? u : 0][0], ib = kp.pairs[uv ? u : 0][1];
                            double va, vb;
                            pair_values<R, VARIANT == 2>(ms, idn, kp.hel[ia != 0xFF ? ia : ib], cpl, mass_r, krow, va,
                                                         vb);
                            ps.add((uv && valid && ia != 0xFF) ? va : 0.0);
                            ps.add((uv && valid && ib != 0xFF) ? vb : 0.0);
                        }
                    }
                }
                for (int k = 0; k < ((pairs || samp_pair) ? 0 : per); ++k) {
                    const int h = samp ? hs : sub * per + k;
                    const bool hv = h < kp.nhel;
                    double v = helicity_value<R, TC, VARIANT == 2>(kp, ms, idn, kp.hel[hv ? h : 0], cpl, mass_r, tcs,
                                                                   krow);
                    if (!(hv && valid)) v = 0.0;
                    if (kp.mode == 2 && hv && valid) kp.f[(int64_t)h * kp.n + tile * BLOCK + ev] = v;
                    ps.add(v);
                }
                double part = ps.total();
                if (samp) {
                    if (valid) s_msq[ev] = part * (double)(samp_pair ? kp.npairs : kp.nhel);
                } else {
#pragma unroll
                    for (int off = 1; off < HT; off <<= 1) {
                        double o = __shfl_xor_sync(0xffffffffu, part, off);
                        // lanes combine (lower block) + (upper block) in that order
                        part = (sub & off) ? (o + part) : (part + o);
                    }
                    if (sub == 0 && slot < npass) s_msq[s_list[slot]] = part;
                }
            }
        }
        __syncthreads();
        // ---------------- phase C: outputs
        if (e < kp.n) {
            double fval = ok ? s_pref[tid] * s_msq[tid] : 0.0;
            if (kp.mode == 0) {
                // a point with a non-finite coordinate gives NaN; any
                // non-finite value raises the non-finite flag (3) unless a
                // more serious error is flagged already
                if (!finite_in) fval = __longlong_as_double(0x7FF8000000000000ll);
                if (!isfinite(fval) && kp.err) atomicCAS(kp.err, 0, 3);
                kp.f[e] = fval;
            } else if (kp.mode == 1) {
                kp.w_out[e] = fval * jv;
#pragma unroll
                for (int j = 0; j < NDIM; ++j) kp.bins_out[bin_base + (int64_t)j * bin_stride] = bins[j];
            }
        }
        __syncthreads();
    }
}

// Whether the launch provided at least `need` bytes of dynamic shared memory;
// if not, flag the error (code 2) and let the whole block return.
MF_DEV bool smem_ok(const KParams &kp, size_t need) {
    uint32_t have;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(have));
    if (have >= need) return true;
    if (threadIdx.x == 0 && kp.err) atomicExch(kp.err, 2);
    return false;
}

// The single-process kernel: a grid-stride loop over tiles (VARIANT 1: the
// leading-colour flow kernel of mode 5; 2: the colour-sampled integrand).
template <typename R, int BLOCK, int HT, int VARIANT = 0>
MF_DEV void kernel_body(const KParams &kp) {
    using namespace MF_PROC;
    if (!smem_ok(kp, tile_smem_bytes<R, BLOCK>())) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_grid[NDIM * 65];
    __shared__ cx<R> cpl[8];
    __shared__ R mass_r[8];
    load_block_constants<R, BLOCK>(kp, s_grid, cpl, mass_r);
    __syncthreads();
    const int64_t ntiles = (kp.n + BLOCK - 1) / BLOCK;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        tile_body<R, BLOCK, HT, false, VARIANT>(kp, tile, smem_raw, s_grid, cpl, mass_r);
}

// The single-process kernel with the colour sum on the tensor cores
// (FP32 amplitudes, 128 threads): tensor memory and the operand buffers are
// set up once per block, after the tile buffers in dynamic shared memory.
template <int HT>
MF_DEV void kernel_body_tc(const KParams &kp) {
    using namespace MF_PROC;
    constexpr int BLOCK = 128;
    // with the stacked operands (many colour flows) the shared memory goes to
    // the tensor-core operands and the grid is read from global memory
    constexpr bool GRID_GLOBAL = tc::Plan<NJAMP>::STACKED;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ double s_grid[GRID_GLOBAL ? 1 : NDIM * 65];
    __shared__ cx<float> cpl[8];
    __shared__ float mass_r[8];
    constexpr size_t tile_bytes = (tile_smem_bytes<float, BLOCK>() + 1023) / 1024 * 1024;
    if (!smem_ok(kp, tile_bytes + tc::Plan<NJAMP>::SMEM)) return;
    tc::State tcs;
    tc::setup<NJAMP>(tcs, smem_raw + tile_bytes, kp.err, kp.wait_polls);
    tc::load_colour<NJAMP>(tcs, COLOUR_NUM);
    load_block_constants<float, BLOCK>(kp, s_grid, cpl, mass_r, !GRID_GLOBAL);
    __syncthreads();
    const double *grid = GRID_GLOBAL ? kp.grid : s_grid;
    const int64_t ntiles = (kp.n + BLOCK - 1) / BLOCK;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        tile_body<float, BLOCK, HT, true>(kp, tile, smem_raw, grid, cpl, mass_r, &tcs);
    tc::teardown<NJAMP>(tcs);
}

}  // namespace MF_BODY
#undef MF_PROC
#undef MF_BODY
