// Kernel parameter block of the generated process kernel, shared verbatim by
// the host library (C++) and the run-time compiled device code, so that both
// sides agree on the layout.  Passed by value to the kernel.
#pragma once

#define MF_KP_MAX_HEL 256
#define MF_KP_MAX_OBS 4

struct mf_kparams {
    int64_t n;                 // events
    int32_t mode;              // 0: integrand of given points, 1: Vegas,
                               // 2: per-helicity |M|^2 of given points into f[h][n],
                               // 3: event records of the Vegas points idx[0..n) into
                               //    f[n][2 + 4 NLEG] (x1, x2, lab-frame momenta),
                               // 4: observable bins of the Vegas points into obs_out,
                               // 5: leading-colour flow drawn for the Vegas points
                               //    idx[0..n) into flow_out
    int32_t nhel;              // helicity rows in hel[]
    int32_t nhel_pow2;         // a power of two >= nhel (pairwise-sum padding)
    int32_t nb;                // Vegas bins per dimension
    const double *x;           // modes 0, 2: points, SoA [NDIM][n]
    double *f;                 // mode 0: f [n]; mode 2: [nhel][n]
    const double *grid;        // mode 1: edges [NDIM][nb+1]
    double *w_out;             // mode 1: w = f J_V [n]
    uint8_t *bins_out;         // mode 1: bin indices, SoA [NDIM][n]
    uint64_t seed, iteration, subprocess;
    int64_t ev0;               // mode 1: Philox counter of the first point
    double S;                  // collider energy squared
    double ln_tau_min;         // ln((sum of final masses)^2 / S)
    double w0_const;           // massless phase-space volume / s-hat^(n-2)
    double pref_const;         // averaging x GeV^-2 -> pb / 2 (flux 1/(2 s-hat))
    double pt_min2, dr_min2;   // cuts
    double pdf_a0, pdf_h;      // first ln-x knot and spacing
    int32_t pdf_nx;
    int32_t pad1;
    const double *pdf_rows;    // [2 beams][2: values, slopes][pdf_nx]
    double *g_dparam;          // gradient kernel: df/dm_t, df/dalpha_s, [2][n]
    double *g_dx;              // gradient kernel: df/dx_j, [NDIM][n] (may be NULL)
    double alpha_s;            // strong coupling the couplings were built with
    int32_t alpha_s_power;     // |M|^2 ~ alpha_s^power
    int32_t pad2;
    int *err;                  // device error flag (expired waits), may be NULL
    const int64_t *idx;        // mode 3: global point indices
    int32_t hel_sample;        // 1: one helicity per point, drawn uniformly, f scaled by nhel
    int32_t npairs;            // modes 0, 1: helicity pairs in pairs[] (0: one helicity at a time)
    int32_t npairs_pow2;       // a power of two >= npairs
    int32_t pad3;
    int64_t wait_polls;        // polls of a bounded wait per tensor-core colour-sum round
    const long long *iter_dev; // if set, the iteration index is read here (graph replays)
    uint16_t *obs_out;         // mode 4: bins [n_obs][n], 0xFFFF: not binned
    int32_t *flow_out;         // mode 5: colour-flow index [n], -1: none
    int32_t variant;           // kernel of the module to launch (host side): 0 the integrand
                               // kernel, 1 the flow kernel (mode 5), 2 the colour-sampled kernel
    int32_t colour_sample;     // the process samples one colour flow per point
    int32_t n_obs;             // mode 4: observables
    int32_t obs_kind[MF_KP_MAX_OBS];   // 0: pT, 1: rapidity, 2: pseudorapidity (collider frame)
    int32_t obs_leg[MF_KP_MAX_OBS];
    int32_t obs_nbins[MF_KP_MAX_OBS];
    int32_t pad4;
    double obs_lo[MF_KP_MAX_OBS];      // bin b = floor((v - lo) * scale) if 0 <= b < nbins
    double obs_scale[MF_KP_MAX_OBS];   // nbins / (hi - lo)
    const int32_t *chan;       // multichannel table (device/mf_channels.cuh), may be NULL
    int32_t channel;           // modes 0, 1: phase-space channel of the points, -1: RAMBO
    int32_t ch_count;          // mode 1 with ch_off: channels of the launch
    double ch_s0, ch_t0;       // channel propagator regulators (GeV^2)
    // mode 1, one launch over every channel: points [ch_off[k], ch_off[k+1])
    // are points 0.. of channel k, mapped through grid ch_grids[k]; their bin
    // indices go to bins_out + ch_off[k] NDIM as SoA [NDIM][n_k]
    const long long *ch_off;
    const double *const *ch_grids;
    double masses[8];
    double couplings[16];      // 8 complex couplings (re, im)
    int8_t hel[MF_KP_MAX_HEL][8];
    // rows of hel[] forming a pair (same helicities except at the process's
    // pair leg, -1 in the first member and +1 in the second); 0xFF: the row
    // is absent (that helicity vanishes)
    uint8_t pairs[MF_KP_MAX_HEL][2];
};

// Parameters of the batched kernel: several processes' parameter blocks, the
// work items of the batch (groups of tiles, fewer tiles per item for the
// costlier processes so that items cost about the same) and the work counter
// the blocks draw items from (zeroed before each launch).
#define MF_KP_MAX_BATCH 8
struct mf_batch_params {
    long long *counter;
    int32_t nproc;
    int32_t pad;
    long long start[MF_KP_MAX_BATCH + 1];     // work items of process k: [start[k], start[k+1])
    long long group[MF_KP_MAX_BATCH];         // tiles per work item of process k
    long long ntiles[MF_KP_MAX_BATCH];        // tiles of process k
    mf_kparams kp[MF_KP_MAX_BATCH];
};
