/*
 * madflow_gb.h -- C ABI of the GB300-native leading-order integrand library.
 *
 * The library evaluates the per-event leading-order integrand of the MadFlow
 * method (arXiv:2106.10279): for each phase-space point, flat RAMBO momenta and
 * weight (Sec. 2.4), the parton luminosity from interpolated PDF tables (Sec. 1,
 * Fig. 1), and the helicity-amplitude matrix element summed over helicities and
 * colours (Sec. 2.3), combined as L(x1,x2) x sigma-hat (Fig. 1); and it drives the
 * Vegas iteration around it (Sec. 2.2: random numbers -> phase space -> matrix
 * element -> histogram accumulation).
 *
 * Conventions shared by every entry point:
 *   - All functions return an mf_status.  Nothing aborts, throws across the ABI
 *     or traps on the device.  mf_last_error() returns a thread-local message.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *     passes; the library owns the objects it creates (mf_process, mf_vegas) and
 *     their internal device scratch, and frees them in the matching destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous on that stream unless stated otherwise.
 *   - Momenta are (E, px, py, pz) in GeV, metric (+,-,-,-).
 *   - Arrays of events are structure-of-arrays: x[j * n + i] is coordinate j of
 *     event i.
 */
#ifndef MADFLOW_GB_H
#define MADFLOW_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MF_OK = 0,
    MF_EINVAL = 1,        /* malformed argument or descriptor */
    MF_ENOMEM = 2,        /* device or host allocation failed */
    MF_ECUDA = 3,         /* a CUDA runtime/driver call failed */
    MF_ENAN = 4,          /* results were written, but some events were not finite */
    MF_ETIMEOUT = 5,      /* a bounded device wait gave up */
    MF_EUNSUPPORTED = 6,  /* valid request outside what this build implements */
    MF_EJIT = 7           /* run-time compilation of the process kernels failed */
} mf_status;

/* Arithmetic of the matrix element (Sec. 2.3).  MF_FP64: everything in double
 * precision.  MF_MIXED: spinors, currents, amplitudes and the colour sum in
 * single precision; phase space, invariants and propagator denominators, PDFs,
 * weights and all accumulators in double precision.  MF_MIXED_TC: MF_MIXED
 * with the colour sum on the tensor cores (tcgen05, split TF32; see
 * mf_colour_sum), 128 threads per block; up to 64 colour flows the operand
 * rows are [Re J | Im J] against diag(C, C), above 64 the real and imaginary
 * parts are stacked as separate rows against C (two MMA rounds per call, the
 * Vegas grid read from global memory).  (Value 2 is the gradient kernel in
 * mf_generate_kernel_source.) */
typedef enum { MF_FP64 = 0, MF_MIXED = 1, MF_MIXED_TC = 3 } mf_precision;

/* ------------------------------------------------------------------------ */
/* Process descriptor: the diagram program of Sec. 2.3 (the Matrix class the   */
/* MadFlow exporter writes, here as data).                                     */
/* ------------------------------------------------------------------------ */

/* Role of an external leg in the fermion flow. */
typedef enum {
    MF_LEG_FERMION_IN = 0,   /* column spinor: u of an incoming fermion, v of an outgoing antifermion */
    MF_LEG_FERMION_OUT = 1,  /* row spinor: u-bar of an outgoing fermion, v-bar of an incoming antifermion */
    MF_LEG_VECTOR = 2        /* massless vector boson: eps (incoming) or eps* (outgoing) */
} mf_leg_kind;

/* Routines of the diagram program (HELAS/ALOHA roles, Sec. 2.3).  Every
 * wavefunction carries the momentum flowing INTO the diagram through the legs it
 * contains.  "coupling" is the complex vertex factor c; "inv_den" below means
 * 1 / (P^2 - M^2) of the current's momentum P and propagator mass M.
 *   MF_R_IXX, MF_R_OXX, MF_R_VXX  external column spinor / row spinor / vector
 *   MF_R_FFV_AMP(row, col, V)     c * row . (gamma^mu V_mu) . col
 *   MF_R_FFV_FIN(col, V)          i inv_den (q-slash + M) c (V-slash) col,  q = P
 *   MF_R_FFV_FOUT(row, V)         i inv_den row c (V-slash) (q-slash + M),  q = -P
 *   MF_R_FFV_VEC(row, col)        -i inv_den c row gamma^mu col
 *   MF_R_VVV_AMP(A, B, C)         c V3(A,B,C),  V3 = (A.B)((kA-kB).C) + (B.C)((kB-kC).A)
 *                                                + (C.A)((kC-kA).B), k = incoming momenta
 *   MF_R_VVV_VEC(A, B)            -i inv_den c [(A.B)(kA-kB) + B ((kB-kC).A) + A ((kC-kA).B)],
 *                                 kC = -(kA+kB)
 *   MF_R_VVVVs_AMP(A, B, C, D)    c x  s=1: (A.C)(B.D)-(A.D)(B.C)   s=2: (A.B)(C.D)-(A.D)(B.C)
 *                                      s=3: (A.B)(C.D)-(A.C)(B.D)   (colour f^abe f^cde,
 *                                      f^ace f^bde, f^ade f^bce of the four-gluon vertex)
 *   MF_R_VVVVs_VEC(A, B, C)       -i inv_den c x  s=1: (A.C)B-(B.C)A  s=2: (A.B)C-(B.C)A
 *                                                  s=3: (A.B)C-(A.C)B
 */
typedef enum {
    MF_R_IXX = 0, MF_R_OXX = 1, MF_R_VXX = 2,
    MF_R_FFV_AMP = 10, MF_R_FFV_FIN = 11, MF_R_FFV_FOUT = 12, MF_R_FFV_VEC = 13,
    MF_R_VVV_AMP = 20, MF_R_VVV_VEC = 21,
    MF_R_VVVV1_AMP = 30, MF_R_VVVV2_AMP = 31, MF_R_VVVV3_AMP = 32,
    MF_R_VVVV1_VEC = 33, MF_R_VVVV2_VEC = 34, MF_R_VVVV3_VEC = 35
} mf_routine;

typedef enum { MF_OP_EXT = 0, MF_OP_CUR = 1, MF_OP_AMP = 2 } mf_op_kind;

/* One op of the program.  Ops are evaluated in order; op k's result is
 * wavefunction k (EXT and CUR ops).  Inputs name earlier ops. */
typedef struct {
    int32_t kind;          /* mf_op_kind */
    int32_t routine;       /* mf_routine */
    int32_t in[4];         /* input op indices, -1 when unused */
    int32_t leg;           /* EXT: external leg index */
    int32_t coupling;      /* CUR/AMP: index into couplings[] */
    int32_t mass_id;       /* CUR: propagator mass = masses[mass_id], -1 = massless */
    int32_t first_term;    /* AMP: colour terms terms[first_term .. first_term+n_terms) */
    int32_t n_terms;
} mf_op;

/* AMP op contributes (re + i im) * amplitude to JAMP[jamp]. */
typedef struct {
    int32_t jamp;
    int32_t pad_;
    double re, im;
} mf_colour_term;

#define MF_MAX_LEGS 8
#define MF_MAX_JAMP 128
#define MF_MAX_DIM 20
#define MF_MAX_ITER 1024        /* Vegas iterations per grid */
#define MF_MAX_TREE_NODES 128  /* tree nodes one shard returns */
#define MF_CHUNK 4096          /* points per accumulation chunk */
#define MF_STATIC_MAX_EVENTS 262144  /* points per mf_vegas_iterate_static call */

/* Code-generation and launch options of a process (the paper has no
 * counterpart: these choose how the diagram program is emitted and launched,
 * never what it computes).  A field set to MF_OPT_AUTO (-1) lets the library
 * decide; mf_process_options_init sets every field to it, and a descriptor
 * whose options pointer is NULL uses the defaults.
 *   amplitude_units  1: FFV amplitudes that share the row and column spinors
 *                    and whose colour coefficients agree up to +-1, +-i are
 *                    evaluated as one amplitude of the summed vector currents;
 *                    0: one amplitude at a time (default 1);
 *   call_routines    0: every vertex routine inlined; 1: every routine called
 *                    as a non-inlined function; 2: the currents called; 3: the
 *                    amplitudes called (default: 1 for long programs, else 3);
 *   order_search     iterations of the local search on the amplitude order
 *                    (default: 4000 where amplitude units exist, else 0);
 *   sync_every       block barrier every this many amplitudes in the program,
 *                    0: none (default: 16 for long programs, else 0);
 *   program_parts    functions the program is split into (default: by size);
 *   min_blocks       minimum of resident blocks per SM the compiler must
 *                    allow (__launch_bounds__), 0: none (default 0);
 *   helicity_pairs   0: helicities one at a time; 1: pairs where they save
 *                    FLOPs (default: 1, except for programs above 1.5e5
 *                    FLOPs per helicity, whose pair program is not
 *                    generated: their single-helicity program alone takes
 *                    minutes to compile);
 *   block            threads per block, 128 or 256 (default: 256 for long
 *                    programs, 128 otherwise and for MF_MIXED_TC);
 *   lanes            lanes per point, 1..32 and a power of two, at most the
 *                    padded count of pairs or helicities (default: that count,
 *                    at most 32);
 *   blocks_per_sm    resident blocks per SM the grid is sized for, 1..8
 *                    (default: the occupancy the compiled kernel reports);
 *   ptxas_level      optimisation level 0..3 of the device assembler for the
 *                    process kernels (default 3);
 *   wait_polls       polls of the bounded wait on each round of tensor-core
 *                    MMAs in MF_MIXED_TC kernels before the round is given up
 *                    and MF_ETIMEOUT flagged, 0 .. 2^30 (default 2^24; the
 *                    wait before tensor memory is released always uses the
 *                    default).
 * Block, lanes and blocks_per_sm never change results; the other fields may
 * change the last bits (the order of floating-point operations). */
#define MF_OPT_AUTO (-1)
typedef struct {
    int32_t amplitude_units;
    int32_t call_routines;
    int32_t order_search;
    int32_t sync_every;
    int32_t program_parts;
    int32_t min_blocks;
    int32_t helicity_pairs;
    int32_t block;
    int32_t lanes;
    int32_t blocks_per_sm;
    int32_t ptxas_level;
    int32_t wait_polls;
} mf_process_options;

/* Set every field of *opt to MF_OPT_AUTO. */
mf_status mf_process_options_init(mf_process_options *opt);

typedef struct {
    /* external legs; legs 0 and 1 are the incoming partons along +z and -z */
    int32_t n_legs;
    const int32_t *leg_kind;        /* host [n_legs] mf_leg_kind */
    const int32_t *leg_incoming;    /* host [n_legs] 1 incoming, 0 outgoing */
    const int32_t *leg_mass_id;     /* host [n_legs] index into masses[], -1 = massless */
    const int32_t *leg_cut;         /* host [n_legs] 1 = subject to the pT / Delta R cuts */
    int32_t n_masses;
    const double *masses;           /* host [n_masses] GeV; masses[0] is the top mass m_t */
    /* diagram program */
    int32_t n_ops;
    const mf_op *ops;               /* host [n_ops] */
    int32_t n_terms;
    const mf_colour_term *terms;    /* host [n_terms] */
    int32_t n_couplings;
    const double *couplings;        /* host [2 * n_couplings] (re, im) pairs */
    /* colour matrix C = colour_num / colour_den, symmetric, [n_jamp][n_jamp] */
    int32_t n_jamp;
    const int32_t *colour_num;      /* host [n_jamp * n_jamp] */
    int32_t colour_den;
    /* helicities: n_hel rows of n_legs values +-1 (NULL: all 2^n_legs); rows
       that vanish are dropped at create time (below 1e-12 of the helicity
       sum at each of 256 seeded points: chirality zeros are rounding residues) */
    int32_t n_hel;
    const int8_t *helicities;
    double average;                 /* 1/(initial spins x colours) x identical-final factor */
    int32_t alpha_s_power;          /* |M|^2 ~ alpha_s^power */
    double alpha_s;
    /* collision */
    double sqrt_s;                  /* collider energy, GeV */
    int32_t hadronic;               /* 1: two PDF beams and the x1, x2 map; 0: fixed sqrt_s */
    const double *pdf[2];           /* host [pdf_nq][pdf_nx] tables of x f(x, Q^2), beam 1 / 2 */
    int32_t pdf_nx, pdf_nq;         /* knots uniform in ln x and in ln Q^2 */
    double pdf_x_min, pdf_x_max, pdf_q2_min, pdf_q2_max;
    double mu_f2;                   /* factorisation scale squared, GeV^2 */
    /* cuts on the legs flagged in leg_cut */
    double pt_min;                  /* pT > pt_min (GeV), 0 = none */
    double dr_min;                  /* Delta R > dr_min between flagged pairs, 0 = none */
    const mf_process_options *options;  /* host, may be NULL (all defaults); copied */
} mf_process_desc;

typedef struct mf_process mf_process;   /* opaque, library-owned */
typedef struct mf_vegas mf_vegas;       /* opaque, library-owned */
typedef struct mf_batch mf_batch;       /* opaque, library-owned */

/* mf_create_process (the process a MadFlow run integrates: the Matrix class
 * of Sec. 2.3 -- external states, vertices and the colour matrix of the
 * helicity-amplitude evaluation -- with the PDF tables and cuts of the
 * integrand of Fig. 1): validate and deep-copy *desc, drop vanishing helicities,
 * generate CUDA source specialised to the diagram program and compile it for
 * sm_103a at run time (NVRTC; compiled binaries are kept for the life of the
 * process, and on disk when the environment variable MF_JIT_CACHE names a
 * directory; MF_NVRTC_LIBRARY names the NVRTC shared library to load instead
 * of the one found at build time; MF_JIT_VERBOSE=1 prints the assembler's
 * resource report of each compilation to stderr).  The process's code-
 * generation and launch options come from desc->options (see
 * mf_process_options).  The kept helicities are grouped into pairs that differ only at
 * one leg where that saves arithmetic (mf_process_info: pair_leg, n_pairs);
 * the helicity sums of mf_integrand and mf_vegas_iterate then evaluate each
 * pair with one program.  Synchronous.  Errors: MF_EINVAL (malformed descriptor),
 * MF_EUNSUPPORTED (more than MF_MAX_LEGS legs, n_jamp > MF_MAX_JAMP),
 * MF_EJIT (compilation failed; mf_last_error has the log), MF_ECUDA, MF_ENOMEM.
 * On error *out is left NULL. */
mf_status mf_create_process(const mf_process_desc *desc, mf_process **out);
mf_status mf_destroy_process(mf_process *p);

typedef struct {
    int32_t ndim;            /* integration dimensions: 3 n_out - 4 (+2 if hadronic) */
    int32_t n_legs;
    int32_t n_hel;           /* helicities kept after filtering */
    int32_t n_hel_all;       /* helicities before filtering */
    int32_t n_jamp;
    int32_t n_ops;
    int32_t n_den;           /* distinct propagator denominators per event */
    double flops_per_hel;    /* algorithmic FLOPs of one helicity (program + colour sum) */
    double flops_kinematics; /* algorithmic FLOPs per event outside the helicity loop */
    int32_t pair_leg;        /* leg at which paired helicities differ, -1: helicities one by one */
    int32_t n_pairs;         /* helicity pairs evaluated per event (0: no pairs) */
    double flops_helicity_sum; /* FLOPs of one event's helicity sum as evaluated (pairs share
                                * the wavefunctions that do not depend on pair_leg) */
    int32_t helicity_sampling; /* sampling mode in effect (mf_process_set_helicity_sampling): 0 sum,
                                * 1 single helicities, 2 helicity pairs (MF_MIXED_TC kernels sample
                                * single helicities in mode 2) */
} mf_process_info;

mf_status mf_process_get_info(const mf_process *p, mf_process_info *info);

/* mf_integrand (Fig. 1: L(x1,x2) x sigma-hat({p})): for n points x in the open
 * unit hypercube (device, SoA [ndim][n]) write the integrand in pb to f (device
 * [n]); sigma = integral of f over the hypercube.  Hadronic processes use x_0,
 * x_1 for the momentum fractions (tau = tau_min^x0, x1 = tau^x1, x2 = tau/x1)
 * and the rest for the phase space; points failing the cuts or below threshold
 * give f = 0.  No Vegas Jacobian is applied.  A point with a non-finite
 * coordinate gives f = NaN; any non-finite f raises the process's
 * non-finite flag, which mf_process_check reports as MF_ENAN.  Asynchronous.
 * n = 0 is a no-op.  MF_EINVAL for NULL pointers with n > 0 or n < 0. */
mf_status mf_integrand(mf_process *p, const double *x, int64_t n, double *f,
                       mf_precision prec, void *stream);

/* mf_helicity_msq (the helicity loop of Sec. 2.3's smatrix, unrolled): for n
 * points x (device, SoA [ndim][n]) write the colour-summed |M|^2 of every
 * helicity row of the unfiltered table (rows of 2^n_legs in the order
 * l_0 l_1 ... with -1 before +1, or the descriptor's rows), without spin or
 * colour averaging, to out (device [n_hel_all][n]).  Rows of points that fail
 * the cuts or the threshold are left untouched (callers zero out first).
 * Asynchronous.  MF_EINVAL for NULL pointers with n > 0 or n < 0. */
mf_status mf_helicity_msq(mf_process *p, const double *x, int64_t n, double *out,
                          mf_precision prec, void *stream);

/* mf_grad: the integrand and its derivatives, all in double precision, for n
 * points x (device SoA [ndim][n]):
 *   f          (device [n])       as mf_integrand;
 *   df_dparam  (device [2][n])    row 0: df/dm_t (m_t = masses[0], entering the
 *              phase-space masses, the threshold tau_min, spinors and
 *              propagators; mu_F held fixed), row 1: df/dalpha_s = k f / alpha_s
 *              (|M|^2 ~ alpha_s^k exactly);
 *   df_dx      (device [ndim][n], or NULL)  df/dx_j.
 * Derivatives are exact to rounding: forward tangents through the per-event
 * kinematics, and the adjoint of the diagram program per helicity (wavefunctions
 * recomputed in the kernel, nothing stored between helicities).  Points failing
 * the cuts give f = 0 and zero derivatives; the moving cut boundary is not a
 * derivative term.  The run-time compiled gradient kernel is built on the
 * first call.  Asynchronous.  MF_EINVAL for NULL x, f or df_dparam with n > 0. */
mf_status mf_grad(mf_process *p, const double *x, int64_t n, double *f, double *df_dparam,
                  double *df_dx, void *stream);

/* mf_grad_channel: mf_grad for points mapped through phase-space channel
 * `channel` (see mf_vegas_iterate_channels): the derivatives follow the
 * channel's momenta and its weight a_i / g_i (through the sampled ranges,
 * the mapped densities and the partition; m_t also enters the top
 * propagators' masses there).  MF_EUNSUPPORTED if the process has no
 * channels, MF_EINVAL for a channel out of range. */
mf_status mf_grad_channel(mf_process *p, int32_t channel, const double *x, int64_t n, double *f, double *df_dparam,
                          double *df_dx, void *stream);

/* ------------------------------------------------------------------------ */
/* Vegas (Sec. 2.2; G.P. Lepage, J. Comput. Phys. 27 (1978) 192).              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t iteration;       /* index of the iteration these numbers belong to */
    int64_t n_events;        /* points sampled (including points with f = 0) */
    int64_t n_nonzero;       /* points with f != 0 */
    int64_t n_nan;           /* points whose weight was not finite (counted as 0) */
    double integral;         /* this iteration's estimate, pb */
    double error;            /* its standard error */
    double sigma;            /* inverse-variance combination of all iterations so far */
    double sigma_error;
    double chi2_dof;
} mf_iter_result;

/* mf_vegas_create: a grid of ndim dimensions x nbins bins (uniform), refinement
 * damping alpha (1.5 is the customary value).  nbins in [2, 64]. */
mf_status mf_vegas_create(int32_t ndim, int32_t nbins, double alpha, mf_vegas **out);
mf_status mf_vegas_destroy(mf_vegas *v);

/* mf_vegas_iterate: one Vegas iteration for each of nproc subprocesses, each
 * with its own grid.  Point i of subprocess k in iteration t draws its unit
 * numbers from Philox4x64-10 with key (seed, 0) and counter (i, t, k, block),
 * maps them through its grid, evaluates the integrand, accumulates sum w,
 * sum w^2 and, per dimension and bin, sum w^2 and counts in a fixed order
 * (bit-reproducible for a given seed whatever the launch configuration: per
 * chunk of MF_CHUNK points a fixed in-chunk order, across chunks the pairwise
 * tree of mf_tree_reduce), then
 * refines the grid (unless refine == 0) and combines the iteration with the
 * previous ones.  Synchronous: returns after out[k] (host [nproc]) is filled.
 * MF_ENAN if any point's weight was not finite (results still written). */
mf_status mf_vegas_iterate(mf_vegas *const *grids, mf_process *const *procs,
                           const int64_t *n_events, int32_t nproc, uint64_t seed,
                           mf_precision prec, int32_t refine, mf_iter_result *out,
                           void *stream);

/* ---- Multichannel phase space (the outlook of Sec. 4 and the caveat of
 * Sec. 2.6 "Scope": a phase space built from the process topology in place
 * of the flat RAMBO of Sec. 2.4, whose unweighting efficiency Sec. 2.5
 * puts at about 5 %; multichannel weights after Kleiss & Pittau, the
 * paper's reference for it).
 *
 * Channels.  Every AMP op of the program is one diagram; its currents are
 * its propagators.  A current holding exactly one of the incoming legs 0, 1
 * is a t-channel propagator; its final legs on the side of leg 0 form the
 * set F_j, and these sets nest, F_1 < .. < F_{k-1}.  Every other current is
 * an s-channel propagator of a cluster of final legs (for a current holding
 * both incoming legs: the final legs outside it).  The clusters
 * c_j = F_j \ F_{j-1} (F_0 = {}, F_k = all final legs) sit along the path
 * from leg 0 to leg 1; inside a cluster the s-channel propagators form a
 * binary tree, whose left child holds the smallest final index.  Diagrams
 * with a four-gluon vertex are left out, and diagrams that give equal
 * channels are merged.  Channels are numbered in ascending order of their
 * key:
 *   (k, masks of c_1..c_k, mass ids of the k-1 t-channel propagators,
 *    number of s-channel clusters, then their (mask, mass id) pairs in
 *    ascending order),
 * where the masks have bit i for final leg i (leg 2 + i) and mass id -1
 * means massless.  A process with more than six final legs has no channels.
 *
 * Map of the 3n-4 phase-space unit numbers (after x1, x2 for hadronic
 * processes; n final legs) to momenta in the partonic centre-of-mass frame,
 * in this order:
 *   (i)   masses s of the clusters c_j with two or more legs, j = 1..k:
 *         range [m(c_j)^2, (sqrt(s-hat) - sum_{i<j} sqrt(s_{c_i})
 *         - sum_{i>j} m(c_i))^2] (m(X): sum of the final masses in X);
 *   (ii)  masses of the remainders R_j = c_{j+1} + .. + c_k, j = 1..k-2,
 *         flat on [(sum_{i>j} sqrt(s_{c_i}))^2,
 *         (sqrt(s_{R_{j-1}}) - sqrt(s_{c_j}))^2], R_0 = all;
 *   (iii) for j = 1..k-1 the split R_{j-1} -> c_j + R_j in the rest frame of
 *         R_{j-1}: the polar angle of c_j about the direction of
 *         q = p_0 - c_1 - .. - c_{j-1} with density proportional to
 *         1 / (M^2 + t0 - t), t = (q - c_j)^2 and M the t-channel
 *         propagator's mass (one number), then the azimuth, flat, in the
 *         frame R_z(phi_q) R_y(theta_q) of that axis (one number);
 *   (iv)  for every cluster in spine order, its nodes X -> (L, R) in
 *         pre-order: s_L (if L is a cluster) on [m(L)^2, (sqrt(s_X) -
 *         m(R))^2], s_R (if R is a cluster) on [m(R)^2, (sqrt(s_X) -
 *         sqrt(s_L))^2], then L's direction, isotropic in X's rest frame
 *         (cos theta, phi about the fixed axes).
 * A cluster mass has density proportional to 1 / (s - M^2 + s0) on its range
 * (M its propagator's mass; flat if the range's lower end has
 * lo - M^2 + s0 <= 0).  Two-body momenta are built in the parent's rest
 * frame and boosted back without rotation.
 *
 * Weight.  A point of channel i weighs a_i / g_i in place of the RAMBO
 * weight: g_i is the channel's density relative to
 * dPhi_n = prod ds/(2 pi) prod lambda^(1/2)/(32 pi^2 s) dOmega, and
 * a_i = P_i / sum_j P_j with P_i the product over channel i's propagators
 * of 1 / (|x - M^2| + r)^2 (x the propagator's s -- s-hat for the
 * propagator into a one-cluster final state -- or t; r = s0 or t0).  The
 * a_i sum to one, so the cross section is the sum of the channels'
 * integrals of f a_i / g_i, each over its own unit hypercube. */

/* mf_process_channels: the number of channels of the process (0 if it has
 * none; the channel calls then return MF_EUNSUPPORTED). */
mf_status mf_process_channels(const mf_process *p, int32_t *n_channels);

/* mf_process_set_channel_regulators: the regulators s0 and t0 (GeV^2, > 0)
 * of the channels' s- and t-channel densities and of the partition
 * (default: (4 max(pt_min, 1 GeV))^2 for both). */
mf_status mf_process_set_channel_regulators(mf_process *p, double s0, double t0);

/* mf_channel_integrand: as mf_integrand (x: device SoA [ndim][n], f: device
 * [n]), with the momenta and weight of channel `channel`. */
mf_status mf_channel_integrand(mf_process *p, int32_t channel, const double *x, int64_t n, double *f,
                               mf_precision prec, void *stream);

/* mf_vegas_iterate_channels: one Vegas iteration of every channel of the
 * process, grids[k] (host [n_channels], distinct, n_channels =
 * mf_process_channels) serving channel k with n_events[k] >= 2 points.
 * Point i of channel k in iteration t draws its unit numbers as point i of
 * subprocess k in mf_vegas_iterate; accumulation, refinement and
 * combination are those of mf_vegas_iterate, per channel.  All channels'
 * points are evaluated in one kernel launch, so the grids must have the
 * same number of bins and the same iteration count (MF_EINVAL otherwise).
 * With refine != 0, a channel's grid is refined only if the channel had at
 * least 100 points per bin (n_events[k] >= 100 nbins): a grid refined on a
 * few points per bin follows the few points that landed and leaves the rest
 * of the channel unsampled.
 * out: host [n_channels].  The iteration's cross section is the sum of the
 * channels' integrals and its variance the sum of theirs.  Synchronous. */
mf_status mf_vegas_iterate_channels(mf_vegas *const *grids, mf_process *p, const int64_t *n_events,
                                    int32_t n_channels, uint64_t seed, mf_precision prec, int32_t refine,
                                    mf_iter_result *out, void *stream);

/* mf_channels_allocate (host only): Neyman's allocation of n_total points
 * over n_channels channels whose weights have per-point standard deviations
 * sigma[k] (host): n_out[k] = n_floor + floor(F * (s[k] / S)), F =
 * n_total - n_channels n_floor, S = s[0] + .. (summed in order); equal
 * shares n_floor + F / n_channels when S = 0.  s = sigma if n_prev is NULL;
 * otherwise each deviation, estimated from n_prev[k] points, is shrunk
 * towards the pooled one as if m0 more points had shown the pooled variance:
 * s[k] = sqrt((n_k sigma_k^2 + m0 P) / (n_k + m0)), P = sum n_k sigma_k^2 /
 * sum n_k (a channel whose few points missed its peak is not starved).
 * MF_EINVAL if F < 0, m0 < 0, or a sigma or count is negative or not
 * finite. */
mf_status mf_channels_allocate(int32_t n_channels, const double *sigma, const int64_t *n_prev, double m0,
                               int64_t n_total, int64_t n_floor, int64_t *n_out);

/* mf_channels_describe (host only): the channels a descriptor's program
 * gives, without creating a process.  *n_channels is set; if keys is not
 * NULL, row k of keys (host [n][key_stride]) holds the key's length and then
 * the key of channel k (lengths are at most 24; MF_EINVAL if key_stride is
 * smaller than a row needs).
 * mf_channels_table (host only): the int32 table the kernels read (the
 * layout of csrc/device/mf_channels.cuh); *len is set to its length, and
 * the table copied if table is not NULL (MF_EINVAL if *len was smaller). */
mf_status mf_channels_describe(const mf_process_desc *d, int32_t *n_channels, int32_t *keys, int32_t key_stride);
mf_status mf_channels_table(const mf_process_desc *d, int32_t *table, int32_t *len);

/* ---- Data-parallel iterations (Sec. 2.3: points are independent, so one
 * iteration splits across devices with one exchange of partial sums).
 *
 * The n_total points of an iteration form nchunks = ceil(n_total / MF_CHUNK)
 * chunks of MF_CHUNK consecutive points.  Their partial sums (K numbers per
 * chunk, K = mf_vegas_partial_size: sum w, sum w^2, non-zero count, nan count,
 * per dimension and bin sum w^2, then per dimension and bin counts) are added
 * along a fixed binary tree: node (l, i) covers chunks [i 2^l, (i+1) 2^l) and
 * exists when i 2^l < nchunks; its value is the sum of its two children, or
 * its left child when the right one does not exist; the root is (L, 0) with
 * 2^L >= nchunks.  A rank that evaluates chunks [c0, c1) returns the maximal
 * aligned nodes inside its range (mf_tree_frontier); any set of ranks whose
 * ranges partition [0, nchunks) then rebuilds exactly the root that
 * mf_vegas_iterate computes on one device, so every rank refines its own copy
 * of the grid to the same bits and no broadcast is needed.
 *
 * A tree node is exchanged as a record of 2 + K doubles: (level, index, K
 * values). */
mf_status mf_vegas_partial_size(const mf_vegas *v, int32_t *K);

/* mf_vegas_shard_accumulate: evaluate chunks [chunk_begin, chunk_end) of the
 * next iteration (points chunk_begin*MF_CHUNK ... min(chunk_end*MF_CHUNK,
 * n_total) - 1, with the Philox counters of their global indices and the
 * subprocess index `subprocess`) through the grid v, and write this range's
 * tree nodes into nodes (host, capacity MF_MAX_TREE_NODES records of 2 + K
 * doubles); *n_nodes receives their number.  An empty range returns no node.
 * Does not advance the iteration counter.  Synchronous on stream. */
mf_status mf_vegas_shard_accumulate(mf_vegas *v, mf_process *p, int64_t n_total, int64_t chunk_begin,
                                    int64_t chunk_end, int32_t subprocess, uint64_t seed, mf_precision prec,
                                    double *nodes, int32_t *n_nodes, void *stream);

/* mf_vegas_shard_finish: combine the nodes of all ranks (host, n_nodes
 * records, in any order) into the iteration totals, then finish the iteration
 * as mf_vegas_iterate does (histogram, estimate, combination, refinement
 * unless refine == 0) and advance the iteration counter.  MF_EINVAL if the
 * nodes do not partition the chunk range exactly (missing, overlapping or
 * duplicate nodes).  MF_ENAN as mf_vegas_iterate.  Synchronous on stream. */
mf_status mf_vegas_shard_finish(mf_vegas *v, int64_t n_total, const double *nodes, int32_t n_nodes,
                                int32_t refine, mf_iter_result *out, void *stream);

/* Host-only helpers of the tree (no device needed).  mf_tree_frontier writes
 * the (level, index) pairs of the maximal aligned nodes of chunks
 * [chunk_begin, chunk_end) of an nchunks-chunk tree into ids (host, capacity
 * pairs; *n receives the count; MF_EINVAL if capacity is too small); the range
 * ending at nchunks also owns the truncated right edge.  mf_tree_reduce
 * combines records (2 + K doubles each) that partition node (level, index)
 * into that node's K values (host out[K]). */
mf_status mf_tree_frontier(int64_t chunk_begin, int64_t chunk_end, int64_t nchunks, int64_t *ids,
                           int32_t capacity, int32_t *n);
mf_status mf_tree_reduce(const double *nodes, int32_t n_nodes, int32_t K, int64_t nchunks, int32_t level,
                         int64_t index, double *out);

/* mf_process_tune: time the kernel of precision prec for every launch shape
 * (128 or 256 threads per block; 8, 16 or 32 lanes per event, at most the
 * padded count of helicity pairs, or of helicities for a process without
 * pairs), then for the fastest a compiled-in minimum of 3 or 4 resident
 * blocks per SM, each on about n_sample (>= 1024) Vegas points of a uniform
 * grid rounded to a whole number of rounds of that shape's resident grid
 * (at least one round), and keep the fastest per point for later calls (and
 * for batches created afterwards).  The helicity sum is a fixed pairwise
 * tree whatever the lanes per point, so block size and lanes never change
 * the results; a minimum of resident blocks changes the compiler's register
 * budget and with it the order of a few multiply-adds, i.e. the last bits.  Each shape is compiled
 * once (cached on disk).  *block and *ht (may be NULL) receive the choice
 * (mf_process_kernel_info gives the rest).  Synchronous on stream. */
mf_status mf_process_tune(mf_process *p, mf_precision prec, int64_t n_sample, void *stream, int32_t *block,
                          int32_t *ht);

/* ---- Batched iterations (the subprocesses of a hadronic cross section
 * summed in Sec. 2.1 evaluated together): mf_batch_create compiles the
 * programs of nproc processes (1..8, each at most once, all on the current
 * device) into one persistent kernel; blocks draw tiles of 128 points from one
 * counter, the tiles of the costliest process first, so the subprocesses share
 * the GPU without a tail per subprocess.  mf_batch_iterate then runs one Vegas
 * iteration of every subprocess k with grid grids[k] and n_events[k] points:
 * same points (subprocess index k), same estimator and same refinement as
 * mf_vegas_iterate with the same arrays, in one kernel launch plus the
 * per-subprocess accumulation.  Synchronous; out[k] (host [nproc]).
 * mf_batch_get_info: the batch order (order[slot] = the caller's index,
 * host [nproc]), the kernel's registers per thread and the device time of
 * its last launch in ms; any pointer may be NULL.  The processes must outlive
 * the batch. */
mf_status mf_batch_create(mf_process *const *procs, int32_t nproc, mf_precision prec, mf_batch **out);
mf_status mf_batch_destroy(mf_batch *b);
mf_status mf_batch_iterate(mf_batch *b, mf_vegas *const *grids, const int64_t *n_events, uint64_t seed,
                           int32_t refine, mf_iter_result *out, void *stream);
mf_status mf_batch_get_info(const mf_batch *b, int32_t *order, int32_t *regs, double *last_kernel_ms);
/* mf_batch_iterate_graph: mf_batch_iterate as one CUDA graph replay.  The
 * first call (and any call whose grids, point counts, seed or refine flag
 * differ from the captured ones) captures the whole iteration — tile counter
 * reset, the persistent kernel, every subprocess's accumulation, tree
 * reduction, finalisation, refinement and the copies of the results — on an
 * internal stream and instantiates it; later calls copy the grids' iteration
 * indices to the device and replay the graph on `stream`.  Same points and
 * results as mf_batch_iterate.  Synchronous. */
mf_status mf_batch_iterate_graph(mf_batch *b, mf_vegas *const *grids, const int64_t *n_events, uint64_t seed,
                                 int32_t refine, mf_iter_result *out, void *stream);

/* ---- Unweighted events and the Les Houches Event writer (Sec. 2.5).
 *
 * mf_lhe_open writes the header and <init> block of an LHE 3.0 text file
 * and starts a writer thread; events handed to it are formatted and written
 * while the caller's GPU work goes on.  mf_lhe_close drains the queue, ends
 * the file, joins the thread and frees the writer (*n_written, may be NULL:
 * the number of events written).  Each event's colour and anticolour tags
 * (ICOLUP) are those of its colour flow (record field 3) in the table
 * colour_tags; an event whose flow is -1 or outside the table gets 0. */
typedef struct mf_lhe_writer mf_lhe_writer;
typedef struct {
    int32_t n_legs;                /* particles per event, incoming first */
    int32_t pdg[MF_MAX_LEGS];      /* PDG ids per leg */
    double mass[MF_MAX_LEGS];      /* masses written per leg (GeV) */
    int32_t beam_pdg[2];
    double beam_energy[2];         /* GeV */
    double xsec, xsec_error;       /* pb */
    double w_max;                  /* maximum event weight (pb) */
    int32_t process_id;
    double scale;                  /* event scale (GeV) */
    double alpha_qed, alpha_s;
    int32_t n_flows;               /* colour flows in colour_tags (0: no tags) */
    int32_t pad;
    const int32_t *colour_tags;    /* host [n_flows][n_legs][2]: per colour flow of the process (the
                                    * descriptor's colour-basis order) and leg, the LHE colour and
                                    * anticolour line numbers (0: none); copied at open */
} mf_lhe_init;
mf_status mf_lhe_open(const char *path, const mf_lhe_init *init, mf_lhe_writer **out);
/* Queue n events given as host records (4 + 4 n_legs doubles each: weight,
 * x1, x2, colour-flow index (-1: none), then per leg E, px, py, pz); the
 * data are copied. */
mf_status mf_lhe_write(mf_lhe_writer *w, const double *records, int64_t n);
mf_status mf_lhe_close(mf_lhe_writer *w, int64_t *n_written);

/* Observables of a final-state leg in the collider frame (the partonic
 * centre-of-mass momenta boosted along the beam axis by the rapidity of the
 * parton pair), for the weighted histograms of mf_vegas_observables (the
 * differential distributions of Sec. 3.1, Fig. 2):
 *   MF_OBS_PT              pT  = sqrt(px^2 + py^2)                (GeV)
 *   MF_OBS_RAPIDITY        y   = (1/2) ln((E + pz) / (E - pz))
 *   MF_OBS_PSEUDORAPIDITY  eta = asinh(pz / pT)
 * nbins (1 .. 64) equal bins on [lo, hi): v goes to bin
 * b = floor((v - lo) * (nbins / (hi - lo))) when 0 <= b < nbins, else nowhere. */
typedef enum { MF_OBS_PT = 0, MF_OBS_RAPIDITY = 1, MF_OBS_PSEUDORAPIDITY = 2 } mf_observable_kind;
#define MF_MAX_OBSERVABLES 4
typedef struct {
    int32_t kind;                  /* mf_observable_kind */
    int32_t leg;                   /* final-state leg: 2 .. n_legs - 1 */
    int32_t nbins;
    int32_t pad;
    double lo, hi;
} mf_observable;

/* mf_vegas_observables: one pass of n_events (>= 2) Vegas points through the
 * grid as it stands (the points mf_vegas_unweight uses: the grid's current
 * iteration index, subprocess index `subprocess`, Philox key seed; the grid is
 * neither refined nor advanced), and for each of n_obs (1 ..
 * MF_MAX_OBSERVABLES) observables the histogram of the points' weights
 * w_i = f J_V over its bins; points failing the threshold or the cuts are
 * not binned.  Per bin b, in observable order (host arrays of sum_k nbins_k):
 *   sigma[b] = (1/N) sum_{i in b} w_i                     (pb in the bin)
 *   error[b] = sqrt((sum_{i in b} w_i^2 / N - sigma[b]^2) / (N - 1))
 *   counts[b] = points in the bin (may be NULL).
 * The sums are taken in a fixed order (per 4096-point chunk, then a pairwise
 * tree over the chunks), so the results do not change from run to run.
 * MF_ENAN if some weights were not finite (those points are not binned).
 * Synchronous. */
mf_status mf_vegas_observables(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed, int32_t subprocess,
                               mf_precision prec, int32_t n_obs, const mf_observable *obs, double *sigma,
                               double *error, int64_t *counts, void *stream);

/* mf_vegas_observables_channel: mf_vegas_observables for phase-space
 * channel `channel` (see mf_vegas_iterate_channels): its own points
 * (subprocess index = channel) through its grid v, with the channel's
 * momenta and weight a_i / g_i.  The histograms of the whole cross section
 * are the sums over the channels (errors in quadrature). */
mf_status mf_vegas_observables_channel(mf_vegas *v, mf_process *p, int32_t channel, int64_t n_events, uint64_t seed,
                                       mf_precision prec, int32_t n_obs, const mf_observable *obs, double *sigma,
                                       double *error, int64_t *counts, void *stream);

/* mf_vegas_unweight: one pass of n_events Vegas points through the grid as it
 * stands (points of the grid's current iteration index, subprocess index
 * `subprocess`, Philox key seed; the grid is neither refined nor advanced),
 * then hit-or-miss unweighting: point i with weight w_i = f J_V is kept when
 * |w_i| > u_i w_max, u_i the first unit number of Philox counter
 * (i, iteration, subprocess, 15).  A kept point becomes an event of weight
 * sign(w_i) max(|w_i|, w_max) / n_events (pb), so the events' weights add up
 * to the integral estimate.  Each kept event also gets a colour flow k of
 * the process's colour basis, drawn with probability proportional to its
 * leading-colour weight sum_h C_kk |J_k,h|^2 (the helicity sum of the flow's
 * diagonal colour-matrix term, Sec. 2.5's colour assignment of events) by
 * the first unit number of Philox counter (i, iteration, subprocess, 13);
 * the LHE writer turns it into colour tags.  Records (host
 * [capacity][4 + 4 n_legs], may be NULL): event weight, x1, x2, colour-flow
 * index, then per leg (E, px, py, pz) in the collider frame, in point order;
 * at most capacity are written, *n_accepted receives the number kept.  With
 * lhe != NULL the events also go to that writer.  Synchronous. */
mf_status mf_vegas_unweight(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed, int32_t subprocess,
                            mf_precision prec, double w_max, mf_lhe_writer *lhe, double *records, int64_t capacity,
                            int64_t *n_accepted, void *stream);

/* mf_vegas_unweight_channel: mf_vegas_unweight for phase-space channel
 * `channel` (see mf_vegas_iterate_channels): the points are those of the
 * channel's own stream (subprocess index = channel) through its grid v, with
 * the channel's momenta and weight a_i / g_i.  To unweight the combined
 * sample of an iteration of N points (n_k in channel k) against one
 * maximum W of the combined weights W = w N / n_k, pass w_max = W n_k / N
 * for channel k: every event then weighs W / N.  MF_EUNSUPPORTED if the
 * process has no channels, MF_EINVAL for a channel out of range. */
mf_status mf_vegas_unweight_channel(mf_vegas *v, mf_process *p, int32_t channel, int64_t n_events, uint64_t seed,
                                    mf_precision prec, double w_max, mf_lhe_writer *lhe, double *records,
                                    int64_t capacity, int64_t *n_accepted, void *stream);

/* mf_process_channel_max_weights: after mf_vegas_iterate_channels with
 * n_events[k] points in channel k, the largest |w| of each channel's points
 * into host w_max[n_channels].  MF_EINVAL if the counts do not add up to
 * that pass's points.  Synchronous. */
mf_status mf_process_channel_max_weights(mf_process *p, const int64_t *n_events, int32_t n_channels, double *w_max,
                                         void *stream);
/* mf_process_read_weights: the weights w = f J_V of chosen points (host
 * idx[n], point indices of the pass) of the process's last Vegas pass, into
 * host w[n] (for checking single points of a large iteration).  Synchronous
 * on the legacy default stream. */
mf_status mf_process_read_weights(mf_process *p, const int64_t *idx, int64_t n, double *w);
/* mf_process_max_weight: max |w| over the points of the process's last
 * Vegas pass (mf_vegas_iterate, shard or unweighting pass).  Synchronous. */
mf_status mf_process_max_weight(mf_process *p, double *w_max, void *stream);

/* ---- mf_vegas_iterate_static: one Vegas iteration of one subprocess (as
 * mf_vegas_iterate with nproc = 1 and subprocess index 0: same points, same
 * results) that allocates no memory.  The paper has no counterpart: this
 * entry point exists for callers that must not have a library allocate
 * device memory while they run (applications whose device memory is all
 * handed out by their own pool, loops that cannot take the device-wide
 * synchronisation of cudaMalloc / cudaFree).
 *
 * Scratch: one array of 8,673,328 bytes compiled into the library
 * (file-scope device memory, one copy per device), enough for
 * n_events <= MF_STATIC_MAX_EVENTS points of up to MF_MAX_DIM dimensions and
 * 64 bins; larger n_events are rejected with MF_EINVAL.  Nothing in it needs
 * to start at zero: every call writes each element before reading it.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, which may load the library's device code) and keeps
 * it for later calls; make that first call before any stream capture.  The
 * kept address belongs to the device's primary context: after a
 * cudaDeviceReset it is stale, and this entry point must not be called again
 * in that process.  The process kernel of the requested precision (MF_FP64,
 * MF_MIXED or MF_MIXED_TC) must already be compiled, by an earlier
 * mf_integrand or mf_vegas_iterate call with that precision (compiling
 * allocates): otherwise MF_EINVAL.
 *
 * Calls that overlap in time on the same device share the one array and race:
 * serialise them (one stream, or synchronise between calls, across all
 * threads).  Synchronous: returns after *out (host) is filled.  MF_ENAN as
 * mf_vegas_iterate; MF_ETIMEOUT or MF_ECUDA when the process kernel flagged
 * an error (see mf_process_check): the iteration is then not counted. */
mf_status mf_vegas_iterate_static(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed,
                                  mf_precision prec, int32_t refine, mf_iter_result *out, void *stream);

/* ---- Checkpoint of a grid (the Vegas state of Sec. 2.2 that VegasFlow
 * carries from one iteration to the next: the adapted bin edges, and the
 * per-iteration estimates that the final result combines): edges, last
 * histogram and counts, and the (I_k, sigma_k) of the iterations so far, so
 * that a run resumes with the same combination.  mf_vegas_save with buf == NULL stores the size needed in *len;
 * otherwise *len is the capacity on entry and the size written on return
 * (MF_EINVAL if too small).  mf_vegas_load checks the record (tag, shape,
 * size, edges) and restores it into a grid of the same ndim and nbins. */
mf_status mf_vegas_save(const mf_vegas *v, void *buf, size_t *len);
mf_status mf_vegas_load(mf_vegas *v, const void *buf, size_t len);

/* Helicity sampling (the Monte Carlo over helicities that Sec. 4 names as a
 * way to cut the cost per point): with on = 1 the integrand kernels of this
 * process evaluate one helicity per point, drawn uniformly from the
 * non-vanishing helicities with the first unit number of Philox counter
 * (i, iteration, subprocess, 14) (Vegas passes: their key; given points:
 * counter (i, 0, 0, 14) with key (seed, 0)), and multiply its |M|^2 by their
 * number: an unbiased estimate of the helicity sum with a larger variance.
 * With on = 2 the same draw picks one helicity pair (mf_process_get_helicity_
 * pairs) and the sum of its members' |M|^2 is multiplied by the number of
 * pairs.  A process without pairs (none differ at one leg, pairs cost more
 * FLOPs than single helicities, or the option helicity_pairs = 0) samples
 * single helicities instead, and so does the MF_MIXED_TC kernel, which
 * evaluates single helicities; mf_process_info.helicity_sampling reports the
 * mode in effect.  on = 0: the
 * full sum.  MF_EINVAL for other values.  mf_helicity_msq and mf_grad always
 * sum over helicities. */
mf_status mf_process_set_helicity_sampling(mf_process *p, int32_t on, uint64_t seed);

/* Colour sampling (the Monte Carlo over colour configurations of Sec. 4,
 * beside the one over helicities): with on = 1 the integrand kernels of this
 * process (mf_integrand, the Vegas passes) replace each helicity's colour sum
 * by NJAMP Re(conj(J_k) sum_l C_kl J_l) / den for one colour flow k per
 * point, drawn uniformly from the first unit number of Philox counter
 * (i, iteration, subprocess, 12) (given points: (i, 0, 0, 12) with the key
 * of mf_process_set_helicity_sampling): an unbiased estimate of the colour
 * sum, with a larger variance (the amplitudes are computed in full; only the
 * colour sum is sampled).  Combines with helicity sampling and with the
 * leading-colour approximation (then NJAMP C_kk |J_k|^2 / den).  on = 0:
 * the full colour sum.  Runs in a kernel of its own in the process module;
 * mf_helicity_msq, mf_grad and batches always sum the colours. */
mf_status mf_process_set_colour_sampling(mf_process *p, int32_t on);

/* The helicity pairs of a process: pairs[2 k], pairs[2 k + 1] (host, may be
 * NULL, else room for 2 * n_hel entries) are the rows of
 * mf_process_get_helicities whose pair leg (mf_process_info.pair_leg) is -1
 * and +1, or -1 where that assignment vanishes; *n_pairs receives the count
 * (0: helicities one at a time). */
mf_status mf_process_get_helicity_pairs(const mf_process *p, int32_t *pairs, int32_t *n_pairs);
/* Leading-colour approximation (the other cut of the cost per point that
 * Sec. 4 names): with on != 0 the integrand kernels keep only the diagonal
 * of the colour matrix in the colour-flow basis, sum_k C_kk |J_k|^2 / den,
 * i.e. the leading term in 1/N_c.  The kernels are regenerated on their next
 * use (synchronises the device); mf_helicity_msq follows the setting,
 * mf_grad and batches created earlier do not. */
mf_status mf_process_set_leading_colour(mf_process *p, int32_t on);
/* The non-vanishing helicity assignments kept at creation, in the order the
 * sampling indexes them (host [n_hel][n_legs], +1/-1; may be NULL to query
 * *n_hel). */
mf_status mf_process_get_helicities(const mf_process *p, int8_t *hel, int32_t *n_hel);

/* The launch shape of the compiled kernel of precision prec: threads per
 * block, lanes per point, registers per thread, resident blocks per SM and
 * the minimum of resident blocks it was compiled for (0: none) (any pointer
 * may be NULL); MF_EINVAL if that kernel is not compiled yet. */
mf_status mf_process_kernel_info(const mf_process *p, mf_precision prec, int32_t *block, int32_t *ht,
                                 int32_t *regs, int32_t *blocks_per_sm, int32_t *min_blocks);

/* mf_process_check: whether a kernel of this process flagged an error: a
 * bounded wait expired (the tensor-core colour sum waits on the completion
 * of its MMAs; that launch's results are unspecified): MF_ETIMEOUT; the
 * launch gave less dynamic shared memory than the kernel needs (nothing
 * written): MF_ECUDA; mf_integrand wrote a non-finite value: MF_ENAN.  Reads and clears the flag (synchronises the device).
 * The synchronous entry points (mf_create_process, mf_vegas_iterate, the
 * shard and batch iterations) check it by themselves. */
mf_status mf_process_check(mf_process *p);

/* Device time, in ms, of the last fused integrand kernel that mf_vegas_iterate
 * launched for this process (CUDA events recorded on the launching stream
 * around that one launch; the accumulation and refinement kernels excluded).
 * Valid after mf_vegas_iterate returned; 0 before the first call. */
mf_status mf_process_last_kernel_ms(const mf_process *p, double *ms);

/* Copy the grid edges (host [ndim][nbins+1]) out of / into the object. */
mf_status mf_vegas_get_grid(const mf_vegas *v, double *edges);
mf_status mf_vegas_set_grid(mf_vegas *v, const double *edges);
/* The last iteration's accumulators: per dimension and bin sum of w^2 (host
 * [ndim][nbins]) and counts (host [ndim][nbins]); either pointer may be NULL. */
mf_status mf_vegas_get_histogram(const mf_vegas *v, double *sum_w2, int64_t *counts);
/* Dimensions, bins and the next iteration's index. */
mf_status mf_vegas_get_shape(const mf_vegas *v, int32_t *ndim, int32_t *nbins, int32_t *iteration);

/* Diagnostic: write the CUDA source that mf_create_process would generate for
 * *desc at precision prec into buf (host, capacity *len bytes; *len receives
 * the size including the terminating NUL).  With compile != 0 the source is
 * also compiled for sm_103a with NVRTC (no GPU needed) and MF_EJIT returned on
 * failure.  buf may be NULL to query the size. */
mf_status mf_generate_kernel_source(const mf_process_desc *desc, mf_precision prec, int32_t compile,
                                    char *buf, size_t *len);

/* Diagnostic: the source of the batched kernel of nproc descriptors (in the
 * given order), as mf_generate_kernel_source. */
mf_status mf_generate_batch_source(const mf_process_desc *const *descs, int32_t nproc, mf_precision prec,
                                   int32_t compile, char *buf, size_t *len);

/* mf_colour_sum: the colour sum of Sec. 2.4 for n rows of colour flows,
 * out[r] = sum_kl Re(conj(J_rk) C_kl J_rl) / den with C = cnum / den (host
 * [nj][nj] integer numerators, symmetric), J (device, FP32, [2 nj][n]: Re J_k
 * in row 2k, Im J_k in row 2k + 1), out (device FP32 [n]).  use_tc != 0: on
 * the tensor cores (tcgen05.mma kind::tf32 with J split into a TF32 high and
 * low part, FP32 accumulation; the fused kernels' MF_MIXED_TC colour sum);
 * use_tc == 0: FP32 FMAs in the symmetric form of the generated kernels.
 * nj in {2, 4, 6, 24} (MF_EUNSUPPORTED otherwise).  MF_ETIMEOUT if a bounded
 * wait on the MMAs' completion expired (results unspecified).  Synchronous
 * on stream. */
mf_status mf_colour_sum(const float *J, int64_t n, const int32_t *cnum, int32_t nj, int32_t den,
                        int32_t use_tc, float *out, void *stream);

/* mf_measure_peak: the device's arithmetic peak measured by the library's
 * own microbenchmark kernels, the denominators of the fused kernels' roofline
 * fractions (the paper has no counterpart).  kind 0: FP32 FFMA (8 independent
 * a = a b + c chains per thread, 4 blocks of 256 threads per SM); kind 1:
 * FP64 DFMA (the same in double precision); kind 3: FP32 FMA on packed
 * pairs (fma.rn.f32x2, two FMAs per instruction, otherwise as kind 0);
 * kind 2: TF32 tensor-core MMA
 * (one 128-thread block per SM issuing tcgen05.mma kind::tf32 M = 128,
 * N = 256, K = 8 back to back from shared memory in the no-swizzle K-major
 * layout of the colour-sum kernel into tensor memory).  One untimed launch,
 * then reps (>= 1) launches each timed with CUDA events on stream; *tflops
 * (host) receives the best rate in TFLOP/s (2 FLOPs per FMA lane, 2 M N K
 * per MMA) and *ms (host, may be NULL) that launch's duration.  Allocates a
 * few bytes of scratch.  MF_ETIMEOUT if the MMA completion wait (bounded by
 * 2 s per block) expired.  Synchronous. */
mf_status mf_measure_peak(int32_t kind, int32_t reps, double *tflops, double *ms, void *stream);

/* mf_debug_fail_allocation: a test hook for the library's allocation-failure
 * paths (the paper has no counterpart).  With after >= 0, the library's next
 * after device or pinned-host allocations succeed and the one after them
 * fails as if the device were out of memory (the entry point that made it
 * returns MF_ENOMEM and releases what it had allocated); later allocations
 * succeed again.  after = -1 disarms the hook.  Process-wide, thread-safe;
 * no device work. */
mf_status mf_debug_fail_allocation(int64_t after);

/* Thread-local description of the last error (empty string if none). */
const char *mf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MADFLOW_GB_H */
