// Internal declarations of libmadflow_gb (host side).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/madflow_gb.h"
#include "device/mf_kparams.h"

namespace mfi {

// thread-local error text
void set_error(const std::string &msg);
mf_status fail(mf_status st, const std::string &msg);

// Every device (and pinned host) allocation of the library goes through
// these, so that a test can make one of them fail (mf_debug_fail_allocation).
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t host_malloc_raw(void **p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
cudaError_t host_malloc(T **p, size_t bytes) {
    return host_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

struct DenSlot {
    uint32_t mask;   // legs whose signed momenta sum to the current's momentum
    int32_t mass_id; // -1 = massless propagator
};

struct Compiled {
    CUmodule module = nullptr;
    CUfunction fn = nullptr;
    CUfunction fn_flow = nullptr;  // the module's leading-colour flow kernel (mode 5), if any
    CUfunction fn_csamp = nullptr; // the module's colour-sampled integrand kernel, if any
    int block = 128;
    int ht = 32;
    size_t smem = 0;
    int max_blocks_per_sm = 1;
    int regs = 0;
    size_t local_bytes = 0;
    int min_blocks = -1;           // __launch_bounds__ minimum (-1: the default)
    int ptxas_level = -1;          // device-assembler level it was built at (-1: the default, 3)
};

struct GenInfo {
    int n_den = 0;
    std::vector<DenSlot> dens;
    std::vector<int> op_den;     // per op: denominator slot (CUR) or -1
    double flops_per_hel = 0.0;
    double flops_kin = 0.0;
    int parts = 1;               // functions the helicity program is split into
    int pair_leg = -1;           // leg of the helicity-pair program (-1: none)
    double flops_pair = 0.0;     // FLOPs of the pair program (both members)
    int peak_live = 0;           // peak of live internal wavefunctions of the schedule
};

double shared_flops(const mf_process &p, int leg);
int pair_leg(const mf_process &p);
bool large_program(const mf_process &p);


// Channels of the multichannel phase space (mf_channels.cpp): the device
// table of device/mf_channels.cuh and each channel's canonical key.
struct ChannelSet {
    int K = 0;
    std::vector<int32_t> table;
    std::vector<std::vector<int>> keys;
};
mf_status derive_channels(int n_legs, const std::vector<mf_op> &ops, ChannelSet &out);
}  // namespace mfi

struct mf_process {
    int device = 0;
    // code-generation and launch options (MF_OPT_AUTO: the library decides)
    mf_process_options opt = {MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO,
                              MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO, MF_OPT_AUTO};
    // deep copy of the descriptor
    int n_legs = 0, n_out = 0, ndim = 0;
    std::vector<int32_t> leg_kind, leg_incoming, leg_mass_id, leg_cut;
    std::vector<double> masses;
    std::vector<mf_op> ops;
    std::vector<mf_colour_term> terms;
    std::vector<double> couplings;
    int n_jamp = 0;
    std::vector<int32_t> colour_num;
    int colour_den = 1;
    std::vector<int8_t> hel_all;   // [n_hel_all][n_legs]
    std::vector<int8_t> hel;       // kept after filtering
    std::vector<uint8_t> pairs;    // [n_pairs][2] rows of hel (0xFF: absent); empty: no pairs
    double average = 1.0;
    int alpha_s_power = 0;
    double alpha_s = 0.0;
    double sqrt_s = 0.0;
    int hadronic = 0;
    double mu_f2 = 0.0, pt_min = 0.0, dr_min = 0.0;
    int pdf_nx = 0;
    double pdf_a0 = 0.0, pdf_h = 0.0;
    double *d_pdf_rows = nullptr;  // device [2][2][nx]
    double ln_tau_min = 0.0, w0_const = 0.0, pref_const = 0.0;
    mfi::GenInfo gen;
    mfi::Compiled kern[4];         // per mf_precision, and [2] the gradient kernel
    std::string source[4];
    int *d_err = nullptr;          // device error flag of the process kernels
    // events around the last process-kernel launch of mf_vegas_iterate
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    double last_kernel_ms = 0.0;
    // device scratch of mf_vegas_iterate (grown on demand)
    double *d_w = nullptr;
    uint8_t *d_bins = nullptr;
    int64_t scratch_n = 0;
    int64_t last_n = 0;            // points of the last Vegas pass held in d_w
    int hel_sample = 0;            // one sampled helicity per point
    int leading_colour = 0;        // generate the leading-colour approximation
    int colour_sample = 0;         // one colour flow per point (the colour-sampled kernel)
    uint64_t hel_seed = 0;         // Philox key of the sampling of given points
    // multichannel phase space: the channels derived from the program, their
    // device table and the propagator regulators (GeV^2)
    mfi::ChannelSet channels;
    int32_t *d_chan = nullptr;
    double ch_s0 = 1.0, ch_t0 = 1.0;
    long long *d_ch_off = nullptr;      // [K+1] point offsets of a launch over every channel
    double **d_ch_grids = nullptr;      // [K] the channels' grids
    long long *d_ch_chunk_off = nullptr;  // [K+1] chunk offsets of the channels' accumulation
    double *d_ch_res = nullptr;         // [K][8] the channels' iteration results
    void *d_ch_acc = nullptr;           // [K] per-channel bookkeeping records (mf_api.cu)
};

struct mf_vegas {
    int device = 0;
    int ndim = 0, nbins = 0;
    double alpha = 1.5;
    int iteration = 0;
    double *d_grid = nullptr;      // [ndim][nbins+1]
    double *d_hist = nullptr;      // [ndim][nbins] sum w^2 of the last iteration
    long long *d_count = nullptr;  // [ndim][nbins]
    double *d_hist_iter = nullptr; // [max_iter][2]: (I_k, sigma_k)
    int max_iter = 0;
    double *d_result = nullptr;    // small result block
    double *d_slots = nullptr;     // chunk partial sums [K][chunks] + K
    int64_t slots_cap = 0;
    int64_t *d_tree_ids = nullptr; // [MF_MAX_TREE_NODES][2] (level, index)
    double *d_tree_out = nullptr;  // [MF_MAX_TREE_NODES][K] node values
    double *d_tot = nullptr;       // [K] combined totals of a sharded iteration
};

// Several processes compiled into one persistent kernel (mf_batch_create).
struct mf_batch {
    int device = 0;
    int precision = 0;
    std::vector<mf_process *> procs;   // caller's order
    std::vector<int> order;            // batch slot -> caller's index, costliest first
    std::vector<double> cost;          // FLOPs per point, caller's order
    mfi::Compiled kern;
    std::string source;
    long long *d_counter = nullptr;    // tile counter of the persistent kernel
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    double last_kernel_ms = 0.0;
    // CUDA graph of one iteration (mf_batch_iterate_graph), valid for the
    // grids, point counts, seed and refine flag it was captured with
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::vector<mf_vegas *> graph_grids;
    std::vector<int64_t> graph_n;
    std::vector<const void *> graph_ptrs;  // scratch and grid buffers the graph writes
    uint64_t graph_seed = 0;
    int graph_refine = -1;
    long long *d_iters = nullptr;      // [nproc] iteration index per grid, read by the graph
    int64_t *d_root_ids = nullptr;     // [nproc][2] root node of each grid's chunk tree
    long long *h_iters = nullptr;      // pinned [nproc]
    double *h_res = nullptr;           // pinned [nproc][8]
    int *h_flags = nullptr;            // pinned [nproc]
};

struct mf_lhe_writer;

namespace mfi {
// the event writer (mf_lhe.cpp)
mf_status lhe_push(mf_lhe_writer *w, std::vector<double> &&records);
int lhe_legs(const mf_lhe_writer *w);
// code generation (mf_codegen.cpp)
std::string generate_source(const mf_process &p, int precision, int block, int ht, GenInfo &info,
                            const char *ns = "proc", bool kernel = true, int min_blocks = -1);
std::string generate_batch_source(const std::vector<const mf_process *> &ps, int precision, int block,
                                  const std::vector<int> &hts, std::vector<GenInfo> &infos);
std::string generate_grad_source(const mf_process &p, int block, GenInfo &info);
// run-time compilation (mf_jit.cpp)
mf_status jit_compile(const std::string &source, const std::string &name, std::vector<char> &cubin,
                      int ptxas_level = -1);
mf_status load_kernel(const std::vector<char> &cubin, Compiled &out, const char *name = "mf_kernel");
void unload_kernel(Compiled &k);
mf_status launch_kernel(const Compiled &k, unsigned grid, void **args, cudaStream_t s, int variant = 0);
}  // namespace mfi
