// C entry points of libmadflow_gb and the statically compiled kernels of the
// Vegas iteration (accumulation, fixed pairwise-tree reduction over chunks,
// refinement and the combination of iterations; Sec. 2.2 and Lepage 1978).
#include <algorithm>
#include <atomic>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mf_internal.h"
#include "device/mf_kinematics.cuh"

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
namespace mfi {
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
mf_status fail(mf_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

// allocations left before the injected failure (-1: none armed)
static std::atomic<long long> g_alloc_countdown{-1};

static bool injected_failure() {
    long long c = g_alloc_countdown.load();
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
    }
    return false;
}

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_malloc_raw(void **p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}
}  // namespace mfi

extern "C" mf_status mf_debug_fail_allocation(int64_t after) {
    if (after < -1) return mfi::fail(MF_EINVAL, "after must be -1 or non-negative");
    mfi::g_alloc_countdown.store(after);
    return MF_OK;
}

using mfi::fail;

extern "C" const char *mf_last_error(void) { return mfi::g_err.c_str(); }

extern "C" mf_status mf_process_options_init(mf_process_options *opt) {
    if (!opt) return fail(MF_EINVAL, "NULL options");
    int32_t *f = &opt->amplitude_units;
    for (size_t i = 0; i < sizeof(mf_process_options) / sizeof(int32_t); ++i) f[i] = MF_OPT_AUTO;
    return MF_OK;
}

#define MF_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

namespace {

constexpr int kChunk = 4096;           // events per accumulation chunk (fixed: results
                                       // do not depend on launch shapes)
constexpr int kAccThreads = 256;
constexpr int kTreeLog = 8;            // vegas_tree_kernel: 2^kTreeLog threads
constexpr int kTreeThreads = 1 << kTreeLog;
constexpr int kTreeMaxLevel = 40;      // at most 2^40 chunks per iteration
constexpr int kChannelRefinePerBin = 100;  // points per bin a channel's grid needs to be refined
constexpr double kGeV2pb = 0.3893793721e9;
constexpr double kPi = 3.14159265358979323846;

// ----------------------------------------------------------------------------
// PDF table collapse at fixed mu_F^2: cubic Hermite weights in ln Q^2 folded
// into one row of x f values over the ln x knots, plus that row's knot slopes
// (central differences, one-sided at the ends).
// ----------------------------------------------------------------------------
__global__ void pdf_collapse_kernel(const double *table, int nx, int nq, double b0, double hb,
                                    double b, double *row, double *slope) {
    // interval j of ln Q^2 and local coordinate t
    double s = (b - b0) / hb;
    int j = (int)floor(s);
    if (j < 0) j = 0;
    if (j > nq - 2) j = nq - 2;
    double t = s - j;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
    // slopes at knots j and j+1 (per unit ln Q^2) are linear in the rows:
    // D_k = (g_hi - g_lo) / (b_hi - b_lo), lo = max(k-1, 0), hi = min(k+1, nq-1)
    auto lo = [&](int k) { return k - 1 >= 0 ? k - 1 : k; };
    auto hi = [&](int k) { return k + 1 <= nq - 1 ? k + 1 : k; };
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        auto g = [&](int k) { return table[(size_t)k * nx + i]; };
        double d0 = (g(hi(j)) - g(lo(j))) / ((hi(j) - lo(j)) * hb);
        double d1 = (g(hi(j + 1)) - g(lo(j + 1))) / ((hi(j + 1) - lo(j + 1)) * hb);
        row[i] = h00 * g(j) + h10 * hb * d0 + h01 * g(j + 1) + h11 * hb * d1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        int l = i - 1 >= 0 ? i - 1 : i, r = i + 1 <= nx - 1 ? i + 1 : i;
        slope[i] = (row[r] - row[l]) / (r - l);   // per knot; divided by h on use below
    }
}

__global__ void scale_kernel(double *v, int n, double s) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] *= s;
}

// ----------------------------------------------------------------------------
// Vegas accumulation: one block per chunk of kChunk events.  Components per
// chunk: [sum w, sum w^2, nonzero, nan, hist[ndim][nb], counts[ndim][nb]],
// stored component-major: slots[k * ld + chunk].  Non-finite weights count as
// nan and contribute 0.
// ----------------------------------------------------------------------------
__device__ double block_tree_sum(double *buf, int m) {
    // fixed pairwise tree over kChunk slots (zero padded): pairs (i, i + s)
    for (int i = m + threadIdx.x; i < kChunk; i += blockDim.x) buf[i] = 0.0;
    __syncthreads();
    for (int s = kChunk / 2; s > 0; s >>= 1) {
        for (int i = threadIdx.x; i < s; i += blockDim.x) buf[i] = buf[i] + buf[i + s];
        __syncthreads();
    }
    double r = buf[0];
    __syncthreads();
    return r;
}

__device__ void accumulate_chunk(const double *w, const uint8_t *bins, int64_t n, int ndim, int nb, double *slots,
                                 int64_t ld, int64_t chunk) {
    extern __shared__ double sh[];
    double *sw = sh;                    // [kChunk] sanitised w
    double *buf = sh + kChunk;          // [kChunk] tree buffer
    __shared__ double whist[kAccThreads / 32][64];
    __shared__ int wcnt[kAccThreads / 32][64];
    __shared__ double stage[kAccThreads / 32][32];
    __shared__ int s_nz, s_nan;
    const int64_t base = chunk * kChunk;
    const int m = (int)((n - base) < kChunk ? (n - base) : kChunk);
    double *slot = slots + chunk;           // component k at slot[k * ld]
    if (threadIdx.x == 0) { s_nz = 0; s_nan = 0; }
    __syncthreads();
    int nz = 0, nn = 0;
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
        double v = 0.0;
        if (i < m) {
            v = w[base + i];
            if (!isfinite(v)) { v = 0.0; ++nn; }
            if (v != 0.0) ++nz;
        }
        sw[i] = v;
        buf[i] = v;
    }
    atomicAdd(&s_nz, nz);
    atomicAdd(&s_nan, nn);
    __syncthreads();
    double s1 = block_tree_sum(buf, m);
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) buf[i] = sw[i] * sw[i];
    __syncthreads();
    double s2 = block_tree_sum(buf, m);
    if (threadIdx.x == 0) {
        slot[0] = s1; slot[ld] = s2; slot[2 * ld] = (double)s_nz; slot[3 * ld] = (double)s_nan;
    }
    // per dimension and bin: warp k sums its kChunk/8 consecutive events in
    // event order (32 at a time; lanes of one bin are added by the lowest of
    // them in lane order), then the 8 warps' sums are added in a fixed tree
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kAccThreads / 32, kPerWarp = kChunk / kWarps;
    for (int j = 0; j < ndim; ++j) {
        for (int q = lane; q < 64; q += 32) {
            whist[warp][q] = 0.0;
            wcnt[warp][q] = 0;
        }
        __syncwarp();
        for (int step = 0; step < kPerWarp / 32; ++step) {
            const int i = warp * kPerWarp + step * 32 + lane;
            const bool valid = i < m;
            const int b = valid ? (int)bins[(int64_t)j * n + base + i] : 255;
            stage[warp][lane] = valid ? sw[i] * sw[i] : 0.0;
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            __syncwarp();
            if (b < 64 && lane == __ffs(peers) - 1) {
                double acc = whist[warp][b];
                int cnt = wcnt[warp][b];
                for (unsigned mk = peers; mk; mk &= mk - 1) {
                    acc += stage[warp][__ffs(mk) - 1];
                    ++cnt;
                }
                whist[warp][b] = acc;
                wcnt[warp][b] = cnt;
            }
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x < nb) {
            const int q = threadIdx.x;
            static_assert(kWarps == 8, "fixed 8-warp tree");
            const double h = ((whist[0][q] + whist[1][q]) + (whist[2][q] + whist[3][q])) +
                             ((whist[4][q] + whist[5][q]) + (whist[6][q] + whist[7][q]));
            int c = 0;
            for (int w = 0; w < kWarps; ++w) c += wcnt[w][q];
            slot[(size_t)(4 + j * nb + q) * ld] = h;
            slot[(size_t)(4 + ndim * nb + j * nb + q) * ld] = (double)c;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kAccThreads) vegas_accumulate_kernel(const double *w, const uint8_t *bins,
                                                                       int64_t n, int ndim, int nb, double *slots,
                                                                       int64_t ld) {
    accumulate_chunk(w, bins, n, ndim, nb, slots, ld, blockIdx.x);
}

// Per-channel state of a multichannel iteration's bookkeeping (one record
// per channel, device memory): its segment of the launch's weights and bin
// indices, its chunk count and tree level, and its grid's buffers.
struct ChanAcc {
    const double *w;
    const uint8_t *bins;
    long long n, nchunks;
    int level, iteration;
    int refine, pad;            // refine this channel's grid
    double alpha;
    double *slots, *tree_out, *hist, *hist_iter, *result, *grid;
    long long *count;
    double *result_copy;        // the 7 results again, in one array for all channels
};

__device__ int chunk_channel(const long long *chunk_off, int nch, long long b) {
    int lo = 0, hi = nch;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (chunk_off[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Every channel's chunks in one launch: block b is chunk b - chunk_off[k] of
// channel k (chunk_off[k] <= b < chunk_off[k+1]).
__global__ void __launch_bounds__(kAccThreads) vegas_accumulate_channels_kernel(const ChanAcc *ca,
                                                                                const long long *chunk_off, int nch,
                                                                                int ndim, int nb) {
    const int k = chunk_channel(chunk_off, nch, blockIdx.x);
    const ChanAcc &c = ca[k];
    accumulate_chunk(c.w, c.bins, c.n, ndim, nb, c.slots, c.nchunks, (int64_t)blockIdx.x - chunk_off[k]);
}

// Reduction over chunks along a fixed pairwise tree (mf_tree_reduce states the
// tree).  Block (k, j) computes component k of node j = (level, index) from the
// chunk partials slots[k * ld + c - c0] of the chunks the node covers: each
// thread folds an aligned segment of 2^s chunks with a binary-counter stack
// (which performs exactly the tree's additions, the last incomplete subtree
// folded from its right end), then the segments are paired in shared memory.
__device__ double tree_node(const double *slots, int64_t ld, int64_t c0, int64_t nchunks, int k, int level,
                            int64_t index) {
    __shared__ double red[kTreeThreads];
    const int64_t first = index << level;
    const int s = level > kTreeLog ? level - kTreeLog : 0;
    const int64_t nseg = ((int64_t)1 << level) >> s;                // <= kTreeThreads
    const int64_t seg_first = first + ((int64_t)threadIdx.x << s);
    // segments whose first chunk exists
    const int64_t exist = (nchunks - first + ((int64_t)1 << s) - 1) >> s;
    int64_t m = exist < nseg ? exist : nseg;
    double v = 0.0;
    if ((int64_t)threadIdx.x < m) {
        double st[kTreeMaxLevel + 2];
        int lv[kTreeMaxLevel + 2];
        int top = 0;
        int64_t end = seg_first + ((int64_t)1 << s);
        if (end > nchunks) end = nchunks;
        for (int64_t c = seg_first; c < end; ++c) {
            double x = slots[(size_t)k * ld + (size_t)(c - c0)];
            int xl = 0;
            while (top > 0 && lv[top - 1] == xl) {
                x = st[top - 1] + x;
                --top;
                ++xl;
            }
            st[top] = x;
            lv[top] = xl;
            ++top;
        }
        v = st[top - 1];
        for (int q = top - 2; q >= 0; --q) v = st[q] + v;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int64_t w = nseg; w > 1; w >>= 1) {
        const int64_t i = threadIdx.x;
        double nv = 0.0;
        if (i < (w >> 1) && 2 * i < m) nv = (2 * i + 1 < m) ? red[2 * i] + red[2 * i + 1] : red[2 * i];
        __syncthreads();
        if (i < (w >> 1)) red[i] = nv;
        m = (m + 1) >> 1;
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kTreeThreads) vegas_tree_kernel(const double *slots, int64_t ld, int64_t c0,
                                                                  int64_t nchunks, int K, const int64_t *node_ids,
                                                                  double *out) {
    const int k = blockIdx.x;
    const double r = tree_node(slots, ld, c0, nchunks, k, (int)node_ids[2 * blockIdx.y], node_ids[2 * blockIdx.y + 1]);
    if (threadIdx.x == 0) out[(size_t)blockIdx.y * K + k] = r;
}

// Block (k, c): component k of channel c's root node.
__global__ void __launch_bounds__(kTreeThreads) vegas_tree_channels_kernel(const ChanAcc *ca, int K) {
    const ChanAcc &c = ca[blockIdx.y];
    const double r = tree_node(c.slots, c.nchunks, 0, c.nchunks, blockIdx.x, c.level, 0);
    if (threadIdx.x == 0) c.tree_out[blockIdx.x] = r;
}

// Iteration estimate, the histogram, and the inverse-variance combination of
// all iterations so far (iterations with zero variance are exact: if any, the
// result is their mean with zero error).  res: [I, err, sigma, sigma_err,
// chi2/dof, nonzero, nan].
__device__ void finalize_body(const double *tot, int64_t n, int ndim, int nb, int it, double *hist,
                              long long *count, double *iters, double *res) {
    for (int i = threadIdx.x; i < ndim * nb; i += blockDim.x) {
        hist[i] = tot[4 + i];
        count[i] = (long long)tot[4 + ndim * nb + i];
    }
    if (threadIdx.x != 0) return;
    double N = (double)n;
    double I = tot[0] / N;
    double var = (tot[1] / N - I * I) / (N - 1.0);
    double err = sqrt(var > 0.0 ? var : 0.0);
    iters[2 * it] = I;
    iters[2 * it + 1] = err;
    int nexact = 0;
    double exact_sum = 0.0;
    for (int k = 0; k <= it; ++k)
        if (iters[2 * k + 1] == 0.0) { ++nexact; exact_sum += iters[2 * k]; }
    double mean, merr, chi2 = 0.0;
    if (nexact > 0) {
        mean = exact_sum / nexact;
        merr = 0.0;
    } else {
        double sw = 0.0, swi = 0.0;
        for (int k = 0; k <= it; ++k) {
            double wk = 1.0 / (iters[2 * k + 1] * iters[2 * k + 1]);
            sw += wk;
            swi += wk * iters[2 * k];
        }
        mean = swi / sw;
        merr = 1.0 / sqrt(sw);
        if (it > 0) {
            for (int k = 0; k <= it; ++k) {
                double d = iters[2 * k] - mean;
                chi2 += d * d / (iters[2 * k + 1] * iters[2 * k + 1]);
            }
            chi2 /= it;
        }
    }
    res[0] = I; res[1] = err; res[2] = mean; res[3] = merr; res[4] = chi2;
    res[5] = tot[2]; res[6] = tot[3];
}

__global__ void vegas_finalize_kernel(const double *tot, int64_t n, int ndim, int nb, int it, double *hist,
                                      long long *count, double *iters, double *res) {
    finalize_body(tot, n, ndim, nb, it, hist, count, iters, res);
}

// Block c: channel c's finalisation.
__global__ void vegas_finalize_channels_kernel(const ChanAcc *ca, int ndim, int nb) {
    const ChanAcc &c = ca[blockIdx.x];
    finalize_body(c.tree_out, c.n, ndim, nb, c.iteration, c.hist, c.count, c.hist_iter, c.result);
    if (threadIdx.x == 0)
        for (int q = 0; q < 7; ++q) c.result_copy[q] = c.result[q];
}

// The same with the iteration index read from device memory (graph replays).
__global__ void vegas_finalize_dev_kernel(const double *tot, int64_t n, int ndim, int nb, const long long *it,
                                          double *hist, long long *count, double *iters, double *res) {
    __shared__ int s_it;
    if (threadIdx.x == 0) s_it = (int)*it;
    __syncthreads();
    const int k = s_it;
    for (int i = threadIdx.x; i < ndim * nb; i += blockDim.x) {
        hist[i] = tot[4 + i];
        count[i] = (long long)tot[4 + ndim * nb + i];
    }
    if (threadIdx.x != 0) return;
    // the rest as vegas_finalize_kernel, for iteration k
    double N = (double)n;
    double I = tot[0] / N;
    double var = (tot[1] / N - I * I) / (N - 1.0);
    double err = sqrt(var > 0.0 ? var : 0.0);
    iters[2 * k] = I;
    iters[2 * k + 1] = err;
    int nexact = 0;
    double exact_sum = 0.0;
    for (int q = 0; q <= k; ++q)
        if (iters[2 * q + 1] == 0.0) { ++nexact; exact_sum += iters[2 * q]; }
    double mean, merr, chi2 = 0.0;
    if (nexact > 0) {
        mean = exact_sum / nexact;
        merr = 0.0;
    } else {
        double sw = 0.0, swi = 0.0;
        for (int q = 0; q <= k; ++q) {
            double wq = 1.0 / (iters[2 * q + 1] * iters[2 * q + 1]);
            sw += wq;
            swi += wq * iters[2 * q];
        }
        mean = swi / sw;
        merr = 1.0 / sqrt(sw);
        if (k > 0) {
            for (int q = 0; q <= k; ++q) {
                double d = iters[2 * q] - mean;
                chi2 += d * d / (iters[2 * q + 1] * iters[2 * q + 1]);
            }
            chi2 /= k;
        }
    }
    res[0] = I; res[1] = err; res[2] = mean; res[3] = merr; res[4] = chi2;
    res[5] = tot[2]; res[6] = tot[3];
}

// Lepage refinement of every dimension (one thread per dimension).
__device__ void refine_dim(double *grid, const double *hist, int ndim, int nb, int64_t n, double alpha, int j);

__global__ void vegas_refine_kernel(double *grid, const double *hist, int ndim, int nb, int64_t n, double alpha) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < ndim) refine_dim(grid, hist, ndim, nb, n, alpha, j);
}

// Block c: channel c's refinement, one thread per dimension.
__global__ void vegas_refine_channels_kernel(const ChanAcc *ca, int ndim, int nb) {
    const ChanAcc &c = ca[blockIdx.x];
    if (c.refine && (int)threadIdx.x < ndim) refine_dim(c.grid, c.hist, ndim, nb, c.n, c.alpha, threadIdx.x);
}

__device__ void refine_dim(double *grid, const double *hist, int ndim, int nb, int64_t n, double alpha, int j) {
    double *g = grid + (size_t)j * (nb + 1);
    const double *d = hist + (size_t)j * nb;
    double sm[256], comp[256], newe[257];
    double N = (double)n;
    for (int i = 0; i < nb; ++i) {
        double a = d[i] / N;
        if (i == 0) sm[i] = (a + d[1] / N) / 2.0;
        else if (i == nb - 1) sm[i] = (d[nb - 2] / N + a) / 2.0;
        else sm[i] = (d[i - 1] / N + a + d[i + 1] / N) / 3.0;
    }
    double tot = 0.0;
    for (int i = 0; i < nb; ++i) tot += sm[i];
    if (!(tot > 0.0)) return;
    double total = 0.0;
    for (int i = 0; i < nb; ++i) {
        double r = sm[i] / tot;
        double c;
        if (r <= 0.0) c = 0.0;
        else if (r == 1.0) c = 1.0;
        else c = pow((r - 1.0) / log(r), alpha);
        comp[i] = c;
        total += c;
    }
    double per = total / nb;
    newe[0] = 0.0;
    double acc = 0.0;
    int io = -1;
    for (int k = 1; k < nb; ++k) {
        double target = k * per;
        while (acc < target && io < nb - 1) { ++io; acc += comp[io]; }
        double lo = g[io], hi = g[io + 1];
        double frac = comp[io] > 0.0 ? (target - (acc - comp[io])) / comp[io] : 1.0;
        newe[k] = lo + frac * (hi - lo);
    }
    newe[nb] = 1.0;
    for (int i = 0; i <= nb; ++i) g[i] = newe[i];
}

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double factorial(int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

mf_status ensure_context() {
    cudaError_t e = cudaFree(nullptr);
    if (e != cudaSuccess) return fail(MF_ECUDA, std::string("CUDA initialisation: ") + cudaGetErrorString(e));
    return MF_OK;
}

size_t smem_bytes_tc(const mf_process &p);

size_t smem_bytes(const mf_process &p, int prec, int block) {
    if (prec == MF_MIXED_TC) return smem_bytes_tc(p);
    size_t R = prec == MF_FP64 ? 8 : 4;
    int nden1 = p.gen.n_den > 0 ? p.gen.n_den : 1;
    size_t a = (size_t)block * p.n_legs * 4 * R + (size_t)block * nden1 * R;
    a += (16 - (((size_t)block * nden1 * R) % 16)) % 16;
    a += (size_t)block * 8 * 2 + (size_t)block * 4 + (block / 32 + 1) * 4;
    return a;
}

// Generate, compile and load the process kernel of precision prec with the
// launch shape (block, ht) into k.
mf_status compile_shape(mf_process *p, int prec, int block, int ht, mfi::Compiled &k, int min_blocks = -1,
                        int level = -1) {
    k.block = block;
    k.ht = ht;
    k.min_blocks = min_blocks;
    k.ptxas_level = level >= 0 ? level : p->opt.ptxas_level;
    mfi::GenInfo info;
    std::string src = mfi::generate_source(*p, prec, k.block, k.ht, info, "proc", true, min_blocks);
    std::vector<char> cubin;
    mf_status st = mfi::jit_compile(src, prec == MF_FP64 ? "mf_proc_f64.cu" : prec == MF_MIXED ? "mf_proc_mixed.cu"
                                                                                  : "mf_proc_mixed_tc.cu", cubin,
                                    k.ptxas_level);
    if (st != MF_OK) return st;
    // the shared-memory size depends on the program's denominator count
    p->source[prec] = src;
    p->gen = info;
    k.smem = smem_bytes(*p, prec, k.block);
    return mfi::load_kernel(cubin, k);
}

// Tile buffers (FP32, 128 threads) rounded up to 1 KB, then the tensor-core
// operands: A_hi and A_lo (128 x KP), B (NP x KP), the round and drain
// barriers and the tensor-memory address (mf::tc::Plan<NJ>::SMEM).
size_t smem_bytes_tc(const mf_process &p) {
    // the operand plan of device/mf_tc.cuh (Plan<NJ>): side by side, or
    // stacked when 2 NJ > 128
    const bool stacked = 2 * p.n_jamp > 128;
    const int K2 = stacked ? p.n_jamp : 2 * p.n_jamp, KP = (K2 + 7) / 8 * 8, NP = (K2 + 15) / 16 * 16;
    const int nden1 = p.gen.n_den > 0 ? p.gen.n_den : 1, block = 128;
    size_t tile = (size_t)block * p.n_legs * 4 * 4 + (size_t)block * nden1 * 4;
    tile += (16 - (((size_t)block * nden1 * 4) % 16)) % 16;
    tile += (size_t)block * 8 * 2 + (size_t)block * 4 + (block / 32 + 1) * 4;
    tile = (tile + 1023) / 1024 * 1024;
    return tile + 2 * (size_t)128 * KP * 4 + (size_t)NP * KP * 4 + (stacked ? 32 + 128 * 4 : 24);
}

int pow2_at_least(int n) {
    int v = 1;
    while (v < n) v <<= 1;
    return v;
}

// Units of helicity work the lanes of one point share (a power of two): the
// helicity pairs if the process uses them, else its helicities.  Before the
// vanishing helicities are known (the double-precision kernel compiled at
// creation), half the unfiltered count when a pair leg exists.
int lane_units(const mf_process *p) {
    if (!p->hel.empty())
        return p->pairs.empty() ? pow2_at_least((int)(p->hel.size() / p->n_legs)) : pow2_at_least((int)p->pairs.size() / 2);
    const int all = pow2_at_least((int)(p->hel_all.size() / p->n_legs));
    return (mfi::pair_leg(*p) >= 0 && all > 1) ? all / 2 : all;
}

// FLOPs of one point's helicity sum as evaluated: the pair program for each
// complete pair, one helicity's program for a pair with an absent member
// (the absent member's work is padding), or every helicity in full.
double helicity_sum_flops(const mf_process *p) {
    const double fh = p->gen.flops_per_hel;
    if (p->pairs.empty()) return fh * (double)(p->hel.size() / p->n_legs);
    double f = 0.0;
    for (size_t u = 0; u < p->pairs.size(); u += 2)
        f += (p->pairs[u] != 0xFF && p->pairs[u + 1] != 0xFF) ? p->gen.flops_pair : fh;
    return f;
}

void fill_common(const mf_process &p, mf_kparams &kp);
void set_hel(mf_kparams &kp, const std::vector<int8_t> &hel, int n_legs);
mf_status launch(mf_process *p, int prec, mf_kparams &kp, cudaStream_t s);
mf_status flag_status(mf_process *p, int flag, bool nonfinite);

// Self-check of a compiled kernel's helicity-pair program.  The same kernel
// evaluates the helicity sum with the pair program (the process's pair
// table) or, given no pairs, one helicity at a time; on 256 seeded points
// the two must agree to rounding.  They did not for one FP64 gg -> tt~g
// program (amplitude units, searched order, amplitude routines called):
// the same source built at device-assembler level 0 or 1 was right, at 2 or
// 3 wrong at every point -- an optimisation of the assembler, not the
// generated program, which also passes on the host.  On disagreement the
// kernel is therefore rebuilt at level 1, then 0; if it still disagrees the
// process cannot be used (MF_EJIT).  Kernels without pairs and the
// tensor-core kernel (single helicities) have nothing to check.
mf_status verify_pairs(mf_process *p, int prec) {
    if (p->pairs.empty() || prec == MF_MIXED_TC || !p->kern[prec].fn) return MF_OK;
    const int npts = 256;
    std::vector<double> hx((size_t)p->ndim * npts);
    uint64_t seed = 0xC0FFEEu;
    for (auto &v : hx) v = ((splitmix64(seed) >> 11) | 1ull) * 0x1p-53;
    double *dx = nullptr, *df = nullptr;
    if (mfi::dev_malloc(&dx, sizeof(double) * hx.size()) != cudaSuccess ||
        mfi::dev_malloc(&df, sizeof(double) * 2 * npts) != cudaSuccess) {
        cudaFree(dx);
        return fail(MF_ENOMEM, "pair-program check scratch");
    }
    mf_status st = MF_OK;
    const double tol = prec == MF_FP64 ? 1e-10 : 1e-3;
    const int levels[3] = {-1, 1, 0};
    bool ok = false;
    for (int attempt = 0; attempt < 3 && st == MF_OK && !ok; ++attempt) {
        mfi::Compiled &k = p->kern[prec];
        if (attempt > 0) {
            if (p->opt.ptxas_level >= 0 && p->opt.ptxas_level <= levels[attempt]) break;
            mfi::Compiled rebuilt;
            st = compile_shape(p, prec, k.block, k.ht, rebuilt, k.min_blocks, levels[attempt]);
            if (st != MF_OK) break;
            mfi::unload_kernel(k);
            k = rebuilt;
        }
        std::vector<double> hf(2 * npts);
        int flag = 0;
        cudaError_t e = cudaMemcpy(dx, hx.data(), sizeof(double) * hx.size(), cudaMemcpyHostToDevice);
        for (int pass = 0; pass < 2 && e == cudaSuccess && st == MF_OK; ++pass) {
            mf_kparams kp;
            fill_common(*p, kp);
            set_hel(kp, p->hel, p->n_legs);
            kp.hel_sample = 0;
            kp.colour_sample = 0;
            kp.variant = 0;
            if (pass == 1) kp.npairs = 0;            // one helicity at a time
            kp.mode = 0;
            kp.n = npts;
            kp.x = dx;
            kp.f = df + pass * npts;
            st = launch(p, prec, kp, nullptr);
        }
        if (st == MF_OK && e == cudaSuccess) e = cudaMemcpy(hf.data(), df, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost);
        if (st == MF_OK && e == cudaSuccess) e = cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (st == MF_OK && e != cudaSuccess) st = fail(MF_ECUDA, std::string("pair-program check: ") + cudaGetErrorString(e));
        // non-finite values (a program that overflows) are the caller's to
        // see, not this check's: the flag they raised is cleared and those
        // points are skipped
        if (st == MF_OK) st = flag_status(p, flag, false);
        if (st == MF_OK && flag == 3) cudaMemset(p->d_err, 0, sizeof(int));
        if (st != MF_OK) break;
        ok = true;
        for (int i = 0; i < npts && ok; ++i) {
            const double a = hf[i], b = hf[npts + i];
            if (!std::isfinite(a) || !std::isfinite(b)) continue;
            ok = (a == 0.0) == (b == 0.0) && std::fabs(a - b) <= tol * std::fabs(b);
        }
    }
    cudaFree(dx);
    cudaFree(df);
    if (st != MF_OK) return st;
    if (!ok)
        return fail(MF_EJIT, "the compiled helicity-pair program disagrees with the single-helicity program "
                             "(device assembler at every level tried)");
    return MF_OK;
}

mf_status compile_precision(mf_process *p, int prec) {
    mfi::Compiled &k = p->kern[prec];
    if (k.fn) return MF_OK;
    // long programs run in blocks of 256 (one per SM at 255 registers): the
    // eight warps of one block share the instruction stream (gg -> tt~gg:
    // 1.04x over two blocks of 128)
    int block = (mfi::large_program(*p) && prec != MF_MIXED_TC) ? 256 : 128;
    const int nhp = lane_units(p);
    int ht = nhp < 32 ? nhp : 32;
    // launch-shape options: block size and lanes per event
    if (p->opt.block > 0 && prec != MF_MIXED_TC) block = p->opt.block;
    if (p->opt.lanes > 0 && p->opt.lanes <= nhp) ht = p->opt.lanes;
    mf_status st = compile_shape(p, prec, block, ht, k);
    if (st != MF_OK) return st;
    return verify_pairs(p, prec);
}

mf_status compile_grad(mf_process *p) {
    mfi::Compiled &k = p->kern[2];
    if (k.fn) return MF_OK;
    k.block = 128;
    k.smem = 0;
    mfi::GenInfo info;
    p->source[2] = mfi::generate_grad_source(*p, k.block, info);
    std::vector<char> cubin;
    mf_status st = mfi::jit_compile(p->source[2], "mf_proc_grad.cu", cubin, p->opt.ptxas_level);
    if (st != MF_OK) return st;
    return mfi::load_kernel(cubin, k, "mf_grad_kernel");
}

void fill_common(const mf_process &p, mf_kparams &kp) {
    std::memset(&kp, 0, sizeof kp);
    kp.wait_polls = p.opt.wait_polls;   // negative: the kernels' default limit
    kp.colour_sample = p.colour_sample;
    kp.variant = p.colour_sample ? 2 : 0;
    kp.S = p.sqrt_s * p.sqrt_s;
    kp.ln_tau_min = p.ln_tau_min;
    kp.w0_const = p.w0_const;
    kp.pref_const = p.pref_const;
    kp.pt_min2 = p.pt_min * p.pt_min;
    kp.dr_min2 = p.dr_min * p.dr_min;
    kp.pdf_a0 = p.pdf_a0;
    kp.pdf_h = p.pdf_h;
    kp.pdf_nx = p.pdf_nx;
    kp.pdf_rows = p.d_pdf_rows;
    for (size_t i = 0; i < p.masses.size() && i < 8; ++i) kp.masses[i] = p.masses[i];
    for (size_t i = 0; i < p.couplings.size() && i < 16; ++i) kp.couplings[i] = p.couplings[i];
    kp.alpha_s = p.alpha_s;
    kp.alpha_s_power = p.alpha_s_power;
    kp.err = p.d_err;
    kp.hel_sample = p.hel_sample;
    kp.npairs = (int32_t)(p.pairs.size() / 2);
    kp.npairs_pow2 = pow2_at_least(kp.npairs);
    for (int u = 0; u < kp.npairs; ++u) {
        kp.pairs[u][0] = p.pairs[2 * u];
        kp.pairs[u][1] = p.pairs[2 * u + 1];
    }
    kp.seed = p.hel_seed;          // Vegas passes overwrite it with their own key
    kp.chan = p.d_chan;
    kp.channel = -1;               // the flat phase space unless a channel call sets one
    kp.ch_s0 = p.ch_s0;
    kp.ch_t0 = p.ch_t0;
}

// Pairs of kept helicities that differ only at the pair leg L, in the order
// of their first row; used when the padded pairs cost fewer FLOPs than the
// padded single helicities (every thread evaluates the padded count).
void build_pairs(mf_process *p) {
    p->pairs.clear();
    const int L = p->gen.pair_leg, n = p->n_legs;
    const int nh = (int)(p->hel.size() / n);
    // (row indices are stored in one byte with 0xFF for an absent member, so
    // a table of 256 kept rows is evaluated one helicity at a time)
    if (L < 0 || nh == 0 || nh > 255) return;
    if (p->opt.helicity_pairs == 0) return;                // the option: helicities one by one
    std::vector<uint8_t> t;
    std::vector<std::vector<int8_t>> keys;
    for (int h = 0; h < nh; ++h) {
        const int8_t *row = &p->hel[(size_t)h * n];
        if (row[L] != -1 && row[L] != 1) return;
        std::vector<int8_t> key(row, row + n);
        key[L] = 0;
        size_t u = 0;
        while (u < keys.size() && keys[u] != key) ++u;
        if (u == keys.size()) {
            keys.push_back(key);
            t.push_back(0xFF);
            t.push_back(0xFF);
        }
        t[2 * u + (row[L] == 1)] = (uint8_t)h;
    }
    const double single = p->gen.flops_per_hel * pow2_at_least(nh);
    const double paired = p->gen.flops_pair * pow2_at_least((int)keys.size());
    if (paired < single) p->pairs = t;
}

bool valid_prec(int prec) { return prec == MF_FP64 || prec == MF_MIXED || prec == MF_MIXED_TC; }

// A process kernel's error flag: 1 = a bounded wait expired, 2 = the launch
// gave less dynamic shared memory than the kernel needs, 3 = mf_integrand
// wrote a non-finite value.  Read after the stream has been synchronised;
// clears the flag.  The synchronous Vegas paths pass nonfinite = false:
// they count their own non-finite weights, and leave a flag 3 raised by an
// earlier mf_integrand call to mf_process_check.
mf_status flag_status(mf_process *p, int flag, bool nonfinite = false) {
    if (!flag || (flag == 3 && !nonfinite)) return MF_OK;
    cudaMemset(p->d_err, 0, sizeof(int));
    if (flag == 2) return fail(MF_ECUDA, "process kernel launched with too little shared memory (results not written)");
    if (flag == 3)
        return fail(MF_ENAN, "the integrand wrote non-finite values (non-finite coordinates, or overflow)");
    return fail(MF_ETIMEOUT, "a bounded wait in a process kernel expired; that launch's results are unspecified");
}

void set_hel(mf_kparams &kp, const std::vector<int8_t> &hel, int n_legs) {
    int nh = (int)(hel.size() / n_legs);
    kp.nhel = nh;
    int nhp = 1;
    while (nhp < nh) nhp <<= 1;
    kp.nhel_pow2 = nhp;
    for (int h = 0; h < nh; ++h)
        for (int l = 0; l < n_legs; ++l) kp.hel[h][l] = hel[(size_t)h * n_legs + l];
}

mf_status launch(mf_process *p, int prec, mf_kparams &kp, cudaStream_t s) {
    mfi::Compiled &k = p->kern[prec];
    int64_t ntiles = (kp.n + k.block - 1) / k.block;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = k.max_blocks_per_sm;
    // launch-shape option: resident blocks per SM the grid is sized for
    if (p->opt.blocks_per_sm >= 1) per_sm = p->opt.blocks_per_sm;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    void *args[] = {&kp};
    return mfi::launch_kernel(k, (unsigned)grid, args, s, kp.mode == 5 ? 1 : kp.variant);
}

// Ranges of the process options (MF_OPT_AUTO allowed everywhere).
mf_status validate_options(const mf_process_options *o) {
    if (!o) return MF_OK;
    auto in = [](int v, int lo, int hi) { return v == MF_OPT_AUTO || (v >= lo && v <= hi); };
    const bool pow2 = o->lanes == MF_OPT_AUTO || (o->lanes >= 1 && o->lanes <= 32 && (o->lanes & (o->lanes - 1)) == 0);
    if (!in(o->amplitude_units, 0, 1) || !in(o->call_routines, 0, 3) || !in(o->order_search, 0, 1 << 24) ||
        !in(o->sync_every, 0, 1 << 20) || !in(o->program_parts, 1, 4096) || !in(o->min_blocks, 0, 8) ||
        !in(o->helicity_pairs, 0, 1) || !(o->block == MF_OPT_AUTO || o->block == 128 || o->block == 256) || !pow2 ||
        !in(o->blocks_per_sm, 1, 8) || !in(o->ptxas_level, 0, 3) || !in(o->wait_polls, 0, 1 << 30))
        return fail(MF_EINVAL, "process option out of range");
    return MF_OK;
}

mf_status validate(const mf_process_desc *d) {
    if (!d) return fail(MF_EINVAL, "NULL descriptor");
    if (validate_options(d->options) != MF_OK) return MF_EINVAL;
    if (d->n_legs < 3) return fail(MF_EINVAL, "need at least 3 legs");
    if (d->n_legs > MF_MAX_LEGS) return fail(MF_EUNSUPPORTED, "too many legs");
    if (!d->leg_kind || !d->leg_incoming || !d->leg_mass_id || !d->leg_cut)
        return fail(MF_EINVAL, "leg arrays must be non-NULL");
    for (int i = 0; i < d->n_legs; ++i) {
        if (d->leg_kind[i] < 0 || d->leg_kind[i] > 2) return fail(MF_EINVAL, "bad leg kind");
        if ((i < 2) != (d->leg_incoming[i] != 0)) return fail(MF_EINVAL, "legs 0 and 1 must be the incoming ones");
        if (d->leg_mass_id[i] < -1 || d->leg_mass_id[i] >= d->n_masses) return fail(MF_EINVAL, "bad leg mass id");
        if (i < 2 && d->leg_mass_id[i] >= 0 && d->masses[d->leg_mass_id[i]] != 0.0)
            return fail(MF_EUNSUPPORTED, "incoming legs must be massless");
        if (d->leg_kind[i] == MF_LEG_VECTOR && d->leg_mass_id[i] >= 0 && d->masses[d->leg_mass_id[i]] != 0.0)
            return fail(MF_EUNSUPPORTED, "only massless vector bosons");
    }
    if (d->n_masses < 0 || d->n_masses > 8 || (d->n_masses > 0 && !d->masses))
        return fail(MF_EINVAL, "n_masses must be in [0, 8]");
    if (d->n_couplings < 1 || d->n_couplings > 8 || !d->couplings) return fail(MF_EINVAL, "n_couplings must be in [1, 8]");
    if (d->n_jamp < 1) return fail(MF_EINVAL, "n_jamp must be positive");
    if (d->n_jamp > MF_MAX_JAMP) return fail(MF_EUNSUPPORTED, "too many colour flows");
    if (!d->colour_num || d->colour_den <= 0) return fail(MF_EINVAL, "bad colour matrix");
    for (int a = 0; a < d->n_jamp; ++a)
        for (int b = 0; b < d->n_jamp; ++b)
            if (d->colour_num[a * d->n_jamp + b] != d->colour_num[b * d->n_jamp + a])
                return fail(MF_EINVAL, "colour matrix must be symmetric");
    if (d->n_ops < 1 || !d->ops) return fail(MF_EINVAL, "empty program");
    if (d->n_terms < 0 || (d->n_terms > 0 && !d->terms)) return fail(MF_EINVAL, "bad colour terms");
    std::vector<int> is_wf(d->n_ops, 0);
    std::vector<int> leg_seen(d->n_legs, 0);
    int n_amp = 0;
    for (int k = 0; k < d->n_ops; ++k) {
        const mf_op &op = d->ops[k];
        int nin = 0;
        switch (op.routine) {
            case MF_R_IXX: case MF_R_OXX: case MF_R_VXX: nin = 0; break;
            case MF_R_FFV_FIN: case MF_R_FFV_FOUT: case MF_R_FFV_VEC: case MF_R_VVV_VEC: nin = 2; break;
            case MF_R_FFV_AMP: case MF_R_VVV_AMP: case MF_R_VVVV1_VEC: case MF_R_VVVV2_VEC: case MF_R_VVVV3_VEC: nin = 3; break;
            case MF_R_VVVV1_AMP: case MF_R_VVVV2_AMP: case MF_R_VVVV3_AMP: nin = 4; break;
            default: return fail(MF_EINVAL, "unknown routine in op " + std::to_string(k));
        }
        bool ext_r = op.routine <= MF_R_VXX;
        bool amp_r = op.routine == MF_R_FFV_AMP || op.routine == MF_R_VVV_AMP ||
                     (op.routine >= MF_R_VVVV1_AMP && op.routine <= MF_R_VVVV3_AMP);
        if (op.kind == MF_OP_EXT) {
            if (!ext_r) return fail(MF_EINVAL, "EXT op with a vertex routine");
            if (op.leg < 0 || op.leg >= d->n_legs || leg_seen[op.leg]) return fail(MF_EINVAL, "bad EXT leg");
            int want = op.routine == MF_R_IXX ? MF_LEG_FERMION_IN : op.routine == MF_R_OXX ? MF_LEG_FERMION_OUT : MF_LEG_VECTOR;
            if (d->leg_kind[op.leg] != want) return fail(MF_EINVAL, "EXT routine does not match the leg kind");
            leg_seen[op.leg] = 1;
            is_wf[k] = 1;
        } else if (op.kind == MF_OP_CUR || op.kind == MF_OP_AMP) {
            if (ext_r || (op.kind == MF_OP_AMP) != amp_r) return fail(MF_EINVAL, "op kind does not match its routine");
            for (int q = 0; q < 4; ++q) {
                if (q < nin) {
                    if (op.in[q] < 0 || op.in[q] >= k || !is_wf[op.in[q]])
                        return fail(MF_EINVAL, "op " + std::to_string(k) + " reads a missing wavefunction");
                } else if (op.in[q] != -1) {
                    return fail(MF_EINVAL, "unused inputs must be -1");
                }
            }
            if (op.coupling < 0 || op.coupling >= d->n_couplings) return fail(MF_EINVAL, "bad coupling index");
            if (op.kind == MF_OP_CUR) {
                if (op.mass_id < -1 || op.mass_id >= d->n_masses) return fail(MF_EINVAL, "bad propagator mass id");
                is_wf[k] = 1;
            } else {
                ++n_amp;
                if (op.first_term < 0 || op.n_terms < 0 || op.first_term + op.n_terms > d->n_terms)
                    return fail(MF_EINVAL, "bad colour-term range");
                for (int t = 0; t < op.n_terms; ++t) {
                    int j = d->terms[op.first_term + t].jamp;
                    if (j < 0 || j >= d->n_jamp) return fail(MF_EINVAL, "colour term outside the flows");
                }
            }
        } else {
            return fail(MF_EINVAL, "bad op kind");
        }
    }
    for (int i = 0; i < d->n_legs; ++i)
        if (!leg_seen[i]) return fail(MF_EINVAL, "every leg needs one EXT op");
    if (n_amp == 0) return fail(MF_EINVAL, "program has no amplitude");
    if (d->n_hel < 0 || (d->n_hel > 0 && !d->helicities)) return fail(MF_EINVAL, "bad helicity table");
    if (d->n_hel > MF_KP_MAX_HEL || (d->n_hel == 0 && (1 << d->n_legs) > MF_KP_MAX_HEL))
        return fail(MF_EUNSUPPORTED, "too many helicity rows");
    for (int h = 0; h < d->n_hel * d->n_legs; ++h)
        if (d->helicities[h] != 1 && d->helicities[h] != -1) return fail(MF_EINVAL, "helicities must be +-1");
    if (!(d->sqrt_s > 0.0)) return fail(MF_EINVAL, "sqrt_s must be positive");
    if (!(d->average > 0.0)) return fail(MF_EINVAL, "average must be positive");
    if (d->pt_min < 0.0 || d->dr_min < 0.0) return fail(MF_EINVAL, "cuts must be non-negative");
    if (d->hadronic) {
        if (!d->pdf[0] || !d->pdf[1]) return fail(MF_EINVAL, "hadronic process needs two PDF tables");
        if (d->pdf_nx < 4 || d->pdf_nq < 4) return fail(MF_EINVAL, "PDF tables need at least 4 knots per axis");
        if (!(d->pdf_x_min > 0.0 && d->pdf_x_max > d->pdf_x_min && d->pdf_q2_min > 0.0 && d->pdf_q2_max > d->pdf_q2_min))
            return fail(MF_EINVAL, "bad PDF axes");
        if (!(d->mu_f2 > 0.0)) return fail(MF_EINVAL, "mu_f2 must be positive");
    }
    int nout = d->n_legs - 2;
    int ndim = 3 * nout - 4 + (d->hadronic ? 2 : 0);
    if (ndim > MF_MAX_DIM) return fail(MF_EUNSUPPORTED, "too many integration dimensions");
    return MF_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// process
// ----------------------------------------------------------------------------
extern "C" mf_status mf_create_process(const mf_process_desc *d, mf_process **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    mf_status st = validate(d);
    if (st != MF_OK) return st;
    st = ensure_context();
    if (st != MF_OK) return st;
    mf_process *p = new (std::nothrow) mf_process();
    if (!p) return fail(MF_ENOMEM, "host allocation");
    cudaGetDevice(&p->device);
    const int n = d->n_legs;
    p->n_legs = n;
    p->n_out = n - 2;
    p->hadronic = d->hadronic ? 1 : 0;
    p->ndim = 3 * p->n_out - 4 + 2 * p->hadronic;
    p->leg_kind.assign(d->leg_kind, d->leg_kind + n);
    p->leg_incoming.assign(d->leg_incoming, d->leg_incoming + n);
    p->leg_mass_id.assign(d->leg_mass_id, d->leg_mass_id + n);
    p->leg_cut.assign(d->leg_cut, d->leg_cut + n);
    p->masses.assign(d->masses, d->masses + d->n_masses);
    p->ops.assign(d->ops, d->ops + d->n_ops);
    if (d->n_terms > 0) p->terms.assign(d->terms, d->terms + d->n_terms);
    p->couplings.assign(d->couplings, d->couplings + 2 * d->n_couplings);
    p->n_jamp = d->n_jamp;
    p->colour_num.assign(d->colour_num, d->colour_num + d->n_jamp * d->n_jamp);
    p->colour_den = d->colour_den;
    if (d->options) p->opt = *d->options;
    if (d->n_hel > 0) {
        p->hel_all.assign(d->helicities, d->helicities + (size_t)d->n_hel * n);
    } else {
        for (int h = 0; h < (1 << n); ++h)
            for (int l = 0; l < n; ++l) p->hel_all.push_back((h >> (n - 1 - l)) & 1 ? 1 : -1);
    }
    p->average = d->average;
    p->alpha_s_power = d->alpha_s_power;
    p->alpha_s = d->alpha_s;
    p->sqrt_s = d->sqrt_s;
    p->mu_f2 = d->mu_f2;
    p->pt_min = d->pt_min;
    p->dr_min = d->dr_min;
    // constants of the phase space and weight
    double msum = 0.0;
    for (int i = 2; i < n; ++i)
        if (p->leg_mass_id[i] >= 0) msum += p->masses[p->leg_mass_id[i]];
    const double S = d->sqrt_s * d->sqrt_s;
    if (p->hadronic) {
        if (!(msum > 0.0) || !(msum < d->sqrt_s)) {
            delete p;
            return fail(MF_EUNSUPPORTED, "the x1, x2 map needs 0 < sum of final masses < sqrt_s");
        }
        p->ln_tau_min = std::log(msum * msum / S);
    }
    const int no = p->n_out;
    p->w0_const = std::pow(2.0 * kPi, 4 - 3 * no) * std::pow(kPi / 2.0, no - 1) / (factorial(no - 1) * factorial(no - 2));
    p->pref_const = p->average * kGeV2pb / 2.0;
    if (mfi::dev_malloc(&p->d_err, sizeof(int)) != cudaSuccess || cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) {
        mf_destroy_process(p);
        return fail(MF_ENOMEM, "error flag");
    }
    // channels of the multichannel phase space (none for programs outside the
    // table's limits; the flat phase space is always available)
    {
        mf_status cst = mfi::derive_channels(p->n_legs, p->ops, p->channels);
        if (cst != MF_OK) {
            p->channels = mfi::ChannelSet();
        } else if (p->channels.K > 0) {
            const size_t bytes = sizeof(int32_t) * p->channels.table.size();
            if (mfi::dev_malloc(&p->d_chan, bytes) != cudaSuccess ||
                cudaMemcpy(p->d_chan, p->channels.table.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
                mf_destroy_process(p);
                return fail(MF_ENOMEM, "channel table");
            }
        }
        const double r = 4.0 * std::max(p->pt_min, 1.0);
        p->ch_s0 = p->ch_t0 = r * r;
    }
    // PDF rows at fixed mu_F^2
    if (p->hadronic) {
        const int nx = d->pdf_nx, nq = d->pdf_nq;
        p->pdf_nx = nx;
        p->pdf_a0 = std::log(d->pdf_x_min);
        p->pdf_h = (std::log(d->pdf_x_max) - std::log(d->pdf_x_min)) / (nx - 1);
        double b0 = std::log(d->pdf_q2_min);
        double hb = (std::log(d->pdf_q2_max) - b0) / (nq - 1);
        double *d_tab = nullptr;
        if (mfi::dev_malloc(&p->d_pdf_rows, sizeof(double) * 4 * nx) != cudaSuccess ||
            mfi::dev_malloc(&d_tab, sizeof(double) * (size_t)nx * nq) != cudaSuccess) {
            cudaFree(d_tab);
            mf_destroy_process(p);
            return fail(MF_ENOMEM, "PDF rows");
        }
        for (int b = 0; b < 2; ++b) {
            cudaMemcpy(d_tab, d->pdf[b], sizeof(double) * (size_t)nx * nq, cudaMemcpyHostToDevice);
            double *row = p->d_pdf_rows + (size_t)(2 * b) * nx;
            pdf_collapse_kernel<<<1, 128>>>(d_tab, nx, nq, b0, hb, std::log(d->mu_f2), row, row + nx);
            scale_kernel<<<1, 128>>>(row + nx, nx, 1.0 / p->pdf_h);
        }
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(d_tab);
        if (e != cudaSuccess) {
            mf_destroy_process(p);
            return fail(MF_ECUDA, std::string("PDF set-up: ") + cudaGetErrorString(e));
        }
    }
    // compile the double-precision kernel and drop vanishing helicities
    st = compile_precision(p, MF_FP64);
    if (st != MF_OK) {
        std::string msg = mf_last_error();
        mf_destroy_process(p);
        return fail(st, msg);
    }
    {
        const int npts = 256;
        std::vector<double> hx((size_t)p->ndim * npts);
        uint64_t s = 0x5EEDu;
        for (auto &v : hx) v = ((splitmix64(s) >> 11) | 1ull) * 0x1p-53;
        const int nh = (int)(p->hel_all.size() / n);
        double *dx = nullptr, *df = nullptr;
        if (mfi::dev_malloc(&dx, sizeof(double) * hx.size()) != cudaSuccess ||
            mfi::dev_malloc(&df, sizeof(double) * (size_t)nh * npts) != cudaSuccess) {
            cudaFree(dx);
            mf_destroy_process(p);
            return fail(MF_ENOMEM, "helicity filter scratch");
        }
        cudaMemcpy(dx, hx.data(), sizeof(double) * hx.size(), cudaMemcpyHostToDevice);
        cudaMemset(df, 0, sizeof(double) * (size_t)nh * npts);
        mf_kparams kp;
        fill_common(*p, kp);
        set_hel(kp, p->hel_all, n);
        kp.mode = 2;
        kp.variant = 0;
    kp.variant = 0;                       // per-helicity values: the integrand kernel
        kp.n = npts;
        kp.x = dx;
        kp.f = df;
        st = launch(p, MF_FP64, kp, nullptr);
        std::vector<double> hf((size_t)nh * npts);
        cudaError_t e = cudaMemcpy(hf.data(), df, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost);
        int flag = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(dx);
        cudaFree(df);
        if (st == MF_OK && e == cudaSuccess) st = flag_status(p, flag);
        if (st != MF_OK || e != cudaSuccess) {
            mf_destroy_process(p);
            return st != MF_OK ? st : fail(MF_ECUDA, std::string("helicity filter run failed: ") + cudaGetErrorString(e));
        }
        // a helicity vanishes when it stays below 1e-12 of the helicity sum at
        // every test point: amplitudes that chirality makes zero come out as
        // rounding residues (~1e-16 of the sum), physical ones far above
        std::vector<double> tot(npts, 0.0);
        for (int h = 0; h < nh; ++h)
            for (int i = 0; i < npts; ++i) tot[i] += std::fabs(hf[(size_t)h * npts + i]);
        bool any = false;
        for (double v : tot) any |= (v > 0.0);
        for (int h = 0; h < nh; ++h) {
            bool keep = !any;
            for (int i = 0; i < npts && !keep; ++i) keep = std::fabs(hf[(size_t)h * npts + i]) > 1e-12 * tot[i];
            if (keep)
                for (int l = 0; l < n; ++l) p->hel.push_back(p->hel_all[(size_t)h * n + l]);
        }
    }
    build_pairs(p);
    st = verify_pairs(p, MF_FP64);
    if (st != MF_OK) {
        std::string msg = mf_last_error();
        mf_destroy_process(p);
        return fail(st, msg);
    }
    *out = p;
    return MF_OK;
}

namespace {
// The parts of a process that code generation reads, from a validated
// descriptor (no device work).
int shell_from_desc(const mf_process_desc *d, mf_process &p) {
    const int n = d->n_legs;
    p.n_legs = n;
    p.n_out = n - 2;
    p.hadronic = d->hadronic ? 1 : 0;
    p.ndim = 3 * p.n_out - 4 + 2 * p.hadronic;
    p.leg_kind.assign(d->leg_kind, d->leg_kind + n);
    p.leg_incoming.assign(d->leg_incoming, d->leg_incoming + n);
    p.leg_mass_id.assign(d->leg_mass_id, d->leg_mass_id + n);
    p.leg_cut.assign(d->leg_cut, d->leg_cut + n);
    p.masses.assign(d->masses, d->masses + d->n_masses);
    p.ops.assign(d->ops, d->ops + d->n_ops);
    if (d->n_terms > 0) p.terms.assign(d->terms, d->terms + d->n_terms);
    p.couplings.assign(d->couplings, d->couplings + 2 * d->n_couplings);
    p.n_jamp = d->n_jamp;
    p.colour_num.assign(d->colour_num, d->colour_num + d->n_jamp * d->n_jamp);
    p.colour_den = d->colour_den;
    if (d->options) p.opt = *d->options;
    int nh = d->n_hel > 0 ? d->n_hel : (1 << n);
    int nhp = 1;
    while (nhp < nh) nhp <<= 1;
    return nhp < 32 ? nhp : 32;
}

mf_status emit_source(const std::string &src, const char *name, int32_t compile, char *buf, size_t *len,
                      int ptxas_level = -1) {
    if (compile) {
        std::vector<char> cubin;
        mf_status st = mfi::jit_compile(src, name, cubin, ptxas_level);
        if (st != MF_OK) return st;
    }
    size_t need = src.size() + 1;
    if (buf && *len >= need) std::memcpy(buf, src.c_str(), need);
    *len = need;
    return MF_OK;
}
}  // namespace

extern "C" mf_status mf_generate_kernel_source(const mf_process_desc *d, mf_precision prec, int32_t compile,
                                               char *buf, size_t *len) {
    if (!len) return fail(MF_EINVAL, "len is NULL");
    if (!valid_prec(prec) && (int)prec != 2) return fail(MF_EINVAL, "bad precision");
    mf_status st = validate(d);
    if (st != MF_OK) return st;
    mf_process p;
    const int ht = shell_from_desc(d, p);
    mfi::GenInfo info;
    std::string src = (int)prec == 2 ? mfi::generate_grad_source(p, 128, info)
                                     : mfi::generate_source(p, prec, 128, ht, info);
    return emit_source(src, (int)prec == 2 ? "mf_proc_grad.cu" : prec == MF_FP64 ? "mf_proc_f64.cu"
                                              : prec == MF_MIXED ? "mf_proc_mixed.cu" : "mf_proc_mixed_tc.cu",
                       compile, buf, len, p.opt.ptxas_level);
}

extern "C" mf_status mf_generate_batch_source(const mf_process_desc *const *descs, int32_t nproc, mf_precision prec,
                                              int32_t compile, char *buf, size_t *len) {
    if (!len || !descs) return fail(MF_EINVAL, "NULL argument");
    if (nproc < 1 || nproc > MF_KP_MAX_BATCH) return fail(MF_EINVAL, "need 1 to 8 processes");
    if (prec != MF_FP64 && prec != MF_MIXED) return fail(MF_EINVAL, "bad precision");
    std::vector<mf_process> shells(nproc);
    std::vector<const mf_process *> ps;
    std::vector<int> hts;
    for (int k = 0; k < nproc; ++k) {
        mf_status st = validate(descs[k]);
        if (st != MF_OK) return st;
        hts.push_back(shell_from_desc(descs[k], shells[k]));
        ps.push_back(&shells[k]);
    }
    std::vector<mfi::GenInfo> infos;
    std::string src = mfi::generate_batch_source(ps, prec, 128, hts, infos);
    return emit_source(src, prec == MF_FP64 ? "mf_batch_f64.cu" : "mf_batch_mixed.cu", compile, buf, len);
}

extern "C" mf_status mf_destroy_process(mf_process *p) {
    if (!p) return MF_OK;
    for (auto &k : p->kern) mfi::unload_kernel(k);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->ev_stop) cudaEventDestroy(p->ev_stop);
    cudaFree(p->d_pdf_rows);
    cudaFree(p->d_err);
    cudaFree(p->d_chan);
    cudaFree(p->d_ch_off);
    cudaFree(p->d_ch_grids);
    cudaFree(p->d_ch_chunk_off);
    cudaFree(p->d_ch_res);
    cudaFree(p->d_ch_acc);
    cudaFree(p->d_w);
    cudaFree(p->d_bins);
    delete p;
    return MF_OK;
}

extern "C" mf_status mf_process_get_info(const mf_process *p, mf_process_info *info) {
    if (!p || !info) return fail(MF_EINVAL, "NULL argument");
    info->ndim = p->ndim;
    info->n_legs = p->n_legs;
    info->n_hel = (int)(p->hel.size() / p->n_legs);
    info->n_hel_all = (int)(p->hel_all.size() / p->n_legs);
    info->n_jamp = p->n_jamp;
    info->n_ops = (int)p->ops.size();
    info->n_den = p->gen.n_den;
    info->flops_per_hel = p->gen.flops_per_hel;
    info->flops_kinematics = p->gen.flops_kin;
    info->pair_leg = p->pairs.empty() ? -1 : p->gen.pair_leg;
    info->n_pairs = (int32_t)(p->pairs.size() / 2);
    info->flops_helicity_sum = helicity_sum_flops(p);
    info->helicity_sampling = p->hel_sample;
    return MF_OK;
}

extern "C" mf_status mf_process_last_kernel_ms(const mf_process *p, double *ms) {
    if (!p || !ms) return fail(MF_EINVAL, "NULL argument");
    *ms = p->last_kernel_ms;
    return MF_OK;
}

extern "C" mf_status mf_process_set_helicity_sampling(mf_process *p, int32_t on, uint64_t seed) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (on < 0 || on > 2) return fail(MF_EINVAL, "helicity sampling mode must be 0, 1 or 2");
    // mode 2 samples helicity pairs; a process without pairs samples single helicities
    p->hel_sample = (on == 2 && p->pairs.empty()) ? 1 : on;
    p->hel_seed = seed;
    return MF_OK;
}

extern "C" mf_status mf_process_set_colour_sampling(mf_process *p, int32_t on) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (on != 0 && on != 1) return fail(MF_EINVAL, "colour sampling must be 0 or 1");
    p->colour_sample = on;
    return MF_OK;
}

extern "C" mf_status mf_process_get_helicity_pairs(const mf_process *p, int32_t *pairs, int32_t *n_pairs) {
    if (!p || !n_pairs) return fail(MF_EINVAL, "NULL argument");
    *n_pairs = (int32_t)(p->pairs.size() / 2);
    if (pairs)
        for (size_t k = 0; k < p->pairs.size(); ++k) pairs[k] = p->pairs[k] == 0xFF ? -1 : (int32_t)p->pairs[k];
    return MF_OK;
}

extern "C" mf_status mf_process_set_leading_colour(mf_process *p, int32_t on) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    const int v = on ? 1 : 0;
    if (v == p->leading_colour) return MF_OK;
    // the integrand kernels are regenerated on their next use
    MF_CUDA(cudaDeviceSynchronize());
    for (int prec : {(int)MF_FP64, (int)MF_MIXED, (int)MF_MIXED_TC}) mfi::unload_kernel(p->kern[prec]);
    p->leading_colour = v;
    return MF_OK;
}

extern "C" mf_status mf_process_kernel_info(const mf_process *p, mf_precision prec, int32_t *block, int32_t *ht,
                                            int32_t *regs, int32_t *blocks_per_sm, int32_t *min_blocks) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    const mfi::Compiled &k = p->kern[prec];
    if (!k.fn) return fail(MF_EINVAL, "the kernel of this precision is not compiled yet");
    if (block) *block = k.block;
    if (ht) *ht = k.ht;
    if (regs) *regs = k.regs;
    if (blocks_per_sm) *blocks_per_sm = k.max_blocks_per_sm;
    if (min_blocks) *min_blocks = k.min_blocks > 0 ? k.min_blocks : 0;
    return MF_OK;
}

extern "C" mf_status mf_process_get_helicities(const mf_process *p, int8_t *hel, int32_t *n_hel) {
    if (!p || !n_hel) return fail(MF_EINVAL, "NULL argument");
    *n_hel = (int32_t)(p->hel.size() / p->n_legs);
    if (hel) std::copy(p->hel.begin(), p->hel.end(), hel);
    return MF_OK;
}

extern "C" mf_status mf_process_check(mf_process *p) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    int flag = 0;
    MF_CUDA(cudaDeviceSynchronize());
    MF_CUDA(cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return flag_status(p, flag, true);
}

extern "C" mf_status mf_integrand(mf_process *p, const double *x, int64_t n, double *f, mf_precision prec,
                                  void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (n < 0) return fail(MF_EINVAL, "negative n");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (n == 0) return MF_OK;
    if (!x || !f) return fail(MF_EINVAL, "NULL x or f");
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    mf_kparams kp;
    fill_common(*p, kp);
    set_hel(kp, p->hel, p->n_legs);
    kp.mode = 0;
    kp.n = n;
    kp.x = x;
    kp.f = f;
    return launch(p, prec, kp, (cudaStream_t)stream);
}

extern "C" mf_status mf_helicity_msq(mf_process *p, const double *x, int64_t n, double *out, mf_precision prec,
                                     void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (n < 0) return fail(MF_EINVAL, "negative n");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (n == 0) return MF_OK;
    if (!x || !out) return fail(MF_EINVAL, "NULL x or out");
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    mf_kparams kp;
    fill_common(*p, kp);
    set_hel(kp, p->hel_all, p->n_legs);
    kp.mode = 2;
    kp.variant = 0;                       // per-helicity values: the integrand kernel
    kp.hel_sample = 0;
    kp.n = n;
    kp.x = x;
    kp.f = out;
    return launch(p, prec, kp, (cudaStream_t)stream);
}

namespace {
mf_status grad_impl(mf_process *p, int32_t channel, const double *x, int64_t n, double *f, double *df_dparam,
                    double *df_dx, void *stream);
}  // namespace

extern "C" mf_status mf_grad(mf_process *p, const double *x, int64_t n, double *f, double *df_dparam,
                             double *df_dx, void *stream) {
    return grad_impl(p, -1, x, n, f, df_dparam, df_dx, stream);
}

extern "C" mf_status mf_grad_channel(mf_process *p, int32_t channel, const double *x, int64_t n, double *f,
                                     double *df_dparam, double *df_dx, void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (p->channels.K == 0) return fail(MF_EUNSUPPORTED, "the process has no phase-space channels");
    if (channel < 0 || channel >= p->channels.K) return fail(MF_EINVAL, "channel out of range");
    return grad_impl(p, channel, x, n, f, df_dparam, df_dx, stream);
}

namespace {
mf_status grad_impl(mf_process *p, int32_t channel, const double *x, int64_t n, double *f, double *df_dparam,
                    double *df_dx, void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (n < 0) return fail(MF_EINVAL, "negative n");
    if (n == 0) return MF_OK;
    if (!x || !f || !df_dparam) return fail(MF_EINVAL, "NULL x, f or df_dparam");
    mf_status st = compile_grad(p);
    if (st != MF_OK) return st;
    mf_kparams kp;
    fill_common(*p, kp);
    set_hel(kp, p->hel, p->n_legs);
    kp.mode = 0;
    kp.n = n;
    kp.x = x;
    kp.f = f;
    kp.g_dparam = df_dparam;
    kp.g_dx = df_dx;
    kp.variant = 0;                       // the gradient always sums the colours
    kp.colour_sample = 0;
    kp.channel = channel;
    return launch(p, 2, kp, (cudaStream_t)stream);
}
}  // namespace

// ----------------------------------------------------------------------------
// Vegas
// ----------------------------------------------------------------------------
namespace {

// The pairwise tree over the chunks of one iteration (host side; the device
// side is vegas_tree_kernel, which performs the same additions).
int tree_levels(int64_t nchunks) {
    int L = 0;
    while (((int64_t)1 << L) < nchunks) ++L;
    return L;
}

// Maximal aligned nodes covering chunks [c0, c1); the shard that ends at the
// last chunk also owns the tree's truncated right edge.
void tree_frontier(int64_t c0, int64_t c1, int64_t nchunks, std::vector<int64_t> &ids) {
    ids.clear();
    const int L = tree_levels(nchunks);
    const int64_t hi = c1 >= nchunks ? ((int64_t)1 << L) : c1;
    int64_t c = c0;
    while (c < hi) {
        int l = 0;
        while (l < L && c % ((int64_t)2 << l) == 0 && c + ((int64_t)2 << l) <= hi) ++l;
        if (c < nchunks) {
            ids.push_back(l);
            ids.push_back(c >> l);
        }
        c += (int64_t)1 << l;
    }
}

// Combine nodes (records [level, index, K values]) that partition the chunks
// of node (level, index) into that node's K values.
mf_status tree_reduce(const double *nodes, int n_nodes, int K, int64_t nchunks, int level, int64_t index,
                      double *out) {
    using Key = std::pair<int, int64_t>;
    std::map<Key, std::vector<double>> cur;
    for (int j = 0; j < n_nodes; ++j) {
        const double *r = nodes + (size_t)j * (2 + K);
        const int l = (int)r[0];
        const int64_t i = (int64_t)r[1];
        if (r[0] != (double)l || r[1] != (double)i || l < 0 || l > kTreeMaxLevel || i < 0)
            return fail(MF_EINVAL, "malformed tree node");
        if ((i << l) >= nchunks) return fail(MF_EINVAL, "tree node beyond the last chunk");
        if (l > level || (i >> (level - l)) != index) return fail(MF_EINVAL, "tree node outside the target node");
        if (!cur.emplace(Key(l, i), std::vector<double>(r + 2, r + 2 + K)).second)
            return fail(MF_EINVAL, "duplicate tree node");
    }
    for (int l = 0; l < level; ++l) {
        std::vector<std::pair<Key, std::vector<double>>> made;
        for (auto it = cur.begin(); it != cur.end() && it->first.first == l; ++it) {
            const int64_t i = it->first.second;
            if (i & 1) {
                if (!cur.count(Key(l, i - 1))) return fail(MF_EINVAL, "tree nodes do not cover the range");
                continue;
            }
            auto sib = cur.find(Key(l, i + 1));
            std::vector<double> v = it->second;
            if (sib != cur.end()) {
                for (int k = 0; k < K; ++k) v[k] = v[k] + sib->second[k];
            } else if (((i + 1) << l) < nchunks) {
                return fail(MF_EINVAL, "tree nodes do not cover the range");
            }
            made.emplace_back(Key(l + 1, i >> 1), std::move(v));
        }
        cur.erase(cur.begin(), cur.lower_bound(Key(l + 1, 0)));
        for (auto &m : made)
            if (!cur.emplace(m.first, std::move(m.second)).second) return fail(MF_EINVAL, "overlapping tree nodes");
    }
    auto root = cur.find(Key(level, index));
    if (root == cur.end() || cur.size() != 1) return fail(MF_EINVAL, "tree nodes do not cover the range");
    std::copy(root->second.begin(), root->second.end(), out);
    return MF_OK;
}

int partial_size(const mf_vegas *v) { return 4 + 2 * v->ndim * v->nbins; }

// Process scratch (w, bins) for n points and grid slots for their chunks.
mf_status ensure_slots(mf_vegas *v, int64_t n);

mf_status ensure_scratch(mf_process *p, mf_vegas *v, int64_t n) {
    if (p->scratch_n < n) {
        cudaFree(p->d_w);
        cudaFree(p->d_bins);
        p->d_w = nullptr;
        p->d_bins = nullptr;
        p->scratch_n = 0;
        MF_CUDA(mfi::dev_malloc(&p->d_w, sizeof(double) * n));
        MF_CUDA(mfi::dev_malloc(&p->d_bins, (size_t)p->ndim * n));
        p->scratch_n = n;
    }
    if (v) {
        mf_status st = ensure_slots(v, n);
        if (st != MF_OK) return st;
    }
    if (!p->ev_start) {
        MF_CUDA(cudaEventCreate(&p->ev_start));
        MF_CUDA(cudaEventCreate(&p->ev_stop));
    }
    return MF_OK;
}

// Chunk slots of a grid for an iteration of n points.
mf_status ensure_slots(mf_vegas *v, int64_t n) {
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    const int K = partial_size(v);
    if (v->slots_cap < nchunks * K + K) {
        cudaFree(v->d_slots);
        v->d_slots = nullptr;
        v->slots_cap = 0;
        MF_CUDA(mfi::dev_malloc(&v->d_slots, sizeof(double) * (nchunks * K + K)));
        v->slots_cap = nchunks * K + K;
    }
    return MF_OK;
}

// Parameters of the Vegas-mode kernel for points [ev0, ev0 + n).
void vegas_params(const mf_process *p, const mf_vegas *v, int64_t n, int64_t ev0, int subprocess, uint64_t seed,
                  mf_kparams &kp) {
    fill_common(*p, kp);
    set_hel(kp, p->hel, p->n_legs);
    kp.mode = 1;
    kp.n = n;
    kp.ev0 = ev0;
    kp.grid = v->d_grid;
    kp.nb = v->nbins;
    kp.w_out = p->d_w;
    kp.bins_out = p->d_bins;
    kp.seed = seed;
    kp.iteration = (uint64_t)v->iteration;
    kp.subprocess = (uint64_t)subprocess;
}

// Dynamic shared memory of vegas_accumulate_kernel and
// vegas_accumulate_channels_kernel (one chunk's w and w^2), and their
// attribute, set once per device.
constexpr size_t kAccSmem = sizeof(double) * 2 * kChunk;
constexpr int kAccMaxDevices = 64;
std::mutex g_acc_mutex;
bool g_acc_attr[kAccMaxDevices];

mf_status accumulate_attribute() {
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kAccMaxDevices) return fail(MF_EUNSUPPORTED, "device index beyond the attribute table");
    std::lock_guard<std::mutex> lock(g_acc_mutex);
    if (!g_acc_attr[dev]) {
        MF_CUDA(cudaFuncSetAttribute(vegas_accumulate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kAccSmem));
        MF_CUDA(cudaFuncSetAttribute(vegas_accumulate_channels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kAccSmem));
        g_acc_attr[dev] = true;
    }
    return MF_OK;
}

// Chunk partial sums of n points (w, bins) into slots [K][nchunks].
mf_status accumulate_into(const double *w, const uint8_t *bins, int64_t n, const mf_vegas *v, double *slots,
                          cudaStream_t s) {
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    mf_status st = accumulate_attribute();
    if (st != MF_OK) return st;
    vegas_accumulate_kernel<<<(unsigned)nchunks, kAccThreads, kAccSmem, s>>>(w, bins, n, v->ndim, v->nbins, slots,
                                                                              nchunks);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// Chunk partial sums of the process scratch's n points into v->d_slots.
mf_status accumulate(mf_process *p, mf_vegas *v, int64_t n, cudaStream_t s) {
    return accumulate_into(p->d_w, p->d_bins, n, v, v->d_slots, s);
}

// Evaluate points [ev0, ev0 + n) of iteration v->iteration into the process
// scratch (w, bins) and accumulate their chunks into v->d_slots.
mf_status run_points(mf_process *p, mf_vegas *v, int prec, int64_t n, int64_t ev0, int subprocess, uint64_t seed,
                     cudaStream_t s) {
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    st = ensure_scratch(p, v, n);
    if (st != MF_OK) return st;
    p->last_n = n;
    if (n == 0) return MF_OK;
    mf_kparams kp;
    vegas_params(p, v, n, ev0, subprocess, seed, kp);
    MF_CUDA(cudaEventRecord(p->ev_start, s));
    st = launch(p, prec, kp, s);
    if (st != MF_OK) return st;
    MF_CUDA(cudaEventRecord(p->ev_stop, s));
    return accumulate(p, v, n, s);
}

// Nodes ids (host, [n][2]) of the accumulated chunks -> device values [n][K].
mf_status tree_nodes(mf_vegas *v, int64_t ld, int64_t c0, int64_t nchunks, const std::vector<int64_t> &ids,
                     cudaStream_t s) {
    const int n = (int)ids.size() / 2;
    if (n == 0) return MF_OK;
    MF_CUDA(cudaMemcpyAsync(v->d_tree_ids, ids.data(), sizeof(int64_t) * ids.size(), cudaMemcpyHostToDevice, s));
    vegas_tree_kernel<<<dim3((unsigned)partial_size(v), (unsigned)n), kTreeThreads, 0, s>>>(
        v->d_slots, ld, c0, nchunks, partial_size(v), v->d_tree_ids, v->d_tree_out);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

// Iteration estimate, histogram, combination and (optionally) refinement from
// the totals tot (device [K]) of n points.
mf_status finish(mf_vegas *v, const double *tot, int64_t n, int refine, cudaStream_t s) {
    vegas_finalize_kernel<<<1, 128, 0, s>>>(tot, n, v->ndim, v->nbins, v->iteration, v->d_hist, v->d_count,
                                            v->d_hist_iter, v->d_result);
    if (refine) vegas_refine_kernel<<<1, 32, 0, s>>>(v->d_grid, v->d_hist, v->ndim, v->nbins, n, v->alpha);
    MF_CUDA(cudaGetLastError());
    return MF_OK;
}

void fill_result(mf_iter_result &o, const mf_vegas *v, int64_t n, const double *r) {
    o.iteration = v->iteration;
    o.n_events = n;
    o.integral = r[0];
    o.error = r[1];
    o.sigma = r[2];
    o.sigma_error = r[3];
    o.chi2_dof = r[4];
    o.n_nonzero = (int64_t)r[5];
    o.n_nan = (int64_t)r[6];
}

}  // namespace

extern "C" mf_status mf_vegas_create(int32_t ndim, int32_t nbins, double alpha, mf_vegas **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (ndim < 1 || ndim > MF_MAX_DIM) return fail(MF_EINVAL, "ndim out of range");
    if (nbins < 2 || nbins > 64) return fail(MF_EINVAL, "nbins must be in [2, 64]");
    if (!(alpha >= 0.0)) return fail(MF_EINVAL, "alpha must be non-negative");
    mf_status st = ensure_context();
    if (st != MF_OK) return st;
    mf_vegas *v = new (std::nothrow) mf_vegas();
    if (!v) return fail(MF_ENOMEM, "host allocation");
    cudaGetDevice(&v->device);
    v->ndim = ndim;
    v->nbins = nbins;
    v->alpha = alpha;
    v->max_iter = MF_MAX_ITER;
    const int K = partial_size(v);
    if (mfi::dev_malloc(&v->d_grid, sizeof(double) * ndim * (nbins + 1)) != cudaSuccess ||
        mfi::dev_malloc(&v->d_hist, sizeof(double) * ndim * nbins) != cudaSuccess ||
        mfi::dev_malloc(&v->d_count, sizeof(long long) * ndim * nbins) != cudaSuccess ||
        mfi::dev_malloc(&v->d_hist_iter, sizeof(double) * 2 * v->max_iter) != cudaSuccess ||
        mfi::dev_malloc(&v->d_result, sizeof(double) * 8) != cudaSuccess ||
        mfi::dev_malloc(&v->d_tree_ids, sizeof(int64_t) * 2 * MF_MAX_TREE_NODES) != cudaSuccess ||
        mfi::dev_malloc(&v->d_tree_out, sizeof(double) * (size_t)K * MF_MAX_TREE_NODES) != cudaSuccess ||
        mfi::dev_malloc(&v->d_tot, sizeof(double) * K) != cudaSuccess) {
        mf_vegas_destroy(v);
        return fail(MF_ENOMEM, "Vegas grid");
    }
    std::vector<double> g((size_t)ndim * (nbins + 1));
    for (int j = 0; j < ndim; ++j)
        for (int i = 0; i <= nbins; ++i) g[(size_t)j * (nbins + 1) + i] = (double)i / nbins;
    cudaMemcpy(v->d_grid, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice);
    cudaMemset(v->d_hist, 0, sizeof(double) * ndim * nbins);
    cudaMemset(v->d_count, 0, sizeof(long long) * ndim * nbins);
    *out = v;
    return MF_OK;
}

extern "C" mf_status mf_vegas_destroy(mf_vegas *v) {
    if (!v) return MF_OK;
    cudaFree(v->d_grid);
    cudaFree(v->d_hist);
    cudaFree(v->d_count);
    cudaFree(v->d_hist_iter);
    cudaFree(v->d_result);
    cudaFree(v->d_slots);
    cudaFree(v->d_tree_ids);
    cudaFree(v->d_tree_out);
    cudaFree(v->d_tot);
    delete v;
    return MF_OK;
}

extern "C" mf_status mf_vegas_get_grid(const mf_vegas *v, double *edges) {
    if (!v || !edges) return fail(MF_EINVAL, "NULL argument");
    MF_CUDA(cudaMemcpy(edges, v->d_grid, sizeof(double) * v->ndim * (v->nbins + 1), cudaMemcpyDeviceToHost));
    return MF_OK;
}

namespace {
mf_status check_edges(const mf_vegas *v, const double *edges) {
    for (int j = 0; j < v->ndim; ++j) {
        const double *g = edges + (size_t)j * (v->nbins + 1);
        if (g[0] != 0.0 || g[v->nbins] != 1.0) return fail(MF_EINVAL, "grid edges must run from 0 to 1");
        for (int i = 0; i < v->nbins; ++i)
            if (!(g[i + 1] > g[i])) return fail(MF_EINVAL, "grid edges must increase");
    }
    return MF_OK;
}
}  // namespace

extern "C" mf_status mf_vegas_set_grid(mf_vegas *v, const double *edges) {
    if (!v || !edges) return fail(MF_EINVAL, "NULL argument");
    mf_status st = check_edges(v, edges);
    if (st != MF_OK) return st;
    MF_CUDA(cudaMemcpy(v->d_grid, edges, sizeof(double) * v->ndim * (v->nbins + 1), cudaMemcpyHostToDevice));
    return MF_OK;
}

extern "C" mf_status mf_vegas_get_histogram(const mf_vegas *v, double *sum_w2, int64_t *counts) {
    if (!v) return fail(MF_EINVAL, "NULL argument");
    if (sum_w2) MF_CUDA(cudaMemcpy(sum_w2, v->d_hist, sizeof(double) * v->ndim * v->nbins, cudaMemcpyDeviceToHost));
    if (counts) MF_CUDA(cudaMemcpy(counts, v->d_count, sizeof(long long) * v->ndim * v->nbins, cudaMemcpyDeviceToHost));
    return MF_OK;
}

extern "C" mf_status mf_vegas_get_shape(const mf_vegas *v, int32_t *ndim, int32_t *nbins, int32_t *iteration) {
    if (!v) return fail(MF_EINVAL, "NULL argument");
    if (ndim) *ndim = v->ndim;
    if (nbins) *nbins = v->nbins;
    if (iteration) *iteration = v->iteration;
    return MF_OK;
}

extern "C" mf_status mf_vegas_iterate(mf_vegas *const *grids, mf_process *const *procs, const int64_t *n_events,
                                      int32_t nproc, uint64_t seed, mf_precision prec, int32_t refine,
                                      mf_iter_result *out, void *stream) {
    if (nproc < 1 || !grids || !procs || !n_events || !out) return fail(MF_EINVAL, "bad arguments");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < nproc; ++k) {
        if (!grids[k] || !procs[k]) return fail(MF_EINVAL, "NULL grid or process");
        if (grids[k]->ndim != procs[k]->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
        if (n_events[k] < 2) return fail(MF_EINVAL, "need at least two events per iteration");
        if ((n_events[k] + kChunk - 1) / kChunk > ((int64_t)1 << kTreeMaxLevel))
            return fail(MF_EINVAL, "too many events per iteration");
        if (grids[k]->iteration >= grids[k]->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
        for (int q = 0; q < k; ++q)
            if (grids[q] == grids[k]) return fail(MF_EINVAL, "a grid appears twice");
    }
    std::vector<std::vector<double>> res(nproc, std::vector<double>(8));
    std::vector<int> flags(nproc, 0);
    for (int k = 0; k < nproc; ++k) {
        mf_process *p = procs[k];
        mf_vegas *v = grids[k];
        const int64_t n = n_events[k];
        mf_status st = run_points(p, v, prec, n, 0, k, seed, s);
        if (st != MF_OK) return st;
        // the whole chunk range is the root node of the tree
        const int64_t nchunks = (n + kChunk - 1) / kChunk;
        const std::vector<int64_t> root = {tree_levels(nchunks), 0};
        st = tree_nodes(v, nchunks, 0, nchunks, root, s);
        if (st != MF_OK) return st;
        st = finish(v, v->d_tree_out, n, refine, s);
        if (st != MF_OK) return st;
        MF_CUDA(cudaMemcpyAsync(res[k].data(), v->d_result, sizeof(double) * 7, cudaMemcpyDeviceToHost, s));
        MF_CUDA(cudaMemcpyAsync(&flags[k], p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    MF_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nproc; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, procs[k]->ev_start, procs[k]->ev_stop) == cudaSuccess)
            procs[k]->last_kernel_ms = ms;
    }
    for (int k = 0; k < nproc; ++k) {
        mf_status st = flag_status(procs[k], flags[k]);
        if (st != MF_OK) return st;
    }
    bool any_nan = false;
    for (int k = 0; k < nproc; ++k) {
        fill_result(out[k], grids[k], n_events[k], res[k].data());
        any_nan |= out[k].n_nan > 0;
        grids[k]->iteration += 1;
    }
    if (any_nan) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}

extern "C" mf_status mf_process_channels(const mf_process *p, int32_t *n_channels) {
    if (!p || !n_channels) return fail(MF_EINVAL, "NULL argument");
    *n_channels = p->channels.K;
    return MF_OK;
}

extern "C" mf_status mf_process_set_channel_regulators(mf_process *p, double s0, double t0) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (!(s0 > 0.0) || !(t0 > 0.0) || !std::isfinite(s0) || !std::isfinite(t0))
        return fail(MF_EINVAL, "regulators must be positive and finite");
    p->ch_s0 = s0;
    p->ch_t0 = t0;
    return MF_OK;
}

extern "C" mf_status mf_channel_integrand(mf_process *p, int32_t channel, const double *x, int64_t n, double *f,
                                          mf_precision prec, void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (p->channels.K == 0) return fail(MF_EUNSUPPORTED, "the process has no phase-space channels");
    if (channel < 0 || channel >= p->channels.K) return fail(MF_EINVAL, "channel out of range");
    if (n < 0) return fail(MF_EINVAL, "negative n");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (n == 0) return MF_OK;
    if (!x || !f) return fail(MF_EINVAL, "NULL x or f");
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    mf_kparams kp;
    fill_common(*p, kp);
    set_hel(kp, p->hel, p->n_legs);
    kp.mode = 0;
    kp.n = n;
    kp.x = x;
    kp.f = f;
    kp.channel = channel;
    return launch(p, prec, kp, (cudaStream_t)stream);
}

extern "C" mf_status mf_vegas_iterate_channels(mf_vegas *const *grids, mf_process *p, const int64_t *n_events,
                                               int32_t n_channels, uint64_t seed, mf_precision prec, int32_t refine,
                                               mf_iter_result *out, void *stream) {
    if (!grids || !p || !n_events || !out) return fail(MF_EINVAL, "bad arguments");
    if (p->channels.K == 0) return fail(MF_EUNSUPPORTED, "the process has no phase-space channels");
    if (n_channels != p->channels.K) return fail(MF_EINVAL, "one grid per channel of the process");
    if (n_channels > 65535) return fail(MF_EUNSUPPORTED, "more channels than one launch's grid rows");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < n_channels; ++k) {
        if (!grids[k]) return fail(MF_EINVAL, "NULL grid");
        if (grids[k]->ndim != p->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
        if (n_events[k] < 2) return fail(MF_EINVAL, "need at least two events per channel");
        if ((n_events[k] + kChunk - 1) / kChunk > ((int64_t)1 << kTreeMaxLevel))
            return fail(MF_EINVAL, "too many events per iteration");
        if (grids[k]->iteration >= grids[k]->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
    }
    {
        // every grid once (a sorted copy: n_channels can be in the hundreds)
        std::vector<const mf_vegas *> g(grids, grids + n_channels);
        std::sort(g.begin(), g.end());
        if (std::adjacent_find(g.begin(), g.end()) != g.end()) return fail(MF_EINVAL, "a grid appears twice");
    }
    for (int k = 1; k < n_channels; ++k)
        if (grids[k]->nbins != grids[0]->nbins || grids[k]->iteration != grids[0]->iteration)
            return fail(MF_EINVAL, "the channels' grids differ in bins or iteration");
    // one launch over every channel's points: channel k takes points
    // [off[k], off[k+1]) of the launch, as points 0.. of its own stream
    std::vector<long long> off(n_channels + 1, 0);
    std::vector<const double *> gptr(n_channels);
    for (int k = 0; k < n_channels; ++k) {
        off[k + 1] = off[k] + n_events[k];
        gptr[k] = grids[k]->d_grid;
    }
    const int64_t N = off[n_channels];
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    st = ensure_scratch(p, nullptr, N);
    if (st != MF_OK) return st;
    for (int k = 0; k < n_channels; ++k) {
        st = ensure_slots(grids[k], n_events[k]);
        if (st != MF_OK) return st;
    }
    // per-process buffers of the channel launches (K is fixed per process)
    if (!p->d_ch_off) MF_CUDA(mfi::dev_malloc(&p->d_ch_off, sizeof(long long) * (n_channels + 1)));
    if (!p->d_ch_grids) MF_CUDA(mfi::dev_malloc(&p->d_ch_grids, sizeof(double *) * n_channels));
    if (!p->d_ch_chunk_off) MF_CUDA(mfi::dev_malloc(&p->d_ch_chunk_off, sizeof(long long) * (n_channels + 1)));
    if (!p->d_ch_res) MF_CUDA(mfi::dev_malloc(&p->d_ch_res, sizeof(double) * 8 * n_channels));
    if (!p->d_ch_acc) MF_CUDA(mfi::dev_malloc(&p->d_ch_acc, sizeof(ChanAcc) * n_channels));
    // pageable sources: the copies are staged before the calls return
    MF_CUDA(cudaMemcpyAsync(p->d_ch_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, s));
    MF_CUDA(cudaMemcpyAsync(p->d_ch_grids, gptr.data(), sizeof(double *) * gptr.size(), cudaMemcpyHostToDevice, s));
    p->last_n = N;
    mf_kparams kp;
    vegas_params(p, grids[0], N, 0, 0, seed, kp);
    kp.grid = nullptr;
    kp.ch_off = p->d_ch_off;
    kp.ch_grids = p->d_ch_grids;
    kp.ch_count = n_channels;
    MF_CUDA(cudaEventRecord(p->ev_start, s));
    st = launch(p, prec, kp, s);
    if (st != MF_OK) return st;
    MF_CUDA(cudaEventRecord(p->ev_stop, s));
    // the channels' bookkeeping, four launches for all of them: chunk
    // partial sums, each channel's root of the chunk tree, finalisation and
    // refinement (the same arithmetic as the one-grid kernels)
    std::vector<ChanAcc> ca(n_channels);
    std::vector<long long> chunk_off(n_channels + 1, 0);
    for (int k = 0; k < n_channels; ++k) {
        mf_vegas *v = grids[k];
        const long long nch = (n_events[k] + kChunk - 1) / kChunk;
        chunk_off[k + 1] = chunk_off[k] + nch;
        ChanAcc &c = ca[k];
        c.w = p->d_w + off[k];
        c.bins = p->d_bins + off[k] * p->ndim;
        c.n = n_events[k];
        c.nchunks = nch;
        c.level = tree_levels(nch);
        c.iteration = v->iteration;
        // a grid refined on a few points per bin chases the few points that
        // landed (and forgets the rest): a channel's grid adapts only from
        // kChannelRefinePerBin points per bin on
        c.refine = refine && n_events[k] >= (int64_t)kChannelRefinePerBin * v->nbins ? 1 : 0;
        c.pad = 0;
        c.alpha = v->alpha;
        c.slots = v->d_slots;
        c.tree_out = v->d_tree_out;
        c.hist = v->d_hist;
        c.hist_iter = v->d_hist_iter;
        c.result = v->d_result;
        c.grid = v->d_grid;
        c.count = v->d_count;
        c.result_copy = p->d_ch_res + (size_t)k * 8;
    }
    MF_CUDA(cudaMemcpyAsync(p->d_ch_acc, ca.data(), sizeof(ChanAcc) * n_channels, cudaMemcpyHostToDevice, s));
    MF_CUDA(cudaMemcpyAsync(p->d_ch_chunk_off, chunk_off.data(), sizeof(long long) * (n_channels + 1),
                            cudaMemcpyHostToDevice, s));
    const ChanAcc *d_ca = static_cast<const ChanAcc *>(p->d_ch_acc);
    st = accumulate_attribute();
    if (st != MF_OK) return st;
    const int nb = grids[0]->nbins, Kp = partial_size(grids[0]);
    vegas_accumulate_channels_kernel<<<(unsigned)chunk_off[n_channels], kAccThreads, kAccSmem, s>>>(
        d_ca, p->d_ch_chunk_off, n_channels, p->ndim, nb);
    vegas_tree_channels_kernel<<<dim3((unsigned)Kp, (unsigned)n_channels), kTreeThreads, 0, s>>>(d_ca, Kp);
    vegas_finalize_channels_kernel<<<(unsigned)n_channels, 128, 0, s>>>(d_ca, p->ndim, nb);
    if (refine) vegas_refine_channels_kernel<<<(unsigned)n_channels, 32, 0, s>>>(d_ca, p->ndim, nb);
    MF_CUDA(cudaGetLastError());
    std::vector<double> res((size_t)n_channels * 8);
    int flag = 0;
    MF_CUDA(cudaMemcpyAsync(res.data(), p->d_ch_res, sizeof(double) * 8 * n_channels, cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev_start, p->ev_stop) == cudaSuccess) p->last_kernel_ms = ms;
    st = flag_status(p, flag);
    if (st != MF_OK) return st;
    bool any_nan = false;
    for (int k = 0; k < n_channels; ++k) {
        fill_result(out[k], grids[k], n_events[k], &res[(size_t)k * 8]);
        any_nan |= out[k].n_nan > 0;
        grids[k]->iteration += 1;
    }
    if (any_nan) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}

extern "C" mf_status mf_vegas_partial_size(const mf_vegas *v, int32_t *K) {
    if (!v || !K) return fail(MF_EINVAL, "NULL argument");
    *K = partial_size(v);
    return MF_OK;
}

extern "C" mf_status mf_vegas_shard_accumulate(mf_vegas *v, mf_process *p, int64_t n_total, int64_t chunk_begin,
                                               int64_t chunk_end, int32_t subprocess, uint64_t seed,
                                               mf_precision prec, double *nodes, int32_t *n_nodes, void *stream) {
    if (!v || !p || !nodes || !n_nodes) return fail(MF_EINVAL, "NULL argument");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (v->ndim != p->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
    if (n_total < 2) return fail(MF_EINVAL, "need at least two events per iteration");
    const int64_t nchunks = (n_total + kChunk - 1) / kChunk;
    if (nchunks > ((int64_t)1 << kTreeMaxLevel)) return fail(MF_EINVAL, "too many events per iteration");
    if (chunk_begin < 0 || chunk_end < chunk_begin || chunk_end > nchunks) return fail(MF_EINVAL, "bad chunk range");
    if (subprocess < 0) return fail(MF_EINVAL, "bad subprocess index");
    if (v->iteration >= v->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t e0 = chunk_begin * kChunk;
    const int64_t e1 = std::min(chunk_end * kChunk, n_total);
    const int64_t n = e1 > e0 ? e1 - e0 : 0;
    mf_status st = run_points(p, v, prec, n, e0, subprocess, seed, s);
    if (st != MF_OK) return st;
    std::vector<int64_t> ids;
    tree_frontier(chunk_begin, chunk_end, nchunks, ids);
    const int nn = (int)ids.size() / 2;
    if (nn > MF_MAX_TREE_NODES) return fail(MF_EUNSUPPORTED, "too many tree nodes");
    st = tree_nodes(v, (n + kChunk - 1) / kChunk, chunk_begin, nchunks, ids, s);
    if (st != MF_OK) return st;
    const int K = partial_size(v);
    std::vector<double> vals((size_t)nn * K);
    if (nn) MF_CUDA(cudaMemcpyAsync(vals.data(), v->d_tree_out, sizeof(double) * vals.size(), cudaMemcpyDeviceToHost, s));
    int flag = 0;
    MF_CUDA(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    st = flag_status(p, flag);
    if (st != MF_OK) return st;
    if (n > 0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev_start, p->ev_stop) == cudaSuccess) p->last_kernel_ms = ms;
    }
    for (int j = 0; j < nn; ++j) {
        double *r = nodes + (size_t)j * (2 + K);
        r[0] = (double)ids[2 * j];
        r[1] = (double)ids[2 * j + 1];
        std::copy(vals.begin() + (size_t)j * K, vals.begin() + (size_t)(j + 1) * K, r + 2);
    }
    *n_nodes = nn;
    return MF_OK;
}

extern "C" mf_status mf_vegas_shard_finish(mf_vegas *v, int64_t n_total, const double *nodes, int32_t n_nodes,
                                           int32_t refine, mf_iter_result *out, void *stream) {
    if (!v || !out || (n_nodes > 0 && !nodes) || n_nodes < 0) return fail(MF_EINVAL, "bad arguments");
    if (n_total < 2) return fail(MF_EINVAL, "need at least two events per iteration");
    if (v->iteration >= v->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
    const int64_t nchunks = (n_total + kChunk - 1) / kChunk;
    if (nchunks > ((int64_t)1 << kTreeMaxLevel)) return fail(MF_EINVAL, "too many events per iteration");
    const int K = partial_size(v);
    std::vector<double> tot(K);
    mf_status st = tree_reduce(nodes, n_nodes, K, nchunks, tree_levels(nchunks), 0, tot.data());
    if (st != MF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    MF_CUDA(cudaMemcpyAsync(v->d_tot, tot.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    st = finish(v, v->d_tot, n_total, refine, s);
    if (st != MF_OK) return st;
    double r[8];
    MF_CUDA(cudaMemcpyAsync(r, v->d_result, sizeof(double) * 7, cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    fill_result(*out, v, n_total, r);
    v->iteration += 1;
    if (out->n_nan > 0) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}

extern "C" mf_status mf_tree_frontier(int64_t chunk_begin, int64_t chunk_end, int64_t nchunks, int64_t *ids,
                                      int32_t capacity, int32_t *n) {
    if (!n || (capacity > 0 && !ids)) return fail(MF_EINVAL, "NULL argument");
    if (nchunks < 1 || nchunks > ((int64_t)1 << kTreeMaxLevel)) return fail(MF_EINVAL, "chunk count out of range");
    if (chunk_begin < 0 || chunk_end < chunk_begin || chunk_end > nchunks) return fail(MF_EINVAL, "bad chunk range");
    std::vector<int64_t> v;
    tree_frontier(chunk_begin, chunk_end, nchunks, v);
    *n = (int32_t)(v.size() / 2);
    if ((int64_t)v.size() > 2 * (int64_t)capacity) return fail(MF_EINVAL, "capacity too small");
    std::copy(v.begin(), v.end(), ids);
    return MF_OK;
}

extern "C" mf_status mf_tree_reduce(const double *nodes, int32_t n_nodes, int32_t K, int64_t nchunks, int32_t level,
                                    int64_t index, double *out) {
    if (!out || (n_nodes > 0 && !nodes) || n_nodes < 0 || K < 1) return fail(MF_EINVAL, "bad arguments");
    if (nchunks < 1 || nchunks > ((int64_t)1 << kTreeMaxLevel)) return fail(MF_EINVAL, "chunk count out of range");
    if (level < 0 || level > kTreeMaxLevel || index < 0 || (index << level) >= nchunks)
        return fail(MF_EINVAL, "target node does not exist");
    return tree_reduce(nodes, n_nodes, K, nchunks, level, index, out);
}

// ----------------------------------------------------------------------------
// Launch-shape tuner: the helicity sum is a fixed pairwise tree whatever the
// lanes per event, and no event's arithmetic depends on the block size, so
// every shape gives the same bits and the fastest one can be kept.
// ----------------------------------------------------------------------------
extern "C" mf_status mf_process_tune(mf_process *p, mf_precision prec, int64_t n_sample, void *stream, int32_t *block,
                                     int32_t *ht) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (n_sample < 1024 || n_sample > ((int64_t)1 << 30)) return fail(MF_EINVAL, "n_sample out of range");
    cudaStream_t s = (cudaStream_t)stream;
    mf_vegas *v = nullptr;
    mf_status st = mf_vegas_create(p->ndim, 50, 1.5, &v);
    if (st != MF_OK) return st;
    // each shape is timed on a whole number of rounds of its resident grid
    // (at least one), so that no shape is favoured by a partial last round
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n_cap = std::max<int64_t>(n_sample, (int64_t)nsm * 2048);
    st = ensure_scratch(p, v, n_cap);
    cudaEvent_t a = nullptr, b = nullptr;
    if (st == MF_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
        st = fail(MF_ECUDA, "events");
    const int nhp = lane_units(p);
    float best_ms = 0.f;
    mfi::Compiled best;
    // stage 1: block size x lanes per point; stage 2: a minimum of resident
    // blocks per SM (fewer registers, more warps) for the best of stage 1
    std::vector<std::array<int, 3>> shapes;
    for (int bl : {128, 256}) {
        if (prec == MF_MIXED_TC && bl != 128) continue;      // one MMA row per thread of 128
        for (int h : {8, 16, 32}) {
            if (h > nhp && h != 8) continue;
            shapes.push_back({bl, h <= nhp ? h : nhp, -1});
        }
    }
    const size_t n_stage1 = shapes.size();
    for (size_t si = 0; si <= shapes.size(); ++si) {
        if (si == n_stage1 && best.fn && best.min_blocks < 0)
            for (int mb : {3, 4}) shapes.push_back({best.block, best.ht, mb});
        if (si == shapes.size()) break;
        {
            const int bl = shapes[si][0], hh = shapes[si][1], mb = shapes[si][2];
            if (st != MF_OK) break;
            if (mb > 0 && bl * mb > 1024) continue;
            mfi::Compiled k;
            st = compile_shape(p, prec, bl, hh, k, mb);
            if (st != MF_OK) break;
            const int64_t round = (int64_t)nsm * std::max(k.max_blocks_per_sm, 1) * k.block;
            const int64_t n_shape = std::min(n_cap, std::max<int64_t>(1, n_sample / round) * round);
            mf_kparams kp;
            vegas_params(p, v, n_shape, 0, 0, 12345, kp);
            float ms = 1e30f;
            mfi::Compiled saved = p->kern[prec];
            p->kern[prec] = k;
            for (int rep = 0; rep < 3 && st == MF_OK; ++rep) {
                if (cudaEventRecord(a, s) != cudaSuccess) st = fail(MF_ECUDA, "event");
                if (st == MF_OK) st = launch(p, prec, kp, s);
                if (st == MF_OK && cudaEventRecord(b, s) != cudaSuccess) st = fail(MF_ECUDA, "event");
                if (st == MF_OK && cudaEventSynchronize(b) != cudaSuccess) st = fail(MF_ECUDA, "tuning launch failed");
                float t = 0.f;
                if (st == MF_OK && rep > 0 && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms = std::min(ms, t);
            }
            ms /= (float)n_shape;                               // time per point
            p->kern[prec] = saved;
            if (st != MF_OK) {
                mfi::unload_kernel(k);
                break;
            }
            if (!best.fn || ms < best_ms) {
                if (best.fn) mfi::unload_kernel(best);
                best = k;
                best_ms = ms;
            } else {
                mfi::unload_kernel(k);
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    mf_vegas_destroy(v);
    if (st != MF_OK) {
        if (best.fn) mfi::unload_kernel(best);
        return st;
    }
    mfi::unload_kernel(p->kern[prec]);
    p->kern[prec] = best;
    // the generated source and counts of the kept shape
    mfi::GenInfo info;
    p->source[prec] = mfi::generate_source(*p, prec, best.block, best.ht, info, "proc", true, best.min_blocks);
    p->gen = info;
    st = verify_pairs(p, prec);
    if (st != MF_OK) return st;
    if (block) *block = best.block;
    if (ht) *ht = best.ht;
    return MF_OK;
}

// ----------------------------------------------------------------------------
// Batched iteration: the subprocesses of one Vegas iteration in one
// persistent launch (tiles of every subprocess drawn from one counter, the
// costliest subprocess first, so that no SM idles while another subprocess's
// tail finishes), then the per-subprocess accumulation and refinement.
// ----------------------------------------------------------------------------
namespace {
// Work items of batch slot `slot` with n points: groups of tiles sized so
// that an item of every process costs about as much as one tile of the
// costliest (the per-item dispatch is then amortised for the cheap ones).
void set_items(const mf_batch *b, int slot, int64_t n, mf_batch_params &bp) {
    const int64_t ntiles = (n + b->kern.block - 1) / b->kern.block;
    int64_t g = (int64_t)std::llround(b->cost[b->order[0]] / std::max(b->cost[b->order[slot]], 1.0));
    g = std::max<int64_t>(1, std::min<int64_t>(g, 64));
    bp.group[slot] = g;
    bp.ntiles[slot] = ntiles;
    bp.start[slot + 1] = bp.start[slot] + (ntiles + g - 1) / g;
}
}  // namespace

extern "C" mf_status mf_batch_create(mf_process *const *procs, int32_t nproc, mf_precision prec, mf_batch **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!procs || nproc < 1 || nproc > MF_KP_MAX_BATCH) return fail(MF_EINVAL, "need 1 to 8 processes");
    if (prec == MF_MIXED_TC) return fail(MF_EUNSUPPORTED, "batches use the FP32 colour sum");
    if (prec != MF_FP64 && prec != MF_MIXED) return fail(MF_EINVAL, "bad precision");
    for (int k = 0; k < nproc; ++k) {
        if (!procs[k]) return fail(MF_EINVAL, "NULL process");
        for (int q = 0; q < k; ++q)
            if (procs[q] == procs[k]) return fail(MF_EINVAL, "a process appears twice");
    }
    std::vector<double> cost(nproc);
    std::vector<int> hts(nproc);
    for (int k = 0; k < nproc; ++k) {
        mf_status st = compile_precision(procs[k], prec);          // also fixes HT and the FLOP counts
        if (st != MF_OK) return st;
        hts[k] = procs[k]->kern[prec].ht;
        cost[k] = helicity_sum_flops(procs[k]) + procs[k]->gen.flops_kin;
    }
    mf_batch *b = new (std::nothrow) mf_batch();
    if (!b) return fail(MF_ENOMEM, "host allocation");
    cudaGetDevice(&b->device);
    b->precision = prec;
    b->procs.assign(procs, procs + nproc);
    b->cost = cost;
    b->order.resize(nproc);
    for (int k = 0; k < nproc; ++k) b->order[k] = k;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<const mf_process *> ps;
    std::vector<int> hs;
    size_t smem = 0;
    for (int slot = 0; slot < nproc; ++slot) {
        const mf_process *p = procs[b->order[slot]];
        ps.push_back(p);
        hs.push_back(hts[b->order[slot]]);
        smem = std::max(smem, smem_bytes(*p, prec, 128));
    }
    std::vector<mfi::GenInfo> infos;
    b->source = mfi::generate_batch_source(ps, prec, 128, hs, infos);
    // the batch holds the same programs: it is built at the lowest
    // device-assembler level any of its processes' kernels needed (see
    // verify_pairs)
    int level = -1;
    for (int k = 0; k < nproc; ++k) {
        const int lk = procs[k]->kern[prec].ptxas_level;
        if (lk >= 0 && (level < 0 || lk < level)) level = lk;
    }
    std::vector<char> cubin;
    mf_status st = mfi::jit_compile(b->source, prec == MF_FP64 ? "mf_batch_f64.cu" : "mf_batch_mixed.cu", cubin,
                                    level);
    if (st == MF_OK) {
        b->kern.block = 128;
        b->kern.smem = smem;
        st = mfi::load_kernel(cubin, b->kern, "mf_batch_kernel");
    }
    if (st == MF_OK && mfi::dev_malloc(&b->d_counter, sizeof(long long)) != cudaSuccess)
        st = fail(MF_ENOMEM, "batch counter");
    if (st == MF_OK && (cudaEventCreate(&b->ev_start) != cudaSuccess || cudaEventCreate(&b->ev_stop) != cudaSuccess))
        st = fail(MF_ECUDA, "batch events");
    if (st != MF_OK) {
        mf_batch_destroy(b);
        return st;
    }
    *out = b;
    return MF_OK;
}

extern "C" mf_status mf_batch_destroy(mf_batch *b) {
    if (!b) return MF_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    cudaFree(b->d_iters);
    cudaFree(b->d_root_ids);
    cudaFreeHost(b->h_iters);
    cudaFreeHost(b->h_res);
    cudaFreeHost(b->h_flags);
    mfi::unload_kernel(b->kern);
    cudaFree(b->d_counter);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_stop) cudaEventDestroy(b->ev_stop);
    delete b;
    return MF_OK;
}

extern "C" mf_status mf_batch_get_info(const mf_batch *b, int32_t *order, int32_t *regs, double *last_kernel_ms) {
    if (!b) return fail(MF_EINVAL, "NULL batch");
    if (order)
        for (size_t k = 0; k < b->order.size(); ++k) order[k] = b->order[k];
    if (regs) *regs = b->kern.regs;
    if (last_kernel_ms) *last_kernel_ms = b->last_kernel_ms;
    return MF_OK;
}

extern "C" mf_status mf_batch_iterate(mf_batch *b, mf_vegas *const *grids, const int64_t *n_events, uint64_t seed,
                                      int32_t refine, mf_iter_result *out, void *stream) {
    if (!b || !grids || !n_events || !out) return fail(MF_EINVAL, "NULL argument");
    const int nproc = (int)b->procs.size();
    for (int k = 0; k < nproc; ++k) {
        if (!grids[k]) return fail(MF_EINVAL, "NULL grid");
        if (grids[k]->ndim != b->procs[k]->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
        if (n_events[k] < 2) return fail(MF_EINVAL, "need at least two events per iteration");
        if ((n_events[k] + kChunk - 1) / kChunk > ((int64_t)1 << kTreeMaxLevel))
            return fail(MF_EINVAL, "too many events per iteration");
        if (grids[k]->iteration >= grids[k]->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
        for (int q = 0; q < k; ++q)
            if (grids[q] == grids[k]) return fail(MF_EINVAL, "a grid appears twice");
    }
    cudaStream_t s = (cudaStream_t)stream;
    mf_batch_params bp;
    std::memset(&bp, 0, sizeof bp);
    bp.counter = b->d_counter;
    bp.nproc = nproc;
    bp.start[0] = 0;
    for (int slot = 0; slot < nproc; ++slot) {
        const int u = b->order[slot];
        mf_process *p = b->procs[u];
        mf_status st = ensure_scratch(p, grids[u], n_events[u]);
        if (st != MF_OK) return st;
        vegas_params(p, grids[u], n_events[u], 0, u, seed, bp.kp[slot]);
        set_items(b, slot, n_events[u], bp);
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    int64_t grid = (int64_t)nsm * b->kern.max_blocks_per_sm;
    if (grid > bp.start[nproc]) grid = bp.start[nproc];
    MF_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(long long), s));
    MF_CUDA(cudaEventRecord(b->ev_start, s));
    void *args[] = {&bp};
    mf_status st = mfi::launch_kernel(b->kern, (unsigned)grid, args, s);
    if (st != MF_OK) return st;
    MF_CUDA(cudaEventRecord(b->ev_stop, s));
    std::vector<std::vector<double>> res(nproc, std::vector<double>(8));
    std::vector<int> flags(nproc, 0);
    for (int k = 0; k < nproc; ++k) {
        mf_process *p = b->procs[k];
        mf_vegas *v = grids[k];
        const int64_t n = n_events[k];
        st = accumulate(p, v, n, s);
        if (st != MF_OK) return st;
        const int64_t nchunks = (n + kChunk - 1) / kChunk;
        const std::vector<int64_t> root = {tree_levels(nchunks), 0};
        st = tree_nodes(v, nchunks, 0, nchunks, root, s);
        if (st != MF_OK) return st;
        st = finish(v, v->d_tree_out, n, refine, s);
        if (st != MF_OK) return st;
        MF_CUDA(cudaMemcpyAsync(res[k].data(), v->d_result, sizeof(double) * 7, cudaMemcpyDeviceToHost, s));
        MF_CUDA(cudaMemcpyAsync(&flags[k], p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    MF_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev_start, b->ev_stop) == cudaSuccess) b->last_kernel_ms = ms;
    for (int k = 0; k < nproc; ++k) {
        st = flag_status(b->procs[k], flags[k]);
        if (st != MF_OK) return st;
    }
    bool any_nan = false;
    for (int k = 0; k < nproc; ++k) {
        fill_result(out[k], grids[k], n_events[k], res[k].data());
        any_nan |= out[k].n_nan > 0;
        grids[k]->iteration += 1;
    }
    if (any_nan) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}

// One batched iteration as a CUDA graph: captured once for given grids,
// point counts, seed and refine flag, then replayed; the only per-iteration
// inputs are the grids' iteration indices, copied to the device before each
// replay (the kernels read them there).
namespace {
// Every device buffer a captured iteration touches: a graph is replayed only
// while all of them are still the ones it was captured with.
std::vector<const void *> graph_buffers(const mf_batch *b, mf_vegas *const *grids) {
    std::vector<const void *> v;
    for (size_t k = 0; k < b->procs.size(); ++k) {
        const mf_process *p = b->procs[k];
        const mf_vegas *g = grids[k];
        v.insert(v.end(), {p->d_w, p->d_bins, p->d_err, g->d_slots, g->d_tree_out, g->d_grid, g->d_hist,
                           g->d_count, g->d_hist_iter, g->d_result});
    }
    return v;
}

mf_status capture_batch(mf_batch *b, mf_vegas *const *grids, const int64_t *n_events, uint64_t seed, int refine) {
    const int nproc = (int)b->procs.size();
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!b->capture_stream) MF_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    if (!b->d_iters) {
        MF_CUDA(mfi::dev_malloc(&b->d_iters, sizeof(long long) * nproc));
        MF_CUDA(mfi::dev_malloc(&b->d_root_ids, sizeof(int64_t) * 2 * nproc));
        MF_CUDA(mfi::host_malloc(&b->h_iters, sizeof(long long) * nproc));
        MF_CUDA(mfi::host_malloc(&b->h_res, sizeof(double) * 8 * nproc));
        MF_CUDA(mfi::host_malloc(&b->h_flags, sizeof(int) * nproc));
    }
    std::vector<int64_t> roots(2 * nproc);
    for (int k = 0; k < nproc; ++k) {
        mf_status st = ensure_scratch(b->procs[k], grids[k], n_events[k]);
        if (st != MF_OK) return st;
        const int64_t nchunks = (n_events[k] + kChunk - 1) / kChunk;
        roots[2 * k] = tree_levels(nchunks);
        roots[2 * k + 1] = 0;
    }
    MF_CUDA(cudaMemcpy(b->d_root_ids, roots.data(), sizeof(int64_t) * roots.size(), cudaMemcpyHostToDevice));
    mf_status ast = accumulate_attribute();
    if (ast != MF_OK) return ast;
    mf_batch_params bp;
    std::memset(&bp, 0, sizeof bp);
    bp.counter = b->d_counter;
    bp.nproc = nproc;
    for (int slot = 0; slot < nproc; ++slot) {
        const int u = b->order[slot];
        vegas_params(b->procs[u], grids[u], n_events[u], 0, u, seed, bp.kp[slot]);
        bp.kp[slot].iter_dev = b->d_iters + u;
        set_items(b, slot, n_events[u], bp);
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    int64_t grid = (int64_t)nsm * b->kern.max_blocks_per_sm;
    if (grid > bp.start[nproc]) grid = bp.start[nproc];
    cudaStream_t c = b->capture_stream;
    MF_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaMemsetAsync(b->d_counter, 0, sizeof(long long), c);
    void *args[] = {&bp};
    mf_status st = ce == cudaSuccess ? mfi::launch_kernel(b->kern, (unsigned)grid, args, c) : MF_ECUDA;
    for (int k = 0; k < nproc && st == MF_OK; ++k) {
        mf_process *p = b->procs[k];
        mf_vegas *v = grids[k];
        const int64_t n = n_events[k];
        const int64_t nchunks = (n + kChunk - 1) / kChunk;
        const int K = partial_size(v);
        vegas_accumulate_kernel<<<(unsigned)nchunks, kAccThreads, kAccSmem, c>>>(p->d_w, p->d_bins, n, v->ndim,
                                                                                  v->nbins, v->d_slots, nchunks);
        vegas_tree_kernel<<<dim3((unsigned)K, 1), kTreeThreads, 0, c>>>(v->d_slots, nchunks, 0, nchunks, K,
                                                                         b->d_root_ids + 2 * k, v->d_tree_out);
        vegas_finalize_dev_kernel<<<1, 128, 0, c>>>(v->d_tree_out, n, v->ndim, v->nbins, b->d_iters + k, v->d_hist,
                                                    v->d_count, v->d_hist_iter, v->d_result);
        if (refine) vegas_refine_kernel<<<1, 32, 0, c>>>(v->d_grid, v->d_hist, v->ndim, v->nbins, n, v->alpha);
        if (cudaMemcpyAsync(b->h_res + 8 * k, v->d_result, sizeof(double) * 7, cudaMemcpyDeviceToHost, c) !=
                cudaSuccess ||
            cudaMemcpyAsync(b->h_flags + k, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, c) != cudaSuccess)
            st = MF_ECUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c, &g);
    if (st != MF_OK || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(MF_ECUDA, std::string("capturing the batched iteration failed: ") + cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        b->graph = nullptr;
        return fail(MF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    b->graph_grids.assign(grids, grids + nproc);
    b->graph_n.assign(n_events, n_events + nproc);
    b->graph_ptrs = graph_buffers(b, grids);
    b->graph_seed = seed;
    b->graph_refine = refine ? 1 : 0;
    return MF_OK;
}
}  // namespace

extern "C" mf_status mf_batch_iterate_graph(mf_batch *b, mf_vegas *const *grids, const int64_t *n_events,
                                            uint64_t seed, int32_t refine, mf_iter_result *out, void *stream) {
    if (!b || !grids || !n_events || !out) return fail(MF_EINVAL, "NULL argument");
    const int nproc = (int)b->procs.size();
    for (int k = 0; k < nproc; ++k) {
        if (!grids[k]) return fail(MF_EINVAL, "NULL grid");
        if (grids[k]->ndim != b->procs[k]->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
        if (n_events[k] < 2) return fail(MF_EINVAL, "need at least two events per iteration");
        if ((n_events[k] + kChunk - 1) / kChunk > ((int64_t)1 << kTreeMaxLevel))
            return fail(MF_EINVAL, "too many events per iteration");
        if (grids[k]->iteration >= grids[k]->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
        for (int q = 0; q < k; ++q)
            if (grids[q] == grids[k]) return fail(MF_EINVAL, "a grid appears twice");
    }
    bool same = b->graph && b->graph_seed == seed && b->graph_refine == (refine ? 1 : 0);
    for (int k = 0; k < nproc && same; ++k) same = b->graph_grids[k] == grids[k] && b->graph_n[k] == n_events[k];
    if (same) same = graph_buffers(b, grids) == b->graph_ptrs;
    if (!same) {
        mf_status st = capture_batch(b, grids, n_events, seed, refine);
        if (st != MF_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < nproc; ++k) b->h_iters[k] = grids[k]->iteration;
    MF_CUDA(cudaMemcpyAsync(b->d_iters, b->h_iters, sizeof(long long) * nproc, cudaMemcpyHostToDevice, s));
    MF_CUDA(cudaGraphLaunch(b->graph, s));
    MF_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nproc; ++k) {
        mf_status st = flag_status(b->procs[k], b->h_flags[k]);
        if (st != MF_OK) return st;
    }
    bool any_nan = false;
    for (int k = 0; k < nproc; ++k) {
        fill_result(out[k], grids[k], n_events[k], b->h_res + 8 * k);
        any_nan |= out[k].n_nan > 0;
        grids[k]->iteration += 1;
    }
    if (any_nan) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}

// ----------------------------------------------------------------------------
// Weighted histograms of observables of a Vegas pass.
// ----------------------------------------------------------------------------
static_assert(MF_KP_MAX_OBS == MF_MAX_OBSERVABLES, "observable table sizes");
namespace {
constexpr int kObsBins = 64;            // bins per observable at most

// One block per chunk of kChunk points: per observable and bin the sums of w
// and w^2 and the count of the chunk's points; each warp adds its kChunk/8
// consecutive points in point order (lanes of one bin by the lowest of them,
// in lane order), then the 8 warps' sums are added in a fixed tree.
// Partials part[chunk][obs][kObsBins][3].  Non-finite weights are not binned.
__global__ void __launch_bounds__(kAccThreads) obs_accumulate_kernel(const double *w, const uint16_t *obs,
                                                                     int64_t n, int n_obs, double *part,
                                                                     int *nan_flag) {
    constexpr int kWarps = kAccThreads / 32, kPerWarp = kChunk / kWarps;
    __shared__ double s1[kWarps][kObsBins], s2[kWarps][kObsBins];
    __shared__ int sc[kWarps][kObsBins];
    __shared__ double stage[kWarps][32];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int m = (int)((n - base) < kChunk ? (n - base) : kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < n_obs; ++k) {
        for (int q = lane; q < kObsBins; q += 32) {
            s1[warp][q] = 0.0;
            s2[warp][q] = 0.0;
            sc[warp][q] = 0;
        }
        __syncwarp();
        for (int step = 0; step < kPerWarp / 32; ++step) {
            const int i = warp * kPerWarp + step * 32 + lane;
            double v = 0.0;
            int b = 0xFFFF;
            if (i < m) {
                v = w[base + i];
                b = obs[(int64_t)k * n + base + i];
                if (!isfinite(v)) {
                    if (k == 0) atomicExch(nan_flag, 1);
                    b = 0xFFFF;
                }
            }
            stage[warp][lane] = v;
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            __syncwarp();
            if (b < kObsBins && lane == __ffs(peers) - 1) {
                double a1 = s1[warp][b], a2 = s2[warp][b];
                int c = sc[warp][b];
                for (unsigned mk = peers; mk; mk &= mk - 1) {
                    const double x = stage[warp][__ffs(mk) - 1];
                    a1 += x;
                    a2 += x * x;
                    ++c;
                }
                s1[warp][b] = a1;
                s2[warp][b] = a2;
                sc[warp][b] = c;
            }
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x < kObsBins) {
            const int q = threadIdx.x;
            static_assert(kWarps == 8, "fixed 8-warp tree");
            double *o = part + (((int64_t)blockIdx.x * n_obs + k) * kObsBins + q) * 3;
            o[0] = ((s1[0][q] + s1[1][q]) + (s1[2][q] + s1[3][q])) + ((s1[4][q] + s1[5][q]) + (s1[6][q] + s1[7][q]));
            o[1] = ((s2[0][q] + s2[1][q]) + (s2[2][q] + s2[3][q])) + ((s2[4][q] + s2[5][q]) + (s2[6][q] + s2[7][q]));
            int c = 0;
            for (int ww = 0; ww < kWarps; ++ww) c += sc[ww][q];
            o[2] = (double)c;
        }
        __syncthreads();
    }
}

// Fixed pairwise sum of v[lo, hi) (halves split at the midpoint).
double pairwise_sum(const std::vector<double> &v, size_t lo, size_t hi) {
    if (hi - lo == 0) return 0.0;
    if (hi - lo == 1) return v[lo];
    const size_t mid = lo + (hi - lo) / 2;
    return pairwise_sum(v, lo, mid) + pairwise_sum(v, mid, hi);
}
}  // namespace

namespace {
mf_status observables_impl(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed, int32_t subprocess,
                           int32_t channel, mf_precision prec, int32_t n_obs, const mf_observable *obs, double *sigma,
                           double *error, int64_t *counts, void *stream);
}  // namespace

extern "C" mf_status mf_vegas_observables(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed,
                                          int32_t subprocess, mf_precision prec, int32_t n_obs,
                                          const mf_observable *obs, double *sigma, double *error, int64_t *counts,
                                          void *stream) {
    return observables_impl(v, p, n_events, seed, subprocess, -1, prec, n_obs, obs, sigma, error, counts, stream);
}

extern "C" mf_status mf_vegas_observables_channel(mf_vegas *v, mf_process *p, int32_t channel, int64_t n_events,
                                                  uint64_t seed, mf_precision prec, int32_t n_obs,
                                                  const mf_observable *obs, double *sigma, double *error,
                                                  int64_t *counts, void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (p->channels.K == 0) return fail(MF_EUNSUPPORTED, "the process has no phase-space channels");
    if (channel < 0 || channel >= p->channels.K) return fail(MF_EINVAL, "channel out of range");
    return observables_impl(v, p, n_events, seed, channel, channel, prec, n_obs, obs, sigma, error, counts, stream);
}

namespace {
mf_status observables_impl(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed, int32_t subprocess,
                           int32_t channel, mf_precision prec, int32_t n_obs, const mf_observable *obs, double *sigma,
                           double *error, int64_t *counts, void *stream) {
    if (!v || !p || !obs || !sigma || !error) return fail(MF_EINVAL, "NULL argument");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (v->ndim != p->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
    if (n_events < 2) return fail(MF_EINVAL, "need at least two points");
    if (subprocess < 0) return fail(MF_EINVAL, "bad subprocess index");
    if (n_obs < 1 || n_obs > MF_KP_MAX_OBS) return fail(MF_EINVAL, "n_obs must be 1 .. MF_MAX_OBSERVABLES");
    for (int k = 0; k < n_obs; ++k) {
        const mf_observable &o = obs[k];
        if (o.kind < MF_OBS_PT || o.kind > MF_OBS_PSEUDORAPIDITY) return fail(MF_EINVAL, "bad observable kind");
        if (o.leg < 2 || o.leg >= p->n_legs) return fail(MF_EINVAL, "observable leg must be a final-state leg");
        if (o.nbins < 1 || o.nbins > kObsBins) return fail(MF_EINVAL, "nbins must be 1 .. 64");
        if (!std::isfinite(o.lo) || !std::isfinite(o.hi) || !(o.hi > o.lo)) return fail(MF_EINVAL, "bad range");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = n_events;
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    st = ensure_scratch(p, v, n);
    if (st != MF_OK) return st;
    // the weights of the pass
    mf_kparams kp;
    vegas_params(p, v, n, 0, subprocess, seed, kp);
    kp.channel = channel;
    st = launch(p, prec, kp, s);
    if (st != MF_OK) return st;
    p->last_n = n;
    // the observables' bins of the same points, recomputed from their Philox
    // counters (no helicity work)
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    uint16_t *d_obs = nullptr;
    double *d_part = nullptr;
    int *d_nan = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_obs);
        cudaFree(d_part);
        cudaFree(d_nan);
    };
#define MF_OB(call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cleanup();                                                                         \
            return fail(MF_ECUDA, std::string("observables: ") + cudaGetErrorString(e_));      \
        }                                                                                      \
    } while (0)
    MF_OB(mfi::dev_malloc(&d_obs, sizeof(uint16_t) * (size_t)n_obs * n));
    MF_OB(mfi::dev_malloc(&d_part, sizeof(double) * (size_t)nchunks * n_obs * kObsBins * 3));
    MF_OB(mfi::dev_malloc(&d_nan, sizeof(int)));
    MF_OB(cudaMemsetAsync(d_nan, 0, sizeof(int), s));
    mf_kparams ko;
    vegas_params(p, v, n, 0, subprocess, seed, ko);
    ko.mode = 4;
    ko.channel = channel;
    ko.obs_out = d_obs;
    ko.n_obs = n_obs;
    for (int k = 0; k < n_obs; ++k) {
        ko.obs_kind[k] = obs[k].kind;
        ko.obs_leg[k] = obs[k].leg;
        ko.obs_nbins[k] = obs[k].nbins;
        ko.obs_lo[k] = obs[k].lo;
        ko.obs_scale[k] = obs[k].nbins / (obs[k].hi - obs[k].lo);
    }
    st = launch(p, prec, ko, s);
    if (st != MF_OK) {
        cleanup();
        return st;
    }
    obs_accumulate_kernel<<<(unsigned)nchunks, kAccThreads, 0, s>>>(p->d_w, d_obs, n, n_obs, d_part, d_nan);
    MF_OB(cudaGetLastError());
    std::vector<double> part((size_t)nchunks * n_obs * kObsBins * 3);
    int flag = 0, any_nan = 0;
    MF_OB(cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s));
    MF_OB(cudaMemcpyAsync(&any_nan, d_nan, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_OB(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_OB(cudaStreamSynchronize(s));
#undef MF_OB
    cleanup();
    st = flag_status(p, flag);
    if (st != MF_OK) return st;
    // chunk partials combined along a fixed pairwise tree over the chunk index
    std::vector<double> col(nchunks);
    size_t out = 0;
    const double N = (double)n;
    for (int k = 0; k < n_obs; ++k)
        for (int b = 0; b < obs[k].nbins; ++b, ++out) {
            double r[3];
            for (int c = 0; c < 3; ++c) {
                for (int64_t ch = 0; ch < nchunks; ++ch)
                    col[ch] = part[(((size_t)ch * n_obs + k) * kObsBins + b) * 3 + c];
                r[c] = pairwise_sum(col, 0, col.size());
            }
            const double sg = r[0] / N;
            const double var = (r[1] / N - sg * sg) / (N - 1.0);
            sigma[out] = sg;
            error[out] = std::sqrt(var > 0.0 ? var : 0.0);
            if (counts) counts[out] = (int64_t)r[2];
        }
    if (any_nan) return fail(MF_ENAN, "some points had non-finite weights (not binned)");
    return MF_OK;
}
}  // namespace

// ----------------------------------------------------------------------------
// Unweighting (hit or miss against w_max) and event records.
// ----------------------------------------------------------------------------
namespace {
constexpr int kUwThreads = 256;
constexpr int kUwPer = kChunk / kUwThreads;          // consecutive points per thread

// Per chunk: the accept decision of every point and the chunk's count.
__global__ void __launch_bounds__(kUwThreads) unweight_count_kernel(const double *w, int64_t n, uint64_t seed,
                                                                    uint64_t iteration, uint64_t subprocess,
                                                                    double w_max, uint8_t *acc, int *count) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int local = 0;
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kUwPer;
    for (int k = 0; k < kUwPer; ++k) {
        const int64_t g = base + k;
        if (g >= n) break;
        uint64_t c[4] = {(uint64_t)g, iteration, subprocess, 15ull};
        mf::philox4x64_10(c, seed, 0ull);
        const double u = mf::unit_from_bits(c[0]);
        const bool a = fabs(w[g]) > u * w_max;
        acc[g] = a ? 1 : 0;
        local += a ? 1 : 0;
    }
    atomicAdd(&s_cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) count[blockIdx.x] = s_cnt;
}

// Indices and weights of the kept points, in point order: chunk offsets from
// the host, within a chunk a block-wide exclusive scan of per-thread counts.
__global__ void __launch_bounds__(kUwThreads) unweight_compact_kernel(const uint8_t *acc, const double *w, int64_t n,
                                                                      const int64_t *offset, int64_t *idx,
                                                                      double *wk) {
    __shared__ int s_scan[kUwThreads];
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kUwPer;
    int mine = 0;
    for (int k = 0; k < kUwPer; ++k) {
        const int64_t g = base + k;
        if (g < n) mine += acc[g];
    }
    s_scan[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < kUwThreads; off <<= 1) {
        const int v = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t pos = offset[blockIdx.x] + s_scan[threadIdx.x] - mine;
    for (int k = 0; k < kUwPer; ++k) {
        const int64_t g = base + k;
        if (g < n && acc[g]) {
            idx[pos] = g;
            wk[pos] = w[g];
            ++pos;
        }
    }
}

__global__ void max_abs_kernel(const double *w, int64_t n, unsigned long long *out) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(w[i]);
        if (a > m) m = a;            // NaN never wins
    }
    // non-negative doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
}  // namespace

namespace {
__global__ void gather_kernel(const double *w, const int64_t *idx, int64_t n, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = w[idx[i]];
}
}  // namespace

extern "C" mf_status mf_process_read_weights(mf_process *p, const int64_t *idx, int64_t n, double *w) {
    if (!p || (n > 0 && (!idx || !w)) || n < 0) return fail(MF_EINVAL, "bad arguments");
    for (int64_t i = 0; i < n; ++i)
        if (idx[i] < 0 || idx[i] >= p->last_n) return fail(MF_EINVAL, "point index outside the last pass");
    if (n == 0) return MF_OK;
    int64_t *d_idx = nullptr;
    double *d_out = nullptr;
    cudaError_t e = mfi::dev_malloc(&d_idx, sizeof(int64_t) * n);
    if (e == cudaSuccess) e = mfi::dev_malloc(&d_out, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_idx, idx, sizeof(int64_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        gather_kernel<<<(unsigned)((n + 255) / 256), 256>>>(p->d_w, d_idx, n, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(w, d_out, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_idx);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail(MF_ECUDA, std::string("reading weights: ") + cudaGetErrorString(e));
    return MF_OK;
}

extern "C" mf_status mf_process_max_weight(mf_process *p, double *w_max, void *stream) {
    if (!p || !w_max) return fail(MF_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    MF_CUDA(mfi::dev_malloc(&d, sizeof(unsigned long long)));
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, s);
    if (e == cudaSuccess && p->last_n > 0) {
        max_abs_kernel<<<304, 256, 0, s>>>(p->d_w, p->last_n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MF_ECUDA, std::string("max weight: ") + cudaGetErrorString(e));
    double m;
    std::memcpy(&m, &h, sizeof m);
    *w_max = m;
    return MF_OK;
}

namespace {

// Unweighting of the points of one subprocess stream; channel >= 0 takes
// the points' momenta and weights from that phase-space channel.
mf_status unweight_impl(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed, int32_t subprocess,
                        int32_t channel, mf_precision prec, double w_max, mf_lhe_writer *lhe, double *records,
                        int64_t capacity, int64_t *n_accepted, void *stream) {
    if (!v || !p || !n_accepted) return fail(MF_EINVAL, "NULL argument");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (v->ndim != p->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
    if (n_events < 1) return fail(MF_EINVAL, "need at least one point");
    if (!(w_max > 0.0) || !std::isfinite(w_max)) return fail(MF_EINVAL, "w_max must be positive and finite");
    if (capacity < 0 || (capacity > 0 && !records)) return fail(MF_EINVAL, "bad record buffer");
    if (subprocess < 0) return fail(MF_EINVAL, "bad subprocess index");
    if (lhe && mfi::lhe_legs(lhe) != p->n_legs) return fail(MF_EINVAL, "LHE writer and process have different legs");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = n_events;
    mf_status st = compile_precision(p, prec);
    if (st != MF_OK) return st;
    st = ensure_scratch(p, v, n);
    if (st != MF_OK) return st;
    // the weights of the pass
    mf_kparams kp;
    vegas_params(p, v, n, 0, subprocess, seed, kp);
    kp.channel = channel;
    st = launch(p, prec, kp, s);
    if (st != MF_OK) return st;
    p->last_n = n;
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    uint8_t *d_acc = nullptr;
    int *d_cnt = nullptr;
    int64_t *d_off = nullptr, *d_idx = nullptr;
    double *d_wk = nullptr, *d_rec = nullptr;
    int32_t *d_flow = nullptr;
    std::vector<int> cnt(nchunks);
    std::vector<int64_t> off(nchunks);
    int64_t nacc = 0;
    const int RW = 2 + 4 * p->n_legs;
    auto cleanup = [&]() {
        cudaFree(d_acc);
        cudaFree(d_cnt);
        cudaFree(d_off);
        cudaFree(d_idx);
        cudaFree(d_wk);
        cudaFree(d_rec);
        cudaFree(d_flow);
    };
#define MF_UW(call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cleanup();                                                                         \
            return fail(MF_ECUDA, std::string("unweighting: ") + cudaGetErrorString(e_));       \
        }                                                                                      \
    } while (0)
    MF_UW(mfi::dev_malloc(&d_acc, (size_t)n));
    MF_UW(mfi::dev_malloc(&d_cnt, sizeof(int) * nchunks));
    MF_UW(mfi::dev_malloc(&d_off, sizeof(int64_t) * nchunks));
    unweight_count_kernel<<<(unsigned)nchunks, kUwThreads, 0, s>>>(p->d_w, n, seed, (uint64_t)v->iteration,
                                                                   (uint64_t)subprocess, w_max, d_acc, d_cnt);
    MF_UW(cudaGetLastError());
    MF_UW(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * nchunks, cudaMemcpyDeviceToHost, s));
    int flag = 0;
    MF_UW(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_UW(cudaStreamSynchronize(s));
    st = flag_status(p, flag);
    if (st != MF_OK) {
        cleanup();
        return st;
    }
    for (int64_t c = 0; c < nchunks; ++c) {
        off[c] = nacc;
        nacc += cnt[c];
    }
    *n_accepted = nacc;
    if (nacc > 0 && (capacity > 0 || lhe)) {
        MF_UW(cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * nchunks, cudaMemcpyHostToDevice, s));
        MF_UW(mfi::dev_malloc(&d_idx, sizeof(int64_t) * nacc));
        MF_UW(mfi::dev_malloc(&d_wk, sizeof(double) * nacc));
        MF_UW(mfi::dev_malloc(&d_rec, sizeof(double) * RW * nacc));
        MF_UW(mfi::dev_malloc(&d_flow, sizeof(int32_t) * nacc));
        unweight_compact_kernel<<<(unsigned)nchunks, kUwThreads, 0, s>>>(d_acc, p->d_w, n, d_off, d_idx, d_wk);
        MF_UW(cudaGetLastError());
        // the kept points' kinematics, recomputed from their Philox counters
        mf_kparams kr;
        vegas_params(p, v, nacc, 0, subprocess, seed, kr);
        kr.mode = 3;
        kr.idx = d_idx;
        kr.f = d_rec;
        kr.channel = channel;
        st = launch(p, prec, kr, s);
        if (st != MF_OK) {
            cleanup();
            return st;
        }
        // their leading-colour flows (the full helicity sum per flow; no
        // helicity sampling), drawn on the device
        mf_kparams kc;
        vegas_params(p, v, nacc, 0, subprocess, seed, kc);
        kc.mode = 5;
        kc.hel_sample = 0;
        kc.idx = d_idx;
        kc.flow_out = d_flow;
        kc.channel = channel;
        st = launch(p, prec, kc, s);
        if (st != MF_OK) {
            cleanup();
            return st;
        }
        std::vector<double> wk(nacc), rec((size_t)RW * nacc);
        std::vector<int32_t> flow(nacc);
        MF_UW(cudaMemcpyAsync(wk.data(), d_wk, sizeof(double) * nacc, cudaMemcpyDeviceToHost, s));
        MF_UW(cudaMemcpyAsync(rec.data(), d_rec, sizeof(double) * RW * nacc, cudaMemcpyDeviceToHost, s));
        MF_UW(cudaMemcpyAsync(flow.data(), d_flow, sizeof(int32_t) * nacc, cudaMemcpyDeviceToHost, s));
        MF_UW(cudaStreamSynchronize(s));
        // record: event weight, x1, x2, colour flow, momenta
        const int OW = RW + 2;
        std::vector<double> out((size_t)OW * nacc);
        for (int64_t k = 0; k < nacc; ++k) {
            const double w = wk[k];
            const double ew = (w < 0.0 ? -1.0 : 1.0) * std::max(std::fabs(w), w_max) / (double)n;
            double *o = out.data() + (size_t)k * OW;
            const double *r = rec.data() + (size_t)k * RW;
            o[0] = ew;
            o[1] = r[0];
            o[2] = r[1];
            o[3] = (double)flow[k];
            std::copy(r + 2, r + RW, o + 4);
        }
        if (capacity > 0)
            std::copy(out.begin(), out.begin() + (size_t)OW * std::min(capacity, nacc), records);
        if (lhe) {
            st = mfi::lhe_push(lhe, std::move(out));
            if (st != MF_OK) {
                cleanup();
                return st;
            }
        }
    }
#undef MF_UW
    cleanup();
    return MF_OK;
}

}  // namespace

extern "C" mf_status mf_vegas_unweight(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed,
                                       int32_t subprocess, mf_precision prec, double w_max, mf_lhe_writer *lhe,
                                       double *records, int64_t capacity, int64_t *n_accepted, void *stream) {
    return unweight_impl(v, p, n_events, seed, subprocess, -1, prec, w_max, lhe, records, capacity, n_accepted,
                         stream);
}

extern "C" mf_status mf_vegas_unweight_channel(mf_vegas *v, mf_process *p, int32_t channel, int64_t n_events,
                                               uint64_t seed, mf_precision prec, double w_max, mf_lhe_writer *lhe,
                                               double *records, int64_t capacity, int64_t *n_accepted,
                                               void *stream) {
    if (!p) return fail(MF_EINVAL, "NULL process");
    if (p->channels.K == 0) return fail(MF_EUNSUPPORTED, "the process has no phase-space channels");
    if (channel < 0 || channel >= p->channels.K) return fail(MF_EINVAL, "channel out of range");
    return unweight_impl(v, p, n_events, seed, channel, channel, prec, w_max, lhe, records, capacity, n_accepted,
                         stream);
}

extern "C" mf_status mf_process_channel_max_weights(mf_process *p, const int64_t *n_events, int32_t n_channels,
                                                    double *w_max, void *stream) {
    if (!p || !n_events || !w_max) return fail(MF_EINVAL, "NULL argument");
    if (n_channels < 1 || n_channels != p->channels.K) return fail(MF_EINVAL, "one count per channel of the process");
    int64_t tot = 0;
    for (int k = 0; k < n_channels; ++k) {
        if (n_events[k] < 0) return fail(MF_EINVAL, "negative count");
        tot += n_events[k];
    }
    if (tot != p->last_n) return fail(MF_EINVAL, "the counts do not add up to the last pass's points");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    MF_CUDA(mfi::dev_malloc(&d, sizeof(unsigned long long) * n_channels));
    std::vector<unsigned long long> h(n_channels, 0);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * n_channels, s);
    int64_t off = 0;
    for (int k = 0; k < n_channels && e == cudaSuccess; ++k) {
        if (n_events[k] > 0) {
            max_abs_kernel<<<304, 256, 0, s>>>(p->d_w + off, n_events[k], d + k);
            e = cudaGetLastError();
        }
        off += n_events[k];
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * n_channels,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MF_ECUDA, std::string("max weights: ") + cudaGetErrorString(e));
    for (int k = 0; k < n_channels; ++k) std::memcpy(&w_max[k], &h[k], sizeof(double));
    return MF_OK;
}

// ----------------------------------------------------------------------------
// Checkpoint: a flat little-endian record of the grid state.
// ----------------------------------------------------------------------------
namespace {
constexpr char kMagic[8] = {'M', 'F', 'V', 'E', 'G', 'A', 'S', '1'};
struct CkptHeader {
    char magic[8];
    int32_t ndim, nbins, iteration, pad;
    double alpha;
};
size_t ckpt_size(const mf_vegas *v) {
    const size_t g = (size_t)v->ndim * (v->nbins + 1), h = (size_t)v->ndim * v->nbins;
    return sizeof(CkptHeader) + sizeof(double) * (g + h) + sizeof(int64_t) * h + sizeof(double) * 2 * v->iteration;
}
}  // namespace

extern "C" mf_status mf_vegas_save(const mf_vegas *v, void *buf, size_t *len) {
    if (!v || !len) return fail(MF_EINVAL, "NULL argument");
    const size_t need = ckpt_size(v);
    if (!buf) {
        *len = need;
        return MF_OK;
    }
    if (*len < need) {
        *len = need;
        return fail(MF_EINVAL, "buffer too small");
    }
    char *b = (char *)buf;
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.ndim = v->ndim;
    h.nbins = v->nbins;
    h.iteration = v->iteration;
    h.alpha = v->alpha;
    std::memcpy(b, &h, sizeof h);
    b += sizeof h;
    const size_t g = (size_t)v->ndim * (v->nbins + 1), hs = (size_t)v->ndim * v->nbins;
    MF_CUDA(cudaMemcpy(b, v->d_grid, sizeof(double) * g, cudaMemcpyDeviceToHost));
    b += sizeof(double) * g;
    MF_CUDA(cudaMemcpy(b, v->d_hist, sizeof(double) * hs, cudaMemcpyDeviceToHost));
    b += sizeof(double) * hs;
    MF_CUDA(cudaMemcpy(b, v->d_count, sizeof(int64_t) * hs, cudaMemcpyDeviceToHost));
    b += sizeof(int64_t) * hs;
    if (v->iteration > 0)
        MF_CUDA(cudaMemcpy(b, v->d_hist_iter, sizeof(double) * 2 * v->iteration, cudaMemcpyDeviceToHost));
    *len = need;
    return MF_OK;
}

extern "C" mf_status mf_vegas_load(mf_vegas *v, const void *buf, size_t len) {
    if (!v || !buf) return fail(MF_EINVAL, "NULL argument");
    CkptHeader h;
    if (len < sizeof h) return fail(MF_EINVAL, "checkpoint too short");
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, kMagic, 8) != 0) return fail(MF_EINVAL, "not a Vegas checkpoint");
    if (h.ndim != v->ndim || h.nbins != v->nbins) return fail(MF_EINVAL, "checkpoint shape differs from the grid");
    if (h.iteration < 0 || h.iteration > v->max_iter) return fail(MF_EINVAL, "bad iteration count");
    if (!(h.alpha >= 0.0)) return fail(MF_EINVAL, "bad alpha");
    mf_vegas tmp;
    tmp.ndim = h.ndim;
    tmp.nbins = h.nbins;
    tmp.iteration = h.iteration;
    if (len != ckpt_size(&tmp)) return fail(MF_EINVAL, "checkpoint size does not match its header");
    const char *b = (const char *)buf + sizeof h;
    const size_t g = (size_t)v->ndim * (v->nbins + 1), hs = (size_t)v->ndim * v->nbins;
    std::vector<double> edges(g);
    std::memcpy(edges.data(), b, sizeof(double) * g);
    mf_status st = check_edges(v, edges.data());
    if (st != MF_OK) return st;
    MF_CUDA(cudaMemcpy(v->d_grid, b, sizeof(double) * g, cudaMemcpyHostToDevice));
    b += sizeof(double) * g;
    MF_CUDA(cudaMemcpy(v->d_hist, b, sizeof(double) * hs, cudaMemcpyHostToDevice));
    b += sizeof(double) * hs;
    MF_CUDA(cudaMemcpy(v->d_count, b, sizeof(int64_t) * hs, cudaMemcpyHostToDevice));
    b += sizeof(int64_t) * hs;
    if (h.iteration > 0) MF_CUDA(cudaMemcpy(v->d_hist_iter, b, sizeof(double) * 2 * h.iteration, cudaMemcpyHostToDevice));
    v->iteration = h.iteration;
    v->alpha = h.alpha;
    return MF_OK;
}

// ----------------------------------------------------------------------------
// One Vegas iteration that allocates nothing.
//
// Some callers cannot let a library allocate device memory while they run:
// an application whose device memory is carved out by its own pool up front
// (a cudaMalloc would fail or fight that pool for memory), and loops that must
// not stall on the implicit device-wide synchronisation that cudaMalloc and
// cudaFree bring.  mf_vegas_iterate_static serves them: the scratch that
// mf_vegas_iterate keeps per process and grid (weights, bin indices, chunk
// partial sums, totals) lives here in one fixed array compiled into the
// library, and the call uses only memory that already exists.
// ----------------------------------------------------------------------------
namespace {
constexpr int64_t kStaticChunks = MF_STATIC_MAX_EVENTS / kChunk;
constexpr int kStaticMaxK = 4 + 2 * MF_MAX_DIM * 64;          // largest partial-sum vector
// layout: w [MAX_EVENTS] doubles | slots [K][chunks] + totals [K] doubles |
//         root node id [2] int64 | bins [MF_MAX_DIM][MAX_EVENTS] bytes
constexpr size_t kStaticW = 0;
constexpr size_t kStaticSlots = kStaticW + sizeof(double) * MF_STATIC_MAX_EVENTS;
constexpr size_t kStaticTot = kStaticSlots + sizeof(double) * (size_t)kStaticMaxK * kStaticChunks;
constexpr size_t kStaticIds = kStaticTot + sizeof(double) * kStaticMaxK;
constexpr size_t kStaticBins = kStaticIds + 2 * sizeof(int64_t);
constexpr size_t kStaticBytes = kStaticBins + (size_t)MF_MAX_DIM * MF_STATIC_MAX_EVENTS;   // 8,673,328 bytes
static_assert(MF_STATIC_MAX_EVENTS % kChunk == 0, "whole chunks");

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_base[kStaticMaxDevices];

// Address of the array on the current device, looked up once per device.
mf_status static_scratch(void **base) {
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(MF_EUNSUPPORTED, "device index beyond the static table");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(MF_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        g_static_base[dev] = p;
    }
    *base = g_static_base[dev];
    return MF_OK;
}

__global__ void static_root_kernel(int64_t *ids, int level) {
    ids[0] = level;
    ids[1] = 0;
}
}  // namespace

extern "C" mf_status mf_vegas_iterate_static(mf_vegas *v, mf_process *p, int64_t n_events, uint64_t seed,
                                             mf_precision prec, int32_t refine, mf_iter_result *out, void *stream) {
    if (!v || !p || !out) return fail(MF_EINVAL, "NULL argument");
    if (!valid_prec(prec)) return fail(MF_EINVAL, "bad precision");
    if (v->ndim != p->ndim) return fail(MF_EINVAL, "grid and process dimensions differ");
    if (n_events < 2) return fail(MF_EINVAL, "need at least two events per iteration");
    if (n_events > MF_STATIC_MAX_EVENTS)
        return fail(MF_EINVAL, "n_events exceeds MF_STATIC_MAX_EVENTS (" + std::to_string(MF_STATIC_MAX_EVENTS) +
                                   " points), the capacity of the static scratch; use mf_vegas_iterate");
    if (v->iteration >= v->max_iter) return fail(MF_EUNSUPPORTED, "too many iterations");
    if (!p->kern[prec].fn)
        return fail(MF_EINVAL, "the process kernel of this precision is not compiled yet (compiling allocates): "
                               "call mf_integrand or mf_vegas_iterate with it once first");
    void *base = nullptr;
    mf_status st = static_scratch(&base);
    if (st != MF_OK) return st;
    unsigned char *b = (unsigned char *)base;
    double *w = (double *)(b + kStaticW);
    double *slots = (double *)(b + kStaticSlots);
    double *tot = (double *)(b + kStaticTot);
    int64_t *ids = (int64_t *)(b + kStaticIds);
    uint8_t *bins = (uint8_t *)(b + kStaticBins);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = n_events;
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    const int K = partial_size(v);

    mf_kparams kp;
    fill_common(*p, kp);
    set_hel(kp, p->hel, p->n_legs);
    kp.mode = 1;
    kp.n = n;
    kp.ev0 = 0;
    kp.grid = v->d_grid;
    kp.nb = v->nbins;
    kp.w_out = w;
    kp.bins_out = bins;
    kp.seed = seed;
    kp.iteration = (uint64_t)v->iteration;
    kp.subprocess = 0;
    st = launch(p, prec, kp, s);
    if (st != MF_OK) return st;
    st = accumulate_into(w, bins, n, v, slots, s);
    if (st != MF_OK) return st;
    static_root_kernel<<<1, 1, 0, s>>>(ids, tree_levels(nchunks));
    vegas_tree_kernel<<<dim3((unsigned)K, 1), kTreeThreads, 0, s>>>(slots, nchunks, 0, nchunks, K, ids, tot);
    MF_CUDA(cudaGetLastError());
    st = finish(v, tot, n, refine, s);
    if (st != MF_OK) return st;
    double r[8];
    int flag = 0;
    MF_CUDA(cudaMemcpyAsync(r, v->d_result, sizeof(double) * 7, cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    // a process-kernel error (expired wait, too little shared memory) leaves
    // the weights unspecified: report it here, the iteration not advanced
    st = flag_status(p, flag);
    if (st != MF_OK) return st;
    fill_result(*out, v, n, r);
    v->iteration += 1;
    if (out->n_nan > 0) return fail(MF_ENAN, "some points had non-finite weights (counted as zero)");
    return MF_OK;
}
