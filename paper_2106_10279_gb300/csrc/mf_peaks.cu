// Arithmetic peaks of the device, measured by the library's own
// microbenchmarks: the denominators of the roofline fractions of the fused
// integrand kernel, which is bound by FP32 FMA (mixed precision), FP64 FMA
// (the all-double path) or, for its colour sum, the TF32 tensor-core MMA.
//
//   FFMA   every thread runs 8 independent chains a <- a * b + c (FP32), 16
//          steps per loop trip; 4 blocks of 256 threads per SM;
//   DFMA   the same in FP64;
//   FFMA2  the FFMA kernel on packed pairs of FP32 values (fma.rn.f32x2: two
//          FMAs per instruction);
//   TF32   one block of 128 threads per SM; one thread issues back-to-back
//          tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8) on operands in
//          shared memory in the no-swizzle K-major layout the colour-sum
//          kernel uses, accumulating into one tensor-memory tile; the block
//          waits (bounded) on the commit of the last MMA.
//
// FLOPs counted: 2 per FMA lane, 2 M N K per MMA.
#include <cstdint>
#include <string>

#include "mf_internal.h"
#include "device/mf_tc.cuh"

using mfi::fail;

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_peak_kernel(T *sink, int trips, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x & 63) * (T)0.001 + (T)k;
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // never true for these inputs; keeps the chains observable
    if (s == (T)-1.0) sink[threadIdx.x] = s;
}

// FP32 FMA on packed pairs (fma.rn.f32x2, sm_100 and later): one instruction
// performs two FP32 FMAs; 8 independent pair chains per thread
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
    return (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
}

__global__ void __launch_bounds__(kFmaThreads) ffma2_peak_kernel(float *sink, int trips, float b, float c) {
    unsigned long long a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = pack2((float)(threadIdx.x & 63) * 0.001f + (float)k, (float)k);
    const unsigned long long b2 = pack2(b, b), c2 = pack2(c, c);
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = ffma2(a[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += __uint_as_float((uint32_t)a[k]) + __uint_as_float((uint32_t)(a[k] >> 32));
    if (s == -1.0f) sink[threadIdx.x] = s;
}

// TF32 MMA peak: operands K = KP = 32 (4 MMA steps of K = 8), N = 256
constexpr int kMmaN = 256;
constexpr int kMmaKP = 32;
constexpr int kMmaABytes = 128 * kMmaKP * 4;
constexpr int kMmaBBytes = kMmaN * kMmaKP * 4;
constexpr int kMmaSmem = kMmaABytes + kMmaBBytes + 16;
constexpr uint64_t kWaitNs = 2000000000ull;   // bound of each completion wait (2 s)

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool wait_parity_bounded(uint64_t *mbar, uint32_t phase) {
    const uint32_t addr = mf::tc::smem_u32(mbar);
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__global__ void __launch_bounds__(128) tf32_mma_peak_kernel(int trips, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *a = smem, *b = smem + kMmaABytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kMmaABytes + kMmaBBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kMmaABytes + kMmaBBytes + 8);
    // operands: small exact values (no overflow over the accumulation)
    for (int i = threadIdx.x; i < 128 * kMmaKP; i += 128)
        *reinterpret_cast<float *>(a + mf::tc::core_offset(i / kMmaKP, i % kMmaKP, kMmaKP)) =
            (float)((i % 7) - 3) * 0.015625f;
    for (int i = threadIdx.x; i < kMmaN * kMmaKP; i += 128)
        *reinterpret_cast<float *>(b + mf::tc::core_offset(i / kMmaKP, i % kMmaKP, kMmaKP)) =
            (float)((i % 5) - 2) * 0.015625f;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mf::tc::smem_u32(tslot)),
                     "r"(kMmaN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mf::tc::smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = mf::tc::InstrDesc<128, kMmaN>::value;
        constexpr uint32_t sbo = (uint32_t)kMmaKP * 32;
        const uint32_t a0 = mf::tc::smem_u32(a), b0 = mf::tc::smem_u32(b);
        for (int t = 0; t < trips; ++t) {
#pragma unroll
            for (int ks = 0; ks < kMmaKP / 8; ++ks) {
                const uint64_t ad = mf::tc::smem_desc(a0 + ks * 256, 128, sbo);
                const uint64_t bd = mf::tc::smem_desc(b0 + ks * 256, 128, sbo);
                const uint32_t acc = (t | ks) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         mf::tc::smem_u32(mbar))
                     : "memory");
    }
    bool ok = wait_parity_bounded(mbar, 0);
    if (!ok) {
        if (err) atomicExch(err, 1);
        // one more bounded wait for the MMAs in flight before the tensor
        // memory is released
        wait_parity_bounded(mbar, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmaN));
}

}  // namespace

extern "C" mf_status mf_measure_peak(int32_t kind, int32_t reps, double *tflops, double *ms, void *stream) {
    if (kind < 0 || kind > 3 || reps < 1 || !tflops) return fail(MF_EINVAL, "mf_measure_peak: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return fail(MF_ECUDA, "mf_measure_peak: no device");
    void *d_sink = nullptr;
    int *d_err = nullptr;
    if (mfi::dev_malloc(&d_sink, kFmaThreads * sizeof(double)) != cudaSuccess ||
        mfi::dev_malloc(&d_err, sizeof(int)) != cudaSuccess) {
        cudaFree(d_sink);
        return fail(MF_ENOMEM, "mf_measure_peak: scratch");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mf_status st = MF_OK;
    double flops = 0.0;
    // trips sized for launches of about 10-30 ms at the nominal rates
    const int fma_trips = (kind == 0 || kind == 3) ? 32768 : 512;
    const int mma_trips = 65536;
    auto launch = [&]() -> cudaError_t {
        if (kind == 0) {
            fma_peak_kernel<float><<<nsm * kFmaBlocksPerSm, kFmaThreads, 0, s>>>((float *)d_sink, fma_trips,
                                                                                 0.9999999f, 1e-7f);
        } else if (kind == 1) {
            fma_peak_kernel<double><<<nsm * kFmaBlocksPerSm, kFmaThreads, 0, s>>>((double *)d_sink, fma_trips,
                                                                                  0.9999999999, 1e-12);
        } else if (kind == 3) {
            ffma2_peak_kernel<<<nsm * kFmaBlocksPerSm, kFmaThreads, 0, s>>>((float *)d_sink, fma_trips, 0.9999999f,
                                                                           1e-7f);
        } else {
            tf32_mma_peak_kernel<<<nsm, 128, kMmaSmem, s>>>(mma_trips, d_err);
        }
        return cudaGetLastError();
    };
    if (kind == 2) {
        flops = 2.0 * 128 * kMmaN * kMmaKP * (double)mma_trips * nsm;
        if (cudaFuncSetAttribute(tf32_mma_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem) !=
            cudaSuccess)
            st = fail(MF_ECUDA, "mf_measure_peak: shared-memory attribute");
    } else {
        flops = 2.0 * kChains * kUnroll * (double)fma_trips * kFmaThreads * kFmaBlocksPerSm * nsm * (kind == 3 ? 2 : 1);
    }
    if (st == MF_OK && (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess ||
                        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(MF_ECUDA, "mf_measure_peak: set-up");
    double best = 0.0;
    if (st == MF_OK && launch() != cudaSuccess) st = fail(MF_ECUDA, "mf_measure_peak: launch");   // warm-up
    for (int r = 0; st == MF_OK && r < reps; ++r) {
        cudaEventRecord(e0, s);
        if (launch() != cudaSuccess) {
            st = fail(MF_ECUDA, "mf_measure_peak: launch");
            break;
        }
        cudaEventRecord(e1, s);
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            st = fail(MF_ECUDA, "mf_measure_peak: timing");
            break;
        }
        if (best == 0.0 || t < best) best = t;
    }
    int herr = 0;
    if (st == MF_OK && cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = fail(MF_ECUDA, "mf_measure_peak: error flag");
    if (st == MF_OK && herr) st = fail(MF_ETIMEOUT, "mf_measure_peak: MMA completion wait expired");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_sink);
    cudaFree(d_err);
    if (st != MF_OK) return st;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return MF_OK;
}
