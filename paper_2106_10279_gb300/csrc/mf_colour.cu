// mf_colour_sum: the colour sum of Sec. 2.4 (per row r, the numerator sum
// sum_kl Re(conj(J_rk) C_kl J_rl) divided by the colour denominator) for a
// batch of rows of amplitudes, on the tensor cores (tcgen05, split TF32) or on
// the CUDA cores (FP32, the symmetric form the generated process kernels use).
// The fused process kernels use the same device code (device/mf_tc.cuh).
#include <cstdint>
#include <string>

#include "mf_internal.h"
#include "device/mf_tc.cuh"

using mfi::fail;

namespace {

// rows: J [2 NJ][n] (Re J_k in row 2k, Im J_k in row 2k + 1)
template <int NJ>
__device__ void load_row(const float *J, int64_t n, int64_t r, mf::cx<float> *Jr) {
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
        Jr[k].re = r < n ? J[(int64_t)(2 * k) * n + r] : 0.f;
        Jr[k].im = r < n ? J[(int64_t)(2 * k + 1) * n + r] : 0.f;
    }
}

template <int NJ>
__global__ void __launch_bounds__(128) colour_tc_kernel(const float *J, int64_t n, const int *cnum, float inv_den,
                                                        float *out, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    mf::tc::State st;
    mf::tc::setup<NJ>(st, smem, err);
    mf::tc::load_colour<NJ>(st, cnum);
    __syncthreads();
    const int64_t ntiles = (n + 127) / 128;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r = t * 128 + threadIdx.x;
        mf::cx<float> Jr[NJ];
        load_row<NJ>(J, n, r, Jr);
        const float m = mf::tc::colour_sum<NJ>(st, Jr);
        if (r < n) out[r] = m * inv_den;
    }
    mf::tc::teardown<NJ>(st);
}

template <int NJ>
__global__ void colour_fp32_kernel(const float *J, int64_t n, const int *cnum, float inv_den, float *out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    mf::cx<float> Jr[NJ];
    load_row<NJ>(J, n, r, Jr);
    float m = 0.f;
    for (int k = 0; k < NJ; ++k) {
        float zr = (float)cnum[k * NJ + k] * Jr[k].re, zi = (float)cnum[k * NJ + k] * Jr[k].im;
        for (int l = k + 1; l < NJ; ++l) {
            const float c = 2.f * (float)cnum[k * NJ + l];
            zr += c * Jr[l].re;
            zi += c * Jr[l].im;
        }
        m += Jr[k].re * zr + Jr[k].im * zi;
    }
    out[r] = m * inv_den;
}

template <int NJ>
mf_status run(const float *J, int64_t n, const int *d_c, float inv_den, int use_tc, float *out, int *d_err,
              cudaStream_t s) {
    if (use_tc) {
        const int smem = mf::tc::Plan<NJ>::SMEM;
        cudaError_t e = cudaFuncSetAttribute(colour_tc_kernel<NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return fail(MF_ECUDA, std::string("colour kernel attribute: ") + cudaGetErrorString(e));
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        int64_t ntiles = (n + 127) / 128;
        int64_t grid = ntiles < nsm ? ntiles : nsm;
        colour_tc_kernel<NJ><<<(unsigned)grid, 128, smem, s>>>(J, n, d_c, inv_den, out, d_err);
    } else {
        colour_fp32_kernel<NJ><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(J, n, d_c, inv_den, out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MF_ECUDA, std::string("colour kernel launch: ") + cudaGetErrorString(e));
    return MF_OK;
}

}  // namespace

extern "C" mf_status mf_colour_sum(const float *J, int64_t n, const int32_t *cnum, int32_t nj, int32_t den,
                                   int32_t use_tc, float *out, void *stream) {
    if (n < 0 || (n > 0 && (!J || !out)) || !cnum || den <= 0) return fail(MF_EINVAL, "bad arguments");
    if (nj != 2 && nj != 4 && nj != 6 && nj != 24) return fail(MF_EUNSUPPORTED, "colour basis size must be 2, 4, 6 or 24");
    if (n == 0) return MF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_c = nullptr, *d_err = nullptr;
    if (mfi::dev_malloc(&d_c, sizeof(int) * nj * nj) != cudaSuccess || mfi::dev_malloc(&d_err, sizeof(int)) != cudaSuccess) {
        cudaFree(d_c);
        return fail(MF_ENOMEM, "colour sum scratch");
    }
    mf_status st = MF_OK;
    int herr = 0;
    if (cudaMemcpyAsync(d_c, cnum, sizeof(int) * nj * nj, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess)
        st = fail(MF_ECUDA, "colour sum upload");
    const float inv = 1.0f / (float)den;
    if (st == MF_OK) {
        switch (nj) {
            case 2: st = run<2>(J, n, d_c, inv, use_tc, out, d_err, s); break;
            case 4: st = run<4>(J, n, d_c, inv, use_tc, out, d_err, s); break;
            case 6: st = run<6>(J, n, d_c, inv, use_tc, out, d_err, s); break;
            default: st = run<24>(J, n, d_c, inv, use_tc, out, d_err, s); break;
        }
    }
    if (st == MF_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail(MF_ECUDA, std::string("colour sum: ") + cudaGetErrorString(e));
    }
    cudaFree(d_c);
    cudaFree(d_err);
    if (st == MF_OK && herr) st = fail(MF_ETIMEOUT, "tensor-core colour sum: completion wait expired");
    return st;
}
