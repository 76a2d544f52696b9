// Measured FP32 CUDA-core throughput: the denominator of the ALU rooflines of
// the batched and matrix-free product passes (2 FMAs per nonzero and slice),
// timed on the GPU the library runs on at whatever clock it runs.
//
// Every thread runs kChains independent FMA chains (enough independent work
// per warp to cover the FMA latency at full occupancy) for `iters` rounds;
// the f32x2 form issues two lanes' worth of FMAs per instruction (the packed
// FP32 FMA of sm_100-class GPUs).  The chains' sums are stored so that no FMA
// is dead code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "bsgdtv_internal.h"

namespace bsgdtv {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 512;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float *out, float a, float b,
                                                                 int iters) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = 1e-3f * (float)threadIdx.x + (float)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) fma2_peak_kernel(float *out, float a, float b,
                                                                  int iters) {
    // kChains / 2 chains of packed pairs: the same number of FMAs per round
    uint64_t acc[kChains / 2];
    const float a2[2] = {a, a}, b2[2] = {b, b};
    uint64_t av, bv;
    memcpy(&av, a2, 8);
    memcpy(&bv, b2, 8);
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        const float v[2] = {1e-3f * (float)threadIdx.x + (float)c, (float)c + 0.5f};
        memcpy(&acc[c], v, 8);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(av), "l"(bv));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) {
        float v[2];
        memcpy(v, &acc[c], 8);
        s += v[0] + v[1];
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bsgdtv

using namespace bsgdtv;

extern "C" int bsgdtv_fp32_fma_peak(double *tflops_scalar, double *tflops_packed) {
    BSG_TRACE();
    if (!tflops_scalar && !tflops_packed) return fail(BSGDTV_ERR_INVALID_ARG, "null outputs");
    int dev = 0, sms = 0;
    BSG_CUDA(cudaGetDevice(&dev));
    BSG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * sms;   // 2048 threads per SM
    const int iters = 4096;       // 8 x 8 FMAs per round: 2^18 FMAs per thread
    float *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BSGDTV_OK;
    double best[2] = {0.0, 0.0};
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * kPeakThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double flops = 2.0 * (double)blocks * kPeakThreads * iters * 8 * kChains;
    for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first one warms up
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) {
                if (form == 0)
                    fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, 0.9999999f, 1e-7f, iters);
                else
                    fma2_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, 0.9999999f, 1e-7f, iters);
                add_launches(1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && ms > 0.f)
                best[form] = std::max(best[form], flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e != cudaSuccess) rc = fail(BSGDTV_ERR_CUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (rc == BSGDTV_OK) {
        if (tflops_scalar) *tflops_scalar = best[0];
        if (tflops_packed) *tflops_packed = best[1];
    }
    return rc;
}
