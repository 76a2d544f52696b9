// bsgdtv_tv_prox_static: the TV prox of Algorithm 1 (FGP) without any allocation.
//
// Some callers cannot allocate device memory at call time: a process whose
// whole device budget is already claimed by its own pool allocator (a raw
// cudaMalloc there may fail or fragment the pool), a latency-critical loop in
// which the implicit device-wide synchronisation of cudaMalloc/cudaFree would
// stall every other stream, or a host runtime that forbids plugins from
// allocating at all.  This entry point serves them: its scratch (the FGP dual
// fields and the momentum table) lives in one file-scope device array that is
// part of the loaded library.  Every GPU that loads the library holds that
// array (about 8 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "bsgdtv_internal.h"

namespace bsgdtv {
namespace {

constexpr int64_t kStaticMaxPixels = 512 * 512;   // largest img_h * img_w accepted
constexpr int kStaticMaxIters = 4096;             // largest FGP iteration count accepted
constexpr int64_t kStaticFloats = kFgpFieldPlanes * kStaticMaxPixels + kStaticMaxIters;

// Two sets of p, q, p_prev, q_prev (kStaticMaxPixels floats each; the tiled
// FGP's launches read one set and write the other) then the momentum table.
static __device__ __align__(256) float g_static_scratch[kStaticFloats];

// Device address of g_static_scratch, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so kernels must be
// given this address, never the symbol itself.
constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(float **out) {
    int dev = 0;
    BSG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(BSGDTV_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(BSGDTV_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                             cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return BSGDTV_OK;
}

}  // namespace
}  // namespace bsgdtv

using namespace bsgdtv;

extern "C" int bsgdtv_tv_prox_static(const float *b, float *x, int img_h, int img_w, double tau,
                                     int iters, void *stream) {
    if (!b || !x || img_h < 1 || img_w < 1 || iters < 0 || !std::isfinite(tau))
        return fail(BSGDTV_ERR_INVALID_ARG, "bad argument");
    if (b == x) return fail(BSGDTV_ERR_INVALID_ARG, "b and x may not alias");
    const int64_t n = (int64_t)img_h * img_w;
    if (n > kStaticMaxPixels)
        return fail(BSGDTV_ERR_INVALID_ARG,
                    "image too large for the static scratch: img_h*img_w must be <= 262144");
    if (iters > kStaticMaxIters)
        return fail(BSGDTV_ERR_INVALID_ARG, "too many FGP iterations for the static scratch: max 4096");
    cudaStream_t s = (cudaStream_t)stream;
    if (tau <= 0.0 || iters == 0) {
        BSG_CUDA(cudaMemcpyAsync(x, b, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        BSG_CUDA(cudaStreamSynchronize(s));
        return BSGDTV_OK;
    }
    float *base = nullptr;
    BSG_CHECK(scratch_for_current_device(&base));
    // The dual fields need no clearing: the first FGP launch starts from zero
    // in registers and every later launch reads only values an earlier launch
    // of this call wrote.  The momentum table is rewritten in full below.
    float *mom_dev = base + kFgpFieldPlanes * kStaticMaxPixels;
    float mom[kStaticMaxIters];
    double t = 1.0;
    mom[0] = 0.f;
    for (int k = 1; k < iters; ++k) {
        const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
        mom[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
    BSG_CUDA(cudaMemcpyAsync(mom_dev, mom, iters * sizeof(float), cudaMemcpyHostToDevice, s));
    const FgpScratch sc = fgp_scratch_planes(base, kStaticMaxPixels);
    BSG_CUDA(launch_fgp(b, x, img_h, img_w, (float)tau, iters, mom_dev, sc, s));
    BSG_CUDA(cudaStreamSynchronize(s));
    return BSGDTV_OK;
}
