// Pieces shared by the product kernels of every stored format (see products.cu).
#pragma once

#include <cuda_runtime.h>

#include "bsgdtv_internal.h"

namespace bsgdtv {
namespace prod {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kCtasPerSm = 2;

// Accumulation of one column group (four nonzeros of this lane's segment):
// z partial in a register, the A^T r contribution into the shared g tile.
// FP32 path: the tile is int32 fixed point (r2 already carries the scale), so
// the shared-memory updates are native integer atomics and the tile's sums
// are exact and independent of their order.  FP64 path: FP64 atomics.
__device__ __forceinline__ void use_group(const float4 v, const int4 i, const float r2s,
                                          const float *xs, int *gs, float &acc) {
    acc = fmaf(v.x, xs[i.x], acc);
    atomicAdd(gs + i.x, __float2int_rn(v.x * r2s));
    acc = fmaf(v.y, xs[i.y], acc);
    atomicAdd(gs + i.y, __float2int_rn(v.y * r2s));
    acc = fmaf(v.z, xs[i.z], acc);
    atomicAdd(gs + i.z, __float2int_rn(v.z * r2s));
    acc = fmaf(v.w, xs[i.w], acc);
    atomicAdd(gs + i.w, __float2int_rn(v.w * r2s));
}

__device__ __forceinline__ void use_group(const float4 v, const int4 i, const double r2,
                                          const double *xs, double *gs, double &acc) {
    acc += (double)v.x * xs[i.x];
    atomicAdd(gs + i.x, (double)v.x * r2);
    acc += (double)v.y * xs[i.y];
    atomicAdd(gs + i.y, (double)v.y * r2);
    acc += (double)v.z * xs[i.z];
    atomicAdd(gs + i.z, (double)v.z * r2);
    acc += (double)v.w * xs[i.w];
    atomicAdd(gs + i.w, (double)v.w * r2);
}

}  // namespace prod
}  // namespace bsgdtv
