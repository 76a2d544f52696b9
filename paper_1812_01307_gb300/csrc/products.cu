// Fused block products of Algorithm 1, lines 2-5 (one pass over A).
//
// For every work item (row group G inside a row block I_i, pixel tile T inside
// a column band J_j) the CTA computes, from a single read of the item's
// nonzeros,
//   z partial:  sum over the row's nonzeros in T of a * x        (line 4)
//   g partial:  sum over G's rows of 2 a r_row, for each pixel of T (line 3)
// where r is the residual of the previous epoch (the paper's stale gradient,
// Eq. 3).  x_T is staged in shared memory and the g tile accumulates there;
// each warp walks one slab of 32 row segments with one lane per segment, so
// the z partial of a segment stays in a register.
#include <cuda_runtime.h>

#include "bsgdtv_internal.h"

namespace bsgdtv {

namespace {

template <typename T>
__device__ __forceinline__ T load_stream(const float *p) {
    return (T)__ldcs(p);
}

template <typename T>
__global__ void __launch_bounds__(256) products_kernel(const DevLayout d, const T *__restrict__ x,
                                                       const T *__restrict__ r,
                                                       T *__restrict__ z_part,
                                                       T *__restrict__ g_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *gs = xs + kTileH * kTileStride;

    const WorkItem it = d.items[blockIdx.x];
    const Tile tl = d.tiles[it.tile];

    for (int e = threadIdx.x; e < kTileH * kTileStride; e += blockDim.x) {
        const int lr = e / kTileStride, lc = e - lr * kTileStride;
        T v = T(0);
        if (lr < tl.h && lc < tl.w) v = x[(int64_t)(tl.r0 + lr) * d.img_w + tl.c0 + lc];
        xs[e] = v;
        gs[e] = T(0);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int *__restrict__ idx = d.idx;
    const float *__restrict__ vals = d.vals;

    for (int sl = it.slab_begin + warp; sl < it.slab_end; sl += nwarps) {
        const int64_t seg = (int64_t)sl * kSlab + lane;
        const int len = d.seg_len[seg];
        const int ray = d.seg_ray[seg];
        const T r2 = (len > 0) ? T(2) * r[ray] : T(0);
        int64_t off = d.slab_off[sl];
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        T acc = T(0);
        int k = 0;
        for (; k + 4 <= maxlen; k += 4) {
            const unsigned a0 = __ballot_sync(0xffffffffu, len > k);
            const unsigned a1 = __ballot_sync(0xffffffffu, len > k + 1);
            const unsigned a2 = __ballot_sync(0xffffffffu, len > k + 2);
            const unsigned a3 = __ballot_sync(0xffffffffu, len > k + 3);
            const int64_t o0 = off + __popc(a0 & lt);
            const int64_t o1 = off + __popc(a0) + __popc(a1 & lt);
            const int64_t o2 = off + __popc(a0) + __popc(a1) + __popc(a2 & lt);
            const int64_t o3 = off + __popc(a0) + __popc(a1) + __popc(a2) + __popc(a3 & lt);
            off += __popc(a0) + __popc(a1) + __popc(a2) + __popc(a3);
            T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
            int i0 = 0, i1 = 0, i2 = 0, i3 = 0;
            if (len > k) { v0 = load_stream<T>(vals + o0); i0 = __ldcs(idx + o0); }
            if (len > k + 1) { v1 = load_stream<T>(vals + o1); i1 = __ldcs(idx + o1); }
            if (len > k + 2) { v2 = load_stream<T>(vals + o2); i2 = __ldcs(idx + o2); }
            if (len > k + 3) { v3 = load_stream<T>(vals + o3); i3 = __ldcs(idx + o3); }
            if (len > k) { acc += v0 * xs[i0]; atomicAdd(gs + i0, v0 * r2); }
            if (len > k + 1) { acc += v1 * xs[i1]; atomicAdd(gs + i1, v1 * r2); }
            if (len > k + 2) { acc += v2 * xs[i2]; atomicAdd(gs + i2, v2 * r2); }
            if (len > k + 3) { acc += v3 * xs[i3]; atomicAdd(gs + i3, v3 * r2); }
        }
        for (; k < maxlen; ++k) {
            const unsigned a0 = __ballot_sync(0xffffffffu, len > k);
            const int64_t o0 = off + __popc(a0 & lt);
            off += __popc(a0);
            if (len > k) {
                const T v0 = load_stream<T>(vals + o0);
                const int i0 = __ldcs(idx + o0);
                acc += v0 * xs[i0];
                atomicAdd(gs + i0, v0 * r2);
            }
        }
        z_part[seg] = acc;
    }
    __syncthreads();

    T *gp = g_part + (int64_t)it.group * d.cols;
    const int npx = tl.h * tl.w;
    for (int e = threadIdx.x; e < npx; e += blockDim.x) {
        const int lr = e / tl.w, lc = e - lr * tl.w;
        gp[(int64_t)(tl.r0 + lr) * d.img_w + tl.c0 + lc] = gs[lr * kTileStride + lc];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_products(const DevLayout &d, const T *x, const T *r, T *z_part, T *g_part,
                            cudaStream_t s) {
    if (d.n_items == 0) return cudaSuccess;
    const size_t smem = 2u * kTileH * kTileStride * sizeof(T);
    products_kernel<T><<<d.n_items, 256, smem, s>>>(d, x, r, z_part, g_part);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t prepare_products_kernels() {
    cudaError_t e = cudaFuncSetAttribute(products_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2u * kTileH * kTileStride * sizeof(float)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(products_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2u * kTileH * kTileStride * sizeof(double)));
}

template cudaError_t launch_products<float>(const DevLayout &, const float *, const float *,
                                            float *, float *, cudaStream_t);
template cudaError_t launch_products<double>(const DevLayout &, const double *, const double *,
                                             double *, double *, cudaStream_t);

}  // namespace bsgdtv
