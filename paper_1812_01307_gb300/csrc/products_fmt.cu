// Fused block products of Algorithm 1 for A stored with 16-bit tile-local
// indices and FP32, binary16 or bfloat16 weights (see products.cu for the
// work decomposition; this kernel differs only in how a column group is
// loaded and decoded: four entries with FP32 weights, eight with 16-bit
// weights).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bsgdtv_internal.h"
#include "products_common.cuh"

namespace bsgdtv {

namespace {

using namespace prod;

// Stored formats of one column group (kN entries of one lane's segment):
// FP32 weights with 16-bit indices in groups of 4 (16 + 8 bytes per lane),
// 16-bit weights with 16-bit indices in groups of 8 (16 + 16 bytes per lane:
// the registers of one FP32 + 32-bit-index group for twice the entries).
// kDepth: column groups loaded ahead of the one in use.
template <int FMT> struct GroupFmt;
template <> struct GroupFmt<BSGDTV_FMT_F32_I16> {
    static constexpr int kN = 4;
    static constexpr int kDepth = 4;
    using VT = float4;
    using IT = uint2;   // four 16-bit indices
    static __device__ __forceinline__ void decode(const VT &v, const IT &i, float (&w)[kN], int (&k)[kN]) {
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
        k[0] = (int)(i.x & 0xFFFFu);
        k[1] = (int)(i.x >> 16);
        k[2] = (int)(i.y & 0xFFFFu);
        k[3] = (int)(i.y >> 16);
    }
};
__device__ __forceinline__ void unpack_idx8(const uint4 &i, int (&k)[8]) {
    const unsigned u[4] = {i.x, i.y, i.z, i.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        k[2 * t] = (int)(u[t] & 0xFFFFu);
        k[2 * t + 1] = (int)(u[t] >> 16);
    }
}
template <> struct GroupFmt<BSGDTV_FMT_F16_I16> {
    static constexpr int kN = 8;
    static constexpr int kDepth = 4;
    using VT = uint4;   // eight binary16 weights
    using IT = uint4;   // eight 16-bit indices
    static __device__ __forceinline__ void decode(const VT &v, const IT &i, float (&w)[kN], int (&k)[kN]) {
        const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&u[t]));
            w[2 * t] = f.x;
            w[2 * t + 1] = f.y;
        }
        unpack_idx8(i, k);
    }
};
template <> struct GroupFmt<BSGDTV_FMT_BF16_I16> {
    static constexpr int kN = 8;
    static constexpr int kDepth = 4;
    using VT = uint4;   // eight bfloat16 weights: the upper halves of FP32 values
    using IT = uint4;
    static __device__ __forceinline__ void decode(const VT &v, const IT &i, float (&w)[kN], int (&k)[kN]) {
        const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            w[2 * t] = __uint_as_float(u[t] << 16);
            w[2 * t + 1] = __uint_as_float(u[t] & 0xFFFF0000u);
        }
        unpack_idx8(i, k);
    }
};

// Accumulation of one column group (see products_common.cuh): z partial in a
// register, the A^T r contributions into the shared g tile.
template <int N>
__device__ __forceinline__ void use_entries(const float (&w)[N], const int (&k)[N], const float r2s,
                                            const float *xs, int *gs, float &acc) {
#pragma unroll
    for (int t = 0; t < N; ++t) {
        acc = fmaf(w[t], xs[k[t]], acc);
        atomicAdd(gs + k[t], __float2int_rn(w[t] * r2s));
    }
}
template <int N>
__device__ __forceinline__ void use_entries(const float (&w)[N], const int (&k)[N], const double r2,
                                            const double *xs, double *gs, double &acc) {
#pragma unroll
    for (int t = 0; t < N; ++t) {
        acc += (double)w[t] * xs[k[t]];
        atomicAdd(gs + k[t], (double)w[t] * r2);
    }
}

template <typename X>
__device__ __forceinline__ X zero_of();
template <> __device__ __forceinline__ float4 zero_of<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ uint2 zero_of<uint2>() { return make_uint2(0u, 0u); }
template <> __device__ __forceinline__ uint4 zero_of<uint4>() { return make_uint4(0u, 0u, 0u, 0u); }

// T: type of x, r, z (float or double); G: shared g tile (int fixed point or
// double); FMT: stored weight / index format.
template <typename T, typename G, int FMT>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    products_kernel(const DevLayout d, const T *__restrict__ x, const T *__restrict__ r,
                    const float *__restrict__ rmax_in, float *__restrict__ rmax_clear,
                    T *__restrict__ z_part, G *__restrict__ g_part, int *__restrict__ item_ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    G *gs = reinterpret_cast<G *>(xs + kTileWords);
    __shared__ int s_item, s_next;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    using VT = typename GroupFmt<FMT>::VT;
    using IT = typename GroupFmt<FMT>::IT;
    const VT *__restrict__ V4 = reinterpret_cast<const VT *>(d.vals);
    const IT *__restrict__ I4 = reinterpret_cast<const IT *>(d.idx);
    pdl_wait_and_release();
    // 2 r scaled to fixed point (FP32 path) or plain 2 r (FP64 path)
    const T scale = rmax_in ? (T)fixed_scale(*rmax_in, d.colsum_max) : T(1);
    if (rmax_clear && blockIdx.x == 0 && threadIdx.x == 0) *rmax_clear = 0.f;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(item_ctr, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= d.n_items) break;
        const WorkItem it = d.items[item];
        const Tile tl = d.tiles[it.tile];

        for (int e = threadIdx.x; e < kTileWords; e += kThreads) {
            const int lr = e / kTileStride, lc = e - lr * kTileStride;
            T v = T(0);
            if (e < kPadBase && lr < tl.h && lc < tl.w)
                v = x[(int64_t)(tl.r0 + lr) * d.img_w + tl.c0 + lc];
            xs[e] = v;
            gs[e] = G(0);
        }
        if (threadIdx.x == 0) s_next = it.slab_begin + kWarps;
        __syncthreads();

        int sl = it.slab_begin + warp;
        while (sl < it.slab_end) {
            const int64_t seg = (int64_t)sl * kSlab + lane;
            const int len = d.seg_len[seg];
            const int ray = d.seg_ray[seg];
            constexpr int kN = GroupFmt<FMT>::kN;
            const int ng = (len + kN - 1) / kN;
            const T r2 = (len > 0) ? T(2) * r[ray] * scale : T(0);
            const int64_t base = d.slab_off[sl] / kN;
            const VT *V = V4 + base;
            const IT *I = I4 + base;
            const int maxg = __reduce_max_sync(0xffffffffu, ng);
            // kDepth column groups in flight ahead of the one in use
            constexpr int kDepth = sizeof(T) == 4 ? GroupFmt<FMT>::kDepth : 2;   // FP64: setup only
            int off = 0;
            T acc = T(0);
            {
                VT vq[kDepth];
                IT iq[kDepth];
#pragma unroll
                for (int t = 0; t < kDepth; ++t) {
                    vq[t] = zero_of<VT>();
                    iq[t] = zero_of<IT>();
                    const unsigned a = __ballot_sync(0xffffffffu, ng > t);
                    const int p = off + __popc(a & lt);
                    off += __popc(a);
                    if (ng > t) { vq[t] = __ldcs(V + p); iq[t] = __ldcs(I + p); }
                }
                for (int kk = 0; kk < maxg; ++kk) {
                    VT vn = zero_of<VT>();
                    IT in_ = zero_of<IT>();
                    const unsigned a = __ballot_sync(0xffffffffu, ng > kk + kDepth);
                    const int p = off + __popc(a & lt);
                    off += __popc(a);
                    if (ng > kk + kDepth) { vn = __ldcs(V + p); in_ = __ldcs(I + p); }
                    if (ng > kk) {
                        float w[kN];
                        int k[kN];
                        GroupFmt<FMT>::decode(vq[0], iq[0], w, k);
                        use_entries<kN>(w, k, r2, xs, gs, acc);
                    }
#pragma unroll
                    for (int t = 0; t + 1 < kDepth; ++t) {
                        vq[t] = vq[t + 1];
                        iq[t] = iq[t + 1];
                    }
                    vq[kDepth - 1] = vn;
                    iq[kDepth - 1] = in_;
                }
            }
            z_part[seg] = acc;
            int nx = 0;
            if (lane == 0) nx = atomicAdd(&s_next, 1);
            sl = __shfl_sync(0xffffffffu, nx, 0);
        }
        __syncthreads();

        G *gp = g_part + (int64_t)it.group * d.cols;
        const int npx = tl.h * tl.w;
        for (int e = threadIdx.x; e < npx; e += kThreads) {
            const int lr = e / tl.w, lc = e - lr * tl.w;
            gp[(int64_t)(tl.r0 + lr) * d.img_w + tl.c0 + lc] = gs[lr * kTileStride + lc];
        }
        __syncthreads();
    }
    // The last CTA out resets both counters for the next launch: every CTA
    // has made its final claim on item_ctr[0] before it counts itself out.
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(item_ctr + 1, 1) == (int)gridDim.x - 1) {
            item_ctr[0] = 0;
            item_ctr[1] = 0;
            __threadfence();
        }
    }
}

template <int FMT>
cudaError_t launch_p32(const DevLayout &d, const float *x, const float *r, const float *rmax_in,
                       float *rmax_clear, float *z_part, int32_t *g_part, cudaStream_t s, bool pdl) {
    const size_t smem = kTileWords * (sizeof(float) + sizeof(int));
    const int grid = std::min(d.n_items, kCtasPerSm * std::max(d.n_sms, 1));
    return launch_kernel(products_kernel<float, int, FMT>, dim3(grid), dim3(kThreads), smem, s, pdl,
                         d, x, r, rmax_in, rmax_clear, z_part, g_part, d.item_ctr);
}

template <int FMT>
cudaError_t launch_p64(const DevLayout &d, const double *x, const double *r, double *z_part,
                       double *g_part, cudaStream_t s) {
    const size_t smem = 2u * kTileWords * sizeof(double);
    const int grid = std::min(d.n_items, kCtasPerSm * std::max(d.n_sms, 1));
    return launch_kernel(products_kernel<double, double, FMT>, dim3(grid), dim3(kThreads), smem, s,
                         false, d, x, r, (const float *)nullptr, (float *)nullptr, z_part, g_part,
                         d.item_ctr);
}

template <int FMT>
cudaError_t prepare_fmt() {
    cudaError_t e = cudaFuncSetAttribute(products_kernel<float, int, FMT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTileWords * (sizeof(float) + sizeof(int))));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(products_kernel<double, double, FMT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2u * kTileWords * sizeof(double)));
}

}  // namespace

cudaError_t launch_products32_fmt(const DevLayout &d, const float *x, const float *r,
                                  const float *rmax_in, float *rmax_clear, float *z_part,
                                  int32_t *g_part, cudaStream_t s, bool pdl) {
    switch (d.fmt) {
        case BSGDTV_FMT_F32_I16:
            return launch_p32<BSGDTV_FMT_F32_I16>(d, x, r, rmax_in, rmax_clear, z_part, g_part, s, pdl);
        case BSGDTV_FMT_F16_I16:
            return launch_p32<BSGDTV_FMT_F16_I16>(d, x, r, rmax_in, rmax_clear, z_part, g_part, s, pdl);
        case BSGDTV_FMT_BF16_I16:
            return launch_p32<BSGDTV_FMT_BF16_I16>(d, x, r, rmax_in, rmax_clear, z_part, g_part, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_products64_fmt(const DevLayout &d, const double *x, const double *r,
                                  double *z_part, double *g_part, cudaStream_t s) {
    switch (d.fmt) {
        case BSGDTV_FMT_F32_I16: return launch_p64<BSGDTV_FMT_F32_I16>(d, x, r, z_part, g_part, s);
        case BSGDTV_FMT_F16_I16: return launch_p64<BSGDTV_FMT_F16_I16>(d, x, r, z_part, g_part, s);
        case BSGDTV_FMT_BF16_I16: return launch_p64<BSGDTV_FMT_BF16_I16>(d, x, r, z_part, g_part, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_products_fmt_kernels() {
    cudaError_t e = prepare_fmt<BSGDTV_FMT_F32_I16>();
    if (e == cudaSuccess) e = prepare_fmt<BSGDTV_FMT_F16_I16>();
    if (e == cudaSuccess) e = prepare_fmt<BSGDTV_FMT_BF16_I16>();
    return e;
}

}  // namespace bsgdtv
