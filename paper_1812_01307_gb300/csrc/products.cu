// Fused block products of Algorithm 1 (one pass over A).
//
// For every work item (row group G inside a row block I_i, pixel tile T inside
// a column band J_j) a CTA computes, from a single read of the item's
// nonzeros,
//   z partial:  sum over the row's nonzeros in T of a * x          (z^j_{I_i})
//   g partial:  sum over G's rows of 2 a r_row, for each pixel of T (g-hat^i_{J_j})
// where r is the residual of the previous epoch (the paper's stale gradient,
// Eq. 3).  x_T is staged in shared memory and the g tile accumulates there.
//
// GPU mapping: persistent CTAs (two per SM) take work items from a global
// counter, largest items first (the counter resets itself at kernel exit).
// Inside an item each warp takes slabs of 32 row segments from a shared
// counter, one lane per segment, so a segment's z
// partial stays in a register.  A slab is read in 16-byte column groups (four
// consecutive nonzeros of each lane's segment per load, coalesced across the
// warp) with the loads of the next groups in flight while the current one is
// used (four groups of 32 B per lane for FP32 weights + 32-bit indices, so each
// warp keeps ~4 KB of A in flight; three or four of 16 B for 16-bit indices).
#include <cuda_runtime.h>

#include <algorithm>

#include "bsgdtv_internal.h"
#include "products_common.cuh"

namespace bsgdtv {

namespace {

using namespace prod;

// FP32 weights with 32-bit indices.  T: type of x, r, z (float or double); G:
// shared g tile (int fixed point or double); kAdd: items may be shares of a
// (group, tile) pair and add their g tile into g_part (int32 atomics) instead
// of storing it.  The 16-bit formats have their own kernel in products_fmt.cu:
// sharing this translation unit with it made this kernel about 10 % slower on
// GB300.
template <typename T, typename G, bool kAdd>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    products_f32_kernel(const DevLayout d, const T *__restrict__ x, const T *__restrict__ r,
                    const float *__restrict__ rmax_in, float *__restrict__ rmax_clear,
                    T *__restrict__ z_part, G *__restrict__ g_part, int *__restrict__ item_ctr) {
    // column groups in flight per lane: 4 x 32 B for the FP32 path (64
    // registers, no spills; measured 0.184 -> 0.168 -> 0.166 ms going from 2
    // to 3 to 4 on the 512 x 512 workload), 2 for the FP64 path
    constexpr int kDepth = sizeof(T) == 4 ? 4 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    G *gs = reinterpret_cast<G *>(xs + kTileWords);
    __shared__ int s_item, s_next;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const float4 *__restrict__ V4 = reinterpret_cast<const float4 *>(d.vals);
    const int4 *__restrict__ I4 = reinterpret_cast<const int4 *>(d.idx);
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
            const int ng = (len + kGroup - 1) / kGroup;
            const T r2 = (len > 0) ? T(2) * r[ray] * scale : T(0);
            const int64_t base = d.slab_off[sl] / kGroup;
            const float4 *V = V4 + base;
            const int4 *I = I4 + base;
            const int maxg = __reduce_max_sync(0xffffffffu, ng);
            // column groups kk .. kk + kDepth - 1 in flight: a queue of
            // registers shifted by one group per iteration (fully unrolled)
            int off = 0;
            float4 v[kDepth];
            int4 ix[kDepth];
#pragma unroll
            for (int k = 0; k < kDepth; ++k) {
                v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                ix[k] = make_int4(0, 0, 0, 0);
                const unsigned a = __ballot_sync(0xffffffffu, ng > k);
                const int p = off + __popc(a & lt);
                off += __popc(a);
                if (ng > k) { v[k] = __ldcs(V + p); ix[k] = __ldcs(I + p); }
            }
            T acc = T(0);
            for (int kk = 0; kk < maxg; ++kk) {
                float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
                int4 in = make_int4(0, 0, 0, 0);
                const unsigned a = __ballot_sync(0xffffffffu, ng > kk + kDepth);
                const int p = off + __popc(a & lt);
                off += __popc(a);
                if (ng > kk + kDepth) { vn = __ldcs(V + p); in = __ldcs(I + p); }
                if (ng > kk) use_group(v[0], ix[0], r2, xs, gs, acc);
#pragma unroll
                for (int k = 0; k < kDepth - 1; ++k) {
                    v[k] = v[k + 1];
                    ix[k] = ix[k + 1];
                }
                v[kDepth - 1] = vn;
                ix[kDepth - 1] = in;
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
            G *dst = gp + (int64_t)(tl.r0 + lr) * d.img_w + tl.c0 + lc;
            if constexpr (kAdd) atomicAdd(dst, gs[lr * kTileStride + lc]);
            else *dst = gs[lr * kTileStride + lc];
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

}  // namespace

static cudaError_t launch_p32_plain(const DevLayout &d, const float *x, const float *r,
                                    const float *rmax_in, float *rmax_clear, float *z_part,
                                    int32_t *g_part, cudaStream_t s, bool pdl) {
    const size_t smem = kTileWords * (sizeof(float) + sizeof(int));
    const int grid = std::min(d.n_items, kCtasPerSm * std::max(d.n_sms, 1));
    return launch_kernel(products_f32_kernel<float, int, false>, dim3(grid), dim3(kThreads), smem, s, pdl,
                         d, x, r, rmax_in, rmax_clear, z_part, g_part, d.item_ctr);
}

static cudaError_t launch_p64_plain(const DevLayout &d, const double *x, const double *r,
                                    double *z_part, double *g_part, cudaStream_t s) {
    const size_t smem = 2u * kTileWords * sizeof(double);
    const int grid = std::min(d.n_items, kCtasPerSm * std::max(d.n_sms, 1));
    return launch_kernel(products_f32_kernel<double, double, false>, dim3(grid), dim3(kThreads), smem, s,
                         false, d, x, r, (const float *)nullptr, (float *)nullptr, z_part, g_part,
                         d.item_ctr);
}

cudaError_t launch_products32(const DevLayout &d, const float *x, const float *r,
                              const float *rmax_in, float *rmax_clear, float *z_part,
                              int32_t *g_part, cudaStream_t s, bool pdl) {
    if (d.n_items == 0) return cudaSuccess;
    const cudaError_t e =
        d.fmt == BSGDTV_FMT_F32_I32
            ? launch_p32_plain(d, x, r, rmax_in, rmax_clear, z_part, g_part, s, pdl)
            : launch_products32_fmt(d, x, r, rmax_in, rmax_clear, z_part, g_part, s, pdl);
    add_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_products32_add(const DevLayout &d, const float *x, const float *r,
                                  const float *rmax_in, float *rmax_clear, float *z_part,
                                  int32_t *g_part, cudaStream_t s, bool pdl) {
    if (d.n_items == 0) return cudaSuccess;
    if (d.fmt != BSGDTV_FMT_F32_I32) return cudaErrorInvalidValue;
    const size_t smem = kTileWords * (sizeof(float) + sizeof(int));
    const int grid = std::min(d.n_items, kCtasPerSm * std::max(d.n_sms, 1));
    const cudaError_t e = launch_kernel(products_f32_kernel<float, int, true>, dim3(grid), dim3(kThreads),
                                        smem, s, pdl, d, x, r, rmax_in, rmax_clear, z_part, g_part,
                                        d.item_ctr);
    add_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_products64(const DevLayout &d, const double *x, const double *r, double *z_part,
                              double *g_part, cudaStream_t s) {
    if (d.n_items == 0) return cudaSuccess;
    const cudaError_t e = d.fmt == BSGDTV_FMT_F32_I32
                              ? launch_p64_plain(d, x, r, z_part, g_part, s)
                              : launch_products64_fmt(d, x, r, z_part, g_part, s);
    add_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t prepare_products_kernels() {
    cudaError_t e = cudaFuncSetAttribute(products_f32_kernel<float, int, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTileWords * (sizeof(float) + sizeof(int))));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(products_f32_kernel<float, int, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kTileWords * (sizeof(float) + sizeof(int))));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(products_f32_kernel<double, double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2u * kTileWords * sizeof(double)));
    if (e == cudaSuccess) e = prepare_products_fmt_kernels();
    return e;
}

}  // namespace bsgdtv
