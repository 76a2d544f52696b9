// Residual update, gradient sum and gradient step of Algorithm 1, plus the
// deterministic FP64 reductions used for u_max (Theorem 1) and the objective
// (Eq. 1).  Every sum runs in a fixed order, so results do not depend on
// scheduling.
#include <cuda_runtime.h>

#include <algorithm>

#include "bsgdtv_internal.h"

namespace bsgdtv {

namespace {

constexpr int kThreads = 256;

// FP64 form (u_max, objective).
// blocks [0, nb_rows): one thread per row,  r = y - sum_j z
// blocks [nb_rows, ..): one thread per pixel, x' = x + mu sum_i g
__global__ void __launch_bounds__(kThreads)
    reduce_update64_kernel(const DevLayout d, const double *__restrict__ z_part,
                           const double *__restrict__ g_part, const double *__restrict__ y,
                           double *r_out, const double *x, double *x_out, double mu, int nb_rows) {
    if ((int)blockIdx.x < nb_rows) {
        const int64_t ray = (int64_t)blockIdx.x * kThreads + threadIdx.x;
        if (ray >= d.rows) return;
        const int e0 = d.ray_seg_ptr[ray], e1 = d.ray_seg_ptr[ray + 1];
        double acc = 0.0;
        for (int e = e0; e < e1; ++e) acc += z_part[d.ray_seg_pos[e]];
        r_out[ray] = y ? (y[ray] - acc) : acc;
    } else {
        const int64_t p = (int64_t)(blockIdx.x - nb_rows) * kThreads + threadIdx.x;
        if (p >= d.cols) return;
        double acc = 0.0;
        for (int g = 0; g < d.n_groups; ++g) acc += g_part[(int64_t)g * d.cols + p];
        x_out[p] = x ? (x[p] + mu * acc) : acc;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(float *dst, float v) {
    // non-negative floats order like their bit patterns
    atomicMax(reinterpret_cast<int *>(dst), __float_as_int(v));
}

// Sum of a row's segment partials in segment (ascending tile) order.  The
// loads of up to eight segments are issued together (predicated), so a row
// of up to eight segments (most rows) costs two dependent round trips.
__device__ __forceinline__ float row_partial_sum(const DevLayout &d, const float *__restrict__ z_part,
                                                 int64_t ray) {
    constexpr int kU = 8;
    const int e0 = d.ray_seg_ptr[ray], e1 = d.ray_seg_ptr[ray + 1];
    float acc = 0.f;
    for (int e = e0; e < e1; e += kU) {
        int pos[kU];
        float z[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) pos[k] = (e + k < e1) ? d.ray_seg_pos[e + k] : -1;
#pragma unroll
        for (int k = 0; k < kU; ++k) z[k] = (pos[k] >= 0) ? z_part[pos[k]] : 0.f;
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (e + k < e1) acc += z[k];
    }
    return acc;
}

// FP32 hot path.  Rows: r = y - sum_j z and max |r| for the next
// product pass.  Pixels: g = exact int64 sum of the groups' fixed-point tiles,
// one rounding to FP32, x' = x + mu g.
__global__ void __launch_bounds__(kThreads)
    reduce_update32_kernel(const DevLayout d, const float *__restrict__ z_part,
                           const int32_t *__restrict__ g_part, const float *__restrict__ rmax_in,
                           const float *__restrict__ y, float *r_out, float *rmax_out,
                           const float *x, float *x_out, float mu, int nb_rows) {
    pdl_wait_and_release();
    if ((int)blockIdx.x < nb_rows) {
        const int64_t ray = (int64_t)blockIdx.x * kThreads + threadIdx.x;
        float rv = 0.f;
        if (ray < d.rows) {
            rv = y[ray] - row_partial_sum(d, z_part, ray);
            r_out[ray] = rv;
        }
        if (rmax_out) {
            // one atomic per block: warp maxima through shared memory
            __shared__ float wmax[kThreads / 32];
            float m = fabsf(rv);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x < 32) {
                m = (threadIdx.x < kThreads / 32) ? wmax[threadIdx.x] : 0.f;
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (threadIdx.x == 0) atomic_max_nonneg(rmax_out, m);
            }
        }
    } else {
        const int64_t p = (int64_t)(blockIdx.x - nb_rows) * kThreads + threadIdx.x;
        if (p >= d.cols) return;
        long long acc = 0;
        for (int g = 0; g < d.n_groups; ++g) acc += g_part[(int64_t)g * d.cols + p];
        const double inv = 1.0 / (double)fixed_scale(*rmax_in, d.colsum_max);
        x_out[p] = x[p] + mu * (float)((double)acc * inv);
    }
}

__device__ __forceinline__ int block_of(const int64_t *__restrict__ bounds, int nb, int64_t v) {
    int lo = 0, hi = nb - 1;   // largest b with bounds[b] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bounds[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Stochastic variant: the same reductions restricted to the drawn blocks.
// Rows of drawn row blocks: r = y - sum of all segment partials (partials of
// undrawn pairs are the last ones computed); other rows keep r_in.  Pixels of
// drawn column blocks: x' = x + mu * (sum over groups of drawn row blocks of
// the fixed-point tiles); other pixels keep x.  clear_g: each tile value read
// is set back to 0, ready for the next pass that adds into g_part.
__global__ void __launch_bounds__(kThreads)
    reduce_subset32_kernel(const DevLayout d, const float *__restrict__ z_part,
                           int32_t *__restrict__ g_part, const float *__restrict__ rmax_in,
                           const float *__restrict__ y, const float *__restrict__ r_in,
                           float *__restrict__ r_out, float *rmax_out, const float *x,
                           float *x_out, float mu, int nb_rows, const int64_t *__restrict__ rb,
                           const int64_t *__restrict__ cb, const uint8_t *__restrict__ sel_i,
                           const uint8_t *__restrict__ sel_j, bool clear_g) {
    pdl_wait_and_release();
    if ((int)blockIdx.x < nb_rows) {
        const int64_t ray = (int64_t)blockIdx.x * kThreads + threadIdx.x;
        float rv = 0.f;
        if (ray < d.rows) {
            if (sel_i[block_of(rb, d.M, ray)]) {
                rv = y[ray] - row_partial_sum(d, z_part, ray);
            } else {
                rv = r_in[ray];
            }
            r_out[ray] = rv;
        }
        __shared__ float wmax[kThreads / 32];
        float m = fabsf(rv);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            m = (threadIdx.x < kThreads / 32) ? wmax[threadIdx.x] : 0.f;
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (threadIdx.x == 0) atomic_max_nonneg(rmax_out, m);
        }
    } else {
        const int64_t p = (int64_t)(blockIdx.x - nb_rows) * kThreads + threadIdx.x;
        if (p >= d.cols) return;
        if (!sel_j[block_of(cb, d.N, p)]) {
            x_out[p] = x[p];
            return;
        }
        long long acc = 0;
        for (int g = 0; g < d.n_groups; ++g)
            if (sel_i[d.group_block[g]]) {
                acc += g_part[(int64_t)g * d.cols + p];
                if (clear_g) g_part[(int64_t)g * d.cols + p] = 0;
            }
        const double inv = 1.0 / (double)fixed_scale(*rmax_in, d.colsum_max);
        x_out[p] = x[p] + mu * (float)((double)acc * inv);
    }
}

// Per-block sums of the block products for the test hook.
__global__ void block_sums_kernel(const DevLayout d, const float *__restrict__ z_part,
                                  const int32_t *__restrict__ g_part,
                                  const float *__restrict__ rmax_in, float *z_blocks,
                                  float *g_blocks, int N, int M, int nb_rows) {
    if ((int)blockIdx.x < nb_rows) {
        const int64_t ray = (int64_t)blockIdx.x * kThreads + threadIdx.x;
        if (ray >= d.rows) return;
        for (int j = 0; j < N; ++j) z_blocks[(int64_t)j * d.rows + ray] = 0.f;
        const int e0 = d.ray_seg_ptr[ray], e1 = d.ray_seg_ptr[ray + 1];
        int band = -1;
        float acc = 0.f;
        for (int e = e0; e < e1; ++e) {
            const int slot = d.ray_seg_pos[e];
            const int pair = d.slab_item[slot / kSlab];
            const int b = d.tiles[pair % d.n_tiles].band;
            if (b != band) {
                if (band >= 0) z_blocks[(int64_t)band * d.rows + ray] = acc;
                band = b;
                acc = 0.f;
            }
            acc += z_part[slot];
        }
        if (band >= 0) z_blocks[(int64_t)band * d.rows + ray] = acc;
    } else {
        const int64_t p = (int64_t)(blockIdx.x - nb_rows) * kThreads + threadIdx.x;
        if (p >= d.cols) return;
        const double inv = 1.0 / (double)fixed_scale(*rmax_in, d.colsum_max);
        for (int i = 0; i < M; ++i) g_blocks[(int64_t)i * d.cols + p] = 0.f;
        int blk = -1;
        long long acc = 0;
        for (int g = 0; g < d.n_groups; ++g) {
            const int b = d.group_block[g];
            if (b != blk) {
                if (blk >= 0) g_blocks[(int64_t)blk * d.cols + p] = (float)((double)acc * inv);
                blk = b;
                acc = 0;
            }
            acc += g_part[(int64_t)g * d.cols + p];
        }
        if (blk >= 0) g_blocks[(int64_t)blk * d.cols + p] = (float)((double)acc * inv);
    }
}

__global__ void absmax_kernel(const float *__restrict__ v, int64_t n, float *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wmax[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (int)(blockDim.x >> 5)) ? wmax[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomic_max_nonneg(out, m);
    }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__global__ void __launch_bounds__(kThreads)
    dot_partial_kernel(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                       double *partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        acc += b ? a[i] * b[i] : a[i] * a[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) final_sum_kernel(const double *partials, int n,
                                                             double *out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc += partials[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = acc;
}

// TV_I of an h x w FP32 image in FP64: sum of sqrt(dv^2 + dh^2) with forward
// differences, zero across the last row / column (Neumann border).
__global__ void __launch_bounds__(kThreads)
    tv_partial_kernel(const float *__restrict__ x, int h, int w, double *partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int64_t n = (int64_t)h * w;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads) {
        const int s = (int)(i / w), t = (int)(i % w);
        const double v = x[i];
        const double dv = (s + 1 < h) ? v - (double)x[i + w] : 0.0;
        const double dh = (t + 1 < w) ? v - (double)x[i + 1] : 0.0;
        acc += sqrt(dv * dv + dh * dh);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void f32_to_f64_kernel(const float *in, double *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

__global__ void fill64_kernel(double *out, double v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

// out = in / sqrt(nrm2[0])
__global__ void scale64_kernel(const double *in, const double *nrm2, double *out, int64_t n) {
    const double inv = 1.0 / sqrt(nrm2[0]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * inv;
}

__global__ void check_finite_kernel(const float *v, int64_t n, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(flag, 1);
}

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_reduce_update64(const DevLayout &d, const double *z_part, const double *g_part,
                                   const double *y, double *r_out, const double *x, double *x_out,
                                   double mu, cudaStream_t s) {
    const int nb_rows = (int)((d.rows + kThreads - 1) / kThreads);
    const int nb_cols = (int)((d.cols + kThreads - 1) / kThreads);
    reduce_update64_kernel<<<nb_rows + nb_cols, kThreads, 0, s>>>(d, z_part, g_part, y, r_out, x,
                                                                  x_out, mu, nb_rows);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_subset32(const DevLayout &d, const float *z_part, int32_t *g_part,
                                   const float *rmax_in, const float *y, const float *r_in,
                                   float *r_out, float *rmax_out, const float *x, float *x_out,
                                   float mu, const int64_t *rb, const int64_t *cb,
                                   const uint8_t *sel_i, const uint8_t *sel_j, bool clear_g,
                                   cudaStream_t s, bool pdl) {
    const int nb_rows = (int)((d.rows + kThreads - 1) / kThreads);
    const int nb_cols = (int)((d.cols + kThreads - 1) / kThreads);
    const cudaError_t e = launch_kernel(reduce_subset32_kernel, dim3(nb_rows + nb_cols), dim3(kThreads), 0,
                                        s, pdl, d, z_part, g_part, rmax_in, y, r_in, r_out, rmax_out, x,
                                        x_out, mu, nb_rows, rb, cb, sel_i, sel_j, clear_g);
    add_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_reduce_update32(const DevLayout &d, const float *z_part, const int32_t *g_part,
                                   const float *rmax_in, const float *y, float *r_out,
                                   float *rmax_out, const float *x, float *x_out, float mu,
                                   cudaStream_t s, bool pdl) {
    const int nb_rows = (int)((d.rows + kThreads - 1) / kThreads);
    const int nb_cols = (int)((d.cols + kThreads - 1) / kThreads);
    cudaError_t e = launch_kernel(reduce_update32_kernel, dim3(nb_rows + nb_cols), dim3(kThreads), 0, s,
                                  pdl, d, z_part, g_part, rmax_in, y, r_out, rmax_out, x, x_out, mu,
                                  nb_rows);
    add_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_block_sums(const DevLayout &d, const float *z_part, const int32_t *g_part,
                              const float *rmax_in, float *z_blocks, float *g_blocks,
                              cudaStream_t s) {
    const int nb_rows = (int)((d.rows + kThreads - 1) / kThreads);
    const int nb_cols = (int)((d.cols + kThreads - 1) / kThreads);
    block_sums_kernel<<<nb_rows + nb_cols, kThreads, 0, s>>>(d, z_part, g_part, rmax_in, z_blocks,
                                                             g_blocks, d.N, d.M, nb_rows);
    add_launches(1);
    return cudaGetLastError();
}

// The initial state of Algorithm 1 in one launch, from y wherever the GPU
// can read it (device memory, or page-locked host memory through its device
// address): y_dst = y (skipped when y is y_dst), r^{-1} = y, x^0 = 0, and
// max |y| as the largest bit pattern with the sign cleared.  Patterns order
// like the magnitudes, and NaN / +-Inf are exactly those >= 0x7f800000, so it
// is max |y| when y is finite and reads as Inf or NaN when it is not.  The
// last block to finish reduces the blocks' maxima, writes the result to
// rmax[0] and to *check (a word the host reads after synchronising) and puts
// the block counter back to 0.  part: kInitBlocks partial maxima and the
// counter.
__global__ void __launch_bounds__(kThreads)
    init_from_kernel(const float *__restrict__ y, float *y_dst, float *__restrict__ r0,
                     float *__restrict__ x, int64_t rows, int64_t cols, float *rmax, float *check,
                     int *part) {
    const int64_t n = rows > cols ? rows : cols;
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < rows) {
            const float v = y[i];
            if (y_dst) y_dst[i] = v;
            r0[i] = v;
            m = max(m, __float_as_int(v) & 0x7fffffff);
        }
        if (i < cols) x[i] = 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ int wmax[kThreads / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) m = max(m, wmax[k]);
        part[blockIdx.x] = m;
        __threadfence();
        last = atomicAdd(part + kInitBlocks, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    m = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x)
        m = max(m, reinterpret_cast<volatile int *>(part)[k]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) m = max(m, wmax[k]);
        *rmax = __int_as_float(m);
        *check = __int_as_float(m);
        part[kInitBlocks] = 0;
    }
}

cudaError_t launch_init_from(const float *y, float *y_dst, float *r0, float *x, int64_t rows,
                             int64_t cols, float *rmax, float *check, int *part, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(kInitBlocks, std::max<int64_t>(1, (std::max(rows, cols) + kThreads - 1) / kThreads));
    init_from_kernel<<<grid, kThreads, 0, s>>>(y, y == y_dst ? nullptr : y_dst, r0, x, rows, cols, rmax,
                                               check, part);
    add_launches(1);
    return cudaGetLastError();
}

// dst[0 .. n) = src (dst: device memory, or page-locked host memory through
// its device address).
__global__ void __launch_bounds__(kThreads) copy_out_kernel(const float *__restrict__ src,
                                                            float *__restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t launch_copy_out(const float *src, float *dst, int64_t n, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(kInitBlocks, std::max<int64_t>(1, (n + kThreads - 1) / kThreads));
    copy_out_kernel<<<grid, kThreads, 0, s>>>(src, dst, n);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float *v, int64_t n, float *out, cudaStream_t s) {
    absmax_kernel<<<grid_for(n), kThreads, 0, s>>>(v, n, out);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dot(const double *a, const double *b, int64_t n, double *partials, double *out,
                       cudaStream_t s) {
    const int g = std::min(grid_for(n), kDotPartials);
    dot_partial_kernel<<<g, kThreads, 0, s>>>(a, b, n, partials);
    final_sum_kernel<<<1, kThreads, 0, s>>>(partials, g, out);
    add_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_tv64(const float *x, int h, int w, double *partials, double *out,
                        cudaStream_t s) {
    const int g = std::min(grid_for((int64_t)h * w), kDotPartials);
    tv_partial_kernel<<<g, kThreads, 0, s>>>(x, h, w, partials);
    final_sum_kernel<<<1, kThreads, 0, s>>>(partials, g, out);
    add_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float *in, double *out, int64_t n, cudaStream_t s) {
    f32_to_f64_kernel<<<grid_for(n), kThreads, 0, s>>>(in, out, n);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill64(double *out, double v, int64_t n, cudaStream_t s) {
    fill64_kernel<<<grid_for(n), kThreads, 0, s>>>(out, v, n);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scale64(const double *in, const double *nrm2, double *out, int64_t n,
                           cudaStream_t s) {
    scale64_kernel<<<grid_for(n), kThreads, 0, s>>>(in, nrm2, out, n);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *v, int64_t n, int *flag, cudaStream_t s) {
    check_finite_kernel<<<grid_for(n), kThreads, 0, s>>>(v, n, flag);
    add_launches(1);
    return cudaGetLastError();
}

}  // namespace bsgdtv
