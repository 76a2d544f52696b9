// Matrix-free parallel-beam projector for the batched passes: the weights of
// A (exact intersection lengths of ray and pixel, as the seeded CSR generator
// defines them) are computed on the fly instead of being read from HBM.
//
// Geometry: pixel (srow, t) of an n x n image covers x in [t - n/2, t + 1 - n/2),
// y in [n/2 - srow - 1, n/2 - srow); ray (k, d) is the line x c + y s = u with
// c = cos(k pi / n_angles), s = sin(k pi / n_angles) (|.| < 1e-15 taken as 0)
// and u = d - (n_bins - 1)/2; row k * n_bins + d, column srow * n + t.
//
// Chord length of a line through a unit square.  In coordinates relative to
// the square's lower-left corner (x0, y0) the line reads x' c + y' s = w with
// w = u - x0 c - y0 s.  The projections of the four corners on the normal are
// 0, c, s, c + s; sorted p0 <= p1 <= p2 <= p3, with a = max(|c|, |s|) and
// b = min(|c|, |s|):
//     L(w) = (w - p0) / (a b)   for p0 <= w <= p1
//          = 1 / a              for p1 <= w <= p2
//          = (p3 - w) / (a b)   for p2 <= w <= p3,   0 outside,
// and for an axis-parallel line (b = 0) L = 1 on the half-open [p0, p3), the
// generator's rule for a ray running along a grid line.  L is as sensitive to w
// as 1/(a b) (up to ~450 for 1440 angles), so w is formed in double-float
// arithmetic (exact products by FMA, two-sums; c, s and the p_i carried as
// float pairs from FP64), which keeps every weight within ~1e-7 of the FP64
// generator's.  Every operation is an explicit round-to-nearest intrinsic, so
// the row pass and the column pass, which both call chord() with the same
// arguments for a (ray, pixel) pair, get bit-identical weights: the A of the
// row pass is exactly the transpose of the A of the column pass.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "bsgdtv_internal.h"
#include "matrix_free.h"

namespace bsgdtv {
namespace mf {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (w - p) for w = (wh, wl) and p = (ph, pl)
__device__ __forceinline__ float dd_diff(float wh, float wl, float ph, float pl) {
    return __fadd_rn(__fsub_rn(wh, ph), __fsub_rn(wl, pl));
}

__device__ __forceinline__ float chord(const AngleGeo &g, float x0, float y0, float u) {
    const float p1 = __fmul_rn(x0, g.c[0]);
    const float e1 = __fmaf_rn(x0, g.c[0], -p1);
    const float p2 = __fmul_rn(y0, g.s[0]);
    const float e2 = __fmaf_rn(y0, g.s[0], -p2);
    float t1, r1, t2, r2;
    two_sum(u, -p1, t1, r1);
    two_sum(t1, -p2, t2, r2);
    float low = __fadd_rn(r1, r2);
    low = __fsub_rn(low, __fadd_rn(e1, e2));
    low = __fmaf_rn(-x0, g.c[1], low);
    low = __fmaf_rn(-y0, g.s[1], low);
    const float d0 = dd_diff(t2, low, g.p[0], g.p[1]);   // w - p0
    const float d3 = dd_diff(g.p[6], g.p[7], t2, low);   // p3 - w
    if (g.axis) return (d0 >= 0.f && d3 > 0.f) ? 1.f : 0.f;
    if (!(d0 > 0.f) || !(d3 > 0.f)) return 0.f;
    if (dd_diff(t2, low, g.p[2], g.p[3]) < 0.f) return __fmul_rn(d0, g.inv_ab);   // w < p1
    if (dd_diff(g.p[4], g.p[5], t2, low) >= 0.f) return g.inv_a;                 // w <= p2
    return __fmul_rn(d3, g.inv_ab);
}

// Up to 3 (element, weight) candidates of one band of ray (k, d): the image
// row srow (|c| > |s|) or column t (|s| >= |c|) with index m.  Returns the
// count; weights may be 0 (pixels the line only grazes).
__device__ __forceinline__ int ray_band(const AngleGeo &g, int n, float h, float u, int m,
                                        int (&col)[3], float (&w)[3]) {
    int cnt = 0;
    const float eps = 1e-3f;
    if (!g.xmajor) {
        // row band: fy = n - 1 - srow, y in [fy - h, fy - h + 1)
        const int fy = n - 1 - m;
        const float ya = (float)fy - h, yb = ya + 1.f;
        const float xa = (u - ya * g.s[0]) / g.c[0], xb = (u - yb * g.s[0]) / g.c[0];
        int t0 = (int)floorf(fminf(xa, xb) + h - eps), t1 = (int)floorf(fmaxf(xa, xb) + h + eps);
        t0 = max(t0, 0);
        t1 = min(t1, n - 1);
        for (int t = t0; t <= t1 && cnt < 3; ++t) {
            col[cnt] = m * n + t;
            w[cnt] = chord(g, (float)t - h, ya, u);
            ++cnt;
        }
    } else {
        // column band: x in [m - h, m - h + 1)
        const float xa = (float)m - h, xb = xa + 1.f;
        const float ya = (u - xa * g.c[0]) / g.s[0], yb = (u - xb * g.c[0]) / g.s[0];
        int f0 = (int)floorf(fminf(ya, yb) + h - eps), f1 = (int)floorf(fmaxf(ya, yb) + h + eps);
        f0 = max(f0, 0);
        f1 = min(f1, n - 1);
        for (int fy = f1; fy >= f0 && cnt < 3; --fy) {   // ascending srow = n - 1 - fy
            col[cnt] = (n - 1 - fy) * n + m;
            w[cnt] = chord(g, xa, (float)fy - h, u);
            ++cnt;
        }
    }
    return cnt;
}

// Up to 3 (ray row, weight) candidates of pixel (srow, t) at angle k.
__device__ __forceinline__ int pixel_angle(const AngleGeo &g, int k, int n_bins, float off,
                                           float x0, float y0, int (&row)[3], float (&w)[3]) {
    const float q = x0 * g.c[0] + y0 * g.s[0];
    const float eps = 1e-3f;
    int d0 = (int)floorf(q + g.p[0] + off - eps), d1 = (int)floorf(q + g.p[6] + off + eps);
    d0 = max(d0, 0);
    d1 = min(d1, n_bins - 1);
    int cnt = 0;
    for (int d = d0; d <= d1 && cnt < 3; ++d) {
        row[cnt] = k * n_bins + d;
        w[cnt] = chord(g, x0, y0, (float)d - off);
        ++cnt;
    }
    return cnt;
}

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ld_keep(const float *ptr, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

constexpr int kWarps = 8;

// Compacts each lane's cnt entries (weight > 0) into stage[0 .. total) in lane
// order and pads to a multiple of G with zero weights aimed at element 0.
template <int G>
__device__ __forceinline__ int stage_entries(int2 *stage, int lane, int cnt, const int (&idx)[3],
                                             const float (&w)[3], int Bp) {
    int mine = 0;
    for (int i = 0; i < cnt; ++i) mine += (w[i] > 0.f);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - mine;
    for (int i = 0; i < cnt; ++i)
        if (w[i] > 0.f) stage[pos++] = make_int2(__float_as_int(w[i]), idx[i] * Bp);
    const int padded = (total + G - 1) / G * G;
    if (lane < padded - total) stage[total + lane] = make_int2(0, 0);
    __syncwarp();
    return padded;
}

template <int LPN>
__device__ __forceinline__ void apply_stage(const int2 *stage, int n_ent, int g, const float *vl,
                                            uint64_t pol, float4 &acc) {
    constexpr int G = 32 / LPN;
    for (int j = g; j < n_ent; j += G) {
        const int2 e = stage[j];
        const float4 x = ld_keep(vl + e.y, pol);
        const float a = __int_as_float(e.x);
        acc.x = fmaf(a, x.x, acc.x);
        acc.y = fmaf(a, x.y, acc.y);
        acc.z = fmaf(a, x.z, acc.z);
        acc.w = fmaf(a, x.w, acc.w);
    }
}

template <int LPN>
__device__ __forceinline__ void reduce_groups(float4 &acc) {
#pragma unroll
    for (int off = LPN; off < 32; off *= 2) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off);
    }
}

// Row pass: one warp per ray; lanes take 32 bands at a time, then apply the
// staged entries to the slices as the stored-matrix pass does.
// r[ray] = y[ray] - sum_pixels a x[pixel] (all slices).
template <int LPN>
__global__ void __launch_bounds__(kWarps * 32, 4)
    mf_row_kernel(const AngleGeo *__restrict__ geo, int n, int n_angles, int n_bins,
                  const float *__restrict__ X, const float *__restrict__ Y, float *__restrict__ R,
                  int Bp) {
    constexpr int G = 32 / LPN;
    __shared__ int2 stage[kWarps][3 * 32 + 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane / LPN, sl = lane % LPN;
    const int64_t ray = (int64_t)blockIdx.x * kWarps + w;
    if (ray >= (int64_t)n_angles * n_bins) return;
    const int k = (int)(ray / n_bins), d = (int)(ray % n_bins);
    const AngleGeo ag = geo[k];
    const float h = 0.5f * (float)n, u = (float)d - 0.5f * (float)(n_bins - 1);
    const uint64_t pol = l2_evict_last_policy();
    for (int c0 = 0; c0 < Bp; c0 += 4 * LPN) {
        const float *vl = X + c0 + sl * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int m0 = 0; m0 < n; m0 += 32) {
            int idx[3];
            float wt[3];
            const int m = m0 + lane;
            const int cnt = (m < n) ? ray_band(ag, n, h, u, m, idx, wt) : 0;
            const int n_ent = stage_entries<G>(stage[w], lane, cnt, idx, wt, Bp);
            apply_stage<LPN>(stage[w], n_ent, g, vl, pol, acc);
            __syncwarp();
        }
        reduce_groups<LPN>(acc);
        if (g == 0) {
            const int64_t o = ray * Bp + c0 + sl * 4;
            const float4 yv = __ldcs(reinterpret_cast<const float4 *>(Y + o));
            *reinterpret_cast<float4 *>(R + o) =
                make_float4(yv.x - acc.x, yv.y - acc.y, yv.z - acc.z, yv.w - acc.w);
        }
    }
}

// Column pass: one warp per pixel; lanes take 32 angles at a time.
// out[pixel] = base[pixel] + mu * 2 * sum_rays a r[ray] (all slices).
template <int LPN>
__global__ void __launch_bounds__(kWarps * 32, 4)
    mf_col_kernel(const AngleGeo *__restrict__ geo, int n, int n_angles, int n_bins,
                  const float *__restrict__ Rv, const float *__restrict__ base,
                  float *__restrict__ out, int Bp, float mu) {
    constexpr int G = 32 / LPN;
    __shared__ int2 stage[kWarps][3 * 32 + 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane / LPN, sl = lane % LPN;
    const int64_t px = (int64_t)blockIdx.x * kWarps + w;
    if (px >= (int64_t)n * n) return;
    const int srow = (int)(px / n), t = (int)(px % n);
    const float h = 0.5f * (float)n, off = 0.5f * (float)(n_bins - 1);
    const float x0 = (float)t - h, y0 = h - (float)srow - 1.f;
    const uint64_t pol = l2_evict_last_policy();
    for (int c0 = 0; c0 < Bp; c0 += 4 * LPN) {
        const float *vl = Rv + c0 + sl * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k0 = 0; k0 < n_angles; k0 += 32) {
            int idx[3];
            float wt[3];
            const int k = k0 + lane;
            int cnt = 0;
            if (k < n_angles) {
                const AngleGeo ag = geo[k];
                cnt = pixel_angle(ag, k, n_bins, off, x0, y0, idx, wt);
            }
            const int n_ent = stage_entries<G>(stage[w], lane, cnt, idx, wt, Bp);
            apply_stage<LPN>(stage[w], n_ent, g, vl, pol, acc);
            __syncwarp();
        }
        reduce_groups<LPN>(acc);
        if (g == 0) {
            const int64_t o = px * Bp + c0 + sl * 4;
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(base + o));
            *reinterpret_cast<float4 *>(out + o) =
                make_float4(b.x + mu * (2.f * acc.x), b.y + mu * (2.f * acc.y),
                            b.z + mu * (2.f * acc.z), b.w + mu * (2.f * acc.w));
        }
    }
}

// The row-pass weights of the listed rays, in the row pass's order (bands
// ascending, candidates ascending): one thread per ray.
__global__ void mf_weights_kernel(const AngleGeo *__restrict__ geo, int n, int n_bins,
                                  const int64_t *__restrict__ rays, int n_rays, int capacity,
                                  int32_t *__restrict__ cols, float *__restrict__ vals,
                                  int *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rays) return;
    const int k = (int)(rays[i] / n_bins), d = (int)(rays[i] % n_bins);
    const AngleGeo ag = geo[k];
    const float h = 0.5f * (float)n, u = (float)d - 0.5f * (float)(n_bins - 1);
    int cnt = 0;
    for (int m = 0; m < n; ++m) {
        int idx[3];
        float wt[3];
        const int c = ray_band(ag, n, h, u, m, idx, wt);
        for (int j = 0; j < c; ++j)
            if (wt[j] > 0.f && cnt < capacity) {
                cols[(int64_t)i * capacity + cnt] = idx[j];
                vals[(int64_t)i * capacity + cnt] = wt[j];
                ++cnt;
            }
    }
    counts[i] = cnt;
}

}  // namespace mf

// Per-angle constants from FP64 (sin/cos snapped to 0 below 1e-15, as the
// generator does).
void mf_angle_table(int n_angles, std::vector<AngleGeo> &out) {
    const double pi = 3.14159265358979323846;
    out.resize(n_angles);
    auto split = [](double v, float *hl) {
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
    };
    for (int k = 0; k < n_angles; ++k) {
        const double th = (double)k * pi / (double)n_angles;
        double c = std::cos(th), s = std::sin(th);
        if (std::fabs(c) < 1e-15) c = 0.0;
        if (std::fabs(s) < 1e-15) s = 0.0;
        double p[4] = {0.0, c, s, c + s};
        for (int i = 0; i < 4; ++i)   // sort the corner projections
            for (int j = i + 1; j < 4; ++j)
                if (p[j] < p[i]) std::swap(p[i], p[j]);
        AngleGeo &g = out[k];
        split(c, g.c);
        split(s, g.s);
        for (int i = 0; i < 4; ++i) split(p[i], g.p + 2 * i);
        const double a = std::max(std::fabs(c), std::fabs(s)), b = std::min(std::fabs(c), std::fabs(s));
        g.inv_a = (float)(1.0 / a);
        g.inv_ab = b > 0.0 ? (float)(1.0 / (a * b)) : 0.f;
        g.axis = (b == 0.0) ? 1 : 0;
        g.xmajor = (std::fabs(s) >= std::fabs(c)) ? 1 : 0;
    }
}

template <int LPN>
static cudaError_t launch_mf_lpn(bool row_pass, const MfGeometry &G, const float *v,
                                 const float *base, float *out, int Bp, float mu, cudaStream_t s) {
    const int64_t n_out = row_pass ? (int64_t)G.n_angles * G.n_bins : (int64_t)G.n * G.n;
    const dim3 grid((unsigned)((n_out + mf::kWarps - 1) / mf::kWarps)), block(mf::kWarps * 32);
    if (row_pass)
        mf::mf_row_kernel<LPN><<<grid, block, 0, s>>>(G.geo, G.n, G.n_angles, G.n_bins, v, base, out, Bp);
    else
        mf::mf_col_kernel<LPN><<<grid, block, 0, s>>>(G.geo, G.n, G.n_angles, G.n_bins, v, base, out,
                                                       Bp, mu);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mf_pass(bool row_pass, int lpn, const MfGeometry &G, const float *v,
                           const float *base, float *out, int Bp, float mu, cudaStream_t s) {
    switch (lpn) {
        case 1: return launch_mf_lpn<1>(row_pass, G, v, base, out, Bp, mu, s);
        case 2: return launch_mf_lpn<2>(row_pass, G, v, base, out, Bp, mu, s);
        case 4: return launch_mf_lpn<4>(row_pass, G, v, base, out, Bp, mu, s);
        case 8: return launch_mf_lpn<8>(row_pass, G, v, base, out, Bp, mu, s);
        case 16: return launch_mf_lpn<16>(row_pass, G, v, base, out, Bp, mu, s);
        case 32: return launch_mf_lpn<32>(row_pass, G, v, base, out, Bp, mu, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mf_weights(const MfGeometry &G, const int64_t *rays, int n_rays, int capacity,
                              int32_t *cols, float *vals, int *counts, cudaStream_t s) {
    mf::mf_weights_kernel<<<(n_rays + 127) / 128, 128, 0, s>>>(G.geo, G.n, G.n_bins, rays, n_rays,
                                                               capacity, cols, vals, counts);
    add_launches(1);
    return cudaGetLastError();
}

}  // namespace bsgdtv
