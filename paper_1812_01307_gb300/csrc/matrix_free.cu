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

#include <algorithm>
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
// row srow (|c| > |s|) or column t (|s| >= |c|) with index m, restricted to
// the image rows [s_lo, s_hi) (all rows by default).  Returns the count;
// weights may be 0 (pixels the line only grazes).
__device__ __forceinline__ int ray_band(const AngleGeo &g, int n, float h, float u, int m,
                                        int (&col)[3], float (&w)[3], int s_lo = 0, int s_hi = -1) {
    if (s_hi < 0) s_hi = n;
    int cnt = 0;
    const float eps = 1e-3f;
    if (!g.xmajor) {
        // row band: fy = n - 1 - srow, y in [fy - h, fy - h + 1)
        const int fy = n - 1 - m;
        const float ya = (float)fy - h, yb = ya + 1.f;
        const float xa = (u - ya * g.s[0]) * g.inv_c, xb = (u - yb * g.s[0]) * g.inv_c;
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
        const float ya = (u - xa * g.c[0]) * g.inv_s, yb = (u - xb * g.c[0]) * g.inv_s;
        int f0 = (int)floorf(fminf(ya, yb) + h - eps), f1 = (int)floorf(fmaxf(ya, yb) + h + eps);
        f0 = max(f0, n - s_hi);        // rows of the stripe [s_lo, s_hi) only
        f1 = min(f1, n - 1 - s_lo);
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

constexpr int kThreads = 256;

// Bands [m_lo, m_hi] of ray (k, d) that can hold pixels of the image rows
// [s_lo, s_hi) (y in [h - s_hi, h - s_lo)): the other coordinate along the
// band must lie within the image, or the stripe, widened by one pixel.
__device__ __forceinline__ void band_range(const AngleGeo &g, int n, float h, float u, int s_lo,
                                           int s_hi, int &m_lo, int &m_hi) {
    const float lim = 2.f * (float)n;   // keeps the float -> int conversions in range
    const float y_bot = h - (float)s_hi - 1.f, y_top = h - (float)s_lo + 1.f;
    if (!g.xmajor) {
        // bands are rows of the stripe; x(y) = (u - y s) / c within [-h - 1, h + 1]
        m_lo = s_lo;
        m_hi = s_hi - 1;
        if (g.s[0] == 0.f) {
            if (fabsf(u * g.inv_c) > h + 1.f) m_hi = -1;
            return;
        }
        const float ya = (u - (h + 1.f) * g.c[0]) * g.inv_s, yb = (u + (h + 1.f) * g.c[0]) * g.inv_s;
        const float y0 = fmaxf(fminf(ya, yb) - 1.f, -lim), y1 = fminf(fmaxf(ya, yb) + 1.f, lim);
        // row srow holds y in [h - srow - 1, h - srow)
        m_lo = max(m_lo, (int)floorf(h - y1) - 1);
        m_hi = min(m_hi, (int)ceilf(h - y0) + 1);
    } else {
        // bands are columns; y(x) = (u - x c) / s within the stripe
        m_lo = 0;
        m_hi = n - 1;
        if (g.c[0] == 0.f) {
            const float y = u * g.inv_s;
            if (y < y_bot || y > y_top) m_hi = -1;
            return;
        }
        const float xa = (u - y_top * g.s[0]) * g.inv_c, xb = (u - y_bot * g.s[0]) * g.inv_c;
        const float x0 = fmaxf(fminf(xa, xb) - 1.f, -lim), x1 = fminf(fmaxf(xa, xb) + 1.f, lim);
        m_lo = max(m_lo, (int)floorf(x0 + h) - 1);
        m_hi = min(m_hi, (int)ceilf(x1 + h) + 1);
    }
}

__device__ __forceinline__ void fma4(float a, const float4 &x, float4 &acc) {
    acc.x = fmaf(a, x.x, acc.x);
    acc.y = fmaf(a, x.y, acc.y);
    acc.z = fmaf(a, x.z, acc.z);
    acc.w = fmaf(a, x.w, acc.w);
}

// Candidates of this lane's band / angle go to its three mailbox slots as
// (weight bits, element offset), zero where there is no entry; the LPN lanes
// of an element then read the group's slots in order and each applies every
// entry to its own 4 slices.
__device__ __forceinline__ void post(int2 (&slot)[3], const int (&idx)[3], const float (&wt)[3],
                                     int Bp) {
#pragma unroll
    for (int e = 0; e < 3; ++e)
        slot[e] = wt[e] > 0.f ? make_int2(__float_as_int(wt[e]), idx[e] * Bp) : make_int2(0, 0);
}

template <int LPN>
__device__ __forceinline__ void apply_group(const int2 (*box)[3], int grp, const float *vl,
                                            uint64_t pol, float4 &acc) {
#pragma unroll
    for (int src = 0; src < LPN; ++src)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int2 t = box[grp * LPN + src][e];
            if (t.x != 0) fma4(__int_as_float(t.x), ld_keep(vl + t.y, pol), acc);
        }
}

// Row pass over the image rows [s_lo, s_hi): LPN lanes per ray, 32/LPN
// neighbouring rays (bins) per warp.  The lanes of a ray take its bands in
// turn (lane j: bands m = j mod LPN of each round), post their entries, and
// every lane applies all of them to its 4 slices of the chunk:
// r[ray] = (first ? y[ray] : r[ray]) - sum over bands ascending, then
// candidates ascending, of a x[pixel] (the same order for every LPN).
template <int LPN>
__global__ void __launch_bounds__(kThreads)
    mf_row_kernel(const AngleGeo *__restrict__ geo, int n, int n_angles, int n_bins,
                  const float *__restrict__ X, const float *__restrict__ Y, float *__restrict__ R,
                  int Bp, int s_lo, int s_hi, int first) {
    constexpr int EPW = 32 / LPN;
    __shared__ int2 box[kThreads / 32][32][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / LPN, j = lane % LPN;
    const int64_t ray = ((int64_t)blockIdx.x * (kThreads / 32) + w) * EPW + grp;
    const bool valid = ray < (int64_t)n_angles * n_bins;
    const int k = valid ? (int)(ray / n_bins) : 0, d = valid ? (int)(ray % n_bins) : 0;
    const AngleGeo g = geo[k];
    const float h = 0.5f * (float)n, u = (float)d - 0.5f * (float)(n_bins - 1);
    const uint64_t pol = l2_evict_last_policy();
    int m_lo = 0, m_hi = -1;
    if (valid) band_range(g, n, h, u, s_lo, s_hi, m_lo, m_hi);
    const int w_lo = __reduce_min_sync(0xffffffffu, m_hi >= m_lo ? m_lo : n);
    const int w_hi = __reduce_max_sync(0xffffffffu, m_hi);
    for (int c0 = 0; c0 < Bp; c0 += 4 * LPN) {
        const float *vl = X + c0 + j * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int mb = w_lo; mb <= w_hi; mb += LPN) {
            const int m = mb + j;
            int idx[3] = {0, 0, 0};
            float wt[3] = {0.f, 0.f, 0.f};
            if (m >= m_lo && m <= m_hi) ray_band(g, n, h, u, m, idx, wt, s_lo, s_hi);
            post(box[w][lane], idx, wt, Bp);
            __syncwarp();
            apply_group<LPN>(box[w], grp, vl, pol, acc);
            __syncwarp();
        }
        if (valid) {
            const int64_t o = ray * Bp + c0 + j * 4;
            const float4 yv = first ? __ldcs(reinterpret_cast<const float4 *>(Y + o))
                                    : *reinterpret_cast<const float4 *>(R + o);
            *reinterpret_cast<float4 *>(R + o) =
                make_float4(yv.x - acc.x, yv.y - acc.y, yv.z - acc.z, yv.w - acc.w);
        }
    }
}

// Column pass over the angles [k_lo, k_hi): LPN lanes per pixel, 32/LPN
// neighbouring pixels of an image row per warp; lane j takes the angles
// k = j mod LPN of each round.  out[pixel] = (first ? base : out)[pixel] +
// mu * 2 * sum over angles ascending, then bins ascending, of a r[ray].
template <int LPN>
__global__ void __launch_bounds__(kThreads)
    mf_col_kernel(const AngleGeo *__restrict__ geo, int n, int n_angles, int n_bins,
                  const float *__restrict__ Rv, const float *base, float *out, int Bp, float mu,
                  int k_lo, int k_hi, int first) {
    constexpr int EPW = 32 / LPN;
    __shared__ int2 box[kThreads / 32][32][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / LPN, j = lane % LPN;
    const int64_t px = ((int64_t)blockIdx.x * (kThreads / 32) + w) * EPW + grp;
    const bool valid = px < (int64_t)n * n;
    const int srow = valid ? (int)(px / n) : 0, t = valid ? (int)(px % n) : 0;
    const float h = 0.5f * (float)n, off = 0.5f * (float)(n_bins - 1);
    const float x0 = (float)t - h, y0 = h - (float)srow - 1.f;
    const uint64_t pol = l2_evict_last_policy();
    for (int c0 = 0; c0 < Bp; c0 += 4 * LPN) {
        const float *vl = Rv + c0 + j * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int kb = k_lo; kb < k_hi; kb += LPN) {
            const int k = kb + j;
            int idx[3] = {0, 0, 0};
            float wt[3] = {0.f, 0.f, 0.f};
            if (valid && k < k_hi) pixel_angle(geo[k], k, n_bins, off, x0, y0, idx, wt);
            post(box[w][lane], idx, wt, Bp);
            __syncwarp();
            apply_group<LPN>(box[w], grp, vl, pol, acc);
            __syncwarp();
        }
        if (valid) {
            const int64_t o = px * Bp + c0 + j * 4;
            const float4 b = *reinterpret_cast<const float4 *>((first ? base : out) + o);
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
        g.inv_c = c != 0.0 ? (float)(1.0 / c) : 0.f;
        g.inv_s = s != 0.0 ? (float)(1.0 / s) : 0.f;
        g.pad[0] = g.pad[1] = 0;
        g.axis = (b == 0.0) ? 1 : 0;
        g.xmajor = (std::fabs(s) >= std::fabs(c)) ? 1 : 0;
    }
}

// Gathered vectors are split so that the slice vectors one launch gathers
// (rows of x for the row pass, angles of r for the column pass) fit about
// half of the L2: beyond that every angle streams the whole vector from HBM.
constexpr int64_t kGatherBudget = 48ll << 20;

template <int LPN>
static cudaError_t launch_mf_lpn(bool row_pass, const MfGeometry &G, const float *v,
                                 const float *base, float *out, int Bp, float mu, cudaStream_t s) {
    const int64_t n_out = row_pass ? (int64_t)G.n_angles * G.n_bins : (int64_t)G.n * G.n;
    const int64_t per_block = (int64_t)(mf::kThreads / 32) * (32 / LPN);
    const dim3 grid((unsigned)((n_out + per_block - 1) / per_block)), block(mf::kThreads);
    const int64_t unit = 4ll * Bp * (row_pass ? G.n : G.n_bins);   // bytes of one image row / angle
    const int total = row_pass ? G.n : G.n_angles;
    const int step = (int)std::max<int64_t>(1, std::min<int64_t>(total, kGatherBudget / unit));
    for (int lo = 0; lo < total; lo += step) {
        const int hi = std::min(total, lo + step), first = (lo == 0);
        if (row_pass)
            mf::mf_row_kernel<LPN><<<grid, block, 0, s>>>(G.geo, G.n, G.n_angles, G.n_bins, v, base,
                                                           out, Bp, lo, hi, first);
        else
            mf::mf_col_kernel<LPN><<<grid, block, 0, s>>>(G.geo, G.n, G.n_angles, G.n_bins, v, base,
                                                           out, Bp, mu, lo, hi, first);
        add_launches(1);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_mf_pass(bool row_pass, int Bp, const MfGeometry &G, const float *v,
                           const float *base, float *out, float mu, cudaStream_t s) {
    // LPN lanes of 4 slices each per element; strides above 32 go in chunks of 32
    switch (Bp) {
        case 4: return launch_mf_lpn<1>(row_pass, G, v, base, out, Bp, mu, s);
        case 8: return launch_mf_lpn<2>(row_pass, G, v, base, out, Bp, mu, s);
        case 16: return launch_mf_lpn<4>(row_pass, G, v, base, out, Bp, mu, s);
        default:
            if (Bp % 32 == 0) return launch_mf_lpn<8>(row_pass, G, v, base, out, Bp, mu, s);
            return cudaErrorInvalidValue;
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
