// FGP iteration body and kernel shared by the single-image TV prox (fgp.cu)
// and the batched one (batch.cu); the algorithm and GPU mapping are described
// in fgp.cu.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "bsgdtv_internal.h"

namespace bsgdtv {
namespace fgpk {

constexpr int RW = 64;      // region width  = threads in x
constexpr int RH = 64;      // region height = TY threads in y x V pixels per thread
constexpr int kMaxChunk = 8;  // iterations per launch when tiled (halo = chunk + 1)

// The neighbour values pass through shared buffers stored column by column
// ([column + 1][row], column stride SC): a thread's strip of V = 4 pixels is
// one 16-byte word, written and read with single 128-bit accesses.  SC = 68
// floats makes 8 consecutive columns' words fall on distinct bank groups (no
// conflicts).  Column 0 (left of the region) and RW + 1 (right of it) are
// zero, as are row 0 of the strip-edge buffer and row TY of the strip-top
// buffer, so neighbour reads need no bounds tests.
constexpr int SC = RH + 4;
static_assert(SC % 8 == 4, "column stride: 16-byte words of consecutive columns on distinct banks");

template <int TY, int V>
struct FgpShared {
    static_assert(TY * V == RH && V == 4, "a region is RH pixels high, 4 per thread");
    float s[RW + 2][SC];        // s of the momentum point, read by the right neighbour
    float u[RW + 2][SC];        // u, read by the left neighbour
    float r_edge[TY + 1][RW];   // r of each strip's last pixel, read by the strip below
    float u_top[TY + 1][RW];    // u of each strip's first pixel, read by the strip above
};

// Two-lane FP32 arithmetic (one instruction for two pixels; each lane rounds
// exactly as the scalar operation would).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 1 / sqrt(max(a, 1)) (a NaN a gives 1, as fmaxf would).  The argument of
// the approximate reciprocal square root is >= 1, never subnormal, so its
// flush-to-zero form returns the same value as the plain one, without the
// instructions the plain form spends on subnormal arguments.
__device__ __forceinline__ float rsqrt_max1(float a) {
    float r;
    asm("{\n\t.reg .f32 m;\n\t"
        "max.f32 m, %1, 0f3F800000;\n\t"
        "rsqrt.approx.ftz.f32 %0, m;\n\t}"
        : "=f"(r)
        : "f"(a));
    return r;
}

// A thread's 4 pixels as two pairs: pixels (0, 1) and (2, 3) of the strip.
struct Strip {
    float2 h[2];
    __device__ __forceinline__ float get(int v) const { return (v & 1) ? h[v >> 1].y : h[v >> 1].x; }
    __device__ __forceinline__ void set(int v, float a) {
        if (v & 1)
            h[v >> 1].y = a;
        else
            h[v >> 1].x = a;
    }
};

// One FGP iteration for this thread's strip.  (p, q) hold the current dual
// iterate and (pp, qp) the previous one; the new iterate is written over
// (pp, qp), so the caller swaps the roles of the two register sets.
//
// The projection is applied jointly everywhere: where only p (last row of the
// image has no p) or only q is defined, the other component is exactly 0
// throughout, because its dual step (cp or cq: 1/(8 tau) where the component
// exists, else 0) keeps it there, and the joint projection then equals the
// single-component clip t/max(1,|t|); outside the image b, p and q are all 0.
// rsqrt_max1(n2) is the scale 1/max(1, sqrt(n2)).
template <int TY, int V>
__device__ __forceinline__ void fgp_step(Strip &p, Strip &pp, Strip &q, Strip &qp,
                                         const Strip &bb, const Strip &cp, const Strip &cq,
                                         float beta, float tau, FgpShared<TY, V> &sh, int tx,
                                         int ty) {
    const float2 beta2 = make_float2(beta, beta), ntau2 = make_float2(-tau, -tau);
    Strip rr, ss, uu;
    // momentum point (r, s) from the last two iterates
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        rr.h[k] = fma2(beta2, sub2(p.h[k], pp.h[k]), p.h[k]);
        ss.h[k] = fma2(beta2, sub2(q.h[k], qp.h[k]), q.h[k]);
    }
    *reinterpret_cast<float4 *>(&sh.s[tx + 1][ty * V]) =
        make_float4(ss.h[0].x, ss.h[0].y, ss.h[1].x, ss.h[1].y);
    sh.r_edge[ty + 1][tx] = rr.h[1].y;
    __syncthreads();
    // u = b - tau L(r, s): r one row up, s one column left
    {
        const float4 sl = *reinterpret_cast<const float4 *>(&sh.s[tx][ty * V]);
        const float r_up0 = sh.r_edge[ty][tx];
        const float2 rup[2] = {make_float2(r_up0, rr.h[0].x), make_float2(rr.h[0].y, rr.h[1].x)};
        const float2 sleft[2] = {make_float2(sl.x, sl.y), make_float2(sl.z, sl.w)};
#pragma unroll
        for (int k = 0; k < 2; ++k)
            uu.h[k] = fma2(ntau2, add2(sub2(rr.h[k], rup[k]), sub2(ss.h[k], sleft[k])), bb.h[k]);
    }
    *reinterpret_cast<float4 *>(&sh.u[tx + 1][ty * V]) =
        make_float4(uu.h[0].x, uu.h[0].y, uu.h[1].x, uu.h[1].y);
    sh.u_top[ty][tx] = uu.h[0].x;
    __syncthreads();
    // (P, Q) = L^T u (u one row down, one column right), gradient step on the
    // dual, projection onto the unit ball
    const float4 ur = *reinterpret_cast<const float4 *>(&sh.u[tx + 2][ty * V]);
    const float u_dn3 = sh.u_top[ty + 1][tx];
    const float2 udn[2] = {make_float2(uu.h[0].y, uu.h[1].x), make_float2(uu.h[1].y, u_dn3)};
    const float2 urt[2] = {make_float2(ur.x, ur.y), make_float2(ur.z, ur.w)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 pt = fma2(sub2(uu.h[k], udn[k]), cp.h[k], rr.h[k]);
        const float2 qt = fma2(sub2(uu.h[k], urt[k]), cq.h[k], ss.h[k]);
        const float2 n2 = fma2(pt, pt, mul2(qt, qt));
        const float2 inv = make_float2(rsqrt_max1(n2.x), rsqrt_max1(n2.y));
        pp.h[k] = mul2(pt, inv);
        qp.h[k] = mul2(qt, inv);
    }
}

// Regions along one image dimension of `len` pixels for regions of R pixels
// with a halo of HL: a region at the image's edge needs no halo on that side
// (outside the image every iterate is exactly zero, as the region's zero
// borders and masks make it), so the first and the last region's interiors
// reach R - HL pixels and only the others' are R - 2 HL wide.
__host__ __device__ inline int fgp_regions_along(int len, int R, int HL) {
    if (len <= R) return 1;
    const int rest = len - 2 * (R - HL);
    return 2 + (rest > 0 ? (rest + R - 2 * HL - 1) / (R - 2 * HL) : 0);
}
// Region b of n along that dimension: its first pixel and its interior [lo, hi)
// in region-local coordinates.
__host__ __device__ __forceinline__ void fgp_place(int b, int n, int len, int R, int HL, int &first,
                                                   int &lo, int &hi) {
    if (n == 1) {
        first = 0;
        lo = 0;
        hi = len;
        return;
    }
    const int inner = R - 2 * HL;
    const int start = (b == 0) ? 0 : (R - HL) + (b - 1) * inner;
    const int end = (b == n - 1) ? len : (R - HL) + b * inner;
    first = (b == 0) ? 0 : start - HL;
    lo = start - first;
    hi = end - first;
}

// One launch of the FGP covers the images of up to kMaxFgpParts parts (a
// part: `slices` images of H x W, `plane` floats apart, with their own
// weights).  CTA blockIdx.x belongs to the last part whose cta_begin it has
// reached and takes, within it, image z and region (bx, by) of the rx x ry
// regions of that image.
struct FgpPart {
    const float *b;       // inputs, image z at + z * plane
    float *x;             // outputs
    const float *tau_z;   // per-image weights, or null: every image uses tau
    float tau;
    FgpFields in, out;    // dual field sets read / written (image z at + z * plane)
    int64_t plane;
    int H, W, rx, ry;     // image size; regions across and down
    int cta_begin;        // first CTA of this part
};
constexpr int kMaxFgpParts = 8;
struct FgpLaunch {
    FgpPart part[kMaxFgpParts];
    int n_parts;
};

// The dual state (p, q, p_prev, q_prev) of a tiled FGP passes between
// launches through global memory.  A launch reads the set the previous launch
// wrote (in; not read when `first`) and writes its regions' interiors to the
// other set (out; not written when `last`): a region's halo is a neighbour's
// interior, and CTAs of one grid run in no fixed order, so reading and
// writing one set in place would let a neighbour that finished first hand
// this region iterates that are a whole launch ahead.  A weight <= 0 makes an
// image's prox the identity (x = b).
// TY x V: threads in y x pixels per thread (TY * V = RH, V = 4).
// kMulti: the launch has several parts; with one part the descriptor's
// fields are read at fixed offsets of the kernel arguments.
template <int TY, int V, bool kMulti>
__global__ void __launch_bounds__(RW *TY)
    fgp_kernel(const __grid_constant__ FgpLaunch L, const float *__restrict__ mom, int k0, int iters,
               int HL, int first, int last) {
    __shared__ __align__(16) FgpShared<TY, V> sh;

    int pi = 0;
    if constexpr (kMulti)
        while (pi + 1 < L.n_parts && (int)blockIdx.x >= L.part[pi + 1].cta_begin) ++pi;
    const FgpPart &P = L.part[pi];
    const int per = P.rx * P.ry, local = (int)blockIdx.x - P.cta_begin;
    const int z = local / per, reg = local - z * per;
    const int by = reg / P.rx, bx = reg - by * P.rx;
    const int H = P.H, W = P.W;
    const int64_t off = (int64_t)z * P.plane;
    const float *__restrict__ b = P.b + off;
    float *__restrict__ x_out = P.x + off;
    const float *__restrict__ p_in = P.in.p + off;
    const float *__restrict__ q_in = P.in.q + off;
    const float *__restrict__ pp_in = P.in.pp + off;
    const float *__restrict__ qp_in = P.in.qp + off;
    float *__restrict__ p_out = P.out.p + off;
    float *__restrict__ q_out = P.out.q + off;
    float *__restrict__ pp_out = P.out.pp + off;
    float *__restrict__ qp_out = P.out.qp + off;
    const float tau = P.tau_z ? P.tau_z[z] : P.tau;
    const float c8 = 1.0f / (8.0f * tau);

    const int tx = threadIdx.x, ty = threadIdx.y;
    int R0, C0, rlo, rhi, clo, chi;
    fgp_place(by, P.ry, H, RH, HL, R0, rlo, rhi);
    fgp_place(bx, P.rx, W, RW, HL, C0, clo, chi);
    const int j = C0 + tx;
    const bool col_in = (j >= 0 && j < W);

    // zero borders (never written afterwards): columns 0 and RW + 1, row 0
    // of the strip-edge buffer, row TY of the strip-top buffer
    if (tx < 2) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            sh.s[tx * (RW + 1)][ty * V + v] = 0.f;
            sh.u[tx * (RW + 1)][ty * V + v] = 0.f;
        }
    }
    if (ty == 0) {
        sh.r_edge[0][tx] = 0.f;
        sh.u_top[TY][tx] = 0.f;
    }
    // b and the dual steps.  Every launch of one prox after the first starts
    // only once the first has passed its wait on the kernel that wrote b, so
    // those launches read b before their own wait (overlapping the previous
    // launch's tail); the first reads it after.
    Strip bb, cp, cq;
    auto load_b = [&]() {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int i = R0 + ty * V + v;
            const bool in = col_in && i >= 0 && i < H;
            bb.set(v, in ? b[(int64_t)i * W + j] : 0.f);
            // per-pixel dual steps: 1/(8 tau) where p (i < H-1) / q (j < W-1) exists
            cp.set(v, (in && i < H - 1) ? c8 : 0.f);
            cq.set(v, (in && j < W - 1) ? c8 : 0.f);
        }
    };
    if (!first) load_b();
    pdl_wait_and_release();
    if (first) load_b();
    if (!(tau > 0.f)) {   // block-uniform: zero weight, x = b
        if (!last) return;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr_ = ty * V + v;
            const int i = R0 + rr_;
            const bool interior = rr_ >= rlo && rr_ < rhi && tx >= clo && tx < chi;
            if (interior && col_in && i >= 0 && i < H) x_out[(int64_t)i * W + j] = b[(int64_t)i * W + j];
        }
        return;
    }

    Strip pa, pb, qa, qb;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int i = R0 + ty * V + v;
        const bool in = col_in && i >= 0 && i < H;
        const int64_t o = (int64_t)i * W + j;
        if (first || !in) {
            pa.set(v, 0.f);
            qa.set(v, 0.f);
            pb.set(v, 0.f);
            qb.set(v, 0.f);
        } else {
            pa.set(v, p_in[o]);
            qa.set(v, q_in[o]);
            pb.set(v, pp_in[o]);
            qb.set(v, qp_in[o]);
        }
    }

    // momentum coefficients are loaded one pair of iterations ahead, so the
    // load's latency hides behind the iterations
    int it = 0;
    float m0 = iters > 0 ? mom[k0] : 0.f, m1 = iters > 1 ? mom[k0 + 1] : 0.f;
    for (; it + 2 <= iters; it += 2) {
        const float n0 = it + 2 < iters ? mom[k0 + it + 2] : 0.f;
        const float n1 = it + 3 < iters ? mom[k0 + it + 3] : 0.f;
        fgp_step<TY, V>(pa, pb, qa, qb, bb, cp, cq, m0, tau, sh, tx, ty);
        fgp_step<TY, V>(pb, pa, qb, qa, bb, cp, cq, m1, tau, sh, tx, ty);
        m0 = n0;
        m1 = n1;
    }
    if (it < iters) {
        fgp_step<TY, V>(pa, pb, qa, qb, bb, cp, cq, m0, tau, sh, tx, ty);
        const Strip t0 = pa, t1 = qa;
        pa = pb;
        qa = qb;
        pb = t0;
        qb = t1;
    }
    // (pa, qa): current iterate, (pb, qb): previous one

    if (last) {
        // x = b - tau L(p, q) with the final iterate
        __syncthreads();
        *reinterpret_cast<float4 *>(&sh.s[tx + 1][ty * V]) =
            make_float4(qa.h[0].x, qa.h[0].y, qa.h[1].x, qa.h[1].y);
        sh.r_edge[ty + 1][tx] = pa.get(V - 1);
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr_ = ty * V + v;
            const int i = R0 + rr_;
            const bool interior = rr_ >= rlo && rr_ < rhi && tx >= clo && tx < chi;
            if (!(interior && col_in && i >= 0 && i < H)) continue;
            const float p_up = (v > 0) ? pa.get(v - 1) : sh.r_edge[ty][tx];
            const float q_left = sh.s[tx][rr_];
            x_out[(int64_t)i * W + j] = bb.get(v) - tau * (pa.get(v) + qa.get(v) - p_up - q_left);
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr_ = ty * V + v;
            const int i = R0 + rr_;
            const bool interior = rr_ >= rlo && rr_ < rhi && tx >= clo && tx < chi;
            if (!(interior && col_in && i >= 0 && i < H)) continue;
            const int64_t o = (int64_t)i * W + j;
            p_out[o] = pa.get(v);
            q_out[o] = qa.get(v);
            pp_out[o] = pb.get(v);
            qp_out[o] = qb.get(v);
        }
    }
}


inline bool fits_one_region(int h, int w) { return h <= RH && w <= RW; }

// Launch `launch` of a tiled FGP reads field set (launch + 1) & 1 and writes
// set launch & 1.
inline const FgpFields &fgp_read_set(const FgpScratch &sc, int launch) {
    return sc.set[(launch + 1) & 1];
}
inline const FgpFields &fgp_write_set(const FgpScratch &sc, int launch) { return sc.set[launch & 1]; }

// Host description of one part of an FGP launch: `slices` images of h x w,
// `plane` floats apart (b in, x out), weights tau_z[0 .. slices) or, with
// tau_z null, tau for all; sc: the part's two dual field sets.
struct FgpImages {
    const float *b;
    float *x;
    const float *tau_z;
    float tau;
    FgpScratch sc;
    int64_t plane;
    int h, w, slices;
};

// K FGP iterations on every image of n_parts parts, each launch covering all
// of them: one launch when every image fits one region, else one launch per
// chunk of <= max_chunk iterations over overlapping regions (halo = chunk +
// 1).  TY x V: the kernel's thread shape (see fgp_kernel): 16 x 4, 1024
// threads with 4-pixel strips (an earlier 8 x 8 shape with 512 threads ran
// 1-3 % slower: twice the warps per SM hide the two barriers of every
// iteration better).
template <int TY = 16, int V = 4>
cudaError_t launch_fgp_parts(const FgpImages *parts, int n_parts, int iters, const float *mom,
                             cudaStream_t s, bool pdl, int max_chunk = kMaxChunk) {
    if (n_parts < 1 || n_parts > kMaxFgpParts) return cudaErrorInvalidValue;
    const dim3 block(RW, TY);
    bool single = true;
    for (int k = 0; k < n_parts; ++k) single = single && fits_one_region(parts[k].h, parts[k].w);
    auto build = [&](int launch, int HL, FgpLaunch &L) -> int {
        int ctas = 0;
        L.n_parts = n_parts;
        for (int k = 0; k < n_parts; ++k) {
            const FgpImages &q = parts[k];
            FgpPart &P = L.part[k];
            P.b = q.b;
            P.x = q.x;
            P.tau_z = q.tau_z;
            P.tau = q.tau;
            P.in = fgp_read_set(q.sc, launch);
            P.out = fgp_write_set(q.sc, launch);
            P.plane = q.plane;
            P.H = q.h;
            P.W = q.w;
            P.rx = fgp_regions_along(q.w, RW, HL);
            P.ry = fgp_regions_along(q.h, RH, HL);
            P.cta_begin = ctas;
            ctas += P.rx * P.ry * q.slices;
        }
        return ctas;
    };
    FgpLaunch L = {};
    if (single) {
        // one launch, no field traffic (first and last)
        const int ctas = build(0, 0, L);
        cudaError_t e = n_parts > 1 ? launch_kernel(fgp_kernel<TY, V, true>, dim3(ctas), block, 0, s, pdl,
                                                    L, mom, 0, iters, 0, 1, 1)
                                    : launch_kernel(fgp_kernel<TY, V, false>, dim3(ctas), block, 0, s, pdl,
                                                    L, mom, 0, iters, 0, 1, 1);
        add_launches(1);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    int done = 0;
    for (int launch = 0; done < iters; ++launch) {
        const int chunk = std::min(max_chunk, iters - done);
        const int HL = chunk + 1;
        const int ctas = build(launch, HL, L);
        const int first = (done == 0), last = (done + chunk == iters);
        const bool p = pdl || done > 0;
        cudaError_t e = n_parts > 1 ? launch_kernel(fgp_kernel<TY, V, true>, dim3(ctas), block, 0, s, p, L,
                                                    mom, done, chunk, HL, first, last)
                                    : launch_kernel(fgp_kernel<TY, V, false>, dim3(ctas), block, 0, s, p, L,
                                                    mom, done, chunk, HL, first, last);
        add_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        done += chunk;
    }
    return cudaSuccess;
}

// The batched form of one part: `planes` images `plane` floats apart with
// weights tau_z.
inline cudaError_t launch_fgp_regions(const float *b, float *x, int h, int w, const float *tau_z,
                                      int planes, int64_t plane, int iters, const float *mom,
                                      FgpScratch sc, cudaStream_t s, bool pdl,
                                      int max_chunk = kMaxChunk) {
    const FgpImages p = {b, x, tau_z, 1.f, sc, plane, h, w, planes};
    return launch_fgp_parts(&p, 1, iters, mom, s, pdl, max_chunk);
}

}  // namespace fgpk
}  // namespace bsgdtv
