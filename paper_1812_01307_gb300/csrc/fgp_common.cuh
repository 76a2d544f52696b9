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

// Shared buffers are padded with a zero border so that neighbour reads need
// no bounds tests: column c of the region is stored at c + 1, row -1 of the
// strip-edge buffer and row RH of u are zero.
template <int TY, int V>
struct FgpShared {
    static_assert(TY * V == RH, "a region is RH pixels high");
    float s[RH][RW + 2];        // s of the momentum point, read by the right neighbour
    float u[RH + 1][RW + 2];    // u, read by the left and upper neighbours
    float r_edge[TY + 1][RW];   // r of each strip's last pixel, read by the strip below
};

// One FGP iteration for this thread's strip.  (p, q) hold the current dual
// iterate and (pp, qp) the previous one; the new iterate is written over
// (pp, qp), so the caller swaps the roles of the two register sets.
//
// The projection is applied jointly everywhere: where only p (last column) or
// only q (last row) is defined, the other component is zeroed first, which
// makes the joint projection exactly the single-component clip t/max(1,|t|);
// outside the image both are zeroed.  rsqrtf(max(n2, 1)) is the scale
// 1/max(1, sqrt(n2)).
//
// kStepRegs: the dual step 1/(8 tau) is held per pixel and component (cp, cq:
// 1/(8 tau) where p / q is defined, else 0) instead of testing mask bits; at
// the undefined places p, q and the momentum point are exactly 0 throughout,
// so fmaf(d, 0, 0) = 0 gives the same bits as the masked form with two
// instructions fewer per component (at 2V more registers).
template <int TY, int V, bool kStepRegs>
__device__ __forceinline__ void fgp_step(float (&p)[V], float (&pp)[V], float (&q)[V],
                                         float (&qp)[V], const float (&bb)[V], unsigned pmask,
                                         unsigned qmask, const float (&cp)[V],
                                         const float (&cq)[V], float beta, float tau, float c8,
                                         FgpShared<TY, V> &sh, int tx, int ty) {
    float rr[V], ss[V], uu[V];
    // momentum point (r, s) from the last two iterates
#pragma unroll
    for (int v = 0; v < V; ++v) {
        rr[v] = fmaf(beta, p[v] - pp[v], p[v]);
        ss[v] = fmaf(beta, q[v] - qp[v], q[v]);
        sh.s[ty * V + v][tx + 1] = ss[v];
    }
    sh.r_edge[ty + 1][tx] = rr[V - 1];
    __syncthreads();
    // u = b - tau L(r, s)
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float r_up = (v > 0) ? rr[v - 1] : sh.r_edge[ty][tx];
        const float s_left = sh.s[ty * V + v][tx];
        uu[v] = fmaf(-tau, (rr[v] - r_up) + (ss[v] - s_left), bb[v]);
        sh.u[ty * V + v][tx + 1] = uu[v];
    }
    __syncthreads();
    // (P, Q) = L^T u, gradient step on the dual, projection onto the unit ball
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float u_down = (v < V - 1) ? uu[v + 1] : sh.u[ty * V + V][tx + 1];
        const float u_right = sh.u[ty * V + v][tx + 2];
        float pt, qt;
        if constexpr (kStepRegs) {
            pt = fmaf(uu[v] - u_down, cp[v], rr[v]);
            qt = fmaf(uu[v] - u_right, cq[v], ss[v]);
        } else {
            pt = (pmask & (1u << v)) ? fmaf(uu[v] - u_down, c8, rr[v]) : 0.f;
            qt = (qmask & (1u << v)) ? fmaf(uu[v] - u_right, c8, ss[v]) : 0.f;
        }
        const float inv = rsqrtf(fmaxf(fmaf(pt, pt, qt * qt), 1.f));
        pp[v] = pt * inv;
        qp[v] = qt * inv;
    }
}

// The dual state (p, q, p_prev, q_prev) of a tiled FGP passes between
// launches through global memory.  A launch reads the set the previous launch
// wrote (*_in; not read when `first`) and writes its regions' interiors to the
// other set (*_out; not written when `last`): a region's halo is a neighbour's
// interior, and CTAs of one grid run in no fixed order, so reading and
// writing one set in place would let a neighbour that finished first hand
// this region iterates that are a whole launch ahead.
// kBatch: blockIdx.z selects one of several images stored `plane` floats
// apart (b, x_out and the dual fields alike), each with its own weight
// tau_z[z]; a weight <= 0 makes that image's prox the identity.
// TY x V: threads in y x pixels per thread (TY * V = RH); kStepRegs: see
// fgp_step.
template <bool kBatch, int TY, int V, bool kStepRegs>
__global__ void __launch_bounds__(RW *TY)
    fgp_kernel(const float *__restrict__ b, float *__restrict__ x_out, int H, int W, float tau,
               float c8, const float *__restrict__ mom, int k0, int iters, int HL, int IH, int IW,
               int first, int last, const float *__restrict__ p_in,
               const float *__restrict__ q_in, const float *__restrict__ pp_in,
               const float *__restrict__ qp_in, float *__restrict__ p_out,
               float *__restrict__ q_out, float *__restrict__ pp_out, float *__restrict__ qp_out,
               const float *__restrict__ tau_z, int64_t plane) {
    __shared__ FgpShared<TY, V> sh;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int R0 = blockIdx.y * IH - HL, C0 = blockIdx.x * IW - HL;
    const int j = C0 + tx;
    const bool col_in = (j >= 0 && j < W);

    // zero borders (never written afterwards) and the masks
    if (ty == 0) {
        sh.r_edge[0][tx] = 0.f;
        sh.u[RH][tx + 1] = 0.f;
        if (tx == 0) sh.u[RH][0] = sh.u[RH][RW + 1] = 0.f;
    }
    if (tx == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            sh.s[ty * V + v][0] = 0.f;
            sh.u[ty * V + v][RW + 1] = 0.f;
            sh.s[ty * V + v][RW + 1] = 0.f;
            sh.u[ty * V + v][0] = 0.f;
        }
    }
    if constexpr (kBatch) {
        const int64_t off = (int64_t)blockIdx.z * plane;
        b += off;
        x_out += off;
        p_in += off;
        q_in += off;
        pp_in += off;
        qp_in += off;
        p_out += off;
        q_out += off;
        pp_out += off;
        qp_out += off;
        tau = tau_z[blockIdx.z];
        c8 = 1.0f / (8.0f * tau);
    }
    pdl_wait_and_release();
    if constexpr (kBatch) {
        if (!(tau > 0.f)) {   // block-uniform: zero weight, x = b
            if (!last) return;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int rr_ = ty * V + v;
                const int i = R0 + rr_;
                const bool interior = rr_ >= HL && rr_ < HL + IH && tx >= HL && tx < HL + IW;
                if (interior && col_in && i >= 0 && i < H) x_out[(int64_t)i * W + j] = b[(int64_t)i * W + j];
            }
            return;
        }
    }

    float bb[V], pa[V], pb[V], qa[V], qb[V];
    unsigned pmask = 0u, qmask = 0u;   // bit v: p / q defined at this strip's pixel v
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int i = R0 + ty * V + v;
        const bool in = col_in && i >= 0 && i < H;
        if (in && i < H - 1) pmask |= 1u << v;
        if (in && j < W - 1) qmask |= 1u << v;
        const int64_t o = (int64_t)i * W + j;
        bb[v] = in ? b[o] : 0.f;
        if (first || !in) {
            pa[v] = qa[v] = pb[v] = qb[v] = 0.f;
        } else {
            pa[v] = p_in[o];
            qa[v] = q_in[o];
            pb[v] = pp_in[o];
            qb[v] = qp_in[o];
        }
    }

    float cp[V], cq[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        cp[v] = (pmask & (1u << v)) ? c8 : 0.f;
        cq[v] = (qmask & (1u << v)) ? c8 : 0.f;
    }

    int it = 0;
    for (; it + 2 <= iters; it += 2) {
        fgp_step<TY, V, kStepRegs>(pa, pb, qa, qb, bb, pmask, qmask, cp, cq, mom[k0 + it], tau, c8,
                                   sh, tx, ty);
        fgp_step<TY, V, kStepRegs>(pb, pa, qb, qa, bb, pmask, qmask, cp, cq, mom[k0 + it + 1], tau,
                                   c8, sh, tx, ty);
    }
    if (it < iters) {
        fgp_step<TY, V, kStepRegs>(pa, pb, qa, qb, bb, pmask, qmask, cp, cq, mom[k0 + it], tau, c8,
                                   sh, tx, ty);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float t0 = pa[v], t1 = qa[v];
            pa[v] = pb[v];
            qa[v] = qb[v];
            pb[v] = t0;
            qb[v] = t1;
        }
    }
    // (pa, qa): current iterate, (pb, qb): previous one

    if (last) {
        // x = b - tau L(p, q) with the final iterate
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) sh.s[ty * V + v][tx + 1] = qa[v];
        sh.r_edge[ty + 1][tx] = pa[V - 1];
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr_ = ty * V + v;
            const int i = R0 + rr_;
            const bool interior = rr_ >= HL && rr_ < HL + IH && tx >= HL && tx < HL + IW;
            if (!(interior && col_in && i >= 0 && i < H)) continue;
            const float p_up = (v > 0) ? pa[v - 1] : sh.r_edge[ty][tx];
            const float q_left = sh.s[rr_][tx];
            x_out[(int64_t)i * W + j] = bb[v] - tau * (pa[v] + qa[v] - p_up - q_left);
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr_ = ty * V + v;
            const int i = R0 + rr_;
            const bool interior = rr_ >= HL && rr_ < HL + IH && tx >= HL && tx < HL + IW;
            if (!(interior && col_in && i >= 0 && i < H)) continue;
            const int64_t o = (int64_t)i * W + j;
            p_out[o] = pa[v];
            q_out[o] = qa[v];
            pp_out[o] = pb[v];
            qp_out[o] = qb[v];
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

// K FGP iterations: one launch when the image fits one region, else one
// launch per chunk of <= kMaxChunk iterations over overlapping regions.
// kBatch: `planes` images `plane` floats apart, weights tau_z[0 .. planes).
// TY x V: the kernel's thread shape (see fgp_kernel).  16 x 4 (1024 threads,
// 4-pixel strips, <= 64 registers) measured 1-3 % faster than 8 x 8 (512
// threads, 8-pixel strips, 78 registers): twice the warps per SM hide the two
// barriers of every iteration better; both give bit-identical iterates.
template <bool kBatch, int TY = 16, int V = 4, bool kStepRegs = true>
cudaError_t launch_fgp_regions(const float *b, float *x, int h, int w, float tau,
                               const float *tau_z, int planes, int64_t plane, int iters,
                               const float *mom, FgpScratch sc, cudaStream_t s, bool pdl,
                               int max_chunk = kMaxChunk) {
    const dim3 block(RW, TY);
    const float c8 = 1.0f / (8.0f * tau);
    if (fits_one_region(h, w)) {
        // one launch, no field traffic (first and last)
        const FgpFields &f = sc.set[0];
        cudaError_t e = launch_kernel(fgp_kernel<kBatch, TY, V, kStepRegs>, dim3(1, 1, planes), block, 0, s, pdl, b,
                                      x, h, w, tau, c8, mom, 0, iters, 0, RH, RW, 1, 1, f.p, f.q,
                                      f.pp, f.qp, f.p, f.q, f.pp, f.qp, tau_z, plane);
        add_launches(1);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    int done = 0;
    for (int launch = 0; done < iters; ++launch) {
        const int chunk = std::min(max_chunk, iters - done);
        const int HL = chunk + 1;
        const int IH = RH - 2 * HL, IW = RW - 2 * HL;
        const dim3 grid((w + IW - 1) / IW, (h + IH - 1) / IH, planes);
        const int first = (done == 0), last = (done + chunk == iters);
        const FgpFields &fi = fgp_read_set(sc, launch), &fo = fgp_write_set(sc, launch);
        cudaError_t e = launch_kernel(fgp_kernel<kBatch, TY, V, kStepRegs>, grid, block, 0, s, pdl || done > 0, b, x,
                                      h, w, tau, c8, mom, done, chunk, HL, IH, IW, first, last,
                                      fi.p, fi.q, fi.pp, fi.qp, fo.p, fo.q, fo.pp, fo.qp, tau_z,
                                      plane);
        add_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        done += chunk;
    }
    return cudaSuccess;
}

}  // namespace fgpk
}  // namespace bsgdtv
