// TV proximal step of Algorithm 1: x = argmin_t ||t - b||^2 + 2 tau TV(t), tau = mu*lambda,
// by Beck & Teboulle's fast gradient projection (FGP, IEEE TIP 18(11), 2009).
//
// One FGP iteration on the dual pair (p, q) (p: (h-1) x w, q: h x (w-1)):
//   u        = b - tau L(r, s)              L(p,q)_{i,j} = p_{i,j}+q_{i,j}-p_{i-1,j}-q_{i,j-1}
//   (P, Q)   = L^T(u)                       P_{i,j} = u_{i,j}-u_{i+1,j}, Q_{i,j} = u_{i,j}-u_{i,j+1}
//   (p, q)   = Proj[(r, s) + (P, Q)/(8 tau)]  per pixel onto the unit l2 ball
//                                            (border p_{i,w-1}, q_{h-1,j} clipped alone)
//   (r, s)   = (p, q) + beta_k (p - p_prev, q - q_prev)
// and finally x = b - tau L(p, q).
//
// GPU mapping: each CTA owns a 64 x 64 pixel region; every thread keeps a
// vertical strip of 8 pixels' fields (b, p, q, p_prev, q_prev, r, s, u) in
// registers for all the iterations of one launch.  Only the values a
// neighbour needs (s to the right neighbour, r across strip boundaries, u to
// the left / upper neighbour) pass through zero-padded shared buffers, two
// barriers per iteration, with no bounds tests in the iteration.  When the image fits one region the whole FGP is one launch;
// otherwise regions overlap by a halo of (iterations per launch + 1) pixels
// (temporal blocking), so each launch runs several iterations with no global
// synchronisation, and the dual fields persist in global memory (L2) between
// launches.  Pixels outside the image hold exact zeros (b = p = q = 0), which
// is the operator's own boundary condition, so no halo is needed there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bsgdtv_internal.h"

namespace bsgdtv {

namespace {

constexpr int RW = 64;      // region width  = threads in x
constexpr int TY = 8;       // threads in y
constexpr int V = 8;        // pixels per thread (vertical strip)
constexpr int RH = TY * V;  // region height
constexpr int kMaxChunk = 8;  // iterations per launch when tiled (halo = chunk + 1)

// Shared buffers are padded with a zero border so that neighbour reads need
// no bounds tests: column c of the region is stored at c + 1, row -1 of the
// strip-edge buffer and row RH of u are zero.
struct FgpShared {
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
__device__ __forceinline__ void fgp_step(float (&p)[V], float (&pp)[V], float (&q)[V],
                                         float (&qp)[V], const float (&bb)[V], unsigned pmask,
                                         unsigned qmask, float beta, float tau, float c8,
                                         FgpShared &sh, int tx, int ty) {
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
        const float pt = (pmask & (1u << v)) ? fmaf(uu[v] - u_down, c8, rr[v]) : 0.f;
        const float qt = (qmask & (1u << v)) ? fmaf(uu[v] - u_right, c8, ss[v]) : 0.f;
        const float inv = rsqrtf(fmaxf(fmaf(pt, pt, qt * qt), 1.f));
        pp[v] = pt * inv;
        qp[v] = qt * inv;
    }
}

__global__ void __launch_bounds__(RW *TY)
    fgp_kernel(const float *__restrict__ b, float *__restrict__ x_out, int H, int W, float tau,
               float c8, const float *__restrict__ mom, int k0, int iters, int HL, int IH, int IW,
               int first, int last, float *__restrict__ p_g, float *__restrict__ q_g,
               float *__restrict__ pp_g, float *__restrict__ qp_g) {
    __shared__ FgpShared sh;

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
    pdl_wait_and_release();

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
            pa[v] = p_g[o];
            qa[v] = q_g[o];
            pb[v] = pp_g[o];
            qb[v] = qp_g[o];
        }
    }

    int it = 0;
    for (; it + 2 <= iters; it += 2) {
        fgp_step(pa, pb, qa, qb, bb, pmask, qmask, mom[k0 + it], tau, c8, sh, tx, ty);
        fgp_step(pb, pa, qb, qa, bb, pmask, qmask, mom[k0 + it + 1], tau, c8, sh, tx, ty);
    }
    if (it < iters) {
        fgp_step(pa, pb, qa, qb, bb, pmask, qmask, mom[k0 + it], tau, c8, sh, tx, ty);
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
            p_g[o] = pa[v];
            q_g[o] = qa[v];
            pp_g[o] = pb[v];
            qp_g[o] = qb[v];
        }
    }
}

}  // namespace

void fgp_momentum_host(int iters, std::vector<float> &mom) {
    // iteration 1 starts from (r_1, s_1) = (p_0, q_0) = 0; iteration k >= 2 uses
    // (t_{k-1} - 1) / t_k with t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    mom.assign(std::max(iters, 1), 0.f);
    double t = 1.0;
    for (int k = 1; k < iters; ++k) {
        const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
        mom[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
}

static bool fits_one_region(int h, int w) { return h <= RH && w <= RW; }

int fgp_plan_launches(int h, int w, int iters) {
    if (iters <= 0) return 0;
    if (fits_one_region(h, w)) return 1;
    return (iters + kMaxChunk - 1) / kMaxChunk;
}

cudaError_t launch_fgp(const float *b, float *x, int h, int w, float tau, int iters,
                       const float *mom, FgpScratch sc, cudaStream_t s, bool pdl) {
    const dim3 block(RW, TY);
    const float c8 = 1.0f / (8.0f * tau);
    if (fits_one_region(h, w)) {
        cudaError_t e = launch_kernel(fgp_kernel, dim3(1, 1), block, 0, s, pdl, b, x, h, w, tau, c8,
                                      mom, 0, iters, 0, RH, RW, 1, 1, sc.p, sc.q, sc.pp, sc.qp);
        add_launches(1);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    int done = 0;
    while (done < iters) {
        const int chunk = std::min(kMaxChunk, iters - done);
        const int HL = chunk + 1;
        const int IH = RH - 2 * HL, IW = RW - 2 * HL;
        const dim3 grid((w + IW - 1) / IW, (h + IH - 1) / IH);
        const int first = (done == 0), last = (done + chunk == iters);
        cudaError_t e = launch_kernel(fgp_kernel, grid, block, 0, s, pdl || done > 0, b, x, h, w, tau,
                                      c8, mom, done, chunk, HL, IH, IW, first, last, sc.p, sc.q,
                                      sc.pp, sc.qp);
        add_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        done += chunk;
    }
    return cudaSuccess;
}

}  // namespace bsgdtv
