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
// GPU mapping: each CTA owns a 64 x 64 pixel region (64 x 16 threads); every
// thread keeps a vertical strip of 4 pixels' fields (b, p, q, p_prev, q_prev,
// r, s, u) in registers for all the iterations of one launch.  Only the values a
// neighbour needs (s to the right neighbour, r across strip boundaries, u to
// the left / upper neighbour) pass through zero-padded shared buffers, two
// barriers per iteration, with no bounds tests in the iteration.  When the image fits one region the whole FGP is one launch;
// otherwise regions overlap by a halo of (iterations per launch + 1) pixels
// (temporal blocking), so each launch runs several iterations with no global
// synchronisation, and the dual fields persist in global memory (L2) between
// launches, in two sets that the launches read and write by turns.  Pixels outside the image hold exact zeros (b = p = q = 0), which
// is the operator's own boundary condition, so no halo is needed there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fgp_common.cuh"

namespace bsgdtv {

using namespace fgpk;

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

int fgp_chunk_for(int h, int w, int iters, int n_sms) {
    if (iters <= 0 || fits_one_region(h, w)) return std::max(iters, 1);
    // cost in iteration-times of one region: per launch, the waves of
    // 1-CTA-per-SM regions times the iterations, plus about two iterations of
    // launch ramp; fewer iterations per launch shrink the halo (more useful
    // pixels per region, fewer regions) but add launches
    int best = kMaxChunk;
    long long best_cost = -1;
    for (int c = 4; c <= 12; ++c) {
        const long long grid =
            (long long)fgp_regions_along(w, RW, c + 1) * fgp_regions_along(h, RH, c + 1);
        const long long waves = (grid + std::max(n_sms, 1) - 1) / std::max(n_sms, 1);
        const long long cost = (long long)((iters + c - 1) / c) * (waves * c + 2);
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

int fgp_plan_launches(int h, int w, int iters, int max_chunk) {
    if (iters <= 0) return 0;
    if (fits_one_region(h, w)) return 1;
    return (iters + max_chunk - 1) / max_chunk;
}

cudaError_t launch_fgp(const float *b, float *x, int h, int w, float tau, int iters,
                       const float *mom, FgpScratch sc, cudaStream_t s, bool pdl, int max_chunk) {
    const FgpImages p = {b, x, nullptr, tau, sc, 0, h, w, 1};
    return launch_fgp_parts(&p, 1, iters, mom, s, pdl, max_chunk);
}

}  // namespace bsgdtv

using namespace bsgdtv;

extern "C" int bsgdtv_fgp_tiling(int len, int halo, int max_regions, int *n_regions, int *first,
                                 int *lo, int *hi) {
    if (len < 1 || halo < 1 || 2 * halo >= fgpk::RW || max_regions < 0 || !n_regions)
        return fail(BSGDTV_ERR_INVALID_ARG, "need len >= 1, 1 <= halo < 32, max_regions >= 0, n_regions");
    const int n = fgpk::fgp_regions_along(len, fgpk::RW, halo);
    *n_regions = n;
    for (int k = 0; k < n && k < max_regions; ++k) {
        int f = 0, l = 0, h = 0;
        fgpk::fgp_place(k, n, len, fgpk::RW, halo, f, l, h);
        if (first) first[k] = f;
        if (lo) lo[k] = l;
        if (hi) hi[k] = h;
    }
    return BSGDTV_OK;
}
