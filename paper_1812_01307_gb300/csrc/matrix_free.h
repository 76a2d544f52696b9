// Matrix-free parallel-beam projector (matrix_free.cu): per-angle constants
// and launchers of the batched row / column passes that compute A's weights
// on the fly.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace bsgdtv {

// Constants of one projection angle, FP64 values carried as (hi, lo) float
// pairs: cos, sin and the sorted projections p0..p3 of a unit square's
// corners on the ray normal; 1/a and 1/(a b) with a = max(|c|, |s|),
// b = min(|c|, |s|); 1/c and 1/s (0 where undefined) for locating the pixels
// a ray crosses; axis = 1 for an axis-parallel ray (b = 0); xmajor = 1 when
// |s| >= |c| (the ray advances at least as fast in x as in y).
struct AngleGeo {
    float c[2], s[2], p[8];
    float inv_a, inv_ab, inv_c, inv_s;
    int axis, xmajor, pad[2];
};

struct MfGeometry {
    const AngleGeo *geo = nullptr;   // device [n_angles]
    int n = 0, n_angles = 0, n_bins = 0;
};

void mf_angle_table(int n_angles, std::vector<AngleGeo> &out);

// Row pass (row_pass = true): out[ray] = base[ray] - (A v)[ray]; column pass:
// out[pixel] = base[pixel] + mu * 2 (A^T v)[pixel]; interleaved [element][Bp]
// vectors (Bp = 4, 8, 16 or a multiple of 32), LPN = min(Bp / 4, 8) lanes
// per output element.
cudaError_t launch_mf_pass(bool row_pass, int Bp, const MfGeometry &G, const float *v,
                           const float *base, float *out, float mu, cudaStream_t s);

// The row pass's weights of the listed rays: per ray up to `capacity`
// (column, weight) pairs at ray_index * capacity, and their count.
cudaError_t launch_mf_weights(const MfGeometry &G, const int64_t *rays, int n_rays, int capacity,
                              int32_t *cols, float *vals, int *counts, cudaStream_t s);

}  // namespace bsgdtv
