// Internal declarations of the BSGD-TV library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/bsgdtv.h"

namespace bsgdtv {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
#define BSG_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::bsgdtv::fail(BSGDTV_ERR_CUDA, std::string(#call) + ": " +               \
                                                       cudaGetErrorString(e_));              \
    } while (0)
#define BSG_CHECK(expr)                \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != BSGDTV_OK) return rc_; \
    } while (0)

void add_launches(int64_t n);

// True if no entry of y[0..n) is NaN or +-Inf (exponent bits all ones);
// branch-free over the whole array so the compiler can vectorise it.
inline bool all_finite(const float *y, int64_t n) {
    uint32_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b;
        std::memcpy(&b, y + i, sizeof(b));
        bad |= (uint32_t)((b & 0x7f800000u) == 0x7f800000u);
    }
    return bad == 0;
}

// Kernel launch with optional programmatic dependent launch (PDL): the grid
// may be scheduled while its predecessor in the stream drains; the kernel
// must execute pdl_wait() before touching memory its predecessor writes.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#ifdef __CUDACC__
// Wait for the predecessor grid (no-op without PDL), then let the successor
// grid be scheduled.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
#endif

// ------------------------------------------------------- tiled operator layout
// The image is cut into pixel tiles (at most kTileH x kTileW, never crossing a
// column-block band J_j) and the rows into groups (sub-ranges of the row blocks
// I_i).  A work item is one (group, tile) pair.  Inside a work item every row
// that touches the tile contributes one segment (its nonzeros in that tile).
// Segments are packed 32 to a slab; a slab is stored in column groups of
// kGroup elements (elements [4kk, 4kk+4) of every segment longer than 4kk, in
// lane order, tails padded with zero weights), so that a warp reads it with
// coalesced 16-byte loads, one lane per segment.
constexpr int kTileH = 64;
constexpr int kTileW = 64;
constexpr int kTileStride = kTileW + 1;   // padded shared-memory row stride (floats)
constexpr int kSlab = 32;
constexpr int kGroup = 4;                            // elements per lane per vector load
constexpr int kPadBase = kTileH * kTileStride;        // per-lane dummy words for padding
constexpr int kTileWords = kPadBase + kSlab;          // shared-memory words per tile array

struct Tile {
    int32_t r0, c0, h, w;   // image rows [r0, r0+h), cols [c0, c0+w)
    int32_t band;           // column block j containing the tile
    int32_t pad_;
};

struct WorkItem {
    int32_t tile;
    int32_t group;
    int32_t slab_begin;
    int32_t slab_end;
};

struct HostLayout {
    int img_h = 0, img_w = 0;
    int64_t rows = 0, cols = 0, nnz = 0, stored = 0;   // stored: nnz + padding
    double colsum_max = 0.0;   // max over row groups and pixels of sum_rows |a| (FP32 weights)
    int M = 0, N = 0;
    std::vector<int64_t> row_bounds, col_bounds;   // I_i, J_j
    std::vector<Tile> tiles;
    std::vector<int64_t> group_bounds;              // [n_groups+1] row ranges
    std::vector<int32_t> group_block;               // block i of each group
    std::vector<WorkItem> items;                    // launch order (nnz descending)
    std::vector<int64_t> item_nnz;
    std::vector<int64_t> slab_off;                  // [n_slabs+1]
    std::vector<int32_t> slab_item;                 // [n_slabs] item index (storage order)
    std::vector<int32_t> seg_ray, seg_len;          // [n_slabs*32]
    int fmt = 0;                                    // BSGDTV_FMT_*
    std::vector<float> vals;                        // [stored] slab-ordered (as stored, in FP32)
    std::vector<int32_t> idx;                       // [stored] tile-local shared-memory word
    std::vector<uint16_t> vals16;                   // binary16 / bfloat16 bits (16-bit formats)
    std::vector<uint16_t> idx16;                    // 16-bit indices (all but FMT_F32_I32)
    std::vector<int32_t> ray_seg_ptr;               // [rows+1]
    std::vector<int32_t> ray_seg_pos;               // [n_segments] segment slots, ascending tile
    int64_t n_groups() const { return (int64_t)group_block.size(); }
    int64_t n_slabs() const { return (int64_t)slab_item.size(); }
};

// Validates the CSR and builds the layout (host, multithreaded).  Returns a
// BSGDTV_* code; on failure set_error has the reason.
int build_layout(HostLayout &L, int64_t rows, int64_t cols, int img_h, int img_w,
                 const int64_t *row_ptr, const int32_t *col_idx, const double *vals, int M, int N,
                 const int64_t *row_bounds, const int64_t *col_bounds, int target_items, int fmt);
// Stored-weight conversions (round to nearest even) and sizes.
uint16_t double_to_half_bits(double v);
uint16_t double_to_bf16_bits(double v);
float stored_weight(double v, int fmt);
int bytes_per_entry(int fmt);

// Decodes the layout back into CSR and compares with the input (host check).
int verify_layout(const HostLayout &L, const int64_t *row_ptr, const int32_t *col_idx,
                  const double *vals);
std::vector<int64_t> default_bounds(int64_t length, int parts, int64_t unit);
int resolve_bounds(int64_t rows, int64_t cols, int M, int N, int64_t row_unit, int64_t col_unit,
                   const int64_t *row_bounds, const int64_t *col_bounds, std::vector<int64_t> &rb,
                   std::vector<int64_t> &cb);

// ------------------------------------------------------------ device views
struct DevLayout {
    const void *vals = nullptr;   // float, or 16-bit weight bits (see fmt)
    const void *idx = nullptr;    // int32, or uint16 (see fmt)
    int fmt = 0;
    const int64_t *slab_off = nullptr;
    const int32_t *seg_ray = nullptr;
    const int32_t *seg_len = nullptr;
    const WorkItem *items = nullptr;
    const Tile *tiles = nullptr;
    const int32_t *ray_seg_ptr = nullptr;
    const int32_t *ray_seg_pos = nullptr;
    const int32_t *slab_item = nullptr;
    const int32_t *group_block = nullptr;
    int *item_ctr = nullptr;   // [2] work-item / exit counters of the product kernel (device)
    float colsum_max = 0.f;    // see HostLayout::colsum_max (rounded up)
    int n_sms = 1;
    int n_items = 0;
    int n_groups = 0;
    int n_tiles = 0;
    int M = 0, N = 0;
    int64_t n_slabs = 0;
    int64_t rows = 0, cols = 0;
    int img_h = 0, img_w = 0;
};

// products.cu: one pass over A.  z_part[slot] = sum over the segment of a*x,
// g_part[group*cols + pixel] = sum over the group's rows of 2*a*r.
cudaError_t prepare_products_kernels();   // sets shared-memory limits (call before capture)
// 16-bit formats (products_fmt.cu), dispatched by launch_products32/64.
cudaError_t launch_products32_fmt(const DevLayout &d, const float *x, const float *r,
                                  const float *rmax_in, float *rmax_clear, float *z_part,
                                  int32_t *g_part, cudaStream_t s, bool pdl);
cudaError_t launch_products64_fmt(const DevLayout &d, const double *x, const double *r,
                                  double *z_part, double *g_part, cudaStream_t s);
cudaError_t prepare_products_fmt_kernels();
// FP64 variant (u_max and objective): g tile accumulated with FP64 atomics.
cudaError_t launch_products64(const DevLayout &d, const double *x, const double *r, double *z_part,
                              double *g_part, cudaStream_t s);
// FP32 hot path: the A^T r tile is accumulated in int32 fixed point with the
// power-of-two scale fixed_scale(*rmax_in, d.colsum_max); g_part holds int32.
// rmax_clear (may be null) is set to 0 for the next reduction to fill.
cudaError_t launch_products32(const DevLayout &d, const float *x, const float *r,
                              const float *rmax_in, float *rmax_clear, float *z_part,
                              int32_t *g_part, cudaStream_t s, bool pdl = false);

// Scale 2^e such that 2 * rmax * colsum_max * 2^e < 2^30: every partial sum of
// the fixed-point A^T r tile stays below 2^31 in magnitude.
__host__ __device__ inline float fixed_scale(float rmax, float colsum_max) {
    const float bound = 2.0f * rmax * colsum_max;
    if (!(bound > 0.0f) || !(bound < 3.0e38f)) return 1.0f;
    int ex = 0;
    frexpf(bound, &ex);   // bound < 2^ex
    int e = 30 - ex;
    if (e > 120) e = 120;
    if (e < -120) e = -120;
    return ldexpf(1.0f, e);
}

// reduce.cu
// r_out = y - sum of each row's segment partials; x_out = x + mu * sum_g g_part
// (x_out may equal x).  y may be null (then r_out = +sum, used for A v).
cudaError_t launch_reduce_update64(const DevLayout &d, const double *z_part, const double *g_part,
                                   const double *y, double *r_out, const double *x, double *x_out,
                                   double mu, cudaStream_t s);
// FP32 hot path: g_part is the fixed-point tile of launch_products32 (scale from
// rmax_in); the new residual's max |r| is folded into rmax_out (pre-zeroed).
cudaError_t launch_reduce_update32(const DevLayout &d, const float *z_part, const int32_t *g_part,
                                   const float *rmax_in, const float *y, float *r_out,
                                   float *rmax_out, const float *x, float *x_out, float mu,
                                   cudaStream_t s, bool pdl = false);
// Stochastic variant: the reductions restricted to the drawn row blocks
// (sel_i [M]) and column blocks (sel_j [N]); rb [M+1], cb [N+1] are the block
// bounds; rows / pixels outside keep r_in / x.
cudaError_t launch_reduce_subset32(const DevLayout &d, const float *z_part, const int32_t *g_part,
                                   const float *rmax_in, const float *y, const float *r_in,
                                   float *r_out, float *rmax_out, const float *x, float *x_out,
                                   float mu, const int64_t *rb, const int64_t *cb,
                                   const uint8_t *sel_i, const uint8_t *sel_j, cudaStream_t s);
cudaError_t launch_block_sums(const DevLayout &d, const float *z_part, const int32_t *g_part,
                              const float *rmax_in, float *z_blocks, float *g_blocks,
                              cudaStream_t s);
// out[0] = max |v| over n (out must be zeroed first; result via integer max on float bits).
cudaError_t launch_absmax(const float *v, int64_t n, float *out, cudaStream_t s);
// Deterministic FP64 reductions: out[0] = sum a*b (b null: sum a*a) over n.
cudaError_t launch_dot(const double *a, const double *b, int64_t n, double *partials,
                       double *out, cudaStream_t s);
cudaError_t launch_tv64(const float *x, int h, int w, double *partials, double *out,
                        cudaStream_t s);
cudaError_t launch_f32_to_f64(const float *in, double *out, int64_t n, cudaStream_t s);
cudaError_t launch_fill64(double *out, double v, int64_t n, cudaStream_t s);
cudaError_t launch_scale64(const double *in, const double *nrm2, double *out, int64_t n,
                           cudaStream_t s);
cudaError_t launch_check_finite(const float *v, int64_t n, int *flag, cudaStream_t s);
constexpr int kDotPartials = 1024;

// fgp.cu: K FGP iterations on an h x w image.  `mom` holds the K momentum
// coefficients (iteration k uses mom[k-1]); p,q,pp,qp are h*w scratch fields.
struct FgpScratch {
    float *p, *q, *pp, *qp;
};
// Iterations per launch for an h x w image on n_sms SMs (a cost model of
// halo recomputation, waves and launches; every choice gives the same iterates).
int fgp_chunk_for(int h, int w, int iters, int n_sms);
int fgp_plan_launches(int h, int w, int iters, int max_chunk = 8);
cudaError_t launch_fgp(const float *b, float *x, int h, int w, float tau, int iters,
                       const float *mom, FgpScratch sc, cudaStream_t s, bool pdl = false,
                       int max_chunk = 8);
void fgp_momentum_host(int iters, std::vector<float> &mom);

// batch.cu: host check of a CSR image operator (sizes, sorted in-range
// columns, finite weights); BSGDTV_* code.
int validate_image_csr(int64_t rows, int64_t cols, int img_h, int img_w, const int64_t *row_ptr,
                       const int32_t *col_idx, const double *vals);

}  // namespace bsgdtv
