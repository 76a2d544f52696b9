// The tiled operator layout of the fused block products: tile and slab
// constants, work items, the host layout built once per A (layout.cpp) and
// its device view.  Everything the product kernels read is defined here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

namespace bsgdtv {

// ------------------------------------------------------- tiled operator layout
// The image is cut into pixel tiles (at most kTileH x kTileW, never crossing a
// column-block band J_j) and the rows into groups (sub-ranges of the row blocks
// I_i).  A work item is one (group, tile) pair.  Inside a work item every row
// that touches the tile contributes one segment (its nonzeros in that tile).
// Segments are packed 32 to a slab; a slab is stored in column groups of G
// elements (elements [G kk, G kk + G) of every segment longer than G kk, in
// lane order, tails padded with zero weights), so that a warp reads it with
// coalesced 16-byte loads, one lane per segment: G = 4 for FP32 weights,
// G = 8 for 16-bit weights with 16-bit indices (16 bytes of weights and 16 of
// indices per lane and group, the same registers per group as FP32 with
// 32-bit indices and twice the nonzeros).
constexpr int kTileH = 64;
constexpr int kTileW = 64;
constexpr int kTileStride = kTileW + 1;   // padded shared-memory row stride (floats)
constexpr int kSlab = 32;
constexpr int kGroup = 4;                            // elements per lane per load (FP32 weights)
constexpr int kGroup16 = 8;                          // the same for 16-bit weights
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
    int group = kGroup;                             // elements per column group (group_size(fmt))
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
// Elements per column group of a slab for a stored format.
inline int group_size(int fmt) { return (fmt == 2 || fmt == 3) ? kGroup16 : kGroup; }

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

}  // namespace bsgdtv
