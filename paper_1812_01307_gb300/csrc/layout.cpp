// Host construction of the tiled, slab-packed operator layout.
//
// Partition (Sec. 2.1 of the paper): rows of A are split into M row blocks
// I_i, columns into N column blocks J_j.  Default bounds follow
// numpy.array_split over whole units (an angle's rays, an image row).
// The GPU layout refines that partition: pixel tiles never cross a J_j band
// and row groups never cross an I_i block, so every block product of lines
// 3-4 of Algorithm 1 is a sum of work-item partials.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <cmath>
#include <numeric>
#include <thread>

#include "bsgdtv_internal.h"

namespace bsgdtv {

static std::vector<int64_t> split_units(int64_t units, int parts, int64_t unit) {
    std::vector<int64_t> b(parts + 1, 0);
    int64_t q = units / parts, rem = units % parts;
    for (int k = 0; k < parts; ++k) b[k + 1] = b[k] + q + (k < rem ? 1 : 0);
    for (auto &v : b) v *= unit;
    return b;
}

std::vector<int64_t> default_bounds(int64_t length, int parts, int64_t unit) {
    return split_units(length / unit, parts, unit);
}

template <typename F>
static void parallel_for(int64_t n, F &&f) {
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int64_t nt = std::min<int64_t>(n, std::min<unsigned>(hw, 32u));
    if (nt <= 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    std::atomic<int64_t> next(0);
    for (int64_t t = 0; t < nt; ++t)
        th.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                f(i);
            }
        });
    for (auto &t : th) t.join();
}

// ------------------------------------------------ stored weight formats
// Round-to-nearest-even conversion of a double to IEEE binary16 / bfloat16
// bits, written from the formats' definitions (sign, biased exponent,
// truncated significand; ties to the even significand).
static uint16_t round_bits(uint64_t mant53, int shift, uint16_t base) {
    // base + (mant53 >> shift), rounded to nearest even on the dropped bits
    if (shift >= 64) return base;
    const uint64_t kept = mant53 >> shift;
    const uint64_t rem = mant53 & ((shift ? (1ull << shift) : 1ull) - 1ull);
    const uint64_t half = shift ? (1ull << (shift - 1)) : 0ull;
    uint64_t r = kept;
    if (shift && (rem > half || (rem == half && (kept & 1ull)))) ++r;
    return (uint16_t)(base + r);
}

uint16_t double_to_half_bits(double v) {
    uint64_t x;
    std::memcpy(&x, &v, 8);
    const uint16_t sign = (uint16_t)((x >> 48) & 0x8000u);
    const int ex = (int)((x >> 52) & 0x7FF);
    const uint64_t m = x & ((1ull << 52) - 1);
    if (ex == 0x7FF) return (uint16_t)(sign | 0x7C00u | (m ? 0x200u : 0u));
    if (ex == 0) return sign;   // zero or double subnormal (far below half's range)
    const int e = ex - 1023;
    const uint64_t full = m | (1ull << 52);
    if (e >= -14) {             // normal half: 10 significand bits, carry may bump the exponent
        if (e > 15) return (uint16_t)(sign | 0x7C00u);
        const uint16_t h = round_bits(full, 42, 0) ;   // 11 bits incl. the implicit one
        const uint32_t biased = (uint32_t)(e + 15);
        uint32_t bits = (biased << 10) + (uint32_t)(h - 0x400u);
        if (bits >= 0x7C00u) bits = 0x7C00u;
        return (uint16_t)(sign | bits);
    }
    // subnormal half: units of 2^-24
    return (uint16_t)(sign | round_bits(full, 28 - e, 0));
}

uint16_t double_to_bf16_bits(double v) {
    uint64_t x;
    std::memcpy(&x, &v, 8);
    const uint16_t sign = (uint16_t)((x >> 48) & 0x8000u);
    const int ex = (int)((x >> 52) & 0x7FF);
    const uint64_t m = x & ((1ull << 52) - 1);
    if (ex == 0x7FF) return (uint16_t)(sign | 0x7F80u | (m ? 0x40u : 0u));
    if (ex == 0) return sign;
    const int e = ex - 1023;
    const uint64_t full = m | (1ull << 52);
    if (e >= -126) {            // normal bfloat16: 7 significand bits
        if (e > 127) return (uint16_t)(sign | 0x7F80u);
        const uint16_t h = round_bits(full, 45, 0);     // 8 bits incl. the implicit one
        const uint32_t biased = (uint32_t)(e + 127);
        uint32_t bits = (biased << 7) + (uint32_t)(h - 0x80u);
        if (bits >= 0x7F80u) bits = 0x7F80u;
        return (uint16_t)(sign | bits);
    }
    return (uint16_t)(sign | round_bits(full, -e - 81, 0));   // units of 2^-133
}

float half_bits_to_float(uint16_t h) {
    const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
    const int ex = (h >> 10) & 0x1F;
    const uint32_t m = h & 0x3FFu;
    float f;
    if (ex == 0) {
        f = std::ldexp((float)m, -24);
    } else if (ex == 31) {
        f = m ? NAN : INFINITY;
    } else {
        f = std::ldexp((float)(m | 0x400u), ex - 25);
    }
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b |= sign;
    std::memcpy(&f, &b, 4);
    return f;
}

float bf16_bits_to_float(uint16_t h) {
    const uint32_t b = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// The weight as the device stores it, widened back to FP32 (exact).
float stored_weight(double v, int fmt) {
    switch (fmt) {
        case BSGDTV_FMT_F16_I16: return half_bits_to_float(double_to_half_bits(v));
        case BSGDTV_FMT_BF16_I16: return bf16_bits_to_float(double_to_bf16_bits(v));
        default: return (float)v;
    }
}

int bytes_per_entry(int fmt) {
    switch (fmt) {
        case BSGDTV_FMT_F32_I32: return 8;
        case BSGDTV_FMT_F32_I16: return 6;
        default: return 4;
    }
}

int build_layout(HostLayout &L, int64_t rows, int64_t cols, int img_h, int img_w,
                 const int64_t *row_ptr, const int32_t *col_idx, const double *vals, int M, int N,
                 const int64_t *row_bounds, const int64_t *col_bounds, int target_items, int fmt) {
    // ---------------------------------------------------------- validation
    if (fmt < BSGDTV_FMT_F32_I32 || fmt > BSGDTV_FMT_BF16_I16)
        return fail(BSGDTV_ERR_INVALID_ARG, "unknown weight format");
    if (rows < 1 || cols < 1 || img_h < 1 || img_w < 1 || (int64_t)img_h * img_w != cols)
        return fail(BSGDTV_ERR_INVALID_ARG, "bad sizes: need rows>=1 and cols == img_h*img_w");
    if (rows >= (int64_t)1 << 31 || cols >= (int64_t)1 << 31)
        return fail(BSGDTV_ERR_INVALID_ARG, "rows and cols must be < 2^31");
    if (M < 1 || N < 1 || M > rows || N > img_h)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= M <= rows and 1 <= N <= img_h");
    if (!row_ptr || (!col_idx && row_ptr[rows] > 0) || (!vals && row_ptr[rows] > 0))
        return fail(BSGDTV_ERR_INVALID_ARG, "null CSR array");
    if (row_ptr[0] != 0) return fail(BSGDTV_ERR_INVALID_ARG, "row_ptr[0] != 0");
    for (int64_t r = 0; r < rows; ++r)
        if (row_ptr[r + 1] < row_ptr[r]) return fail(BSGDTV_ERR_INVALID_ARG, "row_ptr decreasing");
    const int64_t nnz = row_ptr[rows];
    {
        std::atomic<int> bad(0);
        parallel_for(rows, [&](int64_t r) {
            int64_t prev = -1;
            for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                int64_t c = col_idx[e];
                if (c < 0 || c >= cols || c <= prev) bad.store(1);
                if (!std::isfinite(vals[e])) bad.store(2);
                prev = c;
            }
        });
        if (bad.load() == 1)
            return fail(BSGDTV_ERR_INVALID_ARG, "column index out of range or not ascending in a row");
        if (bad.load() == 2) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in A");
    }
    L.fmt = fmt;
    L.img_h = img_h;
    L.img_w = img_w;
    L.rows = rows;
    L.cols = cols;
    L.nnz = nnz;
    L.M = M;
    L.N = N;
    L.row_bounds.assign(row_bounds, row_bounds + M + 1);
    L.col_bounds.assign(col_bounds, col_bounds + N + 1);
    if (L.row_bounds[0] != 0 || L.row_bounds[M] != rows || L.col_bounds[0] != 0 ||
        L.col_bounds[N] != cols)
        return fail(BSGDTV_ERR_INVALID_ARG, "bounds must start at 0 and end at rows / cols");
    for (int i = 0; i < M; ++i)
        if (L.row_bounds[i + 1] < L.row_bounds[i]) return fail(BSGDTV_ERR_INVALID_ARG, "row bounds decreasing");
    for (int j = 0; j < N; ++j) {
        if (L.col_bounds[j + 1] < L.col_bounds[j]) return fail(BSGDTV_ERR_INVALID_ARG, "col bounds decreasing");
        if (L.col_bounds[j] % img_w) return fail(BSGDTV_ERR_INVALID_ARG, "column blocks must be bands of whole image rows");
    }

    // ------------------------------------------------------------- tiles
    // tile rows never cross a band J_j; tiles are stored row-major over
    // (tile row, tile column)
    std::vector<int32_t> tile_row_of(img_h);
    struct TileRow { int32_t r0, h, band; };
    std::vector<TileRow> trows;
    for (int j = 0; j < N; ++j) {
        int b0 = (int)(L.col_bounds[j] / img_w), b1 = (int)(L.col_bounds[j + 1] / img_w);
        for (int r0 = b0; r0 < b1; r0 += kTileH) {
            int h = std::min(kTileH, b1 - r0);
            for (int rr = r0; rr < r0 + h; ++rr) tile_row_of[rr] = (int32_t)trows.size();
            trows.push_back({r0, h, j});
        }
    }
    const int n_tc = (img_w + kTileW - 1) / kTileW;
    L.tiles.clear();
    for (const TileRow &tr : trows) {
        for (int tc = 0; tc < n_tc; ++tc) {
            Tile t;
            t.r0 = tr.r0;
            t.c0 = tc * kTileW;
            t.h = tr.h;
            t.w = std::min(kTileW, img_w - t.c0);
            t.band = tr.band;
            t.pad_ = 0;
            L.tiles.push_back(t);
        }
    }
    const int n_tiles = (int)L.tiles.size();

    // ------------------------------------------------------------ groups
    int64_t pairs = (int64_t)M * n_tiles;
    int n_sub = (int)std::max<int64_t>(1, (target_items + pairs / 2) / std::max<int64_t>(pairs, 1));
    L.group_bounds.assign(1, 0);
    L.group_block.clear();
    for (int i = 0; i < M; ++i) {
        int64_t len = L.row_bounds[i + 1] - L.row_bounds[i];
        int sub = (int)std::min<int64_t>(n_sub, std::max<int64_t>(len, 1));
        std::vector<int64_t> b = split_units(len, sub, 1);
        for (int k = 0; k < sub; ++k) {
            L.group_bounds.push_back(L.row_bounds[i] + b[k + 1]);
            L.group_block.push_back(i);
        }
    }
    const int n_groups = (int)L.group_block.size();
    const int64_t n_pairs = (int64_t)n_groups * n_tiles;

    auto tile_of = [&](int32_t c, int32_t &local) -> int32_t {
        int32_t s = c / img_w, t = c % img_w;
        int32_t tr = tile_row_of[s], tc = t / kTileW;
        int32_t tid = tr * n_tc + tc;
        const Tile &T = L.tiles[tid];
        local = (s - T.r0) * kTileStride + (t - T.c0);
        return tid;
    };

    // ---------------------------------------------- pass 1: counts per pair
    // pair_nnz: stored elements (each segment padded to a multiple of G)
    const int G = group_size(fmt);
    L.group = G;
    std::vector<int64_t> pair_nnz(n_pairs, 0), pair_seg(n_pairs, 0), pair_real(n_pairs, 0);
    // largest column sum of |a| (FP32 weights) within one row group: bounds the
    // fixed-point accumulation of the A^T r tile
    std::vector<double> group_colmax(n_groups, 0.0);
    parallel_for(n_groups, [&](int64_t g) {
        std::vector<int32_t> cnt(n_tiles, 0);
        std::vector<int32_t> touched;
        std::vector<double> colsum(cols, 0.0);
        for (int64_t r = L.group_bounds[g]; r < L.group_bounds[g + 1]; ++r)
            for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
                colsum[col_idx[e]] += std::fabs((double)stored_weight(vals[e], fmt));
        double cm = 0.0;
        for (double v : colsum) cm = std::max(cm, v);
        group_colmax[g] = cm;
        int64_t *pn = &pair_nnz[g * n_tiles], *ps = &pair_seg[g * n_tiles], *pr = &pair_real[g * n_tiles];
        for (int64_t r = L.group_bounds[g]; r < L.group_bounds[g + 1]; ++r) {
            for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                int32_t loc;
                int32_t t = tile_of(col_idx[e], loc);
                if (cnt[t]++ == 0) touched.push_back(t);
            }
            for (int32_t t : touched) {
                ps[t]++;
                pr[t] += cnt[t];
                pn[t] += (int64_t)G * ((cnt[t] + G - 1) / G);
                cnt[t] = 0;
            }
            touched.clear();
        }
    });

    L.colsum_max = 0.0;
    for (double v : group_colmax) L.colsum_max = std::max(L.colsum_max, v);

    // storage order of pairs: group-major, tile ascending
    std::vector<int64_t> pair_slab0(n_pairs + 1, 0), pair_nnz0(n_pairs + 1, 0);
    for (int64_t p = 0; p < n_pairs; ++p) {
        pair_slab0[p + 1] = pair_slab0[p] + (pair_seg[p] + kSlab - 1) / kSlab;
        pair_nnz0[p + 1] = pair_nnz0[p] + pair_nnz[p];
    }
    const int64_t n_slabs = pair_slab0[n_pairs];
    if (n_slabs * kSlab >= ((int64_t)1 << 31))
        return fail(BSGDTV_ERR_UNSUPPORTED, "too many row segments for 32-bit slots");
    L.slab_off.assign(n_slabs + 1, 0);
    L.slab_item.assign(n_slabs, 0);
    L.seg_ray.assign(n_slabs * kSlab, 0);
    L.seg_len.assign(n_slabs * kSlab, 0);
    const int64_t stored = pair_nnz0[n_pairs];
    L.stored = stored;
    L.vals.assign(stored, 0.0f);
    L.idx.assign(stored, 0);

    // ------------------------------------- pass 2: segments, slab packing
    parallel_for(n_groups, [&](int64_t g) {
        // per pair of this group: segment starts (in a row-ordered scratch copy)
        std::vector<int64_t> cursor_nnz(n_tiles, 0);
        int64_t real_total = 0;
        std::vector<int64_t> real0(n_tiles + 1, 0);
        for (int t = 0; t < n_tiles; ++t) real0[t + 1] = real0[t] + pair_real[g * n_tiles + t];
        real_total = real0[n_tiles];
        std::vector<float> tv(real_total);
        std::vector<int32_t> ti(real_total);
        // segments of pair (g,t): row, start (in tv/ti), length
        std::vector<std::vector<int64_t>> srow(n_tiles), sstart(n_tiles), slen(n_tiles);
        for (int t = 0; t < n_tiles; ++t) {
            srow[t].reserve(pair_seg[g * n_tiles + t]);
            sstart[t].reserve(pair_seg[g * n_tiles + t]);
            slen[t].reserve(pair_seg[g * n_tiles + t]);
            cursor_nnz[t] = real0[t];
        }
        std::vector<int64_t> last(n_tiles, -1);
        for (int64_t r = L.group_bounds[g]; r < L.group_bounds[g + 1]; ++r) {
            // first sweep: open one segment per tile touched (in order of first touch)
            for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                int32_t loc;
                int32_t t = tile_of(col_idx[e], loc);
                if (last[t] != r) {
                    last[t] = r;
                    srow[t].push_back(r);
                    sstart[t].push_back(cursor_nnz[t]);
                    slen[t].push_back(0);
                }
                int64_t pos = cursor_nnz[t]++;
                tv[pos] = stored_weight(vals[e], fmt);
                ti[pos] = loc;
                slen[t].back()++;
            }
        }
        // Entries of one segment are contiguous in tv/ti only if no other
        // segment of the same pair was opened in between, which holds because
        // a row is finished before the next row starts.
        for (int t = 0; t < n_tiles; ++t) {
            const int64_t pair = g * n_tiles + t;
            const int64_t nseg = (int64_t)srow[t].size();
            int64_t out = pair_nnz0[pair];
            for (int64_t s0 = 0, sl = pair_slab0[pair]; s0 < nseg; s0 += kSlab, ++sl) {
                int lanes = (int)std::min<int64_t>(kSlab, nseg - s0);
                L.slab_off[sl] = out;
                int maxlen = 0;
                for (int l = 0; l < lanes; ++l) {
                    L.seg_ray[sl * kSlab + l] = (int32_t)srow[t][s0 + l];
                    L.seg_len[sl * kSlab + l] = (int32_t)slen[t][s0 + l];
                    maxlen = std::max<int>(maxlen, (int)slen[t][s0 + l]);
                }
                // column groups of G elements: group kk holds elements
                // [G*kk, G*kk + G) of every lane whose segment is longer than
                // G*kk, in lane order; short tails are padded with zero
                // weights aimed at the lane's private dummy word
                const int maxg = (maxlen + G - 1) / G;
                for (int kk = 0; kk < maxg; ++kk)
                    for (int l = 0; l < lanes; ++l) {
                        const int64_t len = slen[t][s0 + l];
                        if (len <= (int64_t)G * kk) continue;
                        for (int j = 0; j < G; ++j) {
                            const int64_t k = (int64_t)G * kk + j;
                            if (k < len) {
                                const int64_t src = sstart[t][s0 + l] + k;
                                L.vals[out] = tv[src];
                                L.idx[out] = ti[src];
                            } else {
                                L.vals[out] = 0.0f;
                                L.idx[out] = kPadBase + l;
                            }
                            ++out;
                        }
                    }
            }
            for (int64_t sl = pair_slab0[pair]; sl < pair_slab0[pair + 1]; ++sl)
                L.slab_item[sl] = (int32_t)pair;
        }
    });
    L.slab_off[n_slabs] = stored;

    // --------------------------------------- per-ray segment slots (z reduce)
    L.ray_seg_ptr.assign(rows + 1, 0);
    for (int64_t sl = 0; sl < n_slabs; ++sl)
        for (int l = 0; l < kSlab; ++l)
            if (L.seg_len[sl * kSlab + l] > 0) L.ray_seg_ptr[L.seg_ray[sl * kSlab + l] + 1]++;
    for (int64_t r = 0; r < rows; ++r) L.ray_seg_ptr[r + 1] += L.ray_seg_ptr[r];
    L.ray_seg_pos.assign(L.ray_seg_ptr[rows], 0);
    {
        std::vector<int32_t> cur(L.ray_seg_ptr.begin(), L.ray_seg_ptr.end() - 1);
        // slabs are stored group-major with tiles ascending, so each ray meets
        // its segments in ascending tile order
        for (int64_t sl = 0; sl < n_slabs; ++sl)
            for (int l = 0; l < kSlab; ++l)
                if (L.seg_len[sl * kSlab + l] > 0)
                    L.ray_seg_pos[cur[L.seg_ray[sl * kSlab + l]]++] = (int32_t)(sl * kSlab + l);
    }

    // ------------------------------------------------- work items (launch order)
    L.items.resize(n_pairs);
    L.item_nnz.resize(n_pairs);
    std::vector<int64_t> order(n_pairs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return pair_nnz[a] > pair_nnz[b]; });
    for (int64_t k = 0; k < n_pairs; ++k) {
        int64_t p = order[k];
        WorkItem w;
        w.group = (int32_t)(p / n_tiles);
        w.tile = (int32_t)(p % n_tiles);
        w.slab_begin = (int32_t)pair_slab0[p];
        w.slab_end = (int32_t)pair_slab0[p + 1];
        L.items[k] = w;
        L.item_nnz[k] = pair_nnz[p];
    }
    // 16-bit forms: indices fit (kTileWords < 2^16); weights as binary16 / bfloat16 bits
    if (fmt != BSGDTV_FMT_F32_I32) {
        L.idx16.resize(L.idx.size());
        for (size_t k = 0; k < L.idx.size(); ++k) L.idx16[k] = (uint16_t)L.idx[k];
    }
    if (fmt == BSGDTV_FMT_F16_I16 || fmt == BSGDTV_FMT_BF16_I16) {
        L.vals16.resize(L.vals.size());
        for (size_t k = 0; k < L.vals.size(); ++k)
            L.vals16[k] = fmt == BSGDTV_FMT_F16_I16 ? double_to_half_bits(L.vals[k])
                                                     : double_to_bf16_bits(L.vals[k]);
    }
    return BSGDTV_OK;
}

int verify_layout(const HostLayout &L, const int64_t *row_ptr, const int32_t *col_idx,
                  const double *vals) {
    const int n_tiles = (int)L.tiles.size();
    std::vector<std::vector<std::pair<int32_t, float>>> per_row(L.rows);
    std::vector<std::vector<int32_t>> slots_of_row(L.rows);
    for (int64_t sl = 0; sl < L.n_slabs(); ++sl) {
        const int pair = L.slab_item[sl];
        const int g = pair / n_tiles, t = pair % n_tiles;
        const Tile &T = L.tiles[t];
        int maxlen = 0;
        for (int l = 0; l < kSlab; ++l) {
            const int len = L.seg_len[sl * kSlab + l];
            const int ray = L.seg_ray[sl * kSlab + l];
            if (len < 0) return fail(BSGDTV_ERR_STATE, "negative segment length");
            if (len > 0) {
                if (ray < L.group_bounds[g] || ray >= L.group_bounds[g + 1])
                    return fail(BSGDTV_ERR_STATE, "segment row outside its group");
                slots_of_row[ray].push_back((int32_t)(sl * kSlab + l));
            }
            maxlen = std::max(maxlen, len);
        }
        int64_t pos = L.slab_off[sl];
        const int G = L.group;
        const int maxg = (maxlen + G - 1) / G;
        for (int kk = 0; kk < maxg; ++kk)
            for (int l = 0; l < kSlab; ++l) {
                const int len = L.seg_len[sl * kSlab + l];
                if (len <= G * kk) continue;
                for (int j = 0; j < G; ++j, ++pos) {
                    const int32_t loc = L.idx[pos];
                    if (G * kk + j >= len) {
                        if (loc != kPadBase + l || L.vals[pos] != 0.0f)
                            return fail(BSGDTV_ERR_STATE, "bad padding entry");
                        continue;
                    }
                    const int lr = loc / kTileStride, lc = loc % kTileStride;
                    if (loc < 0 || lr >= T.h || lc >= T.w) return fail(BSGDTV_ERR_STATE, "local index outside tile");
                    const int32_t col = (T.r0 + lr) * L.img_w + T.c0 + lc;
                    per_row[L.seg_ray[sl * kSlab + l]].push_back({col, L.vals[pos]});
                }
            }
        if (pos % G) return fail(BSGDTV_ERR_STATE, "slab not aligned");
        if (pos != L.slab_off[sl + 1]) return fail(BSGDTV_ERR_STATE, "slab size mismatch");
    }
    for (int64_t r = 0; r < L.rows; ++r) {
        auto &v = per_row[r];
        std::sort(v.begin(), v.end());
        if ((int64_t)v.size() != row_ptr[r + 1] - row_ptr[r]) return fail(BSGDTV_ERR_STATE, "row nnz mismatch");
        for (size_t k = 0; k < v.size(); ++k) {
            const int64_t e = row_ptr[r] + (int64_t)k;
            if (v[k].first != col_idx[e] || v[k].second != stored_weight(vals[e], L.fmt))
                return fail(BSGDTV_ERR_STATE, "entry mismatch");
        }
        // the reduction visits exactly this row's segments, tiles ascending
        const int32_t b0 = L.ray_seg_ptr[r], b1 = L.ray_seg_ptr[r + 1];
        if (b1 - b0 != (int32_t)slots_of_row[r].size()) return fail(BSGDTV_ERR_STATE, "segment list size");
        int prev_tile = -1;
        for (int32_t e = b0; e < b1; ++e) {
            const int32_t slot = L.ray_seg_pos[e];
            if (L.seg_ray[slot] != r || L.seg_len[slot] <= 0) return fail(BSGDTV_ERR_STATE, "segment list entry");
            const int tile = L.slab_item[slot / kSlab] % n_tiles;
            if (tile <= prev_tile) return fail(BSGDTV_ERR_STATE, "segment list order");
            prev_tile = tile;
        }
    }
    // every (group, tile) pair is exactly one work item
    std::vector<int> seen((size_t)L.n_groups() * n_tiles, 0);
    for (const WorkItem &w : L.items) seen[(size_t)w.group * n_tiles + w.tile]++;
    for (int v : seen)
        if (v != 1) return fail(BSGDTV_ERR_STATE, "work items do not cover the pairs once");
    return BSGDTV_OK;
}

}  // namespace bsgdtv
