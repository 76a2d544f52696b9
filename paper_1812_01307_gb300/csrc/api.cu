// C ABI of the BSGD-TV library: handle lifetime, data, the epoch loop of
// Algorithm 1 (captured once per configuration into CUDA graphs), the FP64
// step-size estimate (Theorem 1) and monitoring (Eq. 1).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

#include "bsgdtv_internal.h"

namespace bsgdtv {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches(0);

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int resolve_bounds(int64_t rows, int64_t cols, int M, int N, int64_t row_unit, int64_t col_unit,
                   const int64_t *row_bounds, const int64_t *col_bounds, std::vector<int64_t> &rb,
                   std::vector<int64_t> &cb) {
    if (rows < 1 || cols < 1 || M < 1 || N < 1)
        return fail(BSGDTV_ERR_INVALID_ARG, "rows, cols, M, N must be >= 1");
    if (!row_bounds && (row_unit < 1 || rows % row_unit || rows / row_unit < M))
        return fail(BSGDTV_ERR_INVALID_ARG, "row_unit must divide rows into at least M units");
    if (!col_bounds && (col_unit < 1 || cols % col_unit || cols / col_unit < N))
        return fail(BSGDTV_ERR_INVALID_ARG, "col_unit must divide cols into at least N units");
    rb = row_bounds ? std::vector<int64_t>(row_bounds, row_bounds + M + 1)
                    : default_bounds(rows, M, row_unit);
    cb = col_bounds ? std::vector<int64_t>(col_bounds, col_bounds + N + 1)
                    : default_bounds(cols, N, col_unit);
    return BSGDTV_OK;
}

}  // namespace bsgdtv

using namespace bsgdtv;

struct bsgdtv_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;     // caller's stream (may be the legacy default)
    cudaStream_t cap_stream = nullptr; // private stream used only for graph capture
    HostLayout host;                   // layout metadata (bulk arrays released after upload)
    DevLayout dl;
    std::vector<void *> allocs;

    float *y = nullptr, *r[2] = {nullptr, nullptr}, *x = nullptr, *xhat = nullptr;
    float *z_part = nullptr, *g_part = nullptr;
    float *fgp = nullptr;   // FGP dual fields: kFgpFieldPlanes planes of cols floats
    float *mom = nullptr;
    int mom_len = 0;
    int *flag = nullptr;
    float *rmax = nullptr;   // [3] max |r| of r[0], r[1] and of a test-hook r
    int *init_part = nullptr;   // [kInitBlocks + 1] block maxima and counter of the init kernel
    float *check_host = nullptr;   // page-locked word: max |y| of the last initialisation
    float *check_dev = nullptr;    // its device address
    int cur = 0;   // r[cur] holds r^{k-1}
    bool z_stale = true;   // z partials not yet A x^0 = 0 or computed by an epoch
    bool has_data = false;
    double lambda = 0.0, mu = 0.0, u_max = 0.0;
    int64_t epoch = 0;
    int64_t seg_count = 0;

    // FP64 scratch (allocated on first use)
    double *v64 = nullptr, *w64 = nullptr, *g64 = nullptr, *z64 = nullptr, *gp64 = nullptr,
           *y64 = nullptr, *x64 = nullptr, *partials = nullptr, *scal = nullptr;

    // stochastic variant: block bounds on the device and a scratch buffer for
    // the per-iteration work-item lists and block masks (grown on demand)
    int64_t *rb_dev = nullptr, *cb_dev = nullptr;
    void *sub_buf = nullptr;
    size_t sub_bytes = 0;

    // graphs: one per parity of the r double buffer
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    // timed variant: event-record nodes around the product kernel and at the
    // end of the epoch, re-pointed to fresh events before every replay
    cudaGraph_t tgraph[2] = {nullptr, nullptr};
    cudaGraphExec_t texec[2] = {nullptr, nullptr};
    cudaGraphNode_t tnode[2][3] = {};
    cudaEvent_t tmark[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> tevents;
    int graph_fgp_iters = -1;
    bool graph_prox = false;
    double graph_mu = 0.0, graph_lambda = 0.0;
    int64_t graph_kernels = 0;
};

namespace {

template <typename T>
int dalloc(bsgdtv_ctx *h, T **out, size_t count) {
    void *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BSGDTV_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                        "): " + cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    *out = static_cast<T *>(p);
    return BSGDTV_OK;
}

template <typename T>
int upload(bsgdtv_ctx *h, T **out, const std::vector<T> &v) {
    BSG_CHECK(dalloc(h, out, v.size()));
    if (!v.empty())
        BSG_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                 h->stream));
    return BSGDTV_OK;
}

void drop_graphs(bsgdtv_ctx *h) {
    for (auto &g : h->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto &g : h->texec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto &g : h->tgraph)
        if (g) {
            cudaGraphDestroy(g);
            g = nullptr;
        }
    for (auto &row : h->tnode)
        for (auto &nd : row) nd = nullptr;
    h->graph_fgp_iters = -1;
}

int ensure_mom(bsgdtv_ctx *h, int iters) {
    if (iters <= h->mom_len) {
        // coefficients are a prefix-stable sequence: reuse
        return BSGDTV_OK;
    }
    std::vector<float> m;
    fgp_momentum_host(iters, m);
    float *d = nullptr;
    BSG_CHECK(dalloc(h, &d, m.size()));
    BSG_CUDA(cudaMemcpy(d, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
    h->mom = d;
    h->mom_len = iters;
    return BSGDTV_OK;
}

// Enqueues one epoch of Algorithm 1 reading r[par] and writing r[1-par].  With
// `marks`, records marks[0] / marks[1] around the product kernel and marks[2]
// at the end of the epoch.  Kernels that follow a kernel are launched with
// programmatic dependent launch (not across the timing marks).
int enqueue_epoch(bsgdtv_ctx *h, int par, int fgp_iters, cudaStream_t s,
                  cudaEvent_t *marks = nullptr) {
    const bool prox = h->lambda > 0.0 && fgp_iters > 0;
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[0], s, cudaEventRecordExternal));
    BSG_CUDA(launch_products32(h->dl, h->x, h->r[par], h->rmax + par, h->rmax + (1 - par),
                               h->z_part, reinterpret_cast<int32_t *>(h->g_part), s, !marks));
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[1], s, cudaEventRecordExternal));
    float *xdst = prox ? h->xhat : h->x;
    BSG_CUDA(launch_reduce_update32(h->dl, h->z_part, reinterpret_cast<const int32_t *>(h->g_part),
                                    h->rmax + par, h->y, h->r[1 - par], h->rmax + (1 - par), h->x,
                                    xdst, (float)h->mu, s, !marks));
    if (prox) {
        const FgpScratch sc = fgp_scratch_planes(h->fgp, h->dl.cols);
        BSG_CUDA(launch_fgp(h->xhat, h->x, h->dl.img_h, h->dl.img_w, (float)(h->mu * h->lambda),
                            fgp_iters, h->mom, sc, s, true,
                            fgp_chunk_for(h->dl.img_h, h->dl.img_w, fgp_iters, h->dl.n_sms)));
    }
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[2], s, cudaEventRecordExternal));
    return BSGDTV_OK;
}

int build_timed_graphs(bsgdtv_ctx *h, int fgp_iters) {
    for (int k = 0; k < 3; ++k)
        if (!h->tmark[k]) BSG_CUDA(cudaEventCreate(&h->tmark[k]));
    const int64_t before = g_launches.load();
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        BSG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_epoch(h, par, fgp_iters, h->cap_stream, h->tmark);
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc != BSGDTV_OK) {
            if (g) cudaGraphDestroy(g);
            g_launches.fetch_sub(g_launches.load() - before);
            return rc;
        }
        if (e != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        h->tgraph[par] = g;
        size_t n = 0;
        BSG_CUDA(cudaGraphGetNodes(g, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        BSG_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            BSG_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            BSG_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < 3; ++k)
                if (ev == h->tmark[k]) h->tnode[par][k] = nd;
        }
        for (int k = 0; k < 3; ++k)
            if (!h->tnode[par][k]) return fail(BSGDTV_ERR_CUDA, "timed graph: event node not found");
        BSG_CUDA(cudaGraphInstantiate(&h->texec[par], g, 0));
    }
    g_launches.fetch_sub(g_launches.load() - before);
    return BSGDTV_OK;
}

int build_graphs(bsgdtv_ctx *h, int fgp_iters) {
    drop_graphs(h);
    BSG_CHECK(ensure_mom(h, std::max(fgp_iters, 1)));
    const int64_t before = g_launches.load();
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        BSG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_epoch(h, par, fgp_iters, h->cap_stream);
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc != BSGDTV_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->gexec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    // capture counted the kernels once per parity; replays are counted in run
    const int64_t per_epoch = (g_launches.load() - before) / 2;
    g_launches.fetch_sub(g_launches.load() - before);
    h->graph_kernels = per_epoch;
    h->graph_fgp_iters = fgp_iters;
    h->graph_prox = h->lambda > 0.0 && fgp_iters > 0;
    h->graph_mu = h->mu;
    h->graph_lambda = h->lambda;
    return BSGDTV_OK;
}

int ensure_fp64(bsgdtv_ctx *h) {
    if (h->v64) return BSGDTV_OK;
    const int64_t c = h->dl.cols, R = h->dl.rows;
    BSG_CHECK(dalloc(h, &h->v64, c));
    BSG_CHECK(dalloc(h, &h->g64, c));
    BSG_CHECK(dalloc(h, &h->x64, c));
    BSG_CHECK(dalloc(h, &h->w64, R));
    BSG_CHECK(dalloc(h, &h->y64, R));
    BSG_CHECK(dalloc(h, &h->z64, h->dl.n_slabs * kSlab));
    BSG_CHECK(dalloc(h, &h->gp64, (size_t)h->dl.n_groups * c));
    BSG_CHECK(dalloc(h, &h->partials, kDotPartials));
    BSG_CHECK(dalloc(h, &h->scal, 8));
    return BSGDTV_OK;
}

int prepare_kernels() {
    BSG_CUDA(prepare_products_kernels());
    return BSGDTV_OK;
}

int set_device(bsgdtv_ctx *h) {
    BSG_CUDA(cudaSetDevice(h->device));
    return BSGDTV_OK;
}

}  // namespace

extern "C" {

const char *bsgdtv_last_error(void) { return g_last_error.c_str(); }

const char *bsgdtv_strerror(int code) {
    switch (code) {
        case BSGDTV_OK: return "ok";
        case BSGDTV_ERR_INVALID_ARG: return "invalid argument";
        case BSGDTV_ERR_OOM: return "out of memory";
        case BSGDTV_ERR_CUDA: return "CUDA error";
        case BSGDTV_ERR_STATE: return "call out of order";
        case BSGDTV_ERR_TIMEOUT: return "device wait timed out";
        case BSGDTV_ERR_NONFINITE: return "non-finite input";
        case BSGDTV_ERR_UNSUPPORTED: return "unsupported";
        case BSGDTV_ERR_CANCELLED: return "cancelled";
        default: return "unknown error";
    }
}

int64_t bsgdtv_launch_count(void) { return g_launches.load(); }

int bsgdtv_partition_bounds(int64_t rows, int64_t cols, int M, int N, int64_t row_unit,
                            int64_t col_unit, int64_t *row_bounds, int64_t *col_bounds) {
    if (!row_bounds || !col_bounds) return fail(BSGDTV_ERR_INVALID_ARG, "null output");
    std::vector<int64_t> rb, cb;
    BSG_CHECK(resolve_bounds(rows, cols, M, N, row_unit, col_unit, nullptr, nullptr, rb, cb));
    std::copy(rb.begin(), rb.end(), row_bounds);
    std::copy(cb.begin(), cb.end(), col_bounds);
    return BSGDTV_OK;
}

float bsgdtv_stored_weight(double v, int format) { return stored_weight(v, format); }

int bsgdtv_layout_check(int64_t rows, int64_t cols, int img_h, int img_w, const int64_t *row_ptr,
                        const int32_t *col_idx, const double *vals, int M, int N,
                        int64_t row_unit, int64_t col_unit, const int64_t *row_bounds,
                        const int64_t *col_bounds, int format, int target_items,
                        int64_t *stats) {
    std::vector<int64_t> rb, cb;
    BSG_CHECK(resolve_bounds(rows, cols, M, N, row_unit, col_unit, row_bounds, col_bounds, rb, cb));
    try {
        HostLayout L;
        BSG_CHECK(build_layout(L, rows, cols, img_h, img_w, row_ptr, col_idx, vals, M, N,
                               rb.data(), cb.data(), target_items, format));
        BSG_CHECK(verify_layout(L, row_ptr, col_idx, vals));
        if (stats) {
            stats[0] = L.nnz;
            stats[1] = (int64_t)L.ray_seg_pos.size();
            stats[2] = L.n_slabs();
            stats[3] = (int64_t)L.items.size();
            stats[4] = L.n_groups();
            stats[5] = (int64_t)L.tiles.size();
        }
    } catch (const std::bad_alloc &) {
        return fail(BSGDTV_ERR_OOM, "host allocation while building the layout");
    }
    return BSGDTV_OK;
}

int bsgdtv_create_csr(bsgdtv_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                      const int64_t *row_ptr, const int32_t *col_idx, const double *vals, int M,
                      int N, int64_t row_unit, int64_t col_unit, const int64_t *row_bounds,
                      const int64_t *col_bounds, void *stream) {
    return bsgdtv_create_csr_ex(out, rows, cols, img_h, img_w, row_ptr, col_idx, vals, M, N,
                                row_unit, col_unit, row_bounds, col_bounds, BSGDTV_FMT_F32_I32,
                                stream);
}

int bsgdtv_create_csr_ex(bsgdtv_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                         const int64_t *row_ptr, const int32_t *col_idx, const double *vals, int M,
                         int N, int64_t row_unit, int64_t col_unit, const int64_t *row_bounds,
                         const int64_t *col_bounds, int format, void *stream) {
    BSG_TRACE();
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    std::vector<int64_t> rb, cb;
    BSG_CHECK(resolve_bounds(rows, cols, M, N, row_unit, col_unit, row_bounds, col_bounds, rb, cb));
    std::unique_ptr<bsgdtv_ctx> h(new (std::nothrow) bsgdtv_ctx());
    if (!h) return fail(BSGDTV_ERR_OOM, "host allocation");
    // the layout is validated and built on the host before any CUDA call
    int sms = 152;
    if (cudaGetDevice(&h->device) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaGetLastError();
    try {
        BSG_CHECK(build_layout(h->host, rows, cols, img_h, img_w, row_ptr, col_idx, vals, M, N,
                               rb.data(), cb.data(), 4 * sms, format));
    } catch (const std::bad_alloc &) {
        return fail(BSGDTV_ERR_OOM, "host allocation while building the layout");
    }
    BSG_CUDA(cudaGetDevice(&h->device));
    h->stream = (cudaStream_t)stream;
    HostLayout &L = h->host;
    BSG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    bsgdtv_ctx *hp = h.get();
    DevLayout &d = h->dl;
    {
        void *v = nullptr, *ix = nullptr;
        int32_t *sr = nullptr, *sln = nullptr, *rsp = nullptr, *rsq = nullptr, *si = nullptr,
                *gb = nullptr;
        int64_t *so = nullptr;
        WorkItem *it = nullptr;
        Tile *tl = nullptr;
        float *v32 = nullptr;
        int32_t *i32 = nullptr;
        uint16_t *v16 = nullptr, *i16 = nullptr;
        int rc = BSGDTV_OK;
        if (format == BSGDTV_FMT_F16_I16 || format == BSGDTV_FMT_BF16_I16) {
            rc = upload(hp, &v16, L.vals16);
            v = v16;
        } else {
            rc = upload(hp, &v32, L.vals);
            v = v32;
        }
        if (!rc) {
            if (format == BSGDTV_FMT_F32_I32) {
                rc = upload(hp, &i32, L.idx);
                ix = i32;
            } else {
                rc = upload(hp, &i16, L.idx16);
                ix = i16;
            }
        }
        if (rc || (rc = upload(hp, &so, L.slab_off)) || (rc = upload(hp, &sr, L.seg_ray)) ||
            (rc = upload(hp, &sln, L.seg_len)) || (rc = upload(hp, &it, L.items)) ||
            (rc = upload(hp, &tl, L.tiles)) || (rc = upload(hp, &rsp, L.ray_seg_ptr)) ||
            (rc = upload(hp, &rsq, L.ray_seg_pos)) || (rc = upload(hp, &si, L.slab_item)) ||
            (rc = upload(hp, &gb, L.group_block)) || (rc = prepare_kernels())) {
            bsgdtv_destroy(h.release());
            return rc;
        }
        d.vals = v;
        d.idx = ix;
        d.fmt = format;
        d.slab_off = so;
        d.seg_ray = sr;
        d.seg_len = sln;
        d.items = it;
        d.tiles = tl;
        d.ray_seg_ptr = rsp;
        d.ray_seg_pos = rsq;
        d.slab_item = si;
        d.group_block = gb;
    }
    d.n_sms = sms;
    d.colsum_max = (float)L.colsum_max;
    if ((double)d.colsum_max < L.colsum_max) d.colsum_max = std::nextafter(d.colsum_max, 3.0e38f);
    d.n_items = (int)L.items.size();
    d.n_groups = (int)L.n_groups();
    d.n_tiles = (int)L.tiles.size();
    d.M = M;
    d.N = N;
    d.n_slabs = L.n_slabs();
    d.rows = rows;
    d.cols = cols;
    d.img_h = img_h;
    d.img_w = img_w;
    h->seg_count = (int64_t)L.ray_seg_pos.size();
    int rc = BSGDTV_OK;
    if ((rc = dalloc(hp, &h->y, rows)) || (rc = dalloc(hp, &h->r[0], rows)) ||
        (rc = dalloc(hp, &h->r[1], rows)) || (rc = dalloc(hp, &h->x, cols)) ||
        (rc = dalloc(hp, &h->xhat, cols)) || (rc = dalloc(hp, &h->z_part, d.n_slabs * kSlab)) ||
        (rc = dalloc(hp, &h->g_part, (size_t)d.n_groups * cols)) || (rc = dalloc(hp, &h->fgp, (size_t)kFgpFieldPlanes * cols)) ||
        (rc = dalloc(hp, &h->flag, 1)) ||
        (rc = dalloc(hp, &d.item_ctr, 2)) || (rc = dalloc(hp, &h->rmax, 3)) ||
        (rc = dalloc(hp, &h->init_part, kInitBlocks + 1))) {
        bsgdtv_destroy(h.release());
        return rc;
    }
    cudaError_t e = cudaMemsetAsync(d.item_ctr, 0, 2 * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->init_part, 0, (kInitBlocks + 1) * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaHostAlloc(&h->check_host, sizeof(float), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&h->check_dev, h->check_host, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        bsgdtv_destroy(h.release());
        return fail(BSGDTV_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    // bulk host arrays are no longer needed
    std::vector<float>().swap(L.vals);
    std::vector<int32_t>().swap(L.idx);
    std::vector<uint16_t>().swap(L.vals16);
    std::vector<uint16_t>().swap(L.idx16);
    std::vector<int32_t>().swap(L.seg_ray);
    std::vector<int32_t>().swap(L.ray_seg_pos);
    *out = h.release();
    return BSGDTV_OK;
}

int bsgdtv_create_parallel_beam(bsgdtv_t *out, int n, int n_angles, int n_bins, int M, int N,
                                int format, void *stream) {
    BSG_TRACE();
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (n < 1 || n > 46340 || n_angles < 1 || n_bins < 1 || (int64_t)n_angles * n_bins > INT32_MAX)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= n <= 46340, n_angles, n_bins >= 1, "
                                            "n_angles * n_bins < 2^31");
    if (M < 1 || M > n_angles || N < 1 || N > n)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= M <= n_angles and 1 <= N <= n");
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_idx;
    std::vector<double> vals;
    try {
        BSG_CHECK(generate_parallel_beam_csr(n, n_angles, n_bins, (cudaStream_t)stream, row_ptr,
                                             col_idx, vals));
    } catch (const std::bad_alloc &) {
        return fail(BSGDTV_ERR_OOM, "host allocation while generating A");
    }
    // blocks of whole angles and whole image rows
    return bsgdtv_create_csr_ex(out, (int64_t)n_angles * n_bins, (int64_t)n * n, n, n, row_ptr.data(),
                                col_idx.data(), vals.data(), M, N, n_bins, n, nullptr, nullptr,
                                format, stream);
}

void bsgdtv_destroy(bsgdtv_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (cudaEvent_t ev : h->tevents) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->tmark)
        if (ev) cudaEventDestroy(ev);
    for (void *p : h->allocs) cudaFree(p);
    if (h->check_host) cudaFreeHost(h->check_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

int bsgdtv_get_partition(bsgdtv_t h, int64_t *row_bounds, int64_t *col_bounds) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (row_bounds) std::memcpy(row_bounds, h->host.row_bounds.data(), (h->host.M + 1) * sizeof(int64_t));
    if (col_bounds) std::memcpy(col_bounds, h->host.col_bounds.data(), (h->host.N + 1) * sizeof(int64_t));
    return BSGDTV_OK;
}

int bsgdtv_get_info(bsgdtv_t h, int64_t *nnz, int64_t *segments, int64_t *work_items,
                    int64_t *min_bytes_per_pass) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (nnz) *nnz = h->host.nnz;
    if (segments) *segments = h->seg_count;
    if (work_items) *work_items = h->dl.n_items;
    if (min_bytes_per_pass)
        *min_bytes_per_pass = (int64_t)bytes_per_entry(h->host.fmt) * h->host.nnz +
                              4 * (2 * h->dl.rows + 2 * h->dl.cols);
    return BSGDTV_OK;
}

int bsgdtv_estimate_umax(bsgdtv_t h, int max_iters, double rel_tol, double *u_max, int *iters) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (max_iters < 1 || !(rel_tol >= 0.0)) return fail(BSGDTV_ERR_INVALID_ARG, "bad max_iters / rel_tol");
    BSG_CHECK(set_device(h));
    BSG_CHECK(ensure_fp64(h));
    cudaStream_t s = h->stream;
    const int64_t c = h->dl.cols, R = h->dl.rows;
    // v = 1 / ||1||
    BSG_CUDA(launch_fill64(h->v64, 1.0 / std::sqrt((double)c), c, s));
    BSG_CUDA(launch_fill64(h->w64, 0.0, R, s));
    double u = 0.0, u_new = 0.0;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        // w = A v
        BSG_CUDA(launch_products64(h->dl, h->v64, h->w64, h->z64, h->gp64, s));
        BSG_CUDA(launch_reduce_update64(h->dl, h->z64, h->gp64, nullptr, h->w64, nullptr, h->g64,
                                        0.0, s));
        // g = 2 A^T w  (the product kernel carries the block gradient's factor 2)
        BSG_CUDA(launch_products64(h->dl, h->v64, h->w64, h->z64, h->gp64, s));
        BSG_CUDA(launch_reduce_update64(h->dl, h->z64, h->gp64, nullptr, h->w64, nullptr, h->g64,
                                        0.0, s));
        BSG_CUDA(launch_dot(h->v64, h->g64, c, h->partials, h->scal + 0, s));
        BSG_CUDA(launch_dot(h->g64, nullptr, c, h->partials, h->scal + 1, s));
        double sc[2];
        BSG_CUDA(cudaMemcpyAsync(sc, h->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BSG_CUDA(cudaStreamSynchronize(s));
        u_new = 0.5 * sc[0];   // v . (A^T A v), ||v|| = 1
        if (sc[1] == 0.0) {
            u = 0.0;
            break;
        }
        BSG_CUDA(launch_scale64(h->g64, h->scal + 1, h->v64, c, s));
        if (it > 1 && std::fabs(u_new - u) <= rel_tol * std::fabs(u_new)) {
            u = u_new;
            break;
        }
        u = u_new;
    }
    if (it > max_iters) it = max_iters;
    BSG_CUDA(cudaStreamSynchronize(s));
    h->u_max = u;
    if (u_max) *u_max = u;
    if (iters) *iters = it;
    return BSGDTV_OK;
}

// The address at which the GPU reads or writes a caller's buffer directly:
// device memory as given, page-locked (pinned or registered) host memory
// through its device address; null for pageable host memory, which goes
// through a copy.
static float *device_view(const float *p, int on_device) {
    if (on_device) return const_cast<float *>(p);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? static_cast<float *>(a.devicePointer) : nullptr;
}

// y into the handle and the initial state (x^0 = 0, r^{-1} = y, max |y| into
// rmax[0] and the check word) on the handle's stream: one kernel reading y
// where it lies when the GPU can, else a copy first.
static int enqueue_init(bsgdtv_ctx *h, const float *y, int y_on_device) {
    cudaStream_t s = h->stream;
    const int64_t R = h->dl.rows, c = h->dl.cols;
    const float *src = device_view(y, y_on_device);
    if (!src) {
        BSG_CUDA(cudaMemcpyAsync(h->y, y, R * sizeof(float), cudaMemcpyHostToDevice, s));
        src = h->y;
    }
    BSG_CUDA(launch_init_from(src, h->y, h->r[0], h->x, R, c, h->rmax, h->check_dev, h->init_part, s));
    return BSGDTV_OK;
}

int bsgdtv_set_data(bsgdtv_t h, const float *y, int y_on_device, double lambda, double mu) {
    BSG_TRACE();
    if (!h || !y) return fail(BSGDTV_ERR_INVALID_ARG, "null handle or y");
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || !std::isfinite(mu))
        return fail(BSGDTV_ERR_INVALID_ARG, "lambda must be finite and >= 0, mu finite");
    BSG_CHECK(set_device(h));
    cudaStream_t s = h->stream;
    h->has_data = false;   // y is overwritten from here on: a failure leaves no data
    // one launch (after a copy when y is pageable host memory) stores y and
    // sets r^{-1} = y - A x^0 = y, x^0 = 0 and the check word max |y| (Inf or
    // NaN exactly when y is not finite); the synchronisation returns after
    // y has been read, so a host y may be reused at once, pageable or
    // pinned.  The last block products are A x^0 = 0 (cleared when the
    // stochastic iteration first needs them).
    BSG_CHECK(enqueue_init(h, y, y_on_device));
    BSG_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(*h->check_host)) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in y");
    h->cur = 0;
    h->z_stale = true;
    if (mu <= 0.0) {
        if (h->u_max <= 0.0) {
            double u;
            BSG_CHECK(bsgdtv_estimate_umax(h, 5000, 1e-12, &u, nullptr));
        }
        if (h->u_max <= 0.0) return fail(BSGDTV_ERR_INVALID_ARG, "A is zero: u_max = 0");
        mu = 0.9 / (2.0 * h->u_max);
    }
    if (h->mu != mu || h->lambda != lambda) drop_graphs(h);
    h->lambda = lambda;
    h->mu = mu;
    h->epoch = 0;
    h->has_data = true;
    return BSGDTV_OK;
}

int bsgdtv_get_params(bsgdtv_t h, double *mu, double *lambda, double *u_max) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (mu) *mu = h->mu;
    if (lambda) *lambda = h->lambda;
    if (u_max) *u_max = h->u_max;
    return BSGDTV_OK;
}

int bsgdtv_run(bsgdtv_t h, int epochs, int fgp_iters) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "bsgdtv_run before bsgdtv_set_data");
    if (epochs < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epochs / fgp_iters");
    if (epochs == 0) return BSGDTV_OK;
    BSG_CHECK(set_device(h));
    if (!h->gexec[0] || h->graph_fgp_iters != fgp_iters || h->graph_mu != h->mu ||
        h->graph_lambda != h->lambda)
        BSG_CHECK(build_graphs(h, fgp_iters));
    for (int e = 0; e < epochs; ++e) {
        BSG_CUDA(cudaGraphLaunch(h->gexec[h->cur], h->stream));
        add_launches(h->graph_kernels);
        h->cur ^= 1;
        h->z_stale = false;   // a full epoch computes every block product
        h->epoch++;
    }
    return BSGDTV_OK;
}

int bsgdtv_run_timed(bsgdtv_t h, int epochs, int fgp_iters, double *products_ms,
                     double *epoch_ms) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "bsgdtv_run_timed before bsgdtv_set_data");
    if (epochs < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epochs / fgp_iters");
    BSG_CHECK(set_device(h));
    if (!h->gexec[0] || h->graph_fgp_iters != fgp_iters || h->graph_mu != h->mu ||
        h->graph_lambda != h->lambda)
        BSG_CHECK(build_graphs(h, fgp_iters));
    if (!h->texec[0]) BSG_CHECK(build_timed_graphs(h, fgp_iters));
    const size_t need = (size_t)3 * epochs;
    while (h->tevents.size() < need) {
        cudaEvent_t ev;
        BSG_CUDA(cudaEventCreate(&ev));
        h->tevents.push_back(ev);
    }
    for (int e = 0; e < epochs; ++e) {
        cudaGraphExec_t ex = h->texec[h->cur];
        for (int k = 0; k < 3; ++k)
            BSG_CUDA(cudaGraphExecEventRecordNodeSetEvent(ex, h->tnode[h->cur][k], h->tevents[3 * e + k]));
        BSG_CUDA(cudaGraphLaunch(ex, h->stream));
        add_launches(h->graph_kernels);
        h->cur ^= 1;
        h->z_stale = false;   // a full epoch computes every block product
        h->epoch++;
    }
    BSG_CUDA(cudaStreamSynchronize(h->stream));
    double pk = 0.0, ep = 0.0;
    for (int e = 0; e < epochs; ++e) {
        float a = 0.f, b = 0.f;
        BSG_CUDA(cudaEventElapsedTime(&a, h->tevents[3 * e], h->tevents[3 * e + 1]));
        BSG_CUDA(cudaEventElapsedTime(&b, h->tevents[3 * e], h->tevents[3 * e + 2]));
        pk += a;
        ep += b;
    }
    if (products_ms) *products_ms = pk;
    if (epoch_ms) *epoch_ms = ep;
    return BSGDTV_OK;
}

}  // extern "C"

namespace {

// The stochastic iterations; with `marks`, marks[0] is recorded once the
// work-item lists are on the device (right before the first iteration's
// kernels) and marks[1] after the last iteration's, and *prep_ms receives the
// host time spent building and uploading the lists.
int run_subsets_impl(bsgdtv_t h, int iters, int fgp_iters, const uint8_t *row_sel,
                     const uint8_t *col_sel, cudaEvent_t *marks, double *prep_ms) {
    const auto t_prep = std::chrono::steady_clock::now();
    if (!h || !row_sel || !col_sel) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "bsgdtv_run_subsets before bsgdtv_set_data");
    if (iters < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative iters / fgp_iters");
    if (iters == 0) return BSGDTV_OK;
    const HostLayout &L = h->host;
    const int M = L.M, N = L.N;
    for (int k = 0; k < iters; ++k) {
        int ni = 0, nj = 0;
        for (int i = 0; i < M; ++i) ni += row_sel[(size_t)k * M + i] != 0;
        for (int j = 0; j < N; ++j) nj += col_sel[(size_t)k * N + j] != 0;
        if (ni == 0 || nj == 0)
            return fail(BSGDTV_ERR_INVALID_ARG, "every iteration must draw at least one row and one column block");
    }
    BSG_CHECK(set_device(h));
    cudaStream_t s = h->stream;
    if (!h->rb_dev) {
        BSG_CHECK(upload(h, &h->rb_dev, L.row_bounds));
        BSG_CHECK(upload(h, &h->cb_dev, L.col_bounds));
    }
    // per iteration: the work items of the drawn pairs (launch order kept), then
    // the masks.  A draw leaves fewer items than the persistent CTAs when the
    // fractions are small, so with FP32 weights and 32-bit indices each item is
    // split into `shares` ranges of its slabs (the count that minimises
    // ceil(items * shares / CTAs) / shares, i.e. the item-times of the pass),
    // which add their g tiles into a zeroed g_part.
    const bool split = h->dl.fmt == BSGDTV_FMT_F32_I32;
    const int ctas = 2 * std::max(h->dl.n_sms, 1);
    const int n_items = (int)L.items.size();
    std::vector<int> drawn(iters, 0), shares(iters, 1);
    int max_list = 1;
    for (int k = 0; k < iters; ++k) {
        const uint8_t *si = row_sel + (size_t)k * M, *sj = col_sel + (size_t)k * N;
        for (const WorkItem &it : L.items)
            drawn[k] += si[L.group_block[it.group]] && sj[L.tiles[it.tile].band];
        if (split) {
            double best = 1e300;
            for (int sh = 1; sh <= 8; ++sh) {
                const double t = (double)((drawn[k] * sh + ctas - 1) / ctas) / sh;
                if (t < best - 1e-12) {
                    best = t;
                    shares[k] = sh;
                }
            }
        }
        max_list = std::max(max_list, drawn[k] * shares[k]);
    }
    const size_t item_bytes = (size_t)std::max(max_list, n_items) * sizeof(WorkItem);
    const size_t stride = (item_bytes + (size_t)M + N + 255) / 256 * 256;
    std::vector<unsigned char> host(stride * iters, 0);
    std::vector<int> count(iters, 0);
    for (int k = 0; k < iters; ++k) {
        unsigned char *base = host.data() + stride * k;
        WorkItem *list = reinterpret_cast<WorkItem *>(base);
        const uint8_t *si = row_sel + (size_t)k * M, *sj = col_sel + (size_t)k * N;
        for (const WorkItem &it : L.items) {
            if (!si[L.group_block[it.group]] || !sj[L.tiles[it.tile].band]) continue;
            if (!split) {
                list[count[k]++] = it;
                continue;
            }
            const int ns = it.slab_end - it.slab_begin;   // an empty item adds nothing
            const int parts = std::min(shares[k], ns);
            for (int q = 0; q < parts; ++q) {
                WorkItem w = it;
                w.slab_begin = it.slab_begin + (int)((int64_t)ns * q / parts);
                w.slab_end = it.slab_begin + (int)((int64_t)ns * (q + 1) / parts);
                list[count[k]++] = w;
            }
        }
        for (int i = 0; i < M; ++i) base[item_bytes + i] = si[i] ? 1 : 0;
        for (int j = 0; j < N; ++j) base[item_bytes + M + j] = sj[j] ? 1 : 0;
    }
    if (host.size() > h->sub_bytes) {
        BSG_CUDA(cudaStreamSynchronize(s));   // the previous buffer may still be read
        unsigned char *p = nullptr;
        BSG_CHECK(dalloc(h, &p, host.size()));
        h->sub_buf = p;
        h->sub_bytes = host.size();
    }
    unsigned char *dev = static_cast<unsigned char *>(h->sub_buf);
    BSG_CUDA(cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    if (h->z_stale) {   // undrawn pairs start from the block products of x^0 = 0
        BSG_CUDA(cudaMemsetAsync(h->z_part, 0, (size_t)h->dl.n_slabs * kSlab * sizeof(float), s));
        h->z_stale = false;
    }
    BSG_CHECK(ensure_mom(h, std::max(fgp_iters, 1)));
    const bool prox = h->lambda > 0.0 && fgp_iters > 0;
    // split items add into g_part: zero it once; each reduction then zeroes
    // the values it consumes.  Consecutive kernels use programmatic
    // dependent launch (each waits for its predecessor before reading).
    if (split)
        BSG_CUDA(cudaMemsetAsync(h->g_part, 0, (size_t)h->dl.n_groups * h->dl.cols * sizeof(int32_t), s));
    if (marks) {
        BSG_CUDA(cudaEventRecord(marks[0], s));
        if (prep_ms)
            *prep_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_prep).count();
    }
    for (int k = 0; k < iters; ++k) {
        const int par = h->cur;
        const bool pdl = k > 0;   // the first follows copies, not a kernel
        unsigned char *base = dev + stride * k;
        DevLayout ds = h->dl;
        ds.items = reinterpret_cast<const WorkItem *>(base);
        ds.n_items = count[k];
        int32_t *gp = reinterpret_cast<int32_t *>(h->g_part);
        if (split)
            BSG_CUDA(launch_products32_add(ds, h->x, h->r[par], h->rmax + par, h->rmax + (1 - par),
                                           h->z_part, gp, s, pdl));
        else
            BSG_CUDA(launch_products32(ds, h->x, h->r[par], h->rmax + par, h->rmax + (1 - par),
                                       h->z_part, gp, s, pdl));
        float *xdst = prox ? h->xhat : h->x;
        BSG_CUDA(launch_reduce_subset32(h->dl, h->z_part, gp, h->rmax + par, h->y, h->r[par],
                                        h->r[1 - par], h->rmax + (1 - par), h->x, xdst, (float)h->mu,
                                        h->rb_dev, h->cb_dev, base + item_bytes, base + item_bytes + M,
                                        split, s, true));
        if (prox) {
            const FgpScratch sc = fgp_scratch_planes(h->fgp, h->dl.cols);
            BSG_CUDA(launch_fgp(h->xhat, h->x, h->dl.img_h, h->dl.img_w, (float)(h->mu * h->lambda),
                                fgp_iters, h->mom, sc, s, true,
                                fgp_chunk_for(h->dl.img_h, h->dl.img_w, fgp_iters, h->dl.n_sms)));
        }
        h->cur ^= 1;
        h->epoch++;
    }
    if (marks) BSG_CUDA(cudaEventRecord(marks[1], s));
    // the host copy of the lists dies here: wait for the upload
    BSG_CUDA(cudaStreamSynchronize(s));
    return BSGDTV_OK;
}

}  // namespace

extern "C" {

int bsgdtv_run_subsets(bsgdtv_t h, int iters, int fgp_iters, const uint8_t *row_sel,
                       const uint8_t *col_sel) {
    BSG_TRACE();
    return run_subsets_impl(h, iters, fgp_iters, row_sel, col_sel, nullptr, nullptr);
}

int bsgdtv_run_subsets_timed(bsgdtv_t h, int iters, int fgp_iters, const uint8_t *row_sel,
                             const uint8_t *col_sel, double *device_ms, double *prep_ms) {
    BSG_TRACE();
    if (!device_ms) return fail(BSGDTV_ERR_INVALID_ARG, "device_ms is null");
    if (h) BSG_CHECK(set_device(h));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    BSG_CUDA(cudaEventCreate(&ev[0]));
    cudaError_t e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(BSGDTV_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    double prep = 0.0;
    int rc = run_subsets_impl(h, iters, fgp_iters, row_sel, col_sel, iters > 0 ? ev : nullptr, &prep);
    float ms = 0.f;
    if (rc == BSGDTV_OK && iters > 0) {
        e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) rc = fail(BSGDTV_ERR_CUDA, std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e));
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc == BSGDTV_OK) {
        *device_ms = ms;
        if (prep_ms) *prep_ms = prep;
    }
    return rc;
}

// Whether the GPU may write page-locked host memory at p through its device
// address (memory registered read-only may not be written by the device),
// asked through the driver's entry point; false when that cannot be asked.
static bool device_writable(const void *p) {
    using Fn = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
    static const Fn fn = []() -> Fn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<Fn>(f);
    }();
    if (!fn) return false;
    unsigned int flags = 0;
    if (fn(&flags, CU_POINTER_ATTRIBUTE_ACCESS_FLAGS, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
    return flags == CU_POINTER_ATTRIBUTE_ACCESS_FLAG_READWRITE;
}

// x into a caller's buffer on the handle's stream: a copy on the device, or a
// kernel writing page-locked host memory through its device address, or a
// copy to pageable host memory.
static int enqueue_x_out(bsgdtv_ctx *h, float *out, int out_on_device) {
    const int64_t c = h->dl.cols;
    if (out_on_device) {
        BSG_CUDA(cudaMemcpyAsync(out, h->x, c * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
        return BSGDTV_OK;
    }
    float *dst = device_view(out, 0);
    if (dst && device_writable(out)) BSG_CUDA(launch_copy_out(h->x, dst, c, h->stream));
    else BSG_CUDA(cudaMemcpyAsync(out, h->x, c * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return BSGDTV_OK;
}

int bsgdtv_get_x(bsgdtv_t h, float *out, int out_on_device, int64_t n) {
    BSG_TRACE();
    if (!h || !out) return fail(BSGDTV_ERR_INVALID_ARG, "null handle or out");
    if (n < h->dl.cols) return fail(BSGDTV_ERR_INVALID_ARG, "out holds fewer than cols floats");
    BSG_CHECK(set_device(h));
    BSG_CHECK(enqueue_x_out(h, out, out_on_device));
    if (!out_on_device) BSG_CUDA(cudaStreamSynchronize(h->stream));
    return BSGDTV_OK;
}

int bsgdtv_reconstruct(bsgdtv_t h, const float *y, int y_on_device, double lambda, double mu,
                       int epochs, int fgp_iters, float *x_out, int x_on_device, int64_t n_x) {
    BSG_TRACE();
    if (!h || !y || !x_out) return fail(BSGDTV_ERR_INVALID_ARG, "null handle, y or x_out");
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || !std::isfinite(mu))
        return fail(BSGDTV_ERR_INVALID_ARG, "lambda must be finite and >= 0, mu finite");
    if (epochs < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epochs / fgp_iters");
    if (n_x < h->dl.cols) return fail(BSGDTV_ERR_INVALID_ARG, "x_out holds fewer than cols floats");
    BSG_CHECK(set_device(h));
    if (mu <= 0.0) {
        if (h->u_max <= 0.0) {
            double u;
            BSG_CHECK(bsgdtv_estimate_umax(h, 5000, 1e-12, &u, nullptr));
        }
        if (h->u_max <= 0.0) return fail(BSGDTV_ERR_INVALID_ARG, "A is zero: u_max = 0");
        mu = 0.9 / (2.0 * h->u_max);
    }
    if (h->mu != mu || h->lambda != lambda) drop_graphs(h);
    h->lambda = lambda;
    h->mu = mu;
    if (epochs > 0 && (!h->gexec[0] || h->graph_fgp_iters != fgp_iters || h->graph_mu != h->mu ||
                       h->graph_lambda != h->lambda))
        BSG_CHECK(build_graphs(h, fgp_iters));
    cudaStream_t s = h->stream;
    h->has_data = false;
    // set_data's initialisation (max |y| into the check word), the epochs,
    // x out; the check word is read after the one synchronisation
    BSG_CHECK(enqueue_init(h, y, y_on_device));
    h->cur = 0;
    h->z_stale = true;
    h->epoch = 0;
    for (int e = 0; e < epochs; ++e) {
        BSG_CUDA(cudaGraphLaunch(h->gexec[h->cur], s));
        add_launches(h->graph_kernels);
        h->cur ^= 1;
        h->z_stale = false;
        h->epoch++;
    }
    BSG_CHECK(enqueue_x_out(h, x_out, x_on_device));
    BSG_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(*h->check_host)) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in y");
    h->has_data = true;
    return BSGDTV_OK;
}

int bsgdtv_get_state(bsgdtv_t h, float *x, float *r, int64_t *epoch, int on_device) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "no data set");
    BSG_CHECK(set_device(h));
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x) BSG_CUDA(cudaMemcpyAsync(x, h->x, h->dl.cols * sizeof(float), k, h->stream));
    if (r) BSG_CUDA(cudaMemcpyAsync(r, h->r[h->cur], h->dl.rows * sizeof(float), k, h->stream));
    if (epoch) *epoch = h->epoch;
    if (!on_device) BSG_CUDA(cudaStreamSynchronize(h->stream));
    return BSGDTV_OK;
}

int bsgdtv_set_state(bsgdtv_t h, const float *x, const float *r, int64_t epoch, int on_device) {
    BSG_TRACE();
    if (!h || !x || !r) return fail(BSGDTV_ERR_INVALID_ARG, "null handle, x or r");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "set_state before set_data");
    if (epoch < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epoch");
    BSG_CHECK(set_device(h));
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    BSG_CUDA(cudaMemcpyAsync(h->x, x, h->dl.cols * sizeof(float), k, h->stream));
    BSG_CUDA(cudaMemcpyAsync(h->r[h->cur], r, h->dl.rows * sizeof(float), k, h->stream));
    BSG_CUDA(cudaMemsetAsync(h->rmax + h->cur, 0, sizeof(float), h->stream));
    BSG_CUDA(launch_absmax(h->r[h->cur], h->dl.rows, h->rmax + h->cur, h->stream));
    if (!on_device) BSG_CUDA(cudaStreamSynchronize(h->stream));
    h->epoch = epoch;
    return BSGDTV_OK;
}

int bsgdtv_run_until(bsgdtv_t h, int max_epochs, int fgp_iters, int check_every, double rel_tol,
                     int *epochs_run, double *objective) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (max_epochs < 0 || fgp_iters < 0 || check_every < 1 || !(rel_tol >= 0.0) ||
        !std::isfinite(rel_tol))
        return fail(BSGDTV_ERR_INVALID_ARG, "need max_epochs, fgp_iters >= 0, check_every >= 1, "
                                            "finite rel_tol >= 0");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "bsgdtv_run_until before bsgdtv_set_data");
    auto F = [&](double *f) -> int {
        double data = 0.0, tv = 0.0;
        BSG_CHECK(bsgdtv_objective(h, &data, &tv));
        *f = data + h->lambda * tv;
        return BSGDTV_OK;
    };
    double f_before = 0.0, f_after = 0.0;
    BSG_CHECK(F(&f_before));
    f_after = f_before;
    int done = 0;
    while (done < max_epochs) {
        const int step = std::min(check_every, max_epochs - done);
        BSG_CHECK(bsgdtv_run(h, step, fgp_iters));
        done += step;
        BSG_CHECK(F(&f_after));
        if (std::fabs(f_before - f_after) <= rel_tol * std::fabs(f_before)) break;
        f_before = f_after;
    }
    if (epochs_run) *epochs_run = done;
    if (objective) *objective = f_after;
    return BSGDTV_OK;
}

int bsgdtv_objective(bsgdtv_t h, double *data_term, double *tv) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "no data set");
    BSG_CHECK(set_device(h));
    BSG_CHECK(ensure_fp64(h));
    cudaStream_t s = h->stream;
    const int64_t c = h->dl.cols, R = h->dl.rows;
    BSG_CUDA(launch_f32_to_f64(h->x, h->x64, c, s));
    BSG_CUDA(launch_f32_to_f64(h->y, h->y64, R, s));
    BSG_CUDA(launch_fill64(h->w64, 0.0, R, s));
    BSG_CUDA(launch_products64(h->dl, h->x64, h->w64, h->z64, h->gp64, s));
    // w = y - A x (FP64)
    BSG_CUDA(launch_reduce_update64(h->dl, h->z64, h->gp64, h->y64, h->w64, nullptr, h->g64, 0.0, s));
    BSG_CUDA(launch_dot(h->w64, nullptr, R, h->partials, h->scal + 2, s));
    BSG_CUDA(launch_tv64(h->x, h->dl.img_h, h->dl.img_w, h->partials, h->scal + 3, s));
    double sc[2];
    BSG_CUDA(cudaMemcpyAsync(sc, h->scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    BSG_CUDA(cudaStreamSynchronize(s));
    if (data_term) *data_term = sc[0];
    if (tv) *tv = sc[1];
    return BSGDTV_OK;
}

int bsgdtv_block_products(bsgdtv_t h, const float *x, const float *r, float *z_blocks,
                          float *g_blocks) {
    BSG_TRACE();
    if (!h || !x || !r || !z_blocks || !g_blocks)
        return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    BSG_CHECK(set_device(h));
    cudaStream_t s = h->stream;
    BSG_CUDA(cudaMemsetAsync(h->rmax + 2, 0, sizeof(float), s));
    BSG_CUDA(launch_absmax(r, h->dl.rows, h->rmax + 2, s));
    BSG_CUDA(launch_products32(h->dl, x, r, h->rmax + 2, nullptr, h->z_part,
                               reinterpret_cast<int32_t *>(h->g_part), s));
    BSG_CUDA(launch_block_sums(h->dl, h->z_part, reinterpret_cast<const int32_t *>(h->g_part),
                               h->rmax + 2, z_blocks, g_blocks, s));
    BSG_CUDA(cudaStreamSynchronize(s));
    return BSGDTV_OK;
}

int bsgdtv_tv_prox(const float *b, float *x, int img_h, int img_w, double tau, int iters,
                   void *stream) {
    BSG_TRACE();
    if (!b || !x || img_h < 1 || img_w < 1 || iters < 0 || !std::isfinite(tau))
        return fail(BSGDTV_ERR_INVALID_ARG, "bad argument");
    if (b == x) return fail(BSGDTV_ERR_INVALID_ARG, "b and x may not alias");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)img_h * img_w;
    if (tau <= 0.0 || iters == 0) {
        BSG_CUDA(cudaMemcpyAsync(x, b, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        BSG_CUDA(cudaStreamSynchronize(s));
        return BSGDTV_OK;
    }
    std::vector<float> m;
    fgp_momentum_host(iters, m);
    float *scratch = nullptr;
    const size_t bytes = (kFgpFieldPlanes * n + m.size()) * sizeof(float);
    BSG_CUDA(cudaMallocAsync((void **)&scratch, bytes, s));
    float *mom = scratch + kFgpFieldPlanes * n;
    cudaError_t e = cudaMemcpyAsync(mom, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const FgpScratch sc = fgp_scratch_planes(scratch, n);
        e = launch_fgp(b, x, img_h, img_w, (float)tau, iters, mom, sc, s);
    }
    cudaError_t e2 = cudaStreamSynchronize(s);   // keeps m alive until the copy is done
    cudaFreeAsync(scratch, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("tv_prox: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("tv_prox: ") + cudaGetErrorString(e2));
    if (e3 != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("tv_prox: ") + cudaGetErrorString(e3));
    return BSGDTV_OK;
}

}  // extern "C"
