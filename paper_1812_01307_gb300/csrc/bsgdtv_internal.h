// Internal declarations of the BSGD-TV library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/bsgdtv.h"
#include "layout.h"

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

// A named NVTX range over a library call, visible to CUDA tools that record
// NVTX (ncu --nvtx, Nsight Systems); a few nanoseconds when none is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define BSG_TRACE() ::bsgdtv::TraceRange bsg_trace_range_(__func__)

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
// The same for FMT_F32_I32 work items that may cover part of a (group, tile)
// pair's slabs: each adds its g tile into g_part (zeroed beforehand) with
// integer atomics, so the sums stay exact and independent of order.
cudaError_t launch_products32_add(const DevLayout &d, const float *x, const float *r,
                                  const float *rmax_in, float *rmax_clear, float *z_part,
                                  int32_t *g_part, cudaStream_t s, bool pdl = false);


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
// bounds; rows / pixels outside keep r_in / x.  clear_g: the g_part values
// read are zeroed for a following launch_products32_add.
cudaError_t launch_reduce_subset32(const DevLayout &d, const float *z_part, int32_t *g_part,
                                   const float *rmax_in, const float *y, const float *r_in,
                                   float *r_out, float *rmax_out, const float *x, float *x_out,
                                   float mu, const int64_t *rb, const int64_t *cb,
                                   const uint8_t *sel_i, const uint8_t *sel_j, bool clear_g,
                                   cudaStream_t s, bool pdl = false);
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
// Start of an iteration: r0 = y [rows], x = 0 [cols] and *rmax = max |y|,
// which is Inf or NaN exactly when y holds a NaN or +-Inf (a memset and one
// launch).
// One launch: y_dst = y (y may be page-locked host memory through its device
// address), r0 = y, x = 0, max |y| into *rmax and *check; part: kInitBlocks + 1
// ints, the last one 0 between launches.
constexpr int kInitBlocks = 512;
cudaError_t launch_init_from(const float *y, float *y_dst, float *r0, float *x, int64_t rows,
                             int64_t cols, float *rmax, float *check, int *part, cudaStream_t s);
// dst = src (dst may be page-locked host memory through its device address).
cudaError_t launch_copy_out(const float *src, float *dst, int64_t n, cudaStream_t s);
constexpr int kDotPartials = 1024;

// fgp.cu: K FGP iterations on an h x w image.  `mom` holds the K momentum
// coefficients (iteration k uses mom[k-1]).  The dual state passes between
// the launches of a tiled FGP through two sets of h*w fields (p, q, p_prev,
// q_prev), read from one and written to the other by turns.
struct FgpFields {
    float *p, *q, *pp, *qp;
};
struct FgpScratch {
    FgpFields set[2];
};
constexpr int kFgpFieldPlanes = 8;   // h*w floats of scratch per image
// The two sets carved out of kFgpFieldPlanes consecutive planes of `plane`
// floats starting at base (+ offset within each plane).
inline FgpScratch fgp_scratch_planes(float *base, int64_t plane, int64_t offset = 0) {
    FgpScratch sc;
    for (int k = 0; k < 2; ++k) {
        float *b = base + offset + (int64_t)4 * k * plane;
        sc.set[k] = FgpFields{b, b + plane, b + 2 * plane, b + 3 * plane};
    }
    return sc;
}
// Iterations per launch for an h x w image on n_sms SMs (a cost model of
// halo recomputation, waves and launches; every choice gives the same iterates).
int fgp_chunk_for(int h, int w, int iters, int n_sms);
int fgp_plan_launches(int h, int w, int iters, int max_chunk = 8);
cudaError_t launch_fgp(const float *b, float *x, int h, int w, float tau, int iters,
                       const float *mom, FgpScratch sc, cudaStream_t s, bool pdl = false,
                       int max_chunk = 8);
void fgp_momentum_host(int iters, std::vector<float> &mom);

// batch.cu: keep the prox stage in a batch's epochs even when every slot has
// lambda = 0 (slots with lambda = 0 pass through the FGP launch unchanged), so
// slots that come and go do not force the epoch graphs to be captured again.
void batch_keep_prox(bsgdtv_batch_t h, bool on);

// ------------------------------------------------ served mode of a batch
// A batch in served mode runs, at the start of every epoch, a device-side
// slot scheduler: it reads per-slot mailboxes in host-mapped memory that the
// host fills at any time (an admission: y in the slot's pinned staging row,
// tau = mu*lambda, an epoch budget; or a cancellation), resets admitted slots
// (y, r^{-1} = y, x = 0), counts every live slot's epochs, and when a slot's
// budget is spent writes its x to the slot's pinned result row and publishes
// a completion record.  Requests therefore join and leave at epoch
// boundaries while the host keeps the group's stream fed with epochs.
// Host-written mailbox of one slot (host-mapped).  The host fills epochs and
// tau (and y) first, then publishes by storing a new seq.
struct ServeSlot {
    int seq;      // bumped by the host for every admission into this slot
    int epochs;   // epoch budget of the admitted request
    float tau;    // mu * lambda of the admitted request
    int cancel;   // == seq: end the request at the next epoch boundary
};
// Device-written records of one slot (host-mapped): seq of the request whose
// x is in the slot's result row and the epochs it ran; seq of the last
// admission the device picked up and the index of the epoch that picked it
// up (the group's epochs count from 0), from which the host knows exactly
// how many more epochs the request needs.
struct ServeDone {
    int seq;
    int epochs_run;
    int picked_seq;
    int picked_epoch;
};
// Control block (host-mapped).  An armed epoch (arm_seq changed) whose slots
// are all idle waits on the device, polling the mailboxes, up to wait_ns for
// an admission; it then stores status (0: work arrived, 1: the wait ran out)
// and status_seq = arm_seq.
struct ServeCtrl {
    long long wait_ns;
    int arm_seq;
    int status_seq;
    int status;
    int pad_[3];
};
constexpr long long kServeMaxWaitNs = 1000000000ll;   // longest device-side wait (1 s)
// Host view of a served batch's mapped memory.
struct ServeView {
    ServeSlot *mb;
    ServeDone *done;
    ServeCtrl *ctrl;
    float *ypin;   // [B][rows] staging rows of admitted y
    float *xpin;   // [B][cols] result rows of retired slots
    int64_t rows, cols;
    int B;
};
// Bytes of host-mapped memory a served batch of B slots needs (mailboxes,
// records, control block, staging and result rows).
size_t batch_serve_host_bytes(int B, int64_t rows, int64_t cols);
// Switches a batch (which has data, e.g. all-zero slots) into served mode:
// host_block is mapped pinned memory (cudaHostAlloc with
// cudaHostAllocMapped) of at least batch_serve_host_bytes bytes, owned by
// the caller and kept until the batch is destroyed; allocates the device slot
// state; the epoch graphs gain the scheduler.  Slots start empty.
int batch_serve_enable(bsgdtv_batch_t h, ServeView *view, void *host_block);

// Part k of a packed batch (a batch handle owned by it), or null.
bsgdtv_batch_t packed_part(bsgdtv_packed_t h, int k);
// batch_serve_enable for part k of a packed batch (every part of a packed
// batch is served or none is); its epochs gain one scheduler launch pair
// for all parts.
int packed_serve_enable(bsgdtv_packed_t h, int k, ServeView *view, void *host_block);

// batch.cu: bsgdtv_batch_set_slice, with check = false for a host y the
// caller has already checked for NaN/Inf (no device check, no wait).
int batch_set_slice(bsgdtv_batch_t h, int b, const float *y, int y_on_device, double lambda,
                    bool check);

// batch.cu: the 2-D parallel-beam A of an n x n image (n_angles x n_bins
// rays) as a host CSR with ascending columns, weights from the matrix-free
// projector; BSGDTV_* code.
int generate_parallel_beam_csr(int n, int n_angles, int n_bins, cudaStream_t s,
                               std::vector<int64_t> &row_ptr, std::vector<int32_t> &col_idx,
                               std::vector<double> &vals);

// batch.cu: host check of a CSR image operator (sizes, sorted in-range
// columns, finite weights); BSGDTV_* code.
int validate_image_csr(int64_t rows, int64_t cols, int img_h, int img_w, const int64_t *row_ptr,
                       const int32_t *col_idx, const double *vals);

}  // namespace bsgdtv
