// Batched BSGD-TV: B slices (independent images, e.g. the slices of a
// parallel-beam volume) that share one projection matrix A, each with its own
// projections y_b, TV weight lambda_b, iterate x_b and residual r_b, and one
// step mu (u_max belongs to A, so one step bound serves every slice).
//
// Every slice runs Algorithm 1 exactly as the single-slice path does.  The
// block partition of Sec. 2.1 only distributes work: summed over the blocks,
// the products of one epoch are r = y - A x and g = 2 A^T r_prev, so the
// batch computes them with two passes over A for all slices at once:
//   row pass     (A in CSR)  r_b  = y_b - A x_b                  (residual)
//   column pass  (A in CSC)  x^_b = x_b + mu * 2 A^T r_b^{prev}  (gradient sum and step)
// One warp handles one row (or one pixel) and its lanes the slices, so each
// nonzero of A is read from HBM once per pass and applied to every slice.  x
// and r are stored interleaved ([element][slice], slice stride Bp, B padded)
// so that gathering element k for all slices is one contiguous 128-512 B
// read, mostly served from L2.  There are no atomics and every sum runs in a
// fixed order: results are deterministic.  The TV prox runs on planar images
// (transposed out and back) with one FGP launch per chunk of iterations
// covering every slice, tau_b = mu * lambda_b.
//
// Why not the single-slice fused kernel: its shared-memory x and g tiles
// (64 x 64 pixels) hold only a handful of slices, and smaller tiles multiply
// the per-segment z partials by the number of slices until they outweigh A.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <type_traits>
#include <cstring>
#include <memory>
#include <new>

#include "bsgdtv_internal.h"
#include "fgp_common.cuh"
#include "matrix_free.h"

namespace bsgdtv {
namespace {

constexpr int kBatchFgpChunk = 5;   // default FGP iterations per launch (halo = chunk + 1)
constexpr int kFgpChunkChoices[] = {3, 4, 5, 6, 8};   // what the autotuner tries
constexpr int64_t kFgpFieldBudget = 48ll << 20;       // bytes of FGP fields per slice group
constexpr int kPassWarps = 8;       // warps (rows or pixels) per CTA
constexpr int kPassMinBlocks = 6;   // 48 resident warps per SM (<= 40 registers): the
                                    // gathers are latency-bound, occupancy beats depth

// Packed nonzero of A for the passes: the weight's FP32 bits and the index of
// the gathered element (its slice vector starts at idx * Bp floats).
// Gathered slice vectors are loaded with an L2 evict-last policy so that they
// stay resident while A streams past them (evict-first).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ld_keep(const float *ptr, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ void fma4(float a, const float4 &x, float4 &acc) {
    acc.x = fmaf(a, x.x, acc.x);
    acc.y = fmaf(a, x.y, acc.y);
    acc.z = fmaf(a, x.z, acc.z);
    acc.w = fmaf(a, x.w, acc.w);
}

// One warp per output element k (a row of A in the row pass, a column in the
// column pass).  Each lane owns 4 consecutive slices; LPN lanes cover the 4*LPN
// slices of one chunk (the warp takes the Bp / (4 LPN) chunks in turn), so the
// warp applies G = 32/LPN nonzeros at a time (group g takes the nonzeros j = g,
// g + G, ...).  acc = sum_e a_e v[idx_e][slices]
// in that fixed order, the G group sums are added by a fixed butterfly, then
//   row pass:    out[k] = base[k] - acc       (base = y, v = x)
//   column pass: out[k] = base[k] + mu*2*acc  (base = x, v = r_prev)
// The 32 nonzeros of a round are staged in shared memory once; a partial last
// round is padded with zero weights aimed at element 0.
// The nonzeros of A as the passes read them.  kW = 0: packed 8-byte entries
// (FP32 weight bits, element index); kW = BSGDTV_FMT_F16_I16 /
// BSGDTV_FMT_BF16_I16: 16-bit weights and 32-bit element indices in two
// arrays (6 bytes per nonzero).  Indices do not depend on the slice stride,
// so one operator serves batches of any size.
struct PassOperand {
    const int64_t *ptr;
    const int2 *ent;
    const uint16_t *w16;
    const int32_t *off;
};

template <int kW>
__device__ __forceinline__ int2 load_entry(const PassOperand &A, int64_t e) {
    if constexpr (kW == 0) {
        return __ldcs(A.ent + e);
    } else {
        const unsigned short wb = __ldcs(reinterpret_cast<const unsigned short *>(A.w16) + e);
        const int off = __ldcs(A.off + e);
        float a;
        if constexpr (kW == BSGDTV_FMT_F16_I16)
            a = __half2float(__ushort_as_half(wb));
        else
            a = __uint_as_float((unsigned)wb << 16);   // bfloat16 = high half of an FP32
        return make_int2(__float_as_int(a), off);
    }
}

// One pass launch covers up to kMaxPassParts parts (operators with their own
// vectors, one slice stride Bp for all): CTA blockIdx.x belongs to the last
// part whose cta_begin it has reached.
struct PassPart {
    PassOperand A;
    const float *v, *base;
    float *out;
    int64_t n_out;
    float mu;
    int cta_begin;
};
constexpr int kMaxPassParts = 8;
struct PassLaunch {
    PassPart part[kMaxPassParts];
    int n_parts;
    int Bp;
};

// kOwnStride: the padded slice stride is 4 * LPN (the batch's own lanes per
// nonzero, one chunk), a compile-time constant; else L.Bp (fewer lanes than
// that, several chunks).
// kMulti: the launch has several parts (a packed batch); with one part the
// descriptor's fields are read at fixed offsets of the kernel arguments.
template <int LPN, bool kRowPass, int kW, bool kOwnStride = true, bool kMulti = false>
__global__ void __launch_bounds__(kPassWarps * 32, kPassMinBlocks)
    pass_kernel(const __grid_constant__ PassLaunch L) {
    constexpr int G = 32 / LPN;
    constexpr int NB = (32 / G < 4) ? 32 / G : 4;
    int pi = 0;
    if constexpr (kMulti)
        while (pi + 1 < L.n_parts && (int)blockIdx.x >= L.part[pi + 1].cta_begin) ++pi;
    // the part's fields are used where needed (read from the kernel
    // arguments), not held in registers across the gather loop
    const PassPart &P = L.part[pi];
    const int Bp = (kOwnStride && LPN < 32) ? 4 * LPN : L.Bp;
    __shared__ int2 stage[kPassWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane / LPN, sl = lane % LPN;
    const int64_t k = (int64_t)(kMulti ? (int)blockIdx.x - P.cta_begin : (int)blockIdx.x) * kPassWarps + w;
    if (k >= P.n_out) return;   // warp-uniform
    const uint64_t pol = l2_evict_last_policy();
    const int64_t e0 = P.A.ptr[k], e1 = P.A.ptr[k + 1];
    for (int c0 = 0; c0 < Bp; c0 += 4 * LPN) {
        const float *vl = P.v + c0 + sl * 4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t r0 = e0; r0 < e1; r0 += 32) {
            const int64_t e = r0 + lane;
            int2 t = make_int2(0, 0);
            if (e < e1) t = load_entry<kW>(P.A, e);
            stage[w][lane] = t;
            __syncwarp();
            // NB gathers issued per lane before their FMAs
#pragma unroll
            for (int q0 = 0; q0 < 32 / G; q0 += NB) {
                int2 st[NB];
                float4 xv[NB];
#pragma unroll
                for (int q = 0; q < NB; ++q) st[q] = stage[w][(q0 + q) * G + g];
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    // below 32 lanes per nonzero the batch has Bp <= 128 and
                    // element * Bp < 2^31 (checked at creation)
                    if constexpr (LPN < 32)
                        xv[q] = ld_keep(vl + st[q].y * Bp, pol);
                    else
                        xv[q] = ld_keep(vl + (int64_t)st[q].y * Bp, pol);
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) fma4(__int_as_float(st[q].x), xv[q], acc);
            }
            __syncwarp();
        }
#pragma unroll
        for (int off = LPN; off < 32; off *= 2) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off);
        }
        if (g == 0) {
            const int64_t o = k * Bp + c0 + sl * 4;
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(P.base + o));
            float4 res;
            if (kRowPass) {
                res = make_float4(b.x - acc.x, b.y - acc.y, b.z - acc.z, b.w - acc.w);
            } else {
                const float mu = P.mu;
                res = make_float4(b.x + mu * (2.f * acc.x), b.y + mu * (2.f * acc.y),
                                  b.z + mu * (2.f * acc.z), b.w + mu * (2.f * acc.w));
            }
            *reinterpret_cast<float4 *>(P.out + o) = res;
        }
    }
}

template <bool kRowPass, int kW>
cudaError_t launch_pass_w(int lpn, const PassLaunch &L, int ctas, cudaStream_t s) {
    const dim3 grid((unsigned)ctas), block(kPassWarps * 32);
    const bool own = lpn == 32 || 4 * lpn == L.Bp;
#define BSG_PASS(LP)                                                                   \
    case LP:                                                                           \
        if (L.n_parts > 1)                                                             \
            pass_kernel<LP, kRowPass, kW, true, true><<<grid, block, 0, s>>>(L);       \
        else                                                                           \
            pass_kernel<LP, kRowPass, kW><<<grid, block, 0, s>>>(L);                   \
        break;
#define BSG_PASS_N(LP)                                                   \
    case LP:                                                             \
        pass_kernel<LP, kRowPass, kW, false><<<grid, block, 0, s>>>(L);  \
        break;
    if (own) {
        switch (lpn) {
            BSG_PASS(1)
            BSG_PASS(2)
            BSG_PASS(4)
            BSG_PASS(8)
            BSG_PASS(16)
            BSG_PASS(32)
            default:
                return cudaErrorInvalidValue;
        }
    } else {
        switch (lpn) {   // fewer lanes than the batch's own count (2 .. 16)
            BSG_PASS_N(2)
            BSG_PASS_N(4)
            BSG_PASS_N(8)
            BSG_PASS_N(16)
            default:
                return cudaErrorInvalidValue;
        }
    }
#undef BSG_PASS
#undef BSG_PASS_N
    add_launches(1);
    return cudaGetLastError();
}

// One pass over the parts' operators (all of format fmt, slice stride Bp):
// row pass out = base - A v, column pass out = base + 2 mu A^T v, per part.
template <bool kRowPass>
cudaError_t launch_pass_parts(int fmt, int lpn, const PassPart *parts, int n_parts, int Bp,
                              cudaStream_t s) {
    if (n_parts < 1 || n_parts > kMaxPassParts) return cudaErrorInvalidValue;
    PassLaunch L = {};
    L.n_parts = n_parts;
    L.Bp = Bp;
    int ctas = 0;
    for (int k = 0; k < n_parts; ++k) {
        L.part[k] = parts[k];
        L.part[k].cta_begin = ctas;
        ctas += (int)((parts[k].n_out + kPassWarps - 1) / kPassWarps);
    }
    if (ctas == 0) return cudaSuccess;
    switch (fmt) {
        case BSGDTV_FMT_F32_I32: return launch_pass_w<kRowPass, 0>(lpn, L, ctas, s);
        case BSGDTV_FMT_F16_I16: return launch_pass_w<kRowPass, BSGDTV_FMT_F16_I16>(lpn, L, ctas, s);
        case BSGDTV_FMT_BF16_I16: return launch_pass_w<kRowPass, BSGDTV_FMT_BF16_I16>(lpn, L, ctas, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool kRowPass>
cudaError_t launch_pass(int fmt, int lpn, const PassOperand &A, const float *v, const float *base,
                        float *out, int64_t n_out, int Bp, float mu, cudaStream_t s) {
    const PassPart p = {A, v, base, out, n_out, mu, 0};
    return launch_pass_parts<kRowPass>(fmt, lpn, &p, 1, Bp, s);
}

// Slot reset: slice b of the interleaved Y, X and R becomes (y_b, 0, y_b),
// with y_b planar [n]; y_b null clears the slice (y = x = r = 0).
__global__ void slice_reset_kernel(const float *__restrict__ yb, float *__restrict__ Y,
                                   float *__restrict__ X, float *__restrict__ R, int64_t rows,
                                   int64_t cols, int Bp, int b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows) {
        const float y = yb ? yb[i] : 0.f;
        Y[i * Bp + b] = y;
        R[i * Bp + b] = y;
    }
    if (i < cols) X[i * Bp + b] = 0.f;
}

// Planar copy of slice b of an interleaved [n][Bp] array.
__global__ void slice_gather_kernel(const float *__restrict__ in, float *__restrict__ out, int64_t n,
                                    int Bp, int b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i * Bp + b];
}

// Planar [B][n] <-> interleaved [n][Bp] (only slices b < B are touched), for
// up to kMaxTransParts parts (arrays of different n, one B and Bp): CTA
// column blockIdx.x belongs to the last part whose x_begin it has reached.
struct TransPart {
    const float *in;
    float *out;
    int64_t n;
    int x_begin;
};
constexpr int kMaxTransParts = 8;
struct TransLaunch {
    TransPart part[kMaxTransParts];
    int n_parts;
};

__global__ void transpose_kernel(const __grid_constant__ TransLaunch L, int B, int Bp, int to_planar) {
    __shared__ float t[32][33];
    int pi = 0;
    while (pi + 1 < L.n_parts && (int)blockIdx.x >= L.part[pi + 1].x_begin) ++pi;
    const float *__restrict__ in = L.part[pi].in;
    float *__restrict__ out = L.part[pi].out;
    const int64_t n = L.part[pi].n;
    const int64_t k0 = (int64_t)((int)blockIdx.x - L.part[pi].x_begin) * 32;
    const int b0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8 threads
    for (int yy = ty; yy < 32; yy += 8) {
        if (to_planar) {   // interleaved rows k, slices along x
            const int64_t k = k0 + yy;
            const int b = b0 + tx;
            if (k < n && b < B) t[yy][tx] = in[k * Bp + b];
        } else {           // planar rows b, elements along x
            const int b = b0 + yy;
            const int64_t k = k0 + tx;
            if (k < n && b < B) t[tx][yy] = in[(int64_t)b * n + k];
        }
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        if (to_planar) {
            const int b = b0 + yy;
            const int64_t k = k0 + tx;
            if (k < n && b < B) out[(int64_t)b * n + k] = t[tx][yy];
        } else {
            const int64_t k = k0 + yy;
            const int b = b0 + tx;
            if (k < n && b < B) out[k * Bp + b] = t[yy][tx];
        }
    }
}

cudaError_t launch_transpose_parts(const TransPart *parts, int n_parts, int B, int Bp,
                                   bool to_planar, cudaStream_t s) {
    if (n_parts < 1 || n_parts > kMaxTransParts) return cudaErrorInvalidValue;
    TransLaunch L = {};
    L.n_parts = n_parts;
    int xs = 0;
    for (int k = 0; k < n_parts; ++k) {
        L.part[k] = parts[k];
        L.part[k].x_begin = xs;
        xs += (int)((parts[k].n + 31) / 32);
    }
    const dim3 grid((unsigned)xs, (unsigned)((B + 31) / 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(L, B, Bp, to_planar ? 1 : 0);
    add_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float *in, float *out, int64_t n, int B, int Bp, bool to_planar,
                             cudaStream_t s) {
    const TransPart p = {in, out, n, 0};
    return launch_transpose_parts(&p, 1, B, Bp, to_planar, s);
}

// ------------------------------------------------ served mode: slot scheduler
// Loads and stores of host-mapped memory with system scope.
__device__ __forceinline__ int ld_acquire_sys(const int *p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_sys(const int *p) {
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_sys64(const long long *p) {
    long long v;
    asm volatile("ld.relaxed.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(int *p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device slot state, [4][B] + 1: admitted seq, epochs still to run, live
// flag, epochs run so far; then the count of epochs the group has run.  acts [B + 1]: this epoch's actions (slot | kind << 24),
// their count last.
enum ServeAct { kActAdmit = 1, kActRetire = 2 };
constexpr int kServeThreads = 256;

// The served state of one part (a batch in served mode) as the scheduler
// kernels see it; a launch covers up to kMaxServeParts parts.
struct ServePart {
    const ServeSlot *mb;
    ServeDone *done;
    ServeCtrl *ctrl;
    int *state;      // [4 * B + 1]
    int *acts;       // [B + 1]
    float *tau;      // [B]
    int *arm_seen;
    const float *ypin;
    float *xpin;
    int *unit_cnt;   // [B]
    float *Y, *X, *R;   // R: the r^{k-1} buffer the epoch reads
    int64_t rows, cols;
    int B, Bp;
};
constexpr int kMaxServeParts = 8;
struct ServeLaunch {
    ServePart part[kMaxServeParts];
    int n_parts;
};

// One CTA per part at the start of every served epoch.  (1) An armed epoch
// with no live slot and no posted admission waits, bounded by ctrl->wait_ns,
// for a mailbox to change.  (2) Per slot: a new seq admits (state latched
// from the mailbox); a live slot whose budget is spent or that was cancelled
// retires (tau = 0 from here on); every live slot then counts this epoch.
__global__ void __launch_bounds__(kServeThreads) serve_decide_kernel(const __grid_constant__ ServeLaunch L) {
    const ServePart &P = L.part[blockIdx.x];
    const ServeSlot *mb = P.mb;
    ServeDone *done = P.done;
    ServeCtrl *ctrl = P.ctrl;
    int *state = P.state, *acts = P.acts, *arm_seen = P.arm_seen;
    float *tau = P.tau;
    const int B = P.B;
    int *seq_s = state, *rem = state + B, *live = state + 2 * B, *ran = state + 3 * B;
    const int epoch = state[4 * B];   // index of this epoch in the group's sequence
    __shared__ int n_act;
    if (threadIdx.x == 0) {
        n_act = 0;
        const int arm = ld_relaxed_sys(&ctrl->arm_seq);
        if (arm != *arm_seen) {
            *arm_seen = arm;
            long long wait = ld_relaxed_sys64(&ctrl->wait_ns);
            wait = wait < 0 ? 0 : (wait > kServeMaxWaitNs ? kServeMaxWaitNs : wait);
            const unsigned long long t0 = global_ns();
            int status = 1;
            for (;;) {
                bool work = false;
                for (int b = 0; b < B && !work; ++b)
                    work = live[b] || ld_relaxed_sys(&mb[b].seq) != seq_s[b];
                if (work) {
                    status = 0;
                    break;
                }
                if ((long long)(global_ns() - t0) > wait) break;   // bounded: the wait ran out
                __nanosleep(2000);
            }
            ctrl->status = status;
            __threadfence_system();
            st_release_sys(&ctrl->status_seq, arm);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int seq = ld_acquire_sys(&mb[b].seq);
        int act = 0;
        if (seq != seq_s[b]) {
            seq_s[b] = seq;
            rem[b] = ld_relaxed_sys(&mb[b].epochs);
            tau[b] = __int_as_float(ld_relaxed_sys(reinterpret_cast<const int *>(&mb[b].tau)));
            live[b] = 1;
            ran[b] = 0;
            act = kActAdmit;
            done[b].picked_epoch = epoch;
            __threadfence_system();
            st_release_sys(&done[b].picked_seq, seq);
        } else if (live[b] && (rem[b] <= 0 || ld_relaxed_sys(&mb[b].cancel) == seq)) {
            live[b] = 0;
            tau[b] = 0.f;
            act = kActRetire;
        }
        if (live[b]) {
            rem[b]--;
            ran[b]++;
        }
        if (act) acts[atomicAdd(&n_act, 1)] = b | (act << 24);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        acts[B] = n_act;
        state[4 * B] = epoch + 1;
    }
}

constexpr int kServeUnroll = 8;                               // elements per thread per unit
constexpr int kServeChunk = kServeThreads * kServeUnroll;    // vector elements per work unit

// Applies this epoch's actions of every part, work units (action, chunk of
// the slot's vectors) spread over a fixed grid.  Admit: Y_b = R_b = y (from
// the slot's pinned staging row in host memory; each thread issues all its
// loads before its stores, so a unit has kServeChunk reads in flight), X_b =
// 0.  Retire: the slot's x to its pinned result row, then Y_b = X_b = R_b =
// 0; the last unit of a retiring slot publishes the completion record (after
// every unit's stores are visible to the host).
__global__ void __launch_bounds__(kServeThreads) serve_apply_kernel(const __grid_constant__ ServeLaunch L) {
    for (int pi = 0; pi < L.n_parts; ++pi) {
        const ServePart &P = L.part[pi];
        const int B = P.B, Bp = P.Bp;
        const int n_act = P.acts[B];
        if (n_act == 0) continue;
        const int64_t rows = P.rows, cols = P.cols;
        const float *__restrict__ ypin = P.ypin;
        float *__restrict__ xpin = P.xpin;
        float *__restrict__ Y = P.Y;
        float *__restrict__ X = P.X;
        float *__restrict__ R = P.R;
        const int64_t n = rows > cols ? rows : cols;
        const int chunks = (int)((n + kServeChunk - 1) / kServeChunk);
        for (int64_t w = blockIdx.x; w < (int64_t)n_act * chunks; w += gridDim.x) {
            const int a = P.acts[w / chunks];
            const int b = a & 0xFFFFFF, kind = a >> 24;
            const int64_t i0 = (w % chunks) * (int64_t)kServeChunk + threadIdx.x;
            float v[kServeUnroll];
            if (kind == kActAdmit) {
#pragma unroll
                for (int k = 0; k < kServeUnroll; ++k) {
                    const int64_t i = i0 + (int64_t)k * kServeThreads;
                    v[k] = i < rows ? __ldcv(ypin + (int64_t)b * rows + i) : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kServeUnroll; ++k) {
                    const int64_t i = i0 + (int64_t)k * kServeThreads;
                    if (i < rows) {
                        Y[i * Bp + b] = v[k];
                        R[i * Bp + b] = v[k];
                    }
                    if (i < cols) X[i * Bp + b] = 0.f;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kServeUnroll; ++k) {
                    const int64_t i = i0 + (int64_t)k * kServeThreads;
                    v[k] = i < cols ? X[i * Bp + b] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kServeUnroll; ++k) {
                    const int64_t i = i0 + (int64_t)k * kServeThreads;
                    if (i < cols) {
                        xpin[(int64_t)b * cols + i] = v[k];
                        X[i * Bp + b] = 0.f;
                    }
                    if (i < rows) {
                        Y[i * Bp + b] = 0.f;
                        R[i * Bp + b] = 0.f;
                    }
                }
                __threadfence_system();
                __syncthreads();
                if (threadIdx.x == 0 && atomicAdd(P.unit_cnt + b, 1) == chunks - 1) {
                    P.unit_cnt[b] = 0;
                    P.done[b].epochs_run = P.state[3 * B + b];
                    __threadfence_system();
                    st_release_sys(&P.done[b].seq, P.state[b]);
                }
                __syncthreads();
            }
        }
    }
}

// Power iteration helpers on slice 0 of interleaved [n][Bp] vectors:
// per-block FP64 partial sums of a*b (fixed grid, summed on the host in block
// order), and v = s * w written to slice 0 (the other slices stay zero).
constexpr int kDotBlocks = 512;

__global__ void slice_dot_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                 int64_t n, int Bp, double *__restrict__ partials) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i * Bp] * (double)b[i * Bp];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void slice_scale_kernel(const float *__restrict__ w, float *__restrict__ v, int64_t n,
                                   int Bp, float scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i * Bp] = w ? scale * w[i * Bp] : scale;
}

__global__ void negate_kernel(float *__restrict__ v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = -v[i];
}

// Slice stride Bp (B padded) and lanes per nonzero: a lane holds 4 slices,
// so Bp = 4 * LPN for B <= 128 (LPN = 1 .. 32), else a multiple of 128 taken
// in chunks of 128 by the full warp.
void slice_stride(int B, int &Bp, int &lpn) {
    lpn = 1;
    while (lpn < 32 && 4 * lpn < B) lpn *= 2;
    Bp = (lpn < 32) ? 4 * lpn : (B + 127) / 128 * 128;
}

}  // namespace
}  // namespace bsgdtv

using namespace bsgdtv;

// A stored once on the device for any number of batches (reference counted:
// the creator and every batch built on it hold one reference).
struct bsgdtv_operator_ctx {
    int device = 0;
    int64_t rows = 0, cols = 0, nnz = 0;
    int img_h = 0, img_w = 0, fmt = BSGDTV_FMT_F32_I32;
    PassOperand op_r = {}, op_c = {};
    std::vector<void *> allocs;
    std::atomic<int> refs{1};
};

struct bsgdtv_batch_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int64_t rows = 0, cols = 0, nnz = 0;
    int img_h = 0, img_w = 0, B = 0, Bp = 0, lpn = 1;
    int lpn_row = 0, lpn_col = 0;       // lanes per nonzero of the passes (0: lpn; autotuned)
    std::vector<void *> allocs;
    int fmt = BSGDTV_FMT_F32_I32;
    bsgdtv_operator_ctx *op = nullptr;  // shared A (one reference held), null if matrix free
    PassOperand op_r = {}, op_c = {};   // A in CSR / CSC: entries (weight, element index)
    bool matrix_free = false;           // weights computed on the fly (parallel beam)
    int fgp_chunk = kBatchFgpChunk;     // FGP iterations per launch (autotuned)
    int fgp_group = 0;                  // slices per FGP launch group (0: by the L2 budget)
    bool keep_prox = false;             // epochs keep the prox stage even if every lambda is 0
    double *dot_part = nullptr;         // power-iteration partial sums (first use)
    float *save_x = nullptr, *save_r[2] = {nullptr, nullptr};   // autotuner state copy (first use)
    MfGeometry mfg;
    float *ystage = nullptr;            // [max(rows, cols)] planar staging for one slice
    float *X = nullptr, *Xhat = nullptr, *Y = nullptr, *R[2] = {nullptr, nullptr};   // interleaved
    float *Xp = nullptr, *Xhp = nullptr;                                           // planar [B][cols]
    float *fgp = nullptr;   // planar FGP duals: kFgpFieldPlanes planes of B * cols floats
    float *tau = nullptr;                                                          // [B]
    int *flag = nullptr;
    float *mom = nullptr;
    int mom_len = 0;
    int cur = 0;
    bool has_data = false;
    double mu = 0.0;
    std::vector<double> lambdas;
    int64_t epoch = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraph_t tgraph[2] = {nullptr, nullptr};
    cudaGraphExec_t texec[2] = {nullptr, nullptr};
    cudaGraphNode_t tnode[2][3] = {};
    cudaEvent_t tmark[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> tevents;
    int graph_fgp_iters = -1;
    int64_t graph_kernels = 0;
    // served mode (batch_serve_enable): host-mapped mailboxes, completion
    // records, control block and staging rows (host / device addresses; the
    // memory is the caller's), device slot state, action list, per-slot unit
    // counters
    bool served = false;
    ServeView view = {};
    ServeSlot *mb_d = nullptr;
    ServeDone *done_d = nullptr;
    ServeCtrl *ctrl_d = nullptr;
    float *ypin_d = nullptr, *xpin_d = nullptr;
    int *slot_state = nullptr, *acts = nullptr, *unit_cnt = nullptr, *arm_seen = nullptr;
    int serve_grid = 1;   // CTAs of the apply kernel (2 per SM)
};

namespace {

template <typename T>
int balloc(bsgdtv_batch_ctx *h, T **out, size_t count) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
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
int bupload(bsgdtv_batch_ctx *h, T **out, const T *src, size_t count) {
    BSG_CHECK(balloc(h, out, count));
    if (count)
        BSG_CUDA(cudaMemcpyAsync(*out, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return BSGDTV_OK;
}

void bdrop_graphs(bsgdtv_batch_ctx *h) {
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

bool any_prox(const bsgdtv_batch_ctx *h, int fgp_iters) {
    if (fgp_iters <= 0) return false;
    if (h->keep_prox) return true;
    for (double l : h->lambdas)
        if (l > 0.0) return true;
    return false;
}

// Slices per FGP launch group whose fields (b and the two sets of p, q,
// p_prev, q_prev: 36 bytes per pixel) fit in about half of the L2, so the
// fields of consecutive chunk launches come from L2 rather than HBM.
int fgp_group_by_budget(const bsgdtv_batch_ctx *h) {
    return std::max<int>(1, (int)std::min<int64_t>(
                                h->B, kFgpFieldBudget / std::max<int64_t>(1, 36 * h->cols)));
}

// The slot scheduler of served parts at the start of an epoch reading
// R[par]: admissions and retirements at this epoch boundary (one launch of
// each scheduler kernel for all parts).
int enqueue_serve_prologue(bsgdtv_batch_ctx *const *parts, int n, int par, cudaStream_t s) {
    if (n < 1 || n > kMaxServeParts) return fail(BSGDTV_ERR_INVALID_ARG, "too many served parts");
    ServeLaunch L = {};
    L.n_parts = n;
    for (int k = 0; k < n; ++k) {
        const bsgdtv_batch_ctx *h = parts[k];
        L.part[k] = {h->mb_d, h->done_d, h->ctrl_d, h->slot_state, h->acts, h->tau, h->arm_seen,
                     h->ypin_d, h->xpin_d, h->unit_cnt, h->Y, h->X, h->R[par], h->rows, h->cols,
                     h->B, h->Bp};
    }
    serve_decide_kernel<<<n, kServeThreads, 0, s>>>(L);
    serve_apply_kernel<<<parts[0]->serve_grid, kServeThreads, 0, s>>>(L);
    add_launches(2);
    BSG_CUDA(cudaGetLastError());
    return BSGDTV_OK;
}

// One epoch of every slice: reads R[par], writes R[1 - par].
int benqueue_epoch(bsgdtv_batch_ctx *h, int par, int fgp_iters, cudaStream_t s,
                   cudaEvent_t *marks) {
    const bool prox = any_prox(h, fgp_iters);
    if (h->served) {
        bsgdtv_batch_ctx *one[1] = {h};
        BSG_CHECK(enqueue_serve_prologue(one, 1, par, s));
    }
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[0], s, cudaEventRecordExternal));
    if (h->matrix_free) {
        BSG_CUDA(launch_mf_pass(true, h->Bp, h->mfg, h->X, h->Y, h->R[1 - par], 0.f, s));
        BSG_CUDA(launch_mf_pass(false, h->Bp, h->mfg, h->R[par], h->X, prox ? h->Xhat : h->X,
                                (float)h->mu, s));
    } else {
        // r^k = y - A x^k (reads x before the column pass updates it)
        BSG_CUDA(launch_pass<true>(h->fmt, h->lpn_row ? h->lpn_row : h->lpn, h->op_r, h->X, h->Y, h->R[1 - par], h->rows,
                                   h->Bp, 0.f, s));
        // x^ = x^k + mu * 2 A^T r^{k-1}
        BSG_CUDA(launch_pass<false>(h->fmt, h->lpn_col ? h->lpn_col : h->lpn, h->op_c, h->R[par], h->X, prox ? h->Xhat : h->X,
                                    h->cols, h->Bp, (float)h->mu, s));
    }
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[1], s, cudaEventRecordExternal));
    if (prox) {
        const int64_t c = h->cols;
        BSG_CUDA(launch_transpose(h->Xhat, h->Xhp, c, h->B, h->Bp, true, s));
        // slices in groups (the autotuner's choice, else by the L2 budget)
        const int sg = h->fgp_group > 0 ? std::min(h->fgp_group, h->B) : fgp_group_by_budget(h);
        for (int b0 = 0; b0 < h->B; b0 += sg) {
            const int nb = std::min(sg, h->B - b0);
            const size_t o = (size_t)b0 * c;
            const FgpScratch sc = fgp_scratch_planes(h->fgp, (int64_t)h->B * c, (int64_t)o);
            BSG_CUDA(fgpk::launch_fgp_regions(h->Xhp + o, h->Xp + o, h->img_h, h->img_w,
                                              h->tau + b0, nb, c, fgp_iters, h->mom, sc, s, false,
                                              h->fgp_chunk));
        }
        BSG_CUDA(launch_transpose(h->Xp, h->X, c, h->B, h->Bp, false, s));
    }
    if (marks) BSG_CUDA(cudaEventRecordWithFlags(marks[2], s, cudaEventRecordExternal));
    return BSGDTV_OK;
}

int bensure_mom(bsgdtv_batch_ctx *h, int iters) {
    if (iters <= h->mom_len) return BSGDTV_OK;
    std::vector<float> m;
    fgp_momentum_host(iters, m);
    float *d = nullptr;
    BSG_CHECK(balloc(h, &d, m.size()));
    BSG_CUDA(cudaMemcpy(d, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
    h->mom = d;
    h->mom_len = iters;
    return BSGDTV_OK;
}

int bbuild_graphs(bsgdtv_batch_ctx *h, int fgp_iters) {
    bdrop_graphs(h);
    BSG_CHECK(bensure_mom(h, std::max(fgp_iters, 1)));
    for (int k = 0; k < 3; ++k)
        if (!h->tmark[k]) BSG_CUDA(cudaEventCreate(&h->tmark[k]));
    const int64_t before = bsgdtv_launch_count();
    for (int timed = 0; timed < 2; ++timed) {
        for (int par = 0; par < 2; ++par) {
            cudaGraph_t g = nullptr;
            BSG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = benqueue_epoch(h, par, fgp_iters, h->cap_stream, timed ? h->tmark : nullptr);
            cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
            if (rc != BSGDTV_OK) {
                if (g) cudaGraphDestroy(g);
                add_launches(before - bsgdtv_launch_count());
                return rc;
            }
            if (e != cudaSuccess)
                return fail(BSGDTV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            if (!timed) {
                e = cudaGraphInstantiate(&h->gexec[par], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess)
                    return fail(BSGDTV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
                continue;
            }
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
    }
    // capture counted each epoch's kernels four times; replays are counted in run
    const int64_t captured = bsgdtv_launch_count() - before;
    add_launches(-captured);
    h->graph_kernels = captured / 4;
    h->graph_fgp_iters = fgp_iters;
    return BSGDTV_OK;
}

// Packed CSR of A and its CSC (rows ascending inside each column): weights
// as the format stores them, element indices.
struct PackedOperator {
    std::vector<int64_t> col_ptr;
    std::vector<int2> ent_r, ent_c;                // FP32 weights
    std::vector<uint16_t> w_r, w_c;                // 16-bit weights
    std::vector<int32_t> off_r, off_c;
};

void pack_operator(int64_t rows, int64_t cols, const int64_t *row_ptr, const int32_t *col_idx,
                   const double *vals, int fmt, PackedOperator &P) {
    const int64_t nnz = row_ptr[rows];
    const bool f32 = (fmt == BSGDTV_FMT_F32_I32);
    auto put = [&](std::vector<int2> &ent, std::vector<uint16_t> &w, std::vector<int32_t> &off,
                   int64_t k, double a, int64_t idx) {
        const int32_t o = (int32_t)idx;
        if (f32) {
            const float f = (float)a;
            int bits;
            std::memcpy(&bits, &f, sizeof(bits));
            ent[k] = make_int2(bits, o);
        } else {
            w[k] = (fmt == BSGDTV_FMT_F16_I16) ? double_to_half_bits(a) : double_to_bf16_bits(a);
            off[k] = o;
        }
    };
    if (f32) {
        P.ent_r.resize(nnz);
        P.ent_c.resize(nnz);
    } else {
        P.w_r.resize(nnz);
        P.w_c.resize(nnz);
        P.off_r.resize(nnz);
        P.off_c.resize(nnz);
    }
    for (int64_t e = 0; e < nnz; ++e) put(P.ent_r, P.w_r, P.off_r, e, vals[e], col_idx[e]);
    P.col_ptr.assign(cols + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) P.col_ptr[col_idx[e] + 1]++;
    for (int64_t c = 0; c < cols; ++c) P.col_ptr[c + 1] += P.col_ptr[c];
    std::vector<int64_t> cur(P.col_ptr.begin(), P.col_ptr.end() - 1);
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
            put(P.ent_c, P.w_c, P.off_c, cur[col_idx[e]]++, vals[e], r);
}

}  // namespace

namespace bsgdtv {

void batch_keep_prox(bsgdtv_batch_t h, bool on) {
    if (h && h->keep_prox != on) {
        h->keep_prox = on;
        bdrop_graphs(h);
    }
}

int validate_image_csr(int64_t rows, int64_t cols, int img_h, int img_w, const int64_t *row_ptr,
                       const int32_t *col_idx, const double *vals) {
    if (!row_ptr || !col_idx || !vals) return fail(BSGDTV_ERR_INVALID_ARG, "null CSR array");
    if (rows < 1 || cols < 1 || img_h < 1 || img_w < 1 || (int64_t)img_h * img_w != cols)
        return fail(BSGDTV_ERR_INVALID_ARG, "bad sizes: need rows >= 1 and cols == img_h*img_w");
    if (rows > INT32_MAX || cols > INT32_MAX)
        return fail(BSGDTV_ERR_INVALID_ARG, "rows and cols must fit int32");
    if (row_ptr[0] != 0) return fail(BSGDTV_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int64_t r = 0; r < rows; ++r) {
        if (row_ptr[r + 1] < row_ptr[r]) return fail(BSGDTV_ERR_INVALID_ARG, "row_ptr decreases");
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= cols)
                return fail(BSGDTV_ERR_INVALID_ARG, "column index out of range");
            if (e > row_ptr[r] && col_idx[e] <= col_idx[e - 1])
                return fail(BSGDTV_ERR_INVALID_ARG, "column indices must ascend within a row");
            if (!std::isfinite(vals[e])) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in A");
        }
    }
    return BSGDTV_OK;
}

}  // namespace bsgdtv

namespace {

// Vectors of a batch (interleaved, planar, FGP fields, staging), zeroed.
int alloc_vectors(bsgdtv_batch_ctx *hp) {
    const size_t Ri = (size_t)hp->rows * hp->Bp, Ci = (size_t)hp->cols * hp->Bp;
    const size_t Cp = (size_t)hp->cols * hp->B;
    BSG_CHECK(balloc(hp, &hp->ystage, (size_t)std::max(hp->rows, hp->cols)));
    for (float **p : {&hp->X, &hp->Xhat}) BSG_CHECK(balloc(hp, p, Ci));
    for (float **p : {&hp->Y, &hp->R[0], &hp->R[1]}) BSG_CHECK(balloc(hp, p, Ri));
    for (float **p : {&hp->Xp, &hp->Xhp}) BSG_CHECK(balloc(hp, p, Cp));
    BSG_CHECK(balloc(hp, &hp->fgp, kFgpFieldPlanes * Cp));
    BSG_CHECK(balloc(hp, &hp->tau, (size_t)hp->B));
    BSG_CHECK(balloc(hp, &hp->flag, 1));
    // padded slices (b >= B) stay zero for good: y = x = r = 0 there
    for (float *p : {hp->X, hp->Xhat}) BSG_CUDA(cudaMemsetAsync(p, 0, Ci * sizeof(float), hp->stream));
    for (float *p : {hp->Y, hp->R[0], hp->R[1]})
        BSG_CUDA(cudaMemsetAsync(p, 0, Ri * sizeof(float), hp->stream));
    return BSGDTV_OK;
}

}  // namespace

namespace bsgdtv {

// The parallel-beam A as a host CSR, weights from the matrix-free projector
// (mf_weights_kernel, chunks of rays on the device), each row's columns
// sorted ascending.  Values are the FP32 weights widened to FP64.
int generate_parallel_beam_csr(int n, int n_angles, int n_bins, cudaStream_t s,
                               std::vector<int64_t> &row_ptr, std::vector<int32_t> &col_idx,
                               std::vector<double> &vals) {
    const int64_t rows = (int64_t)n_angles * n_bins;
    const int capacity = 2 * n + 2;   // a line meets at most 2n - 1 pixels of an n x n grid
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(rows, ((int64_t)256 << 20) / ((int64_t)capacity * 8)));
    std::vector<AngleGeo> table;
    mf_angle_table(n_angles, table);
    std::vector<int64_t> ray_ids((size_t)chunk);
    std::vector<int32_t> h_cols((size_t)chunk * capacity);
    std::vector<float> h_vals((size_t)chunk * capacity);
    std::vector<int> h_cnt((size_t)chunk);
    row_ptr.assign(rows + 1, 0);
    col_idx.clear();
    vals.clear();
    void *buf = nullptr;
    const size_t bytes = table.size() * sizeof(AngleGeo) + chunk * sizeof(int64_t) +
                         (size_t)chunk * capacity * (sizeof(int32_t) + sizeof(float)) + chunk * sizeof(int) + 1024;
    BSG_CUDA(cudaMalloc(&buf, bytes));
    char *p = static_cast<char *>(buf);
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) / 256 * 256;
        return q;
    };
    AngleGeo *geo = reinterpret_cast<AngleGeo *>(take(table.size() * sizeof(AngleGeo)));
    int64_t *d_rays = reinterpret_cast<int64_t *>(take(chunk * sizeof(int64_t)));
    int32_t *d_cols = reinterpret_cast<int32_t *>(take((size_t)chunk * capacity * sizeof(int32_t)));
    float *d_vals = reinterpret_cast<float *>(take((size_t)chunk * capacity * sizeof(float)));
    int *d_cnt = reinterpret_cast<int *>(take(chunk * sizeof(int)));
    const int rc = [&]() -> int {
        BSG_CUDA(cudaMemcpyAsync(geo, table.data(), table.size() * sizeof(AngleGeo), cudaMemcpyHostToDevice, s));
        MfGeometry G;
        G.geo = geo;
        G.n = n;
        G.n_angles = n_angles;
        G.n_bins = n_bins;
        std::vector<std::pair<int32_t, float>> row;
        for (int64_t r0 = 0; r0 < rows; r0 += chunk) {
            const int nr = (int)std::min<int64_t>(chunk, rows - r0);
            for (int i = 0; i < nr; ++i) ray_ids[i] = r0 + i;
            BSG_CUDA(cudaMemcpyAsync(d_rays, ray_ids.data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            BSG_CUDA(launch_mf_weights(G, d_rays, nr, capacity, d_cols, d_vals, d_cnt, s));
            BSG_CUDA(cudaMemcpyAsync(h_cnt.data(), d_cnt, nr * sizeof(int), cudaMemcpyDeviceToHost, s));
            BSG_CUDA(cudaMemcpyAsync(h_cols.data(), d_cols, (size_t)nr * capacity * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
            BSG_CUDA(cudaMemcpyAsync(h_vals.data(), d_vals, (size_t)nr * capacity * sizeof(float),
                                     cudaMemcpyDeviceToHost, s));
            BSG_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i < nr; ++i) {
                const int c = h_cnt[i];
                if (c < 0 || c >= capacity) return fail(BSGDTV_ERR_STATE, "ray meets more pixels than a line can");
                row.clear();
                for (int k = 0; k < c; ++k)
                    row.push_back({h_cols[(size_t)i * capacity + k], h_vals[(size_t)i * capacity + k]});
                std::sort(row.begin(), row.end());
                for (size_t k = 0; k < row.size(); ++k) {
                    if (k > 0 && row[k].first == row[k - 1].first)
                        return fail(BSGDTV_ERR_STATE, "pixel met twice by one ray");
                    col_idx.push_back(row[k].first);
                    vals.push_back((double)row[k].second);
                }
                row_ptr[r0 + i + 1] = (int64_t)col_idx.size();
            }
        }
        return BSGDTV_OK;
    }();
    cudaFree(buf);
    return rc;
}

}  // namespace bsgdtv

namespace bsgdtv {

// Copies n floats of y (host or device) to dst on the handle's stream and
// checks them for NaN/Inf on the device; returns after the check has been
// read back, so the copy has read y (a host y may be reused at once, pageable
// or pinned).  *finite: the check.
int upload_checked(bsgdtv_batch_t h, float *dst, const float *y, int y_on_device, int64_t n,
                   bool *finite) {
    cudaStream_t s = h->stream;
    int hflag = 0;
    BSG_CUDA(cudaMemcpyAsync(dst, y, (size_t)n * sizeof(float),
                             y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    BSG_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    BSG_CUDA(launch_check_finite(dst, n, h->flag, s));
    BSG_CUDA(cudaMemcpyAsync(&hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BSG_CUDA(cudaStreamSynchronize(s));
    *finite = hflag == 0;
    return BSGDTV_OK;
}

// bsgdtv_batch_set_slice; check = false skips the NaN/Inf check of a host y
// (a caller that has checked it) and with it the wait for the copy: a
// pageable y is staged by the copy call itself.
int batch_set_slice(bsgdtv_batch_t h, int b, const float *y, int y_on_device, double lambda,
                    bool check) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "set_slice before set_data");
    if (b < 0 || b >= h->B) return fail(BSGDTV_ERR_INVALID_ARG, "slice index out of range");
    if (!(lambda >= 0.0) || !std::isfinite(lambda))
        return fail(BSGDTV_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    BSG_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t rows = h->rows;
    if (y && (check || y_on_device)) {   // staged: a bad y leaves the slot as it was
        bool finite = false;
        BSG_CHECK(upload_checked(h, h->ystage, y, y_on_device, rows, &finite));
        if (!finite) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in y");
    } else if (y) {
        BSG_CUDA(cudaMemcpyAsync(h->ystage, y, (size_t)rows * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    const double lam = y ? lambda : 0.0;
    const int64_t n = std::max(rows, h->cols);
    slice_reset_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y ? h->ystage : nullptr, h->Y, h->X,
                                                                   h->R[h->cur], rows, h->cols, h->Bp, b);
    add_launches(1);
    BSG_CUDA(cudaGetLastError());
    const float tau = (float)(h->mu * lam);
    BSG_CUDA(cudaMemcpyAsync(h->tau + b, &tau, sizeof(float), cudaMemcpyHostToDevice, s));
    const bool prox_before = any_prox(h, 1);
    h->lambdas[b] = lam;
    if (any_prox(h, 1) != prox_before) bdrop_graphs(h);   // the epoch gains or loses its prox
    return BSGDTV_OK;
}

namespace {
struct ServeLayout {
    size_t mb, done, ctrl, y, x, total;
};
ServeLayout serve_layout(int B, int64_t rows, int64_t cols) {
    auto up256 = [](size_t v) { return (v + 255) / 256 * 256; };
    ServeLayout L;
    L.mb = 0;
    L.done = up256(L.mb + (size_t)B * sizeof(ServeSlot));
    L.ctrl = up256(L.done + (size_t)B * sizeof(ServeDone));
    L.y = up256(L.ctrl + sizeof(ServeCtrl));
    L.x = up256(L.y + (size_t)B * rows * sizeof(float));
    L.total = up256(L.x + (size_t)B * cols * sizeof(float));
    return L;
}
}  // namespace

size_t batch_serve_host_bytes(int B, int64_t rows, int64_t cols) {
    return serve_layout(B, rows, cols).total;
}

int batch_serve_enable(bsgdtv_batch_t h, ServeView *view, void *host_block) {
    if (!h || !view || !host_block) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "served mode before set_data");
    if (h->served) return fail(BSGDTV_ERR_STATE, "batch already served");
    if (h->B > 0xFFFFFF) return fail(BSGDTV_ERR_INVALID_ARG, "too many slots for served mode");
    BSG_CUDA(cudaSetDevice(h->device));
    const int B = h->B;
    const ServeLayout lay = serve_layout(B, h->rows, h->cols);
    void *hp = host_block;
    std::memset(hp, 0, lay.y);   // mailboxes, records and control start at zero
    void *dp = nullptr;
    BSG_CUDA(cudaHostGetDevicePointer(&dp, hp, 0));
    unsigned char *hb = static_cast<unsigned char *>(hp), *db = static_cast<unsigned char *>(dp);
    h->view.mb = reinterpret_cast<ServeSlot *>(hb + lay.mb);
    h->view.done = reinterpret_cast<ServeDone *>(hb + lay.done);
    h->view.ctrl = reinterpret_cast<ServeCtrl *>(hb + lay.ctrl);
    h->view.ypin = reinterpret_cast<float *>(hb + lay.y);
    h->view.xpin = reinterpret_cast<float *>(hb + lay.x);
    h->view.rows = h->rows;
    h->view.cols = h->cols;
    h->view.B = B;
    h->mb_d = reinterpret_cast<ServeSlot *>(db + lay.mb);
    h->done_d = reinterpret_cast<ServeDone *>(db + lay.done);
    h->ctrl_d = reinterpret_cast<ServeCtrl *>(db + lay.ctrl);
    h->ypin_d = reinterpret_cast<float *>(db + lay.y);
    h->xpin_d = reinterpret_cast<float *>(db + lay.x);
    BSG_CHECK(balloc(h, &h->slot_state, (size_t)4 * B + 1));
    BSG_CHECK(balloc(h, &h->acts, (size_t)B + 1));
    BSG_CHECK(balloc(h, &h->unit_cnt, (size_t)B));
    BSG_CHECK(balloc(h, &h->arm_seen, 1));
    BSG_CUDA(cudaMemsetAsync(h->slot_state, 0, ((size_t)4 * B + 1) * sizeof(int), h->stream));
    BSG_CUDA(cudaMemsetAsync(h->acts, 0, ((size_t)B + 1) * sizeof(int), h->stream));
    BSG_CUDA(cudaMemsetAsync(h->unit_cnt, 0, (size_t)B * sizeof(int), h->stream));
    BSG_CUDA(cudaMemsetAsync(h->arm_seen, 0, sizeof(int), h->stream));
    BSG_CUDA(cudaStreamSynchronize(h->stream));
    int sms = 1;
    BSG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->serve_grid = 2 * std::max(sms, 1);
    h->served = true;
    bdrop_graphs(h);   // the epochs gain the scheduler
    *view = h->view;
    return BSGDTV_OK;
}

}  // namespace bsgdtv

extern "C" {

int bsgdtv_operator_create_csr(bsgdtv_operator_t *out, int64_t rows, int64_t cols, int img_h,
                               int img_w, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *vals, int format, void *stream) {
    BSG_TRACE();
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (format != BSGDTV_FMT_F32_I32 && format != BSGDTV_FMT_F16_I16 && format != BSGDTV_FMT_BF16_I16)
        return fail(format == BSGDTV_FMT_F32_I16 ? BSGDTV_ERR_UNSUPPORTED : BSGDTV_ERR_INVALID_ARG,
                    "batch formats: BSGDTV_FMT_F32_I32, BSGDTV_FMT_F16_I16, BSGDTV_FMT_BF16_I16");
    BSG_CHECK(validate_image_csr(rows, cols, img_h, img_w, row_ptr, col_idx, vals));
    std::unique_ptr<bsgdtv_operator_ctx> op(new (std::nothrow) bsgdtv_operator_ctx());
    if (!op) return fail(BSGDTV_ERR_OOM, "host allocation");
    BSG_CUDA(cudaGetDevice(&op->device));
    op->rows = rows;
    op->cols = cols;
    op->nnz = row_ptr[rows];
    op->img_h = img_h;
    op->img_w = img_w;
    op->fmt = format;
    cudaStream_t s = (cudaStream_t)stream;
    bsgdtv_operator_ctx *o = op.get();
    auto up = [&](auto **dst, const auto *src, size_t count) -> int {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(*src);
        const cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BSGDTV_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                            "): " + cudaGetErrorString(e));
        }
        o->allocs.push_back(p);
        *dst = static_cast<std::remove_reference_t<decltype(**dst)> *>(p);
        if (count)
            BSG_CUDA(cudaMemcpyAsync(p, src, count * sizeof(*src), cudaMemcpyHostToDevice, s));
        return BSGDTV_OK;
    };
    int rc = BSGDTV_OK;
    try {
        PackedOperator P;
        pack_operator(rows, cols, row_ptr, col_idx, vals, format, P);
        rc = [&]() -> int {
            int64_t *rp = nullptr, *cp = nullptr;
            BSG_CHECK(up(&rp, row_ptr, (size_t)rows + 1));
            BSG_CHECK(up(&cp, P.col_ptr.data(), (size_t)cols + 1));
            o->op_r.ptr = rp;
            o->op_c.ptr = cp;
            if (format == BSGDTV_FMT_F32_I32) {
                int2 *er = nullptr, *ec = nullptr;
                BSG_CHECK(up(&er, P.ent_r.data(), (size_t)o->nnz));
                BSG_CHECK(up(&ec, P.ent_c.data(), (size_t)o->nnz));
                o->op_r.ent = er;
                o->op_c.ent = ec;
            } else {
                uint16_t *wr = nullptr, *wc = nullptr;
                int32_t *orr = nullptr, *oc = nullptr;
                BSG_CHECK(up(&wr, P.w_r.data(), (size_t)o->nnz));
                BSG_CHECK(up(&orr, P.off_r.data(), (size_t)o->nnz));
                BSG_CHECK(up(&wc, P.w_c.data(), (size_t)o->nnz));
                BSG_CHECK(up(&oc, P.off_c.data(), (size_t)o->nnz));
                o->op_r.w16 = wr;
                o->op_r.off = orr;
                o->op_c.w16 = wc;
                o->op_c.off = oc;
            }
            BSG_CUDA(cudaStreamSynchronize(s));   // the host arrays die here
            return BSGDTV_OK;
        }();
    } catch (const std::bad_alloc &) {
        rc = fail(BSGDTV_ERR_OOM, "host allocation");
    }
    if (rc != BSGDTV_OK) {
        bsgdtv_operator_destroy(op.release());
        return rc;
    }
    *out = op.release();
    return BSGDTV_OK;
}

void bsgdtv_operator_destroy(bsgdtv_operator_t op) {
    if (!op) return;
    if (op->refs.fetch_sub(1) != 1) return;   // batches still use it
    cudaSetDevice(op->device);
    for (void *p : op->allocs) cudaFree(p);
    delete op;
}

int bsgdtv_batch_create_from_operator(bsgdtv_batch_t *out, bsgdtv_operator_t op, int slices,
                                      void *stream) {
    BSG_TRACE();
    if (!out || !op) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (slices < 1 || slices > 4096) return fail(BSGDTV_ERR_INVALID_ARG, "slices must be in [1, 4096]");
    std::unique_ptr<bsgdtv_batch_ctx> h(new (std::nothrow) bsgdtv_batch_ctx());
    if (!h) return fail(BSGDTV_ERR_OOM, "host allocation");
    BSG_CUDA(cudaGetDevice(&h->device));
    if (h->device != op->device) return fail(BSGDTV_ERR_INVALID_ARG, "operator is on another device");
    h->stream = (cudaStream_t)stream;
    h->rows = op->rows;
    h->cols = op->cols;
    h->nnz = op->nnz;
    h->img_h = op->img_h;
    h->img_w = op->img_w;
    h->B = slices;
    h->fmt = op->fmt;
    h->op_r = op->op_r;
    h->op_c = op->op_c;
    op->refs.fetch_add(1);
    h->op = op;
    slice_stride(slices, h->Bp, h->lpn);
    if (h->lpn < 32 && std::max(h->rows, h->cols) * h->Bp > INT32_MAX) {
        // the passes form element * stride in 32 bits below 128 slices
        bsgdtv_batch_destroy(h.release());
        return fail(BSGDTV_ERR_UNSUPPORTED, "max(rows, cols) * padded slices must fit int32");
    }
    bsgdtv_batch_ctx *hp = h.get();
    const int rc = [&]() -> int {
        BSG_CUDA(cudaStreamCreateWithFlags(&hp->cap_stream, cudaStreamNonBlocking));
        BSG_CHECK(alloc_vectors(hp));
        BSG_CUDA(cudaStreamSynchronize(hp->stream));
        return BSGDTV_OK;
    }();
    if (rc != BSGDTV_OK) {
        bsgdtv_batch_destroy(h.release());
        return rc;
    }
    *out = h.release();
    return BSGDTV_OK;
}

int bsgdtv_batch_create_csr_ex(bsgdtv_batch_t *out, int64_t rows, int64_t cols, int img_h,
                               int img_w, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *vals, int slices, int format, void *stream) {
    BSG_TRACE();
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (slices < 1 || slices > 4096) return fail(BSGDTV_ERR_INVALID_ARG, "slices must be in [1, 4096]");
    bsgdtv_operator_t op = nullptr;
    BSG_CHECK(bsgdtv_operator_create_csr(&op, rows, cols, img_h, img_w, row_ptr, col_idx, vals, format,
                                         stream));
    const int rc = bsgdtv_batch_create_from_operator(out, op, slices, stream);
    bsgdtv_operator_destroy(op);   // the batch keeps its own reference
    return rc;
}

int64_t bsgdtv_batch_device_bytes(int64_t rows, int64_t cols, int64_t nnz, int slices, int format) {
    if (rows < 1 || cols < 1 || nnz < 0 || slices < 1) return -1;
    int Bp = 0, lpn = 0;
    slice_stride(slices, Bp, lpn);
    const int64_t per_nz = (format == BSGDTV_FMT_F32_I32) ? 8 : 6;
    const int64_t a = 2 * (nnz * per_nz + 8 * (rows + cols + 2));
    const int64_t inter = 4 * (int64_t)Bp * (2 * cols + 3 * rows);
    const int64_t planar = 4 * (int64_t)slices * (2 + kFgpFieldPlanes) * cols;
    return a + inter + planar + 4 * (std::max(rows, cols) + slices + 64) + 4 * 4096;
}

int bsgdtv_batch_create_parallel_beam(bsgdtv_batch_t *out, int n, int n_angles, int n_bins,
                                      int slices, void *stream) {
    BSG_TRACE();
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (slices < 1 || slices > 4096) return fail(BSGDTV_ERR_INVALID_ARG, "slices must be in [1, 4096]");
    if (n < 1 || n > 16384 || n_angles < 1 || n_bins < 1 || (int64_t)n_angles * n_bins > INT32_MAX)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= n <= 16384, n_angles, n_bins >= 1");
    std::unique_ptr<bsgdtv_batch_ctx> h(new (std::nothrow) bsgdtv_batch_ctx());
    if (!h) return fail(BSGDTV_ERR_OOM, "host allocation");
    BSG_CUDA(cudaGetDevice(&h->device));
    h->stream = (cudaStream_t)stream;
    h->rows = (int64_t)n_angles * n_bins;
    h->cols = (int64_t)n * n;
    h->img_h = h->img_w = n;
    h->B = slices;
    h->matrix_free = true;
    slice_stride(slices, h->Bp, h->lpn);
    if (std::max(h->rows, h->cols) * h->Bp > INT32_MAX)
        return fail(BSGDTV_ERR_UNSUPPORTED, "max(rows, cols) * padded slices must fit int32");
    bsgdtv_batch_ctx *hp = h.get();
    int rc = [&]() -> int {
        std::vector<AngleGeo> table;
        mf_angle_table(n_angles, table);
        AngleGeo *geo = nullptr;
        BSG_CUDA(cudaStreamCreateWithFlags(&hp->cap_stream, cudaStreamNonBlocking));
        BSG_CHECK(bupload(hp, &geo, table.data(), table.size()));
        hp->mfg.geo = geo;
        hp->mfg.n = n;
        hp->mfg.n_angles = n_angles;
        hp->mfg.n_bins = n_bins;
        BSG_CHECK(alloc_vectors(hp));
        BSG_CUDA(cudaStreamSynchronize(hp->stream));   // the host table dies here
        return BSGDTV_OK;
    }();
    if (rc != BSGDTV_OK) {
        bsgdtv_batch_destroy(h.release());
        return rc;
    }
    *out = h.release();
    return BSGDTV_OK;
}

int bsgdtv_mf_ray_weights(int n, int n_angles, int n_bins, const int64_t *rays, int n_rays,
                          int capacity, int32_t *cols, float *vals, int *counts) {
    if (!rays || !cols || !vals || !counts || n < 1 || n_angles < 1 || n_bins < 1 || n_rays < 0 ||
        capacity < 1)
        return fail(BSGDTV_ERR_INVALID_ARG, "bad argument");
    const int64_t total_rays = (int64_t)n_angles * n_bins;
    for (int i = 0; i < n_rays; ++i)
        if (rays[i] < 0 || rays[i] >= total_rays) return fail(BSGDTV_ERR_INVALID_ARG, "ray out of range");
    if (n_rays == 0) return BSGDTV_OK;
    std::vector<AngleGeo> table;
    mf_angle_table(n_angles, table);
    const size_t cap = (size_t)n_rays * capacity;
    void *buf = nullptr;
    const size_t bytes = table.size() * sizeof(AngleGeo) + n_rays * sizeof(int64_t) +
                         cap * (sizeof(int32_t) + sizeof(float)) + n_rays * sizeof(int) + 1024;
    BSG_CUDA(cudaMalloc(&buf, bytes));
    char *p = static_cast<char *>(buf);
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) / 256 * 256;
        return q;
    };
    AngleGeo *geo = reinterpret_cast<AngleGeo *>(take(table.size() * sizeof(AngleGeo)));
    int64_t *d_rays = reinterpret_cast<int64_t *>(take(n_rays * sizeof(int64_t)));
    int32_t *d_cols = reinterpret_cast<int32_t *>(take(cap * sizeof(int32_t)));
    float *d_vals = reinterpret_cast<float *>(take(cap * sizeof(float)));
    int *d_cnt = reinterpret_cast<int *>(take(n_rays * sizeof(int)));
    int rc = [&]() -> int {
        BSG_CUDA(cudaMemcpy(geo, table.data(), table.size() * sizeof(AngleGeo), cudaMemcpyHostToDevice));
        BSG_CUDA(cudaMemcpy(d_rays, rays, n_rays * sizeof(int64_t), cudaMemcpyHostToDevice));
        MfGeometry G;
        G.geo = geo;
        G.n = n;
        G.n_angles = n_angles;
        G.n_bins = n_bins;
        BSG_CUDA(launch_mf_weights(G, d_rays, n_rays, capacity, d_cols, d_vals, d_cnt, 0));
        BSG_CUDA(cudaMemcpy(cols, d_cols, cap * sizeof(int32_t), cudaMemcpyDeviceToHost));
        BSG_CUDA(cudaMemcpy(vals, d_vals, cap * sizeof(float), cudaMemcpyDeviceToHost));
        BSG_CUDA(cudaMemcpy(counts, d_cnt, n_rays * sizeof(int), cudaMemcpyDeviceToHost));
        return BSGDTV_OK;
    }();
    cudaFree(buf);
    return rc;
}

int bsgdtv_batch_create_csr(bsgdtv_batch_t *out, int64_t rows, int64_t cols, int img_h, int img_w,
                            const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                            int slices, void *stream) {
    return bsgdtv_batch_create_csr_ex(out, rows, cols, img_h, img_w, row_ptr, col_idx, vals, slices,
                                      BSGDTV_FMT_F32_I32, stream);
}

void bsgdtv_batch_destroy(bsgdtv_batch_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    bdrop_graphs(h);
    for (cudaEvent_t ev : h->tevents) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->tmark)
        if (ev) cudaEventDestroy(ev);
    for (void *p : h->allocs) cudaFree(p);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    bsgdtv_operator_t op = h->op;
    delete h;
    bsgdtv_operator_destroy(op);
}


int bsgdtv_batch_set_data(bsgdtv_batch_t h, const float *y, int y_on_device,
                          const double *lambdas, double mu) {
    BSG_TRACE();
    if (!h || !y || !lambdas) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (!(mu > 0.0) || !std::isfinite(mu)) return fail(BSGDTV_ERR_INVALID_ARG, "mu must be finite and > 0");
    for (int b = 0; b < h->B; ++b)
        if (!(lambdas[b] >= 0.0) || !std::isfinite(lambdas[b]))
            return fail(BSGDTV_ERR_INVALID_ARG, "every lambda must be finite and >= 0");
    BSG_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t rows = h->rows, n_in = rows * h->B;
    // y arrives slice-major [B][rows]; it is staged in R[1] (rows * Bp >= rows * B
    // floats) and interleaved into Y; the first epoch rewrites R[1] in full.
    // From here on the old state is gone: a failure leaves the handle without data.
    h->has_data = false;
    bool finite = false;
    BSG_CHECK(upload_checked(h, h->R[1], y, y_on_device, n_in, &finite));
    if (!finite) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in y");
    BSG_CUDA(launch_transpose(h->R[1], h->Y, rows, h->B, h->Bp, false, s));
    // x^0 = 0 and r^{-1} = y - A x^0 = y for every slice
    BSG_CUDA(cudaMemsetAsync(h->X, 0, (size_t)h->cols * h->Bp * sizeof(float), s));
    BSG_CUDA(cudaMemcpyAsync(h->R[0], h->Y, (size_t)rows * h->Bp * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
    std::vector<float> tau(h->B);
    for (int b = 0; b < h->B; ++b) tau[b] = (float)(mu * lambdas[b]);
    BSG_CUDA(cudaMemcpyAsync(h->tau, tau.data(), h->B * sizeof(float), cudaMemcpyHostToDevice, s));
    // mu is a kernel argument of the captured epochs and the weights decide
    // whether the epoch has a prox at all: the graphs are rebuilt on next run
    bdrop_graphs(h);
    h->mu = mu;
    h->lambdas.assign(lambdas, lambdas + h->B);
    h->cur = 0;
    h->epoch = 0;
    h->has_data = true;
    BSG_CUDA(cudaStreamSynchronize(s));
    return BSGDTV_OK;
}

int bsgdtv_batch_run_timed(bsgdtv_batch_t h, int epochs, int fgp_iters, double *products_ms,
                           double *epoch_ms) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "run before set_data");
    if (epochs < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epochs / fgp_iters");
    if (epochs == 0) return BSGDTV_OK;
    BSG_CUDA(cudaSetDevice(h->device));
    if (!h->gexec[0] || h->graph_fgp_iters != fgp_iters) BSG_CHECK(bbuild_graphs(h, fgp_iters));
    const bool timed = products_ms || epoch_ms;
    if (timed)
        while (h->tevents.size() < (size_t)3 * epochs) {
            cudaEvent_t ev;
            BSG_CUDA(cudaEventCreate(&ev));
            h->tevents.push_back(ev);
        }
    for (int e = 0; e < epochs; ++e) {
        if (timed) {
            cudaGraphExec_t ex = h->texec[h->cur];
            for (int k = 0; k < 3; ++k)
                BSG_CUDA(cudaGraphExecEventRecordNodeSetEvent(ex, h->tnode[h->cur][k],
                                                              h->tevents[3 * e + k]));
            BSG_CUDA(cudaGraphLaunch(ex, h->stream));
        } else {
            BSG_CUDA(cudaGraphLaunch(h->gexec[h->cur], h->stream));
        }
        add_launches(h->graph_kernels);
        h->cur ^= 1;
        h->epoch++;
    }
    if (timed) {
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
    }
    return BSGDTV_OK;
}

int bsgdtv_batch_run(bsgdtv_batch_t h, int epochs, int fgp_iters) {
    BSG_TRACE();
    return bsgdtv_batch_run_timed(h, epochs, fgp_iters, nullptr, nullptr);
}

int bsgdtv_batch_get_x(bsgdtv_batch_t h, float *x, int out_on_device) {
    BSG_TRACE();
    if (!h || !x) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    BSG_CUDA(cudaSetDevice(h->device));
    const int64_t c = h->cols;
    BSG_CUDA(launch_transpose(h->X, h->Xp, c, h->B, h->Bp, true, h->stream));
    BSG_CUDA(cudaMemcpyAsync(x, h->Xp, (size_t)c * h->B * sizeof(float),
                             out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             h->stream));
    if (!out_on_device) BSG_CUDA(cudaStreamSynchronize(h->stream));
    return BSGDTV_OK;
}

int bsgdtv_batch_set_slice(bsgdtv_batch_t h, int b, const float *y, int y_on_device, double lambda) {
    BSG_TRACE();
    return bsgdtv::batch_set_slice(h, b, y, y_on_device, lambda, true);
}

int bsgdtv_batch_estimate_umax(bsgdtv_batch_t h, int max_iters, double rel_tol, double *u_max,
                               int *iters) {
    BSG_TRACE();
    if (!h || max_iters < 1 || !(rel_tol >= 0.0)) return fail(BSGDTV_ERR_INVALID_ARG, "bad argument");
    BSG_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t c = h->cols, R = h->rows;
    std::vector<double> part(kDotBlocks);
    if (!h->dot_part) BSG_CHECK(balloc(h, &h->dot_part, kDotBlocks));
    double *d_part = h->dot_part;
    auto dot = [&](const float *a, const float *b, double *out) -> int {
        slice_dot_kernel<<<kDotBlocks, 256, 0, s>>>(a, b, c, h->Bp, d_part);
        add_launches(1);
        BSG_CUDA(cudaGetLastError());
        BSG_CUDA(cudaMemcpyAsync(part.data(), d_part, kDotBlocks * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        BSG_CUDA(cudaStreamSynchronize(s));
        double acc = 0.0;
        for (double v : part) acc += v;
        *out = acc;
        return BSGDTV_OK;
    };
    const unsigned grid = (unsigned)((c + 255) / 256);
    // all slices zero; v = ones / sqrt(c) in slice 0 of X; R[0] = 0 stands for y = 0
    BSG_CUDA(cudaMemsetAsync(h->X, 0, (size_t)c * h->Bp * sizeof(float), s));
    BSG_CUDA(cudaMemsetAsync(h->R[0], 0, (size_t)R * h->Bp * sizeof(float), s));
    slice_scale_kernel<<<grid, 256, 0, s>>>(nullptr, h->X, c, h->Bp, (float)(1.0 / std::sqrt((double)c)));
    add_launches(1);
    BSG_CUDA(cudaGetLastError());
    double u = 0.0;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        BSG_CUDA(cudaMemsetAsync(h->Xhat, 0, (size_t)c * h->Bp * sizeof(float), s));
        // R1 = 0 - A v; Xhat = 0 + 2 * 0.5 * A^T R1 = -A^T A v
        if (h->matrix_free) {
            BSG_CUDA(launch_mf_pass(true, h->Bp, h->mfg, h->X, h->R[0], h->R[1], 0.f, s));
            BSG_CUDA(launch_mf_pass(false, h->Bp, h->mfg, h->R[1], h->Xhat, h->Xhat, 0.5f, s));
        } else {
            BSG_CUDA(launch_pass<true>(h->fmt, h->lpn, h->op_r, h->X, h->R[0], h->R[1], R, h->Bp, 0.f, s));
            BSG_CUDA(launch_pass<false>(h->fmt, h->lpn, h->op_c, h->R[1], h->Xhat, h->Xhat, c, h->Bp,
                                        0.5f, s));
        }
        double vw = 0.0, ww = 0.0;
        BSG_CHECK(dot(h->X, h->Xhat, &vw));
        BSG_CHECK(dot(h->Xhat, h->Xhat, &ww));
        const double u_new = -vw;   // Rayleigh quotient, |v| = 1
        if (!(ww > 0.0)) {
            u = 0.0;
            break;
        }
        slice_scale_kernel<<<grid, 256, 0, s>>>(h->Xhat, h->X, c, h->Bp, (float)(-1.0 / std::sqrt(ww)));
        add_launches(1);
        BSG_CUDA(cudaGetLastError());
        const bool done = it > 1 && std::fabs(u_new - u) <= rel_tol * std::fabs(u_new);
        u = u_new;
        if (done) break;
    }
    // the iteration used the batch's vectors: its state must be set again
    BSG_CUDA(cudaMemsetAsync(h->X, 0, (size_t)c * h->Bp * sizeof(float), s));
    BSG_CUDA(cudaMemsetAsync(h->Xhat, 0, (size_t)c * h->Bp * sizeof(float), s));
    for (float *p : {h->R[0], h->R[1]}) BSG_CUDA(cudaMemsetAsync(p, 0, (size_t)R * h->Bp * sizeof(float), s));
    BSG_CUDA(cudaStreamSynchronize(s));
    h->has_data = false;
    if (u_max) *u_max = u;
    if (iters) *iters = std::min(it, max_iters);
    return BSGDTV_OK;
}

int bsgdtv_batch_project(bsgdtv_batch_t h, const float *x, float *y) {
    BSG_TRACE();
    if (!h || !x || !y) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    BSG_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const int64_t c = h->cols, R = h->rows;
    // x (planar) -> X (interleaved); R[0] = 0 stands for y; R[1] = 0 - A x
    BSG_CUDA(cudaMemcpyAsync(h->Xp, x, (size_t)c * h->B * sizeof(float), cudaMemcpyDeviceToDevice, s));
    BSG_CUDA(launch_transpose(h->Xp, h->X, c, h->B, h->Bp, false, s));
    BSG_CUDA(cudaMemsetAsync(h->R[0], 0, (size_t)R * h->Bp * sizeof(float), s));
    if (h->matrix_free)
        BSG_CUDA(launch_mf_pass(true, h->Bp, h->mfg, h->X, h->R[0], h->R[1], 0.f, s));
    else
        BSG_CUDA(launch_pass<true>(h->fmt, h->lpn, h->op_r, h->X, h->R[0], h->R[1], R, h->Bp, 0.f, s));
    BSG_CUDA(launch_transpose(h->R[1], y, R, h->B, h->Bp, true, s));
    const int64_t n = R * h->B;
    negate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, n);
    add_launches(1);
    BSG_CUDA(cudaGetLastError());
    // the projection used the batch's vectors: its state must be set again
    BSG_CUDA(cudaMemsetAsync(h->X, 0, (size_t)c * h->Bp * sizeof(float), s));
    for (float *p : {h->R[0], h->R[1]}) BSG_CUDA(cudaMemsetAsync(p, 0, (size_t)R * h->Bp * sizeof(float), s));
    BSG_CUDA(cudaStreamSynchronize(s));
    h->has_data = false;
    return BSGDTV_OK;
}

int bsgdtv_batch_autotune(bsgdtv_batch_t h, int fgp_iters, int epochs_per_trial, int *fgp_chunk,
                          int *fgp_group, double *epoch_ms) {
    BSG_TRACE();
    if (!h || fgp_iters < 0 || epochs_per_trial < 1)
        return fail(BSGDTV_ERR_INVALID_ARG, "need fgp_iters >= 0 and epochs_per_trial >= 1");
    if (!h->has_data) return fail(BSGDTV_ERR_STATE, "autotune before set_data");
    BSG_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    const size_t xb = (size_t)h->cols * h->Bp * sizeof(float), rb = (size_t)h->rows * h->Bp * sizeof(float);
    // the trials run real epochs: keep x^k, r^{k-1} (and r^k's buffer) to restore after each
    if (!h->save_x) {
        BSG_CHECK(balloc(h, &h->save_x, xb / sizeof(float)));
        BSG_CHECK(balloc(h, &h->save_r[0], rb / sizeof(float)));
        BSG_CHECK(balloc(h, &h->save_r[1], rb / sizeof(float)));
    }
    float *sx = h->save_x, *sr0 = h->save_r[0], *sr1 = h->save_r[1];
    BSG_CUDA(cudaMemcpyAsync(sx, h->X, xb, cudaMemcpyDeviceToDevice, s));
    BSG_CUDA(cudaMemcpyAsync(sr0, h->R[0], rb, cudaMemcpyDeviceToDevice, s));
    BSG_CUDA(cudaMemcpyAsync(sr1, h->R[1], rb, cudaMemcpyDeviceToDevice, s));
    const int cur = h->cur;
    const int64_t epoch = h->epoch;
    auto restore = [&]() -> int {
        BSG_CUDA(cudaMemcpyAsync(h->X, sx, xb, cudaMemcpyDeviceToDevice, s));
        BSG_CUDA(cudaMemcpyAsync(h->R[0], sr0, rb, cudaMemcpyDeviceToDevice, s));
        BSG_CUDA(cudaMemcpyAsync(h->R[1], sr1, rb, cudaMemcpyDeviceToDevice, s));
        h->cur = cur;
        h->epoch = epoch;
        return BSGDTV_OK;
    };
    // lanes per nonzero of each pass: the rule's count (one chunk of 4 * LPN
    // slices = all of them) and fewer lanes covering the slices in 2 or 4
    // chunks (more nonzeros per warp step, the nonzeros reread per chunk);
    // each pass's product time decides, the other pass kept at its choice
    if (h->lpn < 32 && !h->matrix_free) {
        for (int pass = 0; pass < 2; ++pass) {
            int best_l = h->lpn;
            double best_pk = 1e300;
            for (int l = h->lpn; l >= std::max(2, h->lpn / 4); l /= 2) {
                (pass == 0 ? h->lpn_row : h->lpn_col) = l;
                bdrop_graphs(h);
                BSG_CHECK(bsgdtv_batch_run(h, 1, fgp_iters));
                double pk = 0.0, ep = 0.0;
                BSG_CHECK(bsgdtv_batch_run_timed(h, epochs_per_trial, fgp_iters, &pk, &ep));
                BSG_CHECK(restore());
                if (pk < best_pk * 0.99) {   // fewer lanes only when measurably faster
                    best_pk = pk;
                    best_l = l;
                }
            }
            (pass == 0 ? h->lpn_row : h->lpn_col) = best_l;
        }
    }
    // slices per FGP launch group: half, once and twice the L2-budget size, all
    const int per = fgp_group_by_budget(h);
    std::vector<int> groups;
    for (int g : {std::max(1, per / 2), per, 2 * per, h->B}) {
        g = std::min(g, h->B);
        if (std::find(groups.begin(), groups.end(), g) == groups.end()) groups.push_back(g);
    }
    int best = h->fgp_chunk, best_g = h->fgp_group;
    double best_ms = 1e300;
    for (int g : groups)
        for (int chunk : kFgpChunkChoices) {
            h->fgp_chunk = chunk;
            h->fgp_group = g;
            bdrop_graphs(h);
            BSG_CHECK(bsgdtv_batch_run(h, 1, fgp_iters));   // builds the graphs, warms up
            double pk = 0.0, ep = 0.0;
            BSG_CHECK(bsgdtv_batch_run_timed(h, epochs_per_trial, fgp_iters, &pk, &ep));
            BSG_CHECK(restore());
            if (ep < best_ms) {
                best_ms = ep;
                best = chunk;
                best_g = g;
            }
        }
    h->fgp_chunk = best;
    h->fgp_group = best_g;
    bdrop_graphs(h);
    BSG_CUDA(cudaStreamSynchronize(s));
    if (fgp_chunk) *fgp_chunk = best;
    if (fgp_group) *fgp_group = best_g > 0 ? best_g : per;
    if (epoch_ms) *epoch_ms = best_ms / epochs_per_trial;
    return BSGDTV_OK;
}

int bsgdtv_batch_get_tuning(bsgdtv_batch_t h, int *fgp_chunk, int *fgp_group, int *lanes_row,
                            int *lanes_col) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (fgp_chunk) *fgp_chunk = h->fgp_chunk;
    if (fgp_group) *fgp_group = h->fgp_group > 0 ? h->fgp_group : fgp_group_by_budget(h);
    if (lanes_row) *lanes_row = h->lpn_row ? h->lpn_row : h->lpn;
    if (lanes_col) *lanes_col = h->lpn_col ? h->lpn_col : h->lpn;
    return BSGDTV_OK;
}

int bsgdtv_batch_set_pass_lanes(bsgdtv_batch_t h, int lanes_row, int lanes_col) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    auto ok = [&](int l) {
        return l == 0 || l == h->lpn ||
               (l >= 2 && l < h->lpn && (l & (l - 1)) == 0 && h->lpn < 32);
    };
    if (!ok(lanes_row) || !ok(lanes_col))
        return fail(BSGDTV_ERR_INVALID_ARG,
                    "lanes: 0, the batch's lanes per nonzero, or a smaller power of two >= 2");
    h->lpn_row = lanes_row;
    h->lpn_col = lanes_col;
    bdrop_graphs(h);
    return BSGDTV_OK;
}

int bsgdtv_batch_set_tuning(bsgdtv_batch_t h, int fgp_chunk, int fgp_group) {
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (fgp_chunk < 0 || fgp_chunk > fgpk::kMaxChunk || fgp_group < 0)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 0 <= fgp_chunk <= 8 and fgp_group >= 0");
    const int chunk = fgp_chunk > 0 ? fgp_chunk : kBatchFgpChunk;
    if (chunk != h->fgp_chunk || fgp_group != h->fgp_group) {
        BSG_CUDA(cudaSetDevice(h->device));
        BSG_CUDA(cudaStreamSynchronize(h->stream));
        h->fgp_chunk = chunk;
        h->fgp_group = fgp_group;
        bdrop_graphs(h);
    }
    return BSGDTV_OK;
}

int bsgdtv_batch_get_slice_x(bsgdtv_batch_t h, int b, float *x, int out_on_device) {
    BSG_TRACE();
    if (!h || !x) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (b < 0 || b >= h->B) return fail(BSGDTV_ERR_INVALID_ARG, "slice index out of range");
    BSG_CUDA(cudaSetDevice(h->device));
    const int64_t c = h->cols;
    slice_gather_kernel<<<(unsigned)((c + 255) / 256), 256, 0, h->stream>>>(h->X, h->ystage, c, h->Bp, b);
    add_launches(1);
    BSG_CUDA(cudaGetLastError());
    BSG_CUDA(cudaMemcpyAsync(x, h->ystage, (size_t)c * sizeof(float),
                             out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             h->stream));
    if (!out_on_device) BSG_CUDA(cudaStreamSynchronize(h->stream));
    return BSGDTV_OK;
}

}  // extern "C"

// ------------------------------------------------- packed batches
// Several geometries' batches (parts) whose epochs run together: each stage
// of an epoch (row pass, column pass, the transposes around the prox and
// every FGP launch) is one kernel launch over all parts, captured in one
// graph per parity of the residual double buffer.
struct bsgdtv_packed_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<bsgdtv_batch_t> parts;   // one batch per operator, on `stream`
    std::vector<bool> part_data;         // set_part called for the part
    int fmt = BSGDTV_FMT_F32_I32, B = 0, Bp = 0, lpn = 1;
    int fgp_chunk = bsgdtv::kBatchFgpChunk;
    float *mom = nullptr;
    int mom_len = 0;
    int cur = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_fgp_iters = -1;
    bool graph_prox = false;
    int64_t graph_kernels = 0;
};

namespace {

void pdrop_graphs(bsgdtv_packed_ctx *h) {
    for (auto &g : h->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    h->graph_fgp_iters = -1;
}

bool packed_prox(const bsgdtv_packed_ctx *h, int fgp_iters) {
    if (fgp_iters <= 0) return false;
    for (bsgdtv_batch_t p : h->parts)
        if (any_prox(p, fgp_iters)) return true;
    return false;
}

// One epoch of every part: reads R[par], writes R[1 - par] of each.
int penqueue_epoch(bsgdtv_packed_ctx *h, int par, int fgp_iters, cudaStream_t s) {
    const int n = (int)h->parts.size();
    const bool prox = packed_prox(h, fgp_iters);
    if (h->parts[0]->served) BSG_CHECK(enqueue_serve_prologue(h->parts.data(), n, par, s));
    PassPart rowp[kMaxPassParts], colp[kMaxPassParts];
    TransPart tin[kMaxTransParts], tout[kMaxTransParts];
    fgpk::FgpImages img[fgpk::kMaxFgpParts];
    for (int k = 0; k < n; ++k) {
        const bsgdtv_batch_ctx *p = h->parts[k];
        rowp[k] = {p->op_r, p->X, p->Y, p->R[1 - par], p->rows, 0.f, 0};
        colp[k] = {p->op_c, p->R[par], p->X, prox ? p->Xhat : p->X, p->cols, (float)p->mu, 0};
        tin[k] = {p->Xhat, p->Xhp, p->cols, 0};
        tout[k] = {p->Xp, p->X, p->cols, 0};
        img[k] = {p->Xhp, p->Xp, p->tau, 1.f, fgp_scratch_planes(p->fgp, (int64_t)p->B * p->cols),
                  p->cols, p->img_h, p->img_w, p->B};
    }
    // r^k = y - A x^k for every part (reads x before the column pass updates it)
    BSG_CUDA(launch_pass_parts<true>(h->fmt, h->lpn, rowp, n, h->Bp, s));
    // x^ = x^k + mu_part * 2 A^T r^{k-1}
    BSG_CUDA(launch_pass_parts<false>(h->fmt, h->lpn, colp, n, h->Bp, s));
    if (prox) {
        BSG_CUDA(launch_transpose_parts(tin, n, h->B, h->Bp, true, s));
        // the prox over groups of images whose fields (b and both dual sets,
        // 36 bytes per pixel) fit about half of the L2, so consecutive chunk
        // launches of a group find them there; a group may span parts
        fgpk::FgpImages grp[fgpk::kMaxFgpParts];
        int ng = 0;
        int64_t used = 0;
        for (int k = 0; k < n; ++k) {
            const bsgdtv_batch_ctx *p = h->parts[k];
            const int64_t per = 36 * p->cols;
            for (int b0 = 0; b0 < p->B;) {
                if (ng == fgpk::kMaxFgpParts || (ng > 0 && used + per > kFgpFieldBudget)) {
                    BSG_CUDA(fgpk::launch_fgp_parts(grp, ng, fgp_iters, h->mom, s, false, h->fgp_chunk));
                    ng = 0;
                    used = 0;
                }
                const int fit = (int)std::max<int64_t>(1, (kFgpFieldBudget - used) / per);
                const int nb = std::min(p->B - b0, fit);
                fgpk::FgpImages q = img[k];
                q.b = img[k].b + (int64_t)b0 * p->cols;
                q.x = img[k].x + (int64_t)b0 * p->cols;
                q.tau_z = p->tau + b0;
                q.sc = fgp_scratch_planes(p->fgp, (int64_t)p->B * p->cols, (int64_t)b0 * p->cols);
                q.slices = nb;
                grp[ng++] = q;
                used += per * nb;
                b0 += nb;
            }
        }
        if (ng > 0) BSG_CUDA(fgpk::launch_fgp_parts(grp, ng, fgp_iters, h->mom, s, false, h->fgp_chunk));
        BSG_CUDA(launch_transpose_parts(tout, n, h->B, h->Bp, false, s));
    }
    return BSGDTV_OK;
}

int pbuild_graphs(bsgdtv_packed_ctx *h, int fgp_iters) {
    pdrop_graphs(h);
    if (fgp_iters > h->mom_len) {
        std::vector<float> m;
        fgp_momentum_host(fgp_iters, m);
        float *d = nullptr;
        BSG_CHECK(balloc(h->parts[0], &d, m.size()));   // freed with part 0
        BSG_CUDA(cudaMemcpy(d, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice));
        h->mom = d;
        h->mom_len = fgp_iters;
    }
    const int64_t before = bsgdtv_launch_count();
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        BSG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = penqueue_epoch(h, par, fgp_iters, h->cap_stream);
        const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc != BSGDTV_OK) {
            if (g) cudaGraphDestroy(g);
            add_launches(before - bsgdtv_launch_count());
            return rc;
        }
        if (e != cudaSuccess) return fail(BSGDTV_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&h->gexec[par], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess)
            return fail(BSGDTV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    const int64_t captured = bsgdtv_launch_count() - before;
    add_launches(-captured);
    h->graph_kernels = captured / 2;
    h->graph_fgp_iters = fgp_iters;
    h->graph_prox = packed_prox(h, fgp_iters);
    return BSGDTV_OK;
}

}  // namespace

namespace bsgdtv {

bsgdtv_batch_t packed_part(bsgdtv_packed_t h, int k) {
    return (h && k >= 0 && k < (int)h->parts.size()) ? h->parts[k] : nullptr;
}

int packed_serve_enable(bsgdtv_packed_t h, int k, ServeView *view, void *host_block) {
    if (!h || k < 0 || k >= (int)h->parts.size()) return fail(BSGDTV_ERR_INVALID_ARG, "part out of range");
    BSG_CHECK(batch_serve_enable(h->parts[k], view, host_block));
    pdrop_graphs(h);   // the epochs gain the scheduler
    return BSGDTV_OK;
}

}  // namespace bsgdtv

extern "C" {

int bsgdtv_packed_create(bsgdtv_packed_t *out, const bsgdtv_operator_t *ops, int n_parts, int slices,
                         void *stream) {
    BSG_TRACE();
    if (!out || !ops) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_parts < 1 || n_parts > kMaxPassParts)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= n_parts <= 8");
    for (int k = 0; k < n_parts; ++k) {
        if (!ops[k]) return fail(BSGDTV_ERR_INVALID_ARG, "null operator");
        if (ops[k]->fmt != ops[0]->fmt) return fail(BSGDTV_ERR_INVALID_ARG, "parts must share one weight format");
    }
    std::unique_ptr<bsgdtv_packed_ctx> h(new (std::nothrow) bsgdtv_packed_ctx());
    if (!h) return fail(BSGDTV_ERR_OOM, "host allocation");
    BSG_CUDA(cudaGetDevice(&h->device));
    h->stream = (cudaStream_t)stream;
    h->fmt = ops[0]->fmt;
    h->B = slices;
    bsgdtv_packed_ctx *hp = h.get();
    auto cleanup = [&](int rc) {
        bsgdtv_packed_destroy(h.release());
        return rc;
    };
    BSG_CUDA(cudaStreamCreateWithFlags(&hp->cap_stream, cudaStreamNonBlocking));
    for (int k = 0; k < n_parts; ++k) {
        bsgdtv_batch_t b = nullptr;
        const int rc = bsgdtv_batch_create_from_operator(&b, ops[k], slices, stream);
        if (rc != BSGDTV_OK) return cleanup(rc);
        hp->parts.push_back(b);
        hp->part_data.push_back(false);
    }
    hp->Bp = hp->parts[0]->Bp;
    hp->lpn = hp->parts[0]->lpn;
    *out = h.release();
    return BSGDTV_OK;
}

void bsgdtv_packed_destroy(bsgdtv_packed_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    pdrop_graphs(h);
    for (bsgdtv_batch_t p : h->parts) bsgdtv_batch_destroy(p);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

int bsgdtv_packed_set_part(bsgdtv_packed_t h, int part, const float *y, int y_on_device,
                           const double *lambdas, double mu) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (part < 0 || part >= (int)h->parts.size()) return fail(BSGDTV_ERR_INVALID_ARG, "part out of range");
    h->part_data[part] = false;
    BSG_CHECK(bsgdtv_batch_set_data(h->parts[part], y, y_on_device, lambdas, mu));
    bsgdtv_batch_ctx *p = h->parts[part];
    // the packed epochs read r^{k-1} from R[cur] of every part
    if (h->cur != p->cur) {
        BSG_CUDA(cudaMemcpyAsync(p->R[h->cur], p->R[p->cur], (size_t)p->rows * p->Bp * sizeof(float),
                                 cudaMemcpyDeviceToDevice, h->stream));
        BSG_CUDA(cudaStreamSynchronize(h->stream));
        p->cur = h->cur;
    }
    pdrop_graphs(h);   // mu and the weights are baked into the epochs
    h->part_data[part] = true;
    return BSGDTV_OK;
}

int bsgdtv_packed_run(bsgdtv_packed_t h, int epochs, int fgp_iters) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    for (bool d : h->part_data)
        if (!d) return fail(BSGDTV_ERR_STATE, "run before every part has data");
    if (epochs < 0 || fgp_iters < 0) return fail(BSGDTV_ERR_INVALID_ARG, "negative epochs / fgp_iters");
    if (epochs == 0) return BSGDTV_OK;
    BSG_CUDA(cudaSetDevice(h->device));
    if (!h->gexec[0] || h->graph_fgp_iters != fgp_iters) BSG_CHECK(pbuild_graphs(h, fgp_iters));
    for (int e = 0; e < epochs; ++e) {
        BSG_CUDA(cudaGraphLaunch(h->gexec[h->cur], h->stream));
        add_launches(h->graph_kernels);
        h->cur ^= 1;
        for (bsgdtv_batch_t p : h->parts) {
            p->cur = h->cur;
            p->epoch++;
        }
    }
    return BSGDTV_OK;
}

int bsgdtv_packed_get_x(bsgdtv_packed_t h, int part, float *x, int out_on_device) {
    BSG_TRACE();
    if (!h) return fail(BSGDTV_ERR_INVALID_ARG, "null handle");
    if (part < 0 || part >= (int)h->parts.size()) return fail(BSGDTV_ERR_INVALID_ARG, "part out of range");
    return bsgdtv_batch_get_x(h->parts[part], x, out_on_device);
}

int bsgdtv_packed_launches_per_epoch(bsgdtv_packed_t h, int fgp_iters, int64_t *launches) {
    if (!h || !launches) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    for (bool d : h->part_data)
        if (!d) return fail(BSGDTV_ERR_STATE, "every part needs data first");
    BSG_CUDA(cudaSetDevice(h->device));
    if (!h->gexec[0] || h->graph_fgp_iters != fgp_iters) BSG_CHECK(pbuild_graphs(h, fgp_iters));
    *launches = h->graph_kernels;
    return BSGDTV_OK;
}

}  // extern "C"
