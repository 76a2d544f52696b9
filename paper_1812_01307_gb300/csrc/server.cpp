// Continuous-batching reconstruction server.
//
// Requests (projections y of a registered geometry, a TV weight lambda and an
// epoch budget) arrive at any time.  Each geometry owns one or more batch
// groups: a batch handle (one shared A, `slots` slices) in served mode on its
// own stream.  A geometry's A is stored once; a new group is created only
// while the device bytes of all groups stay within the HBM budget, and an
// idle group of another geometry is released to make room.
//
// Admission, epoch counting and retirement run on the device.  Every epoch of
// a served group starts with a slot scheduler kernel that reads the group's
// mailboxes in host-mapped memory: the worker thread admits a request by
// copying y into the slot's pinned staging row and posting (tau, epochs, a
// new sequence number) in the slot's mailbox, at any time, also while the
// group is running; the device resets the slot at the next epoch boundary,
// counts the request's epochs, and after the last one writes x into the
// slot's pinned result row and publishes a completion record, which the
// worker picks up (x in host memory: the end of the request's latency) to
// free the slot.  So requests join and leave at epoch boundaries while the
// worker only keeps each busy group's stream fed with runs of epochs (at
// most two runs in flight per group).  Groups of different geometries run
// concurrently on their streams.  A slice's arithmetic never depends on the
// other slots, so a request's result is the same alone and in any mix.
//
// An armed epoch (bsgdtv_server_arm) is launched on an idle group before any
// request is there: its scheduler waits on the device, polling the
// mailboxes, for at most the requested time; a request submitted meanwhile
// starts at once without a host launch, and a wait that runs out ends the
// epoch with a timeout status.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "bsgdtv_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

constexpr int kMinSlots = 4;   // smallest group the server makes on demand

struct Request {
    int64_t id = 0;
    int geom = 0;
    std::vector<float> y;
    double lambda = 0.0;
    int epochs = 0;
    int remaining = 0;
    int state = kQueued;
    bool cancel = false;   // running, cancelled: the slot is freed after the tick
    int error = BSGDTV_OK;
    std::string message;
    std::vector<float> x;
    Clock::time_point t_submit, t_admit, t_done;
};

constexpr int kMaxRuns = 2;     // runs of epochs in flight per group
constexpr int kMaxParts = 8;    // geometries packed into one group at most

// One geometry's slots inside a group (a part of the group's packed batch).
struct Part {
    int geom = 0;
    bsgdtv::ServeView view = {};     // host-mapped mailboxes, records, staging rows
    void *pinned = nullptr;          // the block behind view (from the server's pool)
    std::vector<int64_t> slot_req;   // request id per slot, -1 = free
    std::vector<int> slot_seq;       // last sequence number posted per slot
    std::vector<int64_t> slot_end;   // epochs the group must have run to retire the slot's
                                     // request (known once the device picked it up; -1 before)
    int arm_seq = 0;                 // last armed epoch's sequence number (this part's control)
};

// A group: a packed batch of one or more geometries' parts with a common slot
// count, on its own stream; every epoch stage is one launch over all parts.
struct Group {
    bsgdtv_packed_t packed = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<Part> parts;
    int slots = 0;
    cudaEvent_t run_ev[kMaxRuns] = {};
    int run_len[kMaxRuns] = {};
    int runs = 0;                    // runs in flight (run_ev[0 .. runs) in launch order)
    int64_t enq = 0;                 // epochs enqueued on the group since it was made
    int armed_part = -1;             // part whose armed wait has not been reported yet
    int64_t bytes = 0;
    int64_t launches_per_epoch = 0;
    Clock::time_point idle_since;
    Part *part_of(int geom) {
        for (Part &p : parts)
            if (p.geom == geom) return &p;
        return nullptr;
    }
};

struct Geometry {
    int64_t rows = 0, cols = 0;
    int img_h = 0, img_w = 0;
    bsgdtv_operator_t op = nullptr;   // A on the device, shared by every group
    int64_t op_bytes = 0;
    int format = BSGDTV_FMT_F32_I32;
    int slots = 1;       // slots of the largest group
    int min_slots = 1;   // slots of the smallest group
    double mu = 0.0;
    int64_t nnz = 0;
    int64_t queued = 0;  // requests of this geometry waiting for a slot
    // device bytes of a group: its vectors (A is the geometry's, counted once)
    int64_t bytes_for(int slots_g) const {
        return bsgdtv_batch_device_bytes(rows, cols, 0, slots_g, format);
    }
};

}  // namespace

struct bsgdtv_server_ctx {
    int device = 0;
    int64_t budget = 0;
    int fgp_iters = 0;
    int max_tick = 1;
    std::mutex mu;
    std::condition_variable cv_work;   // worker: new request or stop
    std::condition_variable cv_done;   // waiters: a request finished
    std::vector<std::unique_ptr<Geometry>> geoms;
    std::vector<std::unique_ptr<Group>> groups;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<int64_t> queue;
    int64_t next_id = 1;
    int64_t hbm_used = 0;
    bool stop = false;
    bool wake = false;   // a cancel for the worker to reap
    std::thread worker;
    // armed epochs asked for by bsgdtv_server_arm: geometry, wait, result
    struct Arm {
        int geom = 0;
        long long wait_ns = 0;
        bool launched = false, finished = false;
        int result = BSGDTV_OK;
        Group *group = nullptr;
    };
    std::vector<Arm *> arms;
    // mapped pinned host blocks of served groups, kept for reuse: pinning
    // memory costs milliseconds per group, groups come and go often
    struct Pinned {
        void *p = nullptr;
        size_t bytes = 0;
        bool used = false;
    };
    std::vector<Pinned> pinned;
    // statistics
    // packing: a new group also takes other waiting geometries of the same
    // slot count whose operators are within cost_ratio (nonzeros) of each
    // other, up to max_parts geometries
    bool hold = false;   // admissions held (bsgdtv_server_hold)
    int pack_max_parts = 1;
    double pack_cost_ratio = 4.0;
    bool priority_by_size = true;   // smaller geometries' groups on higher-priority streams
    int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, ticks = 0, epochs_run = 0, groups_made = 0,
            groups_freed = 0, max_running = 0, slice_epochs = 0, wait_timeouts = 0, armed_epochs = 0,
            packed_groups = 0, max_parts = 0, packed_launches = 0;
};

namespace {

using bsgdtv::fail;

void finish_failed(bsgdtv_server_ctx *s, Request &r, int code, const std::string &msg) {
    r.state = kFailed;
    r.error = code;
    r.message = msg;
    r.t_done = Clock::now();
    s->failed++;
}

bool finished(const Request &r) {
    return r.state == kDone || r.state == kFailed || r.state == kCancelled;
}

// Slot b of a part is free again (the device emptied it when it retired).
void free_slot(Part *p, int b) {
    p->slot_req[b] = -1;
    p->slot_end[b] = -1;
}

void finish_cancelled(bsgdtv_server_ctx *s, Request &r) {
    r.state = kCancelled;
    r.t_done = Clock::now();
    s->cancelled++;
}

// A mapped pinned block of at least `bytes` (a free one of at most twice
// that size is reused), or null.
void *pinned_acquire(bsgdtv_server_ctx *s, size_t bytes) {
    for (auto &b : s->pinned)
        if (!b.used && b.bytes >= bytes && b.bytes <= 2 * bytes) {
            b.used = true;
            return b.p;
        }
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    s->pinned.push_back({p, bytes, true});
    return p;
}

void pinned_release(bsgdtv_server_ctx *s, void *p) {
    for (auto &b : s->pinned)
        if (b.p == p) b.used = false;
}

int destroy_group(bsgdtv_server_ctx *s, Group *g) {
    if (g->packed) bsgdtv_packed_destroy(g->packed);
    for (Part &p : g->parts)
        if (p.pinned) pinned_release(s, p.pinned);
    for (cudaEvent_t &ev : g->run_ev)
        if (ev) cudaEventDestroy(ev);
    if (g->stream) cudaStreamDestroy(g->stream);
    s->hbm_used -= g->bytes;
    s->groups_freed++;
    return BSGDTV_OK;
}

// Creates a group of the geometries `gis` with `slots` slots each (caller
// holds the lock).
int make_group(bsgdtv_server_ctx *s, const std::vector<int> &gis, int slots, Group **out) {
    std::unique_ptr<Group> g(new Group());
    g->slots = slots;
    int64_t bytes = 0;
    std::vector<bsgdtv_operator_t> ops;
    for (int gi : gis) {
        bytes += s->geoms[gi]->bytes_for(slots);
        ops.push_back(s->geoms[gi]->op);
    }
    g->bytes = bytes;
    // stream priority: one step up for every factor of 16 by which the
    // group's largest operator has fewer nonzeros than the largest registered
    // one, within the device's range.  The short kernels of much smaller
    // images are then scheduled ahead of the long ones of large images
    // whenever SMs free up (nothing is preempted), which costs the large ones
    // little: the small ones are a small share of the work.  Geometries within
    // a factor of 16 of each other share a priority.
    int prio = 0;
    if (s->priority_by_size) {
        int least = 0, greatest = 0;
        BSG_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        int64_t own = 1, top = 1;
        for (int gi : gis) own = std::max(own, s->geoms[gi]->nnz);
        for (const auto &G : s->geoms)
            if (G) top = std::max(top, G->nnz);
        int steps = 0;
        for (int64_t v = own; v * 16 <= top; v *= 16) ++steps;
        prio = std::max(greatest, least - steps);
    }
    BSG_CUDA(cudaStreamCreateWithPriority(&g->stream, cudaStreamNonBlocking, prio));
    int rc = BSGDTV_OK;
    for (cudaEvent_t &ev : g->run_ev)
        if (rc == BSGDTV_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            rc = fail(BSGDTV_ERR_CUDA, "event creation");
    if (rc == BSGDTV_OK)
        rc = bsgdtv_packed_create(&g->packed, ops.data(), (int)ops.size(), slots, g->stream);
    g->parts.resize(gis.size());
    for (size_t k = 0; k < gis.size() && rc == BSGDTV_OK; ++k) {
        const Geometry &G = *s->geoms[gis[k]];
        Part &p = g->parts[k];
        p.geom = gis[k];
        bsgdtv::batch_keep_prox(bsgdtv::packed_part(g->packed, (int)k), s->fgp_iters > 0);
        std::vector<float> zeros((size_t)G.rows * slots, 0.f);
        std::vector<double> lam((size_t)slots, 0.0);
        rc = bsgdtv_packed_set_part(g->packed, (int)k, zeros.data(), 0, lam.data(), G.mu);
        if (rc == BSGDTV_OK) {
            p.pinned = pinned_acquire(s, bsgdtv::batch_serve_host_bytes(slots, G.rows, G.cols));
            rc = p.pinned ? bsgdtv::packed_serve_enable(g->packed, (int)k, &p.view, p.pinned)
                          : fail(BSGDTV_ERR_OOM, "pinned host memory for a served group");
        }
        p.slot_req.assign(slots, -1);
        p.slot_seq.assign(slots, 0);
        p.slot_end.assign(slots, -1);
    }
    if (rc == BSGDTV_OK)
        rc = bsgdtv_packed_launches_per_epoch(g->packed, s->fgp_iters, &g->launches_per_epoch);
    if (rc != BSGDTV_OK) {
        if (g->packed) bsgdtv_packed_destroy(g->packed);
        for (Part &p : g->parts)
            if (p.pinned) pinned_release(s, p.pinned);
        for (cudaEvent_t &ev : g->run_ev)
            if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(g->stream);
        return rc;
    }
    g->idle_since = Clock::now();
    s->hbm_used += g->bytes;
    s->groups_made++;
    if (gis.size() > 1) {
        s->packed_groups++;
        s->packed_launches = g->launches_per_epoch;
    }
    s->max_parts = std::max<int64_t>(s->max_parts, (int64_t)gis.size());
    *out = g.get();
    s->groups.push_back(std::move(g));
    return BSGDTV_OK;
}

bool group_idle(const Group *g) {
    if (g->runs > 0 || g->armed_part >= 0) return false;
    for (const Part &p : g->parts)
        for (int64_t id : p.slot_req)
            if (id >= 0) return false;
    return true;
}

int running_of(const bsgdtv_server_ctx *s, int gi) {
    int n = 0;
    for (auto &g : s->groups)
        for (const Part &p : g->parts)
            if (p.geom == gi)
                for (int64_t id : p.slot_req) n += id >= 0;
    return n;
}

bool has_free_slot(const bsgdtv_server_ctx *s, int gi) {
    for (auto &g : s->groups)
        for (const Part &p : g->parts)
            if (p.geom == gi)
                for (int64_t id : p.slot_req)
                    if (id < 0) return true;
    return false;
}

// Slots of a new group for geometry gi: a power of two between min_slots
// and slots covering the geometry's demand (requests waiting plus running).
int demand_slots(const bsgdtv_server_ctx *s, int gi) {
    const Geometry &G = *s->geoms[gi];
    int slots = G.min_slots;
    const int64_t demand = G.queued + running_of(s, gi);
    while (slots < G.slots && slots < demand) slots *= 2;
    return std::min(slots, G.slots);
}

// Finds or makes a free slot for geometry gi.  Returns false if none can be
// had now (the request waits); sets *fatal if the geometry can never fit.
bool find_slot(bsgdtv_server_ctx *s, int gi, Group **gout, int *part, int *slot, int *fatal) {
    *fatal = BSGDTV_OK;
    // any free slot of this geometry, running group or not (admission is
    // posted to the slot's mailbox; an armed group first)
    Group *best = nullptr;
    int best_part = -1, best_slot = -1;
    for (auto &g : s->groups)
        for (int k = 0; k < (int)g->parts.size(); ++k) {
            const Part &p = g->parts[k];
            if (p.geom != gi) continue;
            for (int b = 0; b < (int)p.slot_req.size(); ++b)
                if (p.slot_req[b] < 0) {
                    const bool armed = g->armed_part == k;
                    if (!best || (armed && best->armed_part < 0)) {
                        best = g.get();
                        best_part = k;
                        best_slot = b;
                    }
                    break;
                }
        }
    if (best) {
        *gout = best;
        *part = best_part;
        *slot = best_slot;
        return true;
    }
    const Geometry &G = *s->geoms[gi];
    if (G.op_bytes + G.bytes_for(G.min_slots) > s->budget) {
        *fatal = BSGDTV_ERR_OOM;
        return false;
    }
    // every group of this geometry is full: a new group sized by the
    // geometry's demand (requests waiting plus running), so light load gets
    // small groups with short epochs (low latency) and sustained load large
    // ones that read A once for many slices (throughput); shrunk if the
    // budget cannot hold it.  With packing, other geometries with requests
    // waiting and no free slot, the same slot count and operators of a
    // similar size join it as parts (one launch per epoch stage for all).
    int slots = demand_slots(s, gi);
    std::vector<int> gis = {gi};
    if (s->pack_max_parts > 1) {
        for (int h = 0; h < (int)s->geoms.size() && (int)gis.size() < s->pack_max_parts; ++h) {
            if (h == gi || !s->geoms[h] || s->geoms[h]->queued <= 0 || has_free_slot(s, h)) continue;
            const Geometry &H = *s->geoms[h];
            if (H.format != G.format || demand_slots(s, h) != slots) continue;
            const double r = (double)std::max(H.nnz, G.nnz) / (double)std::max<int64_t>(1, std::min(H.nnz, G.nnz));
            if (r <= s->pack_cost_ratio) gis.push_back(h);
        }
    }
    auto bytes_of = [&](int sl) {
        int64_t b = 0;
        for (int k : gis) b += s->geoms[k]->bytes_for(sl);
        return b;
    };
    while (slots > G.min_slots && s->hbm_used + bytes_of(slots) > s->budget &&
           !std::any_of(s->groups.begin(), s->groups.end(), [&](const std::unique_ptr<Group> &p) {
               return !p->part_of(gi) && group_idle(p.get());
           }))
        slots = std::max(G.min_slots, slots / 2);
    while (gis.size() > 1 && s->hbm_used + bytes_of(slots) > s->budget) gis.pop_back();
    const int64_t need = bytes_of(slots);
    // release idle groups without this geometry (oldest first) until it fits
    while (s->hbm_used + need > s->budget) {
        Group *victim = nullptr;
        for (auto &g : s->groups)
            if (!g->part_of(gi) && group_idle(g.get()) && (!victim || g->idle_since < victim->idle_since))
                victim = g.get();
        if (!victim) return false;
        destroy_group(s, victim);
        s->groups.erase(std::find_if(s->groups.begin(), s->groups.end(),
                                     [&](const std::unique_ptr<Group> &p) { return p.get() == victim; }));
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || (int64_t)free_b < need + (need >> 5)) {
        cudaGetLastError();
        return false;
    }
    Group *g = nullptr;
    const int rc = make_group(s, gis, slots, &g);
    if (rc != BSGDTV_OK) {
        *fatal = rc;
        return false;
    }
    *gout = g;
    *part = 0;
    *slot = 0;
    return true;
}

void admit(bsgdtv_server_ctx *s) {
    if (s->hold) return;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request &r = *s->reqs[*it];
        Group *g = nullptr;
        int part = -1, slot = -1, fatal = BSGDTV_OK;
        if (!find_slot(s, r.geom, &g, &part, &slot, &fatal)) {
            if (fatal != BSGDTV_OK) {
                finish_failed(s, r, fatal, fatal == BSGDTV_ERR_OOM
                                               ? "a group of this geometry exceeds the HBM budget"
                                               : std::string("group creation: ") + bsgdtv_last_error());
                s->geoms[r.geom]->queued--;
                it = s->queue.erase(it);
                s->cv_done.notify_all();
            } else {
                ++it;
            }
            continue;
        }
        // y was checked at submit.  Post the admission: staging row and
        // fields first, then the new sequence number (release)
        const Geometry &G = *s->geoms[r.geom];
        Part &pt = g->parts[part];
        bsgdtv::ServeSlot &m = pt.view.mb[slot];
        std::memcpy(pt.view.ypin + (size_t)slot * G.rows, r.y.data(), (size_t)G.rows * sizeof(float));
        m.epochs = r.epochs;
        m.tau = (float)(G.mu * r.lambda);
        const int seq = ++pt.slot_seq[slot];
        __atomic_store_n(&m.seq, seq, __ATOMIC_RELEASE);
        pt.slot_req[slot] = r.id;
        pt.slot_end[slot] = -1;   // set when the device reports the pickup
        r.state = kRunning;
        r.remaining = r.epochs;
        r.t_admit = Clock::now();
        std::vector<float>().swap(r.y);
        s->geoms[r.geom]->queued--;
        it = s->queue.erase(it);
    }
}

// Keeps every group with occupied slots fed with runs of epochs (at most
// kMaxRuns in flight), each as long as the longest remaining budget there
// (capped at max_tick), and launches the armed epochs asked for.
void feed_groups(bsgdtv_server_ctx *s) {
    int64_t running = 0;
    for (auto &g : s->groups) {
        // epochs still to enqueue: exact for requests the device has picked
        // up (their end epoch is known), one for the others while nothing is
        // in flight (so the device picks them up)
        int64_t need = 0;
        bool occupied = false;
        for (Part &p : g->parts)
            for (size_t b = 0; b < p.slot_req.size(); ++b)
                if (p.slot_req[b] >= 0) {
                    running++;
                    occupied = true;
                    if (p.slot_end[b] >= 0) need = std::max(need, p.slot_end[b] - g->enq);
                }
        if (occupied && need <= 0 && g->runs == 0) need = 1;
        while (need > 0 && g->runs < kMaxRuns) {
            const int len = (int)std::max<int64_t>(1, std::min<int64_t>(need, s->max_tick));
            int rc = bsgdtv_packed_run(g->packed, len, s->fgp_iters);
            if (rc == BSGDTV_OK && cudaEventRecord(g->run_ev[g->runs], g->stream) != cudaSuccess)
                rc = BSGDTV_ERR_CUDA;
            if (rc != BSGDTV_OK) {
                const std::string msg = std::string("run: ") + bsgdtv_last_error();
                for (Part &p : g->parts)
                    for (int64_t &id : p.slot_req)
                        if (id >= 0) {
                            finish_failed(s, *s->reqs[id], rc, msg);
                            id = -1;
                        }
                s->cv_done.notify_all();
                break;
            }
            g->run_len[g->runs++] = len;
            g->enq += len;
            s->ticks++;
            s->epochs_run += len;
            need -= len;
        }
    }
    s->max_running = std::max(s->max_running, running);
    // armed epochs: one epoch on an idle group of the geometry (made if the
    // budget allows)
    for (bsgdtv_server_ctx::Arm *a : s->arms) {
        if (a->launched) continue;
        Group *g = nullptr;
        for (auto &p : s->groups)
            if (p->part_of(a->geom) && group_idle(p.get())) {
                g = p.get();
                break;
            }
        if (!g) {
            int part = -1, slot = -1, fatal = BSGDTV_OK;
            if (!find_slot(s, a->geom, &g, &part, &slot, &fatal) || !group_idle(g)) {
                if (fatal != BSGDTV_OK) {
                    a->launched = a->finished = true;
                    a->result = fatal;
                    s->cv_done.notify_all();
                }
                continue;
            }
        }
        int k = 0;
        while (g->parts[k].geom != a->geom) ++k;
        Part &p = g->parts[k];
        bsgdtv::ServeCtrl &c = *p.view.ctrl;
        c.wait_ns = a->wait_ns;
        p.arm_seq++;
        __atomic_store_n(&c.arm_seq, p.arm_seq, __ATOMIC_RELEASE);
        int rc = bsgdtv_packed_run(g->packed, 1, s->fgp_iters);
        if (rc == BSGDTV_OK && cudaEventRecord(g->run_ev[g->runs], g->stream) != cudaSuccess)
            rc = BSGDTV_ERR_CUDA;
        a->launched = true;
        if (rc != BSGDTV_OK) {
            a->finished = true;
            a->result = rc;
            s->cv_done.notify_all();
            continue;
        }
        g->run_len[g->runs++] = 1;
        g->enq += 1;
        g->armed_part = k;
        a->group = g;
        s->ticks++;
        s->epochs_run += 1;
        s->armed_epochs++;
    }
}

// Retires finished runs, picks up completion records (x copied from the
// slot's result row; the slot is free again), posts cancellations, and
// reports armed epochs whose device-side wait has ended.  Returns true if
// anything changed.
bool harvest(bsgdtv_server_ctx *s) {
    bool any = false;
    for (auto &g : s->groups) {
        // runs complete in launch order
        while (g->runs > 0) {
            const cudaError_t q = cudaEventQuery(g->run_ev[0]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) {
                cudaGetLastError();
                for (Part &p : g->parts)
                    for (int64_t &id : p.slot_req)
                        if (id >= 0) {
                            finish_failed(s, *s->reqs[id], BSGDTV_ERR_CUDA,
                                          std::string("run: ") + cudaGetErrorString(q));
                            id = -1;
                        }
            }
            // the oldest run is done: its event moves to the free end
            cudaEvent_t ev0 = g->run_ev[0];
            for (int k = 0; k + 1 < kMaxRuns; ++k) {
                g->run_ev[k] = g->run_ev[k + 1];
                g->run_len[k] = g->run_len[k + 1];
            }
            g->run_ev[kMaxRuns - 1] = ev0;
            g->runs--;
            any = true;
        }
        for (Part &p : g->parts) {
            const Geometry &G = *s->geoms[p.geom];
            for (int b = 0; b < (int)p.slot_req.size(); ++b) {
                const int64_t id = p.slot_req[b];
                if (id < 0) continue;
                Request &r = *s->reqs[id];
                const bsgdtv::ServeDone &d = p.view.done[b];
                if (p.slot_end[b] < 0 &&
                    __atomic_load_n(&d.picked_seq, __ATOMIC_ACQUIRE) == p.slot_seq[b])
                    // picked up at epoch e: runs epochs e .. e + E - 1, retired at e + E
                    p.slot_end[b] = (int64_t)d.picked_epoch + r.epochs + 1;
                if (__atomic_load_n(&d.seq, __ATOMIC_ACQUIRE) != p.slot_seq[b]) {
                    // still running: post a cancellation once
                    if (r.cancel && __atomic_load_n(&p.view.mb[b].cancel, __ATOMIC_RELAXED) != p.slot_seq[b])
                        __atomic_store_n(&p.view.mb[b].cancel, p.slot_seq[b], __ATOMIC_RELEASE);
                    continue;
                }
                const int ran = d.epochs_run;
                s->slice_epochs += ran;
                r.remaining = r.epochs - ran;
                if (r.cancel) {
                    finish_cancelled(s, r);
                } else {
                    try {
                        r.x.assign(p.view.xpin + (size_t)b * G.cols, p.view.xpin + (size_t)(b + 1) * G.cols);
                        r.state = kDone;
                        r.t_done = Clock::now();
                        s->completed++;
                    } catch (const std::bad_alloc &) {
                        finish_failed(s, r, BSGDTV_ERR_OOM, "host allocation for x");
                    }
                }
                free_slot(&p, b);
                any = true;
            }
        }
        if (g->armed_part >= 0) {
            const Part &p = g->parts[g->armed_part];
            if (__atomic_load_n(&p.view.ctrl->status_seq, __ATOMIC_ACQUIRE) == p.arm_seq) {
                const int timed_out = p.view.ctrl->status;
                g->armed_part = -1;
                if (timed_out) s->wait_timeouts++;
                for (bsgdtv_server_ctx::Arm *a : s->arms)
                    if (a->group == g.get() && !a->finished) {
                        a->finished = true;
                        a->result = timed_out ? BSGDTV_ERR_TIMEOUT : BSGDTV_OK;
                    }
                any = true;
            }
        }
        if (group_idle(g.get()) && any) g->idle_since = Clock::now();
    }
    if (any) s->cv_done.notify_all();
    return any;
}

void worker_main(bsgdtv_server_ctx *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        if (s->stop) break;
        harvest(s);
        admit(s);
        feed_groups(s);
        bool busy = false;
        for (auto &g : s->groups) busy = busy || g->runs > 0;
        if (!busy) {
            if (s->queue.empty()) {
                s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty() || s->wake; });
                s->wake = false;
            } else {
                // queued requests that cannot be placed yet and nothing running:
                // wait for a submit, a stop, or retry shortly (memory may free up)
                s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
            }
            continue;
        }
        // let submitters in while the device works, then poll again
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lock.lock();
    }
    // drain: wait for every group's work before the caller frees them
    for (auto &g : s->groups)
        if (g->stream) cudaStreamSynchronize(g->stream);
}

}  // namespace

extern "C" {

int bsgdtv_server_create(bsgdtv_server_t *out, int64_t hbm_budget_bytes, int fgp_iters,
                         int max_tick_epochs) {
    if (!out) return fail(BSGDTV_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || fgp_iters < 0 || max_tick_epochs < 1)
        return fail(BSGDTV_ERR_INVALID_ARG, "need hbm_budget_bytes > 0, fgp_iters >= 0, max_tick_epochs >= 1");
    std::unique_ptr<bsgdtv_server_ctx> s(new (std::nothrow) bsgdtv_server_ctx());
    if (!s) return fail(BSGDTV_ERR_OOM, "host allocation");
    BSG_CUDA(cudaGetDevice(&s->device));
    s->budget = hbm_budget_bytes;
    s->fgp_iters = fgp_iters;
    s->max_tick = max_tick_epochs;
    try {
        s->worker = std::thread(worker_main, s.get());
    } catch (...) {
        return fail(BSGDTV_ERR_OOM, "cannot start the worker thread");
    }
    *out = s.release();
    return BSGDTV_OK;
}

void bsgdtv_server_destroy(bsgdtv_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &g : s->groups) destroy_group(s, g.get());
    s->groups.clear();
    for (auto &G : s->geoms)
        if (G && G->op) bsgdtv_operator_destroy(G->op);
    for (auto &b : s->pinned) cudaFreeHost(b.p);
    s->cv_done.notify_all();
    delete s;
}

constexpr int kAutoSlotsMax = 32;
constexpr double kAutoSlotsBytes = 64.0 * 1024 * 1024;

int bsgdtv_server_add_geometry(bsgdtv_server_t s, int64_t rows, int64_t cols, int img_h, int img_w,
                               const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                               int format, int slots, double mu, int prewarm, int *geom_id) {
    if (!s || !geom_id || !row_ptr || !col_idx || !vals)
        return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (slots < 0 || slots > 4096 || !(mu > 0.0) || !std::isfinite(mu) || prewarm < 0)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 0 <= slots <= 4096, finite mu > 0, prewarm >= 0");
    if (slots == 0) {
        // the batch passes gather one slots-wide vector of x (row pass) or r
        // (column pass) per nonzero: the largest power of two up to 32 whose
        // vectors (slots x max(rows, cols) floats) stay within 64 MiB of L2
        // (at 1024 x 1024 a 32-slot group's gathers spill to HBM: 16 slots run
        // each slice's products about 10 % faster)
        slots = kAutoSlotsMax;
        while (slots > 1 && (double)slots * (double)std::max(rows, cols) * sizeof(float) > kAutoSlotsBytes)
            slots /= 2;
    }
    BSG_CHECK(bsgdtv::validate_image_csr(rows, cols, img_h, img_w, row_ptr, col_idx, vals));
    if (format != BSGDTV_FMT_F32_I32 && format != BSGDTV_FMT_F16_I16 && format != BSGDTV_FMT_BF16_I16)
        return fail(BSGDTV_ERR_INVALID_ARG, "batch formats: F32_I32, F16_I16, BF16_I16");
    BSG_CUDA(cudaSetDevice(s->device));
    std::unique_ptr<Geometry> G(new (std::nothrow) Geometry());
    if (!G) return fail(BSGDTV_ERR_OOM, "host allocation");
    const int64_t nnz = row_ptr[rows];
    G->rows = rows;
    G->cols = cols;
    G->img_h = img_h;
    G->img_w = img_w;
    G->format = format;
    G->slots = slots;
    G->min_slots = std::min(slots, kMinSlots);
    G->mu = mu;
    G->nnz = nnz;
    G->op_bytes = bsgdtv_batch_device_bytes(rows, cols, nnz, 1, format) -
                  bsgdtv_batch_device_bytes(rows, cols, 0, 1, format);
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t ops = 0;   // every registered A stays resident; groups can be released
    for (auto &g : s->geoms)
        if (g) ops += g->op_bytes;
    if (ops + G->op_bytes + G->bytes_for(G->min_slots) > s->budget)
        return fail(BSGDTV_ERR_OOM, "the geometries' A and one group exceed the HBM budget");
    while (s->hbm_used + G->op_bytes > s->budget) {   // make room: release idle groups
        auto it = std::find_if(s->groups.begin(), s->groups.end(),
                               [](const std::unique_ptr<Group> &p) { return group_idle(p.get()); });
        if (it == s->groups.end()) return fail(BSGDTV_ERR_OOM, "no idle group to release for this A");
        destroy_group(s, it->get());
        s->groups.erase(it);
    }
    // A goes to the device once, on a private stream; every group reads it
    cudaStream_t up = nullptr;
    BSG_CUDA(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
    const int rc_op = bsgdtv_operator_create_csr(&G->op, rows, cols, img_h, img_w, row_ptr, col_idx,
                                                 vals, format, up);
    cudaStreamDestroy(up);
    if (rc_op != BSGDTV_OK) return rc_op;
    s->hbm_used += G->op_bytes;
    const int gi = (int)s->geoms.size();
    s->geoms.push_back(std::move(G));
    // prewarm: as many groups as the budget holds now, up to `prewarm`
    for (int k = 0; k < prewarm && s->hbm_used + s->geoms[gi]->bytes_for(slots) <= s->budget; ++k) {
        Group *g = nullptr;
        const int rc = make_group(s, {gi}, slots, &g);
        if (rc != BSGDTV_OK) return rc;
    }
    *geom_id = gi;
    return BSGDTV_OK;
}

int bsgdtv_server_submit(bsgdtv_server_t s, int geom_id, const float *y, double lambda, int epochs,
                         int64_t *request_id) {
    if (!s || !y || !request_id) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || epochs < 1)
        return fail(BSGDTV_ERR_INVALID_ARG, "need finite lambda >= 0 and epochs >= 1");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(BSGDTV_ERR_OOM, "host allocation");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (geom_id < 0 || geom_id >= (int)s->geoms.size() || !s->geoms[geom_id])
            return fail(BSGDTV_ERR_INVALID_ARG, "unknown geometry");
        if (s->stop) return fail(BSGDTV_ERR_STATE, "server is stopping");
        const int64_t rows = s->geoms[geom_id]->rows;
        if (!bsgdtv::all_finite(y, rows)) return fail(BSGDTV_ERR_NONFINITE, "non-finite value in y");
        try {
            r->y.assign(y, y + rows);
        } catch (const std::bad_alloc &) {
            return fail(BSGDTV_ERR_OOM, "host allocation");
        }
        r->id = s->next_id++;
        r->geom = geom_id;
        r->lambda = lambda;
        r->epochs = epochs;
        r->t_submit = Clock::now();
        *request_id = r->id;
        s->queue.push_back(r->id);
        s->geoms[geom_id]->queued++;
        s->reqs[r->id] = std::move(r);
        s->submitted++;
    }
    s->cv_work.notify_all();
    return BSGDTV_OK;
}

int bsgdtv_server_poll(bsgdtv_server_t s, int64_t request_id, int *state) {
    if (!s || !state) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(BSGDTV_ERR_INVALID_ARG, "unknown request");
    *state = it->second->state;
    return BSGDTV_OK;
}

int bsgdtv_server_cancel(bsgdtv_server_t s, int64_t request_id) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->reqs.find(request_id);
        if (it == s->reqs.end()) return fail(BSGDTV_ERR_INVALID_ARG, "unknown request");
        Request &r = *it->second;
        if (finished(r)) return fail(BSGDTV_ERR_STATE, "request already ended");
        if (r.state == kQueued) {
            auto q = std::find(s->queue.begin(), s->queue.end(), r.id);
            if (q != s->queue.end()) s->queue.erase(q);
            s->geoms[r.geom]->queued--;
            std::vector<float>().swap(r.y);
            finish_cancelled(s, r);
            s->cv_done.notify_all();
            return BSGDTV_OK;
        }
        r.cancel = true;   // running: the worker posts it to the slot's mailbox
        s->wake = true;
    }
    s->cv_work.notify_all();
    return BSGDTV_OK;
}

int bsgdtv_server_wait(bsgdtv_server_t s, int64_t request_id, double timeout_s, float *x,
                       double *times) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(BSGDTV_ERR_INVALID_ARG, "unknown request");
    Request *r = it->second.get();
    auto ended = [&] { return finished(*r); };
    if (timeout_s < 0) {
        s->cv_done.wait(lock, ended);
    } else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ended)) {
        return fail(BSGDTV_ERR_TIMEOUT, "request not finished within the timeout");
    }
    if (times) {
        times[0] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
        times[1] = r->state == kDone ? std::chrono::duration<double>(r->t_admit - r->t_submit).count() : -1.0;
    }
    if (r->state == kCancelled) {
        s->reqs.erase(it);
        return fail(BSGDTV_ERR_CANCELLED, "request was cancelled");
    }
    if (r->state == kFailed) {
        const int code = r->error;
        const std::string msg = r->message;
        s->reqs.erase(it);
        return fail(code, msg);
    }
    if (x) std::memcpy(x, r->x.data(), r->x.size() * sizeof(float));
    s->reqs.erase(it);
    return BSGDTV_OK;
}

int bsgdtv_server_hold(bsgdtv_server_t s, int hold) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->hold = hold != 0;
        s->wake = true;
    }
    s->cv_work.notify_all();
    return BSGDTV_OK;
}

int bsgdtv_server_set_packing(bsgdtv_server_t s, int max_parts, double cost_ratio) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (max_parts < 1 || max_parts > kMaxParts || !(cost_ratio >= 1.0))
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= max_parts <= 8 and cost_ratio >= 1");
    std::lock_guard<std::mutex> lock(s->mu);
    s->pack_max_parts = max_parts;
    s->pack_cost_ratio = cost_ratio;
    return BSGDTV_OK;
}

int bsgdtv_server_set_priority(bsgdtv_server_t s, int by_size) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    s->priority_by_size = by_size != 0;
    return BSGDTV_OK;
}

int bsgdtv_server_arm(bsgdtv_server_t s, int geom_id, double wait_s) {
    if (!s) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (!(wait_s >= 0.0) || wait_s * 1e9 > (double)bsgdtv::kServeMaxWaitNs)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 0 <= wait_s <= 1");
    bsgdtv_server_ctx::Arm a;
    a.geom = geom_id;
    a.wait_ns = (long long)(wait_s * 1e9);
    std::unique_lock<std::mutex> lock(s->mu);
    if (geom_id < 0 || geom_id >= (int)s->geoms.size() || !s->geoms[geom_id])
        return fail(BSGDTV_ERR_INVALID_ARG, "unknown geometry");
    if (s->stop) return fail(BSGDTV_ERR_STATE, "server is stopping");
    s->arms.push_back(&a);
    s->wake = true;
    s->cv_work.notify_all();
    // the device wait is bounded by wait_s; the host allows it that long plus
    // the launch and a margin before giving up on the report
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s + 30.0),
                                        [&] { return a.finished || s->stop; });
    s->arms.erase(std::find(s->arms.begin(), s->arms.end(), &a));
    if (!ok || !a.finished) return fail(BSGDTV_ERR_STATE, "armed epoch not reported (server stopping)");
    if (a.result == BSGDTV_ERR_TIMEOUT)
        return fail(BSGDTV_ERR_TIMEOUT, "no request arrived during the device-side wait");
    if (a.result != BSGDTV_OK) return fail(a.result, "armed epoch failed");
    return BSGDTV_OK;
}

int bsgdtv_server_stats(bsgdtv_server_t s, int64_t *stats) {
    if (!s || !stats) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t running = 0;
    for (auto &g : s->groups)
        for (const Part &p : g->parts)
            for (int64_t id : p.slot_req) running += id >= 0;
    const int64_t v[18] = {s->submitted, s->completed,   s->failed,     (int64_t)s->queue.size(),
                           running,      (int64_t)s->groups.size(), s->hbm_used, s->max_running,
                           s->ticks,     s->epochs_run,  s->slice_epochs, s->groups_made,
                           s->cancelled, s->armed_epochs, s->wait_timeouts, s->packed_groups,
                           s->max_parts, s->packed_launches};
    std::memcpy(stats, v, sizeof(v));
    return BSGDTV_OK;
}

}  // extern "C"
