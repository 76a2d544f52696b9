// Continuous-batching reconstruction server.
//
// Requests (projections y of a registered geometry, a TV weight lambda and an
// epoch budget) arrive at any time.  Each geometry owns one or more batch
// groups: a batch handle (one shared A, `slots` slices) on its own stream.  A
// request is admitted into a free slot of a group of its geometry as soon as
// one exists; a new group is created only while the device bytes of all
// groups stay within the HBM budget, and an idle group of another geometry
// is released to make room.  Admitted requests keep their x, r and FGP state
// on the device in their slot.
//
// One worker thread drives the device.  Every group with occupied slots runs
// a "tick" of E epochs, E = the smallest remaining budget among its slots
// (capped), as one sequence of captured epoch graphs on the group's stream,
// so the groups of different geometries overlap on the GPU.  When a tick
// ends, finished requests are copied out (x to host memory: the end of their
// latency) and their slots are emptied; queued requests are admitted between
// ticks.  A slice's arithmetic never depends on the other slots, so a
// request's result is the same alone and in any mix.  A cancelled request
// leaves the queue at once, or gives up its slot when its group's current
// tick ends.
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

struct Group {
    int geom = 0;
    bsgdtv_batch_t batch = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<int64_t> slot_req;   // request id per slot, -1 = free
    bool busy = false;
    int tick = 0;
    int64_t bytes = 0;
    Clock::time_point idle_since;
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
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, ticks = 0, epochs_run = 0, groups_made = 0,
            groups_freed = 0, max_running = 0, slice_epochs = 0;
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

// Empties slot b of g (its state reset to zeros) after its request ended.
void free_slot(Group *g, int b) {
    g->slot_req[b] = -1;
    bsgdtv_batch_set_slice(g->batch, b, nullptr, 0, 0.0);
}

void finish_cancelled(bsgdtv_server_ctx *s, Request &r) {
    r.state = kCancelled;
    r.t_done = Clock::now();
    s->cancelled++;
}

int destroy_group(bsgdtv_server_ctx *s, Group *g) {
    if (g->batch) bsgdtv_batch_destroy(g->batch);
    if (g->done) cudaEventDestroy(g->done);
    if (g->stream) cudaStreamDestroy(g->stream);
    s->hbm_used -= g->bytes;
    s->groups_freed++;
    return BSGDTV_OK;
}

// Creates a group for geometry gi (caller holds the lock; the A upload runs
// under it, which only delays submitters).
int make_group(bsgdtv_server_ctx *s, int gi, int slots, Group **out) {
    Geometry &G = *s->geoms[gi];
    std::unique_ptr<Group> g(new Group());
    g->geom = gi;
    g->bytes = G.bytes_for(slots);
    BSG_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    BSG_CUDA(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));
    int rc = bsgdtv_batch_create_from_operator(&g->batch, G.op, slots, g->stream);
    if (rc == BSGDTV_OK) bsgdtv::batch_keep_prox(g->batch, s->fgp_iters > 0);
    if (rc == BSGDTV_OK) {
        std::vector<float> zeros((size_t)G.rows * slots, 0.f);
        std::vector<double> lam((size_t)slots, 0.0);
        rc = bsgdtv_batch_set_data(g->batch, zeros.data(), 0, lam.data(), G.mu);
    }
    if (rc != BSGDTV_OK) {
        if (g->batch) bsgdtv_batch_destroy(g->batch);
        cudaEventDestroy(g->done);
        cudaStreamDestroy(g->stream);
        return rc;
    }
    g->slot_req.assign(slots, -1);
    g->idle_since = Clock::now();
    s->hbm_used += g->bytes;
    s->groups_made++;
    *out = g.get();
    s->groups.push_back(std::move(g));
    return BSGDTV_OK;
}

bool group_idle(const Group *g) {
    if (g->busy) return false;
    for (int64_t id : g->slot_req)
        if (id >= 0) return false;
    return true;
}

// Finds or makes a free slot for geometry gi.  Returns false if none can be
// had now (the request waits); sets *fatal if the geometry can never fit.
bool find_slot(bsgdtv_server_ctx *s, int gi, Group **gout, int *slot, int *fatal) {
    *fatal = BSGDTV_OK;
    for (auto &g : s->groups) {
        if (g->geom != gi || g->busy) continue;
        for (int b = 0; b < (int)g->slot_req.size(); ++b)
            if (g->slot_req[b] < 0) {
                *gout = g.get();
                *slot = b;
                return true;
            }
    }
    const Geometry &G = *s->geoms[gi];
    if (G.op_bytes + G.bytes_for(G.min_slots) > s->budget) {
        *fatal = BSGDTV_ERR_OOM;
        return false;
    }
    // a group of this geometry is busy with free slots: wait for its tick
    for (auto &g : s->groups)
        if (g->geom == gi && g->busy)
            for (int64_t id : g->slot_req)
                if (id < 0) return false;
    // a new group sized for the requests of this geometry now waiting (a
    // power of two between min_slots and slots): a short queue gets a small
    // group with short epochs (low latency), a long queue a large one that
    // reads A once for many slices (throughput); shrunk if the budget cannot
    // hold it
    int slots = G.min_slots;
    while (slots < G.slots && slots < G.queued) slots *= 2;
    slots = std::min(slots, G.slots);
    while (slots > G.min_slots && s->hbm_used + G.bytes_for(slots) > s->budget &&
           !std::any_of(s->groups.begin(), s->groups.end(), [&](const std::unique_ptr<Group> &p) {
               return p->geom != gi && group_idle(p.get());
           }))
        slots = std::max(G.min_slots, slots / 2);
    const int64_t need = G.bytes_for(slots);
    // release idle groups of other geometries (oldest first) until it fits
    while (s->hbm_used + need > s->budget) {
        Group *victim = nullptr;
        for (auto &g : s->groups)
            if (g->geom != gi && group_idle(g.get()) &&
                (!victim || g->idle_since < victim->idle_since))
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
    const int rc = make_group(s, gi, slots, &g);
    if (rc != BSGDTV_OK) {
        *fatal = rc;
        return false;
    }
    *gout = g;
    *slot = 0;
    return true;
}

void admit(bsgdtv_server_ctx *s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request &r = *s->reqs[*it];
        Group *g = nullptr;
        int slot = -1, fatal = BSGDTV_OK;
        if (!find_slot(s, r.geom, &g, &slot, &fatal)) {
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
        // y was checked at submit: no second check, no wait for the copy
        const int rc = bsgdtv::batch_set_slice(g->batch, slot, r.y.data(), 0, r.lambda, false);
        if (rc != BSGDTV_OK) {
            finish_failed(s, r, rc, std::string("set_slice: ") + bsgdtv_last_error());
        } else {
            g->slot_req[slot] = r.id;
            r.state = kRunning;
            r.remaining = r.epochs;
            r.t_admit = Clock::now();
            std::vector<float>().swap(r.y);
        }
        s->geoms[r.geom]->queued--;
        it = s->queue.erase(it);
    }
}

// Launches a tick on every group that has occupied slots and is not running.
void launch_ticks(bsgdtv_server_ctx *s) {
    int64_t running = 0;
    for (auto &g : s->groups) {
        int tick = 0;
        for (int64_t id : g->slot_req)
            if (id >= 0) {
                running++;
                const int rem = s->reqs[id]->remaining;
                tick = tick ? std::min(tick, rem) : rem;
            }
        if (g->busy || tick == 0) continue;
        tick = std::min(tick, s->max_tick);
        int rc = bsgdtv_batch_run(g->batch, tick, s->fgp_iters);
        if (rc == BSGDTV_OK && cudaEventRecord(g->done, g->stream) != cudaSuccess) rc = BSGDTV_ERR_CUDA;
        if (rc != BSGDTV_OK) {
            const std::string msg = std::string("run: ") + bsgdtv_last_error();
            for (int64_t &id : g->slot_req)
                if (id >= 0) {
                    finish_failed(s, *s->reqs[id], rc, msg);
                    id = -1;
                }
            s->cv_done.notify_all();
            continue;
        }
        g->busy = true;
        g->tick = tick;
        s->ticks++;
        s->epochs_run += tick;
    }
    s->max_running = std::max(s->max_running, running);
}

// Harvests finished ticks.  Returns true if any group finished.
bool harvest(bsgdtv_server_ctx *s) {
    bool any = false;
    for (auto &g : s->groups) {
        if (!g->busy) continue;
        const cudaError_t q = cudaEventQuery(g->done);
        if (q == cudaErrorNotReady) continue;
        g->busy = false;
        any = true;
        for (int b = 0; b < (int)g->slot_req.size(); ++b) {
            const int64_t id = g->slot_req[b];
            if (id < 0) continue;
            Request &r = *s->reqs[id];
            if (q != cudaSuccess) {
                finish_failed(s, r, BSGDTV_ERR_CUDA, std::string("tick: ") + cudaGetErrorString(q));
                g->slot_req[b] = -1;
                continue;
            }
            r.remaining -= g->tick;
            s->slice_epochs += g->tick;
            if (r.cancel) {
                finish_cancelled(s, r);
                free_slot(g.get(), b);
                continue;
            }
            if (r.remaining > 0) continue;
            r.x.resize((size_t)s->geoms[g->geom]->cols);
            int rc = bsgdtv_batch_get_slice_x(g->batch, b, r.x.data(), 0);
            if (rc == BSGDTV_OK) {
                r.state = kDone;
                r.t_done = Clock::now();
                s->completed++;
            } else {
                finish_failed(s, r, rc, std::string("get_slice_x: ") + bsgdtv_last_error());
            }
            free_slot(g.get(), b);
        }
        if (q != cudaSuccess) cudaGetLastError();
        if (group_idle(g.get())) g->idle_since = Clock::now();
    }
    if (any) s->cv_done.notify_all();
    return any;
}

// Frees the slots of cancelled requests in groups that are not running a
// tick (a busy group's are freed when harvest sees its tick end).
void reap_cancelled(bsgdtv_server_ctx *s) {
    bool any = false;
    for (auto &g : s->groups) {
        if (g->busy) continue;
        bool freed = false;
        for (int b = 0; b < (int)g->slot_req.size(); ++b) {
            const int64_t id = g->slot_req[b];
            if (id < 0 || !s->reqs[id]->cancel) continue;
            finish_cancelled(s, *s->reqs[id]);
            free_slot(g.get(), b);
            freed = true;
        }
        if (freed && group_idle(g.get())) g->idle_since = Clock::now();
        any = any || freed;
    }
    if (any) s->cv_done.notify_all();
}

void worker_main(bsgdtv_server_ctx *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        if (s->stop) break;
        harvest(s);
        reap_cancelled(s);
        admit(s);
        launch_ticks(s);
        bool busy = false;
        for (auto &g : s->groups) busy = busy || g->busy;
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
    s->cv_done.notify_all();
    delete s;
}

int bsgdtv_server_add_geometry(bsgdtv_server_t s, int64_t rows, int64_t cols, int img_h, int img_w,
                               const int64_t *row_ptr, const int32_t *col_idx, const double *vals,
                               int format, int slots, double mu, int prewarm, int *geom_id) {
    if (!s || !geom_id || !row_ptr || !col_idx || !vals)
        return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    if (slots < 1 || slots > 4096 || !(mu > 0.0) || !std::isfinite(mu) || prewarm < 0)
        return fail(BSGDTV_ERR_INVALID_ARG, "need 1 <= slots <= 4096, finite mu > 0, prewarm >= 0");
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
        const int rc = make_group(s, gi, slots, &g);
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
        r.cancel = true;   // running: the worker frees its slot
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

int bsgdtv_server_stats(bsgdtv_server_t s, int64_t *stats) {
    if (!s || !stats) return fail(BSGDTV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t running = 0;
    for (auto &g : s->groups)
        for (int64_t id : g->slot_req) running += id >= 0;
    const int64_t v[13] = {s->submitted, s->completed,   s->failed,     (int64_t)s->queue.size(),
                           running,      (int64_t)s->groups.size(), s->hbm_used, s->max_running,
                           s->ticks,     s->epochs_run,  s->slice_epochs, s->groups_made,
                           s->cancelled};
    std::memcpy(stats, v, sizeof(v));
    return BSGDTV_OK;
}

}  // extern "C"
