// Solve-request queue with continuous batching.
//
// Requests (cg_solve problems on resident gauge fields) are submitted from any
// host thread and run by one scheduler thread.  In each pass the scheduler
// admits waiting requests while free slots and the HBM budget allow (first
// come first served, but a request that fits may pass one that does not),
// sets up the admitted ones (workspace, stream, initial state) and puts each
// into the request group of its gauge, inner precision and inner link format
// (ggroup.cuh).  A group runs the low-precision iterations of all its ready
// members together, one shared-link hop launch per hop for all of them, in a
// device-side loop that stops when any member needs its FP64 reliable update.
// The scheduler then enqueues those updates on the members' own streams, and
// the group's next launch goes on with the others; a member rejoins when its
// update has finished, and newly admitted requests join at the next launch.
// Groups of different gauges run on their own streams, and updates overlap
// the groups' iterations, so all work in flight shares the GPU.  No request
// waits for another's update, and requests join and leave at any launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ggroup.cuh"

namespace {

using clk = std::chrono::steady_clock;

// Scheduler-side state of an admitted request.
enum ReqState { R_INIT, R_READY, R_ACTIVE, R_UPDATING };

struct Req {
    uint64_t ticket = 0;
    wd_solve_desc d{};
    size_t foot = 0;
    bool cancel = false, done = false;
    // ownership (under rq_queue::mu): `listed` while the request is in the
    // scheduler's running list, which the scheduler reads without the lock
    // during a pass; a result taken while listed marks it `taken`, and the
    // scheduler frees it when it drops it from the list
    bool listed = false, taken = false;
    int state = R_INIT;      // scheduler thread only
    int group = -1, slot = -1;
    cudaEvent_t ev = nullptr;   // recorded on its stream when it rejoins after an update
    bool ev_pending = false;
    wd_solve_result res{};
    wd::GSolve gs;
};

// A request group and its members (scheduler thread only).
struct QGroup {
    wd::GGroup g;
    Req *member[wd::GG_MAX] = {};
    int n_members = 0;
    int active[wd::GG_MAX] = {};
    int n_active = 0;
    bool in_flight = false;
};

} // namespace

struct rq_queue {
    wd_ctx *ctx = nullptr;
    size_t budget = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 0;
    std::deque<Req *> waiting;
    std::vector<Req *> running;
    std::unordered_map<uint64_t, Req *> all;
    size_t in_use = 0;
    clk::time_point t0;
    // counters
    uint64_t submitted = 0, completed = 0, stalls = 0, steps = 0, admitted = 0;
    double occupancy_sum = 0.0;   // integral of the running count over time (seconds)
    double busy_s = 0.0;          // time with at least one request running
    int fault_alloc_at = 0;   // WD_FAULT=alloc:N -> the N-th admission fails
    // idle workspaces of finished requests, reused by requests of the same
    // footprint (scheduler thread only); they count against the budget
    struct Idle {
        size_t foot;
        void *mem;
        double *h;
        cudaStream_t s;
    };
    std::vector<Idle> pool;
    size_t pool_bytes = 0;
    std::vector<QGroup *> groups;
    uint64_t group_launches = 0, group_members = 0;
};

namespace wd {
namespace {

double now_s(const rq_queue *q) { return std::chrono::duration<double>(clk::now() - q->t0).count(); }

void finish(rq_queue *q, Req *r, int status)
{
    std::lock_guard<std::mutex> lk(q->mu);
    r->res.status = status;
    r->res.stats.status = status;
    r->res.stats.iters = r->gs.iters;
    r->res.stats.reliable_updates = r->gs.updates;
    r->res.stats.true_rel_resid = r->gs.rel;
    r->res.t_finish = now_s(q);
    if (r->res.t_start == 0.0) r->res.t_start = r->res.t_finish;
    r->res.stats.seconds = r->res.t_finish - r->res.t_submit;
    r->done = true;
    q->in_use -= r->foot;
    q->completed++;
    q->cv_done.notify_all();
}

void free_idle(rq_queue::Idle &e)
{
    cudaStreamSynchronize(e.s);
    cudaStreamDestroy(e.s);
    cudaFree(e.mem);
    cudaFreeHost(e.h);
}

// Workspace for an admitted request: an idle one of the same footprint if
// there is one, else a new allocation after idle ones are freed until the
// budget holds in-use plus idle memory.
int acquire(rq_queue *q, Req *r)
{
    for (size_t k = 0; k < q->pool.size(); ++k)
        if (q->pool[k].foot == r->foot) {
            r->gs.mem = q->pool[k].mem;
            r->gs.h = q->pool[k].h;
            r->gs.s = q->pool[k].s;
            q->pool_bytes -= r->foot;
            q->pool.erase(q->pool.begin() + (long)k);
            return WD_OK;
        }
    size_t in_use;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        in_use = q->in_use;
    }
    while (!q->pool.empty() && in_use + q->pool_bytes > q->budget) {
        q->pool_bytes -= q->pool.front().foot;
        free_idle(q->pool.front());
        q->pool.erase(q->pool.begin());
    }
    return gs_alloc(r->gs);
}

// Returns a finished request's workspace to the pool.
void park(rq_queue *q, Req *r)
{
    gs_release_graph(r->gs);
    if (r->gs.mem) {
        q->pool.push_back({r->foot, r->gs.mem, r->gs.h, r->gs.s});
        q->pool_bytes += r->foot;
    }
    r->gs.mem = nullptr;
    r->gs.h = nullptr;
    r->gs.s = nullptr;
}

// Ends a running request whose work has finished: leaves its group, returns
// its workspace to the pool (or frees it after a CUDA error) and publishes the
// result.
void retire(rq_queue *q, Req *r, int rc)
{
    if (r->group >= 0) {
        QGroup *G = q->groups[r->group];
        G->member[r->slot] = nullptr;
        G->n_members--;
        r->group = r->slot = -1;
    }
    if (r->ev) {
        cudaEventDestroy(r->ev);
        r->ev = nullptr;
    }
    if (rc == WD_ECUDA) gs_release(r->gs);
    else park(q, r);
    finish(q, r, rc != WD_OK ? rc : r->gs.status);
}

// A group for the request's gauge, inner precision and inner links with a free
// member slot (a new one if none has): sets r->group and r->slot.
int join_group(rq_queue *q, Req *r)
{
    const int prec = r->d.opts.inner_prec, recon = r->d.opts.inner_recon;
    int gi = -1;
    for (size_t k = 0; k < q->groups.size(); ++k) {
        const QGroup *G = q->groups[k];
        if (G->g.gauge == r->d.gauge && G->g.prec == prec && G->g.recon == recon && G->n_members < GG_MAX) {
            gi = (int)k;
            break;
        }
    }
    if (gi < 0) {
        QGroup *G = new (std::nothrow) QGroup();
        if (!G) return set_error(WD_ENOMEM, "host allocation failed");
        G->g.gauge = r->d.gauge;
        G->g.prec = prec;
        G->g.recon = recon;
        const int rc = gg_create(q->ctx, G->g);
        if (rc != WD_OK) {
            gg_destroy(G->g);
            delete G;
            return rc;
        }
        q->groups.push_back(G);
        gi = (int)q->groups.size() - 1;
    }
    QGroup *G = q->groups[gi];
    int slot = 0;
    while (G->member[slot]) ++slot;
    G->member[slot] = r;
    G->n_members++;
    G->g.h_table->m[slot] = gg_member(r->gs);
    r->group = gi;
    r->slot = slot;
    return WD_OK;
}

// Advances a request that is not in a group launch and whose own stream is
// idle: initialisation or FP64 update finished, or a cancellation.  Returns
// true if it keeps running.
bool advance_own(rq_queue *q, Req *r)
{
    bool cancel;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        cancel = r->cancel;
    }
    if (cancel) {
        retire(q, r, WD_ECANCELLED);
        return false;
    }
    if (r->state == R_INIT) {
        gs_start(r->gs, 1e300);
        r->res.t_start = now_s(q);
        if (!r->gs.active) {
            retire(q, r, WD_OK);
            return false;
        }
        r->state = R_READY;
        return true;
    }
    if (r->state == R_UPDATING) {
        const int rc = gs_after_update(q->ctx, r->gs);
        if (rc != WD_OK || !r->gs.active || r->gs.status != WD_OK) {
            retire(q, r, rc);
            return false;
        }
        if (r->gs.confirming) return true;   // an FP64 recomputation is in flight on its stream
        // the restart scalars are still being copied on its stream: the group's
        // next launch waits for them
        if (!r->ev && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            retire(q, r, set_error(WD_ECUDA, "event creation failed"));
            return false;
        }
        if (cudaEventRecord(r->ev, r->gs.s) != cudaSuccess) {
            retire(q, r, set_error(WD_ECUDA, "event record failed"));
            return false;
        }
        r->ev_pending = true;
        r->state = R_READY;
        return true;
    }
    return true;   // R_READY: waits for its group's next launch
}

// After a group launch has finished: each member's scalars are handed back;
// members that need their reliable update (or the convergence test) get it
// enqueued on their own streams, the others stay ready for the next launch.
void group_done(rq_queue *q, QGroup *G)
{
    G->in_flight = false;
    for (int t = 0; t < G->n_active; ++t) {
        Req *r = G->member[G->active[t]];
        if (!r || r->state != R_ACTIVE) continue;
        std::memcpy(r->gs.h, G->g.h_hs + (size_t)t * GS_NSCAL, sizeof(double) * GS_NSCAL);
        bool cancel;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            cancel = r->cancel;
        }
        if (cancel) {
            retire(q, r, WD_ECANCELLED);
            continue;
        }
        bool pending = false;
        const int rc = gs_after_begin(q->ctx, r->gs, pending);
        if (rc != WD_OK) {
            retire(q, r, rc);
            continue;
        }
        r->state = pending ? R_UPDATING : R_READY;
        if (pending) {
            std::lock_guard<std::mutex> lk(q->mu);
            q->steps++;
        }
    }
    G->n_active = 0;
}

// Starts a group launch with its ready members.  Returns true if one started.
bool group_start(rq_queue *q, QGroup *G)
{
    int n = 0;
    for (int k = 0; k < GG_MAX; ++k) {
        Req *r = G->member[k];
        if (r && r->state == R_READY) G->active[n++] = k;
    }
    if (n == 0) return false;
    int rc = WD_OK;
    for (int t = 0; t < n && rc == WD_OK; ++t) {
        Req *r = G->member[G->active[t]];
        if (r->ev_pending) {
            if (cudaStreamWaitEvent(G->g.s, r->ev, 0) != cudaSuccess) rc = set_error(WD_ECUDA, "stream wait failed");
            r->ev_pending = false;
        }
    }
    if (rc == WD_OK) rc = gg_launch(G->g, G->active, n);
    if (rc != WD_OK) {
        for (int t = 0; t < n; ++t) retire(q, G->member[G->active[t]], WD_ECUDA);
        return false;
    }
    for (int t = 0; t < n; ++t) G->member[G->active[t]]->state = R_ACTIVE;
    G->n_active = n;
    G->in_flight = true;
    std::lock_guard<std::mutex> lk(q->mu);
    q->steps++;
    q->group_launches++;
    q->group_members += (uint64_t)n;
    return true;
}

void scheduler(rq_queue *q)
{
    cudaSetDevice(q->ctx->device);
    auto last = clk::now();
    for (;;) {
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(q->mu);
            q->cv_work.wait(lk, [q] { return q->stop || !q->waiting.empty() || !q->running.empty(); });
            if (q->stop && q->waiting.empty() && q->running.empty()) break;
            bool stalled = false;
            for (auto it = q->waiting.begin(); it != q->waiting.end();) {
                Req *r = *it;
                if ((int)(q->running.size() + admit.size()) >= q->max_slots) break;
                if (q->in_use + r->foot <= q->budget) {
                    q->in_use += r->foot;
                    admit.push_back(r);
                    it = q->waiting.erase(it);
                } else {
                    stalled = true;
                    ++it;
                }
            }
            if (stalled) q->stalls++;
        }
        // set up the admitted requests outside the lock: workspace, initial
        // state on their own streams, a member slot in their group
        for (Req *r : admit) {
            r->res.t_admit = now_s(q);
            q->admitted++;
            const bool inject = q->fault_alloc_at > 0 && (int)q->admitted == q->fault_alloc_at;
            int rc = inject ? set_error(WD_ENOMEM, "injected allocation failure (WD_FAULT=alloc)") : acquire(q, r);
            if (rc == WD_OK) rc = gs_bind(q->ctx, r->gs, false);
            if (rc == WD_OK) rc = join_group(q, r);
            if (rc != WD_OK) {
                gs_release(r->gs);
                finish(q, r, rc);
                continue;
            }
            r->state = R_INIT;
            std::lock_guard<std::mutex> lk(q->mu);
            q->running.push_back(r);
            r->listed = true;
        }
        std::vector<Req *> running;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            running = q->running;
        }
        // time-weighted occupancy while requests run
        const auto t = clk::now();
        const double dt = std::chrono::duration<double>(t - last).count();
        last = t;
        if (running.empty()) continue;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            q->busy_s += dt;
            q->occupancy_sum += dt * (double)running.size();
        }
        bool progress = !admit.empty();
        // finished group launches
        for (QGroup *G : q->groups) {
            if (!G->in_flight) continue;
            const cudaError_t ge = cudaStreamQuery(G->g.s);
            if (ge == cudaErrorNotReady) continue;
            progress = true;
            if (ge != cudaSuccess) {
                cudaGetLastError();
                G->in_flight = false;
                for (int k = 0; k < G->n_active; ++k)
                    if (G->member[G->active[k]]) retire(q, G->member[G->active[k]], WD_ECUDA);
                G->n_active = 0;
                continue;
            }
            group_done(q, G);
        }
        // requests between group launches whose own streams are idle
        for (Req *r : running) {
            if (r->done || r->state == R_ACTIVE) continue;
            if (r->state == R_READY) {
                bool cancel;
                {
                    std::lock_guard<std::mutex> lk(q->mu);
                    cancel = r->cancel;
                }
                if (!cancel) continue;
            }
            const cudaError_t qe = cudaStreamQuery(r->gs.s);
            if (qe == cudaErrorNotReady) continue;
            progress = true;
            if (qe != cudaSuccess) {
                cudaGetLastError();
                retire(q, r, WD_ECUDA);
                continue;
            }
            advance_own(q, r);
        }
        // next launches of the groups that are idle
        for (QGroup *G : q->groups)
            if (!G->in_flight && group_start(q, G)) progress = true;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            std::vector<Req *> keep;
            for (Req *r : q->running) {
                if (!r->done) {
                    keep.push_back(r);
                    continue;
                }
                r->listed = false;
                if (r->taken) delete r;   // its result was taken during this pass
            }
            q->running.swap(keep);
        }
        // nothing finished: wait briefly, or until a new request arrives
        if (!progress) {
            std::unique_lock<std::mutex> lk(q->mu);
            q->cv_work.wait_for(lk, std::chrono::microseconds(20),
                                [q] { return q->stop || (!q->waiting.empty() && (int)q->running.size() < q->max_slots); });
        }
    }
    for (QGroup *G : q->groups) {
        gg_destroy(G->g);
        delete G;
    }
    q->groups.clear();
    for (auto &e : q->pool) free_idle(e);
    q->pool.clear();
    q->pool_bytes = 0;
}

int check_request(const wd_solve_desc *d)
{
    if (!d || !d->gauge || !d->x_e || !d->b_e) return set_error(WD_EINVAL, "NULL gauge or field in the request");
    if (((uintptr_t)d->x_e & 15u) || ((uintptr_t)d->b_e & 15u)) return set_error(WD_EINVAL, "misaligned field");
    if (!(d->tol > 0.0)) return set_error(WD_EINVAL, "tol must be > 0");
    if (d->opts.maxiter < 1) return set_error(WD_EINVAL, "maxiter must be >= 1");
    if (d->opts.inner_prec != WD_F32 && d->opts.inner_prec != WD_F16 && d->opts.inner_prec != WD_BF16)
        return set_error(WD_EINVAL, "queued solves use mixed precision: inner_prec must be F32, F16 or BF16");
    if (!valid_recon(d->opts.inner_recon) || !valid_recon(d->opts.outer_recon))
        return set_error(WD_EINVAL, "bad link reconstruction");
    if (d->opts.outer_prec != WD_F64 && d->opts.outer_prec != WD_DF)
        return set_error(WD_EINVAL, "outer precision must be WD_F64 or WD_DF");
    if (!(d->opts.delta > 0.0 && d->opts.delta < 1.0)) return set_error(WD_EINVAL, "delta must be in (0, 1)");
    return WD_OK;
}

} // namespace
} // namespace wd

using namespace wd;

extern "C" {

int rq_create(wd_ctx *ctx, size_t hbm_budget_bytes, int max_slots, rq_queue **out)
{
    clear_error();
    if (!ctx || !out || max_slots < 1 || hbm_budget_bytes == 0) return set_error(WD_EINVAL, "bad arguments");
    rq_queue *q = new (std::nothrow) rq_queue();
    if (!q) return set_error(WD_ENOMEM, "host allocation failed");
    q->ctx = ctx;
    q->budget = hbm_budget_bytes;
    q->max_slots = max_slots;
    q->t0 = clk::now();
    if (const char *f = std::getenv("WD_FAULT"))
        if (const char *a = std::strstr(f, "alloc:")) q->fault_alloc_at = std::atoi(a + 6);
    try {
        q->th = std::thread(scheduler, q);
    } catch (...) {
        delete q;
        return set_error(WD_ENOMEM, "could not start the scheduler thread");
    }
    *out = q;
    return WD_OK;
}

int rq_submit(rq_queue *q, const wd_solve_desc *d, uint64_t *ticket)
{
    clear_error();
    if (!q || !ticket) return set_error(WD_EINVAL, "NULL argument");
    WD_TRY(check_request(d));
    const wd_gauge *g = d->gauge;
    // layouts are built here, on the caller's thread, so that the scheduler never allocates them
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_F64, d->opts.outer_recon));
    if (outer_prec_of(d->opts) == WD_DF) WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), WD_DF, d->opts.outer_recon));
    WD_TRY(wd_gauge_prepare(const_cast<wd_gauge *>(g), d->opts.inner_prec, d->opts.inner_recon));
    Req *r = new (std::nothrow) Req();
    if (!r) return set_error(WD_ENOMEM, "host allocation failed");
    r->d = *d;
    r->foot = gs_footprint(g->geo.Vh, d->opts.inner_prec);
    if (r->foot > q->budget) {
        delete r;
        return set_error(WD_ENOMEM, "request needs %zu bytes, more than the queue's HBM budget", gs_footprint(g->geo.Vh, d->opts.inner_prec));
    }
    r->gs.gauge = g;
    r->gs.mass = d->mass;
    r->gs.tol = d->tol;
    r->gs.x = d->x_e;
    r->gs.b = d->b_e;
    r->gs.opts = d->opts;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (q->stop) {
            delete r;
            return set_error(WD_EINVAL, "queue is shutting down");
        }
        r->ticket = ++q->next_ticket;
        r->res.t_submit = now_s(q);
        q->all[r->ticket] = r;
        q->waiting.push_back(r);
        q->submitted++;
        *ticket = r->ticket;
    }
    q->cv_work.notify_one();
    return WD_OK;
}

// Called with q->mu held, for a finished request.  A request the scheduler
// still lists is freed by the scheduler instead (it may be reading it).
static int take_result(rq_queue *q, std::unordered_map<uint64_t, Req *>::iterator it, wd_solve_result *out)
{
    Req *r = it->second;
    if (out) *out = r->res;
    q->all.erase(it);
    if (r->listed) r->taken = true;
    else delete r;
    return WD_OK;
}

int rq_poll(rq_queue *q, uint64_t ticket, wd_solve_result *out)
{
    clear_error();
    if (!q) return set_error(WD_EINVAL, "NULL queue");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->all.find(ticket);
    if (it == q->all.end()) return set_error(WD_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done) return WD_EBUSY;
    return take_result(q, it, out);
}

int rq_wait(rq_queue *q, uint64_t ticket, int timeout_ms, wd_solve_result *out)
{
    clear_error();
    if (!q) return set_error(WD_EINVAL, "NULL queue");
    std::unique_lock<std::mutex> lk(q->mu);
    auto it = q->all.find(ticket);
    if (it == q->all.end()) return set_error(WD_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Req *r = it->second;
    auto ready = [r] { return r->done; };
    if (timeout_ms < 0) q->cv_done.wait(lk, ready);
    else if (!q->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return set_error(WD_ETIMEOUT, "request %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
    return take_result(q, q->all.find(ticket), out);
}

int rq_cancel(rq_queue *q, uint64_t ticket)
{
    clear_error();
    if (!q) return set_error(WD_EINVAL, "NULL queue");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->all.find(ticket);
    if (it == q->all.end()) return set_error(WD_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Req *r = it->second;
    if (r->done) return WD_OK;
    auto w = std::find(q->waiting.begin(), q->waiting.end(), r);
    if (w != q->waiting.end()) {
        q->waiting.erase(w);
        r->res.status = r->res.stats.status = WD_ECANCELLED;
        r->res.t_finish = now_s(q);
        r->done = true;
        q->completed++;
        q->cv_done.notify_all();
    } else {
        r->cancel = true;   // retired by the scheduler once its stream is idle
    }
    return WD_OK;
}

int rq_stats(rq_queue *q, rq_counters *out)
{
    clear_error();
    if (!q || !out) return set_error(WD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    out->submitted = q->submitted;
    out->completed = q->completed;
    out->admission_stalls = q->stalls;
    out->steps = q->steps;
    out->mean_running = q->busy_s > 0.0 ? q->occupancy_sum / q->busy_s : 0.0;
    out->waiting = (int)q->waiting.size();
    out->running = (int)q->running.size();
    out->hbm_in_use = q->in_use;
    out->group_launches = q->group_launches;
    out->mean_group_size = q->group_launches ? (double)q->group_members / (double)q->group_launches : 0.0;
    return WD_OK;
}

int wd_solve_workspace_bytes(const int dims[4], int inner_prec, size_t *out)
{
    clear_error();
    Geometry g;
    WD_TRY(make_geometry(dims, g));
    if (!valid_prec(inner_prec) || inner_prec == WD_F64) return set_error(WD_EINVAL, "inner precision must be F32, F16 or BF16");
    if (!out) return set_error(WD_EINVAL, "out is NULL");
    *out = gs_footprint(g.Vh, inner_prec);
    return WD_OK;
}

int rq_destroy(rq_queue *q)
{
    clear_error();
    if (!q) return WD_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
    }
    q->cv_work.notify_all();
    if (q->th.joinable()) q->th.join();
    for (auto &kv : q->all) delete kv.second;
    delete q;
    return WD_OK;
}

} // extern "C"
