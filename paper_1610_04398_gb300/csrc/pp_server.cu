// Continuous-batching solve server: requests for snapshots of any grid size are queued,
// admitted in arrival order as soon as a stream slot and device memory (the budget) are
// available, and run concurrently on separate streams.  Plans (trees, expansions,
// tables) stay resident between requests of the same grid and are reused; idle plans are
// evicted least-recently-used when a new grid needs room.  One dispatcher thread owns
// every CUDA call; completion is detected by polling events, so no wait blocks the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pp.h"
#include "pp_common.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct Req {
    int64_t id = 0;
    pp_request r{};
    int status = PP_SERVER_QUEUED;
    int error = PP_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct PlanKey {
    int n;
    double h, x0, y0, rho, lift, ux, uy;
    int interp;
    bool operator<(const PlanKey& o) const {
        const double a[] = {double(n), h, x0, y0, rho, lift, ux, uy, double(interp)};
        const double b[] = {double(o.n), o.h, o.x0, o.y0, o.rho, o.lift, o.ux, o.uy, double(o.interp)};
        return std::lexicographical_compare(a, a + 9, b, b + 9);
    }
};

struct PlanEntry {
    PlanKey key;
    pp_plan plan = nullptr;
    int64_t bytes = 0;    // device bytes reserved for the plan (its workspace once it has run)
    int surf_cap = 0;     // surface points its scratch holds after the requests admitted so far
    bool busy = false;
    double last_used = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Req* req = nullptr;
    PlanEntry* pe = nullptr;
};

}  // namespace

struct pp_server_s {
    pp_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Req*> queue;
    std::map<int64_t, Req*> reqs;
    int64_t next_id = 1;
    bool stop = false;
    std::thread th;
    std::vector<Slot> slots;
    std::vector<PlanEntry*> plans;
    int64_t held = 0;
    int64_t completed = 0, failed = 0, plans_created = 0, plans_evicted = 0;
};

namespace {

// Device bytes a new plan for a request needs: the arrays pp_plan_create makes for the
// server's order, theta, precision and tile, and the surface scratch for its points.
int64_t plan_need(const pp_server_config& c, int n, int npts) {
    pp_options o;
    pp_options_default(&o);
    o.precision = c.precision;
    o.tile = c.tile;
    o.theta_surface = c.theta_surface;
    int64_t b = 0;
    return pp_plan_bytes(n, c.order, c.theta, &o, npts, &b) == PP_OK ? b : INT64_MAX;
}

bool device_pointer(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool valid_request(const pp_request* r) {
    const int n = r->grid.n;
    if (n < 8 || n > 16384 || (n & (n - 1)) != 0 || !(r->h > 0.0)) return false;
    if (!r->u || !r->v || !r->chi || !r->us_x || !r->us_y) return false;
    if (r->npts < 0 || r->npts > (1 << 24) || (r->npts > 0 && (!r->points || !r->normals))) return false;
    if (!std::isfinite(r->lambda) || !std::isfinite(r->nu)) return false;
    // forces are written by the kernels: host memory would make the dispatcher copy and
    // synchronise while it holds the server lock
    if (r->npts > 0 && r->forces && !device_pointer(r->forces)) return false;
    return true;
}

// Launch one request on a slot (dispatcher thread only).
int launch(pp_server s, Slot& sl) {
    Req* q = sl.req;
    pp_plan p = sl.pe->plan;
    const pp_request& r = q->r;
    int st = pp_plan_set_stream(p, sl.stream);
    if (st == PP_OK) st = pp_rhs(p, r.u, r.v, r.chi, r.us_x, r.us_y, r.lambda, nullptr);
    if (st == PP_OK) st = pp_pressure_solve(p, r.p_out);
    if (st == PP_OK && r.npts > 0)
        st = pp_surface_traction(p, r.u, r.v, r.npts, r.points, r.normals, r.dS, r.nu, r.per_point, r.forces);
    if (st == PP_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = PP_ERR_CUDA;
    (void)s;
    return st;
}

PlanEntry* find_plan(pp_server s, const PlanKey& k) {
    for (PlanEntry* pe : s->plans)
        if (!pe->busy && !(pe->key < k) && !(k < pe->key)) return pe;
    return nullptr;
}

void drop_plan(pp_server s, PlanEntry* pe) {
    pp_plan_destroy(pe->plan);
    s->held -= pe->bytes;
    s->plans.erase(std::find(s->plans.begin(), s->plans.end(), pe));
    delete pe;
}

// Evict idle plans other than `keep`, least recently used first, until `need` more bytes
// fit in the budget; false if they cannot.
bool make_room(pp_server s, int64_t need, const PlanEntry* keep) {
    while (s->held + need > s->cfg.budget_bytes) {
        PlanEntry* victim = nullptr;
        for (PlanEntry* pe : s->plans)
            if (!pe->busy && pe != keep && (!victim || pe->last_used < victim->last_used)) victim = pe;
        if (!victim) return false;
        drop_plan(s, victim);
        ++s->plans_evicted;
    }
    return true;
}

// Find or make a plan for request r within the budget; nullptr if it has to wait.  The
// bytes a request adds (a new plan, or the growth of a resident plan's surface scratch for
// its points) are reserved before it is admitted, so the plans never hold more than the
// budget.
PlanEntry* acquire_plan(pp_server s, const pp_request& r, int* err) {
    *err = PP_OK;
    PlanKey k{r.grid.n, r.h, r.grid.x0, r.grid.y0, r.rho, r.lift, r.uinf_x, r.uinf_y, r.interp};
    if (PlanEntry* pe = find_plan(s, k)) {
        const int cap = pp::surface_cap_after(pe->surf_cap, r.npts);
        const int64_t grow = pp::surface_scratch_bytes(cap) - pp::surface_scratch_bytes(pe->surf_cap);
        if (make_room(s, grow, pe)) {
            pe->bytes += grow;
            s->held += grow;
            pe->surf_cap = cap;
            return pe;
        }
        // a fresh plan sized for these points may fit where the grown one does not
        if (!std::any_of(s->plans.begin(), s->plans.end(), [](PlanEntry* x) { return x->busy; })) {
            drop_plan(s, pe);
            ++s->plans_evicted;
        } else {
            return nullptr;
        }
    }
    const int64_t need = plan_need(s->cfg, r.grid.n, r.npts);
    if (!make_room(s, need, nullptr)) return nullptr;
    pp_options o;
    pp_options_default(&o);
    o.precision = s->cfg.precision;
    o.rho = r.rho;
    o.lift = r.lift;
    o.interp = r.interp;
    o.uinf_x = r.uinf_x;
    o.uinf_y = r.uinf_y;
    o.tile = s->cfg.tile;
    o.theta_surface = s->cfg.theta_surface;
    pp_plan p = nullptr;
    int st = pp_plan_create(&p, r.grid, r.h, s->cfg.order, s->cfg.theta, &o);
    if (st != PP_OK) {
        *err = st;
        return nullptr;
    }
    PlanEntry* pe = new PlanEntry();
    pe->key = k;
    pe->plan = p;
    pe->bytes = need;
    pe->surf_cap = pp::surface_cap_after(pp::kInitialSurfaceCap, r.npts);
    s->held += pe->bytes;
    s->plans.push_back(pe);
    ++s->plans_created;
    return pe;
}

// After a request: the plan's reservation becomes its actual workspace.
void refresh_bytes(pp_server s, PlanEntry* pe) {
    pp_plan_info_t inf;
    if (pp_plan_info(pe->plan, &inf) != PP_OK) return;
    s->held += inf.workspace_bytes - pe->bytes;
    pe->bytes = inf.workspace_bytes;
}

void dispatcher(pp_server s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. retire finished requests
        bool any_busy = false;
        for (Slot& sl : s->slots) {
            if (!sl.req) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            Req* q = sl.req;
            q->t_done = seconds_since(s->t0);
            if (e == cudaSuccess) {
                q->status = PP_SERVER_DONE;
                ++s->completed;
                refresh_bytes(s, sl.pe);
                sl.pe->busy = false;
                sl.pe->last_used = q->t_done;
            } else {
                cudaGetLastError();
                q->status = PP_SERVER_FAILED;
                q->error = PP_ERR_CUDA;
                ++s->failed;
                drop_plan(s, sl.pe);
            }
            sl.req = nullptr;
            sl.pe = nullptr;
        }
        s->cv_done.notify_all();
        // 2. admit queued requests in arrival order while slots and memory allow
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Slot* free_slot = nullptr;
            for (Slot& sl : s->slots)
                if (!sl.req) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            Req* q = *it;
            int err = PP_OK;
            PlanEntry* pe = acquire_plan(s, q->r, &err);
            if (!pe) {
                if (err != PP_OK) {  // cannot ever run: fail it and move on
                    q->status = PP_SERVER_FAILED;
                    q->error = err;
                    ++s->failed;
                    it = s->queue.erase(it);
                    continue;
                }
                ++it;  // waits for memory; a later, smaller request may still fit
                continue;
            }
            pe->busy = true;
            free_slot->req = q;
            free_slot->pe = pe;
            q->status = PP_SERVER_RUNNING;
            q->t_start = seconds_since(s->t0);
            const int st = launch(s, *free_slot);
            if (st != PP_OK) {
                q->status = PP_SERVER_FAILED;
                q->error = st;
                q->t_done = seconds_since(s->t0);
                ++s->failed;
                drop_plan(s, pe);
                free_slot->req = nullptr;
                free_slot->pe = nullptr;
            } else {
                any_busy = true;
            }
            it = s->queue.erase(it);
        }
        s->cv_done.notify_all();
        if (s->stop && s->queue.empty() && !any_busy) break;
        // 3. sleep: briefly while work is in flight (to poll completions), else until a submit
        if (any_busy)
            s->cv.wait_for(lk, std::chrono::microseconds(20));
        else
            s->cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop || !s->queue.empty(); });
    }
}

}  // namespace

extern "C" {

void pp_server_config_default(pp_server_config* c) {
    if (!c) return;
    c->budget_bytes = int64_t(8) << 30;
    c->slots = 8;
    c->precision = PP_MIXED;
    c->order = 12;
    c->theta = 0.6;
    c->tile = 16;
    c->theta_surface = 0.0;
}

int pp_server_create(const pp_server_config* cfg, pp_server* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    pp_server_config c;
    pp_server_config_default(&c);
    if (cfg) c = *cfg;
    if (c.budget_bytes <= 0 || c.slots < 1 || c.slots > 64) return PP_ERR_ARG;
    if (c.precision != PP_FP64 && c.precision != PP_MIXED) return PP_ERR_ARG;
    if (c.order < 2 || c.order > 40 || !(c.theta >= 0.25 && c.theta <= 0.95)) return PP_ERR_ARG;
    if (c.tile != 8 && c.tile != 16 && c.tile != 128) return PP_ERR_ARG;
    if (c.theta_surface != 0.0 && !(c.theta_surface >= 0.25 && c.theta_surface <= 0.95)) return PP_ERR_ARG;
    pp_server s = new (std::nothrow) pp_server_s();
    if (!s) return PP_ERR_OOM;
    s->cfg = c;
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PP_ERR_CUDA;
    }
    s->slots.resize(c.slots);
    for (Slot& sl : s->slots)
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (Slot& x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
            }
            delete s;
            return PP_ERR_CUDA;
        }
    s->th = std::thread(dispatcher, s);
    *out = s;
    return PP_OK;
}

int pp_server_submit(pp_server s, const pp_request* r, int64_t* id) {
    if (!s || !r || !id) return PP_ERR_ARG;
    *id = 0;
    if (!valid_request(r)) return PP_ERR_ARG;
    if (plan_need(s->cfg, r->grid.n, r->npts) > s->cfg.budget_bytes) return PP_ERR_BUDGET;
    Req* q = new (std::nothrow) Req();
    if (!q) return PP_ERR_OOM;
    q->r = *r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete q;
            return PP_ERR_STATE;
        }
        q->id = s->next_id++;
        q->t_submit = seconds_since(s->t0);
        s->reqs[q->id] = q;
        s->queue.push_back(q);
        *id = q->id;
    }
    s->cv.notify_all();
    return PP_OK;
}

int pp_server_cancel(pp_server s, int64_t id) {
    if (!s) return PP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return PP_ERR_ARG;
    Req* q = it->second;
    if (q->status != PP_SERVER_QUEUED) return PP_ERR_STATE;  // already on the device
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
    q->status = PP_SERVER_CANCELLED;
    q->t_done = seconds_since(s->t0);
    s->cv_done.notify_all();
    return PP_OK;
}

int pp_server_query(pp_server s, int64_t id, int* status, int* error, double times[3]) {
    if (!s) return PP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return PP_ERR_ARG;
    Req* q = it->second;
    if (status) *status = q->status;
    if (error) *error = q->error;
    if (times) {
        times[0] = q->t_submit;
        times[1] = q->t_start;
        times[2] = q->t_done;
    }
    return PP_OK;
}

int pp_server_wait(pp_server s, int64_t id, double timeout_s) {
    if (!s || !(timeout_s >= 0)) return PP_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return PP_ERR_ARG;
    Req* q = it->second;
    auto finished = [&] { return q->status >= PP_SERVER_DONE; };
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) return PP_ERR_TIMEOUT;
    return q->status == PP_SERVER_DONE ? PP_OK : (q->status == PP_SERVER_CANCELLED ? PP_ERR_STATE : q->error);
}

int pp_server_stats(pp_server s, pp_server_stats_t* st) {
    if (!s || !st) return PP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = int64_t(s->queue.size());
    st->running = 0;
    for (Slot& sl : s->slots) st->running += sl.req ? 1 : 0;
    st->completed = s->completed;
    st->failed = s->failed;
    st->plans_resident = int64_t(s->plans.size());
    st->plans_created = s->plans_created;
    st->plans_evicted = s->plans_evicted;
    st->bytes_held = s->held;
    return PP_OK;
}

int pp_server_destroy(pp_server s) {
    if (!s) return PP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req* q : s->queue) {  // not yet started: cancelled, in-flight ones finish
            q->status = PP_SERVER_CANCELLED;
            q->t_done = seconds_since(s->t0);
        }
        s->queue.clear();
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
    if (s->th.joinable()) s->th.join();
    for (PlanEntry* pe : s->plans) {
        pp_plan_destroy(pe->plan);
        delete pe;
    }
    for (Slot& sl : s->slots) {
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
    }
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return PP_OK;
}

}  // extern "C"
