// mg_server.cu -- continuous-batching request loop of the pressure multigrid.
//
// A host thread admits queued solves while slots and the device-memory budget
// allow, and reuses the hierarchy of a finished request for a later request of
// the same grid.  Admitted requests run in size lanes: a lane holds the
// requests whose grids are within a factor 8 in cells of each other and
// advances them together, one refinement step (up to inner_cycles V-cycles and
// the FP64 residual) per launch for the whole set.  Each lane has its own CUDA
// stream, the lanes of smaller grids at a higher stream priority, and the loop
// steps every lane whose previous step has completed (event polling), so a
// small request takes its steps at its own pace while a large one runs and
// their kernels share the GPU.  Requests join and leave a lane between steps.
// Every grid's arithmetic is independent of the other grids in a launch, so a
// request's result is bitwise the same alone and in the mix.
#include <stdlib.h>
#include <string.h>

#include <new>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gbmg.h"
#include "mg_api_internal.h"

using namespace gbmg;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kLanes = 4;

struct Request {
    mg_ticket id;
    mg_grid grid;
    const double *ax, *ay, *az, *rhs;
    double *p;
    double tol;
    size_t bytes;
    int lane = 0;
    Clock::time_point t_submit;
    mg_handle *h = nullptr;
    bool done = false;
    int status = MG_EAGAIN;
    int64_t admit_tick = 0;
    int inflight_at_admit = 0;
    mg_stats st;
};

using GridKey = std::tuple<int, int, int, double, double, double, int, int, int>;

GridKey key_of(const mg_grid &g)
{
    return GridKey(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, g.bc[0], g.bc[1], g.bc[2]);
}

// Size lane of a grid: lane k holds grids of up to 2^(18 + 3k) cells (64^3,
// 128^3, 256^3 and above), so the grids stepped together differ by at most a
// factor 8 in cells.
int lane_of(const mg_grid &g, int lanes)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    int k = 0;
    while (k + 1 < lanes && n > (1ll << (18 + 3 * k))) k++;
    return k;
}

// One size lane: its stream, its plan over its running requests, and the
// event that marks the end of its last step (with the states gathered into
// the plan's host mirror).
struct Lane {
    cudaStream_t stream = nullptr;
    Plan *plan = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<Request *> running;   // the members of the plan, in its grid order
    std::vector<Request *> pending;   // started, joining at the lane's next step
    bool changed = false;  // membership changed: rewrite the plan's tables
    bool fresh = false;    // a request joined: read the states before the next step
    bool busy = false;     // a step is in flight
};

}  // namespace

struct mg_server {
    size_t budget = 0;
    int max_slots = 1;
    mg_params prm;
    bool own_streams = false;
    int nlanes = kLanes;
    Lane lanes[kLanes];
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    int in_flight = 0;  // requests admitted and not yet retired
    std::unordered_map<mg_ticket, Request *> tickets;
    std::multimap<GridKey, mg_handle *> cache;
    size_t bytes_in_use = 0, peak = 0;
    int64_t completed = 0;
    int64_t ticks = 0;  // refinement-step launches of all lanes
    int max_in_flight = 0;
    mg_ticket next_id = 1;
    bool stop = false;
    int loop_error = MG_OK;
    int64_t fail_at = 0;  // test aid: the fail_at-th step launch fails on the host (0: never)
    std::thread th;

    void loop();
    void admit_locked(std::vector<Request *> &fresh);
    int start_fresh(std::vector<Request *> &fresh);
    int finish_lane(Lane &L);
    int step_lane(Lane &L);
    void fail_all(int rc);
    void retire_locked(Request *r, const Clock::time_point &now);
    void release_lanes();
};

// Move queued requests into slots while slots and budget allow (FIFO; a
// request that does not fit yet blocks the ones behind it, so large requests
// are not starved).  Called with the lock held.
void mg_server::admit_locked(std::vector<Request *> &fresh)
{
    while (!queue.empty() && in_flight < max_slots) {
        Request *r = queue.front();
        Lane &L = lanes[r->lane];
        mg_handle *h = nullptr;
        auto it = cache.find(key_of(r->grid));
        if (it != cache.end()) {
            h = it->second;
            cache.erase(it);
        } else {
            while (bytes_in_use + r->bytes > budget && !cache.empty()) {
                auto victim = cache.begin();
                bytes_in_use -= victim->second->bytes;
                mg_destroy(victim->second);
                cache.erase(victim);
            }
            if (bytes_in_use + r->bytes > budget) break;  // wait for running requests
            int rc = handle_alloc(&r->grid, &prm, L.stream, &h);
            if (rc) {
                queue.pop_front();
                r->done = true;
                r->status = rc;
                memset(&r->st, 0, sizeof(r->st));
                r->st.status = rc;
                completed++;
                cv_done.notify_all();
                continue;
            }
            bytes_in_use += h->bytes;
            peak = std::max(peak, bytes_in_use);
        }
        queue.pop_front();
        int rc = set_faces_impl(h, r->ax, r->ay, r->az);
        if (rc) {
            r->done = true;
            r->status = rc;
            memset(&r->st, 0, sizeof(r->st));
            r->st.status = rc;
            cache.emplace(key_of(r->grid), h);
            completed++;
            cv_done.notify_all();
            continue;
        }
        r->h = h;
        r->admit_tick = ticks;
        r->inflight_at_admit = in_flight;
        in_flight++;
        fresh.push_back(r);
    }
    max_in_flight = std::max(max_in_flight, in_flight);
}

// Start the new requests (state reset, mean of b, R_0) on their own
// single-grid plans, on their lane's stream, and add them to their lane.
int mg_server::start_fresh(std::vector<Request *> &fresh)
{
    int rc = MG_OK;
    for (Request *r : fresh) {
        Lane &L = lanes[r->lane];
        Plan &sp = *r->h->plan;
        plan_bind(sp, 0, r->rhs, r->p, r->tol, prm.max_iters);
        if (!rc) rc = plan_upload(sp);
        if (!rc) rc = plan_prologue(sp);
        L.pending.push_back(r);
    }
    return rc;
}

// Record a finished request (lock held).
void mg_server::retire_locked(Request *r, const Clock::time_point &now)
{
    int herr[3] = {0, 0, 0};
    cudaMemcpy(herr, r->h->err, sizeof(herr), cudaMemcpyDeviceToHost);
    GridState s;
    cudaMemcpy(&s, r->h->state, sizeof(s), cudaMemcpyDeviceToHost);
    const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    fill_stats(s, herr, ms, &r->st, &r->status);
    r->st.admit_tick = r->admit_tick;
    r->st.finish_tick = ticks;
    r->st.inflight_at_admit = r->inflight_at_admit;
    r->st.lane = r->lane;
    r->done = true;
    cache.emplace(key_of(r->grid), r->h);
    r->h = nullptr;
    completed++;
    in_flight--;
}

// The lane's last step has completed: its states are in the plan's host
// mirror.  Finish the requests that stopped (p - mean p on their own plans),
// wait for that, and retire them.
int mg_server::finish_lane(Lane &L)
{
    std::vector<Request *> finished, keep;
    for (size_t g = 0; g < L.running.size(); g++) {
        if (!L.plan->st_h[g].active) finished.push_back(L.running[g]);
        else keep.push_back(L.running[g]);
    }
    if (finished.empty()) return MG_OK;
    int rc = MG_OK;
    for (Request *r : finished)
        if (!rc) rc = plan_final(*r->h->plan);
    if (!rc) rc = cudaStreamSynchronize(L.stream) == cudaSuccess ? MG_OK : MG_ECUDA;
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto now = Clock::now();
        for (Request *r : finished) retire_locked(r, now);
    }
    cv_done.notify_all();
    L.running = keep;
    L.changed = true;
    return MG_OK;
}

// Launch one refinement step of the lane's running requests and the gather of
// their states into the plan's host mirror, then mark its end with the event.
int mg_server::step_lane(Lane &L)
{
    int rc = MG_OK;
    if (!L.pending.empty()) {
        L.running.insert(L.running.end(), L.pending.begin(), L.pending.end());
        L.pending.clear();
        L.changed = L.fresh = true;
    }
    if (L.changed) {
        // the plan is allocated once for max_slots grids; a change of the
        // lane's set only rewrites its tables (asynchronously, no allocation)
        if (!L.plan) {
            L.plan = new (std::nothrow) Plan();
            if (!L.plan) return MG_ENOMEM;
            rc = L.plan->alloc(max_slots);
            if (rc) return rc;
        }
        std::vector<mg_handle *> hs;
        for (Request *r : L.running) hs.push_back(r->h);
        rc = L.plan->fill(hs.data(), (int)hs.size());
        for (size_t g = 0; g < L.running.size() && !rc; g++)
            plan_bind(*L.plan, (int)g, L.running[g]->rhs, L.running[g]->p, L.running[g]->tol, prm.max_iters);
        if (!rc) rc = plan_upload(*L.plan);
        L.changed = false;
    }
    // the step's cycle count comes from the states on the host: a request that
    // just joined has none there yet
    if (!rc && L.fresh) {
        rc = plan_sync_states(*L.plan);
        L.fresh = false;
    }
    if (rc) return rc;
    bool any_active = false;
    for (size_t g = 0; g < L.running.size(); g++) any_active |= L.plan->st_h[g].active != 0;
    if (any_active) {
        ticks++;
        if (fail_at > 0 && ticks == fail_at) return MG_ECUDA;  // injected on the host (test aid)
        rc = plan_body(*L.plan);
    }
    if (!rc) rc = plan_gather_states(*L.plan);
    if (!rc) rc = cudaEventRecord(L.ev, L.stream) == cudaSuccess ? MG_OK : MG_ECUDA;
    if (!rc) L.busy = true;
    return rc;
}

// A step or a set-up failed: every admitted and queued request ends with the
// error; the handles of the admitted ones are destroyed (their device state
// is not trusted after a failure) and their bytes released.
void mg_server::fail_all(int rc)
{
    for (int k = 0; k < nlanes; k++) cudaStreamSynchronize(lanes[k].stream);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(mu);
    loop_error = rc;
    for (int k = 0; k < nlanes; k++) {
        Lane &L = lanes[k];
        L.running.insert(L.running.end(), L.pending.begin(), L.pending.end());
        for (Request *r : L.running) {
            r->done = true;
            r->status = rc;
            r->st.status = rc;
            if (r->h) {
                bytes_in_use -= r->h->bytes;
                mg_destroy(r->h);
                r->h = nullptr;
            }
            completed++;
            in_flight--;
        }
        L.running.clear();
        L.pending.clear();
        L.busy = false;
        L.changed = true;
        L.fresh = false;
    }
    for (Request *r : queue) {
        r->done = true;
        r->status = rc;
        r->st.status = rc;
        completed++;
    }
    queue.clear();
    cv_done.notify_all();
}

void mg_server::loop()
{
    cudaSetDevice(device);
    for (;;) {
        std::vector<Request *> fresh;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty() || in_flight > 0; });
            if (stop && queue.empty() && in_flight == 0) break;
            admit_locked(fresh);
        }
        int rc = start_fresh(fresh);
        bool stepped = false, waiting = false;
        for (int k = 0; k < nlanes && !rc; k++) {
            Lane &L = lanes[k];
            if (L.busy) {
                const cudaError_t q = cudaEventQuery(L.ev);
                if (q == cudaErrorNotReady) {
                    waiting = true;
                    continue;
                }
                L.busy = false;
                if (q != cudaSuccess) {
                    rc = MG_ECUDA;
                    break;
                }
                rc = finish_lane(L);
            }
            if (!rc && (!L.running.empty() || !L.pending.empty())) {
                rc = step_lane(L);
                stepped = true;
            }
        }
        if (rc) {
            fail_all(rc);
            continue;
        }
        if (!stepped && waiting) {
            // every lane with work has a step in flight: sleep briefly (a
            // submission wakes the loop at once)
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        } else if (!stepped && !waiting) {
            // nothing fits yet and nothing runs: wait for the next event
            std::unique_lock<std::mutex> lk(mu);
            if (!queue.empty()) cv_work.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
    release_lanes();
}

void mg_server::release_lanes()
{
    for (int k = 0; k < nlanes; k++) {
        Lane &L = lanes[k];
        if (L.plan) {
            if (L.plan->capture_stream) cudaStreamDestroy(L.plan->capture_stream);
            L.plan->release();
            delete L.plan;
            L.plan = nullptr;
        }
    }
}

extern "C" {

int mg_server_create(size_t hbm_budget_bytes, int max_slots, const mg_params *params, void *stream,
                     mg_server **out)
{
    if (!out || max_slots < 1 || hbm_budget_bytes == 0) return MG_EINVAL;
    mg_server *s = new (std::nothrow) mg_server();
    if (!s) return MG_ENOMEM;
    mg_params_default(&s->prm);
    if (params) s->prm = *params;
    if (check_params(&s->prm)) {
        delete s;
        return MG_EINVAL;
    }
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return MG_ECUDA;
    }
    int ok = 1;
    if (stream) {
        // the caller's stream: one lane, every request stepped together
        s->nlanes = 1;
        s->lanes[0].stream = (cudaStream_t)stream;
    } else {
        // a stream per lane; smaller grids at a higher priority (numerically lower)
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) ok = 0;
        s->own_streams = true;
        for (int k = 0; k < s->nlanes && ok; k++) {
            const int prio = std::min(least, greatest + k);
            if (cudaStreamCreateWithPriority(&s->lanes[k].stream, cudaStreamNonBlocking, prio) != cudaSuccess)
                ok = 0;
        }
    }
    for (int k = 0; k < s->nlanes && ok; k++)
        if (cudaEventCreateWithFlags(&s->lanes[k].ev, cudaEventDisableTiming) != cudaSuccess) ok = 0;
    if (const char *f = getenv("MG_SERVER_FAIL_AT_STEP")) s->fail_at = atoll(f);
    if (!ok) {
        for (int k = 0; k < kLanes; k++) {
            if (s->lanes[k].ev) cudaEventDestroy(s->lanes[k].ev);
            if (s->own_streams && s->lanes[k].stream) cudaStreamDestroy(s->lanes[k].stream);
        }
        delete s;
        return MG_ECUDA;
    }
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return MG_OK;
}

int mg_submit(mg_server *s, const mg_grid *grid, const double *ax, const double *ay, const double *az,
              const double *rhs, double *p, double tol, mg_ticket *out)
{
    if (!s || !grid || !ax || !ay || !az || !rhs || !p || !out || !(tol >= 0.0)) return MG_EINVAL;
    size_t bytes = 0;
    int rc = mg_memory_estimate(grid, &s->prm, &bytes);
    if (rc) return rc;
    if (bytes > s->budget) return MG_EBUDGET;
    Request *r = new (std::nothrow) Request();
    if (!r) return MG_ENOMEM;
    r->grid = *grid;
    r->ax = ax;
    r->ay = ay;
    r->az = az;
    r->rhs = rhs;
    r->p = p;
    r->tol = tol;
    r->bytes = bytes;
    r->lane = lane_of(*grid, s->nlanes);
    r->t_submit = Clock::now();
    memset(&r->st, 0, sizeof(r->st));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        s->queue.push_back(r);
        s->tickets[r->id] = r;
    }
    s->cv_work.notify_one();
    *out = r->id;
    return MG_OK;
}

int mg_poll(mg_server *s, mg_ticket t, mg_stats *st)
{
    if (!s) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(t);
    if (it == s->tickets.end()) return MG_ENOTFOUND;
    Request *r = it->second;
    if (!r->done) return MG_EAGAIN;
    if (st) *st = r->st;
    int status = r->status;
    s->tickets.erase(it);
    delete r;
    return status;
}

int mg_server_drain(mg_server *s)
{
    if (!s) return MG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->in_flight == 0; });
    return s->loop_error;
}

int mg_server_info(mg_server *s, int64_t *completed, size_t *bytes_in_use, size_t *peak_bytes,
                   int *max_in_flight)
{
    if (!s) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
    if (peak_bytes) *peak_bytes = s->peak;
    if (max_in_flight) *max_in_flight = s->max_in_flight;
    return MG_OK;
}

int mg_server_destroy(mg_server *s)
{
    if (!s) return MG_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->queue.empty() || s->in_flight > 0) return MG_EBUSY;
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->cache) mg_destroy(kv.second);
    s->cache.clear();
    for (auto &kv : s->tickets) delete kv.second;
    s->tickets.clear();
    for (int k = 0; k < kLanes; k++) {
        if (s->lanes[k].ev) cudaEventDestroy(s->lanes[k].ev);
        if (s->own_streams && s->lanes[k].stream) cudaStreamDestroy(s->lanes[k].stream);
    }
    delete s;
    return MG_OK;
}

}  // extern "C"
