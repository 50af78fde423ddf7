// mg_server.cu -- continuous-batching request loop of the pressure multigrid.
//
// A host thread admits queued solves while slots and the device-memory budget
// allow, reuses the hierarchy of a finished request for a later request of the
// same grid, and advances all admitted requests together one V-cycle at a time
// (one launch per V-cycle stage for the whole set).  Requests join and leave
// between cycles.  Every grid's arithmetic is independent of the other grids in
// the launch, so a request's result is bitwise the same alone and in the mix.
#include <string.h>

#include <new>

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

struct Request {
    mg_ticket id;
    mg_grid grid;
    const double *ax, *ay, *az, *rhs;
    double *p;
    double tol;
    size_t bytes;
    Clock::time_point t_submit;
    mg_handle *h = nullptr;
    bool done = false;
    int status = MG_EAGAIN;
    mg_stats st;
};

using GridKey = std::tuple<int, int, int, double, double, double, int, int, int>;

GridKey key_of(const mg_grid &g)
{
    return GridKey(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, g.bc[0], g.bc[1], g.bc[2]);
}

}  // namespace

struct mg_server {
    size_t budget = 0;
    int max_slots = 1;
    mg_params prm;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<mg_ticket, Request *> tickets;
    std::multimap<GridKey, mg_handle *> cache;
    size_t bytes_in_use = 0, peak = 0;
    int64_t completed = 0;
    int max_in_flight = 0;
    mg_ticket next_id = 1;
    bool stop = false;
    int loop_error = MG_OK;
    std::thread th;
    Plan *plan = nullptr;   // plan over `running`; rebuilt when membership changes

    void loop();
    int admit_locked(std::vector<Request *> &fresh);
    void retire(std::vector<Request *> &finished);
    void drop_plan()
    {
        if (plan) {
            if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
            plan->release();
            delete plan;
            plan = nullptr;
        }
    }
};

// Move queued requests into slots while slots and budget allow (FIFO; a
// request that does not fit yet blocks the ones behind it, so large requests
// are not starved).  Called with the lock held.
int mg_server::admit_locked(std::vector<Request *> &fresh)
{
    while (!queue.empty() && (int)running.size() < max_slots) {
        Request *r = queue.front();
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
            int rc = handle_alloc(&r->grid, &prm, stream, &h);
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
        running.push_back(r);
        fresh.push_back(r);
    }
    max_in_flight = std::max(max_in_flight, (int)running.size());
    return MG_OK;
}

void mg_server::retire(std::vector<Request *> &finished)
{
    auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (Request *r : finished) {
        int herr[3] = {0, 0, 0};
        cudaMemcpy(herr, r->h->err, sizeof(herr), cudaMemcpyDeviceToHost);
        GridState s;
        cudaMemcpy(&s, r->h->state, sizeof(s), cudaMemcpyDeviceToHost);
        const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
        fill_stats(s, herr, ms, &r->st, &r->status);
        r->done = true;
        cache.emplace(key_of(r->grid), r->h);
        r->h = nullptr;
        completed++;
        for (size_t q = 0; q < running.size(); q++)
            if (running[q] == r) {
                running.erase(running.begin() + q);
                break;
            }
    }
    cv_done.notify_all();
}

void mg_server::loop()
{
    cudaSetDevice(device);
    bool changed = true;
    for (;;) {
        std::vector<Request *> fresh;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty() || !running.empty(); });
            if (stop && queue.empty() && running.empty()) break;
            admit_locked(fresh);
            if (!fresh.empty()) changed = true;
            if (running.empty()) {
                // nothing fits yet and nothing runs: wait for the next event
                if (!queue.empty()) cv_work.wait_for(lk, std::chrono::milliseconds(1));
                continue;
            }
        }
        int rc = MG_OK;
        // start the new requests with their own single-grid plans (state lives in the handle)
        for (Request *r : fresh) {
            Plan &sp = *r->h->plan;
            plan_bind(sp, 0, r->rhs, r->p, r->tol, prm.max_iters);
            if (!rc) rc = plan_upload(sp);
            if (!rc) rc = plan_prologue(sp);
        }
        if (changed) {
            // the plan is allocated once for max_slots grids; a change of the
            // running set only rewrites its tables (asynchronously, no allocation)
            if (!plan) {
                plan = new (std::nothrow) Plan();
                if (!plan) rc = MG_ENOMEM;
                else if (!rc) rc = plan->alloc(max_slots);
            }
            std::vector<mg_handle *> hs;
            for (Request *r : running) hs.push_back(r->h);
            if (!rc) rc = plan->fill(hs.data(), (int)hs.size());
            for (size_t g = 0; g < running.size() && !rc; g++)
                plan_bind(*plan, (int)g, running[g]->rhs, running[g]->p, running[g]->tol, prm.max_iters);
            if (!rc) rc = plan_upload(*plan);
            changed = false;
        }
        if (!rc) rc = plan_sync_states(*plan);
        std::vector<Request *> finished;
        if (!rc) {
            for (size_t g = 0; g < running.size(); g++)
                if (!plan->st_h[g].active) finished.push_back(running[g]);
            bool any_active = finished.size() < running.size();
            if (any_active) rc = plan_body(*plan);
        }
        for (Request *r : finished) {
            if (!rc) rc = plan_final(*r->h->plan);
        }
        if (!finished.empty()) {
            if (!rc) rc = cudaStreamSynchronize(stream) == cudaSuccess ? MG_OK : MG_ECUDA;
            retire(finished);
            changed = true;
        }
        if (rc) {
            std::lock_guard<std::mutex> lk(mu);
            loop_error = rc;
            for (Request *r : running) {
                r->done = true;
                r->status = rc;
                r->st.status = rc;
                completed++;
            }
            running.clear();
            for (Request *r : queue) {
                r->done = true;
                r->status = rc;
                r->st.status = rc;
                completed++;
            }
            queue.clear();
            cv_done.notify_all();
            changed = true;
        }
    }
    drop_plan();
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
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return MG_ECUDA;
        }
        s->own_stream = true;
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
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running.empty(); });
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
        if (!s->queue.empty() || !s->running.empty()) return MG_EBUSY;
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->cache) mg_destroy(kv.second);
    s->cache.clear();
    for (auto &kv : s->tickets) delete kv.second;
    s->tickets.clear();
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return MG_OK;
}

}  // extern "C"
