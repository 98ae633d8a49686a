// Serving: independent VBC simulations admitted by a device-memory budget and
// advanced in chunks on slot threads, each with its own CUDA stream.  A client
// of the public C ABI (vbc.h) only: every kernel it runs is the library's.

#include "vbc.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

struct Request {
    int64_t id = 0;
    vbc_config cfg{};
    std::vector<double> pos, vel;  // inputs; the final state once finished
    bool has_vel = false;
    int64_t nsteps = 0;
    double dt = 0, kT = 0, gamma = 0;
    vbc_request_info info{};
    std::string error;
};

using Clock = std::chrono::steady_clock;

}  // namespace

struct vbc_server {
    vbc_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;  // slots: a request may be admissible, or stop
    std::condition_variable cv_done;  // waiters: a request finished
    std::deque<std::shared_ptr<Request>> queue;             // arrival order, not yet admitted
    std::map<int64_t, std::shared_ptr<Request>> requests;   // every request until its result is taken
    int64_t reserved = 0;  // device bytes reserved by admitted requests
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> slots;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    bool finished(const Request& r) const { return r.info.status <= 0; }
    // the head of the queue fits the budget (callers hold mu)
    bool admissible() const
    {
        return !queue.empty() && reserved + queue.front()->info.device_bytes <= cfg.hbm_budget;
    }
    void slot_main();
    int run(Request& r, cudaStream_t stream);
};

namespace {

thread_local std::string g_serve_err;

int serve_fail(int code, const char* msg)
{
    g_serve_err = msg;
    return code;
}

}  // namespace

// One request on one slot: create on the slot's stream, step in chunks,
// copy the state out, release.  Returns VBC_OK or the first error.
int vbc_server::run(Request& r, cudaStream_t stream)
{
    vbc_config c = r.cfg;
    c.pos = r.pos.data();
    c.vel = r.has_vel ? r.vel.data() : nullptr;
    c.stream = (void*)stream;
    c.inputs_on_device = 0;
    vbc_system* s = nullptr;
    int rc = vbc_create_system(&c, &s);
    if (rc != VBC_OK) {
        r.error = vbc_last_error();
        return rc;
    }
    const auto refresh_reservation = [&]() {
        vbc_stats st{};
        if (vbc_get_stats(s, &st) != VBC_OK) return;
        std::lock_guard<std::mutex> lock(mu);
        // the live figure replaces the estimate; a grown system keeps its larger reservation
        const int64_t b = std::max<int64_t>(st.device_bytes, 1);
        reserved += b - r.info.device_bytes;
        r.info.device_bytes = b;
    };
    refresh_reservation();
    int64_t done = 0;
    while (done < r.nsteps) {
        {
            std::lock_guard<std::mutex> lock(mu);
            if (stop) break;
        }
        const int64_t k = std::min<int64_t>(cfg.chunk_steps, r.nsteps - done);
        rc = vbc_step_langevin(s, k, r.dt, r.kT, r.gamma);
        if (rc != VBC_OK) break;
        done += k;
        refresh_reservation();
        std::lock_guard<std::mutex> lock(mu);
        r.info.steps_done = done;
    }
    if (rc == VBC_OK) {
        int64_t step = 0;
        r.vel.resize(r.pos.size());
        rc = vbc_get_state(s, r.pos.data(), r.vel.data(), &step, 0);
    }
    if (rc != VBC_OK) r.error = vbc_last_error();
    vbc_destroy(s);
    return rc;
}

void vbc_server::slot_main()
{
    cudaSetDevice(device);
    cudaStream_t stream = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait(lock, [&] { return stop || admissible(); });
            if (stop) break;
            r = queue.front();
            queue.pop_front();
            reserved += r->info.device_bytes;
            r->info.status = VBC_REQ_RUNNING;
            r->info.t_admit = now();
        }
        cv_work.notify_all();  // the next head may fit as well
        int rc = have_stream ? run(*r, stream) : VBC_ERR_CUDA;
        if (!have_stream) r->error = "cudaStreamCreate failed on a serving slot";
        {
            std::lock_guard<std::mutex> lock(mu);
            reserved -= r->info.device_bytes;
            if (rc == VBC_OK && r->info.steps_done < r->nsteps) {  // stopped by vbc_server_destroy
                rc = VBC_ERR_CANCELLED;
                r->error = "stopped: the server was destroyed";
            }
            r->info.t_done = now();
            r->info.status = rc;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    if (have_stream) cudaStreamDestroy(stream);
}

extern "C" {

int vbc_server_create(const vbc_server_config* cfg, vbc_server** out)
{
    if (!cfg || !out) return serve_fail(VBC_ERR_INVALID_ARG, "cfg and out must not be NULL");
    *out = nullptr;
    if (cfg->hbm_budget <= 0 || cfg->slots < 1 || cfg->slots > 256 || cfg->chunk_steps <= 0)
        return serve_fail(VBC_ERR_INVALID_ARG, "need hbm_budget > 0, 1 <= slots <= 256, chunk_steps > 0");
    auto* srv = new vbc_server();
    srv->cfg = *cfg;
    srv->t0 = Clock::now();
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return serve_fail(VBC_ERR_CUDA, "no CUDA device");
    }
    for (int k = 0; k < cfg->slots; ++k) srv->slots.emplace_back([srv] { srv->slot_main(); });
    *out = srv;
    return VBC_OK;
}

int vbc_server_submit(vbc_server* srv, const vbc_request* req, int64_t* id)
{
    if (!srv || !req || !id) return serve_fail(VBC_ERR_INVALID_ARG, "srv, req and id must not be NULL");
    if (req->nsteps < 0 || !(req->dt > 0) || !std::isfinite(req->dt) || !(req->kT >= 0) ||
        !std::isfinite(req->kT) || !(req->gamma >= 0) || !std::isfinite(req->gamma))
        return serve_fail(VBC_ERR_INVALID_ARG, "need nsteps >= 0, dt > 0, kT >= 0, gamma >= 0 (finite)");
    if (!req->system.pos) return serve_fail(VBC_ERR_INVALID_ARG, "pos must not be NULL");
    int64_t est = 0;
    int rc = vbc_estimate_device_bytes(&req->system, &est);
    if (rc != VBC_OK) return serve_fail(rc, vbc_last_error());
    if (est > srv->cfg.hbm_budget) return serve_fail(VBC_ERR_OOM, "the system alone needs more than the budget");
    auto r = std::make_shared<Request>();
    r->cfg = req->system;
    const size_t n3 = 3 * (size_t)req->system.n;
    r->pos.assign(req->system.pos, req->system.pos + n3);
    if (req->system.vel) {
        r->vel.assign(req->system.vel, req->system.vel + n3);
        r->has_vel = true;
    }
    r->nsteps = req->nsteps;
    r->dt = req->dt;
    r->kT = req->kT;
    r->gamma = req->gamma;
    r->info.status = VBC_REQ_QUEUED;
    r->info.n = req->system.n;
    r->info.device_bytes = std::max<int64_t>(est, 1);
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        r->id = srv->next_id++;
        r->info.t_submit = srv->now();
        srv->queue.push_back(r);
        srv->requests[r->id] = r;
        *id = r->id;
    }
    srv->cv_work.notify_all();
    return VBC_OK;
}

int vbc_server_wait(vbc_server* srv, int64_t id, double timeout_s, vbc_request_info* info)
{
    if (!srv) return serve_fail(VBC_ERR_INVALID_ARG, "srv must not be NULL");
    std::unique_lock<std::mutex> lock(srv->mu);
    std::function<bool()> ready;
    std::shared_ptr<Request> r;
    if (id == -1) {
        ready = [&] {
            for (auto& kv : srv->requests)
                if (!srv->finished(*kv.second)) return false;
            return true;
        };
    } else {
        auto it = srv->requests.find(id);
        if (it == srv->requests.end()) return serve_fail(VBC_ERR_INVALID_ARG, "unknown request id");
        r = it->second;
        ready = [&] { return srv->finished(*r); };
    }
    if (timeout_s < 0) {
        srv->cv_done.wait(lock, ready);
    } else if (!srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)) {
        return serve_fail(VBC_ERR_TIMEOUT, "the request has not finished yet");
    }
    if (info && r) *info = r->info;
    return VBC_OK;
}

int vbc_server_info(vbc_server* srv, int64_t id, vbc_request_info* info)
{
    if (!srv || !info) return serve_fail(VBC_ERR_INVALID_ARG, "srv and info must not be NULL");
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->requests.find(id);
    if (it == srv->requests.end()) return serve_fail(VBC_ERR_INVALID_ARG, "unknown request id");
    *info = it->second->info;
    return VBC_OK;
}

int vbc_server_result(vbc_server* srv, int64_t id, double* pos, double* vel, vbc_request_info* info)
{
    if (!srv) return serve_fail(VBC_ERR_INVALID_ARG, "srv must not be NULL");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        auto it = srv->requests.find(id);
        if (it == srv->requests.end()) return serve_fail(VBC_ERR_INVALID_ARG, "unknown request id");
        if (!srv->finished(*it->second)) return serve_fail(VBC_ERR_INVALID_ARG, "the request has not finished");
        r = it->second;
        srv->requests.erase(it);
    }
    if (info) *info = r->info;
    if (r->info.status != VBC_OK) return serve_fail(r->info.status, r->error.c_str());
    const size_t n3 = 3 * (size_t)r->info.n;
    if (pos) std::memcpy(pos, r->pos.data(), n3 * sizeof(double));
    if (vel) std::memcpy(vel, r->vel.data(), n3 * sizeof(double));
    return VBC_OK;
}

void vbc_server_destroy(vbc_server* srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        for (auto& r : srv->queue) {
            r->info.status = VBC_ERR_CANCELLED;
            r->error = "dropped: the server was destroyed";
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->slots) t.join();
    srv->cv_done.notify_all();
    delete srv;
}

const char* vbc_server_last_error(void) { return g_serve_err.c_str(); }

}  // extern "C"
