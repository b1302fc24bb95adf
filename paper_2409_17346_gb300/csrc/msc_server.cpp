// Serving runtime: a request loop with continuous batching over the fix-loop library.
//
// Jobs are queued by msc_server_submit and admitted by memory: a slot (a host thread with
// its own non-blocking CUDA stream) takes the first queued job whose device bytes fit in
// what the budget has left, runs prepare + fix for it with all of its state resident on the
// device, and frees that state when the job ends.  Slots run concurrently, so the edit
// rounds of different jobs overlap on the GPU; a job that arrives while others run is
// admitted as soon as a slot and enough memory are free.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/msc.h"
#include "msc_runtime.h"

namespace {

struct Job {
    uint64_t id = 0;
    const float *f = nullptr, *fh = nullptr;
    float *g_out = nullptr;
    int nx = 0, ny = 0, nz = 0;
    float xi = 0.f;
    uint64_t bytes = 0;
    int skips = 0;
    bool running = false;
    bool done = false;
    std::atomic<int> cancel{0};
    msc_status status = MSC_OK;
    std::string err;
    msc_edits edits{};
    msc_job_info info{};
};

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct msc_server {
    msc_server_config cfg{};
    int dev = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t reserved = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> slots;

    // first queued job that fits (caller holds mu); a job passed over max_skips times
    // blocks the queue until it fits itself
    std::deque<Job *>::iterator pick()
    {
        for (auto it = pending.begin(); it != pending.end(); ++it) {
            if (reserved + (*it)->bytes <= cfg.mem_budget) return it;
            if ((*it)->skips >= cfg.max_skips) break;
        }
        return pending.end();
    }

    void run_slot(int slot)
    {
        cudaStream_t ws = nullptr;
        cudaError_t ce = cudaSetDevice(dev);
        if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
        for (;;) {
            Job *j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || pick() != pending.end(); });
                if (stop) break;
                auto it = pick();
                for (auto jt = pending.begin(); jt != it; ++jt) (*jt)->skips++;
                j = *it;
                pending.erase(it);
                reserved += j->bytes;
                j->running = true;
            }
            j->info.slot = slot;
            j->info.t_start = seconds_since(t0);
            msc_status st = MSC_OK;
            if (ce != cudaSuccess) {
                st = msc_rt::set_error(MSC_ERR_CUDA, std::string("slot stream: ") + cudaGetErrorString(ce));
            } else {
                msc_options o = cfg.options;
                o.stream = ws;
                msc_handle *h = nullptr;
                msc_rt::set_cancel_flag(&j->cancel);
                if (j->cancel.load()) st = msc_rt::set_error(MSC_ERR_CANCELLED, "the job was cancelled");
                else st = msc_prepare_original(j->f, j->nx, j->ny, j->nz, &o, &h);
                msc_rt::share_device(h, cfg.max_jobs);
                if (st == MSC_OK) st = msc_fix(h, j->fh, j->xi, &o, &j->edits, j->g_out);
                msc_rt::set_cancel_flag(nullptr);
                std::string e = st == MSC_OK ? std::string() : std::string(msc_last_error());
                msc_destroy(h);
                if (st != MSC_OK) msc_rt::set_error(st, e);
            }
            j->info.t_end = seconds_since(t0);
            j->info.status = st;
            j->info.loop_ms = j->edits.loop_ms;
            {
                std::lock_guard<std::mutex> lk(mu);
                j->status = st;
                if (st != MSC_OK) j->err = msc_last_error();
                j->done = true;
                reserved -= j->bytes;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        if (ws) cudaStreamDestroy(ws);
    }
};

extern "C" {

msc_status msc_server_create(const msc_server_config *cfg, msc_server **out)
{
    if (!out) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    msc_server_config c{};
    if (cfg) c = *cfg;
    else {
        c.max_jobs = 8;
        msc_default_options(&c.options);
    }
    if (c.max_jobs < 1 || c.max_jobs > 64) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "max_jobs must be in 1..64");
    if (c.max_skips < 0) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "max_skips must be >= 0");
    if (c.max_skips == 0) c.max_skips = 16;
    int dev = 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return msc_rt::set_error(MSC_ERR_NO_DEVICE, "no CUDA device available");
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return msc_rt::set_error(MSC_ERR_CUDA, "cudaGetDevice failed");
    if (c.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return msc_rt::set_error(MSC_ERR_CUDA, "cudaMemGetInfo failed");
        c.mem_budget = (uint64_t)(0.9 * (double)fr);
    }
    // keep freed job memory (up to the budget) in the library's pool for the next job
    msc_rt::limit_cached_memory(c.mem_budget);
    msc_server *s = new (std::nothrow) msc_server();
    if (!s) return msc_rt::set_error(MSC_ERR_OOM, "server allocation failed");
    s->cfg = c;
    s->dev = dev;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < c.max_jobs; i++) s->slots.emplace_back([s, i] { s->run_slot(i); });
    *out = s;
    return MSC_OK;
}

msc_status msc_server_submit(msc_server *srv, const float *f, const float *f_hat, int nx, int ny, int nz, float xi,
                             float *g_out, uint64_t *ticket)
{
    if (!srv || !f || !f_hat || !g_out || !ticket)
        return msc_rt::set_error(MSC_ERR_INVALID_ARG, "server, f, f_hat, g_out and ticket must be non-NULL");
    if (nx < 2 || ny < 2 || nz < 1) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "dims must satisfy nx, ny >= 2 and nz >= 1");
    if (!(xi > 0.0f) || !(xi < 3.4e38f)) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "xi must be finite and > 0");
    const uint64_t bytes = msc_device_bytes(nx, ny, nz);
    if (bytes > srv->cfg.mem_budget)
        return msc_rt::set_error(MSC_ERR_OOM, "job needs " + std::to_string(bytes) + " device bytes, budget is " +
                                                  std::to_string(srv->cfg.mem_budget));
    Job *j = new (std::nothrow) Job();
    if (!j) return msc_rt::set_error(MSC_ERR_OOM, "job allocation failed");
    j->f = f;
    j->fh = f_hat;
    j->g_out = g_out;
    j->nx = nx; j->ny = ny; j->nz = nz;
    j->xi = xi;
    j->bytes = bytes;
    j->info.bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        j->id = srv->next_id++;
        j->info.t_submit = seconds_since(srv->t0);
        srv->jobs[j->id] = j;
        srv->pending.push_back(j);
    }
    srv->cv_work.notify_all();
    *ticket = j->id;
    return MSC_OK;
}

msc_status msc_server_wait(msc_server *srv, uint64_t ticket, msc_edits *out, msc_job_info *info)
{
    if (!srv) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "server is NULL");
    Job *j = nullptr;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(ticket);
        if (it == srv->jobs.end()) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "unknown ticket");
        j = it->second;
        srv->cv_done.wait(lk, [&] { return j->done; });
        srv->jobs.erase(it);
    }
    if (out) *out = j->edits;
    else msc_free_edits(&j->edits);
    if (info) *info = j->info;
    const msc_status st = j->status;
    if (st != MSC_OK) msc_rt::set_error(st, j->err);
    delete j;
    return st;
}

msc_status msc_server_cancel(msc_server *srv, uint64_t ticket)
{
    if (!srv) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(ticket);
        if (it == srv->jobs.end()) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "unknown ticket");
        Job *j = it->second;
        if (j->done) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "the job has already ended");
        j->cancel.store(1);
        if (!j->running) {                      // still queued: it never starts
            srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), j));
            j->status = MSC_ERR_CANCELLED;
            j->err = "the job was cancelled before it started";
            j->info.status = MSC_ERR_CANCELLED;
            j->info.slot = -1;
            j->info.t_start = j->info.t_end = seconds_since(srv->t0);
            j->done = true;
        }
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    return MSC_OK;
}

void msc_server_destroy(msc_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->slots) t.join();
    for (auto &kv : srv->jobs) {
        msc_free_edits(&kv.second->edits);
        delete kv.second;
    }
    delete srv;
}

}  // extern "C"
