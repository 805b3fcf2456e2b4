// smi_server.cu -- continuous-batching request server over the C ABI.
//
// Requests (forward modelling, RTM images, FWI gradients of any size,
// dimension and nt) are queued in arrival order.  A request is admitted into
// one of the server's slots as soon as a slot is free and its device
// footprint (smi_query) fits in the remaining memory budget; each slot owns a
// CUDA stream and a host thread, so admitted requests run concurrently on the
// GPU while later ones wait.  A request that can never fit (footprint above
// the whole budget) fails with SMI_ERR_NOMEM instead of blocking the queue.
// This is the GPU counterpart of the paper's batchwise job scheduling
// (Sec. 4.3) and of its one-process-per-shot parallelism (Sec. 3.2).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/smi.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    long long ticket;
    smi_request req;
    size_t bytes = 0;
    int state = 0;            // 0 queued, 1 running, 2 done
    int status = SMI_OK;
    std::string error;
    double t_submit = 0, t_start = 0, t_end = 0;   // seconds since server start
};

}  // namespace

struct smi_server {
    size_t budget = 0, in_use = 0;
    int slots = 1;
    int device = 0;               // device current at creation: the workers run their requests there
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<long long> queue;
    std::map<long long, Job> jobs;
    long long next_ticket = 1;
    std::vector<std::thread> workers;
    Clock::time_point t0 = Clock::now();
    long long completed = 0, failed = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // First queued job that fits (FIFO among those that fit); -1 if none.
    long long pick()
    {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Job &j = jobs[*it];
            if (j.bytes <= budget - in_use) {
                const long long t = *it;
                queue.erase(it);
                return t;
            }
        }
        return -1;
    }

    void worker()
    {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            long long t = -1;
            Job job;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || (t = pick()) >= 0; });
                if (t < 0) break;                      // stopping with nothing runnable
                Job &j = jobs[t];
                j.state = 1;
                j.t_start = now();
                in_use += j.bytes;
                job = j;
            }
            smi_request r = job.req;
            r.opts.stream = st;
            int rc;
            if (r.kind == 0) rc = smi_forward(&r.model, &r.geom, &r.wav, &r.opts, r.out);
            else if (r.kind == 1) rc = smi_rtm(&r.model, &r.geom, &r.wav, &r.opts, r.dobs, r.out);
            else rc = smi_fwi_gradient(&r.model, &r.geom, &r.wav, &r.opts, r.dobs, r.misfit, r.out);
            const std::string err = rc ? smi_last_error() : "";
            {
                std::lock_guard<std::mutex> lk(mu);
                Job &j = jobs[t];
                j.state = 2;
                j.status = rc;
                j.error = err;
                j.t_end = now();
                in_use -= j.bytes;
                if (rc) failed++;
                else completed++;
            }
            cv_done.notify_all();
            cv_work.notify_all();                      // memory freed: others may fit now
        }
        cudaStreamDestroy(st);
    }
};

extern "C" {

smi_server *smi_server_create(size_t budget_bytes, int slots)
{
    if (slots < 1) slots = 1;
    auto *s = new smi_server();
    if (budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        budget_bytes = (size_t)(0.8 * (double)free_b);
    }
    cudaGetDevice(&s->device);
    s->budget = budget_bytes;
    s->slots = slots;
    for (int k = 0; k < slots; k++) s->workers.emplace_back([s] { s->worker(); });
    return s;
}

int smi_submit(smi_server *s, const smi_request *req, long long *ticket)
{
    if (!s || !req || !ticket) return SMI_ERR_ARG;
    if (req->kind < 0 || req->kind > 2) return SMI_ERR_ARG;
    size_t bytes = 0;
    const int rc = smi_query(&req->model, &req->geom, &req->wav, &req->opts, req->kind, nullptr, nullptr, &bytes);
    std::lock_guard<std::mutex> lk(s->mu);
    const long long t = s->next_ticket++;
    Job &j = s->jobs[t];
    j.ticket = t;
    j.req = *req;
    j.bytes = bytes;
    j.t_submit = s->now();
    *ticket = t;
    if (rc || bytes > s->budget) {         // invalid, or can never fit: fail now
        j.state = 2;
        j.status = rc ? rc : SMI_ERR_NOMEM;
        j.error = rc ? smi_last_error() : "request footprint exceeds the server's memory budget";
        j.t_start = j.t_end = j.t_submit;
        s->failed++;
        s->cv_done.notify_all();
        return SMI_OK;
    }
    s->queue.push_back(t);
    s->cv_work.notify_one();
    return SMI_OK;
}

int smi_wait(smi_server *s, long long ticket, double timeout_s, smi_result *res)
{
    if (!s) return SMI_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->jobs.find(ticket) == s->jobs.end()) return SMI_ERR_ARG;
    // a finished job leaves the map once its result is returned, so a waiter
    // that wakes up to find it gone lost the race to another waiter
    const auto done = [&] {
        auto f = s->jobs.find(ticket);
        return f == s->jobs.end() || f->second.state == 2;
    };
    if (timeout_s < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return SMI_ERR_TIMEOUT;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return SMI_ERR_ARG;
    const Job &j = it->second;
    if (res) {
        res->status = j.status;
        res->device_bytes = j.bytes;
        res->t_submit = j.t_submit;
        res->t_start = j.t_start;
        res->t_end = j.t_end;
        strncpy(res->error, j.error.c_str(), sizeof res->error - 1);
        res->error[sizeof res->error - 1] = 0;
    }
    s->jobs.erase(it);                // the result is delivered: release the ticket
    return SMI_OK;
}

int smi_poll(smi_server *s, long long ticket, int *state)
{
    if (!s || !state) return SMI_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return SMI_ERR_ARG;
    *state = it->second.state;
    return SMI_OK;
}

int smi_cancel(smi_server *s, long long ticket)
{
    if (!s) return SMI_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == ticket) {
            s->queue.erase(it);
            Job &j = s->jobs[ticket];
            j.state = 2;
            j.status = SMI_ERR_ARG;
            j.error = "cancelled";
            j.t_start = j.t_end = s->now();
            s->cv_done.notify_all();
            return SMI_OK;
        }
    return SMI_ERR_ARG;       // unknown, running or finished: not cancellable
}

int smi_server_info(smi_server *s, size_t *budget, size_t *in_use, long long *queued, long long *completed,
                    long long *failed)
{
    if (!s) return SMI_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (budget) *budget = s->budget;
    if (in_use) *in_use = s->in_use;
    if (queued) *queued = (long long)s->queue.size();
    if (completed) *completed = s->completed;
    if (failed) *failed = s->failed;
    return SMI_OK;
}

void smi_server_destroy(smi_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (long long t : s->queue) {         // unstarted requests are dropped
            Job &j = s->jobs[t];
            j.state = 2;
            j.status = SMI_ERR_ARG;
            j.error = "server destroyed";
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &w : s->workers) w.join();
    delete s;
}

}  // extern "C"
