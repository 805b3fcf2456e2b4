// smi_server.cu -- continuous-batching request server over the C ABI.
//
// Requests (forward modelling, RTM images, FWI gradients of any size,
// dimension and nt) are queued in arrival order.  A request is admitted into
// one of the server's slots as soon as a slot is free and its device
// footprint (smi_query) fits in the remaining memory budget; each slot owns a
// CUDA stream and a host thread, so admitted requests run concurrently on the
// GPU while later ones wait.  A request that can never fit (footprint above
// the whole budget) fails with SMI_ERR_NOMEM instead of blocking the queue.
// Single-shot requests that can share one call -- same kind, model arrays,
// wavelet and options, i.e. shots of one survey -- are taken together when a
// slot admits the first of them, while one launch over all of them would not
// yet fill the GPU (2^24 grid points): their shots are concatenated into one
// shot-batched call (the shots share every launch, blockIdx.z = shot) with
// per-shot results (opts.per_shot), which are then copied to each request's
// own outputs.  This is the GPU counterpart of the paper's batchwise job
// scheduling (Sec. 4.3) and of its one-process-per-shot parallelism (Sec. 3.2).
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

constexpr int kMaxMerge = 64;                 // shots of one merged call
constexpr long long kMergePoints = 1LL << 24;  // extended grid points of all shots of a merged call

// Extended grid points of one shot of a request (the work of one of its
// launches): shots are merged only while their sum stays below
// kMergePoints, i.e. while one launch over all of them does not yet fill the
// GPU on its own -- a 2D shot (about 0.7 M points) joins up to ~20 others, a
// 300^3 shot none.
long long shot_points(const smi_request &r)
{
    const long long e = 2LL * r.opts.nb;
    long long n = (r.model.n1 + e) * (long long)(r.model.n2 + e);
    if (r.model.ndim == 3) n *= r.model.n3 + e;
    return n;
}

// A request that may join a merged call: one shot, and a kind with per-shot results.
bool mergeable(const smi_request &r)
{
    return r.geom.nshot == 1 && (r.kind == 0 || r.kind == 2 || (r.kind == 1 && !r.opts.img_norm)) &&
           !r.opts.per_shot;
}

// Two requests that one call can run: same kind, model arrays, wavelet and
// options (the stream aside).
bool same_call(const smi_request &a, const smi_request &b)
{
    const smi_model &p = a.model, &q = b.model;
    const smi_opts &u = a.opts, &v = b.opts;
    return a.kind == b.kind && p.ndim == q.ndim && p.n1 == q.n1 && p.n2 == q.n2 && p.n3 == q.n3 && p.d1 == q.d1 &&
           p.d2 == q.d2 && p.d3 == q.d3 && p.vp == q.vp && p.rho == q.rho && a.wav.nt == b.wav.nt &&
           a.wav.dt == b.wav.dt && a.wav.fm == b.wav.fm && a.wav.stf == b.wav.stf && u.order == v.order &&
           u.nb == v.nb && u.freesurf == v.freesurf && u.dr == v.dr && u.use_box == v.use_box &&
           u.shell_prec == v.shell_prec && u.kaiser_b == v.kaiser_b && u.cpml_R == v.cpml_R &&
           u.max_batch == v.max_batch && u.profile == v.profile && u.img_norm == v.img_norm &&
           u.kernels == v.kernels && u.per_shot == v.per_shot;
}

int run_one(smi_request r, cudaStream_t st)
{
    r.opts.stream = st;
    if (r.kind == 0) return smi_forward(&r.model, &r.geom, &r.wav, &r.opts, r.out);
    if (r.kind == 1) return smi_rtm(&r.model, &r.geom, &r.wav, &r.opts, r.dobs, r.out);
    return smi_fwi_gradient(&r.model, &r.geom, &r.wav, &r.opts, r.dobs, r.misfit, r.out);
}

// Requests of one survey as one shot-batched call: shots concatenated in the
// requests' order, observed data gathered, per-shot results scattered back.
int run_merged(const std::vector<smi_request> &rs, cudaStream_t st, std::string &err)
{
    const smi_request &r0 = rs[0];
    const int K = (int)rs.size();
    std::vector<double> src(3 * (size_t)K), rec;
    std::vector<int> roff(K + 1, 0);
    for (int k = 0; k < K; k++) {
        const smi_geometry &g = rs[k].geom;
        for (int c = 0; c < 3; c++) src[3 * (size_t)k + c] = g.src[c];
        const int n = g.rec_offset[1] - g.rec_offset[0];
        roff[k + 1] = roff[k] + n;
        rec.insert(rec.end(), g.rec + 3 * (size_t)g.rec_offset[0], g.rec + 3 * (size_t)g.rec_offset[1]);
    }
    const smi_geometry geo{K, src.data(), roff.data(), rec.data()};
    const size_t nt = (size_t)r0.wav.nt;
    const size_t nphys = (size_t)r0.model.n1 * r0.model.n2 * (r0.model.ndim == 3 ? r0.model.n3 : 1);
    const size_t nout = r0.kind == 0 ? nt * roff[K] : nphys * K;
    float *d_dobs = nullptr, *d_out = nullptr;
    double *d_mis = nullptr;
    bool ok = cudaMallocAsync(&d_out, nout * sizeof(float), st) == cudaSuccess;
    if (ok && r0.kind != 0) ok = cudaMallocAsync(&d_dobs, nt * roff[K] * sizeof(float), st) == cudaSuccess;
    if (ok && r0.kind == 2) ok = cudaMallocAsync(&d_mis, K * sizeof(double), st) == cudaSuccess;
    int rc = SMI_OK;
    if (!ok) {
        rc = SMI_ERR_NOMEM;
        err = "device allocation of a merged call's buffers failed";
    }
    for (int k = 0; !rc && r0.kind != 0 && k < K; k++)
        cudaMemcpyAsync(d_dobs + nt * roff[k], rs[k].dobs, nt * (roff[k + 1] - roff[k]) * sizeof(float),
                        cudaMemcpyDefault, st);
    if (!rc) {
        smi_opts o = r0.opts;
        o.stream = st;
        o.per_shot = 1;
        if (r0.kind == 0) rc = smi_forward(&r0.model, &geo, &r0.wav, &o, d_out);
        else if (r0.kind == 1) rc = smi_rtm(&r0.model, &geo, &r0.wav, &o, d_dobs, d_out);
        else rc = smi_fwi_gradient(&r0.model, &geo, &r0.wav, &o, d_dobs, d_mis, d_out);
        if (rc) err = smi_last_error();
    }
    for (int k = 0; !rc && k < K; k++) {
        if (r0.kind == 0)
            cudaMemcpyAsync(rs[k].out, d_out + nt * roff[k], nt * (roff[k + 1] - roff[k]) * sizeof(float),
                            cudaMemcpyDefault, st);
        else
            cudaMemcpyAsync(rs[k].out, d_out + nphys * k, nphys * sizeof(float), cudaMemcpyDefault, st);
        if (r0.kind == 2 && rs[k].misfit) cudaMemcpyAsync(rs[k].misfit, d_mis + k, sizeof(double), cudaMemcpyDefault, st);
    }
    if (d_out) cudaFreeAsync(d_out, st);
    if (d_dobs) cudaFreeAsync(d_dobs, st);
    if (d_mis) cudaFreeAsync(d_mis, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) {
        rc = SMI_ERR_CUDA;
        err = cudaGetErrorString(e);
    }
    return rc;
}

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
    long long completed = 0, failed = 0, merged_calls = 0, merged_requests = 0;

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
            std::vector<long long> group;
            std::vector<smi_request> reqs;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || (t = pick()) >= 0; });
                if (t < 0) break;                      // stopping with nothing runnable
                const double t_now = now();
                auto take = [&](long long u) {
                    Job &j = jobs[u];
                    j.state = 1;
                    j.t_start = t_now;
                    in_use += j.bytes;
                    group.push_back(u);
                    reqs.push_back(j.req);
                };
                take(t);
                // queued shots of the same survey join the call while they fit
                const long long pts = shot_points(reqs[0]);
                if (mergeable(reqs[0]))
                    for (auto it = queue.begin(); it != queue.end() && (int)group.size() < kMaxMerge &&
                                                  (long long)(group.size() + 1) * pts <= kMergePoints;) {
                        const Job &u = jobs[*it];
                        if (mergeable(u.req) && same_call(reqs[0], u.req) && u.bytes <= budget - in_use) {
                            take(*it);
                            it = queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                if (group.size() > 1) {
                    merged_calls++;
                    merged_requests += (long long)group.size();
                }
            }
            std::vector<int> rcs(group.size(), SMI_OK);
            std::vector<std::string> errs(group.size());
            std::string err;
            if (group.size() > 1 && run_merged(reqs, st, err) != SMI_OK) {
                // The merged call failed (a request that is invalid on its own --
                // a position outside the model, CFL -- fails the whole call):
                // run the requests one by one, so that only such a request fails.
                for (size_t k = 0; k < reqs.size(); k++) {
                    rcs[k] = run_one(reqs[k], st);
                    if (rcs[k]) errs[k] = smi_last_error();
                }
            } else if (group.size() == 1) {
                rcs[0] = run_one(reqs[0], st);
                if (rcs[0]) errs[0] = smi_last_error();
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                const double t_now = now();
                for (size_t k = 0; k < group.size(); k++) {
                    Job &j = jobs[group[k]];
                    j.state = 2;
                    j.status = rcs[k];
                    j.error = errs[k];
                    j.t_end = t_now;
                    in_use -= j.bytes;
                    if (rcs[k]) failed++;
                    else completed++;
                }
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
    // sizes only: a submission never waits for the GPU (a query's set-up
    // kernels would queue behind the running requests' kernels)
    const int rc = smi_footprint(&req->model, &req->geom, &req->wav, &req->opts, req->kind, &bytes);
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

int smi_server_merges(smi_server *s, long long *calls, long long *requests)
{
    if (!s) return SMI_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (calls) *calls = s->merged_calls;
    if (requests) *requests = s->merged_requests;
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
