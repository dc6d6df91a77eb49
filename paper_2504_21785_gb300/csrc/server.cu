// Serving: continuous batching of reconstruction requests.
//
// Packet sets are registered once and stay resident in device memory.  A
// scheduler thread admits queued requests in arrival order while (a) a worker
// slot is free and (b) the resident sets plus the footprints of admitted
// requests stay within the memory budget.  Each worker owns a CUDA stream and
// a small cache of contexts, so the kernels of admitted requests overlap on the
// device; a request that arrives while others run starts as soon as a slot and
// memory free up.  Completion is reported through fgr_poll with host
// timestamps (submit, start, done).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct PacketSet {
    int d = 1;
    int64_t m = 0;
    double *buf = nullptr;  // q[d*m] p[d*m] s[m] a[2m]
    size_t bytes = 0;
    int users = 0;
    bool released = false;
};

enum class St { Queued, Running, Done };

struct Job {
    uint64_t ticket = 0;
    fgr_request req{};
    size_t footprint = 0;
    St st = St::Queued;
    fgr_result res{};
};

struct CtxKey {
    int32_t d;
    fgr_grid grid;
    double eps;
    fgr_options opt;
    bool operator==(const CtxKey &o) const { return memcmp(this, &o, sizeof(CtxKey)) == 0; }
};

}  // namespace

struct fgr_server {
    int device = 0;
    size_t budget = 0;
    int max_inflight = 1;
    std::mutex mu;
    std::condition_variable cv_sched, cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;      // arrival order
    std::deque<std::shared_ptr<Job>> admitted;   // waiting for a worker
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::map<uint64_t, PacketSet> sets;
    size_t resident = 0, reserved = 0;
    int running = 0;
    uint64_t next_ticket = 1, next_set = 1;
    bool stop = false;
    std::thread sched;
    std::vector<std::thread> workers;
};

namespace {

size_t footprint(const fgr_request &r, const PacketSet &ps) {
    int64_t total = 1;
    for (int l = 0; l < r.d; ++l) total *= r.grid.n[l];
    const size_t eb = r.opt.precision == FGR_FP64 ? 16 : 8;
    size_t f = 0;
    if (r.method == 0) {
        f = (size_t)ps.m * 112 + ((size_t)total / 64 + 1) * 16;  // records, bins
    } else {
        const int n1 = (r.opt.nq ? r.opt.nq : 4) * (r.opt.np ? r.opt.np : 2);
        size_t cells = (size_t)ps.m;
        for (int l = 0; l < r.d; ++l) cells *= (size_t)n1;
        f = cells * eb + 3 * (size_t)total * eb;  // nodes (at most one per contribution) + passes
    }
    return f + (size_t)total * eb;  // staging of a host output
}

void worker_main(fgr_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t stream;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    std::vector<std::pair<CtxKey, fgr_ctx *>> cache;  // small LRU
    for (;;) {
        std::shared_ptr<Job> job;
        PacketSet ps;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->admitted.empty(); });
            if (S->admitted.empty()) break;  // stop requested and nothing left
            job = S->admitted.front();
            S->admitted.pop_front();
            job->st = St::Running;
            job->res.t_start_ms = now_ms();
            ps = S->sets[job->req.set_id];
        }
        const fgr_request &r = job->req;
        CtxKey key;
        memset(&key, 0, sizeof(key));
        key.d = r.d;
        key.grid = r.grid;
        key.eps = r.eps;
        key.opt = r.opt;
        fgr_ctx *ctx = nullptr;
        for (size_t i = 0; i < cache.size(); ++i)
            if (cache[i].first == key) {
                ctx = cache[i].second;
                std::rotate(cache.begin(), cache.begin() + i, cache.begin() + i + 1);
                break;
            }
        fgr_status st = FGR_OK;
        if (!ctx) {
            st = fgr_create(r.d, &r.grid, r.eps, &r.opt, &ctx);
            if (st == FGR_OK) {
                cache.insert(cache.begin(), {key, ctx});
                if (cache.size() > 8) {
                    fgr_destroy(cache.back().second);
                    cache.pop_back();
                }
            }
        }
        if (st == FGR_OK) {
            fgr_packets pk;
            pk.m = ps.m;
            pk.q = ps.buf;
            pk.p = ps.buf + ps.d * ps.m;
            pk.s = ps.buf + 2 * ps.d * ps.m;
            pk.a = ps.buf + (2 * ps.d + 1) * ps.m;
            pk.on_device = 1;
            pk.reserved = 0;
            st = r.method == 0 ? fgr_reconstruct_direct(ctx, &pk, r.u_out, stream)
                               : fgr_reconstruct_fggc(ctx, &pk, r.u_out, stream);
            cudaError_t e = cudaStreamSynchronize(stream);
            if (st == FGR_OK && e != cudaSuccess) st = FGR_E_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            job->res.status = st;
            job->res.t_done_ms = now_ms();
            job->st = St::Done;
            S->reserved -= job->footprint;
            S->running -= 1;
            S->sets[r.set_id].users -= 1;
        }
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
    for (auto &c : cache) fgr_destroy(c.second);
    cudaStreamDestroy(stream);
}

void scheduler_main(fgr_server *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_sched.wait(lk, [&] {
            if (S->stop) return true;
            if (S->queue.empty()) return false;
            const auto &j = S->queue.front();
            return S->running < S->max_inflight && S->resident + S->reserved + j->footprint <= S->budget;
        });
        if (S->stop) break;
        // admit in arrival order while slots and memory allow
        while (!S->queue.empty() && S->running < S->max_inflight) {
            auto j = S->queue.front();
            if (S->resident + S->reserved + j->footprint > S->budget) break;
            S->queue.pop_front();
            S->reserved += j->footprint;
            S->running += 1;
            S->admitted.push_back(j);
        }
        S->cv_work.notify_all();
    }
}

}  // namespace

using fgr::set_error;
using fgr::clear_error;

extern "C" {

fgr_status fgr_server_create(size_t hbm_budget_bytes, int32_t max_inflight, fgr_server **out) {
    clear_error();
    if (!out || max_inflight < 1 || max_inflight > 64 || hbm_budget_bytes == 0) {
        set_error("server: need out != NULL, 1 <= max_inflight <= 64, budget > 0");
        return FGR_E_INVALID;
    }
    *out = nullptr;
    fgr_server *S = new (std::nothrow) fgr_server();
    if (!S) return FGR_E_NOMEM;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        set_error("server: no CUDA device");
        delete S;
        return FGR_E_CUDA;
    }
    S->budget = hbm_budget_bytes;
    S->max_inflight = max_inflight;
    try {
        S->sched = std::thread(scheduler_main, S);
        for (int i = 0; i < max_inflight; ++i) S->workers.emplace_back(worker_main, S);
    } catch (...) {
        set_error("server: could not start threads");
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_sched.notify_all();
        S->cv_work.notify_all();
        if (S->sched.joinable()) S->sched.join();
        for (auto &w : S->workers) w.join();
        delete S;
        return FGR_E_INTERNAL;
    }
    *out = S;
    return FGR_OK;
}

void fgr_server_destroy(fgr_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (auto &j : S->queue) {  // never started: cancelled
            j->st = St::Done;
            j->res.status = FGR_E_CANCELLED;
            j->res.t_done_ms = now_ms();
        }
        S->queue.clear();
    }
    S->cv_sched.notify_all();
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    S->sched.join();
    for (auto &w : S->workers) w.join();  // admitted jobs finish first
    cudaSetDevice(S->device);
    for (auto &kv : S->sets) cudaFree(kv.second.buf);
    delete S;
}

fgr_status fgr_register_packets(fgr_server *S, int32_t d, const fgr_packets *pk, uint64_t *set_id) {
    clear_error();
    if (!S || !pk || !set_id || d < 1 || d > 3 || pk->m < 0 ||
        (pk->m > 0 && (!pk->q || !pk->p || !pk->s || !pk->a))) {
        set_error("register: bad arguments");
        return FGR_E_INVALID;
    }
    const int64_t m = pk->m;
    const size_t bytes = sizeof(double) * (size_t)std::max<int64_t>(m, 1) * (2 * d + 3);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->resident + S->reserved + bytes > S->budget) {
            set_error("register: %zu bytes exceed the remaining budget", bytes);
            return FGR_E_CAPACITY;
        }
        S->resident += bytes;  // reserve now, release on failure below
    }
    cudaSetDevice(S->device);
    double *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    const cudaMemcpyKind kind = pk->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (e == cudaSuccess && m > 0) {
        e = cudaMemcpy(buf, pk->q, sizeof(double) * d * m, kind);
        if (e == cudaSuccess) e = cudaMemcpy(buf + d * m, pk->p, sizeof(double) * d * m, kind);
        if (e == cudaSuccess) e = cudaMemcpy(buf + 2 * d * m, pk->s, sizeof(double) * m, kind);
        if (e == cudaSuccess) e = cudaMemcpy(buf + (2 * d + 1) * m, pk->a, sizeof(double) * 2 * m, kind);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        S->resident -= bytes;
        set_error("register: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FGR_E_NOMEM : FGR_E_CUDA;
    }
    PacketSet ps;
    ps.d = d;
    ps.m = m;
    ps.buf = buf;
    ps.bytes = bytes;
    const uint64_t id = S->next_set++;
    S->sets[id] = ps;
    *set_id = id;
    return FGR_OK;
}

fgr_status fgr_release_packets(fgr_server *S, uint64_t set_id) {
    clear_error();
    if (!S) return FGR_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->sets.find(set_id);
    if (it == S->sets.end() || it->second.released) {
        set_error("release: unknown set %llu", (unsigned long long)set_id);
        return FGR_E_INVALID;
    }
    it->second.released = true;
    S->cv_done.wait(lk, [&] { return S->sets[set_id].users == 0; });
    cudaSetDevice(S->device);
    cudaFree(it->second.buf);
    S->resident -= it->second.bytes;
    S->sets.erase(it);
    S->cv_sched.notify_all();
    return FGR_OK;
}

fgr_status fgr_submit(fgr_server *S, const fgr_request *req, uint64_t *ticket) {
    clear_error();
    if (!S || !req || !ticket || (req->method != 0 && req->method != 1) || !req->u_out ||
        req->d < 1 || req->d > 3 || req->grid.d != req->d || !(req->eps > 0)) {
        set_error("submit: malformed request");
        return FGR_E_INVALID;
    }
    auto j = std::make_shared<Job>();
    j->req = *req;
    fgr_options o = req->opt;
    if (o.cq == 0 && o.cp == 0 && o.nq == 0 && o.np == 0 && o.rcond == 0) fgr_default_options(&o);
    j->req.opt = o;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        set_error("submit: server is shutting down");
        return FGR_E_CANCELLED;
    }
    auto it = S->sets.find(req->set_id);
    if (it == S->sets.end() || it->second.released || it->second.d != req->d) {
        set_error("submit: unknown packet set or dimension mismatch");
        return FGR_E_INVALID;
    }
    j->footprint = footprint(j->req, it->second);
    if (S->resident + j->footprint > S->budget) {
        set_error("submit: request needs %zu bytes; budget %zu with %zu resident", j->footprint,
                  S->budget, S->resident);
        return FGR_E_CAPACITY;
    }
    it->second.users += 1;
    j->ticket = S->next_ticket++;
    j->res.status = FGR_E_NOT_READY;
    j->res.t_submit_ms = now_ms();
    S->jobs[j->ticket] = j;
    S->queue.push_back(j);
    *ticket = j->ticket;
    S->cv_sched.notify_all();
    return FGR_OK;
}

fgr_status fgr_poll(fgr_server *S, uint64_t ticket, int32_t timeout_ms, fgr_result *out) {
    if (!S || !out) return FGR_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_error("poll: unknown ticket %llu", (unsigned long long)ticket);
        return FGR_E_INVALID;
    }
    auto j = it->second;
    auto done = [&] { return j->st == St::Done; };
    if (timeout_ms < 0)
        S->cv_done.wait(lk, done);
    else if (timeout_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    if (!done()) return FGR_E_NOT_READY;
    *out = j->res;
    S->jobs.erase(it);
    return FGR_OK;
}

fgr_status fgr_cancel(fgr_server *S, uint64_t ticket) {
    if (!S) return FGR_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return FGR_E_INVALID;
    auto j = it->second;
    auto q = std::find(S->queue.begin(), S->queue.end(), j);
    if (q == S->queue.end()) return FGR_E_NOT_READY;  // already admitted or done
    S->queue.erase(q);
    S->sets[j->req.set_id].users -= 1;
    j->st = St::Done;
    j->res.status = FGR_E_CANCELLED;
    j->res.t_done_ms = now_ms();
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
    return FGR_OK;
}

}  // extern "C"
