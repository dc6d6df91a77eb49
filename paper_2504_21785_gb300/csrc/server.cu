// Serving: continuous batching of reconstruction requests.
//
// Packet sets are registered once and stay resident in device memory.  A
// scheduler thread admits queued requests in arrival order while (a) a worker
// slot is free and (b) the resident sets plus the footprints of admitted
// requests stay within the memory budget.  Each worker owns a CUDA stream and
// a small cache of contexts, so the kernels of admitted requests overlap on the
// device; a request that arrives while others run starts as soon as a slot and
// memory free up.  Requests of one method, dimension and precision that wait
// together (device outputs) are admitted as one group of up to max_batch:
// direct sums run as a single persistent launch (fgr_reconstruct_direct_batch),
// FGGC reconstructions through their plans in one fgr_reconstruct_fggc_batch
// call (one launch per stage) with one wait for the group.  Plans are
// cached per (packet set, grid, eps, options): registered sets never change,
// so a plan's node box stays valid until the set is released, and its device
// memory counts as resident within the budget.  A group that fails is retried
// request by request, so each request gets its own status.  Completion is
// reported through fgr_poll with host timestamps (submit, start, done).
//
// Large requests (direct sums estimated above kLargeMs from their packet-point
// pairs) never hold every worker slot: at most max_inflight - 1 run at once,
// and a small request may pass a large one waiting at the head of the queue.
// They run alone, on low-priority streams (small requests on high-priority
// ones), with finer work items; while small requests are queued or running,
// the persistent direct-sum CTAs of a large request past one per SM stop
// between items (a pinned host word the kernel reads), so the small requests'
// kernels find free SM slots instead of waiting for the whole large launch.
#include <algorithm>
#include <chrono>
#include <cmath>
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
    bool dev_out = false;
    bool large = false;  // a long direct sum (see kLargeMs)
    St st = St::Queued;
    fgr_result res{};
};

using Group = std::vector<std::shared_ptr<Job>>;

struct CtxKey {
    int32_t d;
    fgr_grid grid;
    double eps;
    fgr_options opt;
    bool operator==(const CtxKey &o) const { return memcmp(this, &o, sizeof(CtxKey)) == 0; }
};

CtxKey key_of(const fgr_request &r) {
    CtxKey key;
    memset(&key, 0, sizeof(key));
    key.d = r.d;
    key.grid = r.grid;
    key.eps = r.eps;
    key.opt = r.opt;
    return key;
}

// FGGC plan of one (packet set, context key); its bytes count as resident.
struct PlanKey {
    uint64_t set_id;
    CtxKey key;
    bool operator<(const PlanKey &o) const { return memcmp(this, &o, sizeof(PlanKey)) < 0; }
};

struct PlanEntry {
    fgr_fggc_plan *plan = nullptr;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_used = 0;  // plan clock at the last acquisition
};

}  // namespace

struct fgr_server {
    int device = 0;
    size_t budget = 0;
    int max_inflight = 1;
    int max_batch = 16;
    std::mutex mu;
    std::condition_variable cv_sched, cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;      // arrival order
    std::deque<Group> admitted;                  // waiting for a worker
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::map<uint64_t, PacketSet> sets;
    std::map<PlanKey, PlanEntry> plans;
    size_t resident = 0, reserved = 0;
    size_t plan_resident = 0;  // the part of resident held by cached plans (they can be freed)
    uint64_t plan_clock = 0;
    int running = 0;
    int running_large = 0;     // admitted groups of a large request
    int small_pending = 0;     // small requests queued or running
    int *yield_host = nullptr;  // pinned, mapped: small_pending as the kernels see it
    int *yield_dev = nullptr;
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

// Direct sums estimated above this many milliseconds are large requests.
constexpr double kLargeMs = 2.0;
// Work items per SM of a large request's persistent direct sum (finer than a
// lone call's, so that CTAs reach an item boundary sooner).
constexpr int kLargeCtasPerSm = 32;

// Estimated device time of a direct sum: packets x window points per
// dimension (the kernel's window of 2 R sqrt(eps) / h + 2 points), at rates of
// the order this GB300 sustains (1-D: about 1.2e12 pairs/s, 2-D and 3-D with
// their outer-product factors about 8e12; FP64 about a quarter).
double est_direct_ms(const fgr_request &r, int64_t m) {
    const double R = r.opt.window_r > 0 ? r.opt.window_r : (r.opt.precision == FGR_FP64 ? 8.0 : 6.0);
    const double rs = R * std::sqrt(r.eps);
    double pairs = (double)m;
    for (int l = 0; l < r.d; ++l) {
        const double n = (double)r.grid.n[l];
        const double h = (r.grid.hi[l] - r.grid.lo[l]) / n;
        pairs *= h > 0 ? std::min(n, std::floor(2.0 * rs / h) + 2.0) : n;
    }
    double rate = r.d == 1 ? 1.2e12 : 8e12;
    if (r.opt.precision == FGR_FP64) rate *= 0.25;
    return pairs / rate * 1e3;
}

void publish_small(fgr_server *S) {
    if (S->yield_host) __atomic_store_n(S->yield_host, S->small_pending, __ATOMIC_RELEASE);
}

// Bookkeeping of a job that reached Done (called with the lock held).
void job_finished(fgr_server *S, const Job &j) {
    if (!j.large) {
        S->small_pending -= 1;
        publish_small(S);
    }
}

bool batchable(const Job &j) { return j.dev_out && !j.large; }

bool same_batch(const Job &a, const Job &b) {
    return a.req.method == b.req.method && a.req.d == b.req.d && a.req.opt.precision == b.req.opt.precision;
}

fgr_packets packets_of(const PacketSet &ps) {
    fgr_packets pk;
    pk.m = ps.m;
    pk.q = ps.buf;
    pk.p = ps.buf + ps.d * ps.m;
    pk.s = ps.buf + 2 * ps.d * ps.m;
    pk.a = ps.buf + (2 * ps.d + 1) * ps.m;
    pk.on_device = 1;
    pk.reserved = 0;
    return pk;
}

// Contexts a worker keeps (a context holds a few hundred bytes of host state
// and a device error word: keeping many avoids creating them per request).
constexpr size_t kCtxCachePerWorker = 256;

// Contexts keyed by (d, grid, eps, options), most recently used first.
class CtxCache {
  public:
    ~CtxCache() {
        for (auto &c : items_) fgr_destroy(c.second);
    }
    fgr_status get(const fgr_request &r, fgr_ctx **out) {
        const CtxKey key = key_of(r);
        for (size_t i = 0; i < items_.size(); ++i)
            if (items_[i].first == key) {
                std::rotate(items_.begin(), items_.begin() + i, items_.begin() + i + 1);
                *out = items_[0].second;
                return FGR_OK;
            }
        fgr_status st = fgr_create(r.d, &r.grid, r.eps, &r.opt, out);
        if (st == FGR_OK) items_.insert(items_.begin(), {key, *out});
        return st;
    }
    // called between groups, so no context of a running group is destroyed
    void trim(size_t keep) {
        while (items_.size() > keep) {
            fgr_destroy(items_.back().second);
            items_.pop_back();
        }
    }

  private:
    std::vector<std::pair<CtxKey, fgr_ctx *>> items_;
};

// The cached plan of (set, request), created on first use if it fits the
// budget; marked busy until release_plan.  nullptr: run without a plan.
fgr_fggc_plan *acquire_plan(fgr_server *S, const Job &job, fgr_ctx *ctx, const fgr_packets &pk,
                            cudaStream_t stream) {
    if (!S || !job.dev_out) return nullptr;
    const PlanKey k{job.req.set_id, key_of(job.req)};
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->plans.find(k);
        if (it != S->plans.end()) {
            if (it->second.busy) return nullptr;
            it->second.busy = true;
            it->second.last_used = ++S->plan_clock;
            return it->second.plan;
        }
    }
    fgr_fggc_plan *plan = nullptr;
    if (fgr_fggc_plan_create(ctx, &pk, 1, &plan, stream) != FGR_OK) return nullptr;
    const size_t bytes = fgr::plan_device_bytes(plan);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto set = S->sets.find(job.req.set_id);
        const bool fits = S->resident + S->reserved + bytes <= S->budget;
        if (fits && set != S->sets.end() && !set->second.released && !S->plans.count(k)) {
            S->plans[k] = PlanEntry{plan, bytes, true, ++S->plan_clock};
            S->resident += bytes;
            S->plan_resident += bytes;
            return plan;
        }
    }
    fgr_fggc_plan_destroy(plan);
    return nullptr;
}

void release_plan(fgr_server *S, const Job &job) {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->plans.find(PlanKey{job.req.set_id, key_of(job.req)});
    if (it != S->plans.end()) it->second.busy = false;
}

// Enqueues one request (FGGC through its plan when there is one); *planned is
// the plan to release once the stream has finished.
fgr_status enqueue_one(fgr_server *S, const Job &job, const PacketSet &ps, CtxCache &cache, cudaStream_t stream,
                       fgr_fggc_plan **planned) {
    const fgr_request &r = job.req;
    *planned = nullptr;
    fgr_ctx *ctx = nullptr;
    fgr_status st = cache.get(r, &ctx);
    if (st != FGR_OK) return st;
    fgr_packets pk = packets_of(ps);
    if (r.method == 0) {
        if (!job.large || !S) return fgr_reconstruct_direct(ctx, &pk, r.u_out, stream);
        // the launch takes these at enqueue time; the cached context gets its own back
        const int ctas_per_sm = ctx->tune.direct_ctas_per_sm;
        ctx->tune.direct_ctas_per_sm = std::max(ctas_per_sm, kLargeCtasPerSm);
        ctx->yield_flag = S->yield_dev;
        st = fgr_reconstruct_direct(ctx, &pk, r.u_out, stream);
        ctx->yield_flag = nullptr;
        ctx->tune.direct_ctas_per_sm = ctas_per_sm;
        return st;
    }
    fgr_fggc_plan *plan = acquire_plan(S, job, ctx, pk, stream);
    if (!plan) return fgr_reconstruct_fggc(ctx, &pk, r.u_out, stream);
    *planned = plan;
    return fgr_reconstruct_fggc_planned(ctx, plan, &pk, r.u_out, stream);
}

// After the stream has finished: a planned request whose packets left the
// box (they cannot, for an unchanged set) is redone without the plan.
fgr_status finish_one(fgr_server *S, const Job &job, const PacketSet &ps, CtxCache &cache, cudaStream_t stream,
                      fgr_fggc_plan *planned, fgr_status st) {
    if (!planned) return st;
    int32_t over = 0;
    if (st == FGR_OK && fgr_fggc_plan_overflow(planned, &over) == FGR_OK && over) {
        fgr_ctx *ctx = nullptr;
        st = cache.get(job.req, &ctx);
        if (st == FGR_OK) {
            fgr_packets pk = packets_of(ps);
            st = fgr_reconstruct_fggc(ctx, &pk, job.req.u_out, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess && st == FGR_OK) st = FGR_E_CUDA;
        }
    }
    release_plan(S, job);
    return st;
}

fgr_status run_one(fgr_server *S, const Job &job, const PacketSet &ps, CtxCache &cache, cudaStream_t stream) {
    fgr_fggc_plan *planned = nullptr;
    fgr_status st = enqueue_one(S, job, ps, cache, stream, &planned);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (st == FGR_OK && e != cudaSuccess) st = FGR_E_CUDA;
    return finish_one(S, job, ps, cache, stream, planned, st);
}

// FGGC group: the requests that have (or get) a plan in one
// fgr_reconstruct_fggc_batch call, the others alone; one wait.
void run_fggc_group(fgr_server *S, const Group &g, const std::vector<PacketSet> &ps, CtxCache &cache,
                    cudaStream_t stream, std::vector<fgr_status> &st) {
    const size_t n = g.size();
    std::vector<fgr_fggc_plan *> planned(n, nullptr);
    std::vector<fgr_ctx *> bctx;
    std::vector<fgr_fggc_plan *> bplan;
    std::vector<fgr_packets> bpk(n);
    std::vector<const fgr_packets *> bpkp;
    std::vector<void *> bu;
    std::vector<size_t> bidx;
    for (size_t i = 0; i < n; ++i) {
        fgr_ctx *ctx = nullptr;
        st[i] = cache.get(g[i]->req, &ctx);
        if (st[i] != FGR_OK) continue;
        bpk[i] = packets_of(ps[i]);
        planned[i] = acquire_plan(S, *g[i], ctx, bpk[i], stream);
        if (!planned[i]) {
            st[i] = fgr_reconstruct_fggc(ctx, &bpk[i], g[i]->req.u_out, stream);
            continue;
        }
        const fgr_options &o = g[i]->req.opt, &o0 = bidx.empty() ? o : g[bidx[0]]->req.opt;
        if (o.cq != o0.cq || o.cp != o0.cp || o.nq != o0.nq || o.np != o0.np || o.rcond != o0.rcond) {
            // another neighbour strategy: not in this batch
            st[i] = fgr_reconstruct_fggc_planned(ctx, planned[i], &bpk[i], g[i]->req.u_out, stream);
            continue;
        }
        bctx.push_back(ctx);
        bplan.push_back(planned[i]);
        bpkp.push_back(&bpk[i]);
        bu.push_back(g[i]->req.u_out);
        bidx.push_back(i);
    }
    if (!bidx.empty()) {
        const fgr_status rb = fgr_reconstruct_fggc_batch((int32_t)bidx.size(), bctx.data(), bplan.data(), bpkp.data(),
                                                         bu.data(), stream);
        for (size_t k = 0; k < bidx.size(); ++k) st[bidx[k]] = rb;
    }
    const cudaError_t e = cudaStreamSynchronize(stream);
    for (size_t i = 0; i < n; ++i) {
        if (st[i] == FGR_OK && e != cudaSuccess) st[i] = FGR_E_CUDA;
        st[i] = finish_one(S, *g[i], ps[i], cache, stream, planned[i], st[i]);
    }
}

// One persistent launch for the whole group; on failure the requests are
// retried one by one.
void run_group(const Group &g, const std::vector<PacketSet> &ps, CtxCache &cache, cudaStream_t stream,
               std::vector<fgr_status> &st) {
    const size_t n = g.size();
    std::vector<fgr_ctx *> ctxs(n);
    std::vector<fgr_packets> pk(n);
    std::vector<const fgr_packets *> pkp(n);
    std::vector<void *> us(n);
    fgr_status rc = FGR_OK;
    for (size_t i = 0; i < n && rc == FGR_OK; ++i) {
        rc = cache.get(g[i]->req, &ctxs[i]);
        pk[i] = packets_of(ps[i]);
        pkp[i] = &pk[i];
        us[i] = g[i]->req.u_out;
    }
    if (rc == FGR_OK) {
        rc = fgr_reconstruct_direct_batch((int32_t)n, ctxs.data(), pkp.data(), us.data(), stream);
        cudaError_t e = cudaStreamSynchronize(stream);
        if (rc == FGR_OK && e != cudaSuccess) rc = FGR_E_CUDA;
    }
    if (rc == FGR_OK) {
        std::fill(st.begin(), st.end(), FGR_OK);
        return;
    }
    for (size_t i = 0; i < n; ++i) st[i] = run_one(nullptr, *g[i], ps[i], cache, stream);
}

void worker_main(fgr_server *S) {
    cudaSetDevice(S->device);
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    cudaStream_t stream_high, stream_low;  // small requests, large requests
    cudaStreamCreateWithPriority(&stream_high, cudaStreamNonBlocking, prio_high);
    cudaStreamCreateWithPriority(&stream_low, cudaStreamNonBlocking, prio_low);
    CtxCache cache;
    for (;;) {
        Group group;
        std::vector<PacketSet> ps;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->admitted.empty(); });
            if (S->admitted.empty()) break;  // stop requested and nothing left
            group = std::move(S->admitted.front());
            S->admitted.pop_front();
            const double t = now_ms();
            for (auto &job : group) {
                job->st = St::Running;
                job->res.t_start_ms = t;
                ps.push_back(S->sets[job->req.set_id]);
            }
        }
        std::vector<fgr_status> st(group.size(), FGR_OK);
        const bool large = group[0]->large;
        cudaStream_t stream = large ? stream_low : stream_high;
        if (group.size() == 1)
            st[0] = run_one(S, *group[0], ps[0], cache, stream);
        else if (group[0]->req.method == 0)
            run_group(group, ps, cache, stream, st);
        else
            run_fggc_group(S, group, ps, cache, stream, st);
        cache.trim(kCtxCachePerWorker);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = now_ms();
            for (size_t i = 0; i < group.size(); ++i) {
                Job &job = *group[i];
                job.res.status = st[i];
                job.res.t_done_ms = t;
                job.st = St::Done;
                S->reserved -= job.footprint;
                S->sets[job.req.set_id].users -= 1;
                job_finished(S, job);
            }
            S->running -= 1;
            if (large) S->running_large -= 1;
        }
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
    cudaStreamDestroy(stream_high);
    cudaStreamDestroy(stream_low);
}

bool has_idle_plan(const fgr_server *S) {
    for (const auto &kv : S->plans)
        if (!kv.second.busy) return true;
    return false;
}

// Takes idle plans out of the cache, least recently used first, until need
// more bytes fit the budget or no idle plan is left; returns them for
// destruction outside the lock.
std::vector<fgr_fggc_plan *> evict_idle_plans(fgr_server *S, size_t need) {
    std::vector<fgr_fggc_plan *> out;
    while (S->resident + S->reserved + need > S->budget) {
        auto lru = S->plans.end();
        for (auto it = S->plans.begin(); it != S->plans.end(); ++it)
            if (!it->second.busy && (lru == S->plans.end() || it->second.last_used < lru->second.last_used)) lru = it;
        if (lru == S->plans.end()) break;
        S->resident -= lru->second.bytes;
        S->plan_resident -= lru->second.bytes;
        out.push_back(lru->second.plan);
        S->plans.erase(lru);
    }
    return out;
}

// The next request to admit: the head of the queue, unless it is large and the
// large requests already hold all but one worker slot; then the first small
// request behind it (end() if there is none).
std::deque<std::shared_ptr<Job>>::iterator next_candidate(fgr_server *S) {
    auto it = S->queue.begin();
    if (it == S->queue.end() || !(*it)->large || S->running_large < std::max(1, S->max_inflight - 1)) return it;
    return std::find_if(S->queue.begin(), S->queue.end(), [](const std::shared_ptr<Job> &j) { return !j->large; });
}

bool fits(const fgr_server *S, const Job &j) { return S->resident + S->reserved + j.footprint <= S->budget; }

// Completes a queued request with FGR_E_CAPACITY: it does not fit the budget
// even with nothing else admitted and no cached plan left.
void fail_capacity(fgr_server *S, std::deque<std::shared_ptr<Job>>::iterator it) {
    auto j = *it;
    S->queue.erase(it);
    const double t = now_ms();
    j->res.status = FGR_E_CAPACITY;
    j->res.t_start_ms = j->res.t_done_ms = t;
    j->st = St::Done;
    S->sets[j->req.set_id].users -= 1;
    job_finished(S, *j);
    S->cv_done.notify_all();
}

void scheduler_main(fgr_server *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_sched.wait(lk, [&] {
            if (S->stop) return true;
            if (S->queue.empty() || S->running >= S->max_inflight) return false;
            auto c = next_candidate(S);
            if (c == S->queue.end()) return false;  // only large requests wait, and their slots are taken
            if (fits(S, **c)) return true;
            // the candidate does not fit: free idle plans, or fail it when
            // nothing that could free memory is in flight
            return has_idle_plan(S) || (S->running == 0 && S->reserved == 0);
        });
        if (S->stop) break;
        auto c = next_candidate(S);
        if (!fits(S, **c)) {
            std::vector<fgr_fggc_plan *> drop = evict_idle_plans(S, (*c)->footprint);
            if (!drop.empty()) {
                lk.unlock();
                for (fgr_fggc_plan *pl : drop) fgr_fggc_plan_destroy(pl);
                lk.lock();
                continue;  // look again: the queue or the memory may have changed
            }
            if (S->running == 0 && S->reserved == 0) {
                fail_capacity(S, c);
                continue;
            }
        }
        // admit in arrival order (a small request may pass a large one, see
        // next_candidate) while slots and memory allow; a batchable request
        // takes the later compatible ones with it
        while (S->running < S->max_inflight) {
            c = next_candidate(S);
            if (c == S->queue.end() || !fits(S, **c)) break;
            auto j = *c;
            S->queue.erase(c);
            S->reserved += j->footprint;
            Group g{j};
            if (batchable(*j))
                for (auto it = S->queue.begin(); it != S->queue.end() && (int)g.size() < S->max_batch;) {
                    const auto &k = *it;
                    if (batchable(*k) && same_batch(*j, *k) && fits(S, *k)) {
                        S->reserved += k->footprint;
                        g.push_back(k);
                        it = S->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            S->running += 1;
            if (j->large) S->running_large += 1;
            S->admitted.push_back(std::move(g));
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
    int *word = nullptr;  // the yield word; without it large requests simply never yield
    if (cudaHostAlloc((void **)&word, sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
        *word = 0;
        if (cudaHostGetDevicePointer((void **)&S->yield_dev, word, 0) == cudaSuccess) {
            S->yield_host = word;
        } else {
            S->yield_dev = nullptr;
            cudaFreeHost(word);
        }
    }
    cudaGetLastError();
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
        if (S->yield_host) cudaFreeHost(S->yield_host);
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
            job_finished(S, *j);
        }
        S->queue.clear();
    }
    S->cv_sched.notify_all();
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    S->sched.join();
    for (auto &w : S->workers) w.join();  // admitted jobs finish first
    cudaSetDevice(S->device);
    for (auto &kv : S->plans) fgr_fggc_plan_destroy(kv.second.plan);
    for (auto &kv : S->sets) cudaFree(kv.second.buf);
    if (S->yield_host) cudaFreeHost(S->yield_host);
    delete S;
}

fgr_status fgr_server_set_max_batch(fgr_server *S, int32_t max_batch) {
    clear_error();
    if (!S || max_batch < 1 || max_batch > 64) {
        set_error("server: max_batch must be in 1..64");
        return FGR_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_batch = max_batch;
    return FGR_OK;
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
        std::vector<fgr_fggc_plan *> drop;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            drop = evict_idle_plans(S, bytes);  // cached plans give way to a new set
            if (S->resident + S->reserved + bytes > S->budget) {
                set_error("register: %zu bytes exceed the remaining budget", bytes);
                for (fgr_fggc_plan *pl : drop) fgr_fggc_plan_destroy(pl);
                return FGR_E_CAPACITY;
            }
            S->resident += bytes;  // reserve now, release on failure below
        }
        for (fgr_fggc_plan *pl : drop) fgr_fggc_plan_destroy(pl);
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
    // the set's plans (none busy: no request of the set is running)
    for (auto pl = S->plans.begin(); pl != S->plans.end();) {
        if (pl->first.set_id == set_id) {
            fgr_fggc_plan_destroy(pl->second.plan);
            S->resident -= pl->second.bytes;
            S->plan_resident -= pl->second.bytes;
            pl = S->plans.erase(pl);
        } else {
            ++pl;
        }
    }
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
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, req->u_out) == cudaSuccess)
        j->dev_out = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
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
    j->large = j->req.method == 0 && est_direct_ms(j->req, it->second.m) > kLargeMs;
    // cached plans do not count: the scheduler frees them for requests that need their memory
    if (S->resident - S->plan_resident + j->footprint > S->budget) {
        set_error("submit: request needs %zu bytes; budget %zu with %zu resident in packet sets", j->footprint,
                  S->budget, S->resident - S->plan_resident);
        return FGR_E_CAPACITY;
    }
    it->second.users += 1;
    j->ticket = S->next_ticket++;
    j->res.status = FGR_E_NOT_READY;
    j->res.t_submit_ms = now_ms();
    S->jobs[j->ticket] = j;
    S->queue.push_back(j);
    if (!j->large) {
        S->small_pending += 1;
        publish_small(S);
    }
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
    job_finished(S, *j);
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
    return FGR_OK;
}

}  // extern "C"
