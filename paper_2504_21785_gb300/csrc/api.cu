// C ABI entry points of libfgr: argument checks, host<->device staging,
// scratch management and dispatch to the kernel stages.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "fggc_params.h"
#include "internal.h"

namespace fgr {

namespace {
thread_local char g_err[1024] = "";
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

Scratch::~Scratch() {
    for (int i = n_ - 1; i >= 0; --i)
        if (ptrs_[i]) cudaFreeAsync(ptrs_[i], s_);
}

namespace {
// Failure injection for tests: FGR_INJECT_ALLOC_FAILURE=n makes the n-th
// scratch allocation of the process fail (as if the device were out of memory).
std::atomic<long> g_alloc_count{0};
long injected_failure_index() {
    static const long at = [] {
        const char *e = getenv("FGR_INJECT_ALLOC_FAILURE");
        return e ? atol(e) : -1L;
    }();
    return at;
}
}  // namespace

void *Scratch::get(size_t bytes) {
    if (n_ >= 32) {
        set_error("internal: too many scratch buffers");
        return nullptr;
    }
    const long fail_at = injected_failure_index();
    if (fail_at > 0 && ++g_alloc_count == fail_at) {
        set_error("device allocation of %zu bytes failed: injected failure (FGR_INJECT_ALLOC_FAILURE=%ld)",
                  bytes, fail_at);
        return nullptr;
    }
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    // Under stream capture the allocation becomes a graph memory node, which
    // the graph owns; otherwise it comes from the per-device pool.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = s_ ? cudaStreamIsCapturing(s_, &cap) : cudaSuccess;
    if (e == cudaSuccess)
        e = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(&p, bytes, s_)
                                                 : cudaMallocFromPoolAsync(&p, bytes, ctx_->pool, s_);
    if (e != cudaSuccess) {
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        cudaGetLastError();
        return nullptr;
    }
    ptrs_[n_++] = p;
    return p;
}

StageTimer::StageTimer(fgr_ctx *ctx, cudaStream_t s) : ctx_(ctx), s_(s) {
    if (!ctx_->timing.enabled) return;
    cudaEventCreate(&ev_[0]);
    cudaEventRecord(ev_[0], s_);
    n_ = 1;
}

void StageTimer::mark(double *slot) {
    if (!ctx_->timing.enabled || n_ >= 24) return;
    cudaEventCreate(&ev_[n_]);
    cudaEventRecord(ev_[n_], s_);
    slot_[n_] = slot;
    ++n_;
}

void StageTimer::finish() {
    if (!ctx_->timing.enabled || n_ == 0) return;
    cudaEventSynchronize(ev_[n_ - 1]);
    for (int i = 1; i < n_; ++i) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev_[i - 1], ev_[i]);
        if (slot_[i]) *slot_[i] += ms;
    }
    float tot = 0;
    cudaEventElapsedTime(&tot, ev_[0], ev_[n_ - 1]);
    ctx_->timing.last.total_ms = tot;
}

StageTimer::~StageTimer() {
    for (int i = 0; i < n_; ++i)
        if (ev_[i]) cudaEventDestroy(ev_[i]);
}

int64_t rk4_nsteps(double t, double dt) {
    double r = t / dt;
    double n = std::nearbyint(r);
    if (std::fabs(r - n) <= 1e-9 * (n > 1.0 ? n : 1.0)) return (int64_t)n;
    return (int64_t)std::ceil(r);
}

namespace {

// Process-wide resources shared by contexts, so that creating a context costs
// no CUDA allocation after the first one on a device.
std::mutex g_res_mu;
std::map<std::tuple<double, double, int, int, double>, std::shared_ptr<Lsa>> g_lsa_cache;
cudaMemPool_t g_pools[64] = {};
constexpr int kPinnedSlot = 256;                      // bytes per context
std::vector<std::pair<char *, int>> g_pinned_slabs;   // (slab, slots)
std::vector<char *> g_pinned_free;

std::shared_ptr<Lsa> shared_lsa(double cq, double cp, int nq, int np, double rcond) {
    const auto key = std::make_tuple(cq, cp, nq, np, rcond);
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        auto it = g_lsa_cache.find(key);
        if (it != g_lsa_cache.end()) return it->second;
    }
    auto L = std::make_shared<Lsa>();
    if (!build_lsa(cq, cp, nq, np, rcond, L.get())) return nullptr;
    std::lock_guard<std::mutex> lk(g_res_mu);
    return g_lsa_cache.emplace(key, L).first->second;
}

cudaError_t device_pool(int device, cudaMemPool_t *out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_res_mu);
    if (!g_pools[device]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return e;
        g_pools[device] = pool;
    }
    *out = g_pools[device];
    return cudaSuccess;
}

cudaError_t pinned_slot(char **out) {
    std::lock_guard<std::mutex> lk(g_res_mu);
    if (g_pinned_free.empty()) {
        const int slots = 256;
        char *slab = nullptr;
        cudaError_t e = cudaMallocHost((void **)&slab, (size_t)slots * kPinnedSlot);
        if (e != cudaSuccess) return e;
        g_pinned_slabs.push_back({slab, slots});
        for (int i = slots - 1; i >= 0; --i) g_pinned_free.push_back(slab + (size_t)i * kPinnedSlot);
    }
    *out = g_pinned_free.back();
    g_pinned_free.pop_back();
    return cudaSuccess;
}

void release_pinned_slot(char *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_res_mu);
    g_pinned_free.push_back(p);
}

// Device error words of contexts: slabs of kErrWords per device, kept for the
// process, so that creating or destroying a context allocates and frees no
// device memory (cudaFree would wait for the whole device).  A context's word
// is zeroed on a private non-blocking stream when the context takes it.
constexpr int kErrWords = 1024;
std::vector<int *> g_err_free[64];
cudaStream_t g_err_stream[64] = {};

cudaError_t err_word(int device, int **out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_res_mu);
    cudaError_t e = cudaSuccess;
    if (!g_err_stream[device]) {
        e = cudaStreamCreateWithFlags(&g_err_stream[device], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    if (g_err_free[device].empty()) {
        int *slab = nullptr;
        e = cudaMalloc((void **)&slab, sizeof(int) * kErrWords);
        if (e != cudaSuccess) return e;
        for (int i = kErrWords - 1; i >= 0; --i) g_err_free[device].push_back(slab + i);
    }
    int *w = g_err_free[device].back();
    e = cudaMemsetAsync(w, 0, sizeof(int), g_err_stream[device]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g_err_stream[device]);
    if (e != cudaSuccess) return e;
    g_err_free[device].pop_back();
    *out = w;
    return cudaSuccess;
}

void release_err_word(int device, int *w) {
    if (!w || device < 0 || device >= 64) return;
    std::lock_guard<std::mutex> lk(g_res_mu);
    g_err_free[device].push_back(w);
}

bool is_finite(double x) { return std::isfinite(x); }

fgr_status check_grid(int32_t d, const fgr_grid *g, Grid *out) {
    if (!g) {
        set_error("grid is NULL");
        return FGR_E_INVALID;
    }
    if (d < 1 || d > kMaxDim || g->d != d) {
        set_error("dimension d=%d (grid d=%d) must be 1, 2 or 3 and match", d, g->d);
        return FGR_E_INVALID;
    }
    Grid G;
    G.d = d;
    G.total = 1;
    for (int l = 0; l < d; ++l) {
        if (g->n[l] < 1 || g->n[l] > (int64_t(1) << 31) || !is_finite(g->lo[l]) || !is_finite(g->hi[l]) ||
            !(g->hi[l] > g->lo[l])) {
            set_error("grid dimension %d: need n >= 1 and finite lo < hi", l);
            return FGR_E_INVALID;
        }
        G.n[l] = g->n[l];
        G.lo[l] = g->lo[l];
        G.hi[l] = g->hi[l];
        G.h[l] = (g->hi[l] - g->lo[l]) / (double)g->n[l];
        G.total *= g->n[l];
    }
    if (G.total > (int64_t(1) << 34)) {
        set_error("grid has too many points");
        return FGR_E_INVALID;
    }
    *out = G;
    return FGR_OK;
}

fgr_status resolve_options(const fgr_options *in, fgr_options *out) {
    fgr_options o;
    fgr_default_options(&o);
    if (in) {
        o = *in;
        if (o.cq == 0) o.cq = 0.5;
        if (o.cp == 0) o.cp = M_PI / 8;
        if (o.nq == 0) o.nq = 4;
        if (o.np == 0) o.np = 2;
        if (o.rcond == 0) o.rcond = 1e-14;
    }
    if (o.precision != FGR_FP64 && o.precision != FGR_FP32) {
        set_error("precision must be FGR_FP64 or FGR_FP32");
        return FGR_E_INVALID;
    }
    if (o.window_r == 0) o.window_r = o.precision == FGR_FP64 ? 8.0 : 6.0;
    if (!(o.cq > 0) || !(o.cp > 0) || !is_finite(o.cq) || !is_finite(o.cp) || (o.nq != 2 && o.nq != 4) ||
        (o.np != 2 && o.np != 4) || !(o.window_r > 0) || o.window_r > 40 || !(o.rcond > 0) ||
        o.rcond >= 1 || (o.flags & ~(FGR_FLAG_FFT_GRID | FGR_FLAG_SNAP_CP | FGR_FLAG_DIRECT_FMA)) != 0) {
        set_error("options out of range (cq, cp > 0; nq, np in {2,4}; 0 < window_r <= 40; "
                  "0 < rcond < 1; flags of FGR_FLAG_FFT_GRID | FGR_FLAG_SNAP_CP | FGR_FLAG_DIRECT_FMA)");
        return FGR_E_INVALID;
    }
    *out = o;
    return FGR_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// First index i < n with x[i] not finite, or n.  Large arrays are scanned by
// several host threads (a call on 2^24 host packets scans 1.2 GB).
int64_t first_non_finite(const double *x, int64_t n) {
    constexpr int64_t kChunk = int64_t(1) << 20;
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t nt = std::min<int64_t>(std::max(1u, std::min(hw, 32u)), (n + kChunk - 1) / kChunk);
    if (nt <= 1) {
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(x[i])) return i;
        return n;
    }
    std::vector<int64_t> first((size_t)nt, n);
    std::atomic<int64_t> found{n};
    auto scan = [&](int64_t t) {
        const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        for (int64_t i = lo; i < hi; ++i) {
            if (((i - lo) & 0xffff) == 0 && found.load(std::memory_order_relaxed) < lo) return;
            if (!std::isfinite(x[i])) {
                first[(size_t)t] = i;
                int64_t cur = found.load();
                while (i < cur && !found.compare_exchange_weak(cur, i)) {
                }
                return;
            }
        }
    };
    std::vector<std::thread> th;
    try {
        for (int64_t t = 1; t < nt; ++t) th.emplace_back(scan, t);
    } catch (...) {  // no threads to be had: scan the rest here
        for (int64_t t = (int64_t)th.size() + 1; t < nt; ++t) scan(t);
    }
    scan(0);
    for (auto &h : th) h.join();
    int64_t best = n;
    for (int64_t v : first) best = std::min(best, v);
    return best;
}

// Finiteness of host packet data (Q, P, S, A).
fgr_status check_host_finite(const fgr_ctx *ctx, const fgr_packets *pk) {
    const int d = ctx->d;
    const int64_t m = pk->m;
    int64_t i = std::min(first_non_finite(pk->q, d * m), first_non_finite(pk->p, d * m));
    if (i < d * m) {
        set_error("packets: non-finite Q or P at %lld", (long long)i);
        return FGR_E_INVALID;
    }
    i = std::min(first_non_finite(pk->s, m), std::min(first_non_finite(pk->a, m), first_non_finite(pk->a + m, m)));
    if (i < m) {
        set_error("packets: non-finite S or A at %lld", (long long)i);
        return FGR_E_INVALID;
    }
    return FGR_OK;
}

// Arguments of a packet set, without reading the data.
fgr_status check_packet_args(const fgr_packets *pk) {
    if (!pk || pk->m < 0 || (pk->m > 0 && (!pk->q || !pk->p || !pk->s || !pk->a))) {
        set_error("packets: need m >= 0 and non-NULL q, p, s, a");
        return FGR_E_INVALID;
    }
    if (pk->m > (int64_t(1) << 31)) {
        set_error("packets: at most 2^31 packets per call");
        return FGR_E_INVALID;
    }
    if (pk->on_device != 0 && pk->on_device != 1) {
        set_error("packets: on_device must be 0 or 1");
        return FGR_E_INVALID;
    }
    return FGR_OK;
}

fgr_status check_packets(const fgr_ctx *ctx, const fgr_packets *pk) {
    fgr_status rc = check_packet_args(pk);
    if (rc == FGR_OK && pk->on_device == 0 && pk->m > 0) rc = check_host_finite(ctx, pk);  // host data
    return rc;
}

// Makes device copies of host packet arrays (or passes device pointers through).
fgr_status stage_packets(fgr_ctx *ctx, const fgr_packets *pk, cudaStream_t st, Scratch &scratch,
                         PacketsDev *out, double **dq, double **dp, double **ds, double **da) {
    const int d = ctx->d;
    const int64_t m = pk->m;
    if (pk->on_device || m == 0) {
        *out = {m, pk->q, pk->p, pk->s, pk->a};
        *dq = pk->q;
        *dp = pk->p;
        *ds = pk->s;
        *da = pk->a;
        return FGR_OK;
    }
    double *buf = (double *)scratch.get(sizeof(double) * (size_t)m * (2 * d + 3));
    if (!buf) return FGR_E_NOMEM;
    double *q = buf, *p = q + d * m, *s = p + d * m, *a = s + m;
    FGR_CUDA_TRY(cudaMemcpyAsync(q, pk->q, sizeof(double) * d * m, cudaMemcpyHostToDevice, st));
    FGR_CUDA_TRY(cudaMemcpyAsync(p, pk->p, sizeof(double) * d * m, cudaMemcpyHostToDevice, st));
    FGR_CUDA_TRY(cudaMemcpyAsync(s, pk->s, sizeof(double) * m, cudaMemcpyHostToDevice, st));
    FGR_CUDA_TRY(cudaMemcpyAsync(a, pk->a, sizeof(double) * 2 * m, cudaMemcpyHostToDevice, st));
    *out = {m, q, p, s, a};
    *dq = q;
    *dp = p;
    *ds = s;
    *da = a;
    return FGR_OK;
}

// Tensor-product mesh arguments (fgr_decompose_tensor): every axis present
// with n >= 1 and finite host data, a product of at most 2^40 packets, m in
// [0, 2^31], and a host selection inside the product.
fgr_status check_axes(const fgr_ctx *ctx, const fgr_axis *axes, int64_t m, const int64_t *sel, int64_t *total) {
    if (!axes) {
        set_error("axes: NULL");
        return FGR_E_INVALID;
    }
    int64_t tot = 1;
    for (int l = 0; l < ctx->d; ++l) {
        const fgr_axis &A = axes[l];
        if (A.n < 1 || !A.q || !A.p || (A.on_device != 0 && A.on_device != 1)) {
            set_error("axes: axis %d needs n >= 1, non-NULL q and p, on_device 0 or 1", l);
            return FGR_E_INVALID;
        }
        if (A.n > (int64_t(1) << 40) / tot) {
            set_error("axes: more than 2^40 packets in the product");
            return FGR_E_INVALID;
        }
        tot *= A.n;
        if (!A.on_device)
            for (int64_t i = 0; i < A.n; ++i)
                if (!is_finite(A.q[i]) || !is_finite(A.p[i])) {
                    set_error("axes: non-finite q or p at axis %d entry %lld", l, (long long)i);
                    return FGR_E_INVALID;
                }
    }
    if (m < 0 || m > (int64_t(1) << 31)) {
        set_error("decompose_tensor: m must lie in [0, 2^31]");
        return FGR_E_INVALID;
    }
    if (!sel && m != tot) {
        set_error("decompose_tensor: without sel, m (%lld) must equal the product of the axis lengths (%lld)",
                  (long long)m, (long long)tot);
        return FGR_E_INVALID;
    }
    if (sel && m > 0 && !is_device_ptr(sel))
        for (int64_t j = 0; j < m; ++j)
            if (sel[j] < 0 || sel[j] >= tot) {
                set_error("decompose_tensor: sel[%lld] = %lld outside [0, %lld)", (long long)j, (long long)sel[j],
                          (long long)tot);
                return FGR_E_INVALID;
            }
    *total = tot;
    return FGR_OK;
}

// Device views of the axis lists and the selection (host data copied in; a
// device selection range-checked on the device).
fgr_status stage_axes(fgr_ctx *ctx, const fgr_axis *axes, int64_t m, const int64_t *sel, int64_t total,
                      cudaStream_t st, Scratch &scratch, AxisDev *out, const int64_t **sel_dev) {
    for (int l = 0; l < ctx->d; ++l) {
        const fgr_axis &A = axes[l];
        out[l].L = A.n;
        if (A.on_device) {
            out[l].q = A.q;
            out[l].p = A.p;
            continue;
        }
        double *buf = (double *)scratch.get(sizeof(double) * 2 * (size_t)A.n);
        if (!buf) return FGR_E_NOMEM;
        FGR_CUDA_TRY(cudaMemcpyAsync(buf, A.q, sizeof(double) * A.n, cudaMemcpyHostToDevice, st));
        FGR_CUDA_TRY(cudaMemcpyAsync(buf + A.n, A.p, sizeof(double) * A.n, cudaMemcpyHostToDevice, st));
        out[l].q = buf;
        out[l].p = buf + A.n;
    }
    *sel_dev = nullptr;
    if (!sel || m == 0) return FGR_OK;
    if (is_device_ptr(sel)) {
        *sel_dev = sel;
        return check_selection_device(ctx, sel, m, total, st, scratch);
    }
    int64_t *buf = (int64_t *)scratch.get(sizeof(int64_t) * (size_t)m);
    if (!buf) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemcpyAsync(buf, sel, sizeof(int64_t) * m, cudaMemcpyHostToDevice, st));
    *sel_dev = buf;
    return FGR_OK;
}

template <class F>
fgr_status guarded(F f) {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return FGR_E_NOMEM;
    } catch (...) {
        set_error("internal error");
        return FGR_E_INTERNAL;
    }
}

fgr_status reconstruct(fgr_ctx *ctx, const fgr_packets *pk, void *u_out, void *stream, bool fggc) {
    clear_error();
    if (!ctx || !u_out) {
        set_error("ctx and u_out must be non-NULL");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packet_args(pk);
    if (rc != FGR_OK) return rc;
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        memset(&ctx->timing.last, 0, sizeof(ctx->timing.last));
        Scratch scratch(ctx, st);
        PacketsDev dev;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, pk, st, scratch, &dev, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        const bool host_data = !pk->on_device && pk->m > 0;
        if (host_data && !fggc) {
            // host data of a direct sum: scanned while its copy runs, before
            // any kernel reads it
            r = check_host_finite(ctx, pk);
            if (r != FGR_OK) {
                cudaStreamSynchronize(st);  // the copy is done with the caller's arrays
                return r;
            }
        }
        const size_t out_bytes = elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total;
        const bool dev_out = is_device_ptr(u_out);
        void *u_dev = u_out;
        if (!dev_out) {
            u_dev = scratch.get(out_bytes);
            if (!u_dev) return FGR_E_NOMEM;
        }
        // host data of an FGGC call: tested on the device by the bounds
        // reduction, whose readback precedes every write
        r = fggc ? run_fggc(ctx, dev, u_dev, st, scratch, host_data) : run_direct(ctx, dev, u_dev, st, scratch);
        if (r != FGR_OK) return r;
        FGR_CUDA_TRY(cudaGetLastError());
        if (!dev_out) {
            FGR_CUDA_TRY(cudaMemcpyAsync(u_out, u_dev, out_bytes, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        } else if (!stream) {
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return FGR_OK;
    });
}

fgr_status reconstruct_direct_batch(int32_t n, fgr_ctx *const *ctxs, const fgr_packets *const *pks,
                                    void *const *u_outs, void *stream) {
    clear_error();
    if (n < 1 || n > 64 || !ctxs || !pks || !u_outs) {
        set_error("batch: n must be in 1..64 and the arrays non-NULL");
        return FGR_E_INVALID;
    }
    for (int r = 0; r < n; ++r) {
        if (!ctxs[r] || !u_outs[r]) {
            set_error("batch: request %d has a NULL context or output", r);
            return FGR_E_INVALID;
        }
        if (ctxs[r]->d != ctxs[0]->d || ctxs[r]->opt.precision != ctxs[0]->opt.precision ||
            ctxs[r]->device != ctxs[0]->device) {
            set_error("batch: request %d differs from request 0 in dimension, precision or device", r);
            return FGR_E_INVALID;
        }
        if (!is_device_ptr(u_outs[r])) {
            set_error("batch: output of request %d is not device memory", r);
            return FGR_E_INVALID;
        }
        fgr_status rc = check_packets(ctxs[r], pks[r]);
        if (rc != FGR_OK) return rc;
    }
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctxs[0]->device));
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<std::unique_ptr<Scratch>> owned;
        std::vector<Scratch *> scratch;
        std::vector<PacketsDev> dev((size_t)n);
        for (int r = 0; r < n; ++r) {
            owned.emplace_back(new Scratch(ctxs[r], st));
            scratch.push_back(owned.back().get());
            double *q, *p, *s, *a;
            fgr_status rc = stage_packets(ctxs[r], pks[r], st, *owned.back(), &dev[(size_t)r], &q, &p, &s, &a);
            if (rc != FGR_OK) return rc;
        }
        Scratch shared(ctxs[0], st);
        fgr_status rc = run_direct_batch(n, ctxs, dev.data(), u_outs, st, scratch.data(), shared);
        if (rc != FGR_OK) return rc;
        FGR_CUDA_TRY(cudaGetLastError());
        if (!stream) FGR_CUDA_TRY(cudaStreamSynchronize(st));
        return FGR_OK;
    });
}

}  // namespace
}  // namespace fgr

using namespace fgr;

// Steps of Algorithm 3 shared by both mesh forms: decompose(u, a0) writes the
// amplitudes of the mesh packets, then the learned factors and FGGC.
template <class Decompose>
fgr_status multistep_loop(fgr_ctx *ctx, const PacketsDev &df, const void *u_in, void *u_out, int32_t steps,
                          cudaStream_t st, Scratch &scratch, void *stream, Decompose decompose) {
    const int64_t m = df.m;
    const size_t bytes = elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total;
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    void *ua = scratch.get(bytes), *ub = scratch.get(bytes);
    double *a0 = (double *)scratch.get(sizeof(double) * 2 * mm);
    double *aw = (double *)scratch.get(sizeof(double) * 2 * mm);
    if (!ua || !ub || !a0 || !aw) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemcpyAsync(ua, u_in, bytes, cudaMemcpyDefault, st));
    void *cur = ua;
    for (int32_t it = 0; it < steps; ++it) {
        Scratch step_scratch(ctx, st);
        fgr_status r = decompose(cur, a0, step_scratch);                    // Step 1 (eq. 2.8)
        if (r == FGR_OK) r = run_scale_amplitudes(a0, df.a, aw, m, st);      // Step 2: learned flow
        if (r != FGR_OK) return r;
        void *dst = cur == ua ? ub : ua;
        r = run_fggc(ctx, PacketsDev{m, df.q, df.p, df.s, aw}, dst, st, step_scratch);  // Step 3
        if (r != FGR_OK) return r;
        cur = dst;
    }
    FGR_CUDA_TRY(cudaMemcpyAsync(u_out, cur, bytes, cudaMemcpyDefault, st));
    FGR_CUDA_TRY(cudaGetLastError());
    if (!stream || !is_device_ptr(u_out)) FGR_CUDA_TRY(cudaStreamSynchronize(st));
    return FGR_OK;
}

extern "C" {

fgr_status fgr_default_options(fgr_options *opt) {
    if (!opt) return FGR_E_INVALID;
    memset(opt, 0, sizeof(*opt));
    opt->cq = 0.5;
    opt->cp = M_PI / 8;
    opt->nq = 4;
    opt->np = 2;
    opt->window_r = 0;
    opt->rcond = 1e-14;
    opt->precision = FGR_FP64;
    opt->flags = 0;
    return FGR_OK;
}

const char *fgr_last_error(void) { return g_err; }

fgr_status fgr_create(int32_t d, const fgr_grid *grid, double eps, const fgr_options *opt,
                      fgr_ctx **out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return FGR_E_INVALID;
    }
    *out = nullptr;
    Grid G;
    fgr_status rc = check_grid(d, grid, &G);
    if (rc != FGR_OK) return rc;
    if (!(eps > 0) || !is_finite(eps)) {
        set_error("eps must be positive and finite");
        return FGR_E_INVALID;
    }
    fgr_options o;
    rc = resolve_options(opt, &o);
    if (rc != FGR_OK) return rc;
    // commensurate meshes: h dp / eps = 2 pi / N per dimension (N a power of two)
    int fft_logn[kMaxDim] = {0, 0, 0};
    if (o.flags & FGR_FLAG_SNAP_CP) {
        const double n0 = 2 * M_PI * eps / (G.h[0] * o.cp * std::sqrt(eps));
        const double l2 = std::round(std::log2(n0));
        if (!(l2 >= 3 && l2 <= 13)) {
            set_error("snap: 2 pi eps / (h dp) = %g is not near a power of two in [8, 8192]", n0);
            return FGR_E_INVALID;
        }
        o.cp = 2 * M_PI * eps / (G.h[0] * std::ldexp(1.0, (int)l2) * std::sqrt(eps));
    }
    if (o.flags & FGR_FLAG_FFT_GRID) {
        for (int l = 0; l < d; ++l) {
            const double n = 2 * M_PI * eps / (G.h[l] * o.cp * std::sqrt(eps));
            const double l2 = std::round(std::log2(n));
            if (!(l2 >= 3 && l2 <= 13) || std::fabs(n - std::ldexp(1.0, (int)l2)) > 1e-9 * n) {
                set_error("fft grid stage: dimension %d has 2 pi eps / (h dp) = %.12g, not a power of two in "
                          "[8, 8192] (use a commensurate grid or FGR_FLAG_SNAP_CP)", l, n);
                return FGR_E_INVALID;
            }
            fft_logn[l] = (int)l2;
        }
    }
    return guarded([&]() -> fgr_status {
        std::shared_ptr<Lsa> L = shared_lsa(o.cq, o.cp, o.nq, o.np, o.rcond);
        if (!L) {
            set_error("neighbour strategy rejected");
            return FGR_E_INVALID;
        }
        fgr_ctx *c = new fgr_ctx();
        c->d = d;
        c->grid = G;
        c->opt = o;
        for (int l = 0; l < kMaxDim; ++l) c->fft_logn[l] = fft_logn[l];
        c->lsa = *L;
        Mesh &M = c->mesh;
        M.eps = eps;
        M.sigma = std::sqrt(eps);
        M.cq = o.cq;
        M.cp = o.cp;
        M.cqcp = o.cq * o.cp;
        M.dq = o.cq * M.sigma;
        M.dp = o.cp * M.sigma;
        M.pref = std::pow(M.dq * M.dp, d) / std::pow(2.0 * M_PI * eps, 1.5 * d);
        M.R = o.window_r;
        M.rs = o.window_r * M.sigma;
        cudaError_t e = cudaGetDevice(&c->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
        if (e == cudaSuccess) e = device_pool(c->device, &c->pool);
        char *slot = nullptr;
        if (e == cudaSuccess) e = pinned_slot(&slot);
        if (e == cudaSuccess) e = err_word(c->device, &c->dev_err);
        if (e != cudaSuccess) {
            set_error("CUDA initialisation failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            if (slot) release_pinned_slot(slot);
            release_err_word(c->device, c->dev_err);
            delete c;
            return FGR_E_CUDA;
        }
        c->host_pinned = (int64_t *)slot;
        seed_tuning(c);
        *out = c;
        return FGR_OK;
    });
}

void fgr_destroy(fgr_ctx *ctx) {
    if (!ctx) return;
    // Kernels in flight hold no reference to the context (parameters are
    // copied at launch, scratch returns to the pool in stream order) except its
    // error word, which only a kernel whose bounded wait gave up writes; every
    // call that uses the pinned slot waits for it before returning.
    release_pinned_slot((char *)ctx->host_pinned);
    release_err_word(ctx->device, ctx->dev_err);
    delete ctx;
}

fgr_status fgr_get_info(const fgr_ctx *ctx, fgr_info *out) {
    if (!ctx || !out) return FGR_E_INVALID;
    memset(out, 0, sizeof(*out));
    out->d = ctx->d;
    out->n1 = ctx->lsa.n1;
    out->rank = ctx->lsa.rank;
    out->precision = ctx->opt.precision;
    out->eps = ctx->mesh.eps;
    out->dq = ctx->mesh.dq;
    out->dp = ctx->mesh.dp;
    out->pref = ctx->mesh.pref;
    out->window_r = ctx->mesh.R;
    for (int i = 0; i < ctx->lsa.n1; ++i) out->eigenvalues[i] = ctx->lsa.lam[i];
    return FGR_OK;
}

fgr_status fgr_set_timing(fgr_ctx *ctx, int32_t enabled) {
    if (!ctx) return FGR_E_INVALID;
    ctx->timing.enabled = enabled != 0;
    ctx->timing.count_terms = enabled >= 2;
    return FGR_OK;
}

fgr_status fgr_get_stats(const fgr_ctx *ctx, fgr_stats *out) {
    if (!ctx || !out) return FGR_E_INVALID;
    *out = ctx->timing.last;
    return FGR_OK;
}

fgr_status fgr_propagate(fgr_ctx *ctx, fgr_packets *pk, const fgr_potential *v, double t, double dt,
                         void *stream) {
    clear_error();
    if (!ctx || !v) {
        set_error("ctx and potential must be non-NULL");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packets(ctx, pk);
    if (rc != FGR_OK) return rc;
    if (!(t >= 0) || !is_finite(t) || !(dt > 0) || !is_finite(dt) || v->kind < FGR_V_FREE ||
        v->kind > FGR_V_HARMONIC || !is_finite(v->c0) || !is_finite(v->amp) || !is_finite(v->k) ||
        !is_finite(v->omega)) {
        set_error("propagate: need t >= 0, dt > 0, a known potential kind, finite parameters");
        return FGR_E_INVALID;
    }
    if (rk4_nsteps(t, dt) > (int64_t(1) << 31)) {
        set_error("propagate: too many steps");
        return FGR_E_INVALID;
    }
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        memset(&ctx->timing.last, 0, sizeof(ctx->timing.last));
        Scratch scratch(ctx, st);
        PacketsDev dev;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, pk, st, scratch, &dev, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        r = run_propagate(ctx, q, p, s, a, pk->m, v, t, dt, st);
        if (r != FGR_OK) return r;
        FGR_CUDA_TRY(cudaGetLastError());
        const int64_t m = pk->m;
        const int d = ctx->d;
        if (!pk->on_device && m > 0) {
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->q, q, sizeof(double) * d * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->p, p, sizeof(double) * d * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->s, s, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->a, a, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        } else if (!stream) {
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return FGR_OK;
    });
}

fgr_status fgr_decompose(fgr_ctx *ctx, const void *u_in, fgr_packets *pk, void *stream) {
    clear_error();
    if (!ctx || !u_in) {
        set_error("decompose: ctx and u_in must be non-NULL");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packets(ctx, pk);
    if (rc != FGR_OK) return rc;
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        memset(&ctx->timing.last, 0, sizeof(ctx->timing.last));
        Scratch scratch(ctx, st);
        PacketsDev dev;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, pk, st, scratch, &dev, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        const void *u_dev = u_in;
        if (!is_device_ptr(u_in) && pk->m > 0) {
            const size_t bytes = elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total;
            void *buf = scratch.get(bytes);
            if (!buf) return FGR_E_NOMEM;
            FGR_CUDA_TRY(cudaMemcpyAsync(buf, u_in, bytes, cudaMemcpyHostToDevice, st));
            u_dev = buf;
        }
        r = run_decompose(ctx, u_dev, q, p, s, a, pk->m, st);
        if (r != FGR_OK) return r;
        const int64_t m = pk->m;
        if (!pk->on_device && m > 0) {
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->s, s, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaMemcpyAsync(pk->a, a, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        } else if (!stream) {
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return FGR_OK;
    });
}

fgr_status fgr_decompose_tensor(fgr_ctx *ctx, const fgr_axis *axes, const void *u_in, int64_t m, const int64_t *sel,
                                double *a_out, void *stream) {
    clear_error();
    if (!ctx || !u_in || (m > 0 && !a_out)) {
        set_error("decompose_tensor: ctx, u_in and a_out must be non-NULL");
        return FGR_E_INVALID;
    }
    int64_t total = 0;
    fgr_status rc = check_axes(ctx, axes, m, sel, &total);
    if (rc != FGR_OK) return rc;
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        memset(&ctx->timing.last, 0, sizeof(ctx->timing.last));
        Scratch scratch(ctx, st);
        AxisDev ax[FGR_MAX_DIM];
        const int64_t *sel_dev = nullptr;
        fgr_status r = stage_axes(ctx, axes, m, sel, total, st, scratch, ax, &sel_dev);
        if (r != FGR_OK || m == 0) return r;
        const void *u_dev = u_in;
        if (!is_device_ptr(u_in)) {
            const size_t bytes = elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total;
            void *buf = scratch.get(bytes);
            if (!buf) return FGR_E_NOMEM;
            FGR_CUDA_TRY(cudaMemcpyAsync(buf, u_in, bytes, cudaMemcpyHostToDevice, st));
            u_dev = buf;
        }
        const bool dev_out = is_device_ptr(a_out);
        double *a = a_out;
        if (!dev_out) {
            a = (double *)scratch.get(sizeof(double) * 2 * (size_t)m);
            if (!a) return FGR_E_NOMEM;
        }
        r = run_decompose_tensor(ctx, ax, u_dev, m, sel_dev, a, st, scratch);
        if (r != FGR_OK) return r;
        if (!dev_out) {
            FGR_CUDA_TRY(cudaMemcpyAsync(a_out, a, sizeof(double) * 2 * (size_t)m, cudaMemcpyDeviceToHost, st));
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        } else if (!stream) {
            FGR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        return FGR_OK;
    });
}


fgr_status fgr_fggc_multistep(fgr_ctx *ctx, const fgr_packets *mesh, const fgr_packets *flow, const void *u_in,
                              void *u_out, int32_t steps, void *stream) {
    clear_error();
    if (!ctx || !u_in || !u_out || steps < 0) {
        set_error("multistep: need ctx, u_in, u_out and steps >= 0");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packets(ctx, mesh);
    if (rc == FGR_OK) rc = check_packets(ctx, flow);
    if (rc != FGR_OK) return rc;
    if (mesh->m != flow->m) {
        set_error("multistep: mesh and flow must hold the same packets (%lld vs %lld)", (long long)mesh->m,
                  (long long)flow->m);
        return FGR_E_INVALID;
    }
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Scratch scratch(ctx, st);
        PacketsDev dm, df;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, mesh, st, scratch, &dm, &q, &p, &s, &a);
        if (r == FGR_OK) r = stage_packets(ctx, flow, st, scratch, &df, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        double *s0 = (double *)scratch.get(sizeof(double) * (size_t)std::max<int64_t>(mesh->m, 1));
        if (!s0) return FGR_E_NOMEM;
        return multistep_loop(ctx, df, u_in, u_out, steps, st, scratch, stream,
                              [&](const void *u, double *a0, Scratch &) {
                                  return run_decompose(ctx, u, dm.q, dm.p, s0, a0, dm.m, st);
                              });
    });
}

fgr_status fgr_fggc_multistep_tensor(fgr_ctx *ctx, const fgr_axis *axes, const int64_t *sel,
                                     const fgr_packets *flow, const void *u_in, void *u_out, int32_t steps,
                                     void *stream) {
    clear_error();
    if (!ctx || !u_in || !u_out || steps < 0) {
        set_error("multistep: need ctx, u_in, u_out and steps >= 0");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packets(ctx, flow);
    if (rc != FGR_OK) return rc;
    int64_t total = 0;
    rc = check_axes(ctx, axes, flow->m, sel, &total);
    if (rc != FGR_OK) return rc;
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Scratch scratch(ctx, st);
        PacketsDev df;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, flow, st, scratch, &df, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        AxisDev ax[FGR_MAX_DIM];
        const int64_t *sel_dev = nullptr;
        r = stage_axes(ctx, axes, flow->m, sel, total, st, scratch, ax, &sel_dev);
        if (r != FGR_OK) return r;
        return multistep_loop(ctx, df, u_in, u_out, steps, st, scratch, stream,
                              [&](const void *u, double *a0, Scratch &step_scratch) {
                                  return run_decompose_tensor(ctx, ax, u, df.m, sel_dev, a0, st, step_scratch);
                              });
    });
}

fgr_status fgr_reconstruct_direct(fgr_ctx *ctx, const fgr_packets *pk, void *u_out, void *stream) {
    return reconstruct(ctx, pk, u_out, stream, false);
}

fgr_status fgr_reconstruct_direct_batch(int32_t n, fgr_ctx *const *ctxs, const fgr_packets *const *pks,
                                        void *const *u_outs, void *stream) {
    return reconstruct_direct_batch(n, ctxs, pks, u_outs, stream);
}

fgr_status fgr_reconstruct_fggc(fgr_ctx *ctx, const fgr_packets *pk, void *u_out, void *stream) {
    return reconstruct(ctx, pk, u_out, stream, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// FGGC plans: the node box and the working memory of one (context, packet
// set) fixed once, so that later reconstructions wait for nothing on the host
// and can be captured into a CUDA graph.
// ---------------------------------------------------------------------------
struct fgr_fggc_plan {
    int d = 0, precision = 0, device = 0;
    Grid grid;
    Mesh mesh;
    fgr_options opt{};
    FggcBox box;
    FggcBuffers buf;
    int *bnd = nullptr;       // device: the packets' node bounds of the last call
    int *overflow = nullptr;  // device: set when they left the box
    size_t bin_bytes = 0;     // binning buffers (d = 3, FP32)
    // The buffers come from the device's stream-ordered pool (allocating them
    // does not wait for other streams' work); they go back to it once the
    // device has finished the work issued before the release.
    void release() {
        void *ptrs[] = {buf.W,   buf.buf1, buf.buf2, buf.flags,   buf.brange, buf.tables,
                        buf.bin, buf.fft,  buf.twiddle, bnd, overflow};
        bool any = false;
        for (void *p : ptrs) any = any || p;
        if (any && cudaDeviceSynchronize() == cudaSuccess)
            for (void *p : ptrs)
                if (p) cudaFreeAsync(p, 0);
        cudaGetLastError();
        buf = FggcBuffers{};
        bnd = overflow = nullptr;
    }
};

namespace fgr {
size_t plan_device_bytes(const fgr_fggc_plan *pl) {
    const size_t eb = elem_bytes(pl->precision);
    const FggcBox &b = pl->box;
    size_t n = 64;  // bounds and overflow flag
    if (!b.empty)
        n += eb * (size_t)b.cells + (pl->d > 1 ? 2 * eb * (size_t)b.maxbuf : 0) + (size_t)b.rows0 +
             sizeof(int2) * (size_t)b.max_lines + 8 * (size_t)b.table_entries + pl->bin_bytes +
             (b.fft_elems > 0 ? eb * ((size_t)b.fft_elems + 4096) : 0);
    return n;
}
}  // namespace fgr

namespace {

bool plan_matches(const fgr_ctx *ctx, const fgr_fggc_plan *pl) {
    if (ctx->d != pl->d || ctx->opt.precision != pl->precision || ctx->device != pl->device) return false;
    if (ctx->mesh.eps != pl->mesh.eps || ctx->mesh.dq != pl->mesh.dq || ctx->mesh.dp != pl->mesh.dp ||
        ctx->mesh.rs != pl->mesh.rs || ctx->opt.nq != pl->opt.nq || ctx->opt.np != pl->opt.np ||
        (ctx->opt.flags & FGR_FLAG_FFT_GRID) != (pl->opt.flags & FGR_FLAG_FFT_GRID))
        return false;
    for (int l = 0; l < ctx->d; ++l)
        if (ctx->grid.n[l] != pl->grid.n[l] || ctx->grid.lo[l] != pl->grid.lo[l] || ctx->grid.h[l] != pl->grid.h[l])
            return false;
    return true;
}

}  // namespace

extern "C" {

fgr_status fgr_fggc_plan_create(fgr_ctx *ctx, const fgr_packets *pk, int32_t margin, fgr_fggc_plan **out,
                                void *stream) {
    clear_error();
    if (!ctx || !out || margin < 0 || margin > 4096) {
        set_error("plan: need ctx, out and 0 <= margin <= 4096");
        return FGR_E_INVALID;
    }
    *out = nullptr;
    fgr_status rc = check_packets(ctx, pk);
    if (rc != FGR_OK) return rc;
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Scratch scratch(ctx, st);
        PacketsDev dev;
        double *q, *p, *s, *a;
        fgr_status r = stage_packets(ctx, pk, st, scratch, &dev, &q, &p, &s, &a);
        if (r != FGR_OK) return r;
        std::unique_ptr<fgr_fggc_plan> pl(new fgr_fggc_plan());
        pl->d = ctx->d;
        pl->precision = ctx->opt.precision;
        pl->device = ctx->device;
        pl->grid = ctx->grid;
        pl->mesh = ctx->mesh;
        pl->opt = ctx->opt;
        auto fail = [&](cudaError_t e) {
            cudaGetLastError();
            pl->release();
            set_error("plan: device allocation failed: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? FGR_E_NOMEM : FGR_E_CUDA;
        };
        auto palloc = [&](void **ptr, size_t bytes) { return cudaMallocFromPoolAsync(ptr, bytes, ctx->pool, st); };
        cudaError_t e = palloc((void **)&pl->bnd, sizeof(int) * 12);
        if (e == cudaSuccess) e = palloc((void **)&pl->overflow, sizeof(int));
        if (e != cudaSuccess) return fail(e);
        int hb[12];
        r = compute_node_bounds(ctx, dev, pl->bnd, hb, st);
        if (r != FGR_OK) {
            pl->release();
            return r;
        }
        r = make_box(ctx, hb, margin, &pl->box);
        if (r != FGR_OK) {
            pl->release();
            return r;
        }
        if (!pl->box.empty) {
            const size_t eb = elem_bytes(ctx->opt.precision);
            const FggcBox &b = pl->box;
            e = palloc(&pl->buf.W, eb * (size_t)b.cells);
            if (e == cudaSuccess && ctx->d > 1) e = palloc(&pl->buf.buf1, eb * (size_t)b.maxbuf);
            if (e == cudaSuccess && ctx->d > 1) e = palloc(&pl->buf.buf2, eb * (size_t)b.maxbuf);
            if (e == cudaSuccess) e = palloc((void **)&pl->buf.flags, (size_t)b.rows0);
            if (e == cudaSuccess) e = palloc((void **)&pl->buf.brange, sizeof(int2) * (size_t)b.max_lines);
            if (e == cudaSuccess) e = palloc(&pl->buf.tables, 8 * (size_t)b.table_entries);
            if (e == cudaSuccess && b.fft_elems > 0) e = palloc(&pl->buf.fft, eb * (size_t)b.fft_elems);
            if (e == cudaSuccess && b.fft_elems > 0) e = palloc(&pl->buf.twiddle, eb * 4096);
            BinBox bb;
            if (e == cudaSuccess && ctx->opt.precision == FGR_FP32 && make_bin_box(b, ctx->d, &bb)) {
                pl->bin_bytes = bin_buffer_bytes(pk->m, bb);
                e = palloc(&pl->buf.bin, pl->bin_bytes);
                pl->buf.bin_m = pk->m;
            }
            if (e != cudaSuccess) return fail(e);
        }
        // the buffers are stream-ordered on st: valid for every stream once it is done
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(e);
        *out = pl.release();
        return FGR_OK;
    });
}

fgr_status fgr_reconstruct_fggc_planned(fgr_ctx *ctx, fgr_fggc_plan *plan, const fgr_packets *pk, void *u_out,
                                        void *stream) {
    clear_error();
    if (!ctx || !plan || !u_out) {
        set_error("planned: need ctx, plan and u_out");
        return FGR_E_INVALID;
    }
    if (!plan_matches(ctx, plan)) {
        set_error("planned: the plan was made for another dimension, precision, grid, eps or neighbour set");
        return FGR_E_INVALID;
    }
    fgr_status rc = check_packets(ctx, pk);
    if (rc != FGR_OK) return rc;
    if (pk->m > 0 && pk->on_device != 1) {
        set_error("planned: packets must be device memory");
        return FGR_E_INVALID;
    }
    if (!is_device_ptr(u_out)) {
        set_error("planned: u_out must be device memory");
        return FGR_E_INVALID;
    }
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        const PacketsDev dev{pk->m, pk->q, pk->p, pk->s, pk->a};
        fgr_status r = run_fggc_planned(ctx, dev, plan->box, plan->buf, plan->bnd, plan->overflow, u_out, st);
        if (r != FGR_OK) return r;
        FGR_CUDA_TRY(cudaGetLastError());
        if (!stream) FGR_CUDA_TRY(cudaStreamSynchronize(st));
        return FGR_OK;
    });
}

fgr_status fgr_reconstruct_fggc_batch(int32_t n, fgr_ctx *const *ctxs, fgr_fggc_plan *const *plans,
                                      const fgr_packets *const *pks, void *const *u_outs, void *stream) {
    clear_error();
    if (n < 1 || n > 64 || !ctxs || !plans || !pks || !u_outs) {
        set_error("fggc batch: need 1 <= n <= 64 and the arrays ctxs, plans, pks, u_outs");
        return FGR_E_INVALID;
    }
    for (int r = 0; r < n; ++r) {
        fgr_ctx *ctx = ctxs[r];
        if (!ctx || !plans[r] || !u_outs[r] || !pks[r]) {
            set_error("fggc batch: request %d: need ctx, plan, packets and u_out", r);
            return FGR_E_INVALID;
        }
        const fgr_ctx *c0 = ctxs[0];
        if (ctx->device != c0->device || ctx->opt.precision != c0->opt.precision || ctx->opt.nq != c0->opt.nq ||
            ctx->opt.np != c0->opt.np || ctx->opt.cq != c0->opt.cq || ctx->opt.cp != c0->opt.cp ||
            ctx->opt.rcond != c0->opt.rcond) {
            set_error("fggc batch: request %d: device, precision and neighbour strategy (cq, cp, nq, np, rcond) "
                      "must be those of request 0", r);
            return FGR_E_INVALID;
        }
        if (!plan_matches(ctx, plans[r])) {
            set_error("fggc batch: request %d: the plan was made for another dimension, precision, grid, eps or "
                      "neighbour set", r);
            return FGR_E_INVALID;
        }
        fgr_status rc = check_packets(ctx, pks[r]);
        if (rc != FGR_OK) return rc;
        if (pks[r]->m > 0 && pks[r]->on_device != 1) {
            set_error("fggc batch: request %d: packets must be device memory", r);
            return FGR_E_INVALID;
        }
        if (!is_device_ptr(u_outs[r])) {
            set_error("fggc batch: request %d: u_out must be device memory", r);
            return FGR_E_INVALID;
        }
    }
    return guarded([&]() -> fgr_status {
        FGR_CUDA_TRY(cudaSetDevice(ctxs[0]->device));
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<FggcRequest> req;
        for (int r = 0; r < n; ++r) {
            const fgr_packets *pk = pks[r];
            const PacketsDev dev{pk->m, pk->q, pk->p, pk->s, pk->a};
            if (ctxs[r]->fft_logn[0] > 0) {  // the DFT grid stage runs request by request
                fgr_status e = run_fggc_planned(ctxs[r], dev, plans[r]->box, plans[r]->buf, plans[r]->bnd,
                                                plans[r]->overflow, u_outs[r], st);
                if (e != FGR_OK) return e;
                continue;
            }
            req.push_back(FggcRequest{ctxs[r], &plans[r]->box, &plans[r]->buf, plans[r]->bnd, plans[r]->overflow,
                                      dev, u_outs[r]});
        }
        if (!req.empty()) {
            fgr_status e = run_fggc_batch((int)req.size(), req.data(), st);
            if (e != FGR_OK) return e;
        }
        FGR_CUDA_TRY(cudaGetLastError());
        if (!stream) FGR_CUDA_TRY(cudaStreamSynchronize(st));
        return FGR_OK;
    });
}

fgr_status fgr_fggc_plan_overflow(fgr_fggc_plan *plan, int32_t *overflowed) {
    clear_error();
    if (!plan || !overflowed) return FGR_E_INVALID;
    int v = 0;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e == cudaSuccess) e = cudaMemcpy(&v, plan->overflow, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("plan: %s", cudaGetErrorString(e));
        return FGR_E_CUDA;
    }
    *overflowed = v;
    return FGR_OK;
}

fgr_status fgr_fggc_plan_info(const fgr_fggc_plan *plan, int64_t *nodes, int32_t *empty) {
    if (!plan || !nodes || !empty) return FGR_E_INVALID;
    *nodes = plan->box.cells;
    *empty = plan->box.empty ? 1 : 0;
    return FGR_OK;
}

void fgr_fggc_plan_destroy(fgr_fggc_plan *plan) {
    if (!plan) return;
    cudaSetDevice(plan->device);
    plan->release();
    delete plan;
}

}  // extern "C"
