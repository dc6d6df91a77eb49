// Autotuner for the launch shapes of the reconstruction kernels.
//
// fgr_autotune times, with CUDA events on the caller's stream, each candidate
// of (a) the number of CTAs per SM the direct sum aims for when it splits the
// packet lists of its output tiles and (b) the grid passes' tile width (32 or
// 128 grid points per CTA) together with the number of CTAs per SM they aim
// for when they split the node range, on the caller's packets and grid.  The
// fastest of each is kept in the context and in a process-wide table keyed by
// the problem class (dimension, precision, packets and grid points rounded to
// powers of two), from which new contexts of the same class start.  With
// FGR_TUNE_FILE set, the table is read from and appended to that file (one
// line per class: d precision log2(M) log2(points) direct pass tile).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace fgr {
namespace {

using ClassKey = std::tuple<int, int, int, int>;
std::mutex g_tune_mu;
std::map<ClassKey, Tuning> g_tuned;
bool g_loaded = false;

int log2_bucket(int64_t x) {
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= x && b < 62) ++b;
    return b;
}

ClassKey class_of(const fgr_ctx *ctx, int64_t m) {
    return ClassKey(ctx->d, ctx->opt.precision, log2_bucket(std::max<int64_t>(m, 1)),
                    log2_bucket(ctx->grid.total));
}

void load_file_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("FGR_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        int d, pr, lm, lg, a, b, t = 0;
        const int n = sscanf(line, "%d %d %d %d %d %d %d", &d, &pr, &lm, &lg, &a, &b, &t);
        if (n < 6 || a < 1 || a > 256 || b < 1 || b > 256 || (t != 0 && t != 32 && t != 128)) continue;
        g_tuned[ClassKey(d, pr, lm, lg)] = Tuning{a, b, t};
    }
    fclose(f);
}

void save_line(const ClassKey &k, const Tuning &t) {
    const char *path = getenv("FGR_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
            t.direct_ctas_per_sm, t.pass_ctas_per_sm, t.pass_tile);
    fclose(f);
}

}  // namespace

void seed_tuning(fgr_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_file_locked();
    // the closest tuned class of the same dimension and precision (grid size first)
    const ClassKey me = class_of(ctx, 1);
    int best = -1;
    for (const auto &kv : g_tuned) {
        if (std::get<0>(kv.first) != std::get<0>(me) || std::get<1>(kv.first) != std::get<1>(me)) continue;
        const int dist = std::abs(std::get<3>(kv.first) - std::get<3>(me));
        if (best < 0 || dist < best) {
            best = dist;
            ctx->tune = kv.second;
        }
    }
}

}  // namespace fgr

using namespace fgr;

extern "C" {

fgr_status fgr_autotune(fgr_ctx *ctx, const fgr_packets *pk, void *u_out, int32_t methods, void *stream) {
    clear_error();
    if (!ctx || !pk || !u_out || (methods & ~3) != 0 || methods == 0) {
        set_error("autotune: need ctx, packets, u_out and methods in {1 (direct), 2 (fggc), 3 (both)}");
        return FGR_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("autotune: cudaEventCreate failed");
        return FGR_E_CUDA;
    }
    auto time_call = [&](bool fggc, float *ms) -> fgr_status {
        fgr_status r = fggc ? fgr_reconstruct_fggc(ctx, pk, u_out, stream) : fgr_reconstruct_direct(ctx, pk, u_out, stream);
        if (r != FGR_OK) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            r = fggc ? fgr_reconstruct_fggc(ctx, pk, u_out, stream) : fgr_reconstruct_direct(ctx, pk, u_out, stream);
            if (r != FGR_OK) return r;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return FGR_E_CUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        *ms = best;
        return FGR_OK;
    };
    const Tuning saved = ctx->tune;
    Tuning best = saved;
    fgr_status rc = FGR_OK;
    if (methods & 1) {
        float best_ms = 1e30f;
        for (int c : {2, 4, 8, 16, 32}) {
            ctx->tune.direct_ctas_per_sm = c;
            float ms;
            rc = time_call(false, &ms);
            if (rc != FGR_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best.direct_ctas_per_sm = c;
            }
        }
        ctx->tune.direct_ctas_per_sm = best.direct_ctas_per_sm;
    }
    if (rc == FGR_OK && (methods & 2)) {
        float best_ms = 1e30f;
        for (int tile : {128, 32}) {
            for (int c : {4, 8, 16, 32, 64}) {
                ctx->tune.pass_tile = tile;
                ctx->tune.pass_ctas_per_sm = c;
                float ms;
                rc = time_call(true, &ms);
                if (rc != FGR_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best.pass_ctas_per_sm = c;
                    best.pass_tile = tile;
                }
            }
            if (rc != FGR_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FGR_OK) {
        ctx->tune = saved;
        return rc;
    }
    ctx->tune = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_file_locked();
    const ClassKey k = class_of(ctx, pk->m);
    g_tuned[k] = best;
    save_line(k, best);
    return FGR_OK;
}

fgr_status fgr_get_tuning(const fgr_ctx *ctx, int32_t *direct_ctas_per_sm, int32_t *pass_ctas_per_sm,
                          int32_t *pass_tile) {
    if (!ctx || !direct_ctas_per_sm || !pass_ctas_per_sm || !pass_tile) return FGR_E_INVALID;
    *direct_ctas_per_sm = ctx->tune.direct_ctas_per_sm;
    *pass_ctas_per_sm = ctx->tune.pass_ctas_per_sm;
    *pass_tile = ctx->tune.pass_tile;
    return FGR_OK;
}

fgr_status fgr_set_tuning(fgr_ctx *ctx, int32_t direct_ctas_per_sm, int32_t pass_ctas_per_sm, int32_t pass_tile) {
    if (!ctx || direct_ctas_per_sm < 1 || direct_ctas_per_sm > 256 || pass_ctas_per_sm < 1 ||
        pass_ctas_per_sm > 256 || (pass_tile != 0 && pass_tile != 32 && pass_tile != 128)) {
        set_error("set_tuning: CTA targets must lie in 1..256 and the pass tile be 0, 32 or 128");
        return FGR_E_INVALID;
    }
    ctx->tune.direct_ctas_per_sm = direct_ctas_per_sm;
    ctx->tune.pass_ctas_per_sm = pass_ctas_per_sm;
    ctx->tune.pass_tile = pass_tile;
    return FGR_OK;
}

}  // extern "C"
