// Internal declarations of libfgr (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "fgr.h"

namespace fgr {

constexpr int kMaxDim = 3;
constexpr int kMaxN1 = 16;  // 1-D neighbours per packet: nq * np <= 16

// Eigen-factored eps-free Gram matrix of eq. 3.22 (paper convention).
// The Gram A~ is Hermitian PSD: A~ = V diag(lam) V^H, A~^+ = V diag(inv_lam) V^H.
// Degree of the FP32 coefficient surrogate per variable: its truncation error
// (3e-10 for Q4P2 at 10, 4e-13 at 12) lies far below the FP32 rounding of its
// stored coefficients and of its evaluation.
constexpr int kCheb = 10;
// Terms T_i(s) T_j(t) the FP32 kernels evaluate: i + j <= cheb_total<n1>().
// For n1 <= 8 (Q2P2, Q4P2) the triangle i + j <= 11 keeps 72 of the 100 terms
// and the dropped coefficients sum to below 1e-8 of the largest one (Q4P2
// 8.4e-9, Q2P2 7e-12), under the FP32 rounding of the evaluation; n1 = 16
// (Q4P4) keeps the whole table.
template <int N1>
__host__ __device__ constexpr int cheb_total() {
    return N1 <= 8 ? 11 : 2 * (kCheb - 1);
}

struct Lsa {
    int nq = 4, np = 2, n1 = 8, rank = 0;
    double cq = 0.5, cp = 0.0;
    int dq[kMaxN1] = {}, dp[kMaxN1] = {};  // shifts, k = iq*np + ip
    double lam[kMaxN1] = {};               // descending
    double inv_lam[kMaxN1] = {};           // 1/lam above the cut-off, else 0
    double vr[kMaxN1 * kMaxN1] = {};       // V[j][i]: component j of eigenvector i
    double vi[kMaxN1 * kMaxN1] = {};
    // Chebyshev surrogate of the true coefficients c~_k(s,t) = conj(A~^+ f~(s,t))_k
    // on [0,1]^2: c~_k ~= sum_{i,j<kCheb} cheb[k][i][j] T_i(2s-1) T_j(2t-1).
    float cheb_re[kMaxN1][kCheb][kCheb] = {};
    float cheb_im[kMaxN1][kCheb][kCheb] = {};
};

// Builds Lsa (host, long double Jacobi).  Returns false on bad input.
bool build_lsa(double cq, double cp, int nq, int np, double rcond, Lsa *out);

struct Grid {
    int d = 1;
    int64_t n[kMaxDim] = {1, 1, 1};
    double lo[kMaxDim] = {}, hi[kMaxDim] = {}, h[kMaxDim] = {};
    int64_t total = 1;
};

struct Mesh {
    double eps, sigma, dq, dp, cq, cp, cqcp, pref, R, rs;  // rs = R*sqrt(eps)
};

struct Timing {
    bool enabled = false;
    bool count_terms = false;  // also count the grid passes' node-point terms (one kernel per pass)
    fgr_stats last{};
};

// Launch-shape parameters picked by the autotuner (autotune.cu).
struct Tuning {
    int direct_ctas_per_sm = 8;  // direct sum: tiles x slices >= this x SMs
    int pass_ctas_per_sm = 16;   // grid passes: rows x tiles x b-slices >= this x SMs
    int pass_tile = 0;           // grid points per grid-pass CTA: 32, 128, or 0 (by the band width)
};

// Seeds a new context's tuning from the process-wide table (autotune.cu).
void seed_tuning(fgr_ctx *ctx);

}  // namespace fgr

struct fgr_ctx {
    int d = 1;
    int device = 0;
    int num_sms = 1;
    fgr::Grid grid;
    fgr::Mesh mesh;
    fgr::Lsa lsa;
    fgr_options opt{};
    cudaMemPool_t pool = nullptr;
    fgr::Timing timing;
    fgr::Tuning tune;
    int fft_logn[fgr::kMaxDim] = {0, 0, 0};  // log2 N of the DFT grid stage per dimension (0: direct stage)
    int *dev_err = nullptr;          // device word: a kernel's bounded wait gave up (reported by the next call)
    // Device view of a host word (set by the server around a large direct
    // sum): while it is > 0 the persistent direct-sum CTAs past one per SM
    // stop between work items, so that waiting small requests get SM slots.
    const volatile int *yield_flag = nullptr;
    int64_t *host_pinned = nullptr;  // small pinned buffer for device->host sizes
};

namespace fgr {

// thread-local error message
void set_error(const char *fmt, ...);
void clear_error();

#define FGR_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t err__ = (expr);                                                     \
        if (err__ != cudaSuccess) {                                                     \
            ::fgr::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(err__), \
                             __FILE__, __LINE__);                                       \
            return FGR_E_CUDA;                                                          \
        }                                                                               \
    } while (0)

// Device view of a packet set (device pointers).
struct PacketsDev {
    int64_t m;
    const double *q, *p, *s, *a;
};

// Stream-ordered scratch from the context's pool, released when the guard dies.
class Scratch {
  public:
    Scratch(fgr_ctx *ctx, cudaStream_t s) : ctx_(ctx), s_(s) {}
    ~Scratch();
    // returns nullptr and sets the error on failure
    void *get(size_t bytes);

  private:
    fgr_ctx *ctx_;
    cudaStream_t s_;
    void *ptrs_[32] = {};
    int n_ = 0;
};

// Kernel-stage launchers (return FGR_OK or an error with the message set).
fgr_status run_propagate(fgr_ctx *ctx, double *q, double *p, double *s, double *a, int64_t m,
                         const fgr_potential *v, double t, double dt, cudaStream_t st);
// Eq. 2.6 / 2.8 on the grid: a (2 x m) and s (m) of the packets at (q, p) from
// the wave u_dev (complex, the context's precision).
fgr_status run_decompose(fgr_ctx *ctx, const void *u_dev, const double *q, const double *p, double *s, double *a,
                         int64_t m, cudaStream_t st);
// One dimension of a tensor-product mesh (device pointers).
struct AxisDev {
    int64_t L;
    const double *q, *p;
};
// Eq. 2.8 onto the tensor product of d lists: a (2 x m) of the packets with
// row-major indices sel[j] (sel NULL: j); d >= 2 by banded contractions.
fgr_status run_decompose_tensor(fgr_ctx *ctx, const AxisDev *axes, const void *u_dev, int64_t m,
                                const int64_t *sel, double *a, cudaStream_t st, Scratch &scratch);
// FGR_E_INVALID unless every sel[j] (device memory) lies in [0, total); waits
// for the stream.
fgr_status check_selection_device(fgr_ctx *ctx, const int64_t *sel, int64_t m, int64_t total, cudaStream_t st,
                                  Scratch &scratch);
// out = a0 * f, complex, planes [re][m] then [im][m].
fgr_status run_scale_amplitudes(const double *a0, const double *f, double *out, int64_t m, cudaStream_t st);
fgr_status run_direct(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st,
                      Scratch &scratch);
// check_finite: the bounds reduction also tests every packet value and the
// call returns FGR_E_INVALID, before writing anything, if one is not finite.
fgr_status run_fggc(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st,
                    Scratch &scratch, bool check_finite = false);
// Device bytes owned by an FGGC plan (api.cu).
size_t plan_device_bytes(const fgr_fggc_plan *plan);

// n <= 64 requests of one dimension and precision; scratch[r] belongs to request r
fgr_status run_direct_batch(int n, fgr_ctx *const *ctxs, const PacketsDev *pks, void *const *us,
                            cudaStream_t st, Scratch **scratch, Scratch &shared);

// Event-based stage timer (active only when ctx->timing.enabled).
class StageTimer {
  public:
    StageTimer(fgr_ctx *ctx, cudaStream_t s);
    ~StageTimer();
    void mark(double *slot);  // time since the previous mark goes to *slot
    void finish();            // total -> last.total_ms

  private:
    fgr_ctx *ctx_;
    cudaStream_t s_;
    cudaEvent_t ev_[24] = {};
    double *slot_[24] = {};
    int n_ = 0;
};

inline size_t elem_bytes(int precision) { return precision == FGR_FP64 ? 16 : 8; }

int64_t rk4_nsteps(double t, double dt);

}  // namespace fgr
