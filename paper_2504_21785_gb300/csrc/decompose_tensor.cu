// K8: initial decomposition (eq. 2.8) onto a tensor-product packet mesh.
//
// When the packets are the tensor product of d per-dimension lists of
// (q, p) pairs -- packet (i_0, ..., i_{d-1}) at Q_l = q_l[i_l], P_l = p_l[i_l],
// as for the phase-space meshes of Sec. 2.1 and Algorithm 3 -- the kernel of
// eq. 2.8 factorises over dimensions,
//
//   A(i) = 2^{d/2} prod_l h_l  sum_y u(y) prod_l F_l[i_l, y_l],
//   F_l[i, y] = exp(-(x_y - q_i)^2 / (2 eps)) exp(-i p_i (x_y - q_i) / eps)
//
// over the box window of q_i (the window of the reconstruction), and the sum
// is a sequence of d banded contractions, one dimension at a time (last
// dimension first).  Contraction of dimension l maps X[o][y][s] (o over the
// grid extents before l, s over the list lengths after l) to
// Y[o][i][s] = sum_y X[o][y][s] F_l[i, y].
//
// `axis_contract_kernel`: CTA = a chunk of TI consecutive list entries x a
// tile of TS (o, s) positions.  The entries' windows are set up in FP64 (as
// in K7), their union bounds the y loop; per chunk of 16 y values the factors
// F (zero outside an entry's own window) and the X tile are staged in shared
// memory and each thread accumulates an RI x RT register tile of complex
// products (entries of one warp share F values, so those reads broadcast; X
// reads are consecutive).  Lists sorted by q keep the union close to one
// window.  FP32: factors by one ex2 and one MUFU sincos from FP64-reduced
// turns, FP32 sums over at most one window per stage.  FP64: libm exp and
// sincos, FP64 sums.
#include <climits>
#include <cmath>
#include <type_traits>

#include "device_util.cuh"
#include "internal.h"

namespace fgr {
namespace {

constexpr int kKC = 16;   // y values per staged chunk
constexpr int kNT = 256;  // threads per CTA

struct ContractParams {
    const void *X;
    void *Y;
    const double *q, *p;  // the list of this dimension
    int64_t L;            // list entries (Y's extent along the dimension)
    int64_t n;            // grid points (X's extent along the dimension)
    int64_t S_out, S_in;
    int64_t tiles;        // ceil(S_out * S_in / TS)
    double lo, h, rs, inv_2pi_eps, neg_half_inv_eps, inv_eps, two_pow_b, inv_two_pow_b;
    float hf, ce;
    int wcap;
};

constexpr float kTwoPiF = 6.283185307179586f;

template <bool FP64, int RI, int RT>
__global__ void __launch_bounds__(kNT, 2) axis_contract_kernel(const ContractParams C) {
    using Real = typename std::conditional<FP64, double, float>::type;
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    constexpr int TI = 8 * RI, TS = 32 * RT;
    __shared__ C2 Fs[kKC][TI];
    __shared__ C2 Xs[kKC][TS + 1];  // +1: the transposed stores of S_in == 1 spread over banks
    __shared__ int64_t xbase[TS], ybase[TS];
    __shared__ int wlo[TI], wlen[TI];
    __shared__ double sQ[FP64 ? TI : 1], sP[FP64 ? TI : 1];
    __shared__ float sdl[TI], st0[TI], snh[TI], snl[TI];
    __shared__ int ulo_s, uhi_s;
    const int tid = threadIdx.x;
    const int64_t i0 = blockIdx.x * (int64_t)TI;
    const int64_t T = C.S_out * C.S_in;
    if (tid == 0) {
        ulo_s = INT_MAX;
        uhi_s = -1;
    }
    __syncthreads();
    if (tid < TI) {  // windows and phases of the chunk's entries (FP64)
        const int64_t i = i0 + tid;
        int lo = 0, len = 0;
        if (i < C.L) {
            const double Q = C.q[i], Pm = C.p[i];
            int64_t wl, wh;
            window_bounds(Q, C.rs, C.lo, C.h, C.n, &wl, &wh);
            const int64_t ln = wh - wl + 1;
            lo = (int)wl;
            len = ln <= 0 ? 0 : (int)(ln < C.wcap ? ln : C.wcap);
            if (FP64) {
                sQ[tid] = Q;
                sP[tid] = Pm;
            } else {
                const double dx0 = grid_x(C.lo, C.h, wl) - Q;
                double tt = -Pm * dx0 * C.inv_2pi_eps;
                tt -= rint(tt);
                double nu = -Pm * C.h * C.inv_2pi_eps;
                nu -= rint(nu);
                const double hi_part = rint(nu * C.two_pow_b) * C.inv_two_pow_b;
                sdl[tid] = (float)dx0;
                st0[tid] = (float)tt;
                snh[tid] = (float)hi_part;
                snl[tid] = (float)(nu - hi_part);
            }
            if (len > 0) {
                atomicMin(&ulo_s, lo);
                atomicMax(&uhi_s, lo + len - 1);
            }
        }
        wlo[tid] = lo;
        wlen[tid] = len;
    }
    __syncthreads();
    const int ulo = ulo_s, uhi = uhi_s;
    const int tg = tid & 31, ig = tid >> 5;
    for (int64_t tile = blockIdx.y; tile < C.tiles; tile += gridDim.y) {
        const int64_t t0 = tile * TS;
        if (tid < TS) {
            const int64_t t = t0 + tid;
            if (t < T) {
                const int64_t o = t / C.S_in, s = t - o * C.S_in;
                xbase[tid] = o * C.n * C.S_in + s;
                ybase[tid] = o * C.L * C.S_in + s;
            } else {
                xbase[tid] = -1;
                ybase[tid] = -1;
            }
        }
        Real accr[RI][RT], acci[RI][RT];
#pragma unroll
        for (int r = 0; r < RI; ++r)
#pragma unroll
            for (int c = 0; c < RT; ++c) accr[r][c] = acci[r][c] = (Real)0;
        __syncthreads();
        for (int kb = ulo; kb <= uhi; kb += kKC) {
            // factors of the chunk's entries at y = kb .. kb + 15
            for (int e = tid; e < kKC * TI; e += kNT) {
                const int kk = e / TI, ii = e - kk * TI;
                const int rel = kb + kk - wlo[ii];
                C2 f;
                f.x = f.y = (Real)0;
                if (rel >= 0 && rel < wlen[ii]) {
                    if constexpr (FP64) {
                        const double dx = grid_x(C.lo, C.h, kb + kk) - sQ[ii];
                        const double g = exp(dx * dx * C.neg_half_inv_eps);
                        double sn, cs;
                        sincos(-(sP[ii] * dx) * C.inv_eps, &sn, &cs);
                        f.x = g * cs;
                        f.y = g * sn;
                    } else {
                        const float kf = (float)rel;
                        const float dx = fmaf(kf, C.hf, sdl[ii]);
                        const float g = ex2_approx(dx * dx * C.ce);
                        float fr = kf * snh[ii];
                        fr -= rint_fast(fr);
                        float tau = st0[ii] + fmaf(kf, snl[ii], fr);
                        tau -= rint_fast(tau);
                        float sn, cs;
                        __sincosf(kTwoPiF * tau, &sn, &cs);
                        f.x = g * cs;
                        f.y = g * sn;
                    }
                }
                Fs[kk][ii] = f;
            }
            // X tile: consecutive threads along y when the dimension is
            // innermost (S_in == 1), along s otherwise (coalesced either way)
            const C2 *X = reinterpret_cast<const C2 *>(C.X);
            for (int e = tid; e < kKC * TS; e += kNT) {
                int kk, tt;
                if (C.S_in == 1) {
                    tt = e / kKC;
                    kk = e - tt * kKC;
                } else {
                    kk = e / TS;
                    tt = e - kk * TS;
                }
                const int y = kb + kk;
                C2 v;
                v.x = v.y = (Real)0;
                if (y <= uhi && xbase[tt] >= 0) v = X[xbase[tt] + (int64_t)y * C.S_in];
                Xs[kk][tt] = v;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kKC; ++kk) {
                C2 f[RI], x[RT];
#pragma unroll
                for (int r = 0; r < RI; ++r) f[r] = Fs[kk][ig + 8 * r];
#pragma unroll
                for (int c = 0; c < RT; ++c) x[c] = Xs[kk][tg + 32 * c];
#pragma unroll
                for (int r = 0; r < RI; ++r)
#pragma unroll
                    for (int c = 0; c < RT; ++c) {
                        accr[r][c] = fma(f[r].x, x[c].x, fma(-f[r].y, x[c].y, accr[r][c]));
                        acci[r][c] = fma(f[r].x, x[c].y, fma(f[r].y, x[c].x, acci[r][c]));
                    }
            }
            __syncthreads();
        }
        C2 *Y = reinterpret_cast<C2 *>(C.Y);
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int64_t i = i0 + ig + 8 * r;
            if (i >= C.L) continue;
#pragma unroll
            for (int c = 0; c < RT; ++c) {
                const int tt = tg + 32 * c;
                if (ybase[tt] < 0) continue;
                C2 v;
                v.x = accr[r][c];
                v.y = acci[r][c];
                Y[ybase[tt] + i * C.S_in] = v;
            }
        }
        __syncthreads();  // xbase / ybase are rewritten by the next tile
    }
}

// a[j] = weight * Y[sel[j]] (or Y[j]), complex to FP64 planes [re][m], [im][m]
template <bool FP64>
__global__ void gather_scale_kernel(const void *__restrict__ Y_v, const int64_t *__restrict__ sel,
                                    double *__restrict__ a, int64_t m, double weight) {
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const C2 v = reinterpret_cast<const C2 *>(Y_v)[sel ? sel[j] : j];
    a[j] = weight * (double)v.x;
    a[m + j] = weight * (double)v.y;
}

// packet arrays of a one-dimensional mesh: q[j] = axis_q[sel[j]], p likewise
__global__ void gather_axis_kernel(const double *__restrict__ aq, const double *__restrict__ ap,
                                   const int64_t *__restrict__ sel, double *__restrict__ q,
                                   double *__restrict__ p, int64_t m) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t i = sel ? sel[j] : j;
    q[j] = aq[i];
    p[j] = ap[i];
}

__global__ void count_out_of_range_kernel(const int64_t *__restrict__ sel, int64_t m, int64_t total,
                                          unsigned long long *__restrict__ bad) {
    unsigned long long n = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        n += (sel[j] < 0 || sel[j] >= total) ? 1ull : 0ull;
    if (n) atomicAdd(bad, n);
}

template <bool FP64, int RI, int RT>
fgr_status launch_contract(ContractParams C, int num_sms, cudaStream_t st) {
    constexpr int TI = 8 * RI, TS = 32 * RT;
    const int64_t T = C.S_out * C.S_in;
    C.tiles = (T + TS - 1) / TS;
    const int64_t chunks = (C.L + TI - 1) / TI;
    if (chunks == 0 || T == 0) return FGR_OK;
    // enough CTAs for a few waves; each loops over its share of the tiles
    const int64_t want = std::max<int64_t>(1, ((int64_t)num_sms * 8 + chunks - 1) / chunks);
    const unsigned gy = (unsigned)std::min<int64_t>(std::min<int64_t>(C.tiles, want * 4), 65535);
    axis_contract_kernel<FP64, RI, RT><<<dim3((unsigned)chunks, gy), kNT, 0, st>>>(C);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace

fgr_status check_selection_device(fgr_ctx *ctx, const int64_t *sel, int64_t m, int64_t total, cudaStream_t st,
                                  Scratch &scratch) {
    if (m == 0) return FGR_OK;
    auto *bad = (unsigned long long *)scratch.get(sizeof(unsigned long long));
    if (!bad) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st));
    const unsigned blocks = (unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)ctx->num_sms * 8);
    count_out_of_range_kernel<<<blocks, 256, 0, st>>>(sel, m, total, bad);
    FGR_CUDA_TRY(cudaGetLastError());
    FGR_CUDA_TRY(cudaMemcpyAsync(ctx->host_pinned, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    FGR_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t nbad = ctx->host_pinned[0];
    if (nbad != 0) {
        set_error("decompose: %lld selected indices outside [0, %lld)", (long long)nbad, (long long)total);
        return FGR_E_INVALID;
    }
    return FGR_OK;
}

fgr_status run_decompose_tensor(fgr_ctx *ctx, const AxisDev *axes, const void *u_dev, int64_t m,
                                const int64_t *sel, double *a, cudaStream_t st, Scratch &scratch) {
    if (m == 0) return FGR_OK;
    const int D = ctx->d;
    const Grid &G = ctx->grid;
    const Mesh &M = ctx->mesh;
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    if (D == 1) {
        // one dimension: nothing factorises; the per-packet kernel on the
        // listed packets
        double *buf = (double *)scratch.get(sizeof(double) * (size_t)m * 3);
        if (!buf) return FGR_E_NOMEM;
        double *q = buf, *p = buf + m, *s = buf + 2 * m;
        gather_axis_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(axes[0].q, axes[0].p, sel, q, p, m);
        FGR_CUDA_TRY(cudaGetLastError());
        return run_decompose(ctx, u_dev, q, p, s, a, m, st);
    }
    // extents after each contraction: dimensions > l are lists, <= l grid
    int64_t ext[3];
    for (int l = 0; l < D; ++l) ext[l] = G.n[l];
    size_t maxelems = 0;
    for (int l = D - 1; l >= 0; --l) {
        ext[l] = axes[l].L;
        size_t e = 1;
        for (int k = 0; k < D; ++k) e *= (size_t)ext[k];
        maxelems = std::max(maxelems, e);
    }
    const size_t eb = elem_bytes(ctx->opt.precision);
    void *buf0 = scratch.get(eb * std::max<size_t>(maxelems, 1));
    void *buf1 = scratch.get(eb * std::max<size_t>(maxelems, 1));
    if (!buf0 || !buf1) return FGR_E_NOMEM;
    const void *X = u_dev;
    void *Y = buf0;
    for (int l = 0; l < D; ++l) ext[l] = G.n[l];
    for (int l = D - 1; l >= 0; --l) {
        ContractParams C{};
        C.X = X;
        C.Y = Y;
        C.q = axes[l].q;
        C.p = axes[l].p;
        C.L = axes[l].L;
        C.n = G.n[l];
        C.S_out = 1;
        for (int k = 0; k < l; ++k) C.S_out *= ext[k];
        C.S_in = 1;
        for (int k = l + 1; k < D; ++k) C.S_in *= ext[k];
        C.lo = G.lo[l];
        C.h = G.h[l];
        C.hf = (float)G.h[l];
        C.rs = M.rs;
        C.inv_2pi_eps = 1.0 / (2.0 * M_PI * M.eps);
        C.neg_half_inv_eps = -0.5 / M.eps;
        C.inv_eps = 1.0 / M.eps;
        C.ce = (float)(-1.4426950408889634 / (2.0 * M.eps));
        const double wc = std::min<double>(std::floor(2.0 * M.rs / G.h[l]) + 2.0, (double)G.n[l]);
        if (wc > (double)(1 << 30)) {
            set_error("decompose: window of more than 2^30 points");
            return FGR_E_INVALID;
        }
        C.wcap = (int)wc;
        int lbits = 1;
        while ((int64_t(1) << lbits) < (int64_t)C.wcap + 1) ++lbits;
        C.two_pow_b = std::ldexp(1.0, std::max(1, 24 - lbits));
        C.inv_two_pow_b = 1.0 / C.two_pow_b;
        const fgr_status rc = fp64 ? launch_contract<true, 4, 2>(C, ctx->num_sms, st)
                                   : launch_contract<false, 8, 4>(C, ctx->num_sms, st);
        if (rc != FGR_OK) return rc;
        ext[l] = axes[l].L;
        X = Y;
        Y = Y == buf0 ? buf1 : buf0;
    }
    double weight = std::pow(2.0, 0.5 * D);
    for (int l = 0; l < D; ++l) weight *= G.h[l];
    const unsigned blocks = (unsigned)((m + 255) / 256);
    if (fp64)
        gather_scale_kernel<true><<<blocks, 256, 0, st>>>(X, sel, a, m, weight);
    else
        gather_scale_kernel<false><<<blocks, 256, 0, st>>>(X, sel, a, m, weight);
    FGR_CUDA_TRY(cudaGetLastError());
    ctx->timing.last.launches = D + 1;
    return FGR_OK;
}

}  // namespace fgr
