// K7: initial decomposition (eq. 2.6 and 2.8; Step 1 of Algorithms 1-3) of a
// wave given on the grid:
//
//   A(0, q, p) = 2^{d/2} u0hat(q, p),
//   u0hat(q, p) = int u(y) exp(-i p.(y - q)/eps - |y - q|^2/(2 eps)) dy,
//
// evaluated by the rectangle rule on the grid over the same box window
// |y_l - q_l| <= R sqrt(eps) as the reconstruction (window_bounds), so that
// decomposing and summing back (eq. 2.10) use matching truncations.
//
// One warp per packet.  Lanes 0..d-1 set up one dimension each in FP64 (window,
// offset of its first point, phase at that point and phase step per grid point,
// both in turns and reduced modulo 1) and broadcast it.  The warp walks the
// window box row by row; the lanes stride along the last dimension, so the
// reads of u are coalesced.  FP32 contexts: per point one ex2 and one sincos
// in FP32 from the FP64-reduced phase (the step split into a part that FP32
// multiplies exactly by any window index and a remainder), FP32 partial sums
// folded into FP64 every 16 points per lane.  FP64 contexts: every term in FP64.
#include <cmath>

#include "device_util.cuh"
#include "internal.h"

namespace fgr {
namespace {

struct DecParams {
    int64_t n[3];
    double lo[3], h[3];
    float hf[3];
    double rs, inv_eps, inv_2pi_eps, neg_half_inv_eps;
    double weight;     // 2^{d/2} prod_l h_l
    float ce;          // -log2(e) / (2 eps)
    double two_pow_b;  // split of the phase step (FP32 path)
    double inv_two_pow_b;
};

constexpr int kDecWarps = 8;  // packets per 256-thread CTA

template <int D, bool FP64>
__global__ void __launch_bounds__(32 * kDecWarps) decompose_kernel(const void *__restrict__ u_v,
                                                                   const double *__restrict__ q,
                                                                   const double *__restrict__ p,
                                                                   double *__restrict__ a,
                                                                   double *__restrict__ s, int64_t m,
                                                                   const DecParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t j = blockIdx.x * (int64_t)kDecWarps + (threadIdx.x >> 5);
    if (j >= m) return;  // whole warps leave together
    // per-dimension set-up on lane l
    int mlo = 0, wlen = 0;
    double Qd = 0, Pd = 0;
    float delta = 0, nuhi = 0, nulo = 0, tau0 = 0;
    if (lane < D) {
        const int l = lane;
        Qd = q[l * m + j];
        Pd = p[l * m + j];
        int64_t lo, hi;
        window_bounds(Qd, P.rs, P.lo[l], P.h[l], P.n[l], &lo, &hi);
        mlo = (int)lo;
        wlen = (int)(hi - lo + 1);
        if (!FP64) {
            const double dx0 = grid_x(P.lo[l], P.h[l], lo) - Qd;
            delta = (float)dx0;
            double t0 = -Pd * dx0 * P.inv_2pi_eps;
            t0 -= rint(t0);
            tau0 = (float)t0;
            double nu = -Pd * P.h[l] * P.inv_2pi_eps;  // turns per grid step
            nu -= rint(nu);
            const double hi_part = rint(nu * P.two_pow_b) * P.inv_two_pow_b;
            nuhi = (float)hi_part;
            nulo = (float)(nu - hi_part);
        }
    }
    int w[D], base[D];
    double Qs[D], Ps[D];
    float dl[D], nh[D], nl[D];
    float t0sum = 0.f;
    bool empty = false;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        base[l] = __shfl_sync(0xffffffffu, mlo, l);
        w[l] = __shfl_sync(0xffffffffu, wlen, l);
        Qs[l] = __shfl_sync(0xffffffffu, Qd, l);
        Ps[l] = __shfl_sync(0xffffffffu, Pd, l);
        dl[l] = __shfl_sync(0xffffffffu, delta, l);
        nh[l] = __shfl_sync(0xffffffffu, nuhi, l);
        nl[l] = __shfl_sync(0xffffffffu, nulo, l);
        t0sum += __shfl_sync(0xffffffffu, tau0, l);
        empty = empty || w[l] <= 0;
    }
    double accr = 0.0, acci = 0.0;
    if (!empty) {
        int rows = 1;
#pragma unroll
        for (int l = 0; l < D - 1; ++l) rows *= w[l];
        for (int r = 0; r < rows; ++r) {
            // outer indices of this row and their contributions
            int k[D];
            int rem = r;
#pragma unroll
            for (int l = D - 2; l >= 0; --l) {
                k[l] = rem % w[l];
                rem /= w[l];
            }
            int64_t lin = 0;
#pragma unroll
            for (int l = 0; l < D - 1; ++l) lin = lin * P.n[l] + (base[l] + k[l]);
            lin = lin * P.n[D - 1] + base[D - 1];
            if (FP64) {
                double g2o = 0.0, pho = 0.0;
#pragma unroll
                for (int l = 0; l < D - 1; ++l) {
                    const double dx = grid_x(P.lo[l], P.h[l], base[l] + k[l]) - Qs[l];
                    g2o += dx * dx;
                    pho += Ps[l] * dx;
                }
                const double *u = reinterpret_cast<const double *>(u_v);
                constexpr int L = D - 1;
                for (int kl = lane; kl < w[L]; kl += 32) {
                    const double dx = grid_x(P.lo[L], P.h[L], base[L] + kl) - Qs[L];
                    const double g = exp((g2o + dx * dx) * P.neg_half_inv_eps);
                    double sn, cs;
                    sincos(-(pho + Ps[L] * dx) * P.inv_eps, &sn, &cs);
                    const double ur = u[2 * (lin + kl)], ui = u[2 * (lin + kl) + 1];
                    const double gr = g * cs, gi = g * sn;
                    accr += ur * gr - ui * gi;
                    acci += ur * gi + ui * gr;
                }
            } else {
                float eo = 0.f, to = t0sum;
#pragma unroll
                for (int l = 0; l < D - 1; ++l) {
                    const float kf = (float)k[l];
                    const float dx = fmaf(kf, P.hf[l], dl[l]);
                    eo = fmaf(dx, dx, eo);
                    float f = kf * nh[l];
                    f -= rint_fast(f);
                    to += fmaf(kf, nl[l], f);
                }
                const float2 *u = reinterpret_cast<const float2 *>(u_v);
                constexpr int L = D - 1;
                float sr = 0.f, si = 0.f;
                int cnt = 0;
                for (int kl = lane; kl < w[L]; kl += 32) {
                    const float kf = (float)kl;
                    const float dx = fmaf(kf, P.hf[L], dl[L]);
                    float f = kf * nh[L];
                    f -= rint_fast(f);
                    float tau = to + fmaf(kf, nl[L], f);
                    tau -= rint_fast(tau);
                    float sn, cs;
                    __sincosf(6.283185307179586f * tau, &sn, &cs);
                    const float g = ex2_approx(fmaf(dx, dx, eo) * P.ce);
                    const float2 uv = u[lin + kl];
                    const float gr = g * cs, gi = g * sn;
                    sr = fmaf(uv.x, gr, fmaf(-uv.y, gi, sr));
                    si = fmaf(uv.x, gi, fmaf(uv.y, gr, si));
                    if (++cnt == 16) {  // fold into the FP64 totals
                        accr += (double)sr;
                        acci += (double)si;
                        sr = si = 0.f;
                        cnt = 0;
                    }
                }
                accr += (double)sr;
                acci += (double)si;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        accr += __shfl_xor_sync(0xffffffffu, accr, o);
        acci += __shfl_xor_sync(0xffffffffu, acci, o);
    }
    if (lane == 0) {
        a[j] = P.weight * accr;
        a[m + j] = P.weight * acci;
        s[j] = 0.0;
    }
}

// out = a0 * f elementwise (complex planes [re][m], [im][m]): amplitudes of
// the learned flow from freshly decomposed ones (eq. 2.6 is linear in A).
__global__ void scale_amplitudes_kernel(const double *__restrict__ a0, const double *__restrict__ f,
                                        double *__restrict__ out, int64_t m) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double ar = a0[j], ai = a0[m + j], fr = f[j], fi = f[m + j];
    out[j] = ar * fr - ai * fi;
    out[m + j] = ar * fi + ai * fr;
}

}  // namespace

fgr_status run_scale_amplitudes(const double *a0, const double *f, double *out, int64_t m, cudaStream_t st) {
    if (m == 0) return FGR_OK;
    scale_amplitudes_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(a0, f, out, m);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

fgr_status run_decompose(fgr_ctx *ctx, const void *u_dev, const double *q, const double *p, double *s, double *a,
                         int64_t m, cudaStream_t st) {
    if (m == 0) return FGR_OK;
    const Grid &G = ctx->grid;
    const Mesh &M = ctx->mesh;
    const int D = ctx->d;
    DecParams P{};
    double weight = std::pow(2.0, 0.5 * D);
    int wmax = 1;
    for (int l = 0; l < 3; ++l) {
        P.n[l] = l < D ? G.n[l] : 1;
        P.lo[l] = l < D ? G.lo[l] : 0.0;
        P.h[l] = l < D ? G.h[l] : 1.0;
        P.hf[l] = (float)P.h[l];
        if (l < D) {
            weight *= G.h[l];
            wmax = std::max<int>(wmax, (int)std::min<int64_t>((int64_t)std::floor(2.0 * M.rs / G.h[l]) + 2, G.n[l]));
        }
    }
    int64_t rows = 1;
    for (int l = 0; l < D - 1; ++l)
        rows *= std::min<int64_t>((int64_t)std::floor(2.0 * M.rs / G.h[l]) + 2, G.n[l]);
    if (rows > (int64_t)1 << 30) {
        set_error("decompose: window of more than 2^30 rows");
        return FGR_E_INVALID;
    }
    P.rs = M.rs;
    P.inv_eps = 1.0 / M.eps;
    P.inv_2pi_eps = 1.0 / (2.0 * M_PI * M.eps);
    P.neg_half_inv_eps = -0.5 / M.eps;
    P.weight = weight;
    P.ce = (float)(-1.4426950408889634 / (2.0 * M.eps));
    int lbits = 1;
    while ((1 << lbits) < wmax + 1) ++lbits;
    P.two_pow_b = std::ldexp(1.0, std::max(1, 24 - lbits));
    P.inv_two_pow_b = 1.0 / P.two_pow_b;
    const unsigned blocks = (unsigned)((m + kDecWarps - 1) / kDecWarps);
    const bool fp64 = ctx->opt.precision == FGR_FP64;
#define FGR_DEC(DD)                                                                                               \
    if (fp64)                                                                                                     \
        decompose_kernel<DD, true><<<blocks, 32 * kDecWarps, 0, st>>>(u_dev, q, p, a, s, m, P);                   \
    else                                                                                                          \
        decompose_kernel<DD, false><<<blocks, 32 * kDecWarps, 0, st>>>(u_dev, q, p, a, s, m, P);
    switch (D) {
    case 1: FGR_DEC(1); break;
    case 2: FGR_DEC(2); break;
    default: FGR_DEC(3); break;
    }
#undef FGR_DEC
    FGR_CUDA_TRY(cudaGetLastError());
    ctx->timing.last.launches = 1;
    return FGR_OK;
}

}  // namespace fgr
