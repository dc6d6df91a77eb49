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
// One warp per group of G <= 32 consecutive packets.  Lane i sets up packet
// j0 + i in FP64 (per dimension: the window, the offset x_mlo - Q of its first
// point, the phase at that point and the phase step per grid point, both in
// turns reduced modulo 1, the step split into a part that FP32 multiplies
// exactly by any window index and a remainder), so the FP64 work is spread
// over the lanes instead of repeated per packet; the warp then takes the
// group's packets in turn, their parameters broadcast by shuffles.
//
// d = 1: the lanes own the window points lane + 32 i (coalesced reads of u).
// FP32: of every 8 of a lane's points the first gets its Gaussian by one ex2
// and its phase by one MUFU sincos, the next seven the exact recurrences
// over the stride H = 32 h: g_{k+32} = g_k rho, rho <- rho 2^{2 ce H^2},
// e_{k+32} = e_k e^{2 pi i 32 nu}.
// d = 2, 3: the kernel factorises over dimensions, so each packet's
// per-dimension factors f_l(k) = g(dx_l) e^{-i p_l dx_l / eps} are tabulated
// once in the warp's shared memory and every window point costs one complex
// multiply-add of u with the last dimension's factor; the outer factors
// multiply row sums.  FP32 sums are compensated (Kahan), the warp reduction is
// a butterfly of shuffles; FP64 contexts evaluate every factor with libm exp
// and sincos and accumulate in FP64.
#include <cmath>
#include <type_traits>

#include "device_util.cuh"
#include "internal.h"

namespace fgr {
namespace {

struct DecParams {
    int64_t n[3];
    double lo[3], h[3];
    float hf[3];
    int wcap[3];     // upper bound of a window's length per dimension
    int tab_off[3];  // offset of dimension l's factors in a warp's table (d >= 2)
    int tab_len;     // table entries per warp
    int group;       // packets per warp (G)
    int kl_regs;     // d >= 2, FP32: last-dimension factors per lane in registers (2, 4, 8; 0: table)
    double rs, inv_eps, inv_2pi_eps, neg_half_inv_eps;
    double weight;   // 2^{d/2} prod_l h_l
    float ce;        // -log2(e) / (2 eps)
    double two_pow_b, inv_two_pow_b;
};

constexpr int kDecMaxWarps = 8;
constexpr float kTwoPi = 6.283185307179586f;
constexpr int kDecGroup = 8;  // d = 1: points per full evaluation along a lane's stride

// s + x with the running compensation c (Kahan)
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// FP32 factor of dimension l at window index k: g(dx) e^{2 pi i tau}
__device__ __forceinline__ float2 factor32(int k, float hf, float dl, float t0, float nh, float nl, float ce) {
    const float kf = (float)k;
    const float dx = fmaf(kf, hf, dl);
    const float g = ex2_approx(dx * dx * ce);
    float f = kf * nh;
    f -= rint_fast(f);
    float tau = t0 + fmaf(kf, nl, f);
    tau -= rint_fast(tau);
    float sn, cs;
    __sincosf(kTwoPi * tau, &sn, &cs);
    return make_float2(g * cs, g * sn);
}

__device__ __forceinline__ double2 factor64(int k, double lo, double h, int base, double Q, double Pm,
                                            const DecParams &P) {
    const double dx = grid_x(lo, h, base + k) - Q;
    const double g = exp(dx * dx * P.neg_half_inv_eps);
    double sn, cs;
    sincos(-(Pm * dx) * P.inv_eps, &sn, &cs);
    return make_double2(g * cs, g * sn);
}

// Sum over the window of one packet for d = 2, 3 (FP32): rows over the outer
// dimensions, each the product of the outer factors with the row's sum of u
// times the last dimension's factors.  KL > 0: the lane's last-dimension
// factors (points lane + 32 i, i < KL, KL * 32 >= the window) are held in
// registers; KL = 0: read from the warp's table per point.  Rows are summed
// in plain FP32 in chunks of 8 (d = 2) or per slab of the first dimension
// (d = 3), the chunks added with compensation.
template <int D, int KL>
__device__ __forceinline__ void rows32(const float2 *__restrict__ u, const float2 *tab, const DecParams &P,
                                       const int *bb, const int *bw, int lane, float &sr, float &cr, float &si,
                                       float &ci) {
    const float2 *tl = tab + P.tab_off[D - 1];
    const int wL = bw[D - 1];
    float2 fl[KL > 0 ? KL : 1];
    if constexpr (KL > 0) {
#pragma unroll
        for (int i = 0; i < KL; ++i) {
            const int kl = lane + 32 * i;
            fl[i] = kl < wL ? tl[kl] : make_float2(0.f, 0.f);
        }
    }
    const int rows1 = D == 3 ? bw[1] : 1;
    constexpr int CH = D == 2 ? 8 : 1;
    for (int k0c = 0; k0c < bw[0]; k0c += CH) {
        const int k0e = min(k0c + CH, bw[0]);
        float ar = 0.f, ai = 0.f;
        for (int k0 = k0c; k0 < k0e; ++k0) {
            const float2 f0 = tab[P.tab_off[0] + k0];
            const int64_t row0 = (int64_t)(bb[0] + k0);
            for (int k1 = 0; k1 < rows1; ++k1) {
                float2 fo = f0;
                int64_t row = row0;
                if (D == 3) {
                    const float2 f1 = tab[P.tab_off[1] + k1];
                    fo = make_float2(f0.x * f1.x - f0.y * f1.y, f0.x * f1.y + f0.y * f1.x);
                    row = row * P.n[1] + (bb[1] + k1);
                }
                const float2 *urow = u + row * P.n[D - 1] + bb[D - 1];
                float rr = 0.f, ri = 0.f;
                if constexpr (KL > 0) {
#pragma unroll
                    for (int i = 0; i < KL; ++i) {
                        const int kl = lane + 32 * i;
                        if (kl < wL) {
                            const float2 uv = urow[kl];
                            rr = fmaf(uv.x, fl[i].x, fmaf(-uv.y, fl[i].y, rr));
                            ri = fmaf(uv.x, fl[i].y, fmaf(uv.y, fl[i].x, ri));
                        }
                    }
                } else {
                    for (int k = lane; k < wL; k += 32) {
                        const float2 f = tl[k], uv = urow[k];
                        rr = fmaf(uv.x, f.x, fmaf(-uv.y, f.y, rr));
                        ri = fmaf(uv.x, f.y, fmaf(uv.y, f.x, ri));
                    }
                }
                ar = fmaf(fo.x, rr, fmaf(-fo.y, ri, ar));
                ai = fmaf(fo.x, ri, fmaf(fo.y, rr, ai));
            }
        }
        kahan_add(sr, cr, ar);
        kahan_add(si, ci, ai);
    }
}

template <int D, bool FP64>
__global__ void __launch_bounds__(32 * kDecMaxWarps) decompose_kernel(const void *__restrict__ u_v,
                                                                      const double *__restrict__ q,
                                                                      const double *__restrict__ p,
                                                                      double *__restrict__ a,
                                                                      double *__restrict__ s, int64_t m,
                                                                      const DecParams P) {
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char dec_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = P.group;
    const int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * G;
    if (j0 >= m) return;  // whole warps leave together
    const int64_t jl = j0 + lane;
    const bool mine = lane < G && jl < m;
    // set-up of packet jl, every dimension (FP64)
    int base[D], wl[D];
    double Qd[D], Pd[D];
    float dl[D], t0[D], nh[D], nl[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        base[l] = 0;
        wl[l] = 0;
        Qd[l] = Pd[l] = 0.0;
        dl[l] = t0[l] = nh[l] = nl[l] = 0.f;
        if (mine) {
            const double Q = q[l * m + jl], Pm = p[l * m + jl];
            int64_t lo, hi;
            window_bounds(Q, P.rs, P.lo[l], P.h[l], P.n[l], &lo, &hi);
            base[l] = (int)lo;
            const int64_t len = hi - lo + 1;
            wl[l] = len <= 0 ? 0 : (int)(len < P.wcap[l] ? len : P.wcap[l]);
            Qd[l] = Q;
            Pd[l] = Pm;
            if (!FP64) {
                const double dx0 = grid_x(P.lo[l], P.h[l], lo) - Q;
                dl[l] = (float)dx0;
                double tt = -Pm * dx0 * P.inv_2pi_eps;
                tt -= rint(tt);
                t0[l] = (float)tt;
                double nu = -Pm * P.h[l] * P.inv_2pi_eps;  // turns per grid step
                nu -= rint(nu);
                const double hi_part = rint(nu * P.two_pow_b) * P.inv_two_pow_b;
                nh[l] = (float)hi_part;
                nl[l] = (float)(nu - hi_part);
            }
        }
    }
    C2 *tab = reinterpret_cast<C2 *>(dec_smem) + (size_t)warp * P.tab_len;
    double out_r = 0.0, out_i = 0.0;  // this lane's packet
    const int tcount = m - j0 < G ? (int)(m - j0) : G;
    for (int t = 0; t < tcount; ++t) {
        int bb[D], bw[D];
        bool empty = false;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            bb[l] = __shfl_sync(0xffffffffu, base[l], t);
            bw[l] = __shfl_sync(0xffffffffu, wl[l], t);
            empty = empty || bw[l] <= 0;
        }
        if (empty) continue;  // uniform: the amplitude stays 0
        double accr = 0.0, acci = 0.0;
        if constexpr (FP64) {
            double bQ[D], bP[D];
#pragma unroll
            for (int l = 0; l < D; ++l) {
                bQ[l] = __shfl_sync(0xffffffffu, Qd[l], t);
                bP[l] = __shfl_sync(0xffffffffu, Pd[l], t);
            }
            const double2 *u = reinterpret_cast<const double2 *>(u_v);
            if constexpr (D == 1) {
                for (int k = lane; k < bw[0]; k += 32) {
                    const double2 f = factor64(k, P.lo[0], P.h[0], bb[0], bQ[0], bP[0], P);
                    const double2 uv = u[bb[0] + k];
                    accr += uv.x * f.x - uv.y * f.y;
                    acci += uv.x * f.y + uv.y * f.x;
                }
            } else {
#pragma unroll
                for (int l = 0; l < D; ++l)
                    for (int k = lane; k < bw[l]; k += 32)
                        tab[P.tab_off[l] + k] = factor64(k, P.lo[l], P.h[l], bb[l], bQ[l], bP[l], P);
                __syncwarp();
                const double2 *tl = tab + P.tab_off[D - 1];
                const int rows1 = D == 3 ? bw[1] : 1;
                for (int k0 = 0; k0 < bw[0]; ++k0) {
                    const double2 f0 = tab[P.tab_off[0] + k0];
                    for (int k1 = 0; k1 < rows1; ++k1) {
                        double2 fo = f0;
                        int64_t row = (int64_t)(bb[0] + k0);
                        if (D == 3) {
                            const double2 f1 = tab[P.tab_off[1] + k1];
                            fo = make_double2(f0.x * f1.x - f0.y * f1.y, f0.x * f1.y + f0.y * f1.x);
                            row = row * P.n[1] + (bb[1] + k1);
                        }
                        const double2 *urow = u + row * P.n[D - 1] + bb[D - 1];
                        double rr = 0.0, ri = 0.0;
                        for (int k = lane; k < bw[D - 1]; k += 32) {
                            const double2 f = tl[k], uv = urow[k];
                            rr += uv.x * f.x - uv.y * f.y;
                            ri += uv.x * f.y + uv.y * f.x;
                        }
                        accr += fo.x * rr - fo.y * ri;
                        acci += fo.x * ri + fo.y * rr;
                    }
                }
                __syncwarp();  // the next packet rewrites the table
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                accr += __shfl_xor_sync(0xffffffffu, accr, o);
                acci += __shfl_xor_sync(0xffffffffu, acci, o);
            }
        } else {
            float bdl[D], bt0[D], bnh[D], bnl[D];
#pragma unroll
            for (int l = 0; l < D; ++l) {
                bdl[l] = __shfl_sync(0xffffffffu, dl[l], t);
                bt0[l] = __shfl_sync(0xffffffffu, t0[l], t);
                bnh[l] = __shfl_sync(0xffffffffu, nh[l], t);
                bnl[l] = __shfl_sync(0xffffffffu, nl[l], t);
            }
            float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;  // Kahan sums
            const float2 *u = reinterpret_cast<const float2 *>(u_v);
            if constexpr (D == 1) {
                // lane owns the points k = lane + 32 i; every eighth is
                // evaluated in full, the next seven by the recurrences over
                // the stride H = 32 h (coalesced loads of u)
                const float h = P.hf[0], ce = P.ce, H = 32.f * h;
                float nu32 = 32.f * bnh[0];
                nu32 -= rint_fast(nu32);
                nu32 += 32.f * bnl[0];
                float rs_, rc_;
                __sincosf(kTwoPi * nu32, &rs_, &rc_);  // e^{2 pi i 32 nu}
                const float c2 = ex2_approx(2.f * ce * H * H);
                const float2 *ub = u + bb[0];
                const int w = bw[0];
                for (int k = lane; k < w; k += 32 * kDecGroup) {
                    const float dx = fmaf((float)k, h, bdl[0]);
                    float rho = ex2_approx(ce * H * fmaf(2.f, dx, H));
                    float2 e = factor32(k, h, bdl[0], bt0[0], bnh[0], bnl[0], ce);
                    float2 uv = ub[k];
                    float tr = uv.x * e.x - uv.y * e.y, ti = uv.x * e.y + uv.y * e.x;
#pragma unroll
                    for (int i = 1; i < kDecGroup; ++i) {
                        if (k + 32 * i < w) {
                            const float pr = rc_ * rho, pi = rs_ * rho;
                            e = make_float2(e.x * pr - e.y * pi, e.x * pi + e.y * pr);
                            rho *= c2;
                            uv = ub[k + 32 * i];
                            tr = fmaf(uv.x, e.x, fmaf(-uv.y, e.y, tr));
                            ti = fmaf(uv.x, e.y, fmaf(uv.y, e.x, ti));
                        }
                    }
                    kahan_add(sr, cr, tr);
                    kahan_add(si, ci, ti);
                }
            } else {
#pragma unroll
                for (int l = 0; l < D; ++l)
                    for (int k = lane; k < bw[l]; k += 32)
                        tab[P.tab_off[l] + k] = factor32(k, P.hf[l], bdl[l], bt0[l], bnh[l], bnl[l], P.ce);
                __syncwarp();
                switch (P.kl_regs) {
                case 2: rows32<D, 2>(u, tab, P, bb, bw, lane, sr, cr, si, ci); break;
                case 4: rows32<D, 4>(u, tab, P, bb, bw, lane, sr, cr, si, ci); break;
                case 8: rows32<D, 8>(u, tab, P, bb, bw, lane, sr, cr, si, ci); break;
                default: rows32<D, 0>(u, tab, P, bb, bw, lane, sr, cr, si, ci); break;
                }
                __syncwarp();  // the next packet rewrites the table
            }
            sr -= cr;
            si -= ci;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            accr = (double)sr;
            acci = (double)si;
        }
        if (lane == t) {
            out_r = accr;
            out_i = acci;
        }
    }
    if (mine) {
        a[jl] = P.weight * out_r;
        a[m + jl] = P.weight * out_i;
        s[jl] = 0.0;
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

template <int D, bool FP64>
fgr_status launch_decompose(unsigned blocks, int threads, size_t smem, cudaStream_t st, const void *u,
                            const double *q, const double *p, double *a, double *s, int64_t m,
                            const DecParams &P) {
    if (smem > 48 * 1024)
        FGR_CUDA_TRY(cudaFuncSetAttribute(decompose_kernel<D, FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    decompose_kernel<D, FP64><<<blocks, threads, smem, st>>>(u, q, p, a, s, m, P);
    return FGR_OK;
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
    const Grid &Gd = ctx->grid;
    const Mesh &M = ctx->mesh;
    const int D = ctx->d;
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    DecParams P{};
    double weight = std::pow(2.0, 0.5 * D);
    int wmax = 1, tab = 0;
    for (int l = 0; l < 3; ++l) {
        P.n[l] = l < D ? Gd.n[l] : 1;
        P.lo[l] = l < D ? Gd.lo[l] : 0.0;
        P.h[l] = l < D ? Gd.h[l] : 1.0;
        P.hf[l] = (float)P.h[l];
        P.wcap[l] = 1;
        if (l < D) {
            weight *= Gd.h[l];
            // a window holds at most floor(2 rs / h) + 1 points (+1 for the
            // rounding of the two bounds)
            const double wc = std::min<double>(std::floor(2.0 * M.rs / Gd.h[l]) + 2.0, (double)Gd.n[l]);
            if (wc > (double)(1 << 30)) {
                set_error("decompose: window of more than 2^30 points");
                return FGR_E_INVALID;
            }
            P.wcap[l] = (int)wc;
            wmax = std::max(wmax, P.wcap[l]);
            P.tab_off[l] = tab;
            tab += P.wcap[l];
        }
    }
    P.tab_len = D >= 2 ? tab : 0;
    P.kl_regs = 0;
    if (D >= 2)
        for (int kl : {2, 4, 8})
            if (P.kl_regs == 0 && P.wcap[D - 1] <= 32 * kl) P.kl_regs = kl;
    P.rs = M.rs;
    P.inv_eps = 1.0 / M.eps;
    P.inv_2pi_eps = 1.0 / (2.0 * M_PI * M.eps);
    P.neg_half_inv_eps = -0.5 / M.eps;
    P.weight = weight;
    P.ce = (float)(-1.4426950408889634 / (2.0 * M.eps));
    int lbits = 1;
    while ((int64_t(1) << lbits) < (int64_t)wmax + 1) ++lbits;
    P.two_pow_b = std::ldexp(1.0, std::max(1, 24 - lbits));
    P.inv_two_pow_b = 1.0 / P.two_pow_b;
    // warps per CTA: the per-warp factor tables (d >= 2) must fit shared memory
    const size_t per_warp = (size_t)P.tab_len * (fp64 ? sizeof(double2) : sizeof(float2));
    int warps = kDecMaxWarps;
    while (warps > 1 && (size_t)warps * per_warp > (size_t)96 * 1024) warps /= 2;
    if ((size_t)warps * per_warp > (size_t)200 * 1024) {
        set_error("decompose: windows of %d points per dimension exceed the factor tables", wmax);
        return FGR_E_INVALID;
    }
    // packets per warp: amortise the FP64 set-up over up to 32 packets while
    // keeping at least 32 warps per SM busy
    int G = 32;
    while (G > 1 && (m + G - 1) / G < (int64_t)ctx->num_sms * 32) G /= 2;
    P.group = G;
    const int64_t nwarps = (m + G - 1) / G;
    const unsigned blocks = (unsigned)((nwarps + warps - 1) / warps);
    const size_t smem = (size_t)warps * per_warp;
    const int threads = 32 * warps;
    fgr_status rc = FGR_OK;
#define FGR_DEC(DD)                                                                              \
    rc = fp64 ? launch_decompose<DD, true>(blocks, threads, smem, st, u_dev, q, p, a, s, m, P)   \
              : launch_decompose<DD, false>(blocks, threads, smem, st, u_dev, q, p, a, s, m, P);
    switch (D) {
    case 1: FGR_DEC(1); break;
    case 2: FGR_DEC(2); break;
    default: FGR_DEC(3); break;
    }
#undef FGR_DEC
    if (rc != FGR_OK) return rc;
    FGR_CUDA_TRY(cudaGetLastError());
    ctx->timing.last.launches = 1;
    return FGR_OK;
}

}  // namespace fgr
