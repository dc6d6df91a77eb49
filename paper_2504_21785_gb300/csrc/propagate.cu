// K1: per-packet FP64 RK4 of the frozen Gaussian trajectories (eq. 2.3-2.7).
//
// For the separable potentials of the ABI the Hessian of V is diagonal, so the
// Jacobian blocks F = dQ/dq, G = dQ/dp, H = dP/dq, K = dP/dp are diagonal too and
// each dimension carries four scalars.  Per dimension l:
//   Q' = P,  P' = -V_l'(Q),  F' = H,  G' = K,  H' = -V_l''(Q) F,  K' = -V_l''(Q) G,
//   Z_l = F - iG + iH + K,  Z_l' = H - iK - i V_l'' F - V_l'' G,
// and  S' = |P|^2/2 - V(Q),  A' = (A/2) sum_l Z_l'/Z_l  (tr(Z^{-1} Z') for diagonal Z).
// One thread integrates one packet with the whole state in registers.
#include "internal.h"

namespace fgr {
namespace {

struct Pot {
    int kind;
    double c0, amp, k, omega2;
};

template <int D>
struct State {
    double Q[D], P[D], F[D], G[D], H[D], K[D], S, Ar, Ai;
};

template <int D>
__device__ __forceinline__ void rhs(const Pot &v, const State<D> &y, State<D> &dy) {
    double pot = 0.0, p2 = 0.0, tr_r = 0.0, tr_i = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        double g, hs;  // V_l', V_l''
        if (v.kind == FGR_V_COSSUM) {
            double sn, cs;
            sincos(v.k * y.Q[l], &sn, &cs);
            g = -v.amp * v.k * sn;
            hs = -v.amp * v.k * v.k * cs;
            pot += cs;
        } else if (v.kind == FGR_V_HARMONIC) {
            g = v.omega2 * y.Q[l];
            hs = v.omega2;
            pot += y.Q[l] * y.Q[l];
        } else {
            g = 0.0;
            hs = 0.0;
        }
        dy.Q[l] = y.P[l];
        dy.P[l] = -g;
        dy.F[l] = y.H[l];
        dy.G[l] = y.K[l];
        dy.H[l] = -hs * y.F[l];
        dy.K[l] = -hs * y.G[l];
        p2 += y.P[l] * y.P[l];
        // Z and Z'
        double zr = y.F[l] + y.K[l], zi = y.H[l] - y.G[l];
        double wr = y.H[l] - hs * y.G[l], wi = -y.K[l] - hs * y.F[l];
        double den = zr * zr + zi * zi;
        tr_r += (wr * zr + wi * zi) / den;
        tr_i += (wi * zr - wr * zi) / den;
    }
    double V = 0.0;
    if (v.kind == FGR_V_COSSUM) V = v.c0 + v.amp * pot;
    else if (v.kind == FGR_V_HARMONIC) V = 0.5 * v.omega2 * pot;
    dy.S = 0.5 * p2 - V;
    dy.Ar = 0.5 * (y.Ar * tr_r - y.Ai * tr_i);
    dy.Ai = 0.5 * (y.Ar * tr_i + y.Ai * tr_r);
}

template <int D>
__device__ __forceinline__ void axpy(State<D> &out, const State<D> &y, double h, const State<D> &k) {
#pragma unroll
    for (int l = 0; l < D; ++l) {
        out.Q[l] = y.Q[l] + h * k.Q[l];
        out.P[l] = y.P[l] + h * k.P[l];
        out.F[l] = y.F[l] + h * k.F[l];
        out.G[l] = y.G[l] + h * k.G[l];
        out.H[l] = y.H[l] + h * k.H[l];
        out.K[l] = y.K[l] + h * k.K[l];
    }
    out.S = y.S + h * k.S;
    out.Ar = y.Ar + h * k.Ar;
    out.Ai = y.Ai + h * k.Ai;
}

template <int D>
__device__ __forceinline__ void accum(State<D> &acc, double w, const State<D> &k) {
#pragma unroll
    for (int l = 0; l < D; ++l) {
        acc.Q[l] += w * k.Q[l];
        acc.P[l] += w * k.P[l];
        acc.F[l] += w * k.F[l];
        acc.G[l] += w * k.G[l];
        acc.H[l] += w * k.H[l];
        acc.K[l] += w * k.K[l];
    }
    acc.S += w * k.S;
    acc.Ar += w * k.Ar;
    acc.Ai += w * k.Ai;
}

template <int D>
__global__ void __launch_bounds__(128) rk4_kernel(double *__restrict__ q, double *__restrict__ p,
                                                  double *__restrict__ s, double *__restrict__ a,
                                                  int64_t m, Pot v, int64_t nsteps, double h) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    State<D> y;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        y.Q[l] = q[l * m + j];
        y.P[l] = p[l * m + j];
        y.F[l] = 1.0;
        y.G[l] = 0.0;
        y.H[l] = 0.0;
        y.K[l] = 1.0;
    }
    y.S = s[j];
    y.Ar = a[j];
    y.Ai = a[m + j];
    const double h2 = 0.5 * h, h6 = h / 6.0;
    for (int64_t it = 0; it < nsteps; ++it) {
        State<D> k, tmp, acc;
        rhs<D>(v, y, k);
        acc = k;
        axpy<D>(tmp, y, h2, k);
        rhs<D>(v, tmp, k);
        accum<D>(acc, 2.0, k);
        axpy<D>(tmp, y, h2, k);
        rhs<D>(v, tmp, k);
        accum<D>(acc, 2.0, k);
        axpy<D>(tmp, y, h, k);
        rhs<D>(v, tmp, k);
        accum<D>(acc, 1.0, k);
        axpy<D>(y, y, h6, acc);
    }
#pragma unroll
    for (int l = 0; l < D; ++l) {
        q[l * m + j] = y.Q[l];
        p[l * m + j] = y.P[l];
    }
    s[j] = y.S;
    a[j] = y.Ar;
    a[m + j] = y.Ai;
}

}  // namespace

fgr_status run_propagate(fgr_ctx *ctx, double *q, double *p, double *s, double *a, int64_t m,
                         const fgr_potential *vp, double t, double dt, cudaStream_t st) {
    StageTimer timer(ctx, st);
    const int64_t nsteps = rk4_nsteps(t, dt);
    if (m == 0 || nsteps == 0) {
        timer.finish();
        return FGR_OK;
    }
    const double h = t / (double)nsteps;
    Pot v{vp->kind, vp->c0, vp->amp, vp->k, vp->omega * vp->omega};
    const int threads = 128;
    const unsigned blocks = (unsigned)((m + threads - 1) / threads);
    switch (ctx->d) {
    case 1: rk4_kernel<1><<<blocks, threads, 0, st>>>(q, p, s, a, m, v, nsteps, h); break;
    case 2: rk4_kernel<2><<<blocks, threads, 0, st>>>(q, p, s, a, m, v, nsteps, h); break;
    default: rk4_kernel<3><<<blocks, threads, 0, st>>>(q, p, s, a, m, v, nsteps, h); break;
    }
    FGR_CUDA_TRY(cudaGetLastError());
    ctx->timing.last.launches = 1;
    timer.mark(&ctx->timing.last.propagate_ms);
    timer.finish();
    return FGR_OK;
}

}  // namespace fgr
