// K1: per-packet FP64 RK4 of the frozen Gaussian trajectories (eq. 2.3-2.7).
//
// For the separable potentials of the ABI the Hessian of V is diagonal, so the
// Jacobian blocks F = dQ/dq, G = dQ/dp, H = dP/dq, K = dP/dp are diagonal and
// each dimension carries four scalars.  Per dimension l:
//   Q' = P,  P' = -V_l'(Q),  F' = H,  G' = K,  H' = -V_l''(Q) F,  K' = -V_l''(Q) G,
// and S' = |P|^2/2 - V(Q).  RK4 integrates (Q, P, F, G, H, K, S).
//
// Amplitude.  Eq. 2.6, A' = (A/2) tr(Z^{-1} Z'), integrates in closed form:
// tr(Z^{-1} Z') = d/dt log det Z, so A(t) = A(0) (det Z(t) / det Z(0))^{1/2}
// with det Z = prod_l Z_l, Z_l = F - iG + iH + K and Z(0) = 2I.  The square root
// follows the continuous branch: starting from the principal value 1 at t = 0,
// it changes sign each time some Z_l crosses the negative real axis, which the
// kernel counts after every step (Z is never zero, and moves O(dt) per step).
// This replaces a complex division per dimension and stage; it agrees with an
// RK4 integration of eq. 2.6 to the RK4 truncation error, O(dt^4).
//
// Trigonometry (cosine potential).  sin and cos of k Q are evaluated once per
// step; stages 2 and 4 rotate them by the stage offset d = k (Q_stage - Q),
// |d| <= k h (|P| + h |amp| k), with cos d and sin d from their Taylor series:
// to d^4 / d^5 while that bound is below 2e-3 (first omitted terms below
// 1e-19), to d^6 / d^7 below 0.02, and by sincos at every stage above it
// (large steps or momenta).  Stage 3 sits at the same time as stage 2 and its
// position differs from stage 2's by (h/2)^2 |V'| <= k h^2 |amp k| / 4; where
// that is below 1e-6 for every packet (a property of h, k and amp, checked
// once per launch), stage 3 rotates stage 2's values with cos d = 1 - d^2/2
// and sin d = d (omitted terms below 2e-19).  Under the same kind of bound,
// k h^2 |amp k| <= 1e-6, the next step's sin and cos come from stage 4's the
// same way (Q(t+h) - Q_stage4 = h (P1 + 2 P2 + 2 P3 + P4)/6 - h P3, at most
// h^2 |amp k| in size), and sincos is evaluated afresh every 32nd step so that
// the rounding of the chained rotations stays below 1e-14.
//
// One thread integrates one packet with the whole state in registers.
#include "internal.h"

namespace fgr {
namespace {

struct Pot {
    double c0, amp, k, omega2;
    double ampk, ampk2;  // amp*k, amp*k^2
};

template <int D>
struct State {
    double Q[D], P[D], F[D], G[D], H[D], K[D], S;
};

// sin/cos of (x + d) from sin/cos of x by the Taylor series of cos d and sin d
// (to d^6 and d^7; for |d| <= 0.025 the first omitted term is below 2e-18).
__device__ __forceinline__ void rotate_small(double s0, double c0, double d, double &s, double &c) {
    const double d2 = d * d;
    const double cd = 1.0 + d2 * (-0.5 + d2 * (1.0 / 24.0 + d2 * (-1.0 / 720.0)));
    const double sd = d * (1.0 + d2 * (-1.0 / 6.0 + d2 * (1.0 / 120.0 + d2 * (-1.0 / 5040.0))));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
}

// The same to d^4 and d^5 (for |d| <= 2e-3 the first omitted term is below
// 1e-19).
__device__ __forceinline__ void rotate_tiny(double s0, double c0, double d, double &s, double &c) {
    const double d2 = d * d;
    const double cd = 1.0 + d2 * (-0.5 + d2 * (1.0 / 24.0));
    const double sd = d * (1.0 + d2 * (-1.0 / 6.0 + d2 * (1.0 / 120.0)));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
}

// For |d| <= 1e-6: cos d = 1 - d^2/2, sin d = d (omitted terms below 2e-19).
__device__ __forceinline__ void rotate_micro(double s0, double c0, double d, double &s, double &c) {
    const double cd = fma(-0.5 * d, d, 1.0);
    s = fma(c0, d, s0 * cd);
    c = fma(-s0, d, c0 * cd);
}

// per-dimension choice of the stage trigonometry for one step
enum Trig : unsigned char { kTiny = 0, kSmall = 1, kFull = 2 };

// right-hand side; sn/cs = sin/cos(k Q_l) (cosine potential only)
template <int D, int KIND>
__device__ __forceinline__ void rhs(const Pot &v, const State<D> &y, const double *sn, const double *cs,
                                    State<D> &dy) {
    double pot = 0.0, p2 = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        double g, hs;  // V_l', V_l''
        if (KIND == FGR_V_COSSUM) {
            g = -v.ampk * sn[l];
            hs = -v.ampk2 * cs[l];
            pot += cs[l];
        } else if (KIND == FGR_V_HARMONIC) {
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
    }
    double V = 0.0;
    if (KIND == FGR_V_COSSUM) V = v.c0 + v.amp * pot;
    else if (KIND == FGR_V_HARMONIC) V = 0.5 * v.omega2 * pot;
    dy.S = 0.5 * p2 - V;
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
}

// sin/cos of k Q at a stage from their values at the step start (Q0)
template <int D, int KIND>
__device__ __forceinline__ void stage_trig(const Pot &v, const double *Q0, const State<D> &tmp,
                                           const double *s0, const double *c0, const Trig *how, double *sn,
                                           double *cs) {
    if (KIND == FGR_V_COSSUM) {
#pragma unroll
        for (int l = 0; l < D; ++l) {
            if (how[l] == kTiny)
                rotate_tiny(s0[l], c0[l], v.k * (tmp.Q[l] - Q0[l]), sn[l], cs[l]);
            else if (how[l] == kSmall)
                rotate_small(s0[l], c0[l], v.k * (tmp.Q[l] - Q0[l]), sn[l], cs[l]);
            else
                sincos(v.k * tmp.Q[l], &sn[l], &cs[l]);
        }
    }
}

// stage 3 from stage 2 (same time, positions (h/2)^2 |V'| apart)
template <int D, int KIND>
__device__ __forceinline__ void stage3_trig(const Pot &v, bool micro, const double *Q0, const double *Q2,
                                            const State<D> &tmp, const double *s0, const double *c0,
                                            const Trig *how, double *sn, double *cs) {
    if (KIND == FGR_V_COSSUM) {
        if (micro) {
#pragma unroll
            for (int l = 0; l < D; ++l)
                if (how[l] != kFull) rotate_micro(sn[l], cs[l], v.k * (tmp.Q[l] - Q2[l]), sn[l], cs[l]);
                else sincos(v.k * tmp.Q[l], &sn[l], &cs[l]);
        } else {
            stage_trig<D, KIND>(v, Q0, tmp, s0, c0, how, sn, cs);
        }
    }
}

template <int D, int KIND>
__device__ __forceinline__ void rk4_body(double *__restrict__ q, double *__restrict__ p, double *__restrict__ s,
                                         double *__restrict__ a, int64_t m, const Pot &v, int64_t nsteps,
                                         double h) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    State<D> y;
    bool im_pos[D];
    int flips = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        y.Q[l] = q[l * m + j];
        y.P[l] = p[l * m + j];
        y.F[l] = 1.0;
        y.G[l] = 0.0;
        y.H[l] = 0.0;
        y.K[l] = 1.0;
        im_pos[l] = true;  // Z(0) = 2: Im Z = +0
    }
    y.S = s[j];
    const double h2 = 0.5 * h, h6 = h / 6.0;
    double s0[D], c0[D], sn[D], cs[D], Q0[D], Q2[D], Q4[D];
    Trig how[D];
    const double kh = fabs(v.k) * h, kh_margin = kh * h * fabs(v.ampk);
    const bool micro = 0.25 * kh_margin <= 1e-6;  // stage 3 from stage 2
    const bool carry = kh_margin <= 1e-6;         // next step from stage 4
    for (int64_t it = 0; it < nsteps; ++it) {
        if (KIND == FGR_V_COSSUM) {
            const bool fresh = !carry || (it & 31) == 0;
#pragma unroll
            for (int l = 0; l < D; ++l) {
                if (fresh)
                    sincos(v.k * y.Q[l], &s0[l], &c0[l]);
                else
                    rotate_micro(sn[l], cs[l], v.k * (y.Q[l] - Q4[l]), s0[l], c0[l]);
                const double bound = fabs(y.P[l]) * kh + kh_margin;
                how[l] = bound <= 2e-3 ? kTiny : (bound <= 0.02 ? kSmall : kFull);
                Q0[l] = y.Q[l];
            }
        }
        State<D> k, tmp, acc;
        rhs<D, KIND>(v, y, s0, c0, k);
        acc = k;
        axpy<D>(tmp, y, h2, k);
        stage_trig<D, KIND>(v, Q0, tmp, s0, c0, how, sn, cs);
#pragma unroll
        for (int l = 0; l < D; ++l) Q2[l] = tmp.Q[l];
        rhs<D, KIND>(v, tmp, sn, cs, k);
        accum<D>(acc, 2.0, k);
        axpy<D>(tmp, y, h2, k);
        stage3_trig<D, KIND>(v, micro, Q0, Q2, tmp, s0, c0, how, sn, cs);
        rhs<D, KIND>(v, tmp, sn, cs, k);
        accum<D>(acc, 2.0, k);
        axpy<D>(tmp, y, h, k);
        stage_trig<D, KIND>(v, Q0, tmp, s0, c0, how, sn, cs);
#pragma unroll
        for (int l = 0; l < D; ++l) Q4[l] = tmp.Q[l];
        rhs<D, KIND>(v, tmp, sn, cs, k);
        accum<D>(acc, 1.0, k);
        axpy<D>(y, y, h6, acc);
        // branch of sqrt(det Z): count crossings of the negative real axis
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const bool pos = (y.H[l] - y.G[l]) >= 0.0;
            if (pos != im_pos[l] && (y.F[l] + y.K[l]) < 0.0) flips ^= 1;
            im_pos[l] = pos;
        }
    }
    // A = A(0) prod_l sqrt(Z_l / 2), continuous branch
    double wr = 1.0, wi = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const double x = 0.5 * (y.F[l] + y.K[l]), yv = 0.5 * (y.H[l] - y.G[l]);
        const double r = hypot(x, yv);
        double sr, si;
        if (x >= 0.0) {
            sr = sqrt(0.5 * (r + x));
            si = yv / (2.0 * sr);
        } else {
            const double t = sqrt(0.5 * (r - x));
            si = yv >= 0.0 ? t : -t;
            sr = yv / (2.0 * si);
        }
        const double nr = wr * sr - wi * si, ni = wr * si + wi * sr;
        wr = nr;
        wi = ni;
    }
    if (flips) {
        wr = -wr;
        wi = -wi;
    }
#pragma unroll
    for (int l = 0; l < D; ++l) {
        q[l * m + j] = y.Q[l];
        p[l * m + j] = y.P[l];
    }
    s[j] = y.S;
    const double ar = a[j], ai = a[m + j];
    a[j] = ar * wr - ai * wi;
    a[m + j] = ar * wi + ai * wr;
}

template <int D, int KIND>
__global__ void __launch_bounds__(128) rk4_kernel(double *__restrict__ q, double *__restrict__ p,
                                                  double *__restrict__ s, double *__restrict__ a, int64_t m,
                                                  Pot v, int64_t nsteps, double h) {
    rk4_body<D, KIND>(q, p, s, a, m, v, nsteps, h);
}

// (A 1-D variant capped at 80 registers for 6 CTAs per SM ran 4% slower: the
// FP64 pipe stays 86% busy and the cap adds recomputation.)
template <int D, int KIND>
void launch_rk4(unsigned blocks, int threads, cudaStream_t st, double *q, double *p, double *s, double *a,
                int64_t m, const Pot &v, int64_t nsteps, double h) {
    rk4_kernel<D, KIND><<<blocks, threads, 0, st>>>(q, p, s, a, m, v, nsteps, h);
}

template <int D>
void launch_kind(int kind, unsigned blocks, int threads, cudaStream_t st, double *q, double *p, double *s,
                 double *a, int64_t m, Pot v, int64_t nsteps, double h) {
    if (kind == FGR_V_COSSUM)
        launch_rk4<D, FGR_V_COSSUM>(blocks, threads, st, q, p, s, a, m, v, nsteps, h);
    else if (kind == FGR_V_HARMONIC)
        launch_rk4<D, FGR_V_HARMONIC>(blocks, threads, st, q, p, s, a, m, v, nsteps, h);
    else
        launch_rk4<D, FGR_V_FREE>(blocks, threads, st, q, p, s, a, m, v, nsteps, h);
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
    Pot v{vp->c0, vp->amp, vp->k, vp->omega * vp->omega, vp->amp * vp->k, vp->amp * vp->k * vp->k};
    const int threads = 128;
    const unsigned blocks = (unsigned)((m + threads - 1) / threads);
    switch (ctx->d) {
    case 1: launch_kind<1>(vp->kind, blocks, threads, st, q, p, s, a, m, v, nsteps, h); break;
    case 2: launch_kind<2>(vp->kind, blocks, threads, st, q, p, s, a, m, v, nsteps, h); break;
    default: launch_kind<3>(vp->kind, blocks, threads, st, q, p, s, a, m, v, nsteps, h); break;
    }
    FGR_CUDA_TRY(cudaGetLastError());
    ctx->timing.last.launches = 1;
    timer.mark(&ctx->timing.last.propagate_ms);
    timer.finish();
    return FGR_OK;
}

}  // namespace fgr
