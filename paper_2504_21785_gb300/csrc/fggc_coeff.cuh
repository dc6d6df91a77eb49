// K3+K4: FGGC coefficients and scatter (Algorithm 2 Step 3, eq. 2.25).
// Included by fggc_coeff1.cu / fggc_coeff2.cu / fggc_coeff3.cu, one per
// dimension, so the heavily unrolled instantiations compile in parallel.
// See fggc.cu for the layout of the node array and the folded node phase.
#pragma once

#include "device_util.cuh"
#include "fggc_params.h"

namespace fgr {
namespace {

// ---------------------------------------------------------------------------
// coefficients + scatter
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double &cr, double &ci) {
    cr = ar * br - ai * bi;
    ci = ar * bi + ai * br;
}
__device__ __forceinline__ void cmul(float ar, float ai, float br, float bi, float &cr, float &ci) {
    cr = ar * br - ai * bi;
    ci = ar * bi + ai * br;
}

// Parameter views of one request inside a batch: that request's constants
// with the least-squares tables shared by the batch (same strategy).
struct Params64View {
    const Common &c;
    const double *vr, *vi, *inv_lam;
};
struct Params32View {
    const Common &c;
    const float *cre, *cim;
};

// FP64: per-dimension coefficients through the eigen factors (PT: Params64
// or Params64View).
template <int N, class PT>
__device__ __forceinline__ void coeff_dim64(const PT &P, double Q, double Pm, int &a0, int &b0,
                                            double *cr, double *ci) {
    const Common &c = P.c;
    const double r = __ddiv_rn(Q, c.dqv), rp = __ddiv_rn(Pm, c.dpv);
    const double fa = floor(r), fb = floor(rp);
    const double s = r - fa, t = rp - fb;
    a0 = (int)fmin(fmax(fa, -1e9), 1e9);
    b0 = (int)fmin(fmax(fb, -1e9), 1e9);
    constexpr int n = N;
    double fr[N], fi[N];
#pragma unroll
    for (int j = 0; j < n; ++j) {  // eq. 3.23
        const double u = c.dq[j] - s, v = c.dp[j] - t;
        const double mag = exp(-c.cq2_4 * u * u - c.cp2_4 * v * v);
        double sn, cs;
        sincos(c.half_cqcp * (s - c.dq[j]) * (c.dp[j] + t), &sn, &cs);
        fr[j] = mag * cs;
        fi[j] = mag * sn;
    }
    double yr[N], yi[N];
#pragma unroll
    for (int i = 0; i < n; ++i) {  // y = diag(1/lam) V^H f
        double sr = 0, si = 0;
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const double vr = P.vr[j * kMaxN1 + i], vi = P.vi[j * kMaxN1 + i];
            sr += vr * fr[j] + vi * fi[j];
            si += vr * fi[j] - vi * fr[j];
        }
        yr[i] = sr * P.inv_lam[i];
        yi[i] = si * P.inv_lam[i];
    }
    // node phase base (turns): -cc * r * b0 and -cc * a0
    double t0 = -c.cc * (r * fb);
    t0 -= rint(t0);
    double t1 = -c.cc * fa;
    t1 -= rint(t1);
#pragma unroll
    for (int k = 0; k < n; ++k) {  // c~ = conj(V y), times the node phase
        double sr = 0, si = 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const double vr = P.vr[k * kMaxN1 + i], vi = P.vi[k * kMaxN1 + i];
            sr += vr * yr[i] - vi * yi[i];
            si += vr * yi[i] + vi * yr[i];
        }
        si = -si;
        double tk = t0 + c.dp[k] * t1 - c.cc * (double)(c.dq[k] * c.dp[k]);
        tk -= rint(tk);
        double sn, cs;
        sincospi(2.0 * tk, &sn, &cs);
        cmul(sr, si, cs, sn, cr[k], ci[k]);
    }
}

// FP32: per-dimension coefficients through the Chebyshev surrogate (PT:
// Params32 or Params32View).
template <int N, class PT>
__device__ __forceinline__ void coeff_dim32(const PT &P, double Q, double Pm, int &a0, int &b0,
                                            float *cr, float *ci) {
    const Common &c = P.c;
    // the floors of Q/dq and P/dp as the FP64 division decides them (FP32
    // estimate, FP64 only near an integer); the fractions from one FP64
    // product each (within a few ulps of the quotient, which is all the FP32
    // surrogate below can resolve)
    a0 = floor_div_int(Q, c.dqv, c.inv_dq);
    b0 = floor_div_int(Pm, c.dpv, c.inv_dp);
    const double fa = (double)a0, fb = (double)b0;
    const double r = Q * c.inv_dq, rp = Pm * c.inv_dp;
    const float xs = fmaf(2.f, (float)(r - fa), -1.f), xt = fmaf(2.f, (float)(rp - fb), -1.f);
    float Ts[kCheb], Tt[kCheb];
    Ts[0] = 1.f;
    Ts[1] = xs;
    Tt[0] = 1.f;
    Tt[1] = xt;
#pragma unroll
    for (int i = 2; i < kCheb; ++i) {
        Ts[i] = 2.f * xs * Ts[i - 1] - Ts[i - 2];
        Tt[i] = 2.f * xt * Tt[i - 1] - Tt[i - 2];
    }
    double t0 = -c.cc * (r * fb);
    t0 -= rint(t0);
    double t1 = -c.cc * fa;
    t1 -= rint(t1);
    const float t0f = (float)t0, t1f = (float)t1, ccf = (float)c.cc;
    constexpr int n = N;
#pragma unroll
    for (int k = 0; k < n; ++k) {
        float sr = 0.f, si = 0.f;
        const float *Cr = P.cre + k * kCheb * kCheb, *Ci = P.cim + k * kCheb * kCheb;
#pragma unroll
        for (int i = 0; i < kCheb; ++i) {
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int j = 0; j < kCheb; ++j) {
                if (i + j <= cheb_total<N>()) {
                    ur = fmaf(Cr[i * kCheb + j], Tt[j], ur);
                    ui = fmaf(Ci[i * kCheb + j], Tt[j], ui);
                }
            }
            sr = fmaf(Ts[i], ur, sr);
            si = fmaf(Ts[i], ui, si);
        }
        float tk = t0f + (float)c.dp[k] * t1f - ccf * (float)(c.dq[k] * c.dp[k]);
        tk -= rint_fast(tk);
        float sn, cs;
        sincospif(2.f * tk, &sn, &cs);
        cmul(sr, si, cs, sn, cr[k], ci[k]);
    }
}

// The last dimension's N1 contributions of one row of outer neighbours,
// scaled by (pr, pi): cell idx + (a0 + dq_k - amin) sa + (b0 + dp_k - bmin) sb.
template <int L, int N1, class Real, class C2>
__device__ __forceinline__ void emit_row(C2 *__restrict__ W, const Common &c, int a0, int b0, const Real *cl_r,
                                         const Real *cl_i, int64_t idx, Real pr, Real pi) {
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        const int ia = a0 + c.dq[k] - c.amin[L], ib = b0 + c.dp[k] - c.bmin[L];
        if ((unsigned)ia < (unsigned)c.A[L] && (unsigned)ib < (unsigned)c.B[L]) {
            Real vr, vi;
            cmul(pr, pi, cl_r[k], cl_i[k], vr, vi);
            atomic_add_c(W + idx + ia * c.sa[L] + ib * c.sb[L], vr, vi);
        }
    }
}

// Threads per CTA of the scatter kernel: the coefficients of all dimensions
// but the last wait in shared memory ([dim][neighbour][thread], at most 32 KB).
template <bool FP64, int N1>
__host__ __device__ constexpr int coeff_threads() {
    return (FP64 && N1 == 16) ? 64 : 128;
}

template <bool FP64>
using ParamsT = typename std::conditional<FP64, Params64, Params32>::type;

template <int D, bool FP64, int N1, class PT>
__device__ __forceinline__ void coeff_scatter_body(const double *__restrict__ q, const double *__restrict__ p,
                                                   const double *__restrict__ s, const double *__restrict__ a,
                                                   int64_t m, int64_t j, const PT &P,
                                                   void *__restrict__ W_v, uint8_t *__restrict__ row_flag) {
    using Real = typename std::conditional<FP64, double, float>::type;
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    constexpr int kT = coeff_threads<FP64, N1>();
    __shared__ C2 scoef[D > 1 ? D - 1 : 1][N1][kT];
    const int tid = threadIdx.x;
    const Common &c = P.c;
    const double ar = a[j], ai = a[m + j];
    if (ar == 0.0 && ai == 0.0) return;  // contributes exact zeros
    // weight pref * A * e^{i S/eps}
    double ts = s[j] * c.inv_2pi_eps;
    ts -= rint(ts);
    Real wr, wi;
    if (FP64) {
        double sn, cs;
        sincospi(2.0 * ts, &sn, &cs);
        double xr, xi;
        cmul(ar * c.pref, ai * c.pref, cs, sn, xr, xi);
        wr = (Real)xr;
        wi = (Real)xi;
    } else {
        float sn, cs;
        sincospif(2.f * (float)ts, &sn, &cs);
        float xr, xi;
        cmul((float)(ar * c.pref), (float)(ai * c.pref), cs, sn, xr, xi);
        wr = (Real)xr;
        wi = (Real)xi;
    }
    // per-dimension coefficients: the last dimension's stay in registers, the
    // others go to this thread's column of shared memory (read back only by
    // this thread, so no barrier is needed)
    Real cl_r[N1], cl_i[N1];
    int a0[D], b0[D];
    // one dimension at a time (for d = 3 not unrolled: three unrolled copies
    // of the coefficient evaluation do not fit the register file)
#pragma unroll(D == 3 ? 1 : D)
    for (int l = 0; l < D; ++l) {
        Real cr[N1], ci[N1];
        if constexpr (FP64)
            coeff_dim64<N1>(P, q[l * m + j], p[l * m + j], a0[l], b0[l], cr, ci);
        else
            coeff_dim32<N1>(P, q[l * m + j], p[l * m + j], a0[l], b0[l], cr, ci);
        if (l < D - 1) {
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                C2 v;
                v.x = cr[k];
                v.y = ci[k];
                scoef[l][k][tid] = v;
            }
        } else {
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                cl_r[k] = cr[k];
                cl_i[k] = ci[k];
            }
        }
    }
    C2 *W = reinterpret_cast<C2 *>(W_v);
    // tensor product over dimensions, innermost dimension last; the rows of
    // the first grid pass (the last dimension's [a][b] plane) that receive a
    // contribution are marked once per row (the single row of d = 1 is marked
    // by the host)
    if constexpr (D == 1) {
        emit_row<D - 1, N1>(W, c, a0[D - 1], b0[D - 1], cl_r, cl_i, 0, wr, wi);
    } else {
#pragma unroll 1
        for (int k0 = 0; k0 < N1; ++k0) {
            const int ia0 = a0[0] + c.dq[k0] - c.amin[0], ib0 = b0[0] + c.dp[k0] - c.bmin[0];
            const bool in0 = (unsigned)ia0 < (unsigned)c.A[0] && (unsigned)ib0 < (unsigned)c.B[0];
            if (!in0) continue;
            const int64_t idx0 = ia0 * c.sa[0] + ib0 * c.sb[0];
            const int64_t row0 = ia0 * c.ra[0] + ib0 * c.rb[0];
            const C2 c0 = scoef[0][k0][tid];
            Real p0r, p0i;
            cmul(wr, wi, c0.x, c0.y, p0r, p0i);
            if constexpr (D == 2) {
                row_flag[row0] = 1;
                emit_row<D - 1, N1>(W, c, a0[D - 1], b0[D - 1], cl_r, cl_i, idx0, p0r, p0i);
            } else {
#pragma unroll 1
                for (int k1 = 0; k1 < N1; ++k1) {
                    const int ia1 = a0[1] + c.dq[k1] - c.amin[1], ib1 = b0[1] + c.dp[k1] - c.bmin[1];
                    if ((unsigned)ia1 >= (unsigned)c.A[1] || (unsigned)ib1 >= (unsigned)c.B[1]) continue;
                    const C2 c1 = scoef[1][k1][tid];
                    Real p1r, p1i;
                    cmul(p0r, p0i, c1.x, c1.y, p1r, p1i);
                    row_flag[row0 + ia1 * c.ra[1] + ib1 * c.rb[1]] = 1;
                    emit_row<D - 1, N1>(W, c, a0[D - 1], b0[D - 1], cl_r, cl_i, idx0 + ia1 * c.sa[1] + ib1 * c.sb[1],
                                        p1r, p1i);
                }
            }
        }
    }
}

// d = 1, 2: the compiler's own register budget; d = 3: at most 128
// registers (4 CTAs per SM), which the three-dimensional emit loops need
template <int D, bool FP64, int N1>
__global__ void __launch_bounds__(coeff_threads<FP64, N1>()) coeff_scatter_kernel(
    const double *__restrict__ q, const double *__restrict__ p, const double *__restrict__ s,
    const double *__restrict__ a, int64_t m, const __grid_constant__ ParamsT<FP64> P, void *__restrict__ W_v,
    uint8_t *__restrict__ row_flag) {
    const int64_t j = blockIdx.x * (int64_t)coeff_threads<FP64, N1>() + threadIdx.x;
    if (j < m) coeff_scatter_body<D, FP64, N1>(q, p, s, a, m, j, P, W_v, row_flag);
}

template <int D, bool FP64, int N1>
__global__ void __launch_bounds__(coeff_threads<FP64, N1>(), 4) coeff_scatter3_kernel(
    const double *__restrict__ q, const double *__restrict__ p, const double *__restrict__ s,
    const double *__restrict__ a, int64_t m, const __grid_constant__ ParamsT<FP64> P, void *__restrict__ W_v,
    uint8_t *__restrict__ row_flag) {
    const int64_t j = blockIdx.x * (int64_t)coeff_threads<FP64, N1>() + threadIdx.x;
    if (j < m) coeff_scatter_body<D, FP64, N1>(q, p, s, a, m, j, P, W_v, row_flag);
}

// The same over the packets list[0 .. *count) (device count), grid-stride.
template <int D, bool FP64, int N1>
__global__ void __launch_bounds__(coeff_threads<FP64, N1>(), D == 3 ? 4 : 1) coeff_scatter_list_kernel(
    const double *__restrict__ q, const double *__restrict__ p, const double *__restrict__ s,
    const double *__restrict__ a, int64_t m, const __grid_constant__ ParamsT<FP64> P, void *__restrict__ W_v,
    uint8_t *__restrict__ row_flag, const int *__restrict__ list, const int *__restrict__ count) {
    constexpr int kT = coeff_threads<FP64, N1>();
    const int n = *count;
    for (int64_t t = blockIdx.x * (int64_t)kT + threadIdx.x; t < n; t += (int64_t)gridDim.x * kT)
        coeff_scatter_body<D, FP64, N1>(q, p, s, a, m, list[t], P, W_v, row_flag);
}

// Batched form: the CTAs of every request of a launch (same dimension,
// precision and neighbour strategy: shared least-squares tables).
template <int D, bool FP64, int N1>
__global__ void __launch_bounds__(coeff_threads<FP64, N1>(), D == 3 ? 4 : 1) coeff_scatter_batch_kernel(
    const __grid_constant__ typename std::conditional<FP64, ScatterBatch64, ScatterBatch32>::type B) {
    int r = 0;
    while (r + 1 < B.n && (int)blockIdx.x >= B.block0[r + 1]) ++r;
    const int64_t j = (int64_t)(blockIdx.x - B.block0[r]) * coeff_threads<FP64, N1>() + threadIdx.x;
    if (j >= B.m[r]) return;
    if constexpr (FP64) {
        const Params64View v{B.c[r], B.vr, B.vi, B.inv_lam};
        coeff_scatter_body<D, FP64, N1>(B.q[r], B.p[r], B.s[r], B.a[r], B.m[r], j, v, B.W[r], B.flags[r]);
    } else {
        const Params32View v{B.c[r], B.cre, B.cim};
        coeff_scatter_body<D, FP64, N1>(B.q[r], B.p[r], B.s[r], B.a[r], B.m[r], j, v, B.W[r], B.flags[r]);
    }
}

template <int D>
fgr_status launch_scatter_batch_dim(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32) {
    const int nb = b64 ? b64->block0[b64->n] : b32->block0[b32->n];
    if (nb == 0) return FGR_OK;
#define FGR_SB(N)                                                                                      \
    if (b64)                                                                                           \
        coeff_scatter_batch_kernel<D, true, N><<<nb, coeff_threads<true, N>(), 0, st>>>(*b64);         \
    else                                                                                               \
        coeff_scatter_batch_kernel<D, false, N><<<nb, coeff_threads<false, N>(), 0, st>>>(*b32);
    switch (n1) {
    case 4: FGR_SB(4); break;
    case 8: FGR_SB(8); break;
    case 16: FGR_SB(16); break;
    default: set_error("fggc: unsupported neighbour count %d", n1); return FGR_E_INVALID;
    }
#undef FGR_SB
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

template <int D, bool FP64, int N1>
void launch_coeff_kernel(unsigned blocks, cudaStream_t st, const PacketsDev &pk, const ParamsT<FP64> &P, void *W,
                         uint8_t *flags) {
    constexpr int T = coeff_threads<FP64, N1>();
    if constexpr (D == 3)
        coeff_scatter3_kernel<D, FP64, N1><<<blocks, T, 0, st>>>(pk.q, pk.p, pk.s, pk.a, pk.m, P, W, flags);
    else
        coeff_scatter_kernel<D, FP64, N1><<<blocks, T, 0, st>>>(pk.q, pk.p, pk.s, pk.a, pk.m, P, W, flags);
}

template <int D>
fgr_status launch_coeff_d(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64, const Params32 *p32,
                          void *W, uint8_t *flags) {
    if (pk.m == 0) return FGR_OK;
#define FGR_COEFF(N)                                                                                        \
    if (p64)                                                                                                \
        launch_coeff_kernel<D, true, N>((unsigned)((pk.m + coeff_threads<true, N>() - 1) /                  \
                                                   coeff_threads<true, N>()), st, pk, *p64, W, flags);      \
    else                                                                                                    \
        launch_coeff_kernel<D, false, N>((unsigned)((pk.m + coeff_threads<false, N>() - 1) /                \
                                                    coeff_threads<false, N>()), st, pk, *p32, W, flags);
    switch (n1) {
    case 4: FGR_COEFF(4); break;
    case 8: FGR_COEFF(8); break;
    case 16: FGR_COEFF(16); break;
    default: set_error("fggc: unsupported neighbour count %d", n1); return FGR_E_INVALID;
    }
#undef FGR_COEFF
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace
}  // namespace fgr
