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

// FP64: per-dimension coefficients through the eigen factors.
template <int N>
__device__ __forceinline__ void coeff_dim64(const Params64 &P, double Q, double Pm, int &a0, int &b0,
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

// FP32: per-dimension coefficients through the Chebyshev surrogate.
template <int N>
__device__ __forceinline__ void coeff_dim32(const Params32 &P, double Q, double Pm, int &a0, int &b0,
                                            float *cr, float *ci) {
    const Common &c = P.c;
    const double r = quotient_for_floor(Q, c.dqv, c.inv_dq), rp = quotient_for_floor(Pm, c.dpv, c.inv_dp);
    const double fa = floor(r), fb = floor(rp);
    a0 = (int)fmin(fmax(fa, -1e9), 1e9);
    b0 = (int)fmin(fmax(fb, -1e9), 1e9);
    const float xs = (float)(2.0 * (r - fa) - 1.0), xt = (float)(2.0 * (rp - fb) - 1.0);
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
                ur = fmaf(Cr[i * kCheb + j], Tt[j], ur);
                ui = fmaf(Ci[i * kCheb + j], Tt[j], ui);
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

template <int D, bool FP64, int N1>
__global__ void __launch_bounds__(128) coeff_scatter_kernel(
    const double *__restrict__ q, const double *__restrict__ p, const double *__restrict__ s,
    const double *__restrict__ a, int64_t m,
    const __grid_constant__ typename std::conditional<FP64, Params64, Params32>::type P,
    void *__restrict__ W_v, uint8_t *__restrict__ row_flag) {
    using Real = typename std::conditional<FP64, double, float>::type;
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
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
    Real cr[D][N1], ci[D][N1];
    int a0[D], b0[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        if constexpr (FP64)
            coeff_dim64<N1>(P, q[l * m + j], p[l * m + j], a0[l], b0[l], cr[l], ci[l]);
        else
            coeff_dim32<N1>(P, q[l * m + j], p[l * m + j], a0[l], b0[l], cr[l], ci[l]);
    }
    C2 *W = reinterpret_cast<C2 *>(W_v);
    // tensor product over dimensions, innermost dimension last; the rows of
    // the first grid pass (the last dimension's [a][b] plane) that receive a
    // contribution are marked once per row, before its contributions
    auto emit = [&](int64_t idx, bool in, Real vr, Real vi) {
        if (in) atomic_add_c(W + idx, vr, vi);
    };
#pragma unroll(N1 <= 8 ? N1 : 1)
    for (int k0 = 0; k0 < N1; ++k0) {
        const int ia0 = a0[0] + c.dq[k0] - c.amin[0], ib0 = b0[0] + c.dp[k0] - c.bmin[0];
        const bool in0 = (unsigned)ia0 < (unsigned)c.A[0] && (unsigned)ib0 < (unsigned)c.B[0];
        const int64_t idx0 = ia0 * c.sa[0] + ib0 * c.sb[0];
        Real p0r, p0i;
        cmul(wr, wi, cr[0][k0], ci[0][k0], p0r, p0i);
        if constexpr (D == 1) {
            emit(idx0, in0, p0r, p0i);  // the single row is marked by the host
        } else {
            const int64_t row0 = ia0 * c.ra[0] + ib0 * c.rb[0];
            if (D == 2 && in0) row_flag[row0] = 1;
#pragma unroll(N1 <= 8 ? N1 : 1)
            for (int k1 = 0; k1 < N1; ++k1) {
                const int ia1 = a0[1] + c.dq[k1] - c.amin[1], ib1 = b0[1] + c.dp[k1] - c.bmin[1];
                const bool in1 = in0 && (unsigned)ia1 < (unsigned)c.A[1] && (unsigned)ib1 < (unsigned)c.B[1];
                const int64_t idx1 = idx0 + ia1 * c.sa[1] + ib1 * c.sb[1];
                Real p1r, p1i;
                cmul(p0r, p0i, cr[1][k1], ci[1][k1], p1r, p1i);
                if constexpr (D == 2) {
                    emit(idx1, in1, p1r, p1i);
                } else {
                    if (in1) row_flag[row0 + ia1 * c.ra[1] + ib1 * c.rb[1]] = 1;
#pragma unroll
                    for (int k2 = 0; k2 < N1; ++k2) {
                        const int ia2 = a0[2] + c.dq[k2] - c.amin[2], ib2 = b0[2] + c.dp[k2] - c.bmin[2];
                        const bool in2 = in1 && (unsigned)ia2 < (unsigned)c.A[2] && (unsigned)ib2 < (unsigned)c.B[2];
                        Real p2r, p2i;
                        cmul(p1r, p1i, cr[2][k2], ci[2][k2], p2r, p2i);
                        emit(idx1 + ia2 * c.sa[2] + ib2 * c.sb[2], in2, p2r, p2i);
                    }
                }
            }
        }
    }
}

template <int D>
fgr_status launch_coeff_d(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64, const Params32 *p32,
                          void *W, uint8_t *flags) {
    const unsigned blocks = (unsigned)((pk.m + 127) / 128);
    if (pk.m == 0) return FGR_OK;
#define FGR_COEFF(N)                                                                                        \
    if (p64)                                                                                                \
        coeff_scatter_kernel<D, true, N><<<blocks, 128, 0, st>>>(pk.q, pk.p, pk.s, pk.a, pk.m, *p64, W, flags); \
    else                                                                                                    \
        coeff_scatter_kernel<D, false, N><<<blocks, 128, 0, st>>>(pk.q, pk.p, pk.s, pk.a, pk.m, *p32, W, flags);
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
