// K3-K5: frozen Gaussian grid-point correction (Algorithm 2, Steps 3-4).
//
// Node array.  W holds the aggregated amplitudes of eq. 2.25 on a dense box of
// phase-space nodes, stored interleaved as [a_0][b_0][a_1][b_1]...[a_{d-1}][b_{d-1}]
// (a: q-node index, b: p-node index).  The a-range is the part of the packets'
// range whose Gaussians reach the grid (other nodes have empty windows); the
// b-range spans the packets with non-zero amplitude (zero amplitudes add zeros).
//
// K3+K4 (one thread per packet).  Per dimension: r = Q/dq, a0 = floor(r),
// s = r - a0 and likewise b0, t for P (eq. 3.6-3.7, FP64).  The true LSA
// coefficients c~_k(s,t) = conj(A~^+ f~(s,t))_k come from
//   FP64: f~ of eq. 3.23 in FP64 and A~^+ applied through its eigen factors;
//   FP32: a Chebyshev surrogate of c~(s,t) built on the host in long double
//         from the same factors (truncation error below 1e-9), evaluated in FP32.
// The shift back of eq. 3.13 and the node phase of the on-grid packet are
// folded into one phase per coefficient: G(x; a dq, b dp) =
// g(x - a dq) e^{i b dp x/eps} e^{-i cq cp a b}, and with r = a0 + s,
//   -cq cp [(s - dq_k) b0 + (a0 + dq_k)(b0 + dp_k)] = -cq cp [r b0 + (a0 + dq_k) dp_k].
// The weight A e^{iS/eps} pref times the product of the d per-dimension
// coefficients is added to W with atomics.
//
// K5 (separable grid stage).  u(x_m) = sum_{a,b} W'[a,b] prod_l g(x_{m_l} - a_l dq)
// e^{i b_l dp x_{m_l}/eps} is contracted one dimension at a time: a pass maps
// rows [a_l][b_l] to [m_l]; a transpose brings the next dimension innermost.
// Each CTA owns 32 or 128 grid points of one row (one per thread): the band of
// nodes a whose window covers them, g in registers, W staged through shared
// memory in chunks of b, and e^{i b dp x/eps} generated per (m, b) from a
// phase reduced in FP64.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <climits>
#include <memory>
#include <vector>
#include <cmath>

#include "device_util.cuh"
#include "fggc_params.h"
#include "internal.h"

namespace fgr {
namespace {

// ---------------------------------------------------------------------------
// node box
// ---------------------------------------------------------------------------
// Body of the bounds reduction for CTA bid of nblk (a batched launch runs it
// for the CTAs of each request).
// Exponent bits all set: infinity or NaN (an integer test).
__device__ __forceinline__ bool not_finite_d(double x) {
    return ((unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7ff00000u) == 0x7ff00000u;
}

// s: when non-null, every packet's Q, P, S and A are also tested for
// finiteness and out[12] is set to 1 if one is not (out[12] starts at 0).
template <int D>
__device__ __forceinline__ void bounds_body(const double *__restrict__ q, const double *__restrict__ p,
                                            const double *__restrict__ a, int64_t m, const Common &c,
                                            const int *aglo, const int *aghi, int *__restrict__ out, int64_t bid,
                                            int64_t nblk, const double *__restrict__ s = nullptr) {
    bool bad = false;
    int dqmin = INT_MAX, dqmax = INT_MIN, dpmin = INT_MAX, dpmax = INT_MIN;
    for (int k = 0; k < c.n1; ++k) {
        dqmin = min(dqmin, c.dq[k]);
        dqmax = max(dqmax, c.dq[k]);
        dpmin = min(dpmin, c.dp[k]);
        dpmax = max(dpmax, c.dp[k]);
    }
    // grid-stride: each thread folds its packets into running bounds, so the
    // atomics below are one set per CTA (a few thousand in all)
    int lo_a[D], hi_a[D], lo_b[D], hi_b[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        lo_a[l] = INT_MAX;
        hi_a[l] = INT_MIN;
        lo_b[l] = INT_MAX;
        hi_b[l] = INT_MIN;
    }
    for (int64_t j = bid * (int64_t)blockDim.x + threadIdx.x; j < m; j += nblk * blockDim.x) {
        // every load of the packet first (no load waits on the amplitude test)
        double qv[D], pv[D];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            qv[l] = q[l * m + j];
            pv[l] = p[l * m + j];
        }
        if (s) {
            bool nf = not_finite_d(s[j]) || not_finite_d(a[j]) || not_finite_d(a[m + j]);
#pragma unroll
            for (int l = 0; l < D; ++l) nf = nf || not_finite_d(qv[l]) || not_finite_d(pv[l]);
            bad = bad || nf;
            if (nf) continue;
        }
        if (a[j] == 0.0 && a[m + j] == 0.0) continue;
        int pa_lo[D], pa_hi[D], pb_lo[D], pb_hi[D];
        bool use = true;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const int a0 = floor_div_int(qv[l], c.dqv, c.inv_dq);
            const int b0 = floor_div_int(pv[l], c.dpv, c.inv_dp);
            pa_lo[l] = max(a0 + dqmin, aglo[l]);
            pa_hi[l] = min(a0 + dqmax, aghi[l]);
            if (pa_lo[l] > pa_hi[l]) use = false;  // no node of this packet reaches the grid
            pb_lo[l] = b0 + dpmin;
            pb_hi[l] = b0 + dpmax;
        }
        if (!use) continue;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            lo_a[l] = min(lo_a[l], pa_lo[l]);
            hi_a[l] = max(hi_a[l], pa_hi[l]);
            lo_b[l] = min(lo_b[l], pb_lo[l]);
            hi_b[l] = max(hi_b[l], pb_hi[l]);
        }
    }
    if (s && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&out[12], 1);
    // warp, then block reduction; one atomic per block and value
    __shared__ int red[8][kMaxDim * 4];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const int v0 = __reduce_min_sync(0xffffffffu, lo_a[l]);
        const int v1 = __reduce_max_sync(0xffffffffu, hi_a[l]);
        const int v2 = __reduce_min_sync(0xffffffffu, lo_b[l]);
        const int v3 = __reduce_max_sync(0xffffffffu, hi_b[l]);
        if ((threadIdx.x & 31) == 0) {
            red[warp][l * 4 + 0] = v0;
            red[warp][l * 4 + 1] = v1;
            red[warp][l * 4 + 2] = v2;
            red[warp][l * 4 + 3] = v3;
        }
    }
    __syncthreads();
    if (threadIdx.x < D * 4) {
        const int k = threadIdx.x;
        const bool is_min = (k & 1) == 0;
        int v = red[0][k];
        for (int w = 1; w < nwarps; ++w) v = is_min ? min(v, red[w][k]) : max(v, red[w][k]);
        if (is_min ? v != INT_MAX : v != INT_MIN) {
            if (is_min) atomicMin(&out[k], v);
            else atomicMax(&out[k], v);
        }
    }
}

template <int D>
__global__ void bounds_kernel(const double *__restrict__ q, const double *__restrict__ p,
                              const double *__restrict__ a, int64_t m, Common c, int aglo0, int aghi0,
                              int aglo1, int aghi1, int aglo2, int aghi2, int *__restrict__ out,
                              const double *__restrict__ s) {
    const int aglo[3] = {aglo0, aglo1, aglo2}, aghi[3] = {aghi0, aghi1, aghi2};
    bounds_body<D>(q, p, a, m, c, aglo, aghi, out, blockIdx.x, gridDim.x, s);
}

// CTAs of the bounds kernel: enough to fill the GPU, few enough that the
// per-CTA atomics stay negligible
inline unsigned bounds_blocks(const fgr_ctx *ctx, int64_t m) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)ctx->num_sms * 8));
}

// ---------------------------------------------------------------------------
// grid passes
// ---------------------------------------------------------------------------
struct PassParams {
    int64_t rows;
    int A, B, amin, bmin;
    int64_t N;
    double lo, h, dq, rs, neg_half_inv_eps;
    double phi_scale;  // dp / (2 pi eps): phase of e^{i b dp x/eps} in turns per unit b
    double two_pow_b;  // split of the turn increment (FP32 path)
    double inv_two_pow_b;
    double dp_over_eps;
};

constexpr int kCB = 32;

// One grid point per thread keeps the Gaussian factors of the band (MAXBAND
// registers) small enough for several CTAs per SM.  A CTA covers TP = 128 or
// 32 consecutive points (TP threads): the node band of a tile spans its width
// plus one window, so on coarse grids (tile width comparable to the window)
// the narrow tile wastes fewer zero Gaussian factors.
constexpr int kPassPts = 1;  // grid points per thread

// node band of a tile of tp points (nodes whose window can reach it, + margin)
inline int pass_band(int tp, double h, double rs, double dq) {
    return (int)std::ceil(((tp - 1) * h + 2 * rs) / dq) + 3;
}

// Per-pass tables shared by all rows: the grid window of every node a (FP64
// rule of include/fgr.h), the FP64-reduced phase increment of every grid point
// m split into an exact FP32 pair, and the node band of every tile of TP
// points.  They replace per-CTA FP64 divisions and reductions.
struct PassTables {
    int2 *win;     // [A]: (first, last) grid point of node amin + i
    float2 *ph;    // [N]: (hi, lo) turns of e^{i dp x_m / eps} per unit b
    int2 *band;    // [tiles]: (a_lo, a_hi) of tile t (a_lo > a_hi: empty)
};

__device__ __forceinline__ void pass_tables_body(const PassParams &pp, int tp, int64_t tiles, const PassTables &t,
                                                 int64_t i) {
    if (i < pp.A) {
        int64_t wlo, whi;
        window_bounds((double)(pp.amin + i) * pp.dq, pp.rs, pp.lo, pp.h, pp.N, &wlo, &whi);
        t.win[i] = make_int2((int)wlo, (int)whi);
    }
    if (i < pp.N) {
        const double xm = grid_x(pp.lo, pp.h, i);
        double phi = pp.phi_scale * xm;
        phi -= rint(phi);
        const double phi_hi = rint(phi * pp.two_pow_b) * pp.inv_two_pow_b;
        t.ph[i] = make_float2((float)phi_hi, (float)(phi - phi_hi));
    }
    if (i < tiles) {
        const int64_t m0 = i * tp, m1 = min(m0 + tp - 1, pp.N - 1);
        const double x0 = grid_x(pp.lo, pp.h, m0), x1 = grid_x(pp.lo, pp.h, m1);
        const int a_lo = max(pp.amin, (int)ceil((x0 - pp.rs) / pp.dq) - 1);
        const int a_hi = min(pp.amin + pp.A - 1, (int)floor((x1 + pp.rs) / pp.dq) + 1);
        t.band[i] = make_int2(a_lo, a_hi);
    }
}

__global__ void pass_tables_kernel(PassParams pp, int tp, int64_t tiles, PassTables t) {
    pass_tables_body(pp, tp, tiles, t, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

#include "fggc_fft.cuh"

// Body of a grid pass for the CTA (row, tile, b-slice zs of nz); a batched
// launch runs it for the CTAs of each request.
template <bool FP64, int MAXBAND, int TP>
__device__ __forceinline__ void grid_pass_body(const void *__restrict__ in_v, void *__restrict__ out_v,
                                               const PassParams &pp, const uint8_t *__restrict__ flags,
                                               const int2 *__restrict__ brange, const PassTables &tab,
                                               int64_t row, int tile, int zs, int nz) {
    using Real = typename std::conditional<FP64, double, float>::type;
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    __shared__ __align__(16) C2 sw[MAXBAND][kCB];
    __shared__ int swlo[MAXBAND], swhi[MAXBAND];
    __shared__ int s_blo, s_bhi;
    const int64_t m0 = (int64_t)tile * TP;
    int64_t mm[kPassPts];
    bool valid[kPassPts];
#pragma unroll
    for (int r = 0; r < kPassPts; ++r) {
        mm[r] = m0 + threadIdx.x + r * TP;
        valid[r] = mm[r] < pp.N;
    }
    C2 *out = reinterpret_cast<C2 *>(out_v) + row * pp.N;
    const C2 *in = reinterpret_cast<const C2 *>(in_v) + row * (int64_t)pp.A * pp.B;
    C2 zero;
    zero.x = 0;
    zero.y = 0;
    const bool split = nz > 1;  // slices add into a zeroed output
    const int2 bnd = tab.band[tile];
    const int a_lo = bnd.x, a_hi = bnd.y;
    const int nb_total = a_hi - a_lo + 1;
    // occupied b-range: the union over the band of the per-node ranges
    int ulo = 0, uhi = pp.B - 1;
    if (brange && nb_total > 0) {
        if (threadIdx.x == 0) {
            s_blo = INT_MAX;
            s_bhi = INT_MIN;
        }
        __syncthreads();
        int lo = INT_MAX, hi = INT_MIN;
        for (int i = threadIdx.x; i < nb_total; i += TP) {
            const int2 r = brange[row * (int64_t)pp.A + (a_lo - pp.amin) + i];
            lo = min(lo, r.x);
            hi = max(hi, r.y);
        }
        atomicMin(&s_blo, lo);
        atomicMax(&s_bhi, hi);
        __syncthreads();
        ulo = s_blo;
        uhi = s_bhi;
    }
    // b-slice of this CTA: part zs of nz of [ulo, uhi], whole chunks
    const int nchunk = uhi >= ulo ? (uhi - ulo + kCB) / kCB : 0;
    const int per = (nchunk + nz - 1) / nz;
    const int bs = ulo + zs * per * kCB, be = min(uhi + 1, bs + per * kCB);
    if ((flags && !flags[row]) || bs >= be || nb_total <= 0) {
        if (!split) {
#pragma unroll
            for (int r = 0; r < kPassPts; ++r)
                if (valid[r]) out[mm[r]] = zero;
        }
        return;
    }
    double xm[kPassPts], th64[kPassPts];
    float phf[kPassPts], plf[kPassPts];
#pragma unroll
    for (int r = 0; r < kPassPts; ++r) {
        const int64_t mr = valid[r] ? mm[r] : m0;
        xm[r] = grid_x(pp.lo, pp.h, mr);
        // e^{i b dp x_m / eps}: turns per unit b, reduced in FP64 (pass table)
        const float2 ph = tab.ph[mr];
        phf[r] = ph.x;
        plf[r] = ph.y;
        th64[r] = FP64 ? pp.dp_over_eps * xm[r] : 0.0;
    }
    const float cef = (float)(pp.neg_half_inv_eps * 1.4426950408889634);  // log2(e) / (-2 eps)
    const float dqf = (float)pp.dq;

    Real accr[kPassPts], acci[kPassPts];
    double totr[kPassPts], toti[kPassPts];  // chunk partials are folded in here
#pragma unroll
    for (int r = 0; r < kPassPts; ++r) {
        accr[r] = acci[r] = 0;
        totr[r] = toti[r] = 0;
    }
    // the band of nodes is processed MAXBAND at a time (coarse grids need more)
    for (int c0 = 0; c0 < nb_total; c0 += MAXBAND) {
        const int nb = min(MAXBAND, nb_total - c0);
        const int a_first = a_lo + c0;
        // each node's window once per CTA (FP64, the rule of include/fgr.h)
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += TP) {
            const int2 w = tab.win[a_first - pp.amin + i];
            swlo[i] = w.x;
            swhi[i] = w.y;
        }
        __syncthreads();
        Real g[kPassPts][MAXBAND];
#pragma unroll
        for (int r = 0; r < kPassPts; ++r) {
            const double dx0 = xm[r] - (double)a_first * pp.dq;
#pragma unroll
            for (int i = 0; i < MAXBAND; ++i) {
                g[r][i] = 0;
                if (i < nb && valid[r] && mm[r] >= swlo[i] && mm[r] <= swhi[i]) {
                    if constexpr (FP64) {
                        const double dx = xm[r] - (double)(a_first + i) * pp.dq;
                        g[r][i] = exp(dx * dx * pp.neg_half_inv_eps);
                    } else {
                        const float dxf = (float)dx0 - (float)i * dqf;
                        g[r][i] = ex2_approx(dxf * dxf * cef);
                    }
                }
            }
        }
        const int ia0 = a_first - pp.amin;
        for (int b0 = bs; b0 < be; b0 += kCB) {
            const int nbb = min(kCB, be - b0);
            for (int e = threadIdx.x; e < nb * kCB; e += TP) {
                const int i = e / kCB, bb = e % kCB;
                sw[i][bb] = bb < nbb ? in[(int64_t)(ia0 + i) * pp.B + b0 + bb] : zero;
            }
            __syncthreads();
            for (int bb = 0; bb < nbb; bb += 2) {  // b pairs; the padding column is zero
                Real vr[kPassPts][2], vi[kPassPts][2];
#pragma unroll
                for (int r = 0; r < kPassPts; ++r) vr[r][0] = vr[r][1] = vi[r][0] = vi[r][1] = 0;
#pragma unroll
                for (int i = 0; i < MAXBAND; ++i) {
                    if (i < nb) {
                        C2 w0, w1;
                        if constexpr (FP64) {
                            w0 = sw[i][bb];
                            w1 = sw[i][bb + 1];
                        } else {  // one 16-byte shared load for the pair
                            const float4 w = *reinterpret_cast<const float4 *>(&sw[i][bb]);
                            w0.x = w.x;
                            w0.y = w.y;
                            w1.x = w.z;
                            w1.y = w.w;
                        }
#pragma unroll
                        for (int r = 0; r < kPassPts; ++r) {
                            vr[r][0] += g[r][i] * w0.x;
                            vi[r][0] += g[r][i] * w0.y;
                            vr[r][1] += g[r][i] * w1.x;
                            vi[r][1] += g[r][i] * w1.y;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int b = pp.bmin + b0 + bb + u;
#pragma unroll
                    for (int r = 0; r < kPassPts; ++r) {
                        Real er, ei;
                        if constexpr (FP64) {
                            double sn, cs;
                            sincos((double)b * th64[r], &sn, &cs);
                            er = cs;
                            ei = sn;
                        } else {
                            const float bf = (float)b;
                            float f = bf * phf[r];
                            f -= rint_fast(f);
                            float tau = fmaf(bf, plf[r], f);
                            tau -= rint_fast(tau);
                            float sn, cs;
                            __sincosf(6.283185307179586f * tau, &sn, &cs);
                            er = cs;
                            ei = sn;
                        }
                        accr[r] += er * vr[r][u] - ei * vi[r][u];
                        acci[r] += er * vi[r][u] + ei * vr[r][u];
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kPassPts; ++r) {
                totr[r] += (double)accr[r];
                toti[r] += (double)acci[r];
                accr[r] = acci[r] = 0;
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < kPassPts; ++r) {
        if (!valid[r]) continue;
        if (split) {
            atomic_add_c(out + mm[r], (Real)totr[r], (Real)toti[r]);
        } else {
            C2 o;
            o.x = (Real)totr[r];
            o.y = (Real)toti[r];
            out[mm[r]] = o;
        }
    }
}

#include "fggc_tma.cuh"

template <bool FP64, int MAXBAND, int TP>
__global__ void __launch_bounds__(TP) grid_pass_kernel(const void *__restrict__ in_v, void *__restrict__ out_v,
                                                       PassParams pp, const uint8_t *__restrict__ flags,
                                                       const int2 *__restrict__ brange, const PassTables tab) {
    grid_pass_body<FP64, MAXBAND, TP>(in_v, out_v, pp, flags, brange, tab, blockIdx.x, blockIdx.y, blockIdx.z,
                                      gridDim.z);
}

template <class C2>
__device__ __forceinline__ void transpose_body(const C2 *__restrict__ in, C2 *__restrict__ out, int64_t R,
                                               int64_t Cc, int64_t bx, int64_t by) {
    __shared__ C2 tile[32][33];
    const int64_t r0 = bx * 32, c0 = by * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < Cc) tile[i][threadIdx.x] = in[r * Cc + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < Cc) out[c * R + r] = tile[threadIdx.x][i];
    }
}

template <class C2>
__global__ void transpose_kernel(const C2 *__restrict__ in, C2 *__restrict__ out, int64_t R, int64_t Cc) {
    transpose_body<C2>(in, out, R, Cc, blockIdx.x, blockIdx.y);
}

// Occupied b-range of every line [row][a][0..B): first and last b with a
// non-zero value ((B, -1) for an empty line, and without reading it for a line
// of a row the scatter did not mark, when row flags are given).  One warp per
// line.
template <class C2>
__device__ __forceinline__ void brange_body(const C2 *__restrict__ in, int64_t lines, int B,
                                            int2 *__restrict__ out, int64_t bid, const uint8_t *flags = nullptr,
                                            int A = 1) {
    const int64_t line = bid * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= lines) return;
    const int lane = threadIdx.x & 31;
    if (flags && !flags[line / A]) {
        if (lane == 0) out[line] = make_int2(B, -1);
        return;
    }
    const C2 *p = in + line * (int64_t)B;
    int lo = INT_MAX, hi = INT_MIN;
    for (int b = lane; b < B; b += 32) {
        const C2 v = p[b];
        if (v.x != 0 || v.y != 0) {
            lo = min(lo, b);
            hi = max(hi, b);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) out[line] = make_int2(lo == INT_MAX ? B : lo, hi);
}

template <class C2>
__global__ void brange_kernel(const C2 *__restrict__ in, int64_t lines, int B, const uint8_t *__restrict__ flags,
                              int A, int2 *__restrict__ out) {
    brange_body<C2>(in, lines, B, out, blockIdx.x, flags, A);
}

// The same for short lines (B <= 64): one thread per line, so a warp streams
// 32 consecutive lines instead of leaving most of its lanes idle.
template <class C2>
__global__ void brange_short_kernel(const C2 *__restrict__ in, int64_t lines, int B,
                                    const uint8_t *__restrict__ flags, int A, int2 *__restrict__ out) {
    const int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (line >= lines) return;
    const C2 *p = in + line * (int64_t)B;
    int lo = B, hi = -1;
    const int nb = (flags && !flags[line / A]) ? 0 : B;
    for (int b = 0; b < nb; ++b) {
        const C2 v = p[b];
        if (v.x != 0 || v.y != 0) {
            lo = min(lo, b);
            hi = b;
        }
    }
    out[line] = make_int2(lo, hi);
}

// Node-point terms of one pass (timing only): over the (row, a) lines, the
// occupied b-range times the grid points in node a's window, summed into *out.
__global__ void pass_terms_kernel(const int2 *__restrict__ brange, int64_t lines, int A,
                                  const int2 *__restrict__ win, unsigned long long *__restrict__ out) {
    unsigned long long t = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lines;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 r = brange[i], w = win[i % A];
        if (r.y >= r.x && w.y >= w.x) t += (unsigned long long)(r.y - r.x + 1) * (unsigned long long)(w.y - w.x + 1);
    }
    t = __reduce_add_sync(0xffffffffu, (unsigned)(t & 0xffffffffu)) +
        ((unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)(t >> 32)) << 32);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(out, t);
}

// flags: row flags of the first pass (lines of unmarked rows are empty), or null.
template <bool FP64>
fgr_status launch_brange(const void *in, int64_t rows, int A, int B, const uint8_t *flags, int2 *out,
                         cudaStream_t st) {
    const int64_t lines = rows * (int64_t)A;
    if (lines == 0) return FGR_OK;
    if (B <= 64) {
        const unsigned blocks = (unsigned)((lines + 255) / 256);
        if (FP64)
            brange_short_kernel<double2><<<blocks, 256, 0, st>>>((const double2 *)in, lines, B, flags, A, out);
        else
            brange_short_kernel<float2><<<blocks, 256, 0, st>>>((const float2 *)in, lines, B, flags, A, out);
    } else {
        const unsigned blocks = (unsigned)((lines + 7) / 8);
        if (FP64)
            brange_kernel<double2><<<blocks, 256, 0, st>>>((const double2 *)in, lines, B, flags, A, out);
        else
            brange_kernel<float2><<<blocks, 256, 0, st>>>((const float2 *)in, lines, B, flags, A, out);
    }
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

// Entries of the pass tables for a pass over N points and A nodes (int2 /
// float2 units): node windows, point phases and tile bands (at most N / 32 + 1).
inline int64_t pass_table_entries(int64_t A, int64_t N) { return A + N + N / 32 + 1; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor map of a pass input (complex64) as lines x B cells, box kTB cells x
// band lines.  False when the input does not meet the copy engine's rules
// (16-byte aligned base, 16-byte multiple line stride) or encoding fails.
bool pass_tensor_map(const void *in, const PassParams &pp, int band_lines, CUtensorMap *map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const int64_t lines = pp.rows * (int64_t)pp.A;
    if (!enc || ((uintptr_t)in & 15) || (pp.B & 1) || lines >= INT_MAX - 64 || pp.B < 2) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)pp.B, (cuuint64_t)lines};
    const cuuint64_t strides[1] = {(cuuint64_t)pp.B * 8};
    const cuuint32_t box[2] = {(cuuint32_t)kTB, (cuuint32_t)band_lines};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(in), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool FP64>
fgr_status launch_pass(const void *in, void *out, const PassParams &pp, const uint8_t *flags,
                       const int2 *brange, int64_t target_ctas, int tile_pref, void *tables,
                       cudaStream_t st, StageMarks *before_pass = nullptr, int *err = nullptr) {
    if (pp.rows == 0 || pp.N == 0) return FGR_OK;
    if (pp.rows > INT_MAX) {
        set_error("fggc: too many rows in a grid pass");
        return FGR_E_CAPACITY;
    }
    // narrow tiles where they cut the band (the work per grid point) by more
    // than a quarter, unless the autotuner or the caller fixed the tile
    const int band128 = pass_band(128, pp.h, pp.rs, pp.dq), band32 = pass_band(32, pp.h, pp.rs, pp.dq);
    const int tp = tile_pref == 32 || tile_pref == 128 ? tile_pref : (4 * band32 < 3 * band128 ? 32 : 128);
    const int band = tp == 32 ? band32 : band128;
    const int64_t mtiles = (pp.N + tp - 1) / tp;
    if (mtiles > 65535) {
        set_error("fggc: %lld points per grid dimension; at most %d supported", (long long)pp.N, 65535 * tp);
        return FGR_E_INVALID;
    }
    // split the b-range when rows x tiles alone cannot fill the device
    const int64_t target = target_ctas;
    const int nchunk = (pp.B + kCB - 1) / kCB;
    int splits = (int)std::min<int64_t>(std::max<int64_t>(1, (target + pp.rows * mtiles - 1) / (pp.rows * mtiles)),
                                        std::max(1, std::min(nchunk, 64)));
    if (splits > 1) {
        FGR_CUDA_TRY(cudaMemsetAsync(out, 0, (FP64 ? 16 : 8) * (size_t)pp.rows * (size_t)pp.N, st));
    }
    PassTables tab;
    tab.win = reinterpret_cast<int2 *>(tables);
    tab.ph = reinterpret_cast<float2 *>(tab.win + pp.A);
    tab.band = reinterpret_cast<int2 *>(tab.ph + pp.N);
    {
        const int64_t n = std::max<int64_t>(std::max<int64_t>(pp.A, pp.N), mtiles);
        pass_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pp, tp, mtiles, tab);
    }
    if (before_pass) before_pass->binned();
    dim3 grid((unsigned)pp.rows, (unsigned)mtiles, (unsigned)splits);
#define FGR_PASS(MB, TPV) grid_pass_kernel<FP64, MB, TPV><<<grid, TPV, 0, st>>>(in, out, pp, flags, brange, tab)
#define FGR_PASS_TP(TPV)                                                                                    \
    if (band <= 16) FGR_PASS(16, TPV);                                                                      \
    else if (band <= 32) FGR_PASS(32, TPV);                                                                 \
    else if (band <= 48) FGR_PASS(48, TPV);                                                                 \
    else FGR_PASS(64, TPV);  // wider bands are processed in chunks of 64
    CUtensorMap map, map_half;
    const int box_lines = band <= 16 ? 16 : 32;
    if (!FP64 && tp == 32 && splits == 1 && err && pass_tensor_map(in, pp, box_lines, &map) &&
        pass_tensor_map(in, pp, box_lines / 2, &map_half)) {
        // 32-point tiles with the node tiles staged by the copy engine; on
        // short rows (at most 256 points: little work per row and tile) four
        // rows per CTA share one sequence of copies
        const int rows_per_cta = pp.N <= 256 ? 4 : 1;
        const dim3 tgrid((unsigned)((pp.rows + rows_per_cta - 1) / rows_per_cta), (unsigned)mtiles);
#define FGR_TMA(MB, R) \
    grid_pass_tma_kernel<MB, R><<<tgrid, 32, 0, st>>>(map, map_half, out, pp, flags, brange, tab, err)
        if (rows_per_cta == 4) {
            if (band <= 16) FGR_TMA(16, 4);
            else FGR_TMA(32, 4);
        } else {
            if (band <= 16) FGR_TMA(16, 1);
            else FGR_TMA(32, 1);
        }
#undef FGR_TMA
    } else if (tp == 32) {
        // narrow tiles: at most 32 band factors in registers (wider bands in
        // chunks of 32), so that more warps fit an SM
        if (band <= 16) FGR_PASS(16, 32);
        else FGR_PASS(32, 32);
    } else {
        FGR_PASS_TP(128)
    }
#undef FGR_PASS_TP
#undef FGR_PASS
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

// The grid pass of a commensurate dimension (N = 2^logn): pass tables, DFT
// twiddles, one inverse DFT per (row, a) line into F, the banded contraction.
template <bool FP64>
fgr_status launch_fft_pass(const void *in, void *out, const PassParams &pp, const uint8_t *flags,
                           const int2 *brange, int logn, void *F, void *twiddle, void *tables, cudaStream_t st,
                           StageMarks *before_pass) {
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    if (pp.rows == 0 || pp.N == 0) return FGR_OK;
    if (pp.rows > INT_MAX || pp.rows * (int64_t)pp.A > INT_MAX) {
        set_error("fggc: too many lines in a DFT grid pass");
        return FGR_E_CAPACITY;
    }
    constexpr int tp = 128;
    const int64_t mtiles = (pp.N + tp - 1) / tp;
    if (mtiles > 65535) {
        set_error("fggc: %lld points per grid dimension; at most %d supported", (long long)pp.N, 65535 * tp);
        return FGR_E_INVALID;
    }
    const int N = 1 << logn;
    PassTables tab;
    tab.win = reinterpret_cast<int2 *>(tables);
    tab.ph = reinterpret_cast<float2 *>(tab.win + pp.A);
    tab.band = reinterpret_cast<int2 *>(tab.ph + pp.N);
    {
        const int64_t n = std::max<int64_t>(std::max<int64_t>(pp.A, pp.N), mtiles);
        pass_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pp, tp, mtiles, tab);
    }
    fft_twiddle_kernel<C2><<<(unsigned)((N / 2 + 255) / 256), 256, 0, st>>>(N, (C2 *)twiddle);
    if (before_pass) before_pass->binned();
    const int lpc = dft_lines_per_cta(logn);
    const size_t smem = sizeof(C2) * (size_t)N * lpc;
    if (smem > 48 * 1024)
        FGR_CUDA_TRY(cudaFuncSetAttribute(dft_lines_kernel<FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    const double th = pp.phi_scale * pp.lo;  // dp lo / (2 pi eps), turns per unit b
    const int64_t lines = pp.rows * (int64_t)pp.A;
    dft_lines_kernel<FP64><<<(unsigned)((lines + lpc - 1) / lpc), 256, smem, st>>>(in, F, pp.rows, pp.A, pp.B,
                                                                                   pp.bmin, th, logn, brange, flags,
                                                                                   twiddle);
    band_fft_kernel<FP64><<<dim3((unsigned)pp.rows, (unsigned)mtiles), tp, 0, st>>>(F, out, pp, logn, tab);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

template <class C2>
fgr_status launch_transpose(const void *in, void *out, int64_t R, int64_t Cc, cudaStream_t st) {
    if (R == 0 || Cc == 0) return FGR_OK;
    dim3 grid((unsigned)((R + 31) / 32), (unsigned)((Cc + 31) / 32));
    if (grid.y > 65535u) {
        set_error("fggc: transpose too wide");
        return FGR_E_CAPACITY;
    }
    transpose_kernel<C2><<<grid, dim3(32, 8), 0, st>>>((const C2 *)in, (C2 *)out, R, Cc);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

// b[0..12) the empty bounds; b[12] (when present) the non-finite flag.
__global__ void bounds_init_kernel(int *__restrict__ b, int n) {
    if (threadIdx.x < 12) b[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
    if (threadIdx.x == 12 && n > 12) b[12] = 0;
}

// Sets *overflow when the packets' node bounds b[] leave the planned box.
__global__ void box_check_kernel(const int *__restrict__ b, int d, Common c, int *__restrict__ overflow) {
    if (threadIdx.x != 0) return;
    bool out = false;
    for (int l = 0; l < d; ++l) {
        if (b[l * 4] == INT_MAX) continue;  // no packet reaches the grid
        out = out || b[l * 4 + 0] < c.amin[l] || b[l * 4 + 1] > c.amin[l] + c.A[l] - 1 ||
              b[l * 4 + 2] < c.bmin[l] || b[l * 4 + 3] > c.bmin[l] + c.B[l] - 1;
    }
    if (out) *overflow = 1;
}

// LSA and mesh constants of a context (the node box is filled in by make_box).
Common base_common(const fgr_ctx *ctx) {
    const Mesh &M = ctx->mesh;
    const Lsa &L = ctx->lsa;
    Common c{};
    c.n1 = L.n1;
    for (int k = 0; k < L.n1; ++k) {
        c.dq[k] = L.dq[k];
        c.dp[k] = L.dp[k];
    }
    c.dqv = M.dq;
    c.dpv = M.dp;
    c.inv_dq = 1.0 / M.dq;
    c.inv_dp = 1.0 / M.dp;
    c.cq2_4 = M.cq * M.cq / 4;
    c.cp2_4 = M.cp * M.cp / 4;
    c.half_cqcp = M.cqcp / 2;
    c.cc = M.cqcp / (2 * M_PI);
    c.inv_2pi_eps = 1.0 / (2 * M_PI * M.eps);
    c.pref = M.pref;
    return c;
}

// Grid-relevant node range per dimension (other nodes have empty windows).
void grid_node_range(const fgr_ctx *ctx, int *aglo, int *aghi) {
    const Grid &G = ctx->grid;
    const Mesh &M = ctx->mesh;
    for (int l = 0; l < 3; ++l) {
        aglo[l] = 0;
        aghi[l] = -1;
    }
    for (int l = 0; l < ctx->d; ++l) {
        const double xlast = G.lo[l] + (double)(G.n[l] - 1) * G.h[l];
        aglo[l] = (int)std::max(-1e9, std::ceil((G.lo[l] - M.rs) / M.dq) - 1);
        aghi[l] = (int)std::min(1e9, std::floor((xlast + M.rs) / M.dq) + 1);
    }
}

// Launches the node-bounds reduction of the packets into b[12] (device).
// check_finite: also test every packet value (b holds 13 ints, b[12] the flag).
fgr_status launch_bounds_reduction(const fgr_ctx *ctx, const PacketsDev &pk, const Common &c, const int *aglo,
                                   const int *aghi, int *b, cudaStream_t st, bool check_finite = false) {
    bounds_init_kernel<<<1, 32, 0, st>>>(b, check_finite ? 13 : 12);
    const double *sv = check_finite ? pk.s : nullptr;
    if (pk.m > 0) {
        const unsigned blocks = bounds_blocks(ctx, pk.m);
        switch (ctx->d) {
        case 1:
            bounds_kernel<1><<<blocks, 256, 0, st>>>(pk.q, pk.p, pk.a, pk.m, c, aglo[0], aghi[0], aglo[1], aghi[1],
                                                     aglo[2], aghi[2], b, sv);
            break;
        case 2:
            bounds_kernel<2><<<blocks, 256, 0, st>>>(pk.q, pk.p, pk.a, pk.m, c, aglo[0], aghi[0], aglo[1], aghi[1],
                                                     aglo[2], aghi[2], b, sv);
            break;
        default:
            bounds_kernel<3><<<blocks, 256, 0, st>>>(pk.q, pk.p, pk.a, pk.m, c, aglo[0], aghi[0], aglo[1], aghi[1],
                                                     aglo[2], aghi[2], b, sv);
        }
    }
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace

// Node box from the packets' bounds hb[12], widened by margin nodes on every
// side (a-ranges clipped to the grid-relevant range), and the sizes of the
// buffers of one reconstruction.
fgr_status make_box(const fgr_ctx *ctx, const int *hb, int margin, FggcBox *box) {
    const int D = ctx->d;
    const Grid &G = ctx->grid;
    int aglo[3], aghi[3];
    grid_node_range(ctx, aglo, aghi);
    FggcBox &x = *box;
    x = FggcBox{};
    x.c = base_common(ctx);
    Common &c = x.c;
    x.empty = hb[0] == INT_MAX;
    if (x.empty) return FGR_OK;
    int64_t cells = 1;
    for (int l = 0; l < D; ++l) {
        const int alo = std::max(aglo[l], hb[l * 4 + 0] - margin), ahi = std::min(aghi[l], hb[l * 4 + 1] + margin);
        c.amin[l] = alo;
        c.A[l] = ahi - alo + 1;
        c.bmin[l] = hb[l * 4 + 2] - margin;
        // an even b extent keeps every line 16-byte aligned (tile copies)
        c.B[l] = (hb[l * 4 + 3] - hb[l * 4 + 2] + 1 + 2 * margin + 1) & ~1;
        cells *= (int64_t)c.A[l] * c.B[l];
        if (cells > (int64_t(1) << 36)) {
            set_error("fggc: node array of more than 2^36 cells");
            return FGR_E_CAPACITY;
        }
    }
    {
        int64_t stride = 1;
        for (int l = D - 1; l >= 0; --l) {
            c.sb[l] = stride;
            stride *= c.B[l];
            c.sa[l] = stride;
            stride *= c.A[l];
        }
    }
    c.row_len = (int64_t)c.A[D - 1] * c.B[D - 1];
    for (int l = 0; l < D - 1; ++l) {
        c.ra[l] = c.sa[l] / c.row_len;
        c.rb[l] = c.sb[l] / c.row_len;
    }
    x.cells = cells;
    x.rows0 = cells / c.row_len;
    // intermediate sizes of the passes (the node box itself is only read)
    int64_t prodN = 1;
    for (int l = D - 1; l >= 0; --l) {
        int64_t pre = 1;
        for (int j = 0; j < l; ++j) pre *= (int64_t)c.A[j] * c.B[j];
        x.max_lines = std::max(x.max_lines, pre * prodN * c.A[l]);
        prodN *= G.n[l];
        x.maxbuf = std::max(x.maxbuf, prodN * pre);
    }
    if (D == 1) x.maxbuf = 0;
    for (int l = 0; l < D; ++l) x.table_entries = std::max(x.table_entries, pass_table_entries(c.A[l], G.n[l]));
    // DFT grid stage: one N-point line per (row, a) of each pass
    prodN = 1;
    for (int l = D - 1; l >= 0; --l) {
        int64_t pre = 1;
        for (int j = 0; j < l; ++j) pre *= (int64_t)c.A[j] * c.B[j];
        if (ctx->fft_logn[l] > 0) x.fft_elems = std::max(x.fft_elems, pre * prodN * c.A[l] << ctx->fft_logn[l]);
        prodN *= G.n[l];
    }
    return FGR_OK;
}

bool make_bin_box(const FggcBox &box, int d, BinBox *bb) {
    if (d != 3 || box.empty) return false;
    const Common &c = box.c;
    BinBox x;
    x.dqmin = x.dpmin = INT_MAX;
    x.dqmax = x.dpmax = INT_MIN;
    for (int k = 0; k < c.n1; ++k) {
        x.dqmin = std::min(x.dqmin, c.dq[k]);
        x.dqmax = std::max(x.dqmax, c.dq[k]);
        x.dpmin = std::min(x.dpmin, c.dp[k]);
        x.dpmax = std::max(x.dpmax, c.dp[k]);
    }
    // an outer anchor a0 has a node inside [amin, amin + A) for a0 in
    // [amin - dqmax, amin + A - 1 - dqmin] (likewise b0)
    int64_t K = 1;
    for (int l = 0; l < d - 1; ++l) {
        x.ka_lo[l] = c.amin[l] - x.dqmax;
        x.KA[l] = c.A[l] + x.dqmax - x.dqmin;
        x.kb_lo[l] = c.bmin[l] - x.dpmax;
        x.KB[l] = c.B[l] + x.dpmax - x.dpmin;
        K *= (int64_t)x.KA[l] * x.KB[l];
        if (K > kMaxBinKeys) return false;
    }
    x.K = K;
    *bb = x;
    return true;
}

namespace {
inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }
inline int64_t bin_max_items(int64_t m) { return m / 16 + m / 256 + 1; }
}  // namespace

size_t bin_buffer_bytes(int64_t m, const BinBox &bb) {
    const int64_t K = bb.K;
    return 3 * align256(sizeof(int) * (size_t)m) + align256(sizeof(int) * (size_t)K) +
           align256(sizeof(int2) * (size_t)(K + 1)) + align256(sizeof(int2) * (size_t)((K + 1023) / 1024)) +
           align256(sizeof(int4) * (size_t)bin_max_items(m)) + align256(sizeof(int) * 4);
}

void bin_buffers_at(void *block, int64_t m, const BinBox &bb, BinBuffers *out) {
    char *p = (char *)block;
    const int64_t K = bb.K;
    auto take = [&](size_t n) {
        char *r = p;
        p += align256(n);
        return r;
    };
    out->key = (int *)take(sizeof(int) * (size_t)m);
    out->sorted = (int *)take(sizeof(int) * (size_t)m);
    out->loose = (int *)take(sizeof(int) * (size_t)m);
    out->count = (int *)take(sizeof(int) * (size_t)K);
    out->off = (int2 *)take(sizeof(int2) * (size_t)(K + 1));
    out->bsum = (int2 *)take(sizeof(int2) * (size_t)((K + 1023) / 1024));
    out->items = (int4 *)take(sizeof(int4) * (size_t)bin_max_items(m));
    out->ctr = (int *)take(sizeof(int) * 4);
}

fgr_status launch_binned_scatter(int d, int n1, const BinLaunch &L, cudaStream_t st, const PacketsDev &pk,
                                 const Params32 &P, void *W, uint8_t *flags, StageMarks *marks) {
    if (pk.m == 0) return FGR_OK;
    if (d != 3) {
        set_error("fggc: the binned scatter serves d = 3");
        return FGR_E_INTERNAL;
    }
    return launch_binned_d3(n1, L, st, pk, P, W, flags, marks);
}

namespace {

// ---------------------------------------------------------------------------
// batched FGGC: one launch per stage over the planned requests of one
// dimension (fgr_reconstruct_fggc_batch)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_request(const int *block0, int n) {
    int r = 0;
    while (r + 1 < n && (int)blockIdx.x >= block0[r + 1]) ++r;
    return r;
}

// Byte fills of up to 3 segments per request (node array, row flags, output).
struct FillBatch {
    int n;  // segments
    int block0[3 * kBatchMax + 1];
    unsigned char *ptr[3 * kBatchMax];
    int64_t bytes[3 * kBatchMax];
    int value[3 * kBatchMax];
};

__global__ void __launch_bounds__(256) fill_batch_kernel(const __grid_constant__ FillBatch B) {
    const int r = batch_request(B.block0, B.n);
    const int64_t nblk = B.block0[r + 1] - B.block0[r], bid = blockIdx.x - B.block0[r];
    unsigned char *p = B.ptr[r];
    const int64_t bytes = B.bytes[r];
    const unsigned char v = (unsigned char)B.value[r];
    // 16-byte stores from the first 16-byte boundary, single bytes around them
    const int64_t head = min(bytes, (int64_t)((16 - ((uintptr_t)p & 15)) & 15));
    const int64_t n16 = (bytes - head) / 16;
    const unsigned w = v * 0x01010101u;
    uint4 *p16 = reinterpret_cast<uint4 *>(p + head);
    for (int64_t i = bid * 256 + threadIdx.x; i < n16; i += nblk * 256) p16[i] = make_uint4(w, w, w, w);
    if (bid == 0) {
        for (int64_t i = threadIdx.x; i < head; i += 256) p[i] = v;
        for (int64_t i = head + n16 * 16 + threadIdx.x; i < bytes; i += 256) p[i] = v;
    }
}

struct BoundsBatch {
    int n;
    int block0[kBatchMax + 1];
    Common c[kBatchMax];
    const double *q[kBatchMax], *p[kBatchMax], *a[kBatchMax];
    int64_t m[kBatchMax];
    int aglo[kBatchMax][3], aghi[kBatchMax][3];
    int *out[kBatchMax];     // 12 bounds per request
    int *overflow[kBatchMax];
};

// Initial bounds and cleared overflow flags of every request (one CTA).
__global__ void bounds_init_batch_kernel(const __grid_constant__ BoundsBatch B) {
    for (int i = threadIdx.x; i < B.n * 12; i += blockDim.x) B.out[i / 12][i % 12] = (i & 1) ? INT_MIN : INT_MAX;
    for (int r = threadIdx.x; r < B.n; r += blockDim.x) *B.overflow[r] = 0;
}

template <int D>
__global__ void __launch_bounds__(256) bounds_batch_kernel(const __grid_constant__ BoundsBatch B) {
    const int r = batch_request(B.block0, B.n);
    bounds_body<D>(B.q[r], B.p[r], B.a[r], B.m[r], B.c[r], B.aglo[r], B.aghi[r], B.out[r], blockIdx.x - B.block0[r],
                   B.block0[r + 1] - B.block0[r]);
}

// Overflow flag of every request whose packets left its planned box (one CTA).
__global__ void box_check_batch_kernel(const __grid_constant__ BoundsBatch B, int d) {
    for (int r = threadIdx.x; r < B.n; r += blockDim.x) {
        const int *b = B.out[r];
        const Common &c = B.c[r];
        bool out = false;
        for (int l = 0; l < d; ++l) {
            if (b[l * 4] == INT_MAX) continue;
            out = out || b[l * 4 + 0] < c.amin[l] || b[l * 4 + 1] > c.amin[l] + c.A[l] - 1 ||
                  b[l * 4 + 2] < c.bmin[l] || b[l * 4 + 3] > c.bmin[l] + c.B[l] - 1;
        }
        if (out) *B.overflow[r] = 1;
    }
}

// One grid pass (b-range scan, tables, pass or transpose) of every request.
struct PassBatch {
    int n;
    int block0[kBatchMax + 1];
    PassParams pp[kBatchMax];
    PassTables tab[kBatchMax];
    const void *in[kBatchMax];
    void *out[kBatchMax];
    const uint8_t *flags[kBatchMax];
    int2 *brange[kBatchMax];
    int64_t tiles[kBatchMax];  // pass: grid-point tiles per row; tables: table entries
    int64_t tx[kBatchMax];     // transpose: 32-row blocks
};

template <class C2>
__global__ void __launch_bounds__(256) brange_batch_kernel(const __grid_constant__ PassBatch B) {
    const int r = batch_request(B.block0, B.n);
    brange_body<C2>(reinterpret_cast<const C2 *>(B.in[r]), B.pp[r].rows * (int64_t)B.pp[r].A, B.pp[r].B, B.brange[r],
                    blockIdx.x - B.block0[r]);
}

__global__ void __launch_bounds__(256) tables_batch_kernel(const __grid_constant__ PassBatch B, int tp) {
    const int r = batch_request(B.block0, B.n);
    const int64_t mtiles = (B.pp[r].N + tp - 1) / tp;
    pass_tables_body(B.pp[r], tp, mtiles, B.tab[r], (int64_t)(blockIdx.x - B.block0[r]) * 256 + threadIdx.x);
}

template <bool FP64, int MAXBAND, int TP>
__global__ void __launch_bounds__(TP) grid_pass_batch_kernel(const __grid_constant__ PassBatch B) {
    const int r = batch_request(B.block0, B.n);
    const int64_t local = blockIdx.x - B.block0[r];
    const int64_t row = local / B.tiles[r];
    const int tile = (int)(local - row * B.tiles[r]);
    grid_pass_body<FP64, MAXBAND, TP>(B.in[r], B.out[r], B.pp[r], B.flags[r], B.brange[r], B.tab[r], row, tile, 0, 1);
}

template <class C2>
__global__ void transpose_batch_kernel(const __grid_constant__ PassBatch B) {
    const int r = batch_request(B.block0, B.n);
    const int64_t local = blockIdx.x - B.block0[r];
    const int64_t bx = local % B.tx[r], by = local / B.tx[r];
    transpose_body<C2>(reinterpret_cast<const C2 *>(B.in[r]), reinterpret_cast<C2 *>(B.out[r]), B.pp[r].rows,
                       B.pp[r].N, bx, by);
}

// Parameters of the grid pass over dimension l of a node box c; prodN_after =
// product of the grid sizes of the dimensions already contracted.
PassParams pass_params(const fgr_ctx *ctx, const Common &c, int l, int64_t prodN_after) {
    const Mesh &M = ctx->mesh;
    const Grid &G = ctx->grid;
    PassParams pp{};
    int64_t pre = 1;
    for (int j = 0; j < l; ++j) pre *= (int64_t)c.A[j] * c.B[j];
    pp.rows = pre * prodN_after;
    pp.A = c.A[l];
    pp.B = c.B[l];
    pp.amin = c.amin[l];
    pp.bmin = c.bmin[l];
    pp.N = G.n[l];
    pp.lo = G.lo[l];
    pp.h = G.h[l];
    pp.dq = M.dq;
    pp.rs = M.rs;
    pp.neg_half_inv_eps = -0.5 / M.eps;
    pp.phi_scale = M.dp / (2 * M_PI * M.eps);
    pp.dp_over_eps = M.dp / M.eps;
    const int bmax_abs = std::max(std::abs(c.bmin[l]), std::abs(c.bmin[l] + c.B[l] - 1));
    int lb = 1;
    while ((1 << lb) < bmax_abs + 1) ++lb;
    pp.two_pow_b = std::ldexp(1.0, std::max(1, 23 - lb));
    pp.inv_two_pow_b = 1.0 / pp.two_pow_b;
    return pp;
}

// Clears the node box and runs the coefficient scatter and the grid passes
// into u_dev (all stream-ordered: no allocation, no host synchronisation).
template <int D>
fgr_status enqueue_fggc(fgr_ctx *ctx, const PacketsDev &pk, const FggcBox &box, const FggcBuffers &b, void *u_dev,
                        cudaStream_t st, StageTimer *timer, int64_t *launches) {
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    const Grid &G = ctx->grid;
    const Lsa &L = ctx->lsa;
    const size_t eb = elem_bytes(ctx->opt.precision);
    const Common &c = box.c;
    // FP32 3-D: the binned scatter, which marks the rows its packets reach and
    // clears only those (the passes and b-range scans skip unmarked rows);
    // otherwise W is cleared whole and the scatter marks the rows it reaches
    BinLaunch bl;
    const bool binned = !fp64 && D == 3 && b.bin && b.bin_m >= pk.m && pk.m > 0 && (L.n1 == 4 || L.n1 == 8) &&
                        make_bin_box(box, D, &bl.box);
    if (!binned) FGR_CUDA_TRY(cudaMemsetAsync(b.W, 0, eb * (size_t)box.cells, st));
    // the single row of d = 1 is marked here
    FGR_CUDA_TRY(cudaMemsetAsync(b.flags, D == 1 ? 1 : 0, (size_t)box.rows0, st));
    if (timer) timer->mark(&ctx->timing.last.prep_ms);

    if (fp64) {
        Params64 P{};
        P.c = c;
        memcpy(P.vr, L.vr, sizeof(P.vr));
        memcpy(P.vi, L.vi, sizeof(P.vi));
        memcpy(P.inv_lam, L.inv_lam, sizeof(P.inv_lam));
        fgr_status r = launch_coeff_scatter(D, L.n1, st, pk, &P, nullptr, b.W, b.flags);
        if (r != FGR_OK) return r;
    } else {
        Params32 P{};
        P.c = c;
        for (int k = 0; k < kMaxN1; ++k)
            for (int i = 0; i < kCheb; ++i)
                for (int jj = 0; jj < kCheb; ++jj) {
                    P.cre[(k * kCheb + i) * kCheb + jj] = L.cheb_re[k][i][jj];
                    P.cim[(k * kCheb + i) * kCheb + jj] = L.cheb_im[k][i][jj];
                }
        fgr_status r;
        if (binned) {
            bin_buffers_at(b.bin, pk.m, bl.box, &bl.buf);
            bl.num_sms = ctx->num_sms;
            bl.min_count = kBinMinCount;
            bl.clear_rows = box.rows0;
            bl.row_cells = box.cells / box.rows0;
            StageMarks marks{timer, &ctx->timing.last.coeff_ms};
            r = launch_binned_scatter(D, L.n1, bl, st, pk, P, b.W, b.flags, &marks);
            *launches += 8;  // key, 3 scan, place, items, binned, loose
        } else {
            r = launch_coeff_scatter(D, L.n1, st, pk, nullptr, &P, b.W, b.flags);
        }
        if (r != FGR_OK) return r;
    }
    ++*launches;
    if (timer) timer->mark(&ctx->timing.last.scatter_ms);

    // separable passes, last dimension first
    const void *cur = b.W;
    int64_t prodN_after = 1;  // product of N of contracted dimensions
    for (int l = D - 1; l >= 0; --l) {
        const PassParams pp = pass_params(ctx, c, l, prodN_after);
        const bool last = l == 0;
        void *dst = (D == 1) ? u_dev : (cur == b.buf1 ? b.buf2 : b.buf1);
        const uint8_t *fl = l == D - 1 ? b.flags : nullptr;
        fgr_status r = fp64 ? launch_brange<true>(cur, pp.rows, pp.A, pp.B, fl, b.brange, st)
                            : launch_brange<false>(cur, pp.rows, pp.A, pp.B, fl, b.brange, st);
        if (r != FGR_OK) return r;
        ++*launches;
        const int64_t target = (int64_t)ctx->num_sms * ctx->tune.pass_ctas_per_sm;
        StageMarks before{timer, &ctx->timing.last.grid_ms};  // the pass kernel is timed alone
        if (ctx->fft_logn[l] > 0 && b.fft) {
            r = fp64 ? launch_fft_pass<true>(cur, dst, pp, fl, b.brange, ctx->fft_logn[l], b.fft, b.twiddle,
                                             b.tables, st, &before)
                     : launch_fft_pass<false>(cur, dst, pp, fl, b.brange, ctx->fft_logn[l], b.fft, b.twiddle,
                                              b.tables, st, &before);
            ++*launches;  // twiddles + DFT + contraction (tables and pass counted below)
        } else {
            r = fp64 ? launch_pass<true>(cur, dst, pp, fl, b.brange, target, ctx->tune.pass_tile, b.tables, st,
                                         &before, ctx->dev_err)
                     : launch_pass<false>(cur, dst, pp, fl, b.brange, target, ctx->tune.pass_tile, b.tables, st,
                                          &before, ctx->dev_err);
        }
        if (r != FGR_OK) return r;
        *launches += 2;  // tables + pass
        if (timer) {
            timer->mark(&ctx->timing.last.pass_ms);
            if (b.terms) {
                const int64_t lines = pp.rows * (int64_t)pp.A;
                const unsigned blocks = (unsigned)std::max<int64_t>(
                    1, std::min<int64_t>((lines + 255) / 256, (int64_t)ctx->num_sms * 8));
                pass_terms_kernel<<<blocks, 256, 0, st>>>(b.brange, lines, pp.A, (const int2 *)b.tables, b.terms);
                FGR_CUDA_TRY(cudaGetLastError());
            }
        }
        if (D > 1) {
            void *tdst = last ? u_dev : (dst == b.buf1 ? b.buf2 : b.buf1);
            r = fp64 ? launch_transpose<double2>(dst, tdst, pp.rows, pp.N, st)
                     : launch_transpose<float2>(dst, tdst, pp.rows, pp.N, st);
            if (r != FGR_OK) return r;
            ++*launches;
            cur = tdst;
        }
        prodN_after *= G.n[l];
    }
    if (timer) timer->mark(&ctx->timing.last.grid_ms);
    return FGR_OK;
}

template <int D>
fgr_status launch(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st, Scratch &scratch,
                  bool check_finite) {
    const size_t eb = elem_bytes(ctx->opt.precision);
    StageTimer timer(ctx, st);
    int64_t launches = 0;
    const Common c = base_common(ctx);
    int aglo[3], aghi[3];
    grid_node_range(ctx, aglo, aghi);
    int *bnd = (int *)scratch.get(sizeof(int) * 13);
    if (!bnd) return FGR_E_NOMEM;
    fgr_status r = launch_bounds_reduction(ctx, pk, c, aglo, aghi, bnd, st, check_finite);
    if (r != FGR_OK) return r;
    launches += pk.m > 0 ? 2 : 1;
    FGR_CUDA_TRY(cudaMemcpyAsync(ctx->host_pinned, bnd, sizeof(int) * 13, cudaMemcpyDeviceToHost, st));
    int *herr = reinterpret_cast<int *>(ctx->host_pinned) + 16;
    FGR_CUDA_TRY(cudaMemcpyAsync(herr, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FGR_CUDA_TRY(cudaStreamSynchronize(st));
    if (*herr) {  // a kernel of an earlier call gave up one of its bounded waits
        FGR_CUDA_TRY(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), st));
        set_error("fggc: a kernel of an earlier call on this context timed out waiting (grid-pass tile copies "
                  "or the tensor-core direct sum's pipeline); that call's output is incomplete");
        return FGR_E_TIMEOUT;
    }
    int hb[13];
    memcpy(hb, ctx->host_pinned, sizeof(hb));
    if (check_finite && hb[12]) {
        set_error("packets: a non-finite Q, P, S or A value");
        return FGR_E_INVALID;
    }
    FggcBox box;
    r = make_box(ctx, hb, 0, &box);
    if (r != FGR_OK) return r;
    if (box.empty) {  // nothing reaches the grid
        FGR_CUDA_TRY(cudaMemsetAsync(u_dev, 0, eb * (size_t)ctx->grid.total, st));
        timer.finish();
        ctx->timing.last.launches = launches;
        return FGR_OK;
    }
    ctx->timing.last.nodes = box.cells;
    FggcBuffers b{};
    b.W = scratch.get(eb * (size_t)box.cells);
    b.buf1 = D > 1 ? scratch.get(eb * (size_t)box.maxbuf) : nullptr;
    b.buf2 = D > 1 ? scratch.get(eb * (size_t)box.maxbuf) : nullptr;
    b.flags = (uint8_t *)scratch.get((size_t)box.rows0);
    b.brange = (int2 *)scratch.get(sizeof(int2) * (size_t)box.max_lines);
    b.tables = scratch.get(8 * (size_t)box.table_entries);
    if (!b.W || !b.flags || !b.brange || !b.tables || (D > 1 && (!b.buf1 || !b.buf2))) return FGR_E_NOMEM;
    if (box.fft_elems > 0) {
        b.fft = scratch.get(eb * (size_t)box.fft_elems);
        b.twiddle = scratch.get(eb * 4096);
        if (!b.fft || !b.twiddle) return FGR_E_NOMEM;
    }
    BinBox bb;
    if (ctx->opt.precision == FGR_FP32 && make_bin_box(box, D, &bb)) {
        b.bin = scratch.get(bin_buffer_bytes(pk.m, bb));
        if (!b.bin) return FGR_E_NOMEM;
        b.bin_m = pk.m;
    }
    if (ctx->timing.enabled && ctx->timing.count_terms) {
        b.terms = (unsigned long long *)scratch.get(sizeof(unsigned long long));
        if (!b.terms) return FGR_E_NOMEM;
        FGR_CUDA_TRY(cudaMemsetAsync(b.terms, 0, sizeof(unsigned long long), st));
    }
    r = enqueue_fggc<D>(ctx, pk, box, b, u_dev, st, &timer, &launches);
    if (r != FGR_OK) return r;
    ctx->timing.last.launches = launches;
    timer.finish();
    if (ctx->timing.enabled) ctx->timing.last.grid_ms += ctx->timing.last.pass_ms;  // the whole grid stage
    if (b.terms) {
        unsigned long long terms = 0;
        FGR_CUDA_TRY(cudaMemcpy(&terms, b.terms, sizeof(terms), cudaMemcpyDeviceToHost));
        ctx->timing.last.pass_terms = (int64_t)terms;
    }
    return FGR_OK;
}

}  // namespace

namespace {

// Blocks of a batched launch: block0 = prefix of per-request counts.
template <class Batch>
bool set_blocks(Batch &B, const std::vector<int64_t> &counts) {
    int64_t acc = 0;
    for (size_t r = 0; r < counts.size(); ++r) {
        B.block0[r] = (int)acc;
        acc += counts[r];
        if (acc > INT_MAX) return false;
    }
    B.block0[counts.size()] = (int)acc;
    return true;
}

// One chunk (<= kBatchMax requests) of one dimension D: fill, bounds, box
// check, scatter, passes: every stage one launch for the whole chunk.
template <int D>
fgr_status enqueue_fggc_batch(int n, const FggcRequest *req, cudaStream_t st) {
    const fgr_ctx *ctx0 = req[0].ctx;
    const bool fp64 = ctx0->opt.precision == FGR_FP64;
    const size_t eb = elem_bytes(ctx0->opt.precision);
    const int num_sms = ctx0->num_sms;
    auto too_many = [] {
        set_error("fggc batch: too many CTAs in one launch");
        return FGR_E_CAPACITY;
    };
    // fills: the node array and row flags of every non-empty box; the output
    // of an empty one (nothing reaches its grid)
    {
        FillBatch fb{};
        std::vector<int64_t> cnt;
        auto seg = [&](void *ptr, int64_t bytes, int value) {
            if (bytes <= 0) return;
            fb.ptr[fb.n] = (unsigned char *)ptr;
            fb.bytes[fb.n] = bytes;
            fb.value[fb.n] = value;
            cnt.push_back(std::max<int64_t>(1, std::min<int64_t>((bytes + 16383) / 16384, 4 * (int64_t)num_sms)));
            ++fb.n;
        };
        for (int r = 0; r < n; ++r) {
            const FggcRequest &q = req[r];
            if (q.box->empty) {
                seg(q.u, (int64_t)(eb * (size_t)q.ctx->grid.total), 0);
            } else {
                seg(q.buf->W, (int64_t)(eb * (size_t)q.box->cells), 0);
                seg(q.buf->flags, q.box->rows0, D == 1 ? 1 : 0);
            }
        }
        if (fb.n > 0) {
            if (!set_blocks(fb, cnt)) return too_many();
            fill_batch_kernel<<<fb.block0[fb.n], 256, 0, st>>>(fb);
        }
    }
    std::vector<int> live;  // requests with a non-empty box
    for (int r = 0; r < n; ++r)
        if (!req[r].box->empty) live.push_back(r);
    if (live.empty()) {
        FGR_CUDA_TRY(cudaGetLastError());
        return FGR_OK;
    }
    const int nl = (int)live.size();
    // node bounds of the packets, compared with the planned boxes
    {
        BoundsBatch bb{};
        bb.n = nl;
        std::vector<int64_t> cnt;
        for (int i = 0; i < nl; ++i) {
            const FggcRequest &q = req[live[i]];
            bb.c[i] = base_common(q.ctx);
            bb.q[i] = q.pk.q;
            bb.p[i] = q.pk.p;
            bb.a[i] = q.pk.a;
            bb.m[i] = q.pk.m;
            grid_node_range(q.ctx, bb.aglo[i], bb.aghi[i]);
            bb.out[i] = q.bnd;
            bb.overflow[i] = q.overflow;
            cnt.push_back(std::max<int64_t>(1, std::min<int64_t>((q.pk.m + 255) / 256, 8 * (int64_t)num_sms / nl + 1)));
        }
        if (!set_blocks(bb, cnt)) return too_many();
        bounds_init_batch_kernel<<<1, 256, 0, st>>>(bb);
        bounds_batch_kernel<D><<<bb.block0[nl], 256, 0, st>>>(bb);
        for (int i = 0; i < nl; ++i) bb.c[i] = req[live[i]].box->c;  // planned boxes for the check
        box_check_batch_kernel<<<1, 64, 0, st>>>(bb, D);
    }
    // coefficients + scatter (per-packet form)
    {
        const Lsa &L = ctx0->lsa;
        const int T = scatter_threads(fp64, L.n1);
        std::vector<int64_t> cnt;
        ScatterBatchBase *base;
        std::unique_ptr<ScatterBatch64> b64;
        std::unique_ptr<ScatterBatch32> b32;
        if (fp64) {
            b64.reset(new ScatterBatch64());
            memcpy(b64->vr, L.vr, sizeof(b64->vr));
            memcpy(b64->vi, L.vi, sizeof(b64->vi));
            memcpy(b64->inv_lam, L.inv_lam, sizeof(b64->inv_lam));
            base = b64.get();
        } else {
            b32.reset(new ScatterBatch32());
            for (int k = 0; k < kMaxN1; ++k)
                for (int i = 0; i < kCheb; ++i)
                    for (int jj = 0; jj < kCheb; ++jj) {
                        b32->cre[(k * kCheb + i) * kCheb + jj] = L.cheb_re[k][i][jj];
                        b32->cim[(k * kCheb + i) * kCheb + jj] = L.cheb_im[k][i][jj];
                    }
            base = b32.get();
        }
        base->n = nl;
        for (int i = 0; i < nl; ++i) {
            const FggcRequest &q = req[live[i]];
            base->c[i] = q.box->c;
            base->q[i] = q.pk.q;
            base->p[i] = q.pk.p;
            base->s[i] = q.pk.s;
            base->a[i] = q.pk.a;
            base->m[i] = q.pk.m;
            base->W[i] = q.buf->W;
            base->flags[i] = q.buf->flags;
            cnt.push_back((q.pk.m + T - 1) / T);
        }
        if (!set_blocks(*base, cnt)) return too_many();
        fgr_status r = launch_scatter_batch(D, L.n1, st, b64.get(), b32.get());
        if (r != FGR_OK) return r;
    }
    // separable passes, last dimension first
    constexpr int TP = 128;
    std::vector<const void *> cur(nl);
    std::vector<int64_t> prodN(nl, 1);
    for (int i = 0; i < nl; ++i) cur[i] = req[live[i]].buf->W;
    for (int l = D - 1; l >= 0; --l) {
        PassBatch pb{};
        pb.n = nl;
        int band = 1;
        std::vector<void *> dst(nl);
        for (int i = 0; i < nl; ++i) {
            const FggcRequest &q = req[live[i]];
            pb.pp[i] = pass_params(q.ctx, q.box->c, l, prodN[i]);
            const PassParams &pp = pb.pp[i];
            if (pp.rows > INT_MAX) {
                set_error("fggc batch: too many rows in a grid pass");
                return FGR_E_CAPACITY;
            }
            const FggcBuffers &b = *q.buf;
            dst[i] = D == 1 ? q.u : (cur[i] == b.buf1 ? b.buf2 : b.buf1);
            pb.in[i] = cur[i];
            pb.out[i] = dst[i];
            pb.flags[i] = l == D - 1 ? b.flags : nullptr;
            pb.brange[i] = b.brange;
            PassTables tab;
            tab.win = reinterpret_cast<int2 *>(b.tables);
            tab.ph = reinterpret_cast<float2 *>(tab.win + pp.A);
            tab.band = reinterpret_cast<int2 *>(tab.ph + pp.N);
            pb.tab[i] = tab;
            pb.tiles[i] = (pp.N + TP - 1) / TP;
            if (pb.tiles[i] > 65535) {
                set_error("fggc batch: %lld points per grid dimension; at most %d", (long long)pp.N, 65535 * TP);
                return FGR_E_INVALID;
            }
            band = std::max(band, pass_band(TP, pp.h, pp.rs, pp.dq));
        }
        std::vector<int64_t> cnt(nl);
        for (int i = 0; i < nl; ++i) cnt[i] = (pb.pp[i].rows * (int64_t)pb.pp[i].A + 7) / 8;
        if (!set_blocks(pb, cnt)) return too_many();
        if (fp64)
            brange_batch_kernel<double2><<<pb.block0[nl], 256, 0, st>>>(pb);
        else
            brange_batch_kernel<float2><<<pb.block0[nl], 256, 0, st>>>(pb);
        for (int i = 0; i < nl; ++i)
            cnt[i] = (std::max<int64_t>(std::max<int64_t>(pb.pp[i].A, pb.pp[i].N), pb.tiles[i]) + 255) / 256;
        if (!set_blocks(pb, cnt)) return too_many();
        tables_batch_kernel<<<pb.block0[nl], 256, 0, st>>>(pb, TP);
        for (int i = 0; i < nl; ++i) cnt[i] = pb.pp[i].rows * pb.tiles[i];
        if (!set_blocks(pb, cnt)) return too_many();
#define FGR_PB(MB)                                                                                   \
    if (fp64)                                                                                        \
        grid_pass_batch_kernel<true, MB, TP><<<pb.block0[nl], TP, 0, st>>>(pb);                      \
    else                                                                                             \
        grid_pass_batch_kernel<false, MB, TP><<<pb.block0[nl], TP, 0, st>>>(pb);
        if (band <= 16) {
            FGR_PB(16)
        } else if (band <= 32) {
            FGR_PB(32)
        } else if (band <= 48) {
            FGR_PB(48)
        } else {
            FGR_PB(64)
        }
#undef FGR_PB
        if (D > 1) {
            for (int i = 0; i < nl; ++i) {
                const FggcRequest &q = req[live[i]];
                const FggcBuffers &b = *q.buf;
                pb.in[i] = dst[i];
                pb.out[i] = l == 0 ? q.u : (dst[i] == b.buf1 ? b.buf2 : b.buf1);
                pb.tx[i] = (pb.pp[i].rows + 31) / 32;
                cnt[i] = pb.tx[i] * ((pb.pp[i].N + 31) / 32);
                cur[i] = pb.out[i];
            }
            if (!set_blocks(pb, cnt)) return too_many();
            if (fp64)
                transpose_batch_kernel<double2><<<pb.block0[nl], dim3(32, 8), 0, st>>>(pb);
            else
                transpose_batch_kernel<float2><<<pb.block0[nl], dim3(32, 8), 0, st>>>(pb);
        }
        for (int i = 0; i < nl; ++i) prodN[i] *= req[live[i]].ctx->grid.n[l];
    }
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace

fgr_status launch_scatter_batch(int d, int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32) {
    switch (d) {
    case 1: return launch_scatter_batch_d1(n1, st, b64, b32);
    case 2: return launch_scatter_batch_d2(n1, st, b64, b32);
    default: return launch_scatter_batch_d3(n1, st, b64, b32);
    }
}

fgr_status run_fggc_batch(int n, const FggcRequest *req, cudaStream_t st) {
    // requests of one dimension together, kBatchMax per launch
    for (int d = 1; d <= 3; ++d) {
        std::vector<FggcRequest> group;
        for (int r = 0; r < n; ++r)
            if (req[r].ctx->d == d) group.push_back(req[r]);
        for (size_t i0 = 0; i0 < group.size(); i0 += kBatchMax) {
            const int k = (int)std::min<size_t>(kBatchMax, group.size() - i0);
            fgr_status r = d == 1 ? enqueue_fggc_batch<1>(k, group.data() + i0, st)
                         : d == 2 ? enqueue_fggc_batch<2>(k, group.data() + i0, st)
                                  : enqueue_fggc_batch<3>(k, group.data() + i0, st);
            if (r != FGR_OK) return r;
        }
    }
    return FGR_OK;
}

fgr_status launch_coeff_scatter(int d, int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                const Params32 *p32, void *W, uint8_t *flags) {
    switch (d) {
    case 1: return launch_coeff_scatter_d1(n1, st, pk, p64, p32, W, flags);
    case 2: return launch_coeff_scatter_d2(n1, st, pk, p64, p32, W, flags);
    default: return launch_coeff_scatter_d3(n1, st, pk, p64, p32, W, flags);
    }
}

fgr_status run_fggc(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st, Scratch &scratch,
                    bool check_finite) {
    switch (ctx->d) {
    case 1: return launch<1>(ctx, pk, u_dev, st, scratch, check_finite);
    case 2: return launch<2>(ctx, pk, u_dev, st, scratch, check_finite);
    default: return launch<3>(ctx, pk, u_dev, st, scratch, check_finite);
    }
}

// Node bounds of the packets (per dimension: a min, a max, b min, b max; a
// clipped to the grid-relevant range) into hb on the host; waits for them.
fgr_status compute_node_bounds(fgr_ctx *ctx, const PacketsDev &pk, int *bnd_dev, int *hb, cudaStream_t st) {
    const Common c = base_common(ctx);
    int aglo[3], aghi[3];
    grid_node_range(ctx, aglo, aghi);
    fgr_status r = launch_bounds_reduction(ctx, pk, c, aglo, aghi, bnd_dev, st);
    if (r != FGR_OK) return r;
    FGR_CUDA_TRY(cudaMemcpyAsync(ctx->host_pinned, bnd_dev, sizeof(int) * 12, cudaMemcpyDeviceToHost, st));
    FGR_CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(hb, ctx->host_pinned, sizeof(int) * 12);
    return FGR_OK;
}

// Planned reconstruction: the node box and the buffers come from a plan; the
// packets' bounds are recomputed on the device and compared with the box
// (overflow flag), so nothing waits for the host.
fgr_status run_fggc_planned(fgr_ctx *ctx, const PacketsDev &pk, const FggcBox &box, const FggcBuffers &b,
                            int *bnd, int *overflow, void *u_dev, cudaStream_t st) {
    const Common c = base_common(ctx);
    int aglo[3], aghi[3];
    grid_node_range(ctx, aglo, aghi);
    FGR_CUDA_TRY(cudaMemsetAsync(overflow, 0, sizeof(int), st));
    fgr_status r = launch_bounds_reduction(ctx, pk, c, aglo, aghi, bnd, st);
    if (r != FGR_OK) return r;
    if (box.empty) {
        FGR_CUDA_TRY(cudaMemsetAsync(u_dev, 0, elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total, st));
        return FGR_OK;
    }
    box_check_kernel<<<1, 32, 0, st>>>(bnd, ctx->d, box.c, overflow);
    FGR_CUDA_TRY(cudaGetLastError());
    int64_t launches = 0;
    switch (ctx->d) {
    case 1: return enqueue_fggc<1>(ctx, pk, box, b, u_dev, st, nullptr, &launches);
    case 2: return enqueue_fggc<2>(ctx, pk, box, b, u_dev, st, nullptr, &launches);
    default: return enqueue_fggc<3>(ctx, pk, box, b, u_dev, st, nullptr, &launches);
    }
}

}  // namespace fgr

// ---------------------------------------------------------------------------
// fgr_reconstruct_fggc_noalloc: the 1-D FGGC reconstruction with all of its
// working memory in one fixed device array, for callers that must not
// allocate (see include/fgr.h).  It launches the same kernels as
// fgr_reconstruct_fggc; only where the working memory comes from differs.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

// Working memory of the no-allocation entry point: bounds (256 B), row flags
// (256 B), then the node array.  Lives in every device that loads the library.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr size_t kNoAllocNodesOffset = 512;
static __device__ __align__(256) unsigned char fgr_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_base[kNoAllocMaxDevices] = {};

// Device address of fgr_noalloc_scratch on the current device (looked up once
// per device).  Host code must not use the symbol itself as an address.
fgr_status noalloc_base(int device, unsigned char **out) {
    if (device < 0 || device >= kNoAllocMaxDevices) {
        fgr::set_error("noalloc: device ordinal %d out of range", device);
        return FGR_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fgr_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fgr::set_error("noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return FGR_E_CUDA;
        }
        g_noalloc_base[device] = p;
    }
    *out = (unsigned char *)g_noalloc_base[device];
    return FGR_OK;
}

}  // namespace

extern "C" fgr_status fgr_reconstruct_fggc_noalloc(fgr_ctx *ctx, const fgr_packets *pk, void *u_out,
                                                   void *stream) {
    using namespace fgr;
    clear_error();
    if (!ctx || !pk || !u_out) {
        set_error("noalloc: ctx, packets and u_out must be non-NULL");
        return FGR_E_INVALID;
    }
    if (ctx->d != 1) {
        set_error("noalloc: only 1-D contexts are supported (d = %d)", ctx->d);
        return FGR_E_INVALID;
    }
    if (pk->m < 0 || pk->m > (int64_t(1) << 31) || pk->on_device != 1 ||
        (pk->m > 0 && (!pk->q || !pk->p || !pk->s || !pk->a))) {
        set_error("noalloc: packets must be device arrays (on_device = 1), 0 <= m <= 2^31");
        return FGR_E_INVALID;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        set_error("noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
        return FGR_E_CUDA;
    }
    {
        // u_out and the packet arrays: device memory of this context's device
        // (or managed memory)
        const void *ptrs[5] = {u_out, pk->q, pk->p, pk->s, pk->a};
        const char *names[5] = {"u_out", "q", "p", "s", "a"};
        for (int i = 0; i < (pk->m > 0 ? 5 : 1); ++i) {
            cudaPointerAttributes at;
            const bool ok = cudaPointerGetAttributes(&at, ptrs[i]) == cudaSuccess &&
                            ((at.type == cudaMemoryTypeDevice && at.device == ctx->device) ||
                             at.type == cudaMemoryTypeManaged);
            if (!ok) {
                cudaGetLastError();
                set_error("noalloc: %s must be device memory of device %d", names[i], ctx->device);
                return FGR_E_INVALID;
            }
        }
    }
    unsigned char *base = nullptr;
    fgr_status rc = noalloc_base(ctx->device, &base);
    if (rc != FGR_OK) return rc;
    int *bnd = (int *)base;
    uint8_t *flags = base + 256;
    void *W = base + kNoAllocNodesOffset;

    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    const Mesh &M = ctx->mesh;
    const Grid &G = ctx->grid;
    const Lsa &L = ctx->lsa;
    const size_t eb = elem_bytes(ctx->opt.precision);
    const size_t out_bytes = eb * (size_t)G.n[0];

    Common c{};
    c.n1 = L.n1;
    for (int k = 0; k < L.n1; ++k) {
        c.dq[k] = L.dq[k];
        c.dp[k] = L.dp[k];
    }
    c.dqv = M.dq;
    c.dpv = M.dp;
    c.inv_dq = 1.0 / M.dq;
    c.inv_dp = 1.0 / M.dp;
    c.cq2_4 = M.cq * M.cq / 4;
    c.cp2_4 = M.cp * M.cp / 4;
    c.half_cqcp = M.cqcp / 2;
    c.cc = M.cqcp / (2 * M_PI);
    c.inv_2pi_eps = 1.0 / (2 * M_PI * M.eps);
    c.pref = M.pref;
    const double xlast = G.lo[0] + (double)(G.n[0] - 1) * G.h[0];
    const int aglo = (int)std::max(-1e9, std::ceil((G.lo[0] - M.rs) / M.dq) - 1);
    const int aghi = (int)std::min(1e9, std::floor((xlast + M.rs) / M.dq) + 1);

    // bounds start at (+inf, -inf): they are rewritten on every call
    int init[12];
    for (int l = 0; l < 3; ++l) {
        init[l * 4 + 0] = INT_MAX;
        init[l * 4 + 1] = INT_MIN;
        init[l * 4 + 2] = INT_MAX;
        init[l * 4 + 3] = INT_MIN;
    }
    memcpy(ctx->host_pinned, init, sizeof(init));
    FGR_CUDA_TRY(cudaMemcpyAsync(bnd, ctx->host_pinned, sizeof(init), cudaMemcpyHostToDevice, st));
    const int64_t m = pk->m;
    if (m > 0) {
        bounds_kernel<1><<<bounds_blocks(ctx, m), 256, 0, st>>>(pk->q, pk->p, pk->a, m, c, aglo, aghi,
                                                                     0, -1, 0, -1, bnd, nullptr);
        FGR_CUDA_TRY(cudaGetLastError());
    }
    FGR_CUDA_TRY(cudaMemcpyAsync(ctx->host_pinned, bnd, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    FGR_CUDA_TRY(cudaStreamSynchronize(st));
    int hb[4];
    memcpy(hb, ctx->host_pinned, sizeof(hb));
    if (m == 0 || hb[0] == INT_MAX) {
        FGR_CUDA_TRY(cudaMemsetAsync(u_out, 0, out_bytes, st));
        if (!stream) FGR_CUDA_TRY(cudaStreamSynchronize(st));
        return FGR_OK;
    }
    c.amin[0] = hb[0];
    c.A[0] = hb[1] - hb[0] + 1;
    c.bmin[0] = hb[2];
    c.B[0] = hb[3] - hb[2] + 1;
    const int64_t cells = (int64_t)c.A[0] * c.B[0];
    // node array, then the grid pass's tables (8 bytes per node and per grid point)
    const size_t node_bytes = ((size_t)cells * eb + 15) / 16 * 16;
    const size_t table_bytes = 8 * (size_t)pass_table_entries(c.A[0], G.n[0]);
    if ((size_t)cells > (kNoAllocBytes - kNoAllocNodesOffset) / eb ||
        node_bytes + table_bytes > kNoAllocBytes - kNoAllocNodesOffset) {
        set_error("noalloc: the node array needs %lld cells (%zu bytes) and the pass tables %zu bytes; this entry "
                  "point holds at most %zu bytes; use fgr_reconstruct_fggc",
                  (long long)cells, (size_t)cells * eb, table_bytes, kNoAllocBytes - kNoAllocNodesOffset);
        return FGR_E_CAPACITY;
    }
    void *tables = static_cast<unsigned char *>(W) + node_bytes;
    c.sb[0] = 1;
    c.sa[0] = c.B[0];
    c.row_len = cells;
    // the node array accumulates: clear it; the single row is marked non-empty
    FGR_CUDA_TRY(cudaMemsetAsync(W, 0, eb * (size_t)cells, st));
    FGR_CUDA_TRY(cudaMemsetAsync(flags, 1, 1, st));
    if (fp64) {
        Params64 P{};
        P.c = c;
        memcpy(P.vr, L.vr, sizeof(P.vr));
        memcpy(P.vi, L.vi, sizeof(P.vi));
        memcpy(P.inv_lam, L.inv_lam, sizeof(P.inv_lam));
        rc = launch_coeff_scatter(1, L.n1, st, PacketsDev{m, pk->q, pk->p, pk->s, pk->a}, &P, nullptr, W, flags);
        if (rc != FGR_OK) return rc;
    } else {
        Params32 P{};
        P.c = c;
        for (int k = 0; k < kMaxN1; ++k)
            for (int i = 0; i < kCheb; ++i)
                for (int jj = 0; jj < kCheb; ++jj) {
                    P.cre[(k * kCheb + i) * kCheb + jj] = L.cheb_re[k][i][jj];
                    P.cim[(k * kCheb + i) * kCheb + jj] = L.cheb_im[k][i][jj];
                }
        rc = launch_coeff_scatter(1, L.n1, st, PacketsDev{m, pk->q, pk->p, pk->s, pk->a}, nullptr, &P, W, flags);
        if (rc != FGR_OK) return rc;
    }
    PassParams pp{};
    pp.rows = 1;
    pp.A = c.A[0];
    pp.B = c.B[0];
    pp.amin = c.amin[0];
    pp.bmin = c.bmin[0];
    pp.N = G.n[0];
    pp.lo = G.lo[0];
    pp.h = G.h[0];
    pp.dq = M.dq;
    pp.rs = M.rs;
    pp.neg_half_inv_eps = -0.5 / M.eps;
    pp.phi_scale = M.dp / (2 * M_PI * M.eps);
    pp.dp_over_eps = M.dp / M.eps;
    const int bmax_abs = std::max(std::abs(c.bmin[0]), std::abs(c.bmin[0] + c.B[0] - 1));
    int lb = 1;
    while ((1 << lb) < bmax_abs + 1) ++lb;
    pp.two_pow_b = std::ldexp(1.0, std::max(1, 23 - lb));
    pp.inv_two_pow_b = 1.0 / pp.two_pow_b;
    const int64_t target = (int64_t)ctx->num_sms * ctx->tune.pass_ctas_per_sm;
    rc = fp64 ? launch_pass<true>(W, u_out, pp, flags, nullptr, target, ctx->tune.pass_tile, tables, st)
              : launch_pass<false>(W, u_out, pp, flags, nullptr, target, ctx->tune.pass_tile, tables, st);
    if (rc != FGR_OK) return rc;
    if (!stream) FGR_CUDA_TRY(cudaStreamSynchronize(st));
    return FGR_OK;
}
