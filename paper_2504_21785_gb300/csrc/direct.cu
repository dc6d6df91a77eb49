// K2: windowed direct sum of eq. 2.10 with packets binned by output tile.
//
// Binning.  The output grid is cut into tiles of T[0] x ... x T[d-1] points.
// A packet's "home tile" is the tile holding the lower corner of its clipped
// window; a counting sort groups packets by home tile.  An output tile t then
// needs exactly the packets whose home tile lies in the box t - K .. t, with
// K_l = ceil((Wmax_l - 1) / T_l) and Wmax_l the largest window length.  In
// row-major tile order that box is (K+1)^(d-1) contiguous segments.
//
// Evaluation.  Each CTA owns one output tile (4 consecutive points of the last
// dimension per thread) and one of S interleaved slices of the tile's packet
// list; packet records are staged in shared memory 256 at a time.  FP32, 1-D:
// a thread evaluates exp and sincos for the first of its points and reaches the
// other three by the exact recurrences of the Gaussian ratio and the phase
// rotation.  FP32, 2-D and 3-D: the CTA tabulates each record's per-dimension
// factors on its tile and every pair costs one complex multiply-add.  FP64:
// every pair is evaluated in full.  FP32 sums run over one chunk of 256
// records and are folded into FP64 totals (a point can collect 10^4-10^5
// packets: a single FP32 running sum would drift by ~sqrt(N) ulps).  Slices
// are combined with atomic adds into the zeroed output.  This CUDA-core
// evaluation serves FP64, 1-D, batched calls and FGR_FLAG_DIRECT_FMA; a single
// FP32 call with d >= 2 runs the same binned records through the tensor-core
// kernel of direct_tc.cuh (super tiles of several tiles, 3 x TF32 MMAs).
//
// FP32 records carry the per-packet phase reduced in FP64 to turns at the
// window start (tau0) and the per-grid-step increment nu split into a coarse
// part nu_hi (a multiple of 2^-b, so k*nu_hi is exact in FP32 for k < 2^(24-b))
// and a small remainder nu_lo.  FP64 records carry Q, P, S, A and every pair is
// evaluated in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_util.cuh"
#include "internal.h"

namespace fgr {
namespace {

constexpr int kThreads = 256;
constexpr int kTpt = 4;                        // consecutive points per thread (last dimension)
constexpr int kMaxSeg = 1024;                  // segments per tile list

// Output tile extent per dimension (kThreads * kTpt = 1024 points per tile);
// the last dimension's extent is a multiple of kTpt.
template <int D>
__host__ __device__ constexpr int tileT(int l) {
    return D == 1 ? 1024 : (D == 2 ? 32 : (l < 2 ? 8 : 16));
}
static_assert(tileT<1>(0) == kThreads * kTpt && tileT<2>(0) * tileT<2>(1) == kThreads * kTpt &&
                  tileT<3>(0) * tileT<3>(1) * tileT<3>(2) == kThreads * kTpt,
              "tiles hold kThreads * kTpt points");
static_assert(tileT<2>(0) % 4 == 0 && tileT<2>(1) % 4 == 0 && tileT<3>(0) % 4 == 0 && tileT<3>(1) % 4 == 0 &&
                  tileT<3>(2) % 4 == 0,
              "the factor tables of d >= 2 are filled 4 grid lines at a time");

template <int D>
struct __align__(16) RecF {
    float mlo[D];    // window start (grid index, exact in FP32)
    float wlen[D];   // window length
    float delta[D];  // x_{mlo} - Q per dimension
    float nuhi[D];   // turns per grid step, coarse part
    float nulo[D];   // remainder
    float tau0;      // phase of pref * A * e^{i theta} at the window start, turns in [-0.5, 0.5)
    float la;        // log2 |pref * A| (-inf for A = 0)
    float spare;
};

template <int D>
struct __align__(16) RecD {
    int mlo[D];
    int wlen[D];
    double Q[D], P[D];
    double S, ar, ai;  // S, pref * A
};

struct GridDev {
    int64_t n[3];
    double lo[3], h[3];
    int nt[3];   // tiles per dimension
    int K[3];    // home-tile reach
    int ntiles;
};

template <int D>
__device__ __forceinline__ int tile_linear(const GridDev &g, const int *t) {
    int lin = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) lin = lin * g.nt[l] + t[l];
    return lin;
}

// Pass 1: windows, home tile, per-tile counts (one atomic per tile and warp).
template <int D>
__global__ void bin_count_kernel(const double *__restrict__ q, int64_t m, GridDev g, double rs,
                                 int *__restrict__ home, int *__restrict__ counts) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int lin = -1;
    if (j < m) {
        int t[D];
        bool empty = false;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            int64_t lo, hi;
            window_bounds(q[l * m + j], rs, g.lo[l], g.h[l], g.n[l], &lo, &hi);
            if (lo > hi) empty = true;
            t[l] = (int)(lo / tileT<D>(l));
        }
        if (!empty) lin = tile_linear<D>(g, t);
        home[j] = lin;
    }
    const unsigned group = __match_any_sync(0xffffffffu, lin);
    const int lane = threadIdx.x & 31;
    if (lin >= 0 && lane == __ffs(group) - 1) atomicAdd(&counts[lin], __popc(group));
}

// Exclusive scan of n counts into off[0..n] (single CTA, sequential blocks).
__global__ void scan_kernel(const int *__restrict__ counts, int64_t *__restrict__ off, int n) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        int64_t v = i < n ? counts[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < 1024; s <<= 1) {
            int64_t add = threadIdx.x >= s ? part[threadIdx.x - s] : 0;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) off[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

struct RecParams {
    double rs, eps, inv_eps, pref;
    double two_pow_b;  // 2^b for the nu split
    double inv_two_pow_b;
};

// Pass 2: build the records in binned order.
template <int D, bool FP64>
__global__ void bin_scatter_kernel(const double *__restrict__ q, const double *__restrict__ p,
                                   const double *__restrict__ s, const double *__restrict__ a,
                                   int64_t m, GridDev g, RecParams rp, const int *__restrict__ home,
                                   const int64_t *__restrict__ off, int *__restrict__ cursor,
                                   void *__restrict__ recs) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int h = j < m ? home[j] : -1;
    // one atomic per tile and warp; lanes of a group take consecutive slots
    const unsigned group = __match_any_sync(0xffffffffu, h);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(group) - 1;
    int base = 0;
    if (h >= 0 && lane == leader) base = atomicAdd(&cursor[h], __popc(group));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (h < 0) return;
    const int64_t pos = off[h] + base + __popc(group & ((1u << lane) - 1u));
    const double ar = rp.pref * a[j], ai = rp.pref * a[m + j];
    if (FP64) {
        RecD<D> r;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            int64_t lo, hi;
            window_bounds(q[l * m + j], rp.rs, g.lo[l], g.h[l], g.n[l], &lo, &hi);
            r.mlo[l] = (int)lo;
            r.wlen[l] = (int)(hi - lo + 1);
            r.Q[l] = q[l * m + j];
            r.P[l] = p[l * m + j];
        }
        r.S = s[j];
        r.ar = ar;
        r.ai = ai;
        reinterpret_cast<RecD<D> *>(recs)[pos] = r;
    } else {
        RecF<D> r;
        double phase = s[j];
        const double inv_2pi_eps = rp.inv_eps * 0.15915494309189535;  // 1/(2 pi eps)
#pragma unroll
        for (int l = 0; l < D; ++l) {
            int64_t lo, hi;
            const double Q = q[l * m + j], P = p[l * m + j];
            window_bounds(Q, rp.rs, g.lo[l], g.h[l], g.n[l], &lo, &hi);
            r.mlo[l] = (float)lo;
            r.wlen[l] = (float)(hi - lo + 1);
            const double dx = grid_x(g.lo[l], g.h[l], lo) - Q;
            r.delta[l] = (float)dx;
            phase += P * dx;
            double nu = P * g.h[l] * inv_2pi_eps;  // turns per grid step
            nu -= rint(nu);
            const double nuhi = rint(nu * rp.two_pow_b) * rp.inv_two_pow_b;
            r.nuhi[l] = (float)nuhi;
            r.nulo[l] = (float)(nu - nuhi);
        }
        // the amplitude's argument joins the phase, its modulus the Gaussian's exponent
        double tau = phase * inv_2pi_eps;
        tau -= rint(tau);
        tau += atan2(ai, ar) * 0.15915494309189535;
        tau -= rint(tau);
        r.tau0 = (float)tau;
        r.la = (float)log2(hypot(ar, ai));
        r.spare = 0.f;
        reinterpret_cast<RecF<D> *>(recs)[pos] = r;
    }
}

struct DirectParams {
    GridDev g;
    float hf[3];         // grid steps (FP32 path)
    float ce;            // -log2(e) / (2 eps)
    float ce_h;          // ce * h of the last dimension
    float q_last;        // e^{-h^2 / eps} of the last dimension (Gaussian ratio step)
    float q_dim[3];      // e^{-h_l^2 / eps} per dimension (factor tables, d >= 2)
    float q8[3];         // e^{-64 h_l^2 / eps}: Gaussian ratio step over 8 grid lines (tensor-core path)
    double inv_eps;      // FP64 path
    double neg_half_inv_eps;
    int splits;
};

// FP32, d >= 2: the term of a packet factorises over dimensions,
//   pref A e^{i S/eps} prod_l exp(-(x_l - Q_l)^2 / (2 eps) + i P_l (x_l - Q_l) / eps),
// with each factor zero outside the packet's window in that dimension.  For a
// sub-chunk of kSub staged records the CTA tabulates every record's factors
// on the tile's grid lines (sum of the tile extents per record; the amplitude
// and the phase at the window start go into the first dimension's factor),
// then each thread accumulates the products over its 4 points: one complex
// multiply-add per packet-point pair.
template <int D>
__host__ __device__ constexpr int kSumT() {
    return D == 1 ? tileT<1>(0) : (D == 2 ? tileT<2>(0) + tileT<2>(1) : tileT<3>(0) + tileT<3>(1) + tileT<3>(2));
}
template <int D>
__host__ __device__ constexpr int kSub() {
    return D == 3 ? 64 : 32;  // records per factor table (20 KB for d = 2, 16 KB for d = 3)
}

// Points of a thread in the separable path (FP32, d >= 2): a 2 x 2 block of
// the tile, so that each staged record costs two 16-byte factor loads and four
// complex multiply-adds.  d = 2 (32 x 32 tile): rows 2 (tid / 16) + {0, 1},
// columns 2 (tid % 16) + {0, 1}.  d = 3 (8 x 8 x 16 tile): i = tid / 32,
// j = 2 ((tid / 8) % 4) + {0, 1}, k = 2 (tid % 8) + {0, 1}.  Point r of the
// block is (second-to-last + r / 2, last + r % 2).
template <int D>
__device__ __forceinline__ void separable_local(int tid, int *loc) {
    if (D == 2) {
        loc[0] = 2 * (tid / 16);
        loc[1] = 2 * (tid % 16);
    } else {
        loc[0] = tid / 32;
        loc[1] = 2 * ((tid / 8) % 4);
        loc[2] = 2 * (tid % 8);
    }
}

template <int D>
__device__ __forceinline__ void separable_chunk(const int *__restrict__ srec, const int nrec, const DirectParams &P,
                                                const int *t, float2 *__restrict__ sfac, float (*accf)[2]) {
    constexpr int kWords = sizeof(RecF<D>) / 4;
    constexpr int kS = kSub<D>(), kT = kSumT<D>();
    int loc[D];
    separable_local<D>(threadIdx.x, loc);
    // offsets of this thread's factors in a record's table
    const int o_a = loc[0];                                  // d = 2: rows; d = 3: i
    const int o_b = tileT<D>(0) + loc[1];                    // d = 2: columns; d = 3: j
    const int o_c = D == 3 ? tileT<D>(0) + tileT<D>(1) + loc[2] : 0;  // d = 3: k
    for (int s0 = 0; s0 < nrec; s0 += kS) {
        const int ns = min(kS, nrec - s0);
        // factor tables of records s0 .. s0 + ns - 1 (zero outside the window):
        // a thread fills 4 consecutive grid lines of one record and dimension
        // (tile extents are multiples of 4), the first by ex2 and one sincos,
        // the next three by the exact recurrences of the Gaussian ratio
        // (rho_{k+1} = rho_k e^{-h^2/eps}) and the phase rotation e^{2 pi i nu}
        for (int e4 = threadIdx.x; e4 < ns * (kT / 4); e4 += kThreads) {
            const int e = 4 * e4;
            const int jr = s0 + e / kT;
            int qd = e % kT, l = 0;
#pragma unroll
            for (int j = 0; j < D - 1; ++j)
                if (l == j && qd >= tileT<D>(j)) {
                    qd -= tileT<D>(j);
                    l = j + 1;
                }
            const RecF<D> &R = *reinterpret_cast<const RecF<D> *>(&srec[jr * kWords]);
            const float kf = (float)(t[l] * tileT<D>(l) + qd) - R.mlo[l];
            const float wl = R.wlen[l];
            float4 out01 = make_float4(0.f, 0.f, 0.f, 0.f), out23 = out01;
            if (kf + 3.f >= 0.f && kf < wl) {  // some of the four lines lie in the window
                const float dx = fmaf(kf, P.hf[l], R.delta[l]);
                float ex = dx * dx * P.ce;
                float fr = kf * R.nuhi[l];
                fr -= rint_fast(fr);
                float tau = fmaf(kf, R.nulo[l], fr);
                if (l == 0) {
                    ex += R.la;
                    tau += R.tau0;
                }
                tau -= rint_fast(tau);
                float sn, cs;
                __sincosf(6.283185307179586f * tau, &sn, &cs);
                const float ga = ex2_approx(ex);
                float fr0 = ga * cs, fi0 = ga * sn;
                float rs_, rc_;
                __sincosf(6.283185307179586f * (R.nuhi[l] + R.nulo[l]), &rs_, &rc_);
                float rho = ex2_approx(P.ce * P.hf[l] * fmaf(2.f, dx, P.hf[l]));
                float v[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool in = kf + (float)i >= 0.f && kf + (float)i < wl;
                    v[2 * i] = in ? fr0 : 0.f;
                    v[2 * i + 1] = in ? fi0 : 0.f;
                    if (i < 3) {
                        const float pr = rc_ * rho, pi = rs_ * rho;
                        const float nr = fr0 * pr - fi0 * pi;
                        fi0 = fr0 * pi + fi0 * pr;
                        fr0 = nr;
                        rho *= P.q_dim[l];
                    }
                }
                out01 = make_float4(v[0], v[1], v[2], v[3]);
                out23 = make_float4(v[4], v[5], v[6], v[7]);
            }
            *reinterpret_cast<float4 *>(&sfac[e]) = out01;
            *reinterpret_cast<float4 *>(&sfac[e + 2]) = out23;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < ns; ++jj) {
            const float2 *F = sfac + jj * kT;
            float ar[2], ai[2];  // factors of the second-to-last dimension (times the outer one for d = 3)
            float br[2], bi[2];  // factors of the last dimension
            if (D == 2) {
                const float4 a = *reinterpret_cast<const float4 *>(F + o_a);
                const float4 b = *reinterpret_cast<const float4 *>(F + o_b);
                ar[0] = a.x; ai[0] = a.y; ar[1] = a.z; ai[1] = a.w;
                br[0] = b.x; bi[0] = b.y; br[1] = b.z; bi[1] = b.w;
            } else {
                const float2 p = F[o_a];
                const float4 a = *reinterpret_cast<const float4 *>(F + o_b);
                const float4 b = *reinterpret_cast<const float4 *>(F + o_c);
                ar[0] = p.x * a.x - p.y * a.y; ai[0] = p.x * a.y + p.y * a.x;
                ar[1] = p.x * a.z - p.y * a.w; ai[1] = p.x * a.w + p.y * a.z;
                br[0] = b.x; bi[0] = b.y; br[1] = b.z; bi[1] = b.w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int ia = r >> 1, ib = r & 1;
                accf[r][0] = fmaf(ar[ia], br[ib], fmaf(-ai[ia], bi[ib], accf[r][0]));
                accf[r][1] = fmaf(ar[ia], bi[ib], fmaf(ai[ia], br[ib], accf[r][1]));
            }
        }
        __syncthreads();
    }
}

// One (output tile, packet slice) work item of the direct sum, executed by the
// whole CTA; shared by the one-request kernel and the batched persistent kernel.
template <int D, bool FP64>
__device__ __forceinline__ void direct_tile(const void *__restrict__ recs_v, const int64_t *__restrict__ off,
                                            const DirectParams &P, void *__restrict__ u_v, const int tile,
                                            const int split, const int nsplit) {
    using Rec = typename std::conditional<FP64, RecD<D>, RecF<D>>::type;
    constexpr int kWords = sizeof(Rec) / 4;
    __shared__ __align__(16) int srec[kThreads * kWords];
    // record offsets fit 32 bits (at most 2^31 packets per call)
    __shared__ uint32_t seg_start[kMaxSeg];
    __shared__ uint32_t seg_cum[kMaxSeg + 1];
    __shared__ int nseg_s;

    const GridDev &g = P.g;
    const Rec *recs = reinterpret_cast<const Rec *>(recs_v);
    int t[D];
    {
        int rem = tile;
#pragma unroll
        for (int l = D - 1; l >= 0; --l) {
            t[l] = rem % g.nt[l];
            rem /= g.nt[l];
        }
    }
    // home-tile box -> segments (rows along the last dimension)
    if (threadIdx.x == 0) {
        int lo[D], cnt[D];
        int rows = 1;
#pragma unroll
        for (int l = 0; l < D; ++l) {
            lo[l] = max(0, t[l] - g.K[l]);
            cnt[l] = t[l] - lo[l] + 1;
            if (l < D - 1) rows *= cnt[l];
        }
        int ns = 0;
        int64_t cum = 0;
        for (int r = 0; r < rows && ns < kMaxSeg; ++r) {
            int h[D];
            int rem = r;
#pragma unroll
            for (int l = D - 2; l >= 0; --l) {
                h[l] = lo[l] + rem % cnt[l];
                rem /= cnt[l];
            }
            h[D - 1] = lo[D - 1];
            const int first = tile_linear<D>(g, h);
            const int last = first + cnt[D - 1] - 1;
            const int64_t a0 = off[first], a1 = off[last + 1];
            if (a1 > a0) {
                seg_start[ns] = (uint32_t)a0;
                seg_cum[ns] = (uint32_t)cum;
                cum += a1 - a0;
                ++ns;
            }
        }
        seg_cum[ns] = (uint32_t)cum;
        nseg_s = ns;
    }
    __syncthreads();
    const int nseg = nseg_s;
    const int64_t L = (int64_t)seg_cum[nseg];

    // this thread's points: kTpt consecutive points along the last dimension
    // (FP64 and d = 1), or the 2 x 2 block of separable_local (FP32, d >= 2)
    constexpr int kLane = tileT<D>(D - 1) / kTpt;  // threads along the last dimension
    int mi[kTpt][D];
    bool valid[kTpt];
    int64_t lin_out[kTpt];
    {
        int base[D];
        if constexpr (!FP64 && D >= 2) {
            int loc[D];
            separable_local<D>(threadIdx.x, loc);
#pragma unroll
            for (int l = 0; l < D; ++l) base[l] = t[l] * tileT<D>(l) + loc[l];
        } else {
            int i = threadIdx.x / kLane;
            base[D - 1] = t[D - 1] * tileT<D>(D - 1) + (threadIdx.x % kLane) * kTpt;
#pragma unroll
            for (int l = D - 2; l >= 0; --l) {
                base[l] = t[l] * tileT<D>(l) + i % tileT<D>(l);
                i /= tileT<D>(l);
            }
        }
#pragma unroll
        for (int r = 0; r < kTpt; ++r) {
            bool ok = true;
            int64_t lin = 0;
#pragma unroll
            for (int l = 0; l < D; ++l) {
                int off = 0;
                if (!FP64 && D >= 2)
                    off = l == D - 2 ? (r >> 1) : (l == D - 1 ? (r & 1) : 0);
                else
                    off = l == D - 1 ? r : 0;
                mi[r][l] = base[l] + off;
                ok = ok && mi[r][l] < g.n[l];
                lin = lin * g.n[l] + mi[r][l];
            }
            valid[r] = ok;
            lin_out[r] = lin;
        }
    }
    float mf[D];  // first point (FP32 path)
#pragma unroll
    for (int l = 0; l < D; ++l) mf[l] = (float)mi[0][l];
    double xd[kTpt][D];
    if (FP64) {
#pragma unroll
        for (int r = 0; r < kTpt; ++r)
#pragma unroll
            for (int l = 0; l < D; ++l) xd[r][l] = grid_x(g.lo[l], g.h[l], mi[r][l]);
    }
    __shared__ float2 srot[(!FP64 && D == 1) ? kThreads : 1];  // FP32, 1-D: e^{2 pi i nu} per staged record
    __shared__ __align__(16) float2 sfac[(!FP64 && D >= 2) ? kSub<D>() * kSumT<D>() : 2];  // FP32, d >= 2

    float accf[kTpt][2];
    double accd[kTpt][2];
#pragma unroll
    for (int r = 0; r < kTpt; ++r) {
        accf[r][0] = accf[r][1] = 0.f;
        accd[r][0] = accd[r][1] = 0.0;
    }

    const int64_t nchunks = (L + kThreads - 1) / kThreads;
    for (int64_t c = split; c < nchunks; c += nsplit) {
        const int64_t v = c * kThreads + threadIdx.x;
        if (v < L) {
            // segment holding virtual index v
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)seg_cum[mid] <= v) lo = mid;
                else hi = mid - 1;
            }
            const int64_t idx = (int64_t)seg_start[lo] + (v - (int64_t)seg_cum[lo]);
            const int *src = reinterpret_cast<const int *>(recs + idx);
#pragma unroll
            for (int w = 0; w < kWords; w += 4)
                *reinterpret_cast<int4 *>(&srec[threadIdx.x * kWords + w]) =
                    *reinterpret_cast<const int4 *>(src + w);
            if (!FP64 && D == 1) {  // the rotation by one grid step along the last dimension
                const RecF<D> &mine = *reinterpret_cast<const RecF<D> *>(&srec[threadIdx.x * kWords]);
                float sn, cs;
                sincospif(2.f * (mine.nuhi[D - 1] + mine.nulo[D - 1]), &sn, &cs);
                srot[threadIdx.x] = make_float2(cs, sn);
            }
        }
        __syncthreads();
        const int64_t left = L - c * kThreads;
        const int nrec = left < kThreads ? (int)left : kThreads;
        if constexpr (!FP64 && D >= 2)
            separable_chunk<D>(srec, nrec, P, t, sfac, accf);
        else
        for (int jr = 0; jr < nrec; ++jr) {
            const Rec &R = *reinterpret_cast<const Rec *>(&srec[jr * kWords]);
            if (FP64) {
                const RecD<D> &Rd = reinterpret_cast<const RecD<D> &>(R);
#pragma unroll
                for (int r = 0; r < kTpt; ++r) {
                    bool in = valid[r];
#pragma unroll
                    for (int l = 0; l < D; ++l) {
                        const int k = mi[r][l] - Rd.mlo[l];
                        in = in && (unsigned)k < (unsigned)Rd.wlen[l];
                    }
                    if (!in) continue;
                    double phase = Rd.S, g2 = 0.0;
#pragma unroll
                    for (int l = 0; l < D; ++l) {
                        const double dx = xd[r][l] - Rd.Q[l];
                        phase += Rd.P[l] * dx;
                        g2 += dx * dx;
                    }
                    double sn, cs;
                    sincos(phase * P.inv_eps, &sn, &cs);
                    const double ga = exp(g2 * P.neg_half_inv_eps);
                    const double gr = ga * cs, gi = ga * sn;
                    accd[r][0] += Rd.ar * gr - Rd.ai * gi;
                    accd[r][1] += Rd.ar * gi + Rd.ai * gr;
                }
            } else {
                // the first point evaluated in full, the next kTpt - 1 along
                // the last dimension by the exact recurrences of the Gaussian
                // (ratio rho, itself multiplied by e^{-h^2/eps} per step) and of
                // the phase (rotation by e^{2 pi i nu})
                const RecF<D> &Rf = reinterpret_cast<const RecF<D> &>(R);
                float kk[D];
                bool in = true;
#pragma unroll
                for (int l = 0; l < D - 1; ++l) {
                    kk[l] = mf[l] - Rf.mlo[l];
                    in = in && kk[l] >= 0.f && kk[l] < Rf.wlen[l];
                }
                kk[D - 1] = mf[D - 1] - Rf.mlo[D - 1];
                const float wl = Rf.wlen[D - 1];
                in = in && kk[D - 1] > -(float)kTpt && kk[D - 1] < wl;
                if (!in) continue;
                float e = 0.f, tau = Rf.tau0, dxl = 0.f;
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    const float kf = kk[l];
                    const float dx = fmaf(kf, P.hf[l], Rf.delta[l]);
                    e = fmaf(dx, dx, e);
                    float f = kf * Rf.nuhi[l];
                    f -= rint_fast(f);
                    tau += fmaf(kf, Rf.nulo[l], f);
                    dxl = dx;
                }
                tau -= rint_fast(tau);
                float sn, cs;
                __sincosf(6.283185307179586f * tau, &sn, &cs);
                const float ga = ex2_approx(fmaf(e, P.ce, Rf.la));
                float vr = ga * cs, vi = ga * sn;
                const float rho = ex2_approx(P.ce_h * fmaf(2.f, dxl, P.hf[D - 1]));
                const float2 rot = srot[jr];
                float wr = rho * rot.x, wi = rho * rot.y;
#pragma unroll
                for (int r = 0; r < kTpt; ++r) {
                    const float k = kk[D - 1] + (float)r;
                    if (k >= 0.f && k < wl) {
                        accf[r][0] += vr;
                        accf[r][1] += vi;
                    }
                    if (r + 1 < kTpt) {
                        const float nr = vr * wr - vi * wi;
                        vi = vr * wi + vi * wr;
                        vr = nr;
                        wr *= P.q_last;
                        wi *= P.q_last;
                    }
                }
            }
        }
        if (!FP64) {  // fold this chunk's FP32 partial sums into the FP64 totals
#pragma unroll
            for (int r = 0; r < kTpt; ++r) {
                accd[r][0] += (double)accf[r][0];
                accd[r][1] += (double)accf[r][1];
                accf[r][0] = accf[r][1] = 0.f;
            }
        }
        __syncthreads();
    }
    if (L == 0) return;
#pragma unroll
    for (int r = 0; r < kTpt; ++r) {
        if (!valid[r]) continue;
        if (FP64)
            atomic_add_c(reinterpret_cast<double2 *>(u_v) + lin_out[r], accd[r][0], accd[r][1]);
        else
            atomic_add_c(reinterpret_cast<float2 *>(u_v) + lin_out[r], (float)accd[r][0], (float)accd[r][1]);
    }
}

template <int D, bool FP64>
__global__ void __launch_bounds__(kThreads) direct_kernel(const void *__restrict__ recs_v,
                                                          const int64_t *__restrict__ off,
                                                          DirectParams P, void *__restrict__ u_v) {
    direct_tile<D, FP64>(recs_v, off, P, u_v, blockIdx.x, blockIdx.y, P.splits);
}

// Records in the list of every tile (the home-tile box of direct_tile).
template <int D>
__global__ void tile_load_kernel(const int64_t *__restrict__ off, GridDev g, uint32_t *__restrict__ load) {
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile >= g.ntiles) return;
    int t[D];
    int rem = tile;
#pragma unroll
    for (int l = D - 1; l >= 0; --l) {
        t[l] = rem % g.nt[l];
        rem /= g.nt[l];
    }
    int lo[D], cnt[D];
    int rows = 1;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        lo[l] = max(0, t[l] - g.K[l]);
        cnt[l] = t[l] - lo[l] + 1;
        if (l < D - 1) rows *= cnt[l];
    }
    int64_t sum = 0;
    for (int r = 0; r < rows; ++r) {
        int h[D];
        int rr = r;
#pragma unroll
        for (int l = D - 2; l >= 0; --l) {
            h[l] = lo[l] + rr % cnt[l];
            rr /= cnt[l];
        }
        h[D - 1] = lo[D - 1];
        const int first = tile_linear<D>(g, h);
        sum += off[first + cnt[D - 1]] - off[first];
    }
    load[tile] = (uint32_t)sum;
}

// Work items of the balanced launch (one CTA): tile t gets s_t slices in
// proportion to its chunks of 256 records (1 <= s_t <= min(64, chunks)), and
// the items are listed heaviest tiles first (tiles bucketed by the highest bit
// of their record count), so that the persistent kernel finishes with light
// items.  item = (tile, split | nsplit << 8).
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads) plan_items_kernel(const uint32_t *__restrict__ load, int ntiles,
                                                                   int target, int *__restrict__ rank_tile,
                                                                   int *__restrict__ rank_splits,
                                                                   int2 *__restrict__ items,
                                                                   int *__restrict__ n_items) {
    __shared__ unsigned long long s_chunks;
    __shared__ int bucket_cnt[33], bucket_off[33];
    __shared__ int part[kPlanThreads];
    __shared__ int carry;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_chunks = 0;
        carry = 0;
    }
    if (tid < 33) bucket_cnt[tid] = 0;
    __syncthreads();
    unsigned long long mine = 0;
    for (int t = tid; t < ntiles; t += kPlanThreads) {
        const uint32_t L = load[t];
        mine += (L + 255u) / 256u;
        const int b = L == 0 ? 32 : 31 - __clz((int)L);  // empty tiles last
        atomicAdd(&bucket_cnt[b], 1);
    }
    atomicAdd(&s_chunks, mine);
    __syncthreads();
    if (tid == 0) {  // buckets in descending order of size, empty tiles last
        int acc = 0;
        for (int b = 31; b >= 0; --b) {
            bucket_off[b] = acc;
            acc += bucket_cnt[b];
        }
        bucket_off[32] = acc;
    }
    __syncthreads();
    const double total = (double)(s_chunks > 0 ? s_chunks : 1);
    for (int t = tid; t < ntiles; t += kPlanThreads) {
        const uint32_t L = load[t];
        const int b = L == 0 ? 32 : 31 - __clz((int)L);
        const int r = atomicAdd(&bucket_off[b], 1);
        const int chunks = (int)((L + 255u) / 256u);
        int sp = 0;
        if (chunks > 0) {
            sp = (int)ceil((double)chunks * (double)target / total);
            sp = max(1, min(sp, min(64, chunks)));
        }
        rank_tile[r] = t;
        rank_splits[r] = sp;
    }
    __syncthreads();
    // exclusive scan of the slice counts in rank order, items written as we go
    for (int base = 0; base < ntiles; base += kPlanThreads) {
        const int i = base + tid;
        const int v = i < ntiles ? rank_splits[i] : 0;
        part[tid] = v;
        __syncthreads();
        for (int st = 1; st < kPlanThreads; st <<= 1) {
            const int add = tid >= st ? part[tid - st] : 0;
            __syncthreads();
            part[tid] += add;
            __syncthreads();
        }
        if (i < ntiles) {
            const int start = carry + part[tid] - v;
            const int tile = rank_tile[i];
            for (int k = 0; k < v; ++k) items[start + k] = make_int2(tile, k | (v << 8));
        }
        __syncthreads();
        if (tid == kPlanThreads - 1) carry += part[kPlanThreads - 1];
        __syncthreads();
    }
    if (tid == 0) *n_items = carry;
}

// Items plan_items_kernel can write: a tile's slice count is at most
// max(1, ceil(chunks_t * target / chunks)) <= chunks_t * target / chunks + 1,
// so all tiles together hold at most target + tiles (64 of margin for the
// rounding of the quotient).
inline size_t plan_items_capacity(int ntiles, int target) {
    return std::min<size_t>((size_t)64 * ntiles, (size_t)ntiles + (size_t)target + 64);
}

// Balanced direct sum: persistent CTAs pull the planned items in order.  With
// a yield word, the CTAs from index keep on stop before pulling another item
// while the word is > 0; the remaining CTAs finish every item.
template <int D, bool FP64>
__global__ void __launch_bounds__(kThreads) direct_items_kernel(const void *__restrict__ recs_v,
                                                                const int64_t *__restrict__ off, DirectParams P,
                                                                void *__restrict__ u_v,
                                                                const int2 *__restrict__ items,
                                                                const int *__restrict__ n_items,
                                                                unsigned long long *__restrict__ counter,
                                                                const volatile int *yield, int keep) {
    __shared__ long long s_item;
    const long long total = *n_items;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const bool stop = yield != nullptr && (int)blockIdx.x >= keep && *yield > 0;
            s_item = stop ? total : (long long)atomicAdd(counter, 1ULL);
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int2 it = items[item];
        direct_tile<D, FP64>(recs_v, off, P, u_v, it.x, it.y & 0xff, it.y >> 8);
    }
}

// Batched direct sum: one persistent launch over the work items of up to
// kBatchMax requests.  Item i belongs to the request r with
// item_start[r] <= i < item_start[r+1]; within it, tile = j / splits and
// slice = j % splits.  CTAs pull items through one atomic counter.
constexpr int kBatchMax = 64;

struct BatchReq {
    const void *recs;
    const int64_t *off;
    void *u;
    DirectParams P;
    const int2 *items;  // balanced batches (d >= 2): the request's planned items
};

struct BatchParams {
    int n;
    int64_t item_start[kBatchMax + 1];
    BatchReq req[kBatchMax];
};

// kernel parameters may take up to 32764 bytes (sm_70 and later, CUDA 12.1+)
static_assert(sizeof(BatchParams) <= 32000, "batch parameters exceed the kernel parameter space");

template <int D, bool FP64>
__global__ void __launch_bounds__(kThreads) direct_batch_kernel(const __grid_constant__ BatchParams B,
                                                                unsigned long long *__restrict__ counter) {
    __shared__ long long s_item;
    const long long total = B.item_start[B.n];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int lo = 0, hi = B.n - 1;  // request holding this item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.item_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchReq &R = B.req[lo];
        const long long j = item - B.item_start[lo];
        direct_tile<D, FP64>(R.recs, R.off, R.P, R.u, (int)(j / R.P.splits), (int)(j % R.P.splits), R.P.splits);
    }
}

// Balanced batch (d >= 2): request r's items, planned on the device like the
// single call's, occupy [start[r], start[r+1]) of one list whose prefix
// start[] is computed on the device from the per-request item counts.
__global__ void batch_item_start_kernel(const int *__restrict__ nitems, int n, int *__restrict__ start) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < n; ++r) {
            start[r] = acc;
            acc += nitems[r];
        }
        start[n] = acc;
    }
}

template <int D, bool FP64>
__global__ void __launch_bounds__(kThreads) direct_batch_items_kernel(const __grid_constant__ BatchParams B,
                                                                      const int *__restrict__ start,
                                                                      unsigned long long *__restrict__ counter) {
    __shared__ int s_start[kBatchMax + 1];
    __shared__ long long s_item;
    for (int r = threadIdx.x; r <= B.n; r += blockDim.x) s_start[r] = start[r];
    __syncthreads();
    const long long total = s_start[B.n];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int lo = 0, hi = B.n - 1;  // request holding this item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchReq &R = B.req[lo];
        const int2 it = R.items[item - s_start[lo]];
        direct_tile<D, FP64>(R.recs, R.off, R.P, R.u, it.x, it.y & 0xff, it.y >> 8);
    }
}

#include "direct_tc.cuh"

// Zeroes the output and bins one request's packets; fills the parameters of
// its main kernel (pr->empty when nothing remains to sum).
struct Prepared {
    const void *recs = nullptr;
    const int64_t *off = nullptr;
    DirectParams P{};
    int ntiles = 0;
    bool empty = true;
};

template <int D>
fgr_status prepare(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st, Scratch &scratch,
                   Prepared *pr) {
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    const Mesh &M = ctx->mesh;
    GridDev g{};
    int ntiles = 1;
    int wmax_all = 1;
    for (int l = 0; l < D; ++l) {
        g.n[l] = ctx->grid.n[l];
        g.lo[l] = ctx->grid.lo[l];
        g.h[l] = ctx->grid.h[l];
        g.nt[l] = (int)((g.n[l] + tileT<D>(l) - 1) / tileT<D>(l));
        const int64_t wmax = std::min<int64_t>((int64_t)std::floor(2.0 * M.rs / g.h[l]) + 2, g.n[l]);
        wmax_all = std::max<int>(wmax_all, (int)wmax);
        g.K[l] = (int)((wmax - 1 + tileT<D>(l) - 1) / tileT<D>(l));
        g.K[l] = std::min(g.K[l], g.nt[l] - 1);
        ntiles *= g.nt[l];
    }
    g.ntiles = ntiles;
    int64_t rows = 1;
    for (int l = 0; l < D - 1; ++l) rows *= g.K[l] + 1;
    if (rows > kMaxSeg) {
        set_error("direct: window of %d points is too wide for the %d-D tiling", wmax_all, D);
        return FGR_E_INVALID;
    }
    const size_t out_bytes = elem_bytes(ctx->opt.precision) * (size_t)ctx->grid.total;
    FGR_CUDA_TRY(cudaMemsetAsync(u_dev, 0, out_bytes, st));
    pr->empty = true;
    const int64_t m = pk.m;
    if (m == 0) return FGR_OK;
    int *home = (int *)scratch.get(sizeof(int) * m);
    int *counts = (int *)scratch.get(sizeof(int) * 2 * (size_t)ntiles);
    int64_t *off = (int64_t *)scratch.get(sizeof(int64_t) * ((size_t)ntiles + 1));
    const size_t rec_bytes = fp64 ? sizeof(RecD<D>) : sizeof(RecF<D>);
    void *recs = scratch.get(rec_bytes * (size_t)m);
    if (!home || !counts || !off || !recs) return FGR_E_NOMEM;
    int *cursor = counts + ntiles;
    FGR_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * 2 * (size_t)ntiles, st));
    const unsigned pb = (unsigned)((m + 255) / 256);
    bin_count_kernel<D><<<pb, 256, 0, st>>>(pk.q, m, g, M.rs, home, counts);
    scan_kernel<<<1, 1024, 0, st>>>(counts, off, ntiles);
    RecParams rp;
    rp.rs = M.rs;
    rp.eps = M.eps;
    rp.inv_eps = 1.0 / M.eps;
    rp.pref = M.pref;
    int lbits = 1;
    while ((1 << lbits) < wmax_all + 1) ++lbits;
    rp.two_pow_b = std::ldexp(1.0, std::max(1, 24 - lbits));
    rp.inv_two_pow_b = 1.0 / rp.two_pow_b;
    if (fp64)
        bin_scatter_kernel<D, true><<<pb, 256, 0, st>>>(pk.q, pk.p, pk.s, pk.a, m, g, rp, home, off, cursor, recs);
    else
        bin_scatter_kernel<D, false><<<pb, 256, 0, st>>>(pk.q, pk.p, pk.s, pk.a, m, g, rp, home, off, cursor, recs);
    FGR_CUDA_TRY(cudaGetLastError());

    DirectParams &P = pr->P;
    P = DirectParams{};
    P.g = g;
    for (int l = 0; l < D; ++l) P.hf[l] = (float)g.h[l];
    P.ce = (float)(-1.4426950408889634 / (2.0 * M.eps));
    P.ce_h = (float)(-1.4426950408889634 / (2.0 * M.eps) * g.h[D - 1]);
    P.q_last = (float)std::exp(-g.h[D - 1] * g.h[D - 1] / M.eps);
    for (int l = 0; l < D; ++l) P.q_dim[l] = (float)std::exp(-g.h[l] * g.h[l] / M.eps);
    for (int l = 0; l < D; ++l) P.q8[l] = (float)std::exp(-64.0 * g.h[l] * g.h[l] / M.eps);
    P.inv_eps = 1.0 / M.eps;
    P.neg_half_inv_eps = -0.5 / M.eps;
    const int target = ctx->num_sms * ctx->tune.direct_ctas_per_sm;
    P.splits = std::max(1, std::min(64, (target + ntiles - 1) / ntiles));
    pr->recs = recs;
    pr->off = off;
    pr->ntiles = ntiles;
    pr->empty = false;
    return FGR_OK;
}

// Whether the tensor-core kernel can take a grid: a super tile's list is at
// most kSegMax runs of home tiles (windows of up to about 8,000 lines of
// dimension 0 in 2-D, about 110 lines of dimensions 0 and 1 in 3-D); wider
// windows go to the CUDA-core kernel.
template <int D>
bool tc_fits(const GridDev &g, int64_t *nst_out) {
    int64_t runs = 1, nst = 1;
    for (int l = 0; l < D; ++l) {
        const int span = tc::tc_span<D>(l);
        nst *= (g.nt[l] + span - 1) / span;
        if (l < D - 1) runs *= (int64_t)std::min(g.K[l] + span, g.nt[l]);
    }
    if (nst_out) *nst_out = nst;
    return runs <= tc::kSegMax && nst <= ((int64_t)1 << 30);
}

// Tensor-core direct sum (FP32, d = 2, 3): loads of the super tiles, items
// heaviest first, one persistent CTA per SM.
template <int D>
fgr_status launch_tc(fgr_ctx *ctx, const Prepared &pr, void *u_dev, cudaStream_t st, Scratch &scratch) {
    const GridDev &g = pr.P.g;
    int64_t nst = 0;
    if (!tc_fits<D>(g, &nst)) {
        set_error("direct: window too wide for the tensor-core tiling");
        return FGR_E_INTERNAL;
    }
    auto *load = (uint32_t *)scratch.get(sizeof(uint32_t) * (size_t)nst);
    auto *rank = (int *)scratch.get(sizeof(int) * 2 * (size_t)nst);
    const int target = ctx->num_sms * ctx->tune.direct_ctas_per_sm;
    auto *items = (int2 *)scratch.get(sizeof(int2) * plan_items_capacity((int)nst, target));
    auto *cnt = (unsigned long long *)scratch.get(2 * sizeof(unsigned long long));
    if (!load || !rank || !items || !cnt) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    tc_tile_load_kernel<D><<<(unsigned)((nst + 255) / 256), 256, 0, st>>>(pr.off, g, (int)nst, load);
    plan_items_kernel<<<1, kPlanThreads, 0, st>>>(load, (int)nst, target, rank, rank + nst, items,
                                                  reinterpret_cast<int *>(cnt + 1));
    static thread_local int attr_device = -1;
    if (attr_device != ctx->device) {
        FGR_CUDA_TRY(cudaFuncSetAttribute(direct_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc::dyn_smem<2>()));
        FGR_CUDA_TRY(cudaFuncSetAttribute(direct_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc::dyn_smem<3>()));
        attr_device = ctx->device;
    }
    const unsigned ctas = (unsigned)ctx->num_sms;
    // with a yield word (a large request in the server), the CTAs of the
    // second half of the SMs stop between items while it is set: one CTA
    // fills an SM's registers, so that is how small requests get SMs
    const int keep = ctx->yield_flag ? std::max(1, (int)ctas / 2) : (int)ctas;
    direct_tc_kernel<D><<<ctas, tc::kThreadsTc, tc::dyn_smem<D>(), st>>>(
        reinterpret_cast<const RecF<D> *>(pr.recs), pr.off, pr.P, reinterpret_cast<float2 *>(u_dev), items,
        reinterpret_cast<int *>(cnt + 1), cnt, ctx->yield_flag, keep, ctx->dev_err);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

template <int D>
fgr_status launch(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st, Scratch &scratch) {
    const bool fp64 = ctx->opt.precision == FGR_FP64;
    StageTimer timer(ctx, st);
    Prepared pr;
    fgr_status r = prepare<D>(ctx, pk, u_dev, st, scratch, &pr);
    if (r != FGR_OK) return r;
    timer.mark(&ctx->timing.last.prep_ms);
    if (pr.empty) {
        timer.finish();
        return FGR_OK;
    }
    if (D == 1) {
        // 1-D: a few long tiles of similar load; one CTA per (tile, slice)
        dim3 grid((unsigned)pr.ntiles, (unsigned)pr.P.splits);
        if (fp64)
            direct_kernel<D, true><<<grid, kThreads, 0, st>>>(pr.recs, pr.off, pr.P, u_dev);
        else
            direct_kernel<D, false><<<grid, kThreads, 0, st>>>(pr.recs, pr.off, pr.P, u_dev);
        FGR_CUDA_TRY(cudaGetLastError());
        timer.mark(&ctx->timing.last.direct_ms);
        ctx->timing.last.launches = 4;
        timer.finish();
        return FGR_OK;
    }
    if (D >= 2 && !fp64 && !(ctx->opt.flags & FGR_FLAG_DIRECT_FMA) && tc_fits<D == 3 ? 3 : 2>(pr.P.g, nullptr)) {
        fgr_status rt = launch_tc<D == 3 ? 3 : 2>(ctx, pr, u_dev, st, scratch);
        if (rt != FGR_OK) return rt;
        timer.mark(&ctx->timing.last.direct_ms);
        ctx->timing.last.launches = 6;
        timer.finish();
        return FGR_OK;
    }
    // d >= 2, balanced launch: per-tile loads (the dense middle of a wave packet
    // set holds many times the records of its edges), items heaviest first,
    // persistent CTAs
    const int ntiles = pr.ntiles;
    auto *load = (uint32_t *)scratch.get(sizeof(uint32_t) * (size_t)ntiles);
    auto *rank = (int *)scratch.get(sizeof(int) * 2 * (size_t)ntiles);
    const int target = ctx->num_sms * ctx->tune.direct_ctas_per_sm;
    auto *items = (int2 *)scratch.get(sizeof(int2) * plan_items_capacity(ntiles, target));
    auto *cnt = (unsigned long long *)scratch.get(2 * sizeof(unsigned long long));
    if (!load || !rank || !items || !cnt) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    tile_load_kernel<D><<<(unsigned)((ntiles + 255) / 256), 256, 0, st>>>(pr.off, pr.P.g, load);
    plan_items_kernel<<<1, kPlanThreads, 0, st>>>(load, ntiles, target, rank, rank + ntiles, items,
                                                  reinterpret_cast<int *>(cnt + 1));
    int per_sm = 1;
    if (fp64)
        FGR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_items_kernel<D, true>, kThreads, 0));
    else
        FGR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_items_kernel<D, false>, kThreads, 0));
    const unsigned ctas = (unsigned)(ctx->num_sms * std::max(1, per_sm));
    const int keep = std::max(ctx->num_sms, (int)ctas - ctx->num_sms);  // one slot per SM can be given up
    if (fp64)
        direct_items_kernel<D, true><<<ctas, kThreads, 0, st>>>(pr.recs, pr.off, pr.P, u_dev, items,
                                                                reinterpret_cast<int *>(cnt + 1), cnt,
                                                                ctx->yield_flag, keep);
    else
        direct_items_kernel<D, false><<<ctas, kThreads, 0, st>>>(pr.recs, pr.off, pr.P, u_dev, items,
                                                                 reinterpret_cast<int *>(cnt + 1), cnt,
                                                                 ctx->yield_flag, keep);
    FGR_CUDA_TRY(cudaGetLastError());
    timer.mark(&ctx->timing.last.direct_ms);
    ctx->timing.last.launches = 6;
    timer.finish();
    return FGR_OK;
}

// Batched direct sum of n requests of the same dimension and precision: the
// binning of each request, then one persistent launch over all work items.
template <int D>
fgr_status launch_batch(int n, fgr_ctx *const *ctxs, const PacketsDev *pks, void *const *us, cudaStream_t st,
                        Scratch **scratch, Scratch &shared) {
    const bool fp64 = ctxs[0]->opt.precision == FGR_FP64;
    BatchParams B;
    memset(&B, 0, sizeof(B));
    // d >= 2: largest requests first, each cut into items in proportion to
    // its share of the packets (planned on the device, heaviest tiles first)
    int order[kBatchMax];
    for (int r = 0; r < n; ++r) order[r] = r;
    int64_t msum = 0;
    for (int r = 0; r < n; ++r) msum += pks[r].m;
    if (D >= 2)
        std::stable_sort(order, order + n, [&](int x, int y) { return pks[x].m > pks[y].m; });
    int *nitems = nullptr;
    if (D >= 2) {
        nitems = (int *)shared.get(sizeof(int) * (2 * kBatchMax + 2));
        if (!nitems) return FGR_E_NOMEM;
        FGR_CUDA_TRY(cudaMemsetAsync(nitems, 0, sizeof(int) * (2 * kBatchMax + 2), st));
    }
    int64_t total = 0;
    for (int k = 0; k < n; ++k) {
        const int r = order[k];
        Prepared pr;
        fgr_status rc = prepare<D>(ctxs[r], pks[r], us[r], st, *scratch[r], &pr);
        if (rc != FGR_OK) return rc;
        if (pr.empty) continue;
        B.req[B.n] = BatchReq{pr.recs, pr.off, us[r], pr.P, nullptr};
        if (D >= 2) {
            const int ntiles = pr.ntiles;
            auto *load = (uint32_t *)scratch[r]->get(sizeof(uint32_t) * (size_t)ntiles);
            auto *rank = (int *)scratch[r]->get(sizeof(int) * 2 * (size_t)ntiles);
            const int64_t all = (int64_t)ctxs[0]->num_sms * ctxs[0]->tune.direct_ctas_per_sm;
            const int target = (int)std::max<int64_t>(1, all * pks[r].m / std::max<int64_t>(msum, 1));
            auto *items = (int2 *)scratch[r]->get(sizeof(int2) * plan_items_capacity(ntiles, target));
            if (!load || !rank || !items) return FGR_E_NOMEM;
            tile_load_kernel<D><<<(unsigned)((ntiles + 255) / 256), 256, 0, st>>>(pr.off, pr.P.g, load);
            plan_items_kernel<<<1, kPlanThreads, 0, st>>>(load, ntiles, target, rank, rank + ntiles, items,
                                                          nitems + B.n);
            B.req[B.n].items = items;
        } else {
            B.item_start[B.n] = total;
            total += (int64_t)pr.ntiles * pr.P.splits;
        }
        ++B.n;
    }
    B.item_start[B.n] = total;
    if (B.n == 0) return FGR_OK;
    auto *counter = (unsigned long long *)shared.get(sizeof(unsigned long long));
    if (!counter) return FGR_E_NOMEM;
    FGR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    if (D >= 2) {
        int *start = nitems + kBatchMax;
        batch_item_start_kernel<<<1, 32, 0, st>>>(nitems, B.n, start);
        int per_sm = 1;
        if (fp64)
            FGR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_batch_items_kernel<D, true>,
                                                                       kThreads, 0));
        else
            FGR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_batch_items_kernel<D, false>,
                                                                       kThreads, 0));
        const unsigned ctas = (unsigned)(ctxs[0]->num_sms * std::max(1, per_sm));
        if (fp64)
            direct_batch_items_kernel<D, true><<<ctas, kThreads, 0, st>>>(B, start, counter);
        else
            direct_batch_items_kernel<D, false><<<ctas, kThreads, 0, st>>>(B, start, counter);
        FGR_CUDA_TRY(cudaGetLastError());
        return FGR_OK;
    }
    const int64_t ctas = std::min<int64_t>(total, (int64_t)ctxs[0]->num_sms * 8);
    if (fp64)
        direct_batch_kernel<D, true><<<(unsigned)ctas, kThreads, 0, st>>>(B, counter);
    else
        direct_batch_kernel<D, false><<<(unsigned)ctas, kThreads, 0, st>>>(B, counter);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace

fgr_status run_direct_batch(int n, fgr_ctx *const *ctxs, const PacketsDev *pks, void *const *us, cudaStream_t st,
                            Scratch **scratch, Scratch &shared) {
    switch (ctxs[0]->d) {
    case 1: return launch_batch<1>(n, ctxs, pks, us, st, scratch, shared);
    case 2: return launch_batch<2>(n, ctxs, pks, us, st, scratch, shared);
    default: return launch_batch<3>(n, ctxs, pks, us, st, scratch, shared);
    }
}

fgr_status run_direct(fgr_ctx *ctx, const PacketsDev &pk, void *u_dev, cudaStream_t st, Scratch &scratch) {
    switch (ctx->d) {
    case 1: return launch<1>(ctx, pk, u_dev, st, scratch);
    case 2: return launch<2>(ctx, pk, u_dev, st, scratch);
    default: return launch<3>(ctx, pk, u_dev, st, scratch);
    }
}

}  // namespace fgr
