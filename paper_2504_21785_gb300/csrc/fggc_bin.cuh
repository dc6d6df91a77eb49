// K4 for d = 3 (FP32 path): the scatter of eq. 2.25 with the packets binned
// by the anchor cell (a0, b0) of their outer dimensions.
//
// A packet's contributions to one row of the node array (the last dimension's
// [a][b] plane for fixed outer nodes) are the 2 x 4 neighbours of its inner
// anchor cell, and the outer anchor cell fixes which rows it reaches: n1^(d-1)
// rows, one per outer neighbour.  Packets with the same outer anchor cell reach
// the same rows, so after a counting sort by that cell a CTA takes up to
// kBinT packets of one cell, adds their contributions to each row into a
// private plane in shared memory (the box of their inner neighbours) and then
// adds the plane to W: one 8-byte reduction per touched cell instead of one
// per contribution, issued by consecutive threads to consecutive cells of the
// row.  Cells with fewer packets than BinLaunch::min_count go through the
// per-packet kernel (fggc_coeff.cuh) from a list.
//
// Included by fggc_coeff3.cu.  The kernels are written for d >= 2; the
// library uses them for d = 3, where a packet has 512 contributions.
#pragma once

#include <climits>

#include "fggc_coeff.cuh"

namespace fgr {
namespace {

constexpr int kBinT = 256;         // packets (threads) per binned item
constexpr int kBinCtasPerSm = 3;   // resident binned-scatter CTAs per SM (registers, shared memory)

// Warp-aggregated atomicAdd of sign on ctr[k] by the active lanes (one atomic
// per distinct k); returns the old value plus sign times the lane's rank
// among the lanes with the same k.
__device__ __forceinline__ int aggregated_add(int *ctr, int k, int sign) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1));
    int base = 0;
    if (lane == leader) base = atomicAdd(ctr + k, sign * __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + sign * rank;
}

// Per packet: the key of its outer anchor cell in the key box (-1: the packet
// adds nothing: zero amplitude, or every node of an outer dimension lies
// outside the node box), and the count of packets per key.
template <int D>
__global__ void bin_key_kernel(const double *__restrict__ q, const double *__restrict__ p,
                               const double *__restrict__ a, int64_t m, const Common c, const BinBox bb,
                               int *__restrict__ key, int *__restrict__ count) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    int k = -1;
    double qv[D - 1], pv[D - 1];  // every load first (none waits on the amplitude test)
#pragma unroll
    for (int l = 0; l < D - 1; ++l) {
        qv[l] = q[l * m + j];
        pv[l] = p[l * m + j];
    }
    if (a[j] != 0.0 || a[m + j] != 0.0) {
        int64_t kk = 0;
        bool ok = true;
#pragma unroll
        for (int l = 0; l < D - 1; ++l) {
            const int ia = floor_div_int(qv[l], c.dqv, c.inv_dq) - bb.ka_lo[l];
            const int ib = floor_div_int(pv[l], c.dpv, c.inv_dp) - bb.kb_lo[l];
            ok = ok && (unsigned)ia < (unsigned)bb.KA[l] && (unsigned)ib < (unsigned)bb.KB[l];
            kk = (kk * bb.KA[l] + ia) * bb.KB[l] + ib;
        }
        if (ok) k = (int)kk;
    }
    key[j] = k;
    if (k >= 0) aggregated_add(count, k, 1);
}

// Places every binned packet at its sorted position (offset of its key plus
// a slot) and every packet of a small cell on the loose list.  count[] is
// consumed as the per-key cursor.
__global__ void bin_place_kernel(const int *__restrict__ key, int64_t m, const int2 *__restrict__ off,
                                 int *__restrict__ count, int *__restrict__ sorted, int *__restrict__ loose,
                                 int *__restrict__ nloose) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int k = key[j];
    if (k < 0) return;
    const int2 o = off[k], o1 = off[k + 1];
    if (o1.x > o.x) {  // a binned cell: slots counted down from its size
        const int slot = aggregated_add(count, k, -1) - 1;
        sorted[o.x + slot] = (int)j;
    } else {
        loose[aggregated_add(nloose, 0, 1)] = (int)j;
    }
}

// One item (key, first sorted position, packets) per kBinT packets of every
// binned cell.
__global__ void bin_items_kernel(const int2 *__restrict__ off, int64_t K, int4 *__restrict__ items) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int2 o = off[k], o1 = off[k + 1];
    const int n = o1.x - o.x;
    for (int t = 0; t < o1.y - o.y; ++t)
        items[o.y + t] = make_int4((int)k, o.x + t * kBinT, min(kBinT, n - t * kBinT), 0);
}

// Before the scatter: marks every row of W that the packets of an occupied key
// will reach (the n1^(d-1) outer neighbours of its anchor cell that lie in the
// node box), one thread per key.  The binned and per-packet kernels reach
// exactly these rows, so only they need clearing.
template <int D>
__global__ void bin_mark_rows_kernel(const int *__restrict__ count, const Common c, const BinBox bb,
                                     uint8_t *__restrict__ row_flag) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= bb.K || count[k] == 0) return;
    int oa[D - 1], ob[D - 1];
    int64_t kk = k;
#pragma unroll
    for (int l = D - 2; l >= 0; --l) {
        ob[l] = (int)(kk % bb.KB[l]) + bb.kb_lo[l];
        kk /= bb.KB[l];
        oa[l] = (int)(kk % bb.KA[l]) + bb.ka_lo[l];
        kk /= bb.KA[l];
    }
    for (int k0 = 0; k0 < c.n1; ++k0) {
        const int ia0 = oa[0] + c.dq[k0] - c.amin[0], ib0 = ob[0] + c.dp[k0] - c.bmin[0];
        if ((unsigned)ia0 >= (unsigned)c.A[0] || (unsigned)ib0 >= (unsigned)c.B[0]) continue;
        const int64_t row0 = (int64_t)ia0 * c.ra[0] + (int64_t)ib0 * c.rb[0];
        if constexpr (D == 2) {
            row_flag[row0] = 1;
        } else {
            for (int k1 = 0; k1 < c.n1; ++k1) {
                const int ia1 = oa[1] + c.dq[k1] - c.amin[1], ib1 = ob[1] + c.dp[k1] - c.bmin[1];
                if ((unsigned)ia1 >= (unsigned)c.A[1] || (unsigned)ib1 >= (unsigned)c.B[1]) continue;
                row_flag[row0 + (int64_t)ia1 * c.ra[1] + (int64_t)ib1 * c.rb[1]] = 1;
            }
        }
    }
}

// Zeroes the flagged rows of W (row_f4 16-byte words each): a warp reads the
// flags of 32 consecutive rows at once and clears the flagged ones together.
__global__ void __launch_bounds__(256) clear_flagged_rows_kernel(float4 *__restrict__ W,
                                                                 const uint8_t *__restrict__ row_flag,
                                                                 int64_t rows, int64_t row_f4) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < rows;
         base += nwarps * 32) {
        const bool f = base + lane < rows && row_flag[base + lane] != 0;
        unsigned set = __ballot_sync(0xffffffffu, f);
        while (set) {
            const int r = __ffs(set) - 1;
            set &= set - 1;
            float4 *p = W + (base + r) * row_f4;
            for (int64_t i = lane; i < row_f4; i += 32) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// coeff_dim32 with the neighbours evaluated one after the other into
// out[k * stride] (fewer live registers than the unrolled form).
template <int N1>
__device__ __forceinline__ void coeff_dim32_rolled(const Params32 &P, double Q, double Pm, int &a0, int &b0,
                                                   float2 *out, int stride) {
    const Common &c = P.c;
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
#pragma unroll 1
    for (int k = 0; k < N1; ++k) {
        float sr = 0.f, si = 0.f;
        const float *Cr = P.cre + k * kCheb * kCheb, *Ci = P.cim + k * kCheb * kCheb;
#pragma unroll
        for (int i = 0; i < kCheb; ++i) {
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int jj = 0; jj < kCheb; ++jj) {
                if (i + jj <= cheb_total<N1>()) {
                    ur = fmaf(Cr[i * kCheb + jj], Tt[jj], ur);
                    ui = fmaf(Ci[i * kCheb + jj], Tt[jj], ui);
                }
            }
            sr = fmaf(Ts[i], ur, sr);
            si = fmaf(Ts[i], ui, si);
        }
        float tk = t0f + (float)c.dp[k] * t1f - ccf * (float)(c.dq[k] * c.dp[k]);
        tk -= rint_fast(tk);
        float sn, cs;
        sincospif(2.f * tk, &sn, &cs);
        float vr, vi;
        cmul(sr, si, cs, sn, vr, vi);
        out[k * stride] = make_float2(vr, vi);
    }
}

// Target cells of one window (node cells of the inner plane).
constexpr int kWinCells = 1024;

// float2 slots per packet in the coefficient array: D x N1 rounded to an odd
// number of 16-byte words, so that the 16-byte loads of different packets by
// the lanes of a warp spread over all bank groups instead of two
template <int D, int N1>
__host__ __device__ constexpr int coef_stride() {
    return D * N1 + (((D * N1 / 2) % 2 == 0) ? 2 : 0);
}

template <int D, int N1>
__host__ __device__ constexpr int binned_smem_bytes() {
    return kBinT * coef_stride<D, N1>() * 8  // coefficients [packet][dimension][neighbour] (float2)
           + 2 * kWinCells * 4     // per-cell entry start and cursor (int)
           + kWinCells * 4         // active cells (packed line, column)
           + (D == 3 ? N1 * N1 : N1) * 8  // W offsets of the rows (int64)
           + kBinT * N1 * 2;       // entries (packet << 4 | neighbour), uint16
}

__device__ __forceinline__ int2 block_exclusive_scan(int2 v, int2 *total);

// Binned coefficient + scatter: persistent CTAs take items from *work.  All
// packets of an item share the outer anchor cell, so they reach the same
// n1^(d-1) rows, and a target cell of the inner plane receives, in every row,
// sum over its entries (packet j, inner neighbour k) of
//   w_j c_{d-1,j}[k] * c_{0,j}[k0] (* c_{1,j}[k1]).
// Per item (and window of whole inner q-node lines of the target box) the CTA
// lists every target cell's entries (a CSR built once); then each thread takes
// a cell (and a pass over part of the k0 values), accumulates those rows of it
// in registers as a sum of outer products over its entries, and adds each row's
// value to W with one 8-byte reduction (consecutive threads: consecutive cells
// of the row).  No floating-point atomics in shared memory.
template <int D, int N1>
__global__ void __launch_bounds__(kBinT, kBinCtasPerSm) binned_scatter_kernel(
    const double *__restrict__ q, const double *__restrict__ p, const double *__restrict__ s,
    const double *__restrict__ a, int64_t m, const __grid_constant__ Params32 P, const BinBox bb,
    const int *__restrict__ sorted, const int4 *__restrict__ items, const int2 *__restrict__ off_end,
    int *__restrict__ work, float2 *__restrict__ W, uint8_t *__restrict__ row_flag) {
    constexpr int NR = D == 3 ? N1 * N1 : N1;    // rows reached by one outer anchor cell
    constexpr int NA = (D == 3 && N1 == 8) ? 2 : N1;  // k0 values per accumulation pass
    constexpr int NK1 = D == 3 ? N1 : 1;         // k1 values
    constexpr int kPer = kWinCells / kBinT;      // target cells per thread in the CSR build
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int CS = coef_stride<D, N1>();
    // [kBinT][CS]: per packet [D][N1] coefficients (the last dimension's
    // multiplied by the packet's weight w) and padding
    float2 *coef = reinterpret_cast<float2 *>(smem_raw);
    int *cstart = reinterpret_cast<int *>(coef + kBinT * CS);        // [kWinCells]
    int *cend = cstart + kWinCells;                                  // [kWinCells]
    unsigned *act = reinterpret_cast<unsigned *>(cend + kWinCells);  // [kWinCells]
    int64_t *rowoff = reinterpret_cast<int64_t *>(act + kWinCells);  // [NR]
    unsigned short *ent = reinterpret_cast<unsigned short *>(rowoff + NR);  // [kBinT * N1]
    __shared__ int s_item, s_box[4], s_nact;
    __shared__ int4 s_desc;
    __shared__ unsigned long long s_rows;  // bit r: row r lies in the node box
    const Common &c = P.c;
    const int tid = threadIdx.x;
    const int nitems = off_end->y;
    // thread 0 fetches the next item (index and descriptor) while the CTA
    // works on the current one
    int next = 0;
    int4 next_desc = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        next = atomicAdd(work, 1);
        if (next < nitems) next_desc = items[next];
    }
    for (;;) {
        __syncthreads();  // the previous item's shared data are no longer read
        if (tid == 0) {
            s_item = next;
            s_desc = next_desc;
            s_box[0] = s_box[2] = INT_MAX;
            s_box[1] = s_box[3] = INT_MIN;
            s_rows = 0ull;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int4 item = s_desc;
        if (tid == 0) {
            next = atomicAdd(work, 1);
            if (next < nitems) next_desc = items[next];
        }
        const bool valid = tid < item.z;
        // the rows of the item's outer anchor cell: W offsets, flags, in-box bits
        if (tid < NR) {
            int oa[D - 1], ob[D - 1];
            int kk = item.x;
#pragma unroll
            for (int l = D - 2; l >= 0; --l) {
                ob[l] = kk % bb.KB[l] + bb.kb_lo[l];
                kk /= bb.KB[l];
                oa[l] = kk % bb.KA[l] + bb.ka_lo[l];
                kk /= bb.KA[l];
            }
            const int k0 = D == 3 ? tid / N1 : tid, k1 = D == 3 ? tid % N1 : 0;
            const int ia0 = oa[0] + c.dq[k0] - c.amin[0], ib0 = ob[0] + c.dp[k0] - c.bmin[0];
            bool in = (unsigned)ia0 < (unsigned)c.A[0] && (unsigned)ib0 < (unsigned)c.B[0];
            int64_t idx = (int64_t)ia0 * c.sa[0] + (int64_t)ib0 * c.sb[0];
            int64_t row = (int64_t)ia0 * c.ra[0] + (int64_t)ib0 * c.rb[0];
            if constexpr (D == 3) {
                const int ia1 = oa[1] + c.dq[k1] - c.amin[1], ib1 = ob[1] + c.dp[k1] - c.bmin[1];
                in = in && (unsigned)ia1 < (unsigned)c.A[1] && (unsigned)ib1 < (unsigned)c.B[1];
                idx += (int64_t)ia1 * c.sa[1] + (int64_t)ib1 * c.sb[1];
                row += (int64_t)ia1 * c.ra[1] + (int64_t)ib1 * c.rb[1];
            }
            rowoff[tid] = idx;
            if (in) atomicOr(&s_rows, 1ull << tid);
        }
        float wr = 0.f, wi = 0.f;
        int ra = 0, rb = 0;  // inner anchor relative to the node box (set by the last dimension)
        float2 *cj = coef + tid * CS;
        if (valid) {
            const int64_t j = sorted[item.y + tid];
            double ts = s[j] * c.inv_2pi_eps;
            ts -= rint(ts);
            float sn, cs;
            sincospif(2.f * (float)ts, &sn, &cs);
            cmul((float)(a[j] * c.pref), (float)(a[m + j] * c.pref), cs, sn, wr, wi);
            // one dimension at a time (one copy of the evaluation) into this
            // thread's coefficient block
#pragma unroll 1
            for (int l = 0; l < D; ++l) {
                int a0, b0;
                coeff_dim32_rolled<N1>(P, q[l * m + j], p[l * m + j], a0, b0, cj + l * N1, 1);
                ra = a0 - c.amin[D - 1];
                rb = b0 - c.bmin[D - 1];
            }
            // the weight goes with the last dimension's coefficients, once per
            // packet rather than once per entry and accumulation pass
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                float2 &v = cj[(D - 1) * N1 + k];
                float er, ei;
                cmul(wr, wi, v.x, v.y, er, ei);
                v = make_float2(er, ei);
            }
            atomicMin(&s_box[0], ra + bb.dqmin);
            atomicMax(&s_box[1], ra + bb.dqmax);
            atomicMin(&s_box[2], rb + bb.dpmin);
            atomicMax(&s_box[3], rb + bb.dpmax);
        }
        __syncthreads();
        const unsigned long long rows_in = s_rows;
        if (tid < NR && ((rows_in >> tid) & 1ull)) {
            // first-pass rows that receive contributions
            const int k0 = D == 3 ? tid / N1 : tid, k1 = D == 3 ? tid % N1 : 0;
            int kk = item.x;
            int oa[D - 1], ob[D - 1];
#pragma unroll
            for (int l = D - 2; l >= 0; --l) {
                ob[l] = kk % bb.KB[l] + bb.kb_lo[l];
                kk /= bb.KB[l];
                oa[l] = kk % bb.KA[l] + bb.ka_lo[l];
                kk /= bb.KA[l];
            }
            int64_t row = (int64_t)(oa[0] + c.dq[k0] - c.amin[0]) * c.ra[0] +
                          (int64_t)(ob[0] + c.dp[k0] - c.bmin[0]) * c.rb[0];
            if constexpr (D == 3)
                row += (int64_t)(oa[1] + c.dq[k1] - c.amin[1]) * c.ra[1] +
                       (int64_t)(ob[1] + c.dp[k1] - c.bmin[1]) * c.rb[1];
            row_flag[row] = 1;
        }
        const int ta0 = max(0, s_box[0]), ta1 = min(c.A[D - 1] - 1, s_box[1]);
        const int tb0 = max(0, s_box[2]), tb1 = min(c.B[D - 1] - 1, s_box[3]);
        const int TA = ta1 - ta0 + 1, TB = tb1 - tb0 + 1;
        if (TA <= 0 || TB <= 0 || rows_in == 0ull) continue;  // nothing lands in the node box
        const int WH = kWinCells / TB;  // inner q-node lines per window
        if (WH == 0) {
            // a b-range wider than a window: one reduction per contribution
            if (valid) {
                float cr[N1], ci[N1];
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const float2 v = cj[(D - 1) * N1 + k];
                    cr[k] = v.x;
                    ci[k] = v.y;
                }
#pragma unroll 1
                for (int r = 0; r < NR; ++r) {
                    if (!((rows_in >> r) & 1ull)) continue;
                    const int k0 = D == 3 ? r / N1 : r, k1 = D == 3 ? r % N1 : 0;
                    const float2 c0 = cj[k0];  // w is in cr, ci
                    float pr = c0.x, pi = c0.y;
                    if constexpr (D == 3) {
                        const float2 c1 = cj[N1 + k1];
                        cmul(pr, pi, c1.x, c1.y, pr, pi);
                    }
                    emit_row<D - 1, N1>(W, c, ra + c.amin[D - 1], rb + c.bmin[D - 1], cr, ci, rowoff[r], pr, pi);
                }
            }
            continue;
        }
        const int nwin = (TA + WH - 1) / WH;
#pragma unroll 1
        for (int w = 0; w < nwin; ++w) {
            const int wa = w * WH, wn = min(WH, TA - wa), cells = wn * TB;
            // --- entries of this window: count, scan, fill ---------------------
            __syncthreads();  // the previous window's lists are no longer read
            for (int e = tid; e < cells; e += kBinT) cend[e] = 0;
            __syncthreads();
            if (valid) {
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int ia = ra + c.dq[k] - ta0 - wa, ib = rb + c.dp[k] - tb0;
                    if ((unsigned)ia < (unsigned)wn && (unsigned)ib < (unsigned)TB) atomicAdd(&cend[ia * TB + ib], 1);
                }
            }
            __syncthreads();
            {
                // thread t owns cells [t kPer, (t + 1) kPer): entry starts and the
                // ordered list of non-empty cells by one block scan
                int cnt[kPer];
                int2 loc = make_int2(0, 0);
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int e = tid * kPer + i;
                    cnt[i] = e < cells ? cend[e] : 0;
                    loc.x += cnt[i];
                    loc.y += cnt[i] > 0;
                }
                int2 tot;
                int2 base = block_exclusive_scan(loc, &tot);
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int e = tid * kPer + i;
                    if (e < cells) {
                        cstart[e] = base.x;
                        cend[e] = base.x;  // cursor of the fill below
                        if (cnt[i] > 0) {
                            const int ia = e / TB, ib = e - ia * TB;
                            act[base.y++] = ((unsigned)ia << 16) | (unsigned)ib;
                        }
                        base.x += cnt[i];
                    }
                }
                if (tid == 0) s_nact = tot.y;
            }
            __syncthreads();
            if (valid) {
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int ia = ra + c.dq[k] - ta0 - wa, ib = rb + c.dp[k] - tb0;
                    if ((unsigned)ia < (unsigned)wn && (unsigned)ib < (unsigned)TB) {
                        const int pos = atomicAdd(&cend[ia * TB + ib], 1);
                        ent[pos] = (unsigned short)((tid << 4) | k);
                    }
                }
            }
            __syncthreads();
            const int nact = s_nact;
            // --- cells: rows in registers, then one reduction per row ----------
            // work unit = (pass kp over NA values of k0, cell); consecutive
            // threads take consecutive cells of one pass (coalesced reductions)
            constexpr int NP = N1 / NA;
            for (int u0 = tid; u0 < nact * NP; u0 += kBinT) {
                const int kp = u0 / nact, i = u0 - kp * nact;
                const unsigned cell = act[i];
                const int ia = (int)(cell >> 16), ib = (int)(cell & 0xffffu);
                const int e = ia * TB + ib;
                const int x0 = cstart[e], x1 = cend[e];
                float2 *Wc = W + (int64_t)(ta0 + wa + ia) * c.sa[D - 1] + tb0 + ib;
                float accr[NA][NK1], acci[NA][NK1];
#pragma unroll
                for (int u = 0; u < NA; ++u)
#pragma unroll
                    for (int v = 0; v < NK1; ++v) accr[u][v] = acci[u][v] = 0.f;
                for (int x = x0; x < x1; ++x) {
                    const int en = ent[x], jj = en >> 4, kk = en & 15;
                    const float2 ev = coef[jj * CS + (D - 1) * N1 + kk];  // w c_{d-1}[k]
                    // the packet's coefficients, 16-byte loads (two neighbours each)
                    const float4 *cp4 = reinterpret_cast<const float4 *>(coef + jj * CS);
                    float2 c0v[NA];
#pragma unroll
                    for (int u = 0; u < NA; u += 2) {
                        const float4 t = cp4[(kp * NA + u) / 2];
                        c0v[u] = make_float2(t.x, t.y);
                        c0v[u + 1] = make_float2(t.z, t.w);
                    }
                    float2 c1v[NK1];
                    if constexpr (D == 3) {
#pragma unroll
                        for (int v = 0; v < NK1; v += 2) {
                            const float4 t = cp4[(N1 + v) / 2];
                            c1v[v] = make_float2(t.x, t.y);
                            c1v[v + 1] = make_float2(t.z, t.w);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < NA; ++u) {
                        float tr, ti;
                        cmul(ev.x, ev.y, c0v[u].x, c0v[u].y, tr, ti);
                        if constexpr (D == 3) {
#pragma unroll
                            for (int v = 0; v < NK1; ++v) {
                                accr[u][v] = fmaf(tr, c1v[v].x, fmaf(-ti, c1v[v].y, accr[u][v]));
                                acci[u][v] = fmaf(tr, c1v[v].y, fmaf(ti, c1v[v].x, acci[u][v]));
                            }
                        } else {
                            accr[u][0] += tr;
                            acci[u][0] += ti;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < NA; ++u)
#pragma unroll
                    for (int v = 0; v < NK1; ++v) {
                        const int r = (kp * NA + u) * NK1 + v;
                        if ((rows_in >> r) & 1ull) atomicAdd(Wc + rowoff[r], make_float2(accr[u][v], acci[u][v]));
                    }
            }
        }
    }
}

// Exclusive scan of (binned packets, items) per key: a cell with at least
// min_count packets is binned (its packets and ceil(n / kBinT) items count),
// other cells count zero.  off[K] receives the totals.
__device__ __forceinline__ int2 bin_pair(const int *count, int64_t k, int64_t K, int min_count) {
    if (k >= K) return make_int2(0, 0);
    const int n = count[k];
    return n >= min_count ? make_int2(n, (n + kBinT - 1) / kBinT) : make_int2(0, 0);
}

__device__ __forceinline__ int2 block_exclusive_scan(int2 v, int2 *total) {
    __shared__ int2 wsum[32];  // (blockDim.x a multiple of 32, at most 1024)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int2 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int yx = __shfl_up_sync(0xffffffffu, x.x, o), yy = __shfl_up_sync(0xffffffffu, x.y, o);
        if (lane >= o) {
            x.x += yx;
            x.y += yy;
        }
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int2 w = lane < nw ? wsum[lane] : make_int2(0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yx = __shfl_up_sync(0xffffffffu, w.x, o), yy = __shfl_up_sync(0xffffffffu, w.y, o);
            if (lane >= o) {
                w.x += yx;
                w.y += yy;
            }
        }
        if (lane < nw) wsum[lane] = w;  // inclusive warp prefixes
    }
    __syncthreads();
    const int2 before = wid > 0 ? wsum[wid - 1] : make_int2(0, 0);
    *total = wsum[nw - 1];
    __syncthreads();
    return make_int2(before.x + x.x - v.x, before.y + x.y - v.y);
}

__global__ void __launch_bounds__(1024) bin_scan1_kernel(const int *__restrict__ count, int64_t K, int min_count,
                                                         int2 *__restrict__ off, int2 *__restrict__ bsum) {
    const int64_t k = blockIdx.x * (int64_t)1024 + threadIdx.x;
    int2 tot;
    const int2 e = block_exclusive_scan(bin_pair(count, k, K, min_count), &tot);
    if (k < K) off[k] = e;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the block totals (in place); off[K] = total.
__global__ void __launch_bounds__(1024) bin_scan2_kernel(int2 *__restrict__ bsum, int64_t nblk,
                                                         int2 *__restrict__ off, int64_t K) {
    int2 carry = make_int2(0, 0);
    for (int64_t b0 = 0; b0 < nblk; b0 += 1024) {
        const int64_t b = b0 + threadIdx.x;
        const int2 v = b < nblk ? bsum[b] : make_int2(0, 0);
        int2 tot;
        const int2 e = block_exclusive_scan(v, &tot);
        if (b < nblk) bsum[b] = make_int2(carry.x + e.x, carry.y + e.y);
        carry.x += tot.x;
        carry.y += tot.y;
    }
    if (threadIdx.x == 0) off[K] = carry;
}

__global__ void __launch_bounds__(1024) bin_scan3_kernel(int2 *__restrict__ off, int64_t K,
                                                         const int2 *__restrict__ bsum) {
    const int64_t k = blockIdx.x * (int64_t)1024 + threadIdx.x;
    if (k >= K) return;
    const int2 b = bsum[blockIdx.x];
    int2 v = off[k];
    v.x += b.x;
    v.y += b.y;
    off[k] = v;
}

// The binned scatter of d >= 2 (FP32): binning, items, then the binned
// kernel and the per-packet kernel over the loose list, all on stream st.
template <int D, int N1>
fgr_status launch_binned_d(const BinLaunch &L, cudaStream_t st, const PacketsDev &pk, const Params32 &P, void *W,
                           uint8_t *flags, StageMarks *marks) {
    const int64_t m = pk.m, K = L.box.K;
    const BinBuffers &b = L.buf;
    FGR_CUDA_TRY(cudaMemsetAsync(b.count, 0, sizeof(int) * (size_t)K, st));
    FGR_CUDA_TRY(cudaMemsetAsync(b.ctr, 0, sizeof(int) * 4, st));
    const unsigned pblocks = (unsigned)((m + 255) / 256);
    bin_key_kernel<D><<<pblocks, 256, 0, st>>>(pk.q, pk.p, pk.a, m, P.c, L.box, b.key, b.count);
    if (L.clear_rows > 0) {  // the caller cleared the row flags, not W
        bin_mark_rows_kernel<D><<<(unsigned)((K + 255) / 256), 256, 0, st>>>(b.count, P.c, L.box, flags);
        clear_flagged_rows_kernel<<<(unsigned)(L.num_sms * 8), 256, 0, st>>>((float4 *)W, flags, L.clear_rows,
                                                                          L.row_cells / 2);
    }
    const int64_t nblk = (K + 1023) / 1024;
    bin_scan1_kernel<<<(unsigned)nblk, 1024, 0, st>>>(b.count, K, L.min_count, b.off, b.bsum);
    bin_scan2_kernel<<<1, 1024, 0, st>>>(b.bsum, nblk, b.off, K);
    bin_scan3_kernel<<<(unsigned)nblk, 1024, 0, st>>>(b.off, K, b.bsum);
    bin_place_kernel<<<pblocks, 256, 0, st>>>(b.key, m, b.off, b.count, b.sorted, b.loose, b.ctr);
    bin_items_kernel<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(b.off, K, b.items);
    FGR_CUDA_TRY(cudaGetLastError());
    if (marks) marks->binned();
    constexpr int smem = binned_smem_bytes<D, N1>();
    FGR_CUDA_TRY(cudaFuncSetAttribute(binned_scatter_kernel<D, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem));
    binned_scatter_kernel<D, N1><<<(unsigned)(L.num_sms * kBinCtasPerSm), kBinT, smem, st>>>(
        pk.q, pk.p, pk.s, pk.a, m, P, L.box, b.sorted, b.items, b.off + K, b.ctr + 1, (float2 *)W, flags);
    constexpr int T = coeff_threads<false, N1>();
    coeff_scatter_list_kernel<D, false, N1><<<(unsigned)(L.num_sms * 4), T, 0, st>>>(
        pk.q, pk.p, pk.s, pk.a, m, P, W, flags, b.loose, b.ctr);
    FGR_CUDA_TRY(cudaGetLastError());
    return FGR_OK;
}

}  // namespace
}  // namespace fgr
