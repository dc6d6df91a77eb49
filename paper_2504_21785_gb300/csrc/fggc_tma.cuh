// K5 grid pass (FP32, 32-point tiles) with the node-array tiles staged by the
// tensor memory accelerator: the pass input, viewed as a 2-D tensor of
// (row, a) lines by B cells, is read in boxes of kTB b-cells x MAXBAND lines by
// cp.async.bulk.tensor into two shared-memory buffers that alternate, so the
// next tile's copy overlaps the current tile's arithmetic (one warp per CTA:
// lane 0 issues the copies, every lane waits on the buffer's mbarrier).
// Same arithmetic as grid_pass_body.  Waits are bounded: a copy that does not
// complete within the limit sets *err and the CTA returns.
// Included by fggc.cu inside its anonymous namespace, after grid_pass_body
// (fggc.cu includes <cuda.h> for CUtensorMap).
#pragma once

constexpr unsigned kTmaWaitLimit = 1u << 26;  // polls of an mbarrier before giving up
// b cells per staged tile (a 64-byte row per line).  A tile is multiplied
// whole, so its width trades the zero padding past a row's occupied b-range
// against the per-tile overhead: on the 3-D workload 12 or 8 cells took the
// passes from 5.29 to 4.54 ms against 16, and 8 cells keep the CTA's shared
// memory (two tile buffers and the row sums) near 6 KB, so that with at most
// 64 registers about 30 one-warp CTAs fit an SM (3.89 -> 3.76 ms against 12).
constexpr int kTB = 8;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// true once the barrier has completed the phase of parity `phase`
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// 2-D tile copy global -> shared, completion counted on bar (bytes)
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait of the whole warp on a buffer's barrier (the outcome is the
// same for every lane); false, and *err set, if it timed out.
__device__ __forceinline__ bool tma_wait(uint64_t *bar, unsigned phase, int *err) {
    for (unsigned it = 0; it < kTmaWaitLimit; ++it) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, phase))) return true;
        if (it > 64) __nanosleep(64);
    }
    if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
    return false;
}

// Compensated summation (Kahan): s += x with c carrying the negated rounding
// error of the previous additions; the sum is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// map: boxes of MAXBAND lines; map_half: boxes of MAXBAND / 2 lines, for a
// last band chunk that needs no more (half the copy).  A CTA (one warp) takes
// one 32-point tile of RPC consecutive rows: the rows share the tile's node
// band, Gaussian factors and windows, and their tiles form one sequence of
// copies (band chunk, row, b chunk), so the copy of the next tile, also of
// the next row, is in flight while the warp multiplies the current one.
template <int MAXBAND, int RPC>
__global__ void __launch_bounds__(32, 32) grid_pass_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                           const __grid_constant__ CUtensorMap map_half,
                                                           void *__restrict__ out_v, PassParams pp,
                                                           const uint8_t *__restrict__ flags,
                                                           const int2 *__restrict__ brange, const PassTables tab,
                                                           int *__restrict__ err) {
    constexpr int TP = 32;
    static_assert(kTB % 4 == 0, "whole 16-byte words per tile row, four b values per step");
    __shared__ __align__(128) float2 sw[2][MAXBAND][kTB];
    __shared__ __align__(8) uint64_t bar[2];
    // per row and lane: the compensated FP32 sum of the chunk partials (re, im
    // and their running corrections; FP64 runs at 1/64 of the FP32 rate here)
    __shared__ float4 s_tot[RPC][TP];
    const int lane = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * RPC;
    const int tile = blockIdx.y;
    const int64_t m = (int64_t)tile * TP + lane;
    const bool valid = m < pp.N;
    float2 *out = reinterpret_cast<float2 *>(out_v);
    const int2 bnd = tab.band[tile];
    const int a_lo = bnd.x, a_hi = bnd.y;
    const int nb_total = a_hi - a_lo + 1;
    // per row: occupied b-range of the band (empty: no chunks)
    int b_start[RPC], nbc[RPC], S = 0;
#pragma unroll
    for (int r = 0; r < RPC; ++r) {
        const int64_t row = row0 + r;
        bool live = row < pp.rows && nb_total > 0 && !(flags && !flags[row]);
        int ulo = 0, uhi = pp.B - 1;
        if (live && brange) {
            int lo = INT_MAX, hi = INT_MIN;
            for (int i = lane; i < nb_total; i += TP) {
                const int2 rg = brange[row * (int64_t)pp.A + (a_lo - pp.amin) + i];
                lo = min(lo, rg.x);
                hi = max(hi, rg.y);
            }
            ulo = __reduce_min_sync(0xffffffffu, lo);
            uhi = __reduce_max_sync(0xffffffffu, hi);
        }
        live = live && ulo <= uhi;
        // b chunks start at even cells (16-byte copy coordinates); the cell
        // before an odd ulo is zero in every line of the band
        b_start[r] = ulo & ~1;
        nbc[r] = live ? (uhi - b_start[r] + kTB) / kTB : 0;
        S += nbc[r];
        s_tot[r][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int nac = nb_total > 0 ? (nb_total + MAXBAND - 1) / MAXBAND : 0;
    const int ntiles = nac * S;
    constexpr unsigned kBytes = MAXBAND * kTB * sizeof(float2);
    // tile t -> (band chunk ac, row r, b chunk bc)
    auto decode = [&](int t, int &ac, int &r, int &bc) {
        ac = t / S;
        int rem = t - ac * S;
        r = 0;
#pragma unroll
        for (int k = 0; k < RPC; ++k)
            if (r == k && rem >= nbc[k]) {
                rem -= nbc[k];
                r = k + 1;
            }
        bc = rem;
    };
    auto start_of = [&](int r) {
        int v = 0;
#pragma unroll
        for (int k = 0; k < RPC; ++k)
            if (k == r) v = b_start[k];
        return v;
    };
    if (ntiles > 0 && lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncwarp();
    auto issue = [&](int t) {
        int ac, r, bc;
        decode(t, ac, r, bc);
        const bool half = nb_total - ac * MAXBAND <= MAXBAND / 2;
        const int64_t line = (row0 + r) * (int64_t)pp.A + (a_lo - pp.amin) + ac * MAXBAND;
        mbar_expect_tx(&bar[t & 1], half ? kBytes / 2 : kBytes);
        tma_load_2d(&sw[t & 1][0][0], half ? &map_half : &map, start_of(r) + bc * kTB, (int)line, &bar[t & 1]);
    };
    if (lane == 0) {
        if (ntiles > 0) issue(0);
        if (ntiles > 1) issue(1);
    }
    const double xm = grid_x(pp.lo, pp.h, valid ? m : (int64_t)tile * TP);
    const float2 ph = tab.ph[valid ? m : (int64_t)tile * TP];
    // rotation of one b step, e^{2 pi i (ph.x + ph.y)} (accurate sine and cosine)
    float step_r, step_i;
    sincospif(2.f * (ph.x - rint_fast(ph.x) + ph.y), &step_i, &step_r);
    const float cef = (float)(pp.neg_half_inv_eps * 1.4426950408889634);  // log2(e) / (-2 eps)
    const float dqf = (float)pp.dq;
    float g[MAXBAND];
    int nb = 0, ac_cur = -1;
    unsigned phase[2] = {0u, 0u};
    for (int t = 0; t < ntiles; ++t) {
        int ac, r, bc;
        decode(t, ac, r, bc);
        if (ac != ac_cur) {  // Gaussian factors of this band chunk (shared by the rows)
            ac_cur = ac;
            const int a_first = a_lo + ac * MAXBAND;
            nb = min(MAXBAND, nb_total - ac * MAXBAND);
            const double dx0 = xm - (double)a_first * pp.dq;
            // node windows: one coalesced load, then broadcast by shuffles
            const int2 wl = lane < nb ? tab.win[a_first - pp.amin + lane] : make_int2(1, 0);
#pragma unroll
            for (int i = 0; i < MAXBAND; ++i) {
                const int wx = __shfl_sync(0xffffffffu, wl.x, i), wy = __shfl_sync(0xffffffffu, wl.y, i);
                g[i] = 0.f;
                if (i < nb && valid && m >= wx && m <= wy) {
                    const float dxf = (float)dx0 - (float)i * dqf;
                    g[i] = ex2_approx(dxf * dxf * cef);
                }
            }
        }
        const int s = t & 1;
        if (!tma_wait(&bar[s], phase[s], err)) {
            // leave only after this CTA's copies in flight have landed (bounded)
            tma_wait(&bar[s], phase[s], err);
            if (t + 1 < ntiles) tma_wait(&bar[(t + 1) & 1], phase[(t + 1) & 1], err);
            return;
        }
        phase[s] ^= 1u;
        // whole chunks: cells past the band's occupied range are zero in every
        // line of the band (and past the node box the copy fills zeros)
        const int b0 = start_of(r) + bc * kTB;
        float accr = 0.f, acci = 0.f;
#pragma unroll 1
        for (int bb = 0; bb < kTB; bb += 4) {
            float vr[4] = {0.f, 0.f, 0.f, 0.f}, vi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < MAXBAND; ++i) {
                if (i < nb) {
                    const float4 w = *reinterpret_cast<const float4 *>(&sw[s][i][bb]);
                    const float4 w2 = *reinterpret_cast<const float4 *>(&sw[s][i][bb + 2]);
                    vr[0] = fmaf(g[i], w.x, vr[0]);
                    vi[0] = fmaf(g[i], w.y, vi[0]);
                    vr[1] = fmaf(g[i], w.z, vr[1]);
                    vi[1] = fmaf(g[i], w.w, vi[1]);
                    vr[2] = fmaf(g[i], w2.x, vr[2]);
                    vi[2] = fmaf(g[i], w2.y, vi[2]);
                    vr[3] = fmaf(g[i], w2.z, vr[3]);
                    vi[3] = fmaf(g[i], w2.w, vi[3]);
                }
            }
            // e^{i b dp x_m / eps} at the step's first b from the reduced
            // phase, the next three b by rotation with the per-b factor
            float zr, zi;
            {
                const float bf = (float)(pp.bmin + b0 + bb);
                float f = bf * ph.x;
                f -= rint_fast(f);
                float tau = fmaf(bf, ph.y, f);
                tau -= rint_fast(tau);
                __sincosf(6.283185307179586f * tau, &zi, &zr);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                accr += zr * vr[u] - zi * vi[u];
                acci += zr * vi[u] + zi * vr[u];
                if (u < 3) {
                    const float nr = zr * step_r - zi * step_i;
                    zi = fmaf(zr, step_i, zi * step_r);
                    zr = nr;
                }
            }
        }
        float4 tv = s_tot[r][lane];
        kahan_add(tv.x, tv.z, accr);
        kahan_add(tv.y, tv.w, acci);
        s_tot[r][lane] = tv;
        // the buffer is free again: refill it with tile t + 2
        __syncwarp();
        if (lane == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2);
        }
    }
#pragma unroll
    for (int r = 0; r < RPC; ++r) {
        const int64_t row = row0 + r;
        if (row < pp.rows && valid) {
            const float4 tv = s_tot[r][lane];
            out[row * pp.N + m] = make_float2(__fsub_rn(tv.x, tv.z), __fsub_rn(tv.y, tv.w));
        }
    }
}
