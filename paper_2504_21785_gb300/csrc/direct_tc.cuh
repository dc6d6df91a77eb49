// K2 on the fifth-generation tensor cores (FP32 records, d = 2).
//
// The separable form of the direct sum (eq. 2.10 with the box window): a
// packet's term on the grid is the outer product of its per-dimension factors,
//   u[i, j] += F0_r[i] F1_r[j],   F0_r[i] = pref A_r e^{i S_r / eps} g_r(x_i) e^{i P_r (x_i - Q_r) / eps},
// each factor zero outside the packet's window in its dimension.  Over the
// records r of a super tile (128 lines of dimension 0 x 32 lines of dimension 1,
// four tiles of the binning stacked along dimension 0) this is a complex
// matrix product U = F0 F1^T with K = the records, computed as one real
// product on tcgen05.mma (kind::tf32, M = 128, N = 64, K = 8 per instruction):
//   A[i][2r + c]  = (Re F0_r[i], Im F0_r[i])[c]
//   B[j][2r + c]  = (Re F1_r[j], -Im F1_r[j])[c]       (row j: the real part)
//   B[32 + j][..] = (Im F1_r[j],  Re F1_r[j])[c]       (row 32 + j: the imaginary part)
// so D[i][j] = Re u and D[i][32 + j] = Im u, accumulated in tensor memory.
// FP32 accuracy from TF32 operands: every factor x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), and D += A_hi B_hi + A_hi B_lo +
// A_lo B_hi (three instructions per K step; the dropped A_lo B_lo and the
// rounding of x_lo are about 2^-22 of a product).
//
// Pipeline: a persistent CTA of 640 threads takes (super tile, slice) items
// from a device counter.  Records are staged 256 at a time (the next 256 are
// loaded into registers while the current ones are used, and each record's
// phase rotation over 8 grid lines is computed once when it is staged); for
// every 16 of them the CTA writes the factors (hi and lo) into one of two
// shared-memory operand stages in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes; 128 bytes between core matrices along
// K, 1024 bytes between 8-row groups), one thread issues the 12 MMAs and
// commits them to the stage's mbarrier, and the CTA goes on to the other stage
// while the tensor core works.  Factors: one unit of four lines per thread and
// chunk; warps 0-15 tabulate dimension 0 (a thread takes one record and the
// lines i0 + 8m, so the 16 lanes of a half warp store 16 distinct 8-byte words
// of one 128-byte core matrix), warps 16-19 dimension 1; the first line inside
// the window is evaluated in full (ex2 and sincos), the next by the exact
// recurrences over 8 grid lines (Gaussian ratio 2^{ce h (16 dx + 64 h)}, itself
// multiplied by e^{-64 h^2 / eps} per step; phase rotation e^{2 pi i 8 nu}).
//
// Accumulation: the tensor core adds into its FP32 accumulator with truncated
// alignment, so no accumulator sums more than 4 chunks (64 records, 48
// instructions): chunks 4k..4k+3 of an item go to TMEM accumulator k mod 2,
// and while the next four chunks fill the other one, warps 0-15 read the
// finished one back (tcgen05.ld, one row per lane, 8 columns per warp) into
// FP32 registers.  At the end of an item the registers are added to the
// zeroed output with float2 atomics.
//
// Waits on the mbarriers are bounded: on expiry the CTA sets *err, stops
// taking items and releases its tensor memory.
// Included by direct.cu inside its anonymous namespace.
#pragma once

namespace tc {

constexpr int kRows = 128;                       // M: lines of dimension 0 per super tile
constexpr int kSuper0 = kRows / 32;              // binning tiles stacked along dimension 0
constexpr int kCols = 32;                        // lines of dimension 1 per super tile
constexpr int kN = 2 * kCols;                    // N: real and imaginary outputs
constexpr int kRec = 16;                         // records per MMA chunk
constexpr int kK = 2 * kRec;                     // TF32 elements of K per chunk
constexpr int kGenThreads = 640;                 // producers: 16 warps for dimension 0, 4 for dimension 1
constexpr int kThreadsTc = kGenThreads + 32;     // + one warp that issues the MMAs
constexpr int kStageRec = 256;                   // records staged in shared memory at a time
constexpr int kPhase = 4;                        // chunks summed in one TMEM accumulator
constexpr int kABytes = kRows * kK * 4;          // 16 KB
constexpr int kBBytes = kN * kK * 4;             // 8 KB
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr int kStages = 3;
constexpr int kTmemCols = 2 * kN;                // two accumulators
constexpr unsigned kWaitLimit = 1u << 24;        // polls of an mbarrier before giving up
constexpr size_t kDynSmem =
    (size_t)kStages * kStageBytes + (size_t)kStageRec * sizeof(RecF<2>) + (size_t)kStageRec * sizeof(float4);
static_assert(kTmemCols == 128, "two accumulators of N 32-bit columns");

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// byte offset of element (row, kk) of a K-major operand, no swizzle, kK wide
__device__ __forceinline__ unsigned kmaj(int row, int kk) {
    return (unsigned)((kk >> 2) * 128 + (row >> 3) * 1024 + (row & 7) * 16 + (kk & 3) * 4);
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte
// offsets, fixed field 0b001 at bit 46, no swizzle
__device__ __forceinline__ uint64_t sdesc(unsigned addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46);
}

// x rounded to TF32 (10 explicit mantissa bits), nearest with ties away from
// zero, for finite x: add half a TF32 unit to the magnitude bits and clear the
// 13 dropped bits
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool bar_try(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of parity `parity`; false on expiry
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        if (bar_try(bar, parity)) return true;
        if (it > 32) __nanosleep(32);
    }
    return false;
}

// 8 consecutive 32-bit TMEM columns of the warp's 32 lanes (one row per lane)
__device__ __forceinline__ void tmem_ld8(unsigned taddr, float *v) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Factor of dimension l of record R at the grid lines k0 + 8 m, m = 0..3 (zero
// outside the window); rot = e^{2 pi i 8 nu_l} of the record; fold: dimension 0
// carries log2|pref A| and the phase of pref A e^{i theta} at the window start.
__device__ __forceinline__ void factor4(const RecF<2> &R, const int l, const int k0, const float2 rot,
                                        const DirectParams &P, const bool fold, float2 *out) {
    const float kf0 = (float)k0 - R.mlo[l];
    const float wl = R.wlen[l];
    // first of the four lines inside the window (kf0 is integral)
    const int m0 = kf0 >= 0.f ? 0 : (int)ceilf(-0.125f * kf0);
    float vr = 0.f, vi = 0.f, rho = 0.f;
    const bool any = m0 < 4 && kf0 + 8.f * (float)m0 < wl;
    if (any) {
        const float h = P.hf[l];
        const float kf = kf0 + 8.f * (float)m0;
        const float dx = fmaf(kf, h, R.delta[l]);
        float ex = dx * dx * P.ce;
        float fr = kf * R.nuhi[l];
        fr -= rint_fast(fr);
        float tau = fmaf(kf, R.nulo[l], fr);
        if (fold) {
            ex += R.la;
            tau += R.tau0;
        }
        tau -= rint_fast(tau);
        float sn, cs;
        __sincosf(6.283185307179586f * tau, &sn, &cs);
        const float ga = ex2_approx(ex);
        vr = ga * cs;
        vi = ga * sn;
        rho = ex2_approx(P.ce * h * fmaf(16.f, dx, 64.f * h));
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const bool in = any && m >= m0 && kf0 + 8.f * (float)m < wl;
        out[m] = in ? make_float2(vr, vi) : make_float2(0.f, 0.f);
        if (m < 3 && m >= m0) {
            const float pr = rot.x * rho, pi = rot.y * rho;
            const float nr = vr * pr - vi * pi;
            vi = vr * pi + vi * pr;
            vr = nr;
            rho *= P.q8[l];
        }
    }
}

// Writes the factors of records rec[0 .. nrec-1] (zeros for r >= nrec) into
// one operand stage: A_hi, A_lo (128 x kK), B_hi, B_lo (64 x kK); one unit of
// four lines per thread.
__device__ __forceinline__ void fill_stage(unsigned char *stage, const RecF<2> *rec, const float4 *rot,
                                           const int nrec, const int T0, const int T1, const DirectParams &P) {
    const int tid = threadIdx.x;
    float2 f[4];
    if (tid < 512) {
        // dimension 0: record 2 (tid >> 5 & 7) + (tid >> 3 & 1), rows 32 blk + (tid & 7) + 8 m,
        // blk = 2 (tid >> 8) + (tid >> 4 & 1)
        const int r = 2 * ((tid >> 5) & 7) + ((tid >> 3) & 1);
        const int i0 = 32 * (2 * (tid >> 8) + ((tid >> 4) & 1)) + (tid & 7);
        if (r < nrec) {
            const float4 rr = rot[r];
            factor4(rec[r], 0, T0 + i0, make_float2(rr.x, rr.y), P, true, f);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) f[m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned o = kmaj(i0 + 8 * m, 2 * r);
            const float hr = tf32_round(f[m].x), hi = tf32_round(f[m].y);
            const float lr = tf32_round(f[m].x - hr), li = tf32_round(f[m].y - hi);
            *reinterpret_cast<float2 *>(stage + o) = make_float2(hr, hi);
            *reinterpret_cast<float2 *>(stage + kABytes + o) = make_float2(lr, li);
        }
    } else {
        // dimension 1: record v >> 3, columns (v & 7) + 8 m
        const int v = tid - 512;
        const int r = v >> 3, j0 = v & 7;
        unsigned char *Bh = stage + 2 * kABytes;
        unsigned char *Bl = Bh + kBBytes;
        if (r < nrec) {
            const float4 rr = rot[r];
            factor4(rec[r], 1, T1 + j0, make_float2(rr.z, rr.w), P, false, f);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) f[m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = j0 + 8 * m;
            const unsigned o_re = kmaj(j, 2 * r), o_im = kmaj(kCols + j, 2 * r);
            const float hr = tf32_round(f[m].x), hi = tf32_round(f[m].y);
            const float lr = tf32_round(f[m].x - hr), li = tf32_round(f[m].y - hi);
            *reinterpret_cast<float2 *>(Bh + o_re) = make_float2(hr, -hi);
            *reinterpret_cast<float2 *>(Bh + o_im) = make_float2(hi, hr);
            *reinterpret_cast<float2 *>(Bl + o_re) = make_float2(lr, -li);
            *reinterpret_cast<float2 *>(Bl + o_im) = make_float2(li, lr);
        }
    }
}

}  // namespace tc

// Records in the list of every super tile (union of the home-tile boxes of its
// kSuper0 tiles).
__global__ void tc_tile_load_kernel(const int64_t *__restrict__ off, GridDev g, uint32_t *__restrict__ load) {
    const int nst1 = g.nt[1];
    const int nst0 = (g.nt[0] + tc::kSuper0 - 1) / tc::kSuper0;
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile >= nst0 * nst1) return;
    const int s0 = tile / nst1, s1 = tile % nst1;
    const int h0lo = max(0, tc::kSuper0 * s0 - g.K[0]);
    const int h0hi = min(g.nt[0] - 1, tc::kSuper0 * s0 + tc::kSuper0 - 1);
    const int h1lo = max(0, s1 - g.K[1]);
    int64_t sum = 0;
    for (int h0 = h0lo; h0 <= h0hi; ++h0) sum += off[h0 * nst1 + s1 + 1] - off[h0 * nst1 + h1lo];
    load[tile] = (uint32_t)(sum < 0xffffffffLL ? sum : 0xffffffffLL);
}

// what the MMA warp needs to know about the chunk in a stage
struct ChunkInfo {
    int phase;      // accumulator phase (accumulator phase & 1)
    int first;      // first chunk of the phase: the first MMA overwrites the accumulator
    int phase_end;  // last chunk of the phase: commit the accumulator's barrier too
    int stop;       // no more chunks
};

// bounded wait that also gives up once another thread has reported a failure
__device__ __forceinline__ bool bar_wait_or_abort(uint64_t *bar, unsigned parity, const volatile int *abort) {
    for (unsigned it = 0; it < tc::kWaitLimit; ++it) {
        if (tc::bar_try(bar, parity)) return true;
        if ((it & 63) == 63 && *abort) return false;
        if (it > 32) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(bar)) : "memory");
}

// named barrier of the producer threads; returns the OR of v over them
__device__ __forceinline__ bool producers_sync_or(bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "n"(tc::kGenThreads)
        : "memory");
    return r != 0;
}

// Persistent tensor-core direct sum (FP32, d = 2); items as in
// direct_items_kernel, with super tiles in place of tiles.  Warps 0-19 produce
// the operands and read the accumulators back; warp 20 issues the MMAs.
// Stage s is handed over through full[s] (640 producer arrivals) and back
// through empty[s] (the MMA commit); accumulator a through acc_full[a] (MMA
// commit after the last chunk of a phase) and acc_empty[a] (512 reader
// arrivals after the read-back).
__global__ void __launch_bounds__(tc::kThreadsTc, 1)
    direct_tc_kernel(const RecF<2> *__restrict__ recs, const int64_t *__restrict__ off, DirectParams P,
                     float2 *__restrict__ u, const int2 *__restrict__ items, const int *__restrict__ n_items,
                     unsigned long long *__restrict__ counter, const volatile int *yield, int keep,
                     int *__restrict__ err) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *stages = smem;
    RecF<2> *srec = reinterpret_cast<RecF<2> *>(smem + kStages * kStageBytes);
    float4 *srot = reinterpret_cast<float4 *>(smem + kStages * kStageBytes + kStageRec * sizeof(RecF<2>));
    constexpr int kSegMax = 64;  // rows of a super tile's home-tile box (checked on the host)
    __shared__ uint32_t seg_start[kSegMax];
    __shared__ uint32_t seg_cum[kSegMax + 1];
    __shared__ int nseg_s;
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
    __shared__ ChunkInfo info[kStages];
    __shared__ unsigned s_tmem;
    __shared__ long long s_item;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GridDev &g = P.g;
    const int nst1 = g.nt[1];
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[s])), "r"(kGenThreads) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])) : "memory");
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&acc_full[a])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 512;" ::"r"(saddr(&acc_empty[a])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = s_tmem;

    if (warp == kGenThreads / 32) {
        // ---- MMA issuer (one thread) ----
        if (lane == 0) {
            for (uint32_t gc = 0;; ++gc) {
                const int s = gc % kStages;
                if (!bar_wait_or_abort(&full[s], (gc / kStages) & 1, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                const volatile ChunkInfo *vi = &info[s];
                const ChunkInfo ci{vi->phase, vi->first, vi->phase_end, vi->stop};
                if (ci.stop) break;
                const int a = ci.phase & 1;
                if (ci.first && ci.phase >= 2 &&
                    !bar_wait_or_abort(&acc_empty[a], ((ci.phase >> 1) - 1) & 1, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                fence_after();
                const unsigned sa = saddr(stages + s * kStageBytes);
                const unsigned d = tmem + (unsigned)(a * kN);
#pragma unroll
                for (int ks = 0; ks < kK / 8; ++ks) {
                    const unsigned o = 256u * ks;
                    const uint64_t ah = sdesc(sa + o), al = sdesc(sa + kABytes + o);
                    const uint64_t bh = sdesc(sa + 2 * kABytes + o), bl = sdesc(sa + 2 * kABytes + kBBytes + o);
                    mma_tf32(d, al, bh, (ci.first && ks == 0) ? 0u : 1u);
                    mma_tf32(d, ah, bl, 1u);
                    mma_tf32(d, ah, bh, 1u);
                }
                mma_commit(&empty[s]);
                if (ci.phase_end) mma_commit(&acc_full[a]);
            }
        }
    } else {
        // ---- producers and accumulator readers ----
        uint32_t gc = 0;   // chunks produced by this CTA
        int phase = 0;     // accumulator phases started by this CTA
        bool abort = false;
        const long long total = *n_items;
        // warps 0-15 read the accumulators: lane quarter q (rows 32 q + lane), columns 8 cg .. 8 cg + 7
        const int q = warp & 3, cg = (warp >> 2) & 3;
        const bool reader = warp < 16;
        float acc_re[8], acc_im[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc_re[k] = acc_im[k] = 0.f;
        auto read_acc = [&](int ph) {
            if (!reader || abort) return;
            const int a = ph & 1;
            if (!bar_wait_or_abort(&acc_full[a], (ph >> 1) & 1, &s_abort)) {
                abort = true;
                s_abort = 1;
                return;
            }
            fence_after();
            const unsigned base = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(a * kN);
            float re[8], im[8];
            tmem_ld8(base + 8 * cg, re);
            tmem_ld8(base + kCols + 8 * cg, im);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc_re[k] += re[k];
                acc_im[k] += im[k];
            }
            fence_before();
            bar_arrive(&acc_empty[a]);
        };
        // waits for stage s to be free and hands chunk info over with the stage
        auto stage_free = [&](int s) {
            if (gc >= (uint32_t)kStages && !abort &&
                !bar_wait_or_abort(&empty[s], ((gc / kStages) - 1) & 1, &s_abort)) {
                abort = true;
                s_abort = 1;
            }
        };
        for (;;) {
            if (tid == 0) {
                const bool stop = abort || (yield != nullptr && (int)blockIdx.x >= keep && *yield > 0);
                s_item = stop ? total : (long long)atomicAdd(counter, 1ULL);
            }
            if (producers_sync_or(abort)) {
                abort = true;
                break;
            }
            const long long item = s_item;
            if (item >= total) break;
            const int2 it = items[item];
            const int split = it.y & 0xff, nsplit = it.y >> 8;
            const int s0 = it.x / nst1, s1 = it.x % nst1;
            if (tid == 0) {  // segments: rows of the home-tile box, each a run of tiles along dimension 1
                const int h0lo = max(0, kSuper0 * s0 - g.K[0]);
                const int h0hi = min(g.nt[0] - 1, kSuper0 * s0 + kSuper0 - 1);
                const int h1lo = max(0, s1 - g.K[1]);
                int ns = 0;
                int64_t cum = 0;
                for (int h0 = h0lo; h0 <= h0hi && ns < kSegMax; ++h0) {
                    const int64_t a0 = off[h0 * nst1 + h1lo], a1 = off[h0 * nst1 + s1 + 1];
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
            asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory");
            const int nseg = nseg_s;
            const int64_t L = (int64_t)seg_cum[nseg];
            const int64_t nch = (L + kStageRec - 1) / kStageRec;
            const int T0 = s0 * kRows, T1 = s1 * kCols;
            int4 pf[sizeof(RecF<2>) / 16];
#pragma unroll
            for (int w = 0; w < (int)(sizeof(RecF<2>) / 16); ++w) pf[w] = make_int4(0, 0, 0, 0);
            auto fetch = [&](int64_t c) {
                const int64_t v = c * kStageRec + tid;
                if (tid < kStageRec && c < nch && v < L) {
                    int lo = 0, hi = nseg - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((int64_t)seg_cum[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    const int64_t idx = (int64_t)seg_start[lo] + (v - (int64_t)seg_cum[lo]);
                    const int4 *src = reinterpret_cast<const int4 *>(recs + idx);
#pragma unroll
                    for (int w = 0; w < (int)(sizeof(RecF<2>) / 16); ++w) pf[w] = __ldg(src + w);
                }
            };
            fetch(split);
            int ci = 0;            // chunk of this item
            int pend = -1;         // a finished phase not yet read back
            int pend_ci = 0;       // its last chunk
            for (int64_t c = split; c < nch; c += nsplit) {
                if (tid < kStageRec) {
                    int4 *dst = reinterpret_cast<int4 *>(srec + tid);
#pragma unroll
                    for (int w = 0; w < (int)(sizeof(RecF<2>) / 16); ++w) dst[w] = pf[w];
                    // the record's phase rotations over 8 grid lines, per dimension
                    const RecF<2> &R = *reinterpret_cast<const RecF<2> *>(pf);
                    float4 rr;
                    float t0 = 8.f * R.nuhi[0];
                    t0 -= rint_fast(t0);
                    sincospif(2.f * fmaf(8.f, R.nulo[0], t0), &rr.y, &rr.x);
                    float t1 = 8.f * R.nuhi[1];
                    t1 -= rint_fast(t1);
                    sincospif(2.f * fmaf(8.f, R.nulo[1], t1), &rr.w, &rr.z);
                    srot[tid] = rr;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory");
                fetch(c + nsplit);
                const int64_t left = L - c * kStageRec;
                const int nrec = left < kStageRec ? (int)left : kStageRec;
                const bool last_block = c + nsplit >= nch;
                for (int sub = 0; sub < nrec; sub += kRec, ++ci, ++gc) {
                    const int s = gc % kStages;
                    stage_free(s);  // the MMAs of chunk gc - kStages are complete
                    // a phase whose last chunk is 3 chunks back: its MMAs are complete
                    if (pend >= 0 && ci >= pend_ci + kStages) {
                        read_acc(pend);
                        pend = -1;
                    }
                    const bool first = ci % kPhase == 0;
                    const bool end = ci % kPhase == kPhase - 1 || (last_block && sub + kRec >= nrec);
                    if (!abort) tc::fill_stage(stages + s * kStageBytes, srec + sub, srot + sub, min(kRec, nrec - sub),
                                               T0, T1, P);
                    if (tid == 0) info[s] = ChunkInfo{phase, first ? 1 : 0, end ? 1 : 0, 0};
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(&full[s]);
                    if (end) {
                        if (pend >= 0) {  // (a phase of fewer than kStages chunks follows another)
                            read_acc(pend);
                        }
                        pend = phase;
                        pend_ci = ci;
                        ++phase;
                    }
                }
                if (producers_sync_or(abort)) abort = true;  // srec is restaged next
                if (abort) break;
            }
            if (abort) break;
            if (ci > 0) {
                if (pend >= 0) read_acc(pend);
                if (reader && !abort) {
                    const int64_t gi = (int64_t)s0 * kRows + 32 * q + lane;
                    if (gi < g.n[0]) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int64_t gj = (int64_t)s1 * kCols + 8 * cg + k;
                            if (gj < g.n[1]) atomic_add_c(u + gi * g.n[1] + gj, acc_re[k], acc_im[k]);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) acc_re[k] = acc_im[k] = 0.f;
            }
        }
        // tell the MMA warp to stop
        if (!abort) {
            const int s = gc % kStages;
            stage_free(s);
            if (tid == 0) info[s] = ChunkInfo{0, 0, 0, 1};
            bar_arrive(&full[s]);
        }
        if (abort) {
            s_abort = 1;
            if (tid == 0) atomicExch(err, 1);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}
