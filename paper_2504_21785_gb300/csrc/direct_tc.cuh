// K2 on the fifth-generation tensor cores (FP32 records, d = 2 and 3).
//
// The separable form of the direct sum (eq. 2.10 with the box window): a
// packet's term on the grid is the product of its per-dimension factors,
//   F_l,r(x) = g_r(x - Q_l) e^{i P_l (x - Q_l) / eps}, zero outside the window,
// with pref A_r e^{i S_r / eps} folded into dimension 0.  A super tile of 128
// "rows" x 64 lines of the last dimension is a complex matrix product over the
// records r of its list, U = F_row F_last^T: d = 2, rows = 128 lines of
// dimension 0 (four tiles of the binning); d = 3, rows = the 8 x 16 (i, j)
// pairs of dimensions 0 and 1 (one tile x two tiles) with F_row = F_0 F_1; the
// last dimension spans two tiles (d = 2) or four (d = 3).  It runs as one real
// product on tcgen05.mma (kind::tf32, M = 128, N = 128, K = 8 per instruction):
//   A[row][2r + c]  = (Re F_row, Im F_row)[c]
//   B[j][2r + c]    = (Re F_last,r[j], -Im F_last,r[j])[c]   (row j: the real part)
//   B[64 + j][..]   = (Im F_last,r[j],  Re F_last,r[j])[c]   (row 64 + j: the imaginary part)
// so D[row][j] = Re u and D[row][64 + j] = Im u, accumulated in tensor memory.
// N = 128 rather than 64: an MMA of N = 64 takes 48 clocks against 64 at
// N = 128 (twice the work), and a wider last dimension lists each record in
// fewer super tiles.
// FP32 accuracy from TF32 operands: every factor x is split into x_hi (x
// truncated to TF32) and x_lo = x - x_hi, and D += A_lo B_hi + A_hi B_lo +
// A_hi B_hi (three instructions per K step; the dropped A_lo B_lo and the
// truncation of x_lo to TF32 are below 2^-20 of a product each).
//
// Pipeline: a persistent CTA takes (super tile, slice) items from a device
// counter.  20 producer warps stage the records 256 at a time (the next 256
// are loaded into registers while the current ones are used; each record's
// phase rotation over 8 grid lines of the dimensions tabulated with stride 8 is
// computed once when it is staged, and for d = 3 the factors of dimensions 0
// and 1 on the super tile's 8 + 16 lines too); for every 16 records they write
// the operands (hi and lo) into one of three (d = 2) or two (d = 3) stages in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes; 128 bytes between core matrices along K, 1024 bytes between 8-row
// groups) and arrive on the stage's "full" mbarrier; one MMA warp waits on it,
// issues the 12 MMAs and commits them to the stage's "empty" mbarrier, which
// the producers wait on before they reuse the stage.  Operands: per thread and
// chunk, warps 0-15 take four A rows (one record, the rows i0 + 8m, so the 16
// lanes of a half warp store 16 distinct 8-byte words of one 128-byte core
// matrix) and warps 16-19 eight lines of the last dimension (one record, the
// lines j0 + 8m, the same pattern).  A factor along a stride-8 run of lines is evaluated in full at
// the first line inside the window (ex2 and sincos) and by the exact
// recurrences over 8 grid lines after it (Gaussian ratio
// 2^{ce h (16 dx + 64 h)}, itself multiplied by e^{-64 h^2 / eps} per step;
// phase rotation e^{2 pi i 8 nu}); the d = 3 tables of dimensions 0 and 1 use
// the same recurrences over single grid steps.
//
// Accumulation: the tensor core adds into its FP32 accumulator with truncated
// alignment, so no accumulator sums more than 4 chunks (64 records, 48
// instructions): chunks 4k..4k+3 of an item go to TMEM accumulator k mod 2
// (committed to that accumulator's "full" mbarrier after its last chunk), and
// while the next chunks fill the other one, warps 0-15 add the finished one
// (tcgen05.ld, one row per lane, 16 complex columns per warp, 8 TMEM columns
// at a time) to the item's FP32 running sums, which live in a third TMEM
// region (tcgen05.st), and arrive on its "empty" mbarrier, which the MMA warp
// waits on before it starts the accumulator again.  At the end of an item the
// running sums are added to the zeroed output with float2 atomics.
//
// Waits on the mbarriers are bounded: on expiry the CTA sets *err, stops
// taking items and releases its tensor memory.
// Included by direct.cu inside its anonymous namespace.
#pragma once

namespace tc {

// super tile: tiles of the binning per dimension
template <int D>
__host__ __device__ constexpr int tc_span(int l) {
    return D == 2 ? (l == 0 ? 4 : 2) : (l == 0 ? 1 : (l == 1 ? 2 : 4));
}
template <int D>
__host__ __device__ constexpr int tc_lines(int l) {
    return tc_span<D>(l) * tileT<D>(l);
}
constexpr int kRows = 128;                       // M: rows of a super tile
constexpr int kCols = 64;                        // lines of the last dimension per super tile
static_assert(tc_lines<2>(0) == kRows && tc_lines<2>(1) == kCols, "2-D super tile");
static_assert(tc_lines<3>(0) * tc_lines<3>(1) == kRows && tc_lines<3>(1) == 16 && tc_lines<3>(2) == kCols,
              "3-D super tile");
constexpr int kN = 2 * kCols;                    // N: real and imaginary outputs
constexpr int kRec = 16;                         // records per MMA chunk
constexpr int kK = 2 * kRec;                     // TF32 elements of K per chunk
constexpr int kGenThreads = 640;                 // producers: 16 warps for the rows, 4 for the last dimension
constexpr int kThreadsTc = kGenThreads + 32;     // + one warp that issues the MMAs
constexpr int kStageRec = 256;                   // records staged in shared memory at a time
constexpr int kPhase = 4;                        // chunks summed in one TMEM accumulator
constexpr int kABytes = kRows * kK * 4;          // 16 KB
constexpr int kBBytes = kN * kK * 4;             // 16 KB
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr int kMaxStages = 3;
// operand stages: three for d = 2; two for d = 3, whose factor tables take
// the shared memory of the third
template <int D>
__host__ __device__ constexpr int tc_stages() {
    return D == 2 ? 3 : 2;
}
constexpr int kTmemCols = 4 * kN;                // two accumulators, the running sums, one unused
constexpr int kSegMax = 256;                     // runs of home tiles in a super tile's list
constexpr int kF01 = 8 + 16;                     // d = 3: factor lines of dimensions 0 and 1 per record
constexpr unsigned kWaitLimit = 1u << 24;        // polls of an mbarrier before giving up
template <int D>
constexpr size_t dyn_smem() {
    return (size_t)tc_stages<D>() * kStageBytes + (size_t)kStageRec * (sizeof(RecF<D>) + sizeof(float4)) +
           (D == 3 ? (size_t)kStageRec * kF01 * sizeof(float2) : 0);
}
static_assert(kTmemCols == 512, "two accumulators and the running sums of N 32-bit columns each");
static_assert(dyn_smem<2>() + 4096 <= 227 * 1024 && dyn_smem<3>() + 4096 <= 227 * 1024, "shared memory of one CTA");

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 128, M = 128
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

// x truncated to TF32 (10 explicit mantissa bits): the 13 dropped bits cleared
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

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

__device__ __forceinline__ void tmem_st8(unsigned taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of the warp's 32 lanes (one row per lane)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Factor of dimension l of record R at the grid lines k0 + S m, m = 0..NL-1
// (zero outside the window), each handed to sink(m, value) as soon as it is
// known; rot = e^{2 pi i S nu_l} and qs = e^{-S^2 h^2 / eps}; fold: dimension 0
// carries log2|pref A| and the phase of pref A e^{i theta} at the window
// start.  The first line inside the window (kf0 is integral) is evaluated in
// full, the next by the recurrences.
template <int D, int S, int NL, class Sink>
__device__ __forceinline__ void factor_run_to(const RecF<D> &R, const int l, const int k0, const float2 rot,
                                              const float qs, const DirectParams &P, const bool fold, Sink sink) {
    const float kf0 = (float)k0 - R.mlo[l];
    const float wl = R.wlen[l];
    const int m0 = kf0 >= 0.f ? 0 : (S == 1 ? (int)(-kf0) : (int)ceilf(-kf0 * (1.f / S)));
    float vr = 0.f, vi = 0.f, rho = 0.f;
    const bool any = m0 < NL && kf0 + (float)(S * m0) < wl;
    if (any) {
        const float h = P.hf[l];
        const float kf = kf0 + (float)(S * m0);
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
        rho = ex2_approx(P.ce * h * (float)S * fmaf(2.f, dx, (float)S * h));
    }
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        const bool in = any && m >= m0 && kf0 + (float)(S * m) < wl;
        sink(m, in ? make_float2(vr, vi) : make_float2(0.f, 0.f));
        if (m < NL - 1 && m >= m0) {
            const float pr = rot.x * rho, pi = rot.y * rho;
            const float nr = vr * pr - vi * pi;
            vi = vr * pi + vi * pr;
            vr = nr;
            rho *= qs;
        }
    }
}

// factor_run_to into an array
template <int D, int S, int NL>
__device__ __forceinline__ void factor_run(const RecF<D> &R, const int l, const int k0, const float2 rot,
                                           const float qs, const DirectParams &P, const bool fold, float2 *out) {
    factor_run_to<D, S, NL>(R, l, k0, rot, qs, P, fold, [&](int m, float2 v) { out[m] = v; });
}

// hi and lo TF32 parts of a complex value: hi = x truncated to TF32, lo = x - hi
// (exact in FP32; the tensor core reads its leading 11 bits, so lo is
// truncated once more there): |x - hi - lo_tf32| < 2^-20 |x|
__device__ __forceinline__ void split_c(const float2 v, float2 &hi, float2 &lo) {
    hi = make_float2(tf32_trunc(v.x), tf32_trunc(v.y));
    lo = make_float2(v.x - hi.x, v.y - hi.y);
}

// Writes the operands of records rec[0 .. nrec-1] (zeros for r >= nrec) into
// one stage: A_hi, A_lo (128 x kK), B_hi, B_lo (128 x kK); per thread one
// unit of four rows (A) or eight lines of the last dimension (B).  rot[r]: e^{2 pi i 8 nu} of dimension 0 (.x, .y;
// d = 2) and of the last dimension (.z, .w); f01[r] (d = 3): the record's
// factors on the super tile's 8 lines of dimension 0 and 16 of dimension 1.
template <int D>
__device__ __forceinline__ void fill_stage(unsigned char *stage, const RecF<D> *rec, const float4 *rot,
                                           const float2 *f01, const int nrec, const int *T,
                                           const DirectParams &P) {
    const int tid = threadIdx.x;
    float2 f[4];
    if (tid < 512) {
        // rows 32 blk + (tid & 7) + 8 m of record 2 (tid >> 5 & 7) + (tid >> 3 & 1),
        // blk = 2 (tid >> 8) + (tid >> 4 & 1)
        const int r = 2 * ((tid >> 5) & 7) + ((tid >> 3) & 1);
        const int i0 = 32 * (2 * (tid >> 8) + ((tid >> 4) & 1)) + (tid & 7);
        if (r < nrec) {
            if (D == 2) {
                const float4 rr = rot[r];
                factor_run<D, 8, 4>(rec[r], 0, T[0] + i0, make_float2(rr.x, rr.y), P.q8[0], P, true, f);
            } else {
                // row = 16 i + j: F_0[i] F_1[j] from the record's tables
                const float2 *F = f01 + r * kF01;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int row = i0 + 8 * m;
                    const float2 a = F[row >> 4], b = F[8 + (row & 15)];
                    f[m] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) f[m] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned o = kmaj(i0 + 8 * m, 2 * r);
            float2 hi, lo;
            split_c(f[m], hi, lo);
            *reinterpret_cast<float2 *>(stage + o) = hi;
            *reinterpret_cast<float2 *>(stage + kABytes + o) = lo;
        }
    } else {
        // last dimension: record v >> 3, lines (v & 7) + 8 m, m = 0..7
        const int v = tid - 512;
        const int r = v >> 3, j0 = v & 7;
        unsigned char *Bh = stage + 2 * kABytes;
        unsigned char *Bl = Bh + kBBytes;
        auto put = [&](int m, float2 val) {
            const int j = j0 + 8 * m;
            const unsigned o_re = kmaj(j, 2 * r), o_im = kmaj(kCols + j, 2 * r);
            float2 hi, lo;
            split_c(val, hi, lo);
            *reinterpret_cast<float2 *>(Bh + o_re) = make_float2(hi.x, -hi.y);
            *reinterpret_cast<float2 *>(Bh + o_im) = make_float2(hi.y, hi.x);
            *reinterpret_cast<float2 *>(Bl + o_re) = make_float2(lo.x, -lo.y);
            *reinterpret_cast<float2 *>(Bl + o_im) = make_float2(lo.y, lo.x);
        };
        if (r < nrec) {
            const float4 rr = rot[r];
            factor_run_to<D, 8, 8>(rec[r], D - 1, T[D - 1] + j0, make_float2(rr.z, rr.w), P.q8[D - 1], P, false, put);
        } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) put(m, make_float2(0.f, 0.f));
        }
    }
}

// Super tile coordinates of linear index t (row-major over the super tiles).
template <int D>
__device__ __forceinline__ void super_coords(const GridDev &g, int t, int *s) {
#pragma unroll
    for (int l = D - 1; l >= 0; --l) {
        const int n = (g.nt[l] + tc_span<D>(l) - 1) / tc_span<D>(l);
        s[l] = t % n;
        t /= n;
    }
}

// Home-tile box of super tile s: lo[l] .. hi[l] per dimension.
template <int D>
__device__ __forceinline__ void super_box(const GridDev &g, const int *s, int *lo, int *hi) {
#pragma unroll
    for (int l = 0; l < D; ++l) {
        lo[l] = max(0, tc_span<D>(l) * s[l] - g.K[l]);
        hi[l] = min(g.nt[l] - 1, tc_span<D>(l) * s[l] + tc_span<D>(l) - 1);
    }
}

// Record range of the r-th run (along the last dimension) of the box.
template <int D>
__device__ __forceinline__ void box_run(const GridDev &g, const int64_t *off, const int *lo, const int *hi, int r,
                                        int64_t *a0, int64_t *a1) {
    int h[D];
#pragma unroll
    for (int l = D - 2; l >= 0; --l) {
        const int cnt = hi[l] - lo[l] + 1;
        h[l] = lo[l] + r % cnt;
        r /= cnt;
    }
    h[D - 1] = lo[D - 1];
    const int first = tile_linear<D>(g, h);
    *a0 = off[first];
    *a1 = off[first + hi[D - 1] - lo[D - 1] + 1];
}

template <int D>
__device__ __forceinline__ int box_runs(const int *lo, const int *hi) {
    int rows = 1;
#pragma unroll
    for (int l = 0; l < D - 1; ++l) rows *= hi[l] - lo[l] + 1;
    return rows;
}

}  // namespace tc

// Records in the list of every super tile (union of the home-tile boxes of its
// tiles).
template <int D>
__global__ void tc_tile_load_kernel(const int64_t *__restrict__ off, GridDev g, int nst,
                                    uint32_t *__restrict__ load) {
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile >= nst) return;
    int s[D], lo[D], hi[D];
    tc::super_coords<D>(g, tile, s);
    tc::super_box<D>(g, s, lo, hi);
    int64_t sum = 0;
    const int runs = tc::box_runs<D>(lo, hi);
    for (int r = 0; r < runs; ++r) {
        int64_t a0, a1;
        tc::box_run<D>(g, off, lo, hi, r, &a0, &a1);
        sum += a1 - a0;
    }
    load[tile] = (uint32_t)(sum < 0xffffffffLL ? sum : 0xffffffffLL);
}

// what the MMA warp needs to know about the chunk in a stage, in one word:
// bits 0-27 the accumulator phase (accumulator = phase & 1); bit 28: first
// chunk of the phase (the first MMA overwrites the accumulator); bit 29: last
// chunk of the phase (commit the accumulator's barrier too); bit 30: no more
// chunks
constexpr unsigned kInfoFirst = 1u << 28, kInfoEnd = 1u << 29, kInfoStop = 1u << 30;

// Bounded wait that also gives up once another thread has reported a failure.
// SLEEP (the producers): back off after every failed poll, so that waiting
// warps leave the issue slots to the MMA warp, which polls without a pause.
template <bool SLEEP>
__device__ __forceinline__ bool bar_wait_or_abort(uint64_t *bar, unsigned parity, const volatile int *abort) {
    for (unsigned it = 0; it < tc::kWaitLimit; ++it) {
        if (tc::bar_try(bar, parity)) return true;
        if ((it & 63) == 63 && *abort) return false;
        if (SLEEP) __nanosleep(64);
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
template <int D>
__global__ void __launch_bounds__(tc::kThreadsTc, 1)
    direct_tc_kernel(const RecF<D> *__restrict__ recs, const int64_t *__restrict__ off, DirectParams P,
                     float2 *__restrict__ u, const int2 *__restrict__ items, const int *__restrict__ n_items,
                     unsigned long long *__restrict__ counter, const volatile int *yield, int keep,
                     int *__restrict__ err) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *stages = smem;
    constexpr int kStages = tc_stages<D>();
    RecF<D> *srec = reinterpret_cast<RecF<D> *>(smem + kStages * kStageBytes);
    float4 *srot = reinterpret_cast<float4 *>(smem + kStages * kStageBytes + kStageRec * sizeof(RecF<D>));
    float2 *f01 = reinterpret_cast<float2 *>(srot + kStageRec);  // d = 3
    __shared__ uint32_t seg_start[kSegMax];
    __shared__ uint32_t seg_cum[kSegMax + 1];
    __shared__ int nseg_s;
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2];
    __shared__ unsigned info[kMaxStages];
    __shared__ unsigned s_tmem;
    __shared__ long long s_item;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GridDev &g = P.g;
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
            int s = 0;
            unsigned fpar = 0;  // parity of full[s]'s phase for this pass over the stages
            for (;;) {
                if (!bar_wait_or_abort<false>(&full[s], fpar, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                const unsigned ci = *const_cast<const volatile unsigned *>(&info[s]);
                if (ci & kInfoStop) break;
                const int phase = (int)(ci & (kInfoFirst - 1));
                const bool first = (ci & kInfoFirst) != 0;
                const int a = phase & 1;
                if (first && phase >= 2 &&
                    !bar_wait_or_abort<false>(&acc_empty[a], ((phase >> 1) - 1) & 1, &s_abort)) {
                    s_abort = 1;
                    break;
                }
                fence_after();
                // descriptors of the stage's four operands; a K step of 8 TF32
                // (256 bytes) adds 16 to the start-address field
                const unsigned sa = saddr(stages + s * kStageBytes);
                const uint64_t ah = sdesc(sa), al = sdesc(sa + kABytes);
                const uint64_t bh = sdesc(sa + 2 * kABytes), bl = sdesc(sa + 2 * kABytes + kBBytes);
                const unsigned d = tmem + (unsigned)(a * kN);
#pragma unroll
                for (int ks = 0; ks < kK / 8; ++ks) {
                    const uint64_t o = 16u * ks;
                    mma_tf32(d, al + o, bh + o, (first && ks == 0) ? 0u : 1u);
                    mma_tf32(d, ah + o, bl + o, 1u);
                    mma_tf32(d, ah + o, bh + o, 1u);
                }
                mma_commit(&empty[s]);
                if (ci & kInfoEnd) mma_commit(&acc_full[a]);
                if (++s == kStages) {
                    s = 0;
                    fpar ^= 1u;
                }
            }
        }
    } else {
        // ---- producers and accumulator readers ----
        uint32_t gc = 0;   // chunks produced by this CTA
        int st = 0;        // their stage: gc mod kStages
        unsigned epar = 1; // parity of empty[st]'s phase to wait for (the first pass waits for nothing)
        int phase = 0;     // accumulator phases started by this CTA
        bool abort = false;
        const long long total = *n_items;
        // warps 0-15 read the accumulators: lane quarter q (rows 32 q + lane),
        // complex columns kRC cg .. kRC cg + kRC - 1; the item's running sums
        // stay in TMEM columns [2 kN, 3 kN) of the same lanes
        const int q = warp & 3, cg = (warp >> 2) & 3;
        const bool reader = warp < 16;
        constexpr int kRC = kCols / 4;  // complex columns per reader
        const unsigned lanes = tmem + ((unsigned)(32 * q) << 16);
        const unsigned run = lanes + 2 * kN;
        bool fresh = true;              // the item's first read-back stores instead of adding
        auto read_acc = [&](int ph) {
            if (!reader || abort) return;
            const int a = ph & 1;
            if (!bar_wait_or_abort<true>(&acc_full[a], (ph >> 1) & 1, &s_abort)) {
                abort = true;
                s_abort = 1;
                return;
            }
            fence_after();
            const unsigned acc = lanes + (unsigned)(a * kN);
#pragma unroll
            for (int part = 0; part < 2 * kRC / 8; ++part) {
                const unsigned col = (part / (kRC / 8)) * kCols + kRC * cg + 8 * (part % (kRC / 8));
                float p[8], r[8];
                tmem_ld8(acc + col, p);
                if (!fresh) tmem_ld8(run + col, r);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 8; ++k) r[k] = fresh ? p[k] : r[k] + p[k];
                tmem_st8(run + col, r);
            }
            tmem_wait_st();
            fresh = false;
            fence_before();
            bar_arrive(&acc_empty[a]);
        };
        // waits for stage s to be free and hands chunk info over with the stage
        auto stage_free = [&](int s) {
            if (gc >= (uint32_t)kStages && !abort && !bar_wait_or_abort<true>(&empty[s], epar, &s_abort)) {
                abort = true;
                s_abort = 1;
            }
        };
        auto next_stage = [&]() {
            ++gc;
            if (++st == kStages) {
                st = 0;
                epar ^= 1u;
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
            int sc[D];
            super_coords<D>(g, it.x, sc);
            if (tid == 0) {  // runs of home tiles along the last dimension
                int lo[D], hi[D];
                super_box<D>(g, sc, lo, hi);
                const int runs = box_runs<D>(lo, hi);
                int ns = 0;
                int64_t cum = 0;
                for (int r = 0; r < runs && ns < kSegMax; ++r) {
                    int64_t a0, a1;
                    box_run<D>(g, off, lo, hi, r, &a0, &a1);
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
            int T[D];
#pragma unroll
            for (int l = 0; l < D; ++l) T[l] = sc[l] * tc_lines<D>(l);
            int4 pf[sizeof(RecF<D>) / 16];
#pragma unroll
            for (int w = 0; w < (int)(sizeof(RecF<D>) / 16); ++w) pf[w] = make_int4(0, 0, 0, 0);
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
                    for (int w = 0; w < (int)(sizeof(RecF<D>) / 16); ++w) pf[w] = __ldg(src + w);
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
                    for (int w = 0; w < (int)(sizeof(RecF<D>) / 16); ++w) dst[w] = pf[w];
                    // the record's phase rotations over 8 grid lines
                    const RecF<D> &R = *reinterpret_cast<const RecF<D> *>(pf);
                    float4 rr = make_float4(1.f, 0.f, 1.f, 0.f);
                    if (D == 2) {
                        float t0 = 8.f * R.nuhi[0];
                        t0 -= rint_fast(t0);
                        sincospif(2.f * fmaf(8.f, R.nulo[0], t0), &rr.y, &rr.x);
                    }
                    float t1 = 8.f * R.nuhi[D - 1];
                    t1 -= rint_fast(t1);
                    sincospif(2.f * fmaf(8.f, R.nulo[D - 1], t1), &rr.w, &rr.z);
                    srot[tid] = rr;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory");
                if (D == 3) {
                    // factors of dimensions 0 and 1 on the super tile's lines: six
                    // units of four consecutive lines per record
                    for (int e = tid; e < kStageRec * 6; e += kGenThreads) {
                        const int r = e / 6, k = e % 6;
                        const int l = k < 2 ? 0 : 1;
                        const int first = l == 0 ? 4 * k : 4 * (k - 2);
                        const RecF<D> &R = srec[r];
                        float t = R.nuhi[l];
                        t -= rint_fast(t);
                        float sn, cs;
                        __sincosf(6.283185307179586f * (t + R.nulo[l]), &sn, &cs);
                        float2 fv[4];
                        factor_run<D, 1, 4>(R, l, T[l] + first, make_float2(cs, sn), P.q_dim[l], P, l == 0, fv);
                        float2 *dst = f01 + r * kF01 + (l == 0 ? 0 : 8) + first;
#pragma unroll
                        for (int m = 0; m < 4; ++m) dst[m] = fv[m];
                    }
                    asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory");
                }
                fetch(c + nsplit);
                const int64_t left = L - c * kStageRec;
                const int nrec = left < kStageRec ? (int)left : kStageRec;
                const bool last_block = c + nsplit >= nch;
                for (int sub = 0; sub < nrec; sub += kRec, ++ci, next_stage()) {
                    const int s = st;
                    stage_free(s);  // the MMAs of chunk gc - kStages are complete
                    // a phase whose last chunk is 3 chunks back: its MMAs are complete
                    if (pend >= 0 && ci >= pend_ci + kStages) {
                        read_acc(pend);
                        pend = -1;
                    }
                    const bool first = ci % kPhase == 0;
                    const bool end = ci % kPhase == kPhase - 1 || (last_block && sub + kRec >= nrec);
                    if (!abort)
                        fill_stage<D>(stages + s * kStageBytes, srec + sub, srot + sub, f01 + sub * kF01,
                                      min(kRec, nrec - sub), T, P);
                    if (tid == 0) info[s] = (unsigned)phase | (first ? kInfoFirst : 0u) | (end ? kInfoEnd : 0u);
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
                    const int row = 32 * q + lane;
                    int64_t gi;
                    bool ok;
                    if (D == 2) {
                        gi = (int64_t)T[0] + row;
                        ok = gi < g.n[0];
                    } else {
                        const int64_t i = (int64_t)T[0] + (row >> 4), j = (int64_t)T[1] + (row & 15);
                        gi = i * g.n[1] + j;
                        ok = i < g.n[0] && j < g.n[1];
                    }
                    fence_after();
#pragma unroll
                    for (int h = 0; h < kRC / 8; ++h) {
                        const unsigned col = kRC * cg + 8 * h;
                        float re[8], im[8];
                        tmem_ld8(run + col, re);
                        tmem_ld8(run + kCols + col, im);
                        tmem_wait_ld();
                        const int64_t gj0 = (int64_t)T[D - 1] + col;
                        if (ok) {
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                if (gj0 + k < g.n[D - 1])
                                    atomic_add_c(u + gi * g.n[D - 1] + gj0 + k, re[k], im[k]);
                        }
                    }
                    fence_before();
                }
                fresh = true;
            }
        }
        // tell the MMA warp to stop
        if (!abort) {
            const int s = st;
            stage_free(s);
            if (tid == 0) info[s] = kInfoStop;
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
