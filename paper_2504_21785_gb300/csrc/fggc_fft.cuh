// K5 on commensurate meshes: the grid stage of eq. 2.24 with the sum over the
// p-nodes of each q-node done by an inverse DFT (the route Sec. 2.3 and
// Remark 3 point to for the on-grid packets).
//
// A pass maps rows [a][b] of the (phase-folded) node array W' to [m]:
//   u[m] = sum_a g(x_m - a dq) sum_b W'[a, b] e^{i b dp x_m / eps}.
// With x_m = lo + m h and h dp / eps = 2 pi / N (N an integer: the mesh is
// commensurate with the grid), e^{i b dp x_m / eps} = e^{i b dp lo / eps}
// e^{2 pi i b m / N}, so for every node a
//   F_a[m mod N] = sum_b (W'[a, b] e^{i b dp lo / eps}) e^{2 pi i b m / N}
// is an N-point inverse DFT of the node's b-vector folded modulo N (exact: the
// kernel is N-periodic in b), and
//   u[m] = sum_{a : m in window(a)} g(x_m - a dq) F_a[m mod N],
// a banded real contraction.  dft_lines_kernel does one radix-2 FFT per
// (row, a) line in shared memory; band_fft_kernel does the contraction.
// Included by fggc.cu inside its anonymous namespace, after the grid-pass
// parameter blocks (PassParams, PassTables) it uses.
#pragma once

// e^{2 pi i j / N}, j < N / 2, evaluated in FP64.
template <class C2>
__global__ void fft_twiddle_kernel(int N, C2 *__restrict__ tw) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N / 2) return;
    double sn, cs;
    sincospi(2.0 * (double)j / (double)N, &sn, &cs);
    C2 v;
    v.x = cs;
    v.y = sn;
    tw[j] = v;
}

__device__ __forceinline__ unsigned bit_reverse(unsigned x, int logn) { return __brev(x) >> (32 - logn); }

// Lines (row, a) of one CTA: 512 / N of them for N <= 512 (N / 2 threads per
// line, one butterfly each per stage), else one.
__host__ __device__ constexpr int dft_lines_per_cta(int logn) { return logn <= 9 ? (1 << (9 - logn)) : 1; }

// Per line: x[k] = sum_{b = k mod N, b in the line's occupied range}
// W'[a, b] e^{2 pi i b th}, th = dp lo / (2 pi eps); then the inverse DFT of
// length N = 2^logn into F[line][0..N).  Lines without contributions (empty
// b-range, or a first-pass row without a flag) get zeros.  256 threads.
template <bool FP64>
__global__ void __launch_bounds__(256) dft_lines_kernel(const void *__restrict__ in_v, void *__restrict__ F_v,
                                                        int64_t rows, int A, int B, int bmin, double th, int logn,
                                                        const int2 *__restrict__ brange,
                                                        const uint8_t *__restrict__ flags,
                                                        const void *__restrict__ tw_v) {
    using Real = typename std::conditional<FP64, double, float>::type;
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    const int N = 1 << logn;
    const int lpc = dft_lines_per_cta(logn);
    const int tpl = blockDim.x / lpc;  // threads per line
    const int sub = threadIdx.x / tpl, t = threadIdx.x - sub * tpl;
    C2 *x = reinterpret_cast<C2 *>(fft_smem) + (int64_t)sub * N;
    const int64_t lines = rows * (int64_t)A;
    const int64_t line = (int64_t)blockIdx.x * lpc + sub;
    const bool here = line < lines;
    const C2 *in = reinterpret_cast<const C2 *>(in_v) + (here ? line : 0) * (int64_t)B;
    C2 *F = reinterpret_cast<C2 *>(F_v) + (here ? line : 0) * (int64_t)N;
    const C2 *tw = reinterpret_cast<const C2 *>(tw_v);
    int lo = 0, hi = B - 1;
    if (here && brange) {
        const int2 r = brange[line];
        lo = r.x;
        hi = r.y;
    }
    const bool active = here && !(flags && !flags[line / A]) && lo <= hi;
    C2 zero;
    zero.x = 0;
    zero.y = 0;
    // fold the occupied b-range modulo N (thread per residue: no collisions)
    for (int k = t; k < N; k += tpl) {
        Real sr = 0, si = 0;
        if (active) {
            const int b_lo = bmin + lo, b_hi = bmin + hi;
            for (int b = b_lo + ((k - b_lo) % N + N) % N; b <= b_hi; b += N) {
                const C2 w = in[b - bmin];
                if (w.x == 0 && w.y == 0) continue;
                double tt = (double)b * th;
                tt -= rint(tt);
                Real sn, cs;
                if constexpr (FP64) {
                    sincospi(2.0 * tt, &sn, &cs);
                } else {
                    sincospif(2.f * (float)tt, &sn, &cs);
                }
                sr += w.x * cs - w.y * sn;
                si += w.x * sn + w.y * cs;
            }
        }
        C2 v;
        v.x = sr;
        v.y = si;
        x[bit_reverse((unsigned)k, logn)] = v;
    }
    __syncthreads();
    // radix-2 butterflies, decimation in time (bit-reversed input, natural order out)
    for (int s = 1; s <= logn; ++s) {
        const int half = 1 << (s - 1);
        const int stride = N >> s;  // twiddle index step
        if (active) {
            for (int i = t; i < N / 2; i += tpl) {
                const int grp = i >> (s - 1), pos = i & (half - 1);
                const int i0 = (grp << s) + pos, i1 = i0 + half;
                const C2 w = tw[pos * stride];
                const C2 u = x[i0], v = x[i1];
                C2 vt;
                vt.x = v.x * w.x - v.y * w.y;
                vt.y = v.x * w.y + v.y * w.x;
                C2 r0, r1;
                r0.x = u.x + vt.x;
                r0.y = u.y + vt.y;
                r1.x = u.x - vt.x;
                r1.y = u.y - vt.y;
                x[i0] = r0;
                x[i1] = r1;
            }
        }
        __syncthreads();
    }
    if (here)
        for (int k = t; k < N; k += tpl) F[k] = active ? x[k] : zero;
}

// u[row][m] = sum over the tile's node band of g(x_m - a dq) F[row][a][m mod N]
// (nodes whose window holds m); one grid point per thread, 128 per CTA.
template <bool FP64>
__global__ void __launch_bounds__(128) band_fft_kernel(const void *__restrict__ F_v, void *__restrict__ out_v,
                                                       PassParams pp, int logn, const PassTables tab) {
    using C2 = typename std::conditional<FP64, double2, float2>::type;
    const int64_t row = blockIdx.x;
    const int64_t m = (int64_t)blockIdx.y * 128 + threadIdx.x;
    if (m >= pp.N) return;
    const int N = 1 << logn;
    const int mf = (int)(m & (N - 1));
    const C2 *F = reinterpret_cast<const C2 *>(F_v) + row * (int64_t)pp.A * N;
    const int2 bnd = tab.band[blockIdx.y];
    const double xm = grid_x(pp.lo, pp.h, m);
    double sr = 0, si = 0;
    float fr = 0.f, fi = 0.f;
    const float cef = (float)(pp.neg_half_inv_eps * 1.4426950408889634);  // log2(e) / (-2 eps)
    for (int a = bnd.x; a <= bnd.y; ++a) {
        const int ia = a - pp.amin;
        const int2 w = tab.win[ia];
        if (m < w.x || m > w.y) continue;
        const C2 v = F[(int64_t)ia * N + mf];
        const double dx = xm - (double)a * pp.dq;
        if constexpr (FP64) {
            const double g = exp(dx * dx * pp.neg_half_inv_eps);
            sr += g * v.x;
            si += g * v.y;
        } else {
            const float dxf = (float)dx;
            const float g = ex2_approx(dxf * dxf * cef);
            fr = fmaf(g, v.x, fr);
            fi = fmaf(g, v.y, fi);
        }
    }
    C2 o;
    if constexpr (FP64) {
        o.x = sr;
        o.y = si;
    } else {
        o.x = fr;
        o.y = fi;
    }
    reinterpret_cast<C2 *>(out_v)[row * pp.N + m] = o;
}

