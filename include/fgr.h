/*
 * fgr.h -- frozen Gaussian reconstruction on one GB300 (sm_103a).
 *
 * C ABI of libfgr.so.  The library computes the hot path of the frozen Gaussian
 * grid-point correction (FGGC) of Chai & Deng, "Frozen Gaussian Grid-point
 * Correction For Semi-classical Schroedinger Equation":
 *
 *   fgr_propagate           per-packet Hamiltonian flow of Q, P, S and A (eq. 2.3-2.7)
 *   fgr_reconstruct_direct  windowed direct sum of the packets on a grid (eq. 2.10)
 *   fgr_reconstruct_fggc    least-squares on-grid correction (Algorithm 2,
 *                           eq. 2.21-2.25 with eq. 3.13 / 3.22 / 3.23)
 *   fgr_submit / fgr_poll   continuous-batching server over resident packet sets
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: per dimension l < d, x_{m,l} = lo[l] + m*(hi[l]-lo[l])/n[l], m in [0, n[l]);
 *   outputs are row-major with the last dimension fastest.  Free space: points
 *   outside [lo, hi) do not exist and nothing wraps around.
 * Mesh (eq. 3.5): dq = cq*sqrt(eps), dp = cp*sqrt(eps).
 * Prefactor (eq. 2.10): (dq dp)^d / (2 pi eps)^{3d/2}; the library applies it.
 * Window: each Gaussian is summed over the box |x_l - Q_l| <= R sqrt(eps),
 *   decided in FP64 as m_lo = ceil(((Q - R sqrt(eps)) - lo)/h),
 *   m_hi = floor(((Q + R sqrt(eps)) - lo)/h), clipped to the grid.
 * Packets: structure of arrays, FP64, caller-owned:
 *   q[d*m], p[d*m] dimension-major (q[l*m + j]); s[m]; a[2*m] (real plane, then
 *   imaginary plane).  on_device = 1: CUDA device pointers; 0: host pointers
 *   (the library copies in and, for fgr_propagate, back out).
 * Output u_out: interleaved complex, complex128 for FGR_FP64 and complex64 for
 *   FGR_FP32, n[0]*...*n[d-1] values.  Device or host memory (detected); the
 *   caller owns it.  On error its contents are undefined.
 * Streams: the cuda_stream argument is a cudaStream_t.  Work is stream-ordered
 *   and the call returns once it is enqueued, except that (a) host inputs or
 *   outputs, (b) fgr_reconstruct_fggc's sizing of its node array, and (c) a NULL
 *   stream make the call wait for its own work.
 * Errors: invalid arguments return FGR_E_INVALID before any launch.  CUDA
 *   failures return FGR_E_CUDA.  fgr_last_error() gives a message for the
 *   calling thread, valid until that thread's next call.  No C++ exception
 *   crosses this interface.
 * Threads: one fgr_ctx must not be used by two threads at once.  A server is
 *   safe to call from any number of threads.
 */
#ifndef FGR_H
#define FGR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FGR_OK = 0,
    FGR_E_INVALID = 1,   /* bad argument; nothing was launched */
    FGR_E_NOMEM = 2,     /* device or host allocation failed */
    FGR_E_CUDA = 3,      /* a CUDA call failed; see fgr_last_error() */
    FGR_E_NOT_READY = 4, /* fgr_poll: request still running */
    FGR_E_TIMEOUT = 5,   /* a bounded wait ran out */
    FGR_E_CAPACITY = 6,  /* the request does not fit the configured memory budget */
    FGR_E_CANCELLED = 7, /* the request was cancelled or the server shut down */
    FGR_E_INTERNAL = 8   /* library bug */
} fgr_status;

#define FGR_MAX_DIM 3

typedef struct fgr_ctx fgr_ctx;       /* opaque, library-owned */
typedef struct fgr_server fgr_server; /* opaque, library-owned */

typedef struct {
    int32_t d;                /* 1, 2 or 3 */
    int32_t reserved;
    int64_t n[FGR_MAX_DIM];   /* points per dimension, >= 1 */
    double lo[FGR_MAX_DIM];   /* first point */
    double hi[FGR_MAX_DIM];   /* end of the half-open interval, > lo */
} fgr_grid;

typedef enum { FGR_FP64 = 0, FGR_FP32 = 1 } fgr_precision;

typedef struct {
    double cq, cp;      /* mesh constants of eq. 3.5; defaults 1/2 and pi/8 */
    int32_t nq, np;     /* q- and p-shifts per dimension (Def. 1): 2 -> {0,1},
                           4 -> {-1,0,1,2}; defaults 4 and 2 */
    double window_r;    /* R of the box window; 0 -> 8 (FP64) or 6 (FP32) */
    double rcond;       /* relative singular-value cut-off of the pseudo-inverse
                           (Remark 2); 0 -> 1e-14 */
    int32_t precision;  /* fgr_precision; FP64 default */
    int32_t flags;      /* FGR_FLAG_* bits, 0 by default */
} fgr_options;
/* Option flags.
 * FGR_FLAG_FFT_GRID: FGGC's grid stage (eq. 2.24) evaluates the sum over the
 *   p-nodes of every q-node by an inverse DFT, the route of Sec. 2.3 (after
 *   eq. 2.25) and Remark 3 for meshes commensurate with the grid: with
 *   x_m = lo + m h, e^{i b dp x_m / eps} = e^{i b dp lo / eps} e^{2 pi i b m / N}
 *   when h dp / eps = 2 pi / N.  fgr_create returns FGR_E_INVALID unless, in
 *   every dimension, N = 2 pi eps / (h dp) is a power of two in [8, 8192]
 *   (relative tolerance 1e-9); the meshes of Sec. 4.4 (h = eps, dp =
 *   pi sqrt(eps) / 8, so N = 16 / sqrt(eps)) are.  Same results as the direct
 *   grid stage up to rounding.  fgr_reconstruct_fggc_noalloc ignores the flag.
 * FGR_FLAG_SNAP_CP: before anything else, cp is replaced by the nearest value
 *   that makes dimension 0 commensurate (N a power of two, as above); the
 *   least-squares constants (Tables 1-4) then belong to that cp.
 * FGR_FLAG_DIRECT_FMA: the FP32 direct sum of a 2-D context runs on the
 *   CUDA cores (one complex multiply-add per packet-point pair) instead of the
 *   tensor cores (the outer products of eq. 2.10's per-dimension factors as a
 *   3 x TF32 matrix product); both meet the FP32 tolerance. */
#define FGR_FLAG_FFT_GRID 1
#define FGR_FLAG_SNAP_CP 2
#define FGR_FLAG_DIRECT_FMA 4


typedef struct {
    int64_t m;          /* number of packets, >= 0 */
    double *q, *p;      /* [d][m] */
    double *s;          /* [m] */
    double *a;          /* [2][m] */
    int32_t on_device;  /* 1: device pointers, 0: host pointers */
    int32_t reserved;
} fgr_packets;

typedef enum { FGR_V_FREE = 0, FGR_V_COSSUM = 1, FGR_V_HARMONIC = 2 } fgr_potential_kind;

/* Separable potentials:  FREE  V = 0;
 *   COSSUM    V = c0 + amp * sum_l cos(k x_l);
 *   HARMONIC  V = omega^2 |x|^2 / 2. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double c0, amp, k, omega;
} fgr_potential;

/* Fills *opt with the defaults listed in fgr_options. */
fgr_status fgr_default_options(fgr_options *opt);

/* Creates a context for one (d, grid, eps, options) problem.  Precomputes the
 * eps-free Gram matrix of eq. 3.22 for the chosen neighbour strategy and its
 * pseudo-inverse by an eigen-decomposition (the Gram is Hermitian positive
 * semi-definite, so this is its SVD; Remark 2, Algorithm 2 Step 0), on the host
 * in extended precision (cached per strategy, so later contexts with the same
 * mesh constants and strategy reuse it).  Binds to the current CUDA device.
 * opt may be NULL (defaults).  *out receives the context; free it with
 * fgr_destroy.  FGR_E_INVALID if d is not in 1..3, grid->d != d, eps <= 0 or
 * not finite, any n < 1, hi <= lo, or the options are out of range. */
fgr_status fgr_create(int32_t d, const fgr_grid *grid, double eps, const fgr_options *opt,
                      fgr_ctx **out);

/* Frees the context; NULL is a no-op.  Work already enqueued by the context
 * completes normally (scratch memory is stream-ordered and returns to a
 * per-device pool shared by all contexts). */
void fgr_destroy(fgr_ctx *ctx);

/* Message describing the calling thread's last failure ("" if none). */
const char *fgr_last_error(void);

/* Eq. 2.3-2.7: integrates every packet from 0 to t with the classical RK4
 * scheme, nsteps = round(t/dt) when t/dt is within 1e-9 of an integer (else
 * ceil(t/dt)), step length t/nsteps, all in FP64.  On entry q, p, s, a hold
 * Q(0) = q, P(0) = p, S(0) (normally 0) and A(0); the Jacobians start at the
 * identity (Z(0) = 2I).  On return they hold Q, P, S, A at time t (in place).
 * FGR_E_INVALID if t < 0, dt <= 0, or the potential kind is unknown. */
fgr_status fgr_propagate(fgr_ctx *ctx, fgr_packets *inout, const fgr_potential *v, double t,
                         double dt, void *cuda_stream);

/* Eq. 2.6 and 2.8 (Step 1 of Algorithms 1-3): the initial decomposition of a
 * wave u given on the context's grid (complex128 for FP64 contexts, complex64
 * for FP32, row-major, last dimension fastest; host or device memory).  For
 * every packet j of inout, whose q and p are read, it writes
 *   a_j = 2^{d/2} prod_l h_l sum_m u(x_m) exp(-i p_j.(x_m - q_j)/eps - |x_m - q_j|^2/(2 eps))
 * (the rectangle rule of eq. 2.8 on the grid) over the same box window
 * |x_l - q_l| <= R sqrt(eps) as the reconstructions, and s_j = 0; packets
 * whose window misses the grid get a_j = 0.  FP64: every term in FP64.  FP32:
 * the phase is reduced in FP64 per packet, each term evaluated in FP32 (d = 1:
 * every eighth point along the lane's stride by ex2 and sincos, the others by
 * the exact recurrences of the Gaussian and the phase; d = 2, 3: per-dimension
 * factors, since the term factorises), compensated FP32 sums.  Host packets
 * are copied back before the call returns.  FGR_E_INVALID for NULL arguments
 * or non-finite host packet data. */
fgr_status fgr_decompose(fgr_ctx *ctx, const void *u_in, fgr_packets *inout, void *cuda_stream);

/* One dimension of a tensor-product packet mesh: n (q, p) pairs. */
typedef struct {
    int64_t n;          /* entries, >= 1 */
    const double *q;    /* [n] centres along this dimension */
    const double *p;    /* [n] momenta along this dimension */
    int32_t on_device;  /* 1: device pointers, 0: host pointers */
    int32_t reserved;
} fgr_axis;

/* Eq. 2.8, as fgr_decompose, for packets on a tensor-product mesh (the
 * phase-space meshes of Sec. 2.1 and Algorithm 3 are of this form).  Packet
 * (i_0, ..., i_{d-1}) sits at Q_l = axes[l].q[i_l], P_l = axes[l].p[i_l]; its
 * index is row-major, ((i_0 n_1 + i_1) n_2 + i_2) for d = 3.  For j < m,
 * a_out[j] and a_out[m + j] receive the real and imaginary parts of A(0) of
 * the packet with index sel[j] (sel NULL: index j, and m must equal
 * n_0 ... n_{d-1}).  The kernel of eq. 2.8 factorises over dimensions, so for
 * d >= 2 the sum runs as d banded contractions, last dimension first (work
 * proportional to the grid and list sizes times the window length, not to the
 * packets times the window volume); d = 1 runs fgr_decompose's kernel on the
 * listed packets.  The results equal fgr_decompose's on the same packets to
 * rounding.  Axes sorted by q keep each block of 64 consecutive entries
 * within about one window (unsorted axes are correct but slower).  u_in, sel
 * and a_out: host or device memory (detected).  The library allocates two
 * intermediate arrays of at most the largest partial product of grid and list
 * extents (complex, the context's precision).  FGR_E_INVALID for NULL
 * arguments, an axis with n < 1, a product of more than 2^40 packets, m < 0 or
 * m > 2^31, sel NULL with m != n_0 ... n_{d-1}, non-finite host axis data, or
 * a sel entry outside [0, n_0 ... n_{d-1}) (a device sel is checked on the
 * device, and that check waits for the stream). */
fgr_status fgr_decompose_tensor(fgr_ctx *ctx, const fgr_axis *axes, const void *u_in, int64_t m,
                                const int64_t *sel, double *a_out, void *cuda_stream);

/* Algorithm 3 (multi-step FGGC) with a fixed phase-space mesh and the flow
 * learned once.  mesh: packets at the mesh positions (q, p) onto which every
 * step decomposes the current wave (only q and p are read); flow: the same
 * packets, in the same order, propagated over one step from unit amplitude
 * (fgr_propagate with a = 1): their Q, P, S and amplitude factor A(T_evo)
 * (eq. 2.6 is linear in A).  Each of the `steps` steps decomposes u (as
 * fgr_decompose), multiplies the amplitudes by the factors and reconstructs by
 * FGGC (as fgr_reconstruct_fggc); u_out receives the wave after the last step
 * (u_in itself when steps = 0).  u_in and u_out: the context's grid and
 * complex type, host or device.  Waits like fgr_reconstruct_fggc (once per
 * step).  FGR_E_INVALID if mesh and flow hold different numbers of packets,
 * steps < 0 or an argument is NULL. */
fgr_status fgr_fggc_multistep(fgr_ctx *ctx, const fgr_packets *mesh, const fgr_packets *flow, const void *u_in,
                              void *u_out, int32_t steps, void *cuda_stream);

/* Algorithm 3 as fgr_fggc_multistep, with the fixed mesh given as a tensor
 * product (axes and sel as in fgr_decompose_tensor, m = flow->m): each step
 * decomposes by fgr_decompose_tensor's contractions.  flow packet j is mesh
 * packet sel[j] (j without sel) propagated over one step from unit
 * amplitude.  Errors as fgr_decompose_tensor and fgr_fggc_multistep. */
fgr_status fgr_fggc_multistep_tensor(fgr_ctx *ctx, const fgr_axis *axes, const int64_t *sel,
                                     const fgr_packets *flow, const void *u_in, void *u_out, int32_t steps,
                                     void *cuda_stream);

/* Eq. 2.10 over the box window: u(x_m) = pref * sum_j A_j exp(i/eps (S_j +
 * P_j.(x_m - Q_j)) - |x_m - Q_j|^2/(2 eps)).  FP64: every term in FP64.
 * FP32: the phase is reduced in FP64 per packet and evaluated in FP32 turns.
 * d = 1: of every 4 consecutive grid points the first term is evaluated with
 * exp, sin and cos in FP32 and the next three by the exact recurrences of the
 * Gaussian factor and the phase (one complex multiply each).  d = 2, 3: the
 * term factorises over dimensions, so on a tile of the grid the sum is a
 * complex matrix product of the packets' per-dimension factors (tabulated on
 * the tile's grid lines by the same recurrences).  By default it runs on the
 * tensor cores: super tiles of 128 x 64 points (d = 2) or 8 x 16 x 64
 * (d = 3), each factor split into two TF32 parts and the product taken
 * as three TF32 products into FP32 accumulators of 64 packets each, summed in
 * FP32; with FGR_FLAG_DIRECT_FMA (and for windows too wide for the super
 * tiles' lists: beyond about 110 lines of dimensions 0 and 1 in 3-D) on the
 * CUDA cores, one complex multiply-add per packet-point pair, partial sums
 * folded into FP64.  Complex64 out.  The
 * work is cut into (tile, packet slice) items: d = 1 the same number of
 * slices per tile, d >= 2 slices in proportion to each tile's packet count,
 * heaviest first, taken by persistent CTAs (no host wait).  A tensor-core
 * launch that gives up waiting on its own pipeline (a bounded wait) sets the
 * context's error word; the next FGGC call on the context reports it. */
fgr_status fgr_reconstruct_direct(fgr_ctx *ctx, const fgr_packets *pk, void *u_out,
                                  void *cuda_stream);

/* Batched eq. 2.10 (not in the paper: it serves many small reconstructions
 * at once).  Request r sums the packets pks[r] onto the grid of ctxs[r] into
 * u_outs[r], exactly as fgr_reconstruct_direct would, but all n requests share
 * one persistent launch of the summation kernel whose CTAs take (request,
 * tile, packet-split) items from a device counter until none remain, so many
 * requests with small grids fill the GPU together (d >= 2: the largest
 * requests first, each tile's packet list cut on the device into slices in
 * proportion to its length, heaviest tiles first).  1 <= n <= 64; all contexts
 * must have the same dimension, precision and device; every u_outs[r] must be
 * device memory of its context's output size and the outputs must not
 * overlap.  Packets may be host memory (staged like fgr_reconstruct_direct);
 * with device packets and a non-NULL stream the call enqueues only
 * stream-ordered work, so it can be captured into a CUDA graph.  The caller
 * owns every array; nothing is retained after the call.  FGR_E_INVALID names
 * the first offending request in fgr_last_error(). */
fgr_status fgr_reconstruct_direct_batch(int32_t n, fgr_ctx *const *ctxs, const fgr_packets *const *pks,
                                        void *const *u_outs, void *cuda_stream);

/* Algorithm 2 Steps 3-4.  Per packet and dimension: int/frac split (eq. 3.6-3.7),
 * right-hand side f~ (eq. 3.23), c~ = A~^+ f~ through the eigen factors,
 * conjugated (true L2 normal equations) and shifted back by
 * exp(-i cq cp (s - dq_k) b0) (eq. 3.13); d-dimensional coefficients are
 * products over dimensions.  The weights A_j e^{iS_j/eps} c_j^(k) are summed
 * onto grid nodes (eq. 2.25) and the node Gaussians are summed on the grid
 * (eq. 2.24) one dimension at a time.  FP64: all FP64.  FP32: the coefficients
 * come from a Chebyshev surrogate of c~(s,t) built on the host from the same
 * pseudo-inverse (degree 10, truncation error about 3e-10: below FP32 rounding;
 * evaluated in FP32 over the terms i + j <= 11 for n1 <= 8), phases are reduced
 * in FP64, node array and grid sums in complex64.  Host packets are copied to
 * the device and tested there for non-finite values before anything is
 * written: FGR_E_INVALID if one is found. */
fgr_status fgr_reconstruct_fggc(fgr_ctx *ctx, const fgr_packets *pk, void *u_out,
                                void *cuda_stream);

/* FGGC reconstruction that allocates no memory (the paper has no counterpart:
 * this is a deployment variant of fgr_reconstruct_fggc).
 * Some callers cannot allocate device memory once they are running: a host
 * whose device memory is committed up front to a fixed budget, a plugin inside
 * a framework that owns every allocation on the device, or a latency-bound
 * loop that cannot afford cudaMalloc/cudaFree and the synchronisation they can
 * cause.  This entry point serves them: it computes exactly what
 * fgr_reconstruct_fggc computes, with all of its working memory (bounds, row
 * flag and node array) in one static device array of 8 MiB that the library
 * reserves on every device that loads it, for as long as the process lives.
 * Limits: 1-D contexts only; packets and u_out must be device memory of the
 * context's device (or managed memory; FGR_E_INVALID otherwise); the node
 * array (16 bytes per complex128 or 8 per complex64 cell) and the grid pass's
 * tables (8 bytes per node of the box's a-range and per grid point) must fit
 * in 8 MiB - 512 B together; larger problems return FGR_E_CAPACITY with the
 * required sizes in fgr_last_error() (use fgr_reconstruct_fggc for them).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call clears and reuses the same array, so calls whose work overlaps on
 * the device (any streams, any contexts) race and must be serialised by the
 * caller.  The call waits for its own bounds readback like fgr_reconstruct_fggc.
 * No cudaMalloc, cudaFree or other allocating routine is called. */
fgr_status fgr_reconstruct_fggc_noalloc(fgr_ctx *ctx, const fgr_packets *pk, void *u_out,
                                        void *cuda_stream);

/* FGGC plans (not in the paper: a serving and graph-capture aid).  A plan
 * fixes, for one context and one packet set, the node box of the FGGC
 * reconstruction (the packets' node ranges widened by margin nodes on every
 * side) and owns its working memory (device memory allocated here, freed by
 * fgr_fggc_plan_destroy).  fgr_fggc_plan_create waits for the packets' node
 * bounds, like fgr_reconstruct_fggc; packets may be host or device memory.
 * FGR_E_INVALID for margin outside 0..4096; FGR_E_NOMEM / FGR_E_CAPACITY when
 * the box cannot be allocated. */
typedef struct fgr_fggc_plan fgr_fggc_plan;
fgr_status fgr_fggc_plan_create(fgr_ctx *ctx, const fgr_packets *pk, int32_t margin, fgr_fggc_plan **out,
                                void *cuda_stream);
/* FGGC reconstruction through a plan: the same arithmetic as
 * fgr_reconstruct_fggc on the plan's box, with only stream-ordered work (no
 * allocation, no host wait: it can be captured into a CUDA graph and replayed
 * with new packet values in the same buffers).  Packets (device memory) may
 * differ from the plan's; their node bounds are recomputed on the device, and
 * if they leave the box the plan's overflow flag is set (contributions
 * outside the box are then missing from u_out; re-plan).  Calls that share a
 * plan share its memory and must not overlap on the device.  FGR_E_INVALID if
 * the plan belongs to another dimension, precision, grid, eps or neighbour
 * set, or if packets or u_out are not device memory. */
fgr_status fgr_reconstruct_fggc_planned(fgr_ctx *ctx, fgr_fggc_plan *plan, const fgr_packets *pk, void *u_out,
                                        void *cuda_stream);
/* Many FGGC reconstructions in one go (not in the paper: a batching and
 * serving aid).  Request r is fgr_reconstruct_fggc_planned(ctxs[r], plans[r],
 * pks[r], u_outs[r]): the same arithmetic on the plan's box, with packets and
 * outputs in device memory.  Requests of one dimension run together, up to 32
 * per launch: every stage (clearing the node arrays, node bounds and box
 * checks, coefficients and scatter, b-range scans, pass tables, grid passes,
 * transposes) is one launch for all of them, whose CTAs find their request by
 * a prefix over per-request CTA counts; requests of different dimensions may
 * be mixed (one sequence of launches per dimension).  Only stream-ordered work:
 * no allocation and no host wait, so a batch can be captured into a CUDA
 * graph.  Contexts with FGR_FLAG_FFT_GRID run their request alone inside the
 * call.  Overflow flags are set per plan as for planned calls; calls that
 * share a plan must not overlap.  FGR_E_INVALID (naming the request) if n is
 * outside 1..64, an argument is NULL, a plan does not match its context,
 * packets or u_out are not device memory, or a request's device, precision or
 * neighbour strategy (cq, cp, nq, np, rcond) differs from request 0's. */
fgr_status fgr_reconstruct_fggc_batch(int32_t n, fgr_ctx *const *ctxs, fgr_fggc_plan *const *plans,
                                      const fgr_packets *const *pks, void *const *u_outs, void *cuda_stream);
/* 1 if the packets of the plan's last completed call left its box (waits for
 * the device). */
fgr_status fgr_fggc_plan_overflow(fgr_fggc_plan *plan, int32_t *overflowed);
/* Node cells of the plan's box; empty = 1 if no packet reached the grid. */
fgr_status fgr_fggc_plan_info(const fgr_fggc_plan *plan, int64_t *nodes, int32_t *empty);
void fgr_fggc_plan_destroy(fgr_fggc_plan *plan);

/* Autotuner of the launch shapes (not in the paper: it serves the batching and
 * serving side of the library).  Times, with CUDA events on the given stream,
 * the candidate work-item targets per SM of the direct sum (methods & 1: 2, 4,
 * 8, 16, 32; fgr_reconstruct_direct cuts each output tile's packet list into
 * slices in proportion to its length so that about that many items per SM
 * exist, heaviest first, and persistent CTAs pull them; the batched call gives
 * every tile of a request the same number of slices) and, for the FGGC grid passes (methods & 2), the tile width (128 or 32
 * grid points per CTA) with each CTA-per-SM target (4, 8, 16, 32, 64) on these
 * packets and this context's grid (u_out receives the last result), keeps the
 * fastest in the context and in a process-wide table keyed by (d, precision,
 * packets and grid points rounded to powers of two) that seeds later contexts;
 * with FGR_TUNE_FILE set, the table is loaded from and appended to that file.
 * Waits for its own timing runs. */
fgr_status fgr_autotune(fgr_ctx *ctx, const fgr_packets *pk, void *u_out, int32_t methods,
                        void *cuda_stream);
/* The context's launch shapes: work-item (direct sum) and CTA (grid passes)
 * targets per SM (1..256), and the grid-pass tile (32 or 128 grid points per
 * CTA; 0 = chosen from the node band width, the default).  FGR_E_INVALID for
 * values outside those ranges. */
fgr_status fgr_get_tuning(const fgr_ctx *ctx, int32_t *direct_ctas_per_sm, int32_t *pass_ctas_per_sm,
                          int32_t *pass_tile);
fgr_status fgr_set_tuning(fgr_ctx *ctx, int32_t direct_ctas_per_sm, int32_t pass_ctas_per_sm,
                          int32_t pass_tile);

/* Read-only facts about a context. */
typedef struct {
    int32_t d, n1, rank, precision;
    double eps, dq, dp, pref, window_r;
    double eigenvalues[16]; /* of the eps-free Gram, descending; n1 are valid */
} fgr_info;
fgr_status fgr_get_info(const fgr_ctx *ctx, fgr_info *out);

/* Per-stage device times (milliseconds, CUDA events) of the context's last
 * reconstruct or propagate call, when timing is enabled with fgr_set_timing.
 * FGGC: prep_ms = clearing the node array, coeff_ms = binning the packets by
 * anchor cell (d = 3, FP32), scatter_ms = the coefficient and scatter
 * kernels, grid_ms = the whole grid stage (eq. 2.24), of which pass_ms is the
 * grid-pass kernels alone; pass_terms = node-point terms of the grid passes
 * (per pass, over every (row, node a) line: the occupied b-range times the
 * grid points in node a's window; counted on the device, by one extra kernel
 * per pass, when timing is set to 2).  fgr_set_timing: 0 off, 1 per-stage
 * events, 2 per-stage events and pass_terms. */
typedef struct {
    double prep_ms, coeff_ms, scatter_ms, grid_ms, direct_ms, propagate_ms, total_ms;
    int64_t launches;       /* kernels launched by the last call */
    int64_t pairs;          /* FGR direct: packet-point pairs inside windows */
    int64_t nodes;          /* FGGC: cells of the node array */
    double pass_ms;         /* FGGC: grid-pass kernels alone (part of grid_ms) */
    int64_t pass_terms;     /* FGGC: node-point terms of the grid passes */
} fgr_stats;
fgr_status fgr_set_timing(fgr_ctx *ctx, int32_t enabled);
fgr_status fgr_get_stats(const fgr_ctx *ctx, fgr_stats *out);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of reconstructions over resident packet sets.
 * ------------------------------------------------------------------------- */

/* Starts a server on the current device with a scheduler thread and
 * max_inflight worker streams.  Requests are admitted while the resident packet
 * sets (and the FGGC plans the server keeps for them) plus the footprints of
 * the admitted requests stay within hbm_budget_bytes; others wait in arrival
 * order.  Requests of one method, dimension and precision with device outputs
 * that wait together run as one group (see fgr_server_set_max_batch); FGGC
 * requests go through a plan cached per (packet set, grid, eps, options) when
 * the budget allows, freed with the set.  Large requests (direct sums whose
 * packets x window points put them above about 2 ms) run alone on
 * low-priority streams and hold at most max_inflight - 1 slots; a small request
 * may pass a waiting large one, and while small requests wait or run, a large
 * 2-D / 3-D direct sum gives up one CTA slot per SM between its work items.
 * Free with fgr_server_destroy, which cancels what has not started and waits
 * for what has.  Not in the paper: a serving policy. */
fgr_status fgr_server_create(size_t hbm_budget_bytes, int32_t max_inflight, fgr_server **out);
void fgr_server_destroy(fgr_server *srv);

/* Largest group of waiting requests (same method, d and precision, device
 * outputs) that one worker takes at once: direct sums run as a single
 * fgr_reconstruct_direct_batch launch, FGGC reconstructions through their
 * cached plans as one fgr_reconstruct_fggc_batch call, with one wait
 * (default 16; 1 turns grouping off; at most 64).  Applies to
 * requests admitted after the call.  Not in the paper: a serving policy. */
fgr_status fgr_server_set_max_batch(fgr_server *srv, int32_t max_batch);

/* Copies a packet set (host or device, see fgr_packets) into device memory owned
 * by the server and returns its id.  FGR_E_CAPACITY if it would exceed the budget. */
fgr_status fgr_register_packets(fgr_server *srv, int32_t d, const fgr_packets *pk,
                                uint64_t *set_id);
/* Frees a registered set once no admitted request uses it. */
fgr_status fgr_release_packets(fgr_server *srv, uint64_t set_id);

typedef struct {
    int32_t method;      /* 0: direct sum, 1: FGGC */
    int32_t d;
    fgr_grid grid;
    double eps;
    fgr_options opt;     /* precision etc.; zeroed -> defaults */
    uint64_t set_id;     /* a registered packet set of dimension d */
    void *u_out;         /* device or host buffer of the output, caller-owned;
                            must stay valid until fgr_poll reports completion */
} fgr_request;

typedef struct {
    int32_t status;      /* fgr_status of the request */
    int32_t reserved;
    double t_submit_ms, t_start_ms, t_done_ms; /* host steady clock, ms */
} fgr_result;

/* Queues a request and returns a ticket at once.  FGR_E_INVALID for a malformed
 * request or unknown set; FGR_E_CAPACITY if it can never fit the budget. */
fgr_status fgr_submit(fgr_server *srv, const fgr_request *req, uint64_t *ticket);

/* Waits up to timeout_ms (0: just look; < 0: no limit) for the ticket.  Returns
 * FGR_OK with *out filled once done (the ticket is then retired), or
 * FGR_E_NOT_READY.  FGR_E_INVALID for an unknown ticket. */
fgr_status fgr_poll(fgr_server *srv, uint64_t ticket, int32_t timeout_ms, fgr_result *out);

/* Cancels a queued request (no effect once it has started). */
fgr_status fgr_cancel(fgr_server *srv, uint64_t ticket);

#ifdef __cplusplus
}
#endif

#endif /* FGR_H */
