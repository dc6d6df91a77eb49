// Parameter blocks of the FGGC kernels, shared by the node-box / grid-pass
// code (fggc.cu) and the coefficient + scatter kernels (fggc_coeff*.cu).
#pragma once

#include "internal.h"

namespace fgr {

struct Common {
    int n1;
    int dq[kMaxN1], dp[kMaxN1];
    double dqv, dpv;                 // mesh steps
    double inv_dq, inv_dp;
    double cq2_4, cp2_4, half_cqcp;  // eq. 3.23 constants
    double cc;                       // cq cp / (2 pi): node phase in turns
    double inv_2pi_eps, pref;
    int amin[kMaxDim], A[kMaxDim], bmin[kMaxDim], B[kMaxDim];
    int64_t sa[kMaxDim], sb[kMaxDim];  // W strides of a_l and b_l
    int64_t row_len;                   // cells per row of the first grid pass
    int64_t ra[kMaxDim], rb[kMaxDim];  // sa / row_len, sb / row_len (dimensions before the last)
};

struct Params64 {
    Common c;
    double vr[kMaxN1 * kMaxN1], vi[kMaxN1 * kMaxN1], inv_lam[kMaxN1];
};

struct Params32 {
    Common c;
    float cre[kMaxN1 * kCheb * kCheb], cim[kMaxN1 * kCheb * kCheb];
};

// Node box of one FGGC reconstruction and the sizes of its buffers.
struct FggcBox {
    Common c;               // constants and box (amin, A, bmin, B, strides)
    int64_t cells = 0;      // node cells
    int64_t rows0 = 0;      // rows of the first grid pass
    int64_t maxbuf = 0;     // elements of each pass buffer (d > 1)
    int64_t max_lines = 0;  // (row, a) lines of the b-range scan
    int64_t table_entries = 0;  // 8-byte entries of the largest pass table
    int64_t fft_elems = 0;      // complex elements of the DFT lines of the largest pass (0: no DFT stage)
    bool empty = true;      // no packet reaches the grid
};

struct FggcBuffers {
    void *W = nullptr, *buf1 = nullptr, *buf2 = nullptr;
    uint8_t *flags = nullptr;
    int2 *brange = nullptr;
    void *tables = nullptr;  // per-pass tables (node windows, point phases, tile bands)
    void *bin = nullptr;     // binning buffers of the 3-D FP32 scatter (NULL: per-packet scatter)
    int64_t bin_m = 0;       // packets the binning buffers hold
    unsigned long long *terms = nullptr;  // node-point terms of the passes (timed calls only)
    void *fft = nullptr;      // DFT lines of the commensurate grid stage (box.fft_elems complex)
    void *twiddle = nullptr;  // e^{2 pi i j / N}, j < N / 2 <= 4096 (complex)
};

// Binning of the 3-D scatter (fggc_bin.cuh): key box of the outer anchor
// cells (a0, b0) of dimensions 0..d-2 whose neighbours can reach the node box,
// key = row-major index over (a0_0, b0_0, a0_1, b0_1).
struct BinBox {
    int ka_lo[2] = {}, KA[2] = {1, 1}, kb_lo[2] = {}, KB[2] = {1, 1};
    int dqmin = 0, dqmax = 0, dpmin = 0, dpmax = 0;  // neighbour shift ranges
    int64_t K = 0;                                   // keys
};

// Device buffers of the binning (m packets, K keys).
struct BinBuffers {
    int *key = nullptr;     // [m] key of each packet (-1: adds nothing)
    int *count = nullptr;   // [K] packets per key, then the placement cursor
    int2 *off = nullptr;    // [K + 1] (first sorted packet, first item) per key; totals at K
    int2 *bsum = nullptr;   // [ceil(K / 1024)] block totals of the scan
    int *sorted = nullptr;  // [m] binned packets by key
    int *loose = nullptr;   // [m] packets of small cells
    int4 *items = nullptr;  // [max items] (key, first sorted packet, packets)
    int *ctr = nullptr;     // [4] loose count, work counter
};

struct BinLaunch {
    BinBox box;
    BinBuffers buf;
    int min_count = 8;   // smallest binned cell (kBinMinCount)
    int num_sms = 1;
    // rows of W (each row_cells cells) to clear before the scatter: only the
    // rows the binned packets reach are marked and zeroed (0: W is cleared by
    // the caller)
    int64_t clear_rows = 0;
    int64_t row_cells = 0;
};

// Largest key box of the binned scatter; larger boxes use the per-packet kernel.
constexpr int64_t kMaxBinKeys = int64_t(1) << 26;
// Smallest binned cell (packets); smaller cells take the per-packet kernel.
constexpr int kBinMinCount = 8;

// Key box of a node box (false when the binned scatter does not apply).
bool make_bin_box(const FggcBox &box, int d, BinBox *bb);
// Bytes of the binning buffers for m packets and key box bb.
size_t bin_buffer_bytes(int64_t m, const BinBox &bb);
// Carves the binning buffers out of one device block of bin_buffer_bytes.
void bin_buffers_at(void *block, int64_t m, const BinBox &bb, BinBuffers *out);

// Stage marks of the timed FGGC call (the binning ends where binned() is called).
struct StageMarks {
    StageTimer *timer = nullptr;
    double *slot = nullptr;
    void binned() {
        if (timer) timer->mark(slot);
    }
};

// Batched FGGC (fgr_reconstruct_fggc_batch): per-request parameters of one
// launch over up to kBatchMax requests of one dimension; CTA b of the launch
// belongs to the request r with block0[r] <= b < block0[r + 1].
constexpr int kBatchMax = 32;

struct ScatterBatchBase {
    int n;
    int block0[kBatchMax + 1];
    Common c[kBatchMax];
    const double *q[kBatchMax], *p[kBatchMax], *s[kBatchMax], *a[kBatchMax];
    int64_t m[kBatchMax];
    void *W[kBatchMax];
    uint8_t *flags[kBatchMax];
};
struct ScatterBatch64 : ScatterBatchBase {
    double vr[kMaxN1 * kMaxN1], vi[kMaxN1 * kMaxN1], inv_lam[kMaxN1];
};
struct ScatterBatch32 : ScatterBatchBase {
    float cre[kMaxN1 * kCheb * kCheb], cim[kMaxN1 * kCheb * kCheb];
};

// One request of a batched FGGC call: its context, planned box and buffers,
// bounds and overflow flag (device), packets and output (device).
struct FggcRequest {
    const fgr_ctx *ctx;
    const FggcBox *box;
    const FggcBuffers *buf;
    int *bnd, *overflow;
    PacketsDev pk;
    void *u;
};
// Enqueues the requests (any dimensions, one precision and neighbour
// strategy): per dimension and kBatchMax requests, one launch per stage.
fgr_status run_fggc_batch(int n, const FggcRequest *req, cudaStream_t st);

// Launches the batched per-packet coefficient + scatter kernel of dimension d
// (grid: batch.block0[batch.n] CTAs of coeff_threads); exactly one batch is non-NULL.
fgr_status launch_scatter_batch(int d, int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32);
fgr_status launch_scatter_batch_d1(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32);
fgr_status launch_scatter_batch_d2(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32);
fgr_status launch_scatter_batch_d3(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32);
// Threads per CTA of the per-packet scatter kernel.
int scatter_threads(bool fp64, int n1);

// Box from the packets' node bounds hb[12] (per dimension: a min, a max, b min,
// b max), widened by margin nodes on every side.
fgr_status make_box(const fgr_ctx *ctx, const int *hb, int margin, FggcBox *box);

// Node bounds of the packets into hb[12] on the host (waits for them).
fgr_status compute_node_bounds(fgr_ctx *ctx, const PacketsDev &pk, int *bnd_dev, int *hb, cudaStream_t st);

// FGGC into u_dev with a planned box and buffers: stream-ordered only; sets
// *overflow (device) when the packets' nodes leave the box (their
// contributions outside it are then missing).  bnd: 12 device ints.
fgr_status run_fggc_planned(fgr_ctx *ctx, const PacketsDev &pk, const FggcBox &box, const FggcBuffers &b,
                            int *bnd, int *overflow, void *u_dev, cudaStream_t st);

// Launches the coefficient + scatter kernel (K3+K4) for dimension d, one
// thread per packet; exactly one of p64 / p32 is non-NULL.
fgr_status launch_coeff_scatter(int d, int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                const Params32 *p32, void *W, uint8_t *flags);
fgr_status launch_coeff_scatter_d1(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags);
fgr_status launch_coeff_scatter_d2(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags);
fgr_status launch_coeff_scatter_d3(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags);
// The binned scatter (FP32, d = 3, n1 = 4 or 8): binning kernels, then the
// binned kernel and the per-packet kernel over the loose list.  (In 2-D a
// packet has only 64 contributions and an outer cell reaches 8 rows: the
// per-packet kernel is faster there, measured on the 2-D workload.)
fgr_status launch_binned_scatter(int d, int n1, const BinLaunch &L, cudaStream_t st, const PacketsDev &pk,
                                 const Params32 &P, void *W, uint8_t *flags, StageMarks *marks);
fgr_status launch_binned_d3(int n1, const BinLaunch &L, cudaStream_t st, const PacketsDev &pk, const Params32 &P,
                            void *W, uint8_t *flags, StageMarks *marks);

}  // namespace fgr
