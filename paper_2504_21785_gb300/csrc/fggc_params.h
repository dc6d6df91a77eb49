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
    bool empty = true;      // no packet reaches the grid
};

struct FggcBuffers {
    void *W = nullptr, *buf1 = nullptr, *buf2 = nullptr;
    uint8_t *flags = nullptr;
    int2 *brange = nullptr;
    void *tables = nullptr;  // per-pass tables (node windows, point phases, tile bands)
};

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

}  // namespace fgr
