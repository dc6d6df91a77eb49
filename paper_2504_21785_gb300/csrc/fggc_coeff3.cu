// K3+K4 instantiations for 3-D problems (see fggc_coeff.cuh).
#include "fggc_bin.cuh"

namespace fgr {
fgr_status launch_coeff_scatter_d3(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags) {
    return launch_coeff_d<3>(n1, st, pk, p64, p32, W, flags);
}
fgr_status launch_binned_d3(int n1, const BinLaunch &L, cudaStream_t st, const PacketsDev &pk, const Params32 &P,
                            void *W, uint8_t *flags, StageMarks *marks) {
    switch (n1) {
    case 4: return launch_binned_d<3, 4>(L, st, pk, P, W, flags, marks);
    case 8: return launch_binned_d<3, 8>(L, st, pk, P, W, flags, marks);
    default: set_error("fggc: no binned scatter for %d neighbours", n1); return FGR_E_INVALID;
    }
}
fgr_status launch_scatter_batch_d3(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32) {
    return launch_scatter_batch_dim<3>(n1, st, b64, b32);
}
}  // namespace fgr
