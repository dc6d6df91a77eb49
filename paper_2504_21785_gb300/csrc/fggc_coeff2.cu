// K3+K4 instantiations for 2-D problems (see fggc_coeff.cuh).
#include "fggc_bin.cuh"

namespace fgr {
fgr_status launch_coeff_scatter_d2(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags) {
    return launch_coeff_d<2>(n1, st, pk, p64, p32, W, flags);
}
fgr_status launch_binned_d2(int n1, const BinLaunch &L, cudaStream_t st, const PacketsDev &pk, const Params32 &P,
                            void *W, uint8_t *flags, StageMarks *marks) {
    switch (n1) {
    case 4: return launch_binned_d<2, 4>(L, st, pk, P, W, flags, marks);
    case 8: return launch_binned_d<2, 8>(L, st, pk, P, W, flags, marks);
    default: set_error("fggc: no binned scatter for %d neighbours", n1); return FGR_E_INVALID;
    }
}
}  // namespace fgr
