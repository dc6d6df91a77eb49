// K3+K4 instantiations for 1-D problems (see fggc_coeff.cuh).
#include "fggc_coeff.cuh"

namespace fgr {
fgr_status launch_coeff_scatter_d1(int n1, cudaStream_t st, const PacketsDev &pk, const Params64 *p64,
                                   const Params32 *p32, void *W, uint8_t *flags) {
    return launch_coeff_d<1>(n1, st, pk, p64, p32, W, flags);
}
fgr_status launch_scatter_batch_d1(int n1, cudaStream_t st, const ScatterBatch64 *b64, const ScatterBatch32 *b32) {
    return launch_scatter_batch_dim<1>(n1, st, b64, b32);
}
int scatter_threads(bool fp64, int n1) {
    if (fp64) return n1 == 16 ? coeff_threads<true, 16>() : coeff_threads<true, 8>();
    return coeff_threads<false, 8>();
}
}  // namespace fgr
