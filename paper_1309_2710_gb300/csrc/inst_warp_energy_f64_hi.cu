// inst_warp_energy_f64_hi.cu -- the warp-per-cell RKC kernels with the
// energy equation (Eq. (E:energy)), double rate arithmetic and the high-occupancy
// register budget (own translation unit so the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_f64_en_o1(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return warp_launch<double, 1, true>(L, blocks, threads, st);
}

cudaError_t occ_warp_f64_en_o1(const MechDev& M, int nV, int threads, int* bps)
{
    return warp_occ<double, 1, true>(M, nV, KIN_FP64, threads, bps);
}

}  // namespace kin
