// inst_warp_rkck_f64.cu -- the warp-per-cell RKCK kernel with double rate
// arithmetic, isothermal and with the energy equation (own translation unit so
// the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_rkck_f64(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return L.energy ? warp_rkck_launch<double, true>(L, blocks, threads, st)
                    : warp_rkck_launch<double, false>(L, blocks, threads, st);
}

cudaError_t occ_warp_rkck_f64(const MechDev& M, int nV, int energy, int threads, int* bps)
{
    return energy ? warp_rkck_occ<double, true>(M, nV, KIN_FP64, threads, bps)
                  : warp_rkck_occ<double, false>(M, nV, KIN_FP64, threads, bps);
}

}  // namespace kin
