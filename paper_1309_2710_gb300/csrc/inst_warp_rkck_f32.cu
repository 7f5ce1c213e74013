// inst_warp_rkck_f32.cu -- the warp-per-cell RKCK kernel with float rate
// arithmetic, isothermal and with the energy equation (own translation unit so
// the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_rkck_f32(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return L.energy ? warp_rkck_launch<float, true>(L, blocks, threads, st)
                    : warp_rkck_launch<float, false>(L, blocks, threads, st);
}

cudaError_t occ_warp_rkck_f32(const MechDev& M, int nV, int energy, int threads, int* bps)
{
    return energy ? warp_rkck_occ<float, true>(M, nV, KIN_MIXED, threads, bps)
                  : warp_rkck_occ<float, false>(M, nV, KIN_MIXED, threads, bps);
}

}  // namespace kin
