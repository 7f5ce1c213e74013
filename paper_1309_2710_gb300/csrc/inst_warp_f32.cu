// inst_warp_f32.cu -- instantiation of the warp-per-cell RKC kernels with float
// rate arithmetic (own translation unit so the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_f32(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return warp_launch<float>(L, blocks, threads, st);
}

cudaError_t occ_warp_f32(const MechDev& M, int threads, int* bps)
{
    return warp_occ<float>(M, KIN_MIXED, threads, bps);
}

}  // namespace kin
