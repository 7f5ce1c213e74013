// inst_warp_f32.cu -- the warp-per-cell RKC kernels with float rate arithmetic and the
// default register budget (own translation unit so the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_f32_o0(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return warp_launch<float, 0, false>(L, blocks, threads, st);
}

cudaError_t occ_warp_f32_o0(const MechDev& M, int nV, int threads, int* bps)
{
    return warp_occ<float, 0, false>(M, nV, KIN_MIXED, threads, bps);
}

}  // namespace kin
