// inst_warp_f64.cu -- instantiation of the warp-per-cell RKC kernels with double
// rate arithmetic (own translation unit so the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_f64(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return warp_launch<double>(L, blocks, threads, st);
}

cudaError_t occ_warp_f64(const MechDev& M, int threads, int* bps)
{
    return warp_occ<double>(M, KIN_FP64, threads, bps);
}

}  // namespace kin

namespace kin {

size_t warp_smem(const MechDev& M, int precision, int threads)
{
    return warp_smem_bytes(M, precision, threads);
}

}  // namespace kin
