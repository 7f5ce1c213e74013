// inst_warp_f64.cu -- the warp-per-cell RKC kernels with double rate arithmetic and the
// default register budget (own translation unit so the build runs in parallel).
#include "warp.cuh"

namespace kin {

cudaError_t launch_warp_f64_o0(Launch& L, int blocks, int threads, cudaStream_t st)
{
    return warp_launch<double, 0, false>(L, blocks, threads, st);
}

cudaError_t occ_warp_f64_o0(const MechDev& M, int nV, int threads, int* bps)
{
    return warp_occ<double, 0, false>(M, nV, KIN_FP64, threads, bps);
}

size_t warp_smem(const MechDev& M, int precision, int energy, int threads)
{
    if (energy)
        return precision == KIN_MIXED ? warp_smem_bytes<float, true>(M, threads)
                                      : warp_smem_bytes<double, true>(M, threads);
    return precision == KIN_MIXED ? warp_smem_bytes<float, false>(M, threads)
                                  : warp_smem_bytes<double, false>(M, threads);
}

}  // namespace kin
