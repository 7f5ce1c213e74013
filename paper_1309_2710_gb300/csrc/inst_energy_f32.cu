// inst_energy_f32.cu -- the lane-per-cell kernels with the energy equation
// (Eq. (E:energy)) and float rate arithmetic, for both methods (own translation
// unit so the build runs in parallel).
#include "kernels.cuh"

namespace kin {

cudaError_t launch_rkc_f32_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st)
{
    return launch_energy<KIN_RKC, float>(L, occ, blocks, threads, st);
}

cudaError_t launch_rkck_f32_en(Launch& L, int occ, int blocks, int threads, cudaStream_t st)
{
    return launch_energy<KIN_RKCK, float>(L, occ, blocks, threads, st);
}

cudaError_t occ_rkc_f32_en(int occ, int threads, size_t sm, int* bps)
{
    return occ_energy<KIN_RKC, float>(occ, threads, sm, bps);
}

cudaError_t occ_rkck_f32_en(int occ, int threads, size_t sm, int* bps)
{
    return occ_energy<KIN_RKCK, float>(occ, threads, sm, bps);
}

}  // namespace kin
