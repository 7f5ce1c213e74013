// inst_rkck_f32.cu -- instantiation of the integrator kernels for one method and
// rate precision (compiled as its own translation unit so the build runs in
// parallel).
#include "kernels.cuh"

namespace kin {

cudaError_t launch_rkck_f32(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st)
{
    return launch_occ<KIN_RKCK, float>(L, stg, occ, blocks, threads, st);
}

cudaError_t occ_rkck_f32(int stg, int occ, int threads, size_t sm, int* bps)
{
    return occ_sel<KIN_RKCK, float>(stg, occ, threads, sm, bps);
}

}  // namespace kin
