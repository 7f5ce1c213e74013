// inst_rkc_f64.cu -- instantiation of the integrator kernels for one method and
// rate precision (compiled as its own translation unit so the build runs in
// parallel).
#include "kernels.cuh"

namespace kin {

cudaError_t launch_rkc_f64(Launch& L, int stg, int occ, int blocks, int threads, cudaStream_t st)
{
    return launch_occ<KIN_RKC, double>(L, stg, occ, blocks, threads, st);
}

cudaError_t occ_rkc_f64(int stg, int occ, int threads, size_t sm, int* bps)
{
    return occ_sel<KIN_RKC, double>(stg, occ, threads, sm, bps);
}

}  // namespace kin
