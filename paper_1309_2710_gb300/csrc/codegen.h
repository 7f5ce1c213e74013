// codegen.h -- run-time generated f for the lane-per-cell FP64 integrator
// (codegen.cu): source generation, NVRTC compilation and launch.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kin_dev.cuh"

namespace kin {

// Kernels of one compiled mechanism, per form of f (isothermal; with the
// energy equation when `energy`): pre-pass per method (RKCK, RKC) and the
// persistent integrator per method and register budget.
struct GenKernels {
    cudaLibrary_t lib;
    bool energy;
    cudaKernel_t init[2][2];
    cudaKernel_t integrate[2][2][2];
};

// Mechanisms small enough for a register-resident generated f.
bool gen_eligible(int n_species, int n_reactions);
// The CUDA source of the generated f (a policy class kin::GenF) for `d`.
std::string gen_f_source(const kin_mech_desc* d);
// Compile f_src with the kernel templates to a cubin for sm_103a; `lowered`
// receives the kernels' symbol names (per form of f: init RKCK, init RKC,
// integrate [method][occupancy]). Returns KIN_OK, KIN_EUNSUPPORTED (no NVRTC) or
// KIN_ECUDA (compilation failed; `log` has the compiler output).
int gen_compile(const std::string& f_src, std::vector<char>* cubin, std::vector<std::string>* lowered,
                std::string* log);
// Compile (once per device and source) and load the kernels.
int gen_kernels(int device, const std::string& f_src, GenKernels* out, std::string* log);
// Whether gen_kernels has already compiled and loaded f_src on `device` (a
// lookup: compiles nothing, allocates nothing).
bool gen_loaded(int device, const std::string& f_src);
// Pre-pass, longest-first sort (RKC) and integrator of one call.
cudaError_t gen_launch(const GenKernels& g, Launch& L, int occ, int blocks, int threads, cudaStream_t st);

}  // namespace kin
