// no_alloc.cu -- an integration entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they integrate: a solver running
// under a memory manager that owns every device byte (a CFD code with its own
// pool), code executing while another component forbids allocation, or a host
// that must not grow the device footprint after start-up. For them,
// kin_integrate_noalloc takes the integrator's working memory from a fixed
// array that the library reserves once per device, instead of a caller
// workspace.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <mutex>

#include "kin_dev.cuh"

namespace {

// Fixed working memory. Every GPU that loads the library holds it until the
// process exits.
constexpr int64_t kStaticBytes = (int64_t)KIN_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[KIN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device. In host code the
// symbol g_scratch is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int kin_integrate_noalloc(const kin_mech* m, int64_t cells, double* T,
                                     const double* p, double* Y, int64_t ldY, double dt,
                                     double rtol, double atol, const kin_opts* opts,
                                     uint8_t* status, int32_t* stats)
{
    if (!m || !opts)  // let the regular entry point report the argument error
        return kin_integrate(m, cells, T, p, Y, ldY, dt, rtol, atol, opts, status, stats, nullptr, 0);
    // Fewer persistent blocks per SM shrink the per-lane part of the working
    // memory: take the largest count (up to the requested one) that fits.
    kin_opts o = *opts;
    o.blocks_per_sm = 1;
    int64_t need = kin_workspace_bytes(m, &o, cells);
    if (need < 0) return (int)need;  // invalid options or cell count; message set
    if (need > kStaticBytes)
        return kin::set_last_error(KIN_ENOMEM,
                                   "kin_integrate_noalloc: %lld cells need %lld bytes of working "
                                   "memory, more than the %lld-byte fixed array",
                                   (long long)cells, (long long)need, (long long)kStaticBytes);
    const int top = opts->blocks_per_sm > 0 ? opts->blocks_per_sm : 4;
    for (int bps = top; bps > 1; --bps) {
        kin_opts t = *opts;
        t.blocks_per_sm = bps;
        const int64_t n = kin_workspace_bytes(m, &t, cells);
        if (n >= 0 && n <= kStaticBytes) {
            o = t;
            break;
        }
    }
    void* ws = nullptr;
    const cudaError_t e = scratch_address(&ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return kin::set_last_error(KIN_ECUDA, "kin_integrate_noalloc: cudaGetSymbolAddress: %s",
                                   cudaGetErrorString(e));
    }
    return kin_integrate(m, cells, T, p, Y, ldY, dt, rtol, atol, &o, status, stats, ws, kStaticBytes);
}
