// no_alloc.cu -- an integration entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they integrate: a solver running
// under a memory manager that owns every device byte (a CFD code with its own
// pool), code executing while another component forbids allocation, or a host
// that must not grow the device footprint after start-up. For them,
// kin_integrate_noalloc takes the integrator's working memory from a fixed
// array that the library reserves once per device, instead of a caller
// workspace, and never compiles a generated f (NVRTC and the library load
// behind it allocate).
#include <cuda_runtime.h>

#include <mutex>

#include "kin_dev.cuh"

namespace {

// Fixed working memory. Every GPU that loads the library holds it until the
// process exits. The module that holds it is loaded, and the memory taken,
// at the first address lookup on a device (lazy module loading), so the
// first call on each device is where a lack of memory shows.
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
    // the caller's options, with the f evaluation and the blocks per SM
    // chosen so that the call neither compiles nor outgrows the array
    kin_opts o;
    const int rc = kin::noalloc_opts(m, opts, cells, kStaticBytes, &o);
    if (rc) return rc;
    void* ws = nullptr;
    const cudaError_t e = scratch_address(&ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return kin::set_last_error(e == cudaErrorMemoryAllocation ? KIN_ENOMEM : KIN_ECUDA,
                                   "kin_integrate_noalloc: loading the %lld-byte fixed array: %s",
                                   (long long)kStaticBytes, cudaGetErrorString(e));
    }
    return kin_integrate(m, cells, T, p, Y, ldY, dt, rtol, atol, &o, status, stats, ws, kStaticBytes);
}
