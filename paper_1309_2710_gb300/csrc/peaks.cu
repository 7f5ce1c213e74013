// peaks.cu -- fused multiply-add throughput of the FP64 and FP32 pipes
// (include/kin_peaks.h), the denominators of the benchmark's roofline.
//
// Every thread advances kChains independent chains of dependent FMAs, so
// each warp keeps kChains instructions in flight; with several warps per
// scheduler that covers the pipes' latency and the issue rate of the pipe is
// what the kernel measures. The chains stay bounded (x -> b / (1 - a)), and
// their sum is stored only under a condition the compiler cannot decide, so
// no chain is removed as dead code and nothing is written in practice.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "../../include/kin_peaks.h"

namespace {

constexpr int kChains = 8;

// Target of the store that keeps the chains alive (never executed).
__device__ double g_sink64;
__device__ float g_sink32;

thread_local char g_err[256] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

template <typename F>
__global__ void __launch_bounds__(1024) fma_chains(F* sink, long long iters, F a, F b, F never)
{
    F x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = F(threadIdx.x & 7) * F(0.125) + F(c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    F s = F(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == never) sink[0] = s;  // never taken for the arguments the host passes
}

}  // namespace

extern "C" int kinpk_fma_rate(int32_t precision, int64_t iters, int32_t blocks_per_sm,
                              int32_t threads, void* stream, double* ms, double* fma_per_s)
{
    g_err[0] = 0;
    if (precision != KINPK_FP64 && precision != KINPK_FP32)
        return fail(-1, "unknown precision %d", precision);
    if (threads < 32 || threads > 1024 || threads % 32) return fail(-1, "threads must be 32..1024, a multiple of 32");
    if (iters < 1 || blocks_per_sm < 1) return fail(-1, "iters and blocks_per_sm must be >= 1");
    if (!ms || !fma_per_s) return fail(-1, "ms and fma_per_s must be non-NULL");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(-3, "device query: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = nsm * blocks_per_sm;
    // a = 1 - 2^-20 keeps every chain in [0, 8] (it decays towards 1), so
    // the sum of the eight chains is never -1 and the store is never executed
    double* s64 = nullptr;
    float* s32 = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s64, g_sink64);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s32, g_sink32);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        if (precision == KINPK_FP64)
            fma_chains<double><<<blocks, threads, 0, st>>>(s64, iters, 1.0 - 0x1p-20, 0x1p-20, -1.0);
        else
            fma_chains<float><<<blocks, threads, 0, st>>>(s32, iters, 1.0f - 0x1p-20f, 0x1p-20f, -1.0f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(-3, "FMA probe: %s", cudaGetErrorString(e));
    *ms = t;
    *fma_per_s = (double)blocks * threads * kChains * (double)iters / (t * 1e-3);
    return 0;
}

extern "C" const char* kinpk_last_error(void) { return g_err; }
