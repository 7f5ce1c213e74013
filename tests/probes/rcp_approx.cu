// Relative error of the approximate FP64 reciprocal instruction
// (rcp.approx.ftz.f64), alone and after the one Newton step the kernels'
// step control applies, over 4M log-uniform inputs in [2^-120, 2^120].
// Every thread touches only element i < n; no waits. Prints two numbers.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <random>
#include <vector>
#include <cuda_runtime.h>

__global__ void k(const double* x, double* r0, double* r1, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = x[i], r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    r0[i] = r;
    r1[i] = fma(r, fma(-a, r, 1.0), r);
}

int main()
{
    const int n = 1 << 22;
    std::vector<double> x(n), r0(n), r1(n);
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> u(std::log(std::ldexp(1.0, -120)), std::log(std::ldexp(1.0, 120)));
    for (int i = 0; i < n; ++i) x[i] = std::exp(u(g));
    double *dx, *d0, *d1;
    cudaMalloc(&dx, 8 * n); cudaMalloc(&d0, 8 * n); cudaMalloc(&d1, 8 * n);
    cudaMemcpy(dx, x.data(), 8 * n, cudaMemcpyHostToDevice);
    k<<<(n + 255) / 256, 256>>>(dx, d0, d1, n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(e)); return 1; }
    cudaMemcpy(r0.data(), d0, 8 * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(r1.data(), d1, 8 * n, cudaMemcpyDeviceToHost);
    double m0 = 0, m1 = 0;
    for (int i = 0; i < n; ++i) {
        long double ex = 1.0L / (long double)x[i];
        double e0 = (double)fabsl((r0[i] - ex) / ex), e1 = (double)fabsl((r1[i] - ex) / ex);
        if (e0 > m0) m0 = e0;
        if (e1 > m1) m1 = e1;
    }
    printf("%.6e %.6e\n", m0, m1);
    return 0;
}
