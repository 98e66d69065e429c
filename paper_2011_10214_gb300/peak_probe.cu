// FP64 / FP32 FMA throughput probe for the roofline denominators of ALU-bound kernels:
// independent FMA chains on registers, 152 x 16 blocks of 256 threads, CUDA-event timed.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void k(T* out, int iters, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T> double run(const char* name, int iters) {
    int blocks = 152 * 16, threads = 256;
    T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
    k<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0);
    k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 8 * (double)iters * blocks * threads;
    printf("%s FMA peak: %.1f GFLOP/s (%.3f ms)\n", name, flops / ms / 1e6, ms);
    cudaFree(out);
    return flops / ms / 1e6;
}
int main() {
    run<double>("fp64", 4000);
    run<float>("fp32", 40000);
    return 0;
}
