// Test helper: raw output words of cuRAND's device-side Philox4_32_10
// generator, run as a black box.  For each i the state is initialised with
// curand_init(seed, subsequence[i], offset[i]) and the first curand4() result
// is returned.  Built and loaded by tests/test_gpu_philox.py only.
#include <cstdint>

#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void words_kernel(unsigned long long seed, const unsigned long long *sub,
                             const unsigned long long *off, int n, uint4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub[i], off[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_device_words(unsigned long long seed, const unsigned long long *sub,
                                   const unsigned long long *off, int n, unsigned int *out)
{
    unsigned long long *d_sub = nullptr, *d_off = nullptr;
    uint4 *d_out = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_sub, sizeof(*d_sub) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_off, sizeof(*d_off) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_out, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_sub, sub, sizeof(*d_sub) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_off, off, sizeof(*d_off) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        words_kernel<<<(n + 127) / 128, 128>>>(seed, d_sub, d_off, n, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_sub);
    cudaFree(d_off);
    cudaFree(d_out);
    return (int)e;
}
