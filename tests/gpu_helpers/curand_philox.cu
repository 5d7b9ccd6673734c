// Test helper: evaluates cuRAND's device Philox4x32-10 (curand_Philox4x32_10)
// on given counters and keys, so the tests can pin the CPU oracle's Philox
// against an independent implementation.  Built by the GPU test at run time.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void philox_kernel(const uint4* ctr, const uint2* key, uint4* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_many(int n, const uint32_t* h_ctr, const uint32_t* h_key, uint32_t* h_out)
{
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    uint2* d_key = nullptr;
    cudaError_t e = cudaMalloc(&d_ctr, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_key, sizeof(uint2) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_ctr, h_ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_key, h_key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_kernel<<<(n + 255) / 256, 256>>>(d_ctr, d_key, d_out, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_ctr);
    cudaFree(d_out);
    cudaFree(d_key);
    return int(e);
}
