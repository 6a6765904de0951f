// Test helper: Philox4x32-10 outputs of cuRAND's device function, to check
// the oracle's implementation against an independent one.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <cstdint>

__global__ void k_curand_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox(const void *h_ctr, const void *h_key, void *h_out, int m)
{
    uint4 *c = nullptr, *o = nullptr;
    uint2 *k = nullptr;
    if (cudaMalloc(&c, m * sizeof(uint4)) || cudaMalloc(&k, m * sizeof(uint2)) || cudaMalloc(&o, m * sizeof(uint4))) return 1;
    cudaMemcpy(c, h_ctr, m * sizeof(uint4), cudaMemcpyHostToDevice);
    cudaMemcpy(k, h_key, m * sizeof(uint2), cudaMemcpyHostToDevice);
    k_curand_philox<<<(m + 255) / 256, 256>>>(c, k, o, m);
    cudaError_t e = cudaMemcpy(h_out, o, m * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(c); cudaFree(k); cudaFree(o);
    return e == cudaSuccess ? 0 : 2;
}
