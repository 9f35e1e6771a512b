// Test helper: Philox4x32-10 as CUDA's curand implements it, for a third,
// independent check of the library's and the oracle's generators (called,
// not copied).  Host arrays in and out; built by tests/test_gpu_trace.py.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_philox(const uint4* ctr, const uint2* key, int64_t n, uint4* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_batch(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    if (n <= 0) return 0;
    if (cudaMalloc(&dc, 16 * (size_t)n) != cudaSuccess) return 1;
    if (cudaMalloc(&dk, 8 * (size_t)n) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 16 * (size_t)n) != cudaSuccess) return 1;
    cudaMemcpy(dc, ctr, 16 * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, key, 8 * (size_t)n, cudaMemcpyHostToDevice);
    k_curand_philox<<<(unsigned)((n + 255) / 256), 256>>>(dc, dk, n, dout);
    const cudaError_t e = cudaMemcpy(out, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 1;
}
