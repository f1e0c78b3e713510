// Test helper: cuRAND's Philox4x32-10 round function on a batch of
// (counter, key) pairs, as an independent reference for the oracle's Philox
// (Salmon et al., SC'11).  Built by tests/test_gpu_philox_curand.py.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_philox(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_batch(const void *d_ctr, const void *d_key, void *d_out, int n) {
    if (n <= 0) return 0;
    k_curand_philox<<<(n + 255) / 256, 256>>>(static_cast<const uint4 *>(d_ctr),
                                               static_cast<const uint2 *>(d_key),
                                               static_cast<uint4 *>(d_out), n);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
