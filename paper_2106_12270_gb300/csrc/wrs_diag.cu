// wrs_diag.cu - a measurement kernel for the sampler's roofline.
//
// The naive sampler (Sec. 5 "baseline") is bound by random 8-byte row
// gathers from HBM.  This kernel performs the same access pattern without
// the method around it -- uniformly random 8-byte reads from an array of
// rows and one 4-byte store per read -- so the bench can report the sampler
// against the random-gather rate this GPU actually sustains, not only
// against the streaming copy bandwidth.  The row index comes from a cheap
// integer hash, not Philox, so that the kernel is bound by memory alone.
#include "wrs_internal.cuh"

namespace wrs {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // splitmix64 finaliser (Steele, Lea, Flood, OOPSLA'14)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

template <int kFlavor>
__device__ __forceinline__ uint2 load_row(const uint2 *p) {
    if (kFlavor == 0) return __ldg(p);    // read-only (non-coherent) path
    if (kFlavor == 1) return __ldcg(p);   // cache in L2 only
    return __ldcs(p);                     // streaming (evict first)
}

template <int kFlavor>
__global__ void __launch_bounds__(256)
k_random_gather(const uint2 *__restrict__ rows, uint64_t nrows, uint64_t count, uint64_t seed,
                uint32_t *__restrict__ out) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    constexpr int U = 8;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += U * T) {
        uint2 r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint64_t q = i + u * T;
            uint64_t row = __umul64hi(mix64(q ^ seed), nrows);
            r[u] = q < count ? load_row<kFlavor>(rows + row) : make_uint2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint64_t q = i + u * T;
            if (q < count) out[q] = r[u].x ^ r[u].y;
        }
    }
}

extern int num_sms();

cudaError_t launch_random_gather(const void *rows, uint64_t nrows, uint64_t count, uint64_t seed,
                                 int flavor, uint32_t *out, cudaStream_t st) {
    unsigned blocks = (unsigned)num_sms() * 8;
    const uint2 *r = reinterpret_cast<const uint2 *>(rows);
    if (flavor == 0)
        k_random_gather<0><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
    else if (flavor == 1)
        k_random_gather<1><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
    else
        k_random_gather<2><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
    return cudaGetLastError();
}

}  // namespace wrs
