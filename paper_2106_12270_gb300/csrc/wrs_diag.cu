// wrs_diag.cu - measurement kernels for the samplers' rooflines.
//
// The naive sampler (Sec. 5 "baseline") is bound by random 8-byte row
// gathers from HBM.  This kernel performs the same access pattern without
// the method around it -- uniformly random 8-byte reads from an array of
// rows and one 4-byte store per read -- so the bench can report the sampler
// against the random-gather rate this GPU actually sustains, not only
// against the streaming copy bandwidth.  The row index comes from a cheap
// integer hash, not Philox, so that the kernel is bound by memory alone.
//
// The sectioned samplers read their rows from L2 and are bound by Philox
// arithmetic instead.  The second kernel makes the same Philox-4x32-10 calls
// (two per thread and step, two 32-bit outputs per call) and writes the same
// 4 bytes per sample, without the rows.
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

template <int kFlavor, int U>
__global__ void __launch_bounds__(256)
k_random_gather(const uint2 *__restrict__ rows, uint64_t nrows, uint64_t count, uint64_t seed,
                uint32_t *__restrict__ out) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
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

// Philox rate: call c (counter (c_lo, c_hi, 0, WRS_TAG_DIAG), key (k0, k1))
// writes out[2c] = x.x ^ x.y and out[2c+1] = x.z ^ x.w.
__global__ void __launch_bounds__(256)
k_philox_rate(uint64_t count, uint32_t k0, uint32_t k1, uint32_t *__restrict__ out) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t calls = (count + 1) >> 1;
    auto put = [&](uint64_t c, uint4 x) {
        const uint64_t q = 2 * c;
        const uint32_t a = x.x ^ x.y, b = x.z ^ x.w;
        if (q + 1 < count) *reinterpret_cast<uint2 *>(out + q) = make_uint2(a, b);
        else out[q] = a;
    };
    uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; c + T < calls; c += 2 * T) {
        const uint64_t c2 = c + T;
        const uint4 x1 =
            philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0u, WRS_TAG_DIAG), k0, k1);
        const uint4 x2 =
            philox4x32_10(make_uint4((uint32_t)c2, (uint32_t)(c2 >> 32), 0u, WRS_TAG_DIAG), k0, k1);
        put(c, x1);
        put(c2, x2);
    }
    if (c < calls)
        put(c, philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0u, WRS_TAG_DIAG), k0, k1));
}

extern int num_sms();

cudaError_t launch_philox_rate(uint64_t count, uint64_t seed, uint32_t *out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_philox_rate<<<(unsigned)num_sms() * 8, 256, 0, st>>>(count, (uint32_t)seed,
                                                           (uint32_t)(seed >> 32), out);
    return cudaGetLastError();
}


template <int kFlavor>
static void launch_gather_u(const uint2 *r, uint64_t nrows, uint64_t count, uint64_t seed,
                            unsigned blocks, uint32_t unroll, uint32_t *out, cudaStream_t st) {
    if (unroll == 4)
        k_random_gather<kFlavor, 4><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
    else if (unroll == 8)
        k_random_gather<kFlavor, 8><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
    else
        k_random_gather<kFlavor, 16><<<blocks, 256, 0, st>>>(r, nrows, count, seed, out);
}

// Launch shape: ctas_per_sm CTAs of 256 threads per SM (a grid-stride loop),
// `unroll` independent loads in flight per thread.
cudaError_t launch_random_gather(const void *rows, uint64_t nrows, uint64_t count, uint64_t seed,
                                 int flavor, uint32_t ctas_per_sm, uint32_t unroll, uint32_t *out,
                                 cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    unsigned blocks = (unsigned)num_sms() * ctas_per_sm;
    const uint2 *r = reinterpret_cast<const uint2 *>(rows);
    if (flavor == 0) launch_gather_u<0>(r, nrows, count, seed, blocks, unroll, out, st);
    else if (flavor == 1) launch_gather_u<1>(r, nrows, count, seed, blocks, unroll, out, st);
    else launch_gather_u<2>(r, nrows, count, seed, blocks, unroll, out, st);
    return cudaGetLastError();
}

}  // namespace wrs
