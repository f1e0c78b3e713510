// wrs_sample.cu - alias-table sampling on GB300 (sm_103a).
//
// a6, naive sampling (Sec. 2.2 Walker's rule, Sec. 5 "baseline"): every
// sample draws one 64-bit uniform u from Philox-4x32-10, takes the integer
// part of u*N as the row and the fraction's top 32 bits as the coin, and
// gathers one 8-byte row.  Once the table is larger than L2 each sample costs
// one random 32-byte DRAM sector, so the kernel keeps many independent row
// gathers in flight per thread.
#include "wrs_internal.cuh"

namespace wrs {

constexpr int kSampleThreads = 256;
constexpr int kSampleUnroll = 4;   // Philox calls (2 samples each) in flight per thread

__global__ void __launch_bounds__(kSampleThreads)
k_sample_naive(const uint2 *__restrict__ rows, uint64_t n, uint64_t first, uint64_t count,
               uint32_t k0, uint32_t k1, uint32_t slo, uint32_t shi,
               uint32_t *__restrict__ out, int vec_ok) {
    const uint64_t cb = first >> 1, ce = (first + count + 1) >> 1;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t end = first + count;
    for (uint64_t c = cb + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ce;
         c += kSampleUnroll * T) {
        uint64_t row[2 * kSampleUnroll];
        uint32_t coin[2 * kSampleUnroll];
        uint2 r[2 * kSampleUnroll];
#pragma unroll
        for (int u = 0; u < kSampleUnroll; ++u) {
            uint64_t cc = c + u * T;
            if (cc < ce) {
                uint4 x = philox4x32_10(make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), slo, shi),
                                        k0, k1);
                walker_split(((uint64_t)x.x << 32) | x.y, n, row[2 * u], coin[2 * u]);
                walker_split(((uint64_t)x.z << 32) | x.w, n, row[2 * u + 1], coin[2 * u + 1]);
            } else {
                row[2 * u] = row[2 * u + 1] = 0;
                coin[2 * u] = coin[2 * u + 1] = 0;
            }
        }
#pragma unroll
        for (int h = 0; h < 2 * kSampleUnroll; ++h) r[h] = __ldg(rows + row[h]);
#pragma unroll
        for (int u = 0; u < kSampleUnroll; ++u) {
            uint64_t cc = c + u * T;
            if (cc >= ce) break;
            uint64_t q0 = 2 * cc;
            uint32_t s0 = walker_pick((uint32_t)row[2 * u], coin[2 * u], r[2 * u]);
            uint32_t s1 = walker_pick((uint32_t)row[2 * u + 1], coin[2 * u + 1], r[2 * u + 1]);
            if (vec_ok && q0 >= first && q0 + 1 < end && ((q0 - first) & 1) == 0) {
                *reinterpret_cast<uint2 *>(out + (q0 - first)) = make_uint2(s0, s1);
            } else {
                if (q0 >= first && q0 < end) out[q0 - first] = s0;
                if (q0 + 1 >= first && q0 + 1 < end) out[q0 + 1 - first] = s1;
            }
        }
    }
}

extern int num_sms();

cudaError_t launch_sample_naive(const wrs_row *d_rows, uint64_t n, uint64_t first,
                                uint64_t count, uint64_t seed, uint32_t slo, uint32_t shi,
                                uint32_t *d_out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    uint64_t calls = ((first + count + 1) >> 1) - (first >> 1);
    uint64_t per_block = (uint64_t)kSampleThreads * kSampleUnroll;
    uint64_t want = (calls + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)num_sms() * 16;
    unsigned blocks = (unsigned)(want < cap ? want : cap);
    int vec_ok = ((uintptr_t)d_out & 7u) == 0;   // pairs of samples as one 8-byte store
    k_sample_naive<<<blocks, kSampleThreads, 0, st>>>(
        reinterpret_cast<const uint2 *>(d_rows), n, first, count, (uint32_t)seed,
        (uint32_t)(seed >> 32), slo, shi, d_out, vec_ok);
    return cudaGetLastError();
}

}  // namespace wrs
