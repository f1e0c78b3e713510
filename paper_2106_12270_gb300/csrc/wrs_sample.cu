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


// ===========================================================================
// a7: sectioned sampling (Sec. 5)
// ===========================================================================
//
// The rows are cut into nsec sections of near-equal size (section s covers
// rows [floor(s*n/nsec), floor((s+1)*n/nsec))).  Every row is equally likely
// to be picked, so the number of samples that fall into the left half of any
// range of sections is binomial with p = rows(left)/rows(range); splitting
// recursively (as Algorithm R does for uniform sampling) gives each section
// its count with no communication.  A tree node with c samples takes its
// left share from Philox counters keyed by the node: exact Bernoulli trials
// for c <= 96, otherwise the normal approximation round(c p + z sqrt(c p
// (1-p))) clamped to [0, c] (the paper uses the normal approximation; z comes
// from the Box-Muller transform).  Walking from the root to a leaf also sums
// the left shares passed on the way, which is the section's output offset.

constexpr uint32_t kExactBinomialMax = 96;

__device__ __forceinline__ uint64_t sec_row(uint64_t s, uint64_t n, uint64_t nsec) {
    return (uint64_t)(((u128)s * n) / nsec);
}

// Left share of a node holding c samples over sections [lo, hi), split at mid.
__device__ uint64_t node_left(uint64_t c, uint64_t lo, uint64_t mid, uint64_t hi, uint64_t n,
                              uint64_t nsec, uint32_t node, uint32_t k0, uint32_t k1) {
    if (c == 0) return 0;
    const uint64_t rl = sec_row(mid, n, nsec) - sec_row(lo, n, nsec);
    const uint64_t rt = sec_row(hi, n, nsec) - sec_row(lo, n, nsec);
    if (rl == 0) return 0;
    if (rl == rt) return c;
    if (c <= kExactBinomialMax) {
        // c Bernoulli(rl/rt) trials, four 32-bit uniforms per Philox call:
        // success iff u * rt < rl * 2^32 (exact integer comparison)
        uint64_t left = 0;
        for (uint32_t call = 0; 4 * call < c; ++call) {
            uint4 x = philox4x32_10(make_uint4(node, call, 0u, WRS_TAG_COUNTS), k0, k1);
            uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                if (4 * call + h < c)
                    left += ((u128)u[h] * rt < ((u128)rl << 32)) ? 1u : 0u;
            }
        }
        return left;
    }
    uint4 x = philox4x32_10(make_uint4(node, 0xffffffffu, 0u, WRS_TAG_COUNTS), k0, k1);
    // z ~ N(0,1) by Box-Muller in FP32 (SFU); the mean is formed in FP64
    // because counts reach 1e10
    float u1 = ((float)(x.x >> 8) + 1.0f) * 5.9604644775390625e-8f;   // (0, 1]
    float u2 = (float)(x.y >> 8) * 5.9604644775390625e-8f;            // [0, 1)
    float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    double p = (double)rl / (double)rt;
    double mean = (double)c * p;
    float sd = sqrtf((float)(mean * (1.0 - p)));
    double v = rint(mean + (double)(z * sd));
    if (v < 0.0) v = 0.0;
    if (v > (double)c) v = (double)c;
    return (uint64_t)v;
}

__global__ void __launch_bounds__(256)
k_sec_counts(uint64_t n, uint64_t nsec, uint64_t count, uint32_t k0, uint32_t k1,
             uint64_t *__restrict__ counts, uint64_t *__restrict__ offsets) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsec) return;
    uint64_t lo = 0, hi = nsec, c = count, off = 0;
    uint32_t node = 1;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        uint64_t left = node_left(c, lo, mid, hi, n, nsec, node, k0, k1);
        if (s < mid) {
            hi = mid;
            c = left;
            node = 2 * node;
        } else {
            lo = mid;
            off += left;
            c -= left;
            node = 2 * node + 1;
        }
    }
    counts[s] = c;
    offsets[s] = off;
}

// One CTA per section: draw its samples from its rows.  kSmem stages the
// section's rows in shared memory first (coalesced 8-byte loads; each row
// becomes its integer keep threshold and alias, so a draw needs no
// float-to-integer conversion), otherwise the rows are gathered through the
// caches.
template <bool kSmem>
__global__ void __launch_bounds__(256)
k_sample_sec(const uint2 *__restrict__ rows, uint64_t n, uint64_t nsec,
             const uint64_t *__restrict__ counts, const uint64_t *__restrict__ offsets,
             uint32_t k0, uint32_t k1, uint32_t *__restrict__ out, int vec_ok) {
    extern __shared__ uint2 srow[];
    const uint64_t s = blockIdx.x;
    const uint64_t r0 = sec_row(s, n, nsec), r1 = sec_row(s + 1, n, nsec);
    const uint64_t R = r1 - r0;
    const uint64_t c = counts[s], o = offsets[s];
    if (kSmem) {
        // each row once: its keep threshold ceil(prob 2^32) as an integer and
        // its alias; a row with prob 1 keeps itself as the alias, so that
        // coin < 0xffffffff or not picks the same item
        for (uint64_t r = threadIdx.x; r < R; r += blockDim.x) {
            const uint2 v = __ldg(rows + r0 + r);
            const float t = __uint_as_float(v.x) * 4294967296.0f;
            srow[r] = t >= 4294967296.0f ? make_uint2(0xffffffffu, (uint32_t)(r0 + r))
                                         : make_uint2(__float2uint_ru(t), v.y);
        }
        __syncthreads();
    }
    auto pick = [&](uint32_t row, uint32_t coin, uint2 v) {
        return kSmem ? (coin < v.x ? row : v.y) : walker_pick(row, coin, v);
    };
    const uint64_t calls = (c + 1) >> 1;
    // two independent Philox calls per thread and step (interleaved chains)
    auto one = [&](uint64_t cc, uint4 x) {
        uint64_t ra, rb;
        uint32_t ca, cb;
        walker_split(((uint64_t)x.x << 32) | x.y, R, ra, ca);
        walker_split(((uint64_t)x.z << 32) | x.w, R, rb, cb);
        uint2 va = kSmem ? srow[ra] : __ldg(rows + r0 + ra);
        uint2 vb = kSmem ? srow[rb] : __ldg(rows + r0 + rb);
        uint32_t sa = pick((uint32_t)(r0 + ra), ca, va);
        uint32_t sb = pick((uint32_t)(r0 + rb), cb, vb);
        uint64_t q = o + 2 * cc;
        if (2 * cc + 1 < c) {
            if (vec_ok && (q & 1) == 0) *reinterpret_cast<uint2 *>(out + q) = make_uint2(sa, sb);
            else { out[q] = sa; out[q + 1] = sb; }
        } else {
            out[q] = sa;
        }
    };
    const uint64_t B = blockDim.x;
    uint64_t cc = threadIdx.x;
    for (; cc + B < calls; cc += 2 * B) {
        const uint64_t c2 = cc + B;
        const uint4 x1 = philox4x32_10(
            make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), (uint32_t)s, WRS_TAG_SECTION), k0, k1);
        const uint4 x2 = philox4x32_10(
            make_uint4((uint32_t)c2, (uint32_t)(c2 >> 32), (uint32_t)s, WRS_TAG_SECTION), k0, k1);
        one(cc, x1);
        one(c2, x2);
    }
    if (cc < calls)
        one(cc, philox4x32_10(
                    make_uint4((uint32_t)cc, (uint32_t)(cc >> 32), (uint32_t)s, WRS_TAG_SECTION),
                    k0, k1));
}

// Shared memory a LIMITED-mode CTA requests (and does not use) so that only
// one CTA runs per SM (Sec. 5 "cached limited sectioned sampling").
constexpr uint32_t kLimitedSmem = 120 * 1024;

cudaError_t launch_sample_sectioned(const wrs_row *d_rows, uint64_t n, uint64_t count,
                                    uint64_t seed, uint32_t mode, uint64_t nsec,
                                    uint64_t *d_counts, uint64_t *d_offsets, uint32_t *d_out,
                                    cudaStream_t st) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    k_sec_counts<<<(unsigned)((nsec + 255) / 256), 256, 0, st>>>(n, nsec, count, k0, k1,
                                                                 d_counts, d_offsets);
    cudaError_t e = cudaGetLastError();
    if (e || count == 0) return e;
    const uint2 *rows = reinterpret_cast<const uint2 *>(d_rows);
    const int vec_ok = ((uintptr_t)d_out & 7u) == 0;
    if (mode == WRS_SAMPLE_SMEM) {
        uint64_t maxR = (n + nsec - 1) / nsec;
        uint32_t smem = (uint32_t)(maxR * sizeof(uint2));
        e = ensure_dynamic_smem<k_sample_sec<true>>(smem);
        if (e) return e;
        k_sample_sec<true><<<(unsigned)nsec, 256, smem, st>>>(rows, n, nsec, d_counts, d_offsets,
                                                              k0, k1, d_out, vec_ok);
    } else {
        uint32_t smem = 0;
        if (mode == WRS_SAMPLE_LIMITED) {
            smem = kLimitedSmem;
            e = ensure_dynamic_smem<k_sample_sec<false>>(smem);
            if (e) return e;
        }
        k_sample_sec<false><<<(unsigned)nsec, 256, smem, st>>>(rows, n, nsec, d_counts,
                                                               d_offsets, k0, k1, d_out, vec_ok);
    }
    return cudaGetLastError();
}

}  // namespace wrs
