// wrs_internal.cuh - device helpers and internal layouts of the GB300
// alias-table library.  Not part of the public ABI (include/wrs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/wrs.h"

namespace wrs {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Status bits raised by kernels (combined with atomicOr, turned into one
// wrs_status by the info step; the worst error wins).
// ---------------------------------------------------------------------------
enum : uint32_t {
    ERR_NEGATIVE = 1u,   // a weight with the sign bit set (other than -0)
    ERR_NONFINITE = 2u,  // NaN or Inf
    ERR_ZEROSUM = 4u,    // W == 0
    ERR_INTERNAL = 16u   // an invariant failed (reported as EINVAL)
};

// ---------------------------------------------------------------------------
// Build parameters, computed on the device by the total-weight and q-sum
// steps and read by every later step.  Lives at the start of the workspace.
//
// Fixed point: q_i = round(w_i * 2^S) with S chosen so that W*2^S lies in
// [2^61, 2^62); every q_i fits 64 bits.  The bucket Q is the exact sum of the
// q_i, so the scaled light deficits and heavy excesses balance exactly.
// ---------------------------------------------------------------------------
struct __align__(16) BuildParams {
    u128 Dtot;         // D'(nl): total scaled light deficit
    u128 Etot;         // E'(nh): total scaled heavy excess
    double W;          // exact total weight rounded to FP64
    double avg;        // W / N
    uint64_t Q;        // sum of all q_i: one bucket in fixed point (< 2^63)
    uint64_t Qn;       // floor(Q / N): largest q a light item may carry
    uint64_t n;
    uint64_t nl, nh;   // written by the segment scan
    uint32_t status;   // ERR_* bits
    int32_t scale;     // S
    int32_t qshift;    // q_i = m_i * 2^(e'_i + qshift) (e' = max(biased exp, 1))
    float light_max;   // largest FP32 <= avg
    float inv_avg;     // (float)(1 / avg)
    float Qf;          // (float)Q
    float invQ;        // 1 / Qf: a heavy row keeps 1 - delta * invQ
    uint32_t sections; // s
    uint32_t nseg;     // partition segments
    uint32_t sum_done; // blocks of the total-weight kernel that are done
    // Every weight whose light/heavy clamp of q is not the identity lies in
    // [tmid - thalf, tmid + thalf] (a superset, see k_qsum).
    float tmid, thalf;
};

// Workspace layout (all offsets 256-byte aligned).
struct Layout {
    uint64_t params;     // BuildParams
    uint64_t sum_bins;   // kSumMaxBlocks * kBands u128
    uint64_t seg_cnt;    // kMaxSegs uint32 light counts per segment
    uint64_t seg_q;      // kMaxSegs uint64 q sums per segment (all items)
    uint64_t seg_loff;   // (kMaxSegs + 1) uint64 global light rank at each segment start
    uint64_t seg_sum;    // kMaxSegs SegVal (segment clamped q sums)
    uint64_t seg_pre;    // (kMaxSegs + 1) SegVal (exclusive prefixes)
    uint64_t lh;         // n Entry
    uint64_t ckl;        // (n/32 + 2) CkRec
    uint64_t ckh;        // (n/32 + 2) CkRec
    uint64_t splits;     // (s+1) SplitRec
    uint64_t total;
    uint64_t sections;
};

struct __align__(8) Entry {   // one slot of the l/h array
    uint32_t item;
    float w;
};

struct __align__(16) SegVal {   // per-segment partition sums / prefixes
    u128 sl;      // sum of light q (clamped); < 2^64
    u128 sh;      // sum of heavy q (clamped); < 2^64
    uint64_t nl;  // light count
    uint64_t pad;
};

// Checkpoint of a prefix sum every 32 list entries: the q sum of the entries
// before it, relative to the start of the partition segment `seg` that holds
// it (the segment's own prefix is in seg_pre).
struct __align__(16) CkRec {
    uint32_t seg;
    uint32_t pad;
    uint64_t s;   // local q sum
};

struct __align__(16) SplitRec {  // Vose state after k_t buckets
    uint32_t i, j;
    uint32_t pad[2];
    u128 D;       // D'(i)
    u128 E;       // E'(j)
};

// Segmented batched build: each table of a batch is built by the single-
// table split and pack kernels over its own sections (of kBSeg buckets).
// The partition kernel leaves, per table, a BuildParams record, its place in
// the batch and its first section and split record.
constexpr uint32_t kBSeg = 1024;
struct __align__(16) BatchTab {
    uint64_t base;   // first item of the table in the batch
    uint32_t sec0;   // first section
    uint32_t rec0;   // first split record (sections + 1 per table)
};
// Workspace of the segmented batched build for up to `cap` items and ntab
// tables (all offsets 256-byte aligned); the counters and lh sit where the
// chunked kernel expects its counter and lh.
struct BatchSegLayout {
    uint64_t counters;   // [0] large tables taken, [1] sections, [2] split records,
                         // [3] small tables taken, [4] large tables, [5] small tables
    uint64_t lh;         // cap Entry
    uint64_t tp;         // ntab BuildParams
    uint64_t tabs;       // ntab BatchTab
    uint64_t sec_tab;    // cap / kBSeg + ntab + 1 uint32: table of each section
    uint64_t ckl, ckh;   // (cap >> 5) + 2 ntab + 2 CkRec each
    uint64_t recs;       // cap / kBSeg + 2 ntab + 1 SplitRec
    uint64_t zero;       // one zero SegVal (the checkpoints' segment prefix)
    uint64_t lists;      // 2 ntab uint32: the large tables, then the small ones
    uint64_t total;
    uint64_t cap;
};
BatchSegLayout batch_seg_layout(uint64_t cap, uint32_t ntab);
// Checkpoint index of checkpoint c of the table at `base` (table t).
__host__ __device__ inline uint64_t bseg_ck(uint64_t base, uint32_t t, uint64_t c) {
    return (base >> 5) + 2ull * t + c;
}

// One sampling request of the request loop (device-resident descriptor).
struct __align__(16) SampleReq {
    const wrs_row *rows;
    uint64_t n;
    uint64_t count;
    uint32_t *out;
    uint32_t k0, k1, slo, shi;
};

// Sizes shared by host and device code.
constexpr int kBands = 11;            // exponent bands of width 24
constexpr int kSumThreads = 256;
constexpr int kSumBands = 16;   // total weight: bands of 16 binades
constexpr int kSumMaxBlocks = 1216;   // 8 x 152 SMs
constexpr int kPartThreads = 256;
constexpr int kPartItems = 16;
constexpr int kSegPerSM = 3;          // partition CTAs resident per SM (8 warps, one sub-segment each)
constexpr int kMaxSegs = 8192;        // sub-segments (a multiple of 1024)
constexpr int kChunk = 512;           // items a partition warp handles at a time
constexpr int kSplitThreads = 256;    // also p of the partial p-ary search

static inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Host: grant kernel Kern at least `bytes` of dynamic shared memory on the
// current device.  The attribute is per device; the largest grant so far is
// remembered per kernel and device, so the CUDA call happens once, and
// concurrent callers are safe (a repeated grant is harmless).
constexpr int kMaxDevices = 64;
template <auto Kern>
inline cudaError_t ensure_dynamic_smem(uint32_t bytes) {
    static std::atomic<uint32_t> granted[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    uint32_t cur = granted[dev].load(std::memory_order_acquire);
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e) return e;
    while (cur < bytes && !granted[dev].compare_exchange_weak(cur, bytes, std::memory_order_acq_rel)) {
    }
    return cudaSuccess;
}

Layout make_layout(uint64_t n, uint32_t section_size);

// Batched build, chunked kernel (wrs_batched.cu); tune == nullptr is its
// default tiling (256 threads, chunks of 1024).
bool batch_tuning_valid(const wrs_batch_tuning &t);
cudaError_t launch_build_batched(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                 const uint32_t *d_order, uint32_t *d_counter, Entry *d_lh,
                                 wrs_row *d_rows, wrs_row *const *d_row_ptrs,
                                 wrs_table_summary *d_info, const wrs_batch_tuning *tune,
                                 cudaStream_t st);
// The segmented batched build (wrs_batched.cu, wrs_build.cu) in a workspace
// laid out by batch_seg_layout.
cudaError_t launch_build_batched_seg(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                     const uint32_t *d_order, unsigned char *ws,
                                     const BatchSegLayout &L, wrs_row *d_rows,
                                     wrs_row *const *d_row_ptrs, wrs_table_summary *d_info,
                                     cudaStream_t st);

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_up_sync(0xffffffffu, lo, d);
    hi = __shfl_up_sync(0xffffffffu, hi, d);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return ((u128)hi << 64) | lo;
}

// Fixed point of an FP32 weight: q = round(w * 2^S) < 2^62, halves rounded
// up.  S = qshift + 150 lies in [-97, 210] (the total W is in [2^-149,
// 2^159)); 2^S is applied as two exact power-of-two factors, so x = w * 2^S
// is exact unless it falls below the FP32 normal range, where it is far
// below 1/2 and q = 0 however it rounds (x <= W 2^S < 2^62: no overflow).
// q is assembled from 32-bit conversions, which issue about eight times as
// fast as a float to 64-bit integer conversion on sm_103 (that one runs on
// the FP64 unit):
//   hi = floor(x / 2^32) < 2^30 (the scaling is exact; below the normal
//        range hi is 0 either way), a float of at most 24 significant bits;
//   lo = x - hi 2^32 in [0, 2^32), one fused multiply-add, exact: lo is x
//        itself below 2^32, 0 from 2^56 on (x is then a multiple of 2^33),
//        and between, a multiple of ulp(x) below 2^32, at most 24 bits;
//   q  = hi 2^32 + floor(lo + 1/2), the addition rounded down: from 2^23 on
//        lo is an integer and the sum is exact or rounds back to lo; below,
//        floor(lo + 1/2) is itself a float <= lo + 1/2, so rounding down
//        never crosses it.
// Needs IEEE subnormals (no flush to zero).  The weight must be finite and
// not negative (checked by the total-weight step before any caller runs; -0
// gives 0).
struct QScale {
    float c1, c2;   // 2^min(S, 127), 2^(S - min(S, 127))
};
__device__ __forceinline__ QScale qscale(int qshift) {
    const int S = qshift + 150;
    const int s1 = S < 127 ? S : 127;
    QScale r;
    r.c1 = __int_as_float((s1 + 127) << 23);
    r.c2 = __int_as_float((S - s1 + 127) << 23);
    return r;
}
__device__ __forceinline__ uint64_t fixed_q(float w, QScale qs) {
    const float x = __fmul_rn(__fmul_rn(w, qs.c1), qs.c2);
    const uint32_t hi = __float2uint_rz(__fmul_rn(x, 0x1p-32f));
    const float lo = __fmaf_rn(__uint2float_rz(hi), -0x1p32f, x);
    return ((uint64_t)hi << 32) | __float2uint_rd(__fadd_rd(lo, 0.5f));
}

// q of a light item clamped to at most Qn = floor(Q/N), so that its scaled
// deficit d' = Q - N*q >= 0; q of a heavy item clamped to at least Qn+1, so
// that its scaled excess e' = N*q - Q > 0.
__device__ __forceinline__ uint64_t light_q(float w, QScale qs, uint64_t Qn) {
    uint64_t q = fixed_q(w, qs);
    return q > Qn ? Qn : q;
}
__device__ __forceinline__ uint64_t heavy_q(float w, QScale qs, uint64_t Qn) {
    uint64_t q = fixed_q(w, qs);
    return q <= Qn ? Qn + 1 : q;
}
// The sweep's comparison (Sec. 2.2): heavy h[j] closes before light l[i]
// iff its excess prefix E'(j+1) does not exceed the deficit prefix D'(i).
// Both are compared rounded down to multiples of 2^kKeyShift: a bucket is
// Q >= 2^61 units, so this differs from the unrounded comparison only when
// the two agree to 2^-46 of a bucket, ties stay ties, and the 64-bit keys of
// the pack kernel implement it exactly.  Every kernel (split, pack, batched)
// uses this one rule, so the table does not depend on the section size or
// the code path.
constexpr int kKeyShift = 15;
__device__ __forceinline__ bool sweep_le(u128 E, u128 D) {
    return (E >> kKeyShift) <= (D >> kKeyShift);
}

// N * q as 128 bits (q < 2^63, N < 2^31).
__device__ __forceinline__ u128 mul_nq(uint32_t N, uint64_t q) { return (u128)q * N; }

// floor((c + p) / 2^15) for the 128-bit two's-complement sum c + p, capped
// at 2^62 (the true value is above -2^48): a heavy's sweep key relative to
// its section (the pack and its sequential variants).
constexpr int kKeyCap62 = 62;
__device__ __forceinline__ int64_t sweep_key(u128 c, u128 p) {
    const __int128 v = (__int128)(c + p) >> kKeyShift;
    return v < ((__int128)1 << kKeyCap62) ? (int64_t)v : ((int64_t)1 << kKeyCap62);
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with fixed odd constants, mixing the high halves with
// the other two words and the round key; the key advances by fixed Weyl
// increments after every round.
// ---------------------------------------------------------------------------
struct Philox {
    static constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    static constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(Philox::kMul0, c.x), lo0 = Philox::kMul0 * c.x;
        uint32_t hi1 = __umulhi(Philox::kMul1, c.z), lo1 = Philox::kMul1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += Philox::kWeyl0;
        k1 += Philox::kWeyl1;
    }
    return c;
}

// Walker's rule on one 64-bit uniform u for `rows` rows starting at `base`:
// P = u * rows; row = P >> 64; coin = bits 32..63 of P.
__device__ __forceinline__ void walker_split(uint64_t u, uint64_t rows,
                                             uint64_t &row, uint32_t &coin) {
    row = __umul64hi(u, rows);
    coin = (uint32_t)((u * rows) >> 32);
}

// Keep the row iff coin < ceil(prob * 2^32).  prob * 2^32 is exact in FP32
// (power-of-two scaling) and the conversion rounds up, so this is the ceiling.
__device__ __forceinline__ uint32_t walker_pick(uint32_t row, uint32_t coin,
                                                uint2 r) {
    const float t = __uint_as_float(r.x) * 4294967296.0f;
    // below 2^32 the ceiling fits 32 bits (the largest such float is
    // 2^32 - 256); prob = 1 keeps the row for every coin
    return (t >= 4294967296.0f || coin < __float2uint_ru(t)) ? row : r.y;
}

}  // namespace wrs
