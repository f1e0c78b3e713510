// wrs_device.cuh - device routines shared by the construction kernels
// (single table and batched).
#pragma once

#include "wrs_internal.cuh"

namespace wrs {

__device__ __forceinline__ int pad32(int e) { return e + (e >> 5); }
__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

// The partition works on chunks of kChunk items; a warp owns a contiguous
// run of chunks (a sub-segment).  Sub-segment s of NS covers chunks
// [s*C/NS, (s+1)*C/NS) of the C chunks.
__device__ __forceinline__ void sub_range(uint32_t s, uint32_t NS, uint64_t C, uint64_t n,
                                          uint64_t &a, uint64_t &b) {
    uint64_t c0 = (uint64_t)s * C / NS, c1 = (uint64_t)(s + 1) * C / NS;
    a = c0 * kChunk;
    b = min(c1 * kChunk, n);
    if (a > b) a = b;
}

// Exponent band of an FP32 weight for the exact sum: a weight m * 2^(e'-150)
// (e' = max(biased exponent, 1)) is added to band e'/24 as m << (e' mod 24),
// a value below 2^47.  Sets error bits for NaN/Inf and negative weights.
__device__ __forceinline__ void band_of(float x, uint32_t &band, uint64_t &val, uint32_t &bad) {
    uint32_t u = __float_as_uint(x);
    uint32_t e = (u >> 23) & 0xffu;
    bad |= (e == 0xffu) ? ERR_NONFINITE : 0u;
    bad |= ((u >> 31) && (u & 0x7fffffffu)) ? ERR_NEGATIVE : 0u;
    uint32_t ee = e ? e : 1u;
    uint32_t m = (e == 0xffu) ? 0u : ((u & 0x7fffffu) | (e ? 0x800000u : 0u));
    band = (ee * 2731u) >> 16;   // ee / 24 for ee < 256
    val = (uint64_t)m << (ee - 24u * band);
}

// Bits [pos, pos+cnt) of a 384-bit integer held in 12 32-bit limbs, low
// limb first (cnt <= 128; bits outside the integer read as 0).
__device__ inline u128 big_bits(const uint32_t *big, int pos, int cnt) {
    int li = pos >= 0 ? pos / 32 : -((31 - pos) / 32);   // floor(pos / 32)
    int s = pos - 32 * li;                                // 0..31
    u128 lo = 0;
    for (int k = 0; k < 4; ++k) {
        int idx = li + k;
        uint32_t v = (idx >= 0 && idx < 12) ? big[idx] : 0u;
        lo |= (u128)v << (32 * k);
    }
    int idx5 = li + 4;
    uint32_t v5 = (idx5 >= 0 && idx5 < 12) ? big[idx5] : 0u;
    u128 r = lo >> s;
    if (s) r |= (u128)v5 << (128 - s);
    if (cnt < 128) r &= (((u128)1) << cnt) - 1;
    return r;
}

// Any set bit strictly below position pos?
__device__ inline int big_any_below(const uint32_t *big, int pos) {
    for (int k = 0; k < 12 && 32 * k < pos; ++k) {
        int nb = pos - 32 * k;   // bits of limb k that lie below pos
        uint32_t m = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
        if (big[k] & m) return 1;
    }
    return 0;
}

// W from the per-band sums (band b of kWidth binades counts in units of
// 2^(kWidth b - 150); below 2^128 each, kNB * kWidth + 128 <= 384): the
// exact total assembled in a 384-bit integer and rounded once to FP64, ties
// to even.  Returns false when the total is zero; `top` is the index of the
// total's highest set bit (units of 2^-150).
template <int kNB = kBands, int kWidth = 24>
__device__ inline bool exact_total(const u128 *band, double &W, int &top) {
    uint32_t big[12];
    for (int k = 0; k < 12; ++k) big[k] = 0;
    for (int b = 0; b < kNB; ++b) {
        u128 v = band[b];
        int shift = kWidth * b;
        uint64_t carry = 0;
        for (int k = 0; k < 12; ++k) {
            int o = 32 * k - shift;  // bit of v that lands at bit 0 of limb k
            uint32_t part = 0;
            if (o >= 0 && o < 128) part = (uint32_t)(v >> o);
            else if (o < 0 && o > -32) part = (uint32_t)(v << (-o));
            uint64_t sum = (uint64_t)big[k] + part + carry;
            big[k] = (uint32_t)sum;
            carry = sum >> 32;
        }
    }
    top = -1;
    for (int k = 11; k >= 0 && top < 0; --k)
        if (big[k]) top = 32 * k + 31 - __clz(big[k]);
    if (top < 0) {
        W = 0.0;
        return false;
    }
    uint64_t mant = (uint64_t)big_bits(big, top - 52, 53);
    int t = top;
    if (top >= 53) {
        int half = (int)big_bits(big, top - 53, 1);
        int sticky = big_any_below(big, top - 53);
        if (half && (sticky || (mant & 1u))) {
            ++mant;
            if (mant >> 53) { mant >>= 1; ++t; }
        }
    }
    uint64_t bits = ((uint64_t)(t + 873) << 52) | (mant & ((1ull << 52) - 1));
    W = __longlong_as_double((long long)bits);
    return true;
}

// Multi-word helpers of the sweep keys (pack and greedy pass): a 128-bit two's-complement
// value in four 32-bit limbs, low limb first.
struct Limbs4 {
    uint32_t w0, w1, w2, w3;
};
__device__ __forceinline__ Limbs4 to_limbs(u128 v) {
    return Limbs4{(uint32_t)v, (uint32_t)(v >> 32), (uint32_t)(v >> 64), (uint32_t)(v >> 96)};
}
__device__ __forceinline__ u128 from_limbs(const Limbs4 &a) {
    return ((u128)(((uint64_t)a.w3 << 32) | a.w2) << 64) | (((uint64_t)a.w1 << 32) | a.w0);
}
// low 64 bits of N q (exact when N q < 2^64)
__device__ __forceinline__ uint64_t mul_lo_nq(uint32_t N, uint64_t q) {
    const uint64_t lo = (uint64_t)(uint32_t)q * N;
    return lo + ((uint64_t)((uint32_t)(q >> 32) * N) << 32);
}
// a += v for v < 2^64, where the sum stays below 2^96 (the top limb is left as is)
__device__ __forceinline__ void add96(Limbs4 &a, uint64_t v) {
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2)
        : "r"((uint32_t)v), "r"((uint32_t)(v >> 32)));
}
// a += N q - Q (a heavy's scaled excess, below 2^95; q < 2^63, Q < 2^63)
__device__ __forceinline__ void add_excess(Limbs4 &a, uint32_t N, uint64_t q, uint64_t Q) {
    const uint64_t lo = (uint64_t)(uint32_t)q * N;           // bits 0..63
    const uint64_t hi = (uint64_t)(uint32_t)(q >> 32) * N;   // bits 32..95
    uint32_t e0, e1, e2;
    asm("add.cc.u32 %1, %4, %6;\n\t"     // e1 = lo.hi + hi.lo
        "addc.u32 %2, %7, 0;\n\t"        // e2 = hi.hi + carry
        "sub.cc.u32 %0, %3, %8;\n\t"     // e0 = lo.lo - Q.lo
        "subc.cc.u32 %1, %1, %9;\n\t"    // e1 -= Q.hi
        "subc.u32 %2, %2, 0;"
        : "=r"(e0), "=r"(e1), "=r"(e2)
        : "r"((uint32_t)lo), "r"((uint32_t)(lo >> 32)), "r"(0u), "r"((uint32_t)hi),
          "r"((uint32_t)(hi >> 32)), "r"((uint32_t)Q), "r"((uint32_t)(Q >> 32)));
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(e0), "r"(e1), "r"(e2));
}
// floor(a / 2^15) as a signed 64-bit key, for |a| < 2^78
__device__ __forceinline__ int64_t key15(const Limbs4 &a) {
    const uint32_t lo = __funnelshift_r(a.w0, a.w1, kKeyShift);
    const uint32_t hi = __funnelshift_r(a.w1, a.w2, kKeyShift);
    return (int64_t)(((uint64_t)hi << 32) | lo);
}
// the same, capped at 2^62 (a heavy that cannot close in its section)
__device__ __forceinline__ int64_t key15_capped(const Limbs4 &a) {
    const bool big = (int32_t)a.w3 > 0 || (a.w3 == 0 && a.w2 >= (1u << (kKeyCap62 + kKeyShift - 64)));
    return big ? ((int64_t)1 << kKeyCap62) : key15(a);
}


// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel of the stream is still running; it calls
// pdl_wait() before it reads anything that kernel (or an earlier one) wrote,
// which returns once the previous grid has finished and its writes are
// visible.  pdl_trigger() lets the next kernel start; it is issued at entry,
// so that kernel's blocks only fill the room this grid's last blocks leave.
// Neither waits on a flag: the wait ends when the previous grid ends, whose
// blocks are all resident by the time a dependent starts.  Without a
// programmatic launch both return at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
    if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {
        (void)cudaGetLastError();   // no programmatic launches: an ordinary one
        cfg.numAttrs = 0;
        e = cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
    }
    return e;
}

}  // namespace wrs
