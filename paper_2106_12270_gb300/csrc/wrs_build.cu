// wrs_build.cu - alias-table construction on GB300 (sm_103a).
//
// The PSA method (Sec. 2.2, Sec. 4 of "Weighted Random Sampling on GPUs")
// in four kernels, with integer fixed-point prefix sums:
//
//   k_sum                a1: W = sum w_i, exact (per-exponent-band integer
//                        sums, assembled by the last CTA), rounded once to
//                        FP64; avg = W/N; the scale S of the fixed point
//                        q_i = round(w_i 2^S).
//   k_count / k_scatter  a2+a3: light iff w_i <= W/N; stable partition into
//   / k_segscan          one array (lights from the front, heavies from the
//                        back, Sec. 4.2 "weight in l and h").  Persistent
//                        CTAs own contiguous segments: k_count counts each
//                        segment's lights, k_scatter places every item and
//                        writes a checkpoint of the q prefix sum every 32
//                        list entries (relative to its segment), k_segscan
//                        scans the segment sums.  No CTA waits on another,
//                        and the result does not depend on timing.
//   k_split              a4: for every section boundary k the Vose state
//                        (i lights, k-i heavies closed) by a monotone search
//                        over the checkpoints -- partial p-ary search
//                        (Algorithm 1) or plain binary search -- followed by
//                        a warp-cooperative search inside one checkpoint.
//   k_pack               a5: one CTA per section sweeps the section as a
//                        merge of the light deficit prefix D' and the heavy
//                        excess prefix E' (Sec. 2.2 "pack"), staged in shared
//                        memory (Sec. 4.2), writing rows by item index.
//
// Fixed point.  q_i = round(w_i 2^S) < 2^63 with W 2^S in [2^61, 2^62); the
// bucket is Q = sum of all q_i (exactly, so deficits and excesses balance).
// For light items d'_a = Q - N q_a >= 0 (N times its deficit) and for heavy
// items e'_b = N q_b - Q > 0.  D'(i) = sum of the first i light d', E'(j) =
// sum of the first j heavy e' (both < 2^95), exact in 128-bit integers.  The
// sweep closes heavy h[j] (its remaining weight fits in one bucket) iff
// E'(j+1) <= D'(i), both rounded down to multiples of 2^15 (sweep_le: a
// bucket is >= 2^61 units), else light l[i]; a heavy row keeps 1 - (D'(i) -
// E'(j+1)) / Q of its bucket, on the same rounded prefixes.  The split search
// and the pack use this one rule, so the splits and every section end agree
// exactly, and no FP64 unit is used per item.  The rounding of q costs at
// most N/(2Q) <= 2^-32 of a bucket per item, far below the FP32 rounding of
// the stored probabilities.
#include <stdio.h>

#include <algorithm>
#include <type_traits>

#include "wrs_device.cuh"
#include "wrs_scatter.cuh"


namespace wrs {

Layout make_layout(uint64_t n, uint32_t S) {
    Layout L;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    L.sections = (n + S - 1) / S;
    L.params = take(sizeof(BuildParams));
    L.sum_bins = take((uint64_t)kSumMaxBlocks * kSumBands * sizeof(u128));
    L.seg_cnt = take((uint64_t)kMaxSegs * 4);
    L.seg_q = take((uint64_t)kMaxSegs * 8);
    L.seg_loff = take((uint64_t)(kMaxSegs + 1) * 8);
    L.seg_sum = take((uint64_t)kMaxSegs * sizeof(SegVal));
    L.seg_pre = take((uint64_t)(kMaxSegs + 1) * sizeof(SegVal));
    L.lh = take(n * sizeof(Entry));
    L.ckl = take((n / 32 + 2) * sizeof(CkRec));
    L.ckh = take((n / 32 + 2) * sizeof(CkRec));
    L.splits = take((L.sections + 1) * sizeof(SplitRec));
    L.total = off;
    return L;
}

// ===========================================================================
// a1: exact total weight
// ===========================================================================

// Each FP32 weight m * 2^(e'-150) (e' = max(biased exponent, 1), m the
// 24-bit significand with its leading bit) goes into band e'/16 as
// m << (e' mod 16) < 2^39.  A thread sees at most 2^25 items, so its
// per-band sum stays below 2^64; blocks reduce to 128-bit sums.  NaN/Inf and
// negative weights are found from two running maxima of the bit patterns.
// The last block to finish assembles W exactly (units of 2^-150), rounds it
// to FP64 (ties to even) and derives avg, the light threshold and the
// fixed-point scale.
__global__ void __launch_bounds__(kSumThreads)
k_sum(const float *__restrict__ w, uint64_t n, u128 *__restrict__ bins_out,
      BuildParams *__restrict__ P, int aligned, uint32_t sections) {
    __shared__ uint64_t bins[kSumBands][kSumThreads];
    __shared__ u128 band[kSumBands];
    __shared__ uint32_t s_last;
    pdl_trigger();
    const int tid = threadIdx.x;
#pragma unroll
    for (int b = 0; b < kSumBands; ++b) bins[b][tid] = 0;
    uint32_t umax = 0, amax = 0;
    auto add = [&](float x) {
        const uint32_t u = __float_as_uint(x);
        const uint32_t a = u & 0x7fffffffu;
        umax = max(umax, u);
        amax = max(amax, a);
        const uint32_t ee = max(a >> 23, 1u);
        const uint32_t m = a - ((ee - 1u) << 23);
        bins[ee >> 4][tid] += (uint64_t)m << (ee & 15u);
    };
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + tid;
    uint64_t tail = 0;
    if (aligned) {
        const uint64_t n4 = n / 4;
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        for (uint64_t i = g; i < n4; i += T) {
            float4 v = __ldg(w4 + i);
            add(v.x); add(v.y); add(v.z); add(v.w);
        }
        tail = n4 * 4;
    }
    for (uint64_t i = tail + g; i < n; i += T) add(__ldg(w + i));
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int b = warp; b < kSumBands; b += kSumThreads / 32) {
        u128 s = 0;
#pragma unroll
        for (int k = 0; k < kSumThreads / 32; ++k) s += bins[b][lane + 32 * k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)s, d);
            uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(s >> 64), d);
            s += ((u128)hi << 64) | lo;
        }
        if (lane == 0) bins_out[(uint64_t)blockIdx.x * kSumBands + b] = s;
    }
    // non-finite: |bits| >= the Inf pattern; negative: a set sign bit on a
    // nonzero pattern (-0 is allowed)
    uint32_t bad = (amax >= 0x7f800000u ? ERR_NONFINITE : 0u) |
                   (umax > 0x80000000u ? ERR_NEGATIVE : 0u);
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicOr(&P->status, bad);

    // last block: reduce the bands over all blocks and assemble W
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&P->sum_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int b = warp; b < kSumBands; b += kSumThreads / 32) {
        u128 s = 0;
        for (uint32_t k = lane; k < gridDim.x; k += 32) {
            const ulonglong2 v =
                __ldcg(reinterpret_cast<const ulonglong2 *>(bins_out + (uint64_t)k * kSumBands + b));
            s += ((u128)v.y << 64) | v.x;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)s, d);
            uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(s >> 64), d);
            s += ((u128)hi << 64) | lo;
        }
        if (lane == 0) band[b] = s;
    }
    __syncthreads();
    if (tid != 0) return;
    P->n = n;
    P->sections = sections;
    double W;
    int top;
    if (!exact_total<kSumBands, 16>(band, W, top)) {
        P->W = 0.0;
        P->avg = 0.0;
        atomicOr(&P->status, ERR_ZEROSUM);
        return;
    }
    double avg = W / (double)n;
    // q_i = round(w_i 2^S) with W 2^S in [2^61, 2^62): S = 211 - top
    P->W = W;
    P->avg = avg;
    P->scale = 211 - top;
    P->qshift = 61 - top;
    P->light_max = __double2float_rd(avg);
    P->inv_avg = __double2float_rn(1.0 / avg);
}

// ===========================================================================
// a2 + a3: classify, stable partition, prefix sums (per-warp sub-segments)
// ===========================================================================



// Per sub-segment (one warp each, coalesced 16-byte loads): the number of
// light items and the sum of q over all its items (unclamped).
__global__ void __launch_bounds__(kPartThreads)
k_count(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
        uint32_t *__restrict__ seg_cnt, uint64_t *__restrict__ seg_q, uint64_t C, uint32_t NS,
        int aligned) {
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const int lane = threadIdx.x & 31;
    const uint32_t s = blockIdx.x * (kPartThreads / 32) + (threadIdx.x >> 5);
    if (s >= NS) return;
    const float lmax = P->light_max;
    const QScale qsc = qscale(P->qshift);
    uint64_t a, b;
    sub_range(s, NS, C, n, a, b);
    uint32_t cnt = 0;
    uint64_t qs = 0;
    uint64_t tail = a;
    if (aligned) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        const uint64_t b4 = b / 4;
        uint64_t i = a / 4 + lane;
        // groups of eight 16-byte loads per lane, all in flight before use
        for (; i + 7 * 32 < b4; i += 8 * 32) {
            float4 v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) v[r] = __ldg(w4 + i + 32 * r);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                cnt += (v[r].x <= lmax) + (v[r].y <= lmax) + (v[r].z <= lmax) + (v[r].w <= lmax);
                qs += fixed_q(v[r].x, qsc) + fixed_q(v[r].y, qsc) + fixed_q(v[r].z, qsc) +
                      fixed_q(v[r].w, qsc);
            }
        }
        for (; i < b4; i += 32) {
            float4 v = __ldg(w4 + i);
            cnt += (v.x <= lmax) + (v.y <= lmax) + (v.z <= lmax) + (v.w <= lmax);
            qs += fixed_q(v.x, qsc) + fixed_q(v.y, qsc) + fixed_q(v.z, qsc) + fixed_q(v.w, qsc);
        }
        tail = b4 * 4 > a ? b4 * 4 : a;
    }
    for (uint64_t i = tail + lane; i < b; i += 32) {
        float x = __ldg(w + i);
        cnt += (x <= lmax);
        qs += fixed_q(x, qsc);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, d);
    if (lane == 0) {
        seg_cnt[s] = cnt;
        seg_q[s] = qs;
    }
}

// The single-CTA scans over the sub-segments (1024 threads, kMaxSegs =
// 8 * 1024 values at most): warp w holds values 256 w + 32 k + lane, k =
// 0..7, so every load and store of a warp is contiguous; each warp scans its
// 256 values in order (eight warp scans), then one step over the 32 warp
// totals.  warp_excl_scan8 returns, for each k, the exclusive prefix of value
// (k, lane) within the warp's run, and the run's total.
template <typename T>
__device__ __forceinline__ T warp_excl_scan8(T (&v)[kMaxSegs / 1024]) {
    const int lane = threadIdx.x & 31;
    T run = 0;
#pragma unroll
    for (int k = 0; k < kMaxSegs / 1024; ++k) {
        T inc = v[k];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        const T x = v[k];
        v[k] = run + inc - x;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    return run;
}

// Exclusive prefix of this warp's run among the 32 runs, and the sum of all
// runs (two barriers; wtot holds 32 values).
template <typename T>
__device__ __forceinline__ T block_runs_prefix(T run, T *wtot, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wtot[warp] = run;
    __syncthreads();
    T pre = 0, tot = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        const T c = wtot[k];
        pre += (k < warp) ? c : (T)0;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return pre;
}

// One CTA (1024 threads): Q = sum of all q, its derived constants, and the
// global light offset of every sub-segment (exclusive scan of the counts).
__global__ void __launch_bounds__(1024)
k_qsum(BuildParams *__restrict__ P, const uint32_t *__restrict__ seg_cnt,
       const uint64_t *__restrict__ seg_q, uint64_t *__restrict__ seg_loff, uint32_t NS,
       uint64_t n) {
    __shared__ uint64_t wtot[32];
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    constexpr int kPer = kMaxSegs / 1024;
    const uint32_t s0 = (threadIdx.x >> 5) * (32 * kPer) + (threadIdx.x & 31);
    uint64_t c[kPer], qs = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        c[k] = sidx < NS ? seg_cnt[sidx] : 0;
        qs += sidx < NS ? seg_q[sidx] : 0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, d);
    uint64_t Q, ctot;
    block_runs_prefix(qs, wtot, Q);
    const uint64_t cpre = block_runs_prefix(warp_excl_scan8(c), wtot, ctot);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        if (sidx <= NS) seg_loff[sidx] = cpre + c[k];
    }
    if (threadIdx.x == 0) {
        const uint64_t Qn = Q / n;
        P->Q = Q;
        P->Qn = Qn;
        P->Qf = __ull2float_rn(Q);
        P->invQ = __frcp_rn(P->Qf);
        P->nseg = NS;
        // Clamps: a light (w <= lmax) changes only if q > Qn, i.e. w >= wq
        // with wq the least weight of q >= Qn + 1, about (Qn + 1/2) 2^-S;
        // a heavy only if w < wq.  Both lie between lmax and wq; the
        // interval covers that range (threshold_interval).
        float mid, half;
        threshold_interval(ldexp((double)Qn + 0.5, -P->scale), (double)P->light_max, mid, half);
        P->tmid = mid;
        P->thalf = half;
    }
}

// Place every item (scatter_range, wrs_scatter.cuh): each warp works alone
// on its sub-segment, whose light offset the count pass found; checkpoints
// are relative to the sub-segment (its prefix comes from the segment scan).
template <bool kAligned>
__global__ void __launch_bounds__(kPartThreads, 3)
k_scatter(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
          const uint64_t *__restrict__ seg_loff, Entry *__restrict__ lh, CkRec *__restrict__ ckl,
          CkRec *__restrict__ ckh, SegVal *__restrict__ seg_sum, uint64_t C, uint32_t NS) {
    __shared__ WarpStage stage[kPartThreads / 32];
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const int lane = threadIdx.x & 31;
    const uint32_t s = blockIdx.x * (kPartThreads / 32) + (threadIdx.x >> 5);
    if (s >= NS) return;
    ScatterCtx X;
    X.w = w;
    X.n = n;
    X.lh = lh;
    X.ckl = ckl;
    X.ckh = ckh;
    X.qsc = qscale(P->qshift);
    X.Qn = P->Qn;
    X.lmax = P->light_max;
    X.tmid = P->tmid;
    X.thalf = P->thalf;
    uint64_t a, b;
    sub_range(s, NS, C, n, a, b);
    uint64_t sl, sh;
    scatter_range<kAligned>(X, stage[threadIdx.x >> 5], s, a, b, seg_loff[s], sl, sh);
    if (lane == 0) {
        SegVal v;
        v.sl = sl;
        v.sh = sh;
        v.nl = 0;
        v.pad = 0;
        seg_sum[s] = v;
    }
}

// One CTA (1024 threads): exclusive scan over the sub-segments of (light q
// sum, heavy q sum); totals nl, nh, D'(nl), E'(nh); the checkpoints that fall
// on the very end of a list.
__global__ void __launch_bounds__(1024)
k_segscan(BuildParams *__restrict__ P, const uint64_t *__restrict__ seg_loff,
          const SegVal *__restrict__ seg_sum, SegVal *__restrict__ seg_pre,
          CkRec *__restrict__ ckl, CkRec *__restrict__ ckh, uint64_t n, uint32_t NS) {
    __shared__ uint64_t wtot[32];
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    constexpr int kPer = kMaxSegs / 1024;
    const uint32_t s0 = (threadIdx.x >> 5) * (32 * kPer) + (threadIdx.x & 31);
    // the light sums, then the heavy sums (one array of values live at a time)
    uint64_t v[kPer], Ltot, Htot;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        v[k] = sidx < NS ? (uint64_t)seg_sum[sidx].sl : 0;
    }
    const uint64_t lpre = block_runs_prefix(warp_excl_scan8(v), wtot, Ltot);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        if (sidx <= NS) seg_pre[sidx].sl = lpre + v[k];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        v[k] = sidx < NS ? (uint64_t)seg_sum[sidx].sh : 0;
    }
    const uint64_t hpre = block_runs_prefix(warp_excl_scan8(v), wtot, Htot);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t sidx = s0 + 32 * k;
        if (sidx <= NS) {
            seg_pre[sidx].sh = hpre + v[k];
            seg_pre[sidx].nl = seg_loff[sidx];
            seg_pre[sidx].pad = 0;
        }
    }
    if (threadIdx.x == 0) {
        const uint64_t Q = P->Q;
        const uint64_t nl = seg_loff[NS], nh = n - nl;
        P->nl = nl;
        P->nh = nh;
        P->Dtot = (u128)nl * Q - (u128)Ltot * n;
        P->Etot = (u128)Htot * n - (u128)nh * Q;
        if ((nl & 31u) == 0) put_ck(ckl, nl >> 5, NS, 0);
        if ((nh & 31u) == 0) put_ck(ckh, nh >> 5, NS, 0);
    }
}

// ===========================================================================
// a4: splits
// ===========================================================================

struct SplitCtx {
    const CkRec *ckl, *ckh;
    const SegVal *seg_pre;
    const Entry *lh;
    uint64_t n, nl, nh;
    uint64_t Q;
};

// D'(32c) = 32c*Q - N*(q sum of the first 32c light entries).
__device__ __forceinline__ u128 ck_D(const SplitCtx &C, uint64_t c) {
    uint4 r = __ldg(reinterpret_cast<const uint4 *>(C.ckl + c));
    uint64_t local = ((uint64_t)r.w << 32) | r.z;
    uint64_t sig = __ldg(reinterpret_cast<const unsigned long long *>(&C.seg_pre[r.x].sl)) + local;
    return (u128)(32 * c) * C.Q - (u128)sig * C.n;
}
// E'(32c) = N*(q sum of the first 32c heavy entries) - 32c*Q.
__device__ __forceinline__ u128 ck_E(const SplitCtx &C, uint64_t c) {
    uint4 r = __ldg(reinterpret_cast<const uint4 *>(C.ckh + c));
    uint64_t local = ((uint64_t)r.w << 32) | r.z;
    uint64_t sig = __ldg(reinterpret_cast<const unsigned long long *>(&C.seg_pre[r.x].sh)) + local;
    return (u128)sig * C.n - (u128)(32 * c) * C.Q;
}

// P(32c) for bucket count k: monotone in c; false below the valid range of
// i, true from its upper end on, E'(k-32c) <= D'(32c) inside.
__device__ __forceinline__ bool pred_c(const SplitCtx &C, uint64_t k, uint64_t c) {
    uint64_t lo = k > C.nh ? k - C.nh : 0;
    uint64_t hi = k < C.nl ? k : C.nl;
    uint64_t i = 32 * c;
    if (i < lo) return false;
    if (i >= hi) return true;
    return sweep_le(ck_E(C, (k - i) >> 5), ck_D(C, c));
}

__device__ __forceinline__ void crange(const SplitCtx &C, uint64_t k, uint64_t &clo,
                                       uint64_t &chi) {
    uint64_t lo = k > C.nh ? k - C.nh : 0;
    uint64_t hi = k < C.nl ? k : C.nl;
    clo = lo / 32;
    chi = (hi + 31) / 32;
}

// Given the smallest c with P(32c), finish the split for bucket count k with
// one warp: the answer is in (32(c-1), 32c]; lane x tests i = 32(c-1)+1+x.
__device__ void split_fine(const SplitCtx &C, const BuildParams &Pm, uint64_t k, uint64_t c,
                           u128 Dbase, u128 Ebase, SplitRec *out, int lane) {
    uint64_t lo = k > C.nh ? k - C.nh : 0;
    uint64_t hi = k < C.nl ? k : C.nl;
    const uint32_t N = (uint32_t)C.n;
    uint64_t ans;
    u128 Dv, Ev;
    if (c == 0) {
        ans = 0;
        Dv = 0;
        Ev = Ebase;   // E'(k)
    } else {
        uint64_t lb = 32 * (c - 1);  // light base
        uint64_t hb = k - 32 * c;    // heavy base, multiple of 32
        u128 d = 0, e = 0;
        if (lb + lane < C.nl) {
            Entry en = C.lh[lb + lane];
            d = (u128)(Pm.Q - N * light_q(en.w, qscale(Pm.qshift), Pm.Qn));   // <= Q
        }
        if (hb + lane < C.nh) {
            Entry en = C.lh[C.n - 1 - (hb + lane)];
            e = mul_nq(N, heavy_q(en.w, qscale(Pm.qshift), Pm.Qn)) - Pm.Q;
        }
        u128 dinc = d, einc = e;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            u128 a = shfl_up_u128(dinc, s), b = shfl_up_u128(einc, s);
            if (lane >= s) { dinc += a; einc += b; }
        }
        u128 eexc = einc - e;
        // Dbase = D'(32(c-1)) and Ebase = E'(hb), found by the coarse phase
        u128 Dl = Dbase + dinc;                                   // D'(lb + 1 + lane)
        u128 Eh = Ebase + shfl_u128(eexc, 31 - lane);             // E'(k - (lb + 1 + lane))
        uint64_t i = lb + 1 + lane;
        bool ok = i >= lo && i <= hi && (i == hi || sweep_le(Eh, Dl));
        uint32_t bal = __ballot_sync(0xffffffffu, ok);
        int first = bal ? __ffs(bal) - 1 : 31;
        ans = lb + 1 + first;
        Dv = shfl_u128(Dl, first);
        Ev = shfl_u128(Eh, first);
    }
    if (lane == 0) {
        SplitRec r;
        r.i = (uint32_t)ans;
        r.j = (uint32_t)(k - ans);
        r.pad[0] = r.pad[1] = 0;
        r.D = Dv;
        r.E = Ev;
        *out = r;
    }
}

// Interior splits t = 1..s-1, one thread each (k = t*S is a multiple of 32).
// kPary: Algorithm 1 first narrows the block's shared range of c with
// kSplitThreads pivots, judging "below every answer" with the block's first
// split and "at or above every answer" with its last; it repeats while the
// range shrinks to at most half.  Then each thread binary-searches its own c
// inside the shared range.  Without kPary each thread searches alone.
template <bool kPary>
__global__ void __launch_bounds__(kSplitThreads)
k_split(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
        const CkRec *__restrict__ ckl, const CkRec *__restrict__ ckh,
        const SegVal *__restrict__ seg_pre, SplitRec *__restrict__ splits, uint64_t n,
        uint64_t S, uint32_t sections) {
    __shared__ unsigned long long s_a, s_b;
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const BuildParams Pm = *P;
    SplitCtx C;
    C.ckl = ckl; C.ckh = ckh; C.seg_pre = seg_pre; C.lh = lh; C.n = n; C.nl = Pm.nl;
    C.nh = Pm.nh; C.Q = Pm.Q;
    const int tid = threadIdx.x;
    const uint64_t t0 = 1 + (uint64_t)blockIdx.x * kSplitThreads;   // first split of block
    const uint64_t t = t0 + tid;
    const uint64_t tlast_blk = min((uint64_t)sections - 1, t0 + kSplitThreads - 1);
    const bool active = t < sections;
    const uint64_t k = t * S;
    uint64_t clo = 0, chi = 0;
    if (active) crange(C, k, clo, chi);

    uint64_t a = clo, b = chi;   // the answer c* of this split lies in [a, b]
    if (kPary) {
        uint64_t kf = t0 * S, kl = tlast_blk * S, dummy;
        uint64_t A, B;
        crange(C, kf, A, dummy);
        crange(C, kl, dummy, B);
        if (A > B) A = B;
        for (;;) {
            uint64_t width = B - A;
            if (width < kSplitThreads) break;
            if (tid == 0) { s_a = A; s_b = B; }
            __syncthreads();
            uint64_t s = A + (width * (uint64_t)tid) / (kSplitThreads - 1);
            if (!pred_c(C, kf, s)) atomicMax(&s_a, (unsigned long long)(s + 1));
            else if (pred_c(C, kl, s)) atomicMin(&s_b, (unsigned long long)s);
            __syncthreads();
            uint64_t nA = s_a, nB = s_b;
            __syncthreads();
            if (nB < nA) nB = nA;
            bool shrink = 2 * (nB - nA) <= width;
            A = nA;
            B = nB;
            if (!shrink) break;
        }
        if (A > a) a = A;
        if (B < b) b = B;
        if (a > b) a = b;
    }
    if (active) {
        while (a < b) {
            uint64_t m = a + (b - a) / 2;
            if (pred_c(C, k, m)) b = m;
            else a = m + 1;
        }
        // the checkpoint index for the fine search (< 2^26) and the two exact
        // prefixes it starts from, parked in the record the fine search
        // then writes in full
        SplitRec &r = splits[t];
        r.pad[0] = (uint32_t)a;
        if (a > 0) {
            r.D = ck_D(C, a - 1);
            r.E = ck_E(C, (k - 32 * a) >> 5);
        } else {
            r.D = 0;
            r.E = ck_E(C, k >> 5);
        }
    }
}

// Fine phase of the interior splits: one warp per split (many in flight, so
// the dependent loads of the warp search overlap across the GPU).
__global__ void __launch_bounds__(kSplitThreads, 8)
k_split_fine(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
             const CkRec *__restrict__ ckl, const CkRec *__restrict__ ckh,
             const SegVal *__restrict__ seg_pre, SplitRec *__restrict__ splits, uint64_t n,
             uint64_t S, uint32_t sections) {
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    const uint64_t t = 1 + (uint64_t)blockIdx.x * (kSplitThreads / 32) + (threadIdx.x >> 5);
    if (t >= sections) return;
    const BuildParams Pm = *P;
    SplitCtx C;
    C.ckl = ckl; C.ckh = ckh; C.seg_pre = seg_pre; C.lh = lh; C.n = n; C.nl = Pm.nl;
    C.nh = Pm.nh; C.Q = Pm.Q;
    const uint64_t c = splits[t].pad[0];
    const u128 Dbase = splits[t].D, Ebase = splits[t].E;
    __syncwarp();
    split_fine(C, Pm, t * S, c, Dbase, Ebase, splits + t, threadIdx.x & 31);
}

// Splits 0 and s (the whole table's ends).
__global__ void k_split_ends(const BuildParams *__restrict__ P, SplitRec *__restrict__ splits,
                             uint32_t sections) {
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    SplitRec r0, rs;
    r0.i = r0.j = 0; r0.pad[0] = r0.pad[1] = 0; r0.D = 0; r0.E = 0;
    rs.i = (uint32_t)P->nl; rs.j = (uint32_t)P->nh; rs.pad[0] = rs.pad[1] = 0;
    rs.D = P->Dtot; rs.E = P->Etot;
    splits[0] = r0;
    splits[sections] = rs;
}

// ===========================================================================
// a5: pack
// ===========================================================================

// Pack (Sec. 2.2 "pack", staged in shared memory as in Sec. 4.2): each
// section of up to S buckets is swept by one CTA of S/kPer threads, each
// owning kPer consecutive positions of the sweep.
//
// The sweep closes heavy h[j] before light l[i] iff its excess prefix does
// not exceed the deficit prefix, compared at a resolution of 2^kKeyShift
// units (wrs_internal.cuh, sweep_le): floor(E'(j+1) / 2^15) <= floor(D'(i) /
// 2^15).  Inside a section the keys are those floors relative to the
// section start, as 64-bit integers:
//   A(x) = floor(D'(i0+x) / 2^15) - floor(D0 / 2^15)   in [0, 2^61]
//   B(y) = floor(E'(j0+y+1) / 2^15) - floor(D0 / 2^15) > -2^48
// (B(0) > -Q because the split took the smallest i; B is capped at 2^62,
// above every A: a capped heavy cannot close in the section.  A sentinel
// key after the section's last heavy lies above every A as well.)  The
// prefix sums themselves are exact (128-bit); only the stored keys are
// rounded, the same way everywhere, so the table does not depend on the
// section size.

// Shared memory: sK (keys: slot x = A(x), slot L+y+1 = B(y)) and sE (the
// section's entries: lights, heavies, then the first heavy after the
// section); both pad one 8-byte slot in 16 against bank conflicts.
__host__ __device__ inline uint32_t pk16(uint32_t e) { return e + (e >> 4); }
__host__ __device__ inline uint32_t pack_per(uint32_t S) { return S <= 4096 ? 8 : 16; }
__host__ __device__ inline uint32_t pack_slots(uint32_t S) { return pk16(S + 1) + 1; }
__host__ __device__ inline uint32_t pack_smem_bytes(uint32_t S) { return 16 * pack_slots(S); }


template <int kPer>
__device__ __forceinline__ void pack_section(const BuildParams *__restrict__ P,
                                             const Entry *__restrict__ lh,
                                             const SplitRec *__restrict__ splits,
                                             uint2 *__restrict__ rows, uint64_t n, uint32_t S,
                                             uint32_t t) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u128 s_w[16];
    pdl_trigger();
    pdl_wait();
    if (P->status) return;
    int64_t *sK = reinterpret_cast<int64_t *>(smem);
    uint2 *sE = reinterpret_cast<uint2 *>(smem + 8 * pack_slots(S));

    const uint32_t T = blockDim.x;
    const uint32_t tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t nh = P->nh;
    const uint64_t Q = P->Q, Qn = P->Qn;
    const uint32_t N = (uint32_t)n;
    const QScale qsc = qscale(P->qshift);
    const float inv_avg = P->inv_avg;
    const float invQk = P->invQ * (float)(1u << kKeyShift);   // 1/Q per key unit
    const SplitRec R0 = splits[t], R1 = splits[t + 1];
    const uint32_t i0 = R0.i, j0 = R0.j;
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j, K = L + H;
    const uint32_t extra = (R1.j < nh) ? 1u : 0u;
    if (R1.i < R0.i || R1.j < R0.j || K > S || R1.i > P->nl || R1.j > nh) {
        if (tid == 0) atomicOr(const_cast<uint32_t *>(&P->status), ERR_INTERNAL);
        return;   // inconsistent splits: write nothing
    }

    // phase 1: asynchronous copies of the section's lights, heavies and the
    // next heavy item straight into shared memory
    {
        const uint2 *lh2 = reinterpret_cast<const uint2 *>(lh);
#pragma unroll
        for (int r = 0; r <= kPer; ++r) {
            const uint32_t e = tid + r * T;
            if (e < K + extra) {
                const uint2 *src = lh2 + (e < L ? (uint64_t)i0 + e : n - 1 - ((uint64_t)j0 + (e - L)));
                const uint32_t d = (uint32_t)__cvta_generic_to_shared(sE + pk16(e));
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();

    // phase 2: the clamped fixed point q of each owned position (kept in
    // registers) and the thread's exact value sum: sum over lights of d' = Q
    // - N q and over heavies of e' = N q - Q, i.e. (nl - nh) Q + N (sum of
    // heavy q - sum of light q); then a block scan of the thread sums.
    const uint32_t b0 = tid * kPer;
    // positions b0 .. b0+nlt-1 are lights, b0+nlt .. b0+nvt-1 heavies
    const uint32_t nlt = L > b0 ? min(L - b0, (uint32_t)kPer) : 0u;
    const uint32_t nvt = K > b0 ? min(K - b0, (uint32_t)kPer) : 0u;
    uint64_t qv[kPer];
    uint64_t sql = 0, sqh = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        uint64_t q = fixed_q(__uint_as_float(sE[pk16(b0 + k)].y), qsc);
        if ((uint32_t)k < nlt) {
            q = q > Qn ? Qn : q;
            sql += q;
        } else {
            q = q <= Qn ? Qn + 1 : q;
            sqh += (uint32_t)k < nvt ? q : 0ull;
        }
        qv[k] = q;
    }
    // the thread's value sum N (sqh - sql) + (nlt - nht) Q, two's complement
    u128 run;
    {
        const bool neg = sqh < sql;
        const uint64_t mag = neg ? sql - sqh : sqh - sql;   // < 2^63
        const uint64_t lo = (uint64_t)(uint32_t)mag * N;
        const uint64_t hi = (uint64_t)(uint32_t)(mag >> 32) * N;
        u128 v = (u128)lo + ((u128)hi << 32);
        const int c = 2 * (int)nlt - (int)nvt;                // nlt - nht
        const uint64_t cm = (uint64_t)(c < 0 ? -c : c);
        const u128 cq = (u128)((uint64_t)(uint32_t)Q * cm) + ((u128)((Q >> 32) * cm) << 32);
        run = (neg ? (u128)0 - v : v) + (c < 0 ? (u128)0 - cq : cq);
    }
    u128 inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u128 o = shfl_up_u128(inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();

    // phase 3: keys.  With P(e) the exact prefix of the values: D'(i0+x) =
    // D0 + P(x), so A(x) = floor((D0 mod 2^15 + P(x)) / 2^15); E'(j0+y+1) =
    // E0 + P(L+y+1) - P(L) with P(L) = D1 - D0 (the section's light deficit,
    // fixed by the split), so B(y) = floor((E0 - D1 + D0 mod 2^15 +
    // P(L+y+1)) / 2^15).  The running value is kept in 32-bit limbs: a light
    // adds its deficit Q - N q (< 2^63), a heavy its excess N q - Q; the heavy
    // keys run on ch + p.
    {
        const u128 d0l = R0.D & (u128)((1u << kKeyShift) - 1);
        u128 p = inc - run + d0l;
        for (int k = 0; k < warp; ++k) p += s_w[k];
        const u128 ch = R0.E - R1.D;
        if (tid == 0) {
            sK[pk16(0)] = 0;
            sK[pk16(K + 1)] = INT64_MAX;   // after the last heavy: never closes
        }
        Limbs4 a = to_limbs(nlt > 0 ? p : ch + p);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t e = b0 + k;
            if ((uint32_t)k < nlt) {
                add96(a, Q - mul_lo_nq(N, qv[k]));
                sK[pk16(e + 1)] = key15(a);   // < 2^61
                if ((uint32_t)k + 1 == nlt && nlt < nvt) a = to_limbs(ch + from_limbs(a));
            } else if ((uint32_t)k < nvt) {
                add_excess(a, N, qv[k], Q);
                sK[pk16(e + 1)] = key15_capped(a);
            }
        }
        // the section's own sums must meet the split's: the thread holding
        // position K-1 has P(K) = D1 - D0 + E1 - E0
        if (b0 < K && b0 + kPer >= K) {
            const u128 pend = from_limbs(a) - (nvt > nlt ? ch : (u128)0);
            if (pend - d0l != (R1.D - R0.D) + (R1.E - R0.E))
                atomicOr(const_cast<uint32_t *>(&P->status), ERR_INTERNAL);
        }
    }
    __syncthreads();

    // phase 4: merge path.  The number x of lights closed before position d0
    // is the smallest x with B(d0-x-1) <= A(x) (or x = L, or x = d0).
    auto Av = [&](uint32_t x) { return sK[pk16(x)]; };
    auto Bv = [&](uint32_t y) { return sK[pk16(L + y + 1)]; };
    const uint32_t d0 = b0;
    if (d0 < K) {
        uint32_t lo = d0 > H ? d0 - H : 0, hi = d0 < L ? d0 : L;
        while (lo < hi) {
            const uint32_t m = (lo + hi) >> 1;
            // m < hi <= min(d0, L): both neighbours exist
            const bool p = Bv(d0 - m - 1) <= Av(m);
            if (p) hi = m;
            else lo = m + 1;
        }
        uint32_t x = lo, y = d0 - lo;
        int64_t a = Av(x);
        int64_t b = Bv(y);   // y = H reads the sentinel
        // one output per step: close heavy y (b <= a, or no light left) or
        // light x.  The next heavy in the list fills the bucket's rest: list
        // offset y+1 for a heavy, y for a light (sE slot K holds the first
        // heavy after the section); without one the item keeps its bucket.
        // A heavy keeps 1 - (A - B) 2^15 / Q of its bucket.
        const uint32_t hleft = (uint32_t)min(nh - (uint64_t)j0, (uint64_t)K + 1);
        // hcur: item of heavy y, the one that fills the next light bucket
        uint32_t hcur = y < hleft ? sE[pk16(L + y)].x : 0u;
        auto merge = [&](auto kFull) {
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                if (d0 + k < K) {
                    // (y = H leaves b at the sentinel, above every key)
                    const bool heavy = x == L || b <= a;
                    // one entry load per step: the closed light (item and
                    // weight), or the heavy after the closed one (its item)
                    const uint2 ld = sE[pk16(heavy ? L + y + 1 : x)];
                    const uint32_t item = heavy ? hcur : ld.x;
                    const bool has = decltype(kFull)::value || (heavy ? y + 1 : y) < hleft;
                    uint32_t alias = item;
                    float prob = 1.0f;
                    if (has) {
                        alias = heavy ? ld.x : hcur;
                        prob = heavy ? fminf(fmaxf(1.0f - __ll2float_rn(a - b) * invQk, 0.0f), 1.0f)
                                     : fminf(__uint_as_float(ld.y) * inv_avg, 1.0f);
                    }
                    rows[item] = make_uint2(__float_as_uint(prob), alias);
                    const int64_t v = sK[pk16(heavy ? L + y + 2 : x + 1)];
                    if (heavy) { ++y; b = v; hcur = ld.x; }
                    else { ++x; a = v; }
                }
            }
        };
        // every closed item has a next heavy unless the heavy list ends
        // within K + 1 entries of the section's first heavy
        if (hleft > K) merge(std::true_type());
        else merge(std::false_type());
    }
}

// Sections of up to 4096 buckets: 8 positions per thread, at most 48
// registers (10 CTAs of 128 threads per SM at S = 1024).
__global__ void __maxnreg__(48)
k_pack8(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
        const SplitRec *__restrict__ splits, uint2 *__restrict__ rows, uint64_t n, uint32_t S) {
    pack_section<8>(P, lh, splits, rows, n, S, blockIdx.x);
}
// Larger sections: 16 positions per thread, 512 threads.
__global__ void __launch_bounds__(512)
k_pack16(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
         const SplitRec *__restrict__ splits, uint2 *__restrict__ rows, uint64_t n, uint32_t S) {
    pack_section<16>(P, lh, splits, rows, n, S, blockIdx.x);
}


// ===========================================================================
// Segmented batched build: split and pack of every table's sections
// ===========================================================================

BatchSegLayout batch_seg_layout(uint64_t cap, uint32_t ntab) {
    BatchSegLayout L;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    L.cap = cap;
    L.counters = take(256);
    L.lh = take(cap * sizeof(Entry));
    L.tp = take((uint64_t)ntab * sizeof(BuildParams));
    L.tabs = take((uint64_t)ntab * sizeof(BatchTab));
    L.sec_tab = take((cap / kBSeg + ntab + 1) * 4);
    L.ckl = take(((cap >> 5) + 2ull * ntab + 2) * sizeof(CkRec));
    L.ckh = take(((cap >> 5) + 2ull * ntab + 2) * sizeof(CkRec));
    L.recs = take((cap / kBSeg + 2ull * ntab + 1) * sizeof(SplitRec));
    L.zero = take(sizeof(SegVal));
    L.lists = take(2ull * ntab * 4);
    L.total = off;
    return L;
}

__device__ __forceinline__ SplitCtx bseg_ctx(const BuildParams &Pm, const BatchTab &tb, uint32_t t,
                                             const Entry *lh, const CkRec *ckl, const CkRec *ckh,
                                             const SegVal *zero) {
    SplitCtx C;
    const uint64_t ckb = bseg_ck(tb.base, t, 0);
    C.ckl = ckl + ckb;
    C.ckh = ckh + ckb;
    C.seg_pre = zero;   // checkpoints hold table-local sums (segment 0, prefix 0)
    C.lh = lh + tb.base;
    C.n = Pm.n;
    C.nl = Pm.nl;
    C.nh = Pm.nh;
    C.Q = Pm.Q;
    return C;
}

// Interior splits of every table: one warp per section j >= 1 of a table
// finds split j (k = j kBSeg buckets): a 32-ary search over the table's
// checkpoints for the smallest c with E'(k - 32c) <= D'(32c) (under the
// sweep's rule), then the fine search inside 32 entries (split_fine).  The
// partition kernel wrote splits 0 and s of each table.
__global__ void __launch_bounds__(256)
k_bseg_split(const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ sec_tab,
             const BatchTab *__restrict__ tabs, const BuildParams *__restrict__ tp,
             const Entry *__restrict__ lh, const CkRec *__restrict__ ckl,
             const CkRec *__restrict__ ckh, const SegVal *__restrict__ zero,
             SplitRec *__restrict__ recs) {
    pdl_trigger();
    pdl_wait();
    const uint32_t sec = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (sec >= ctr[1]) return;
    const uint32_t t = sec_tab[sec];
    const BatchTab tb = tabs[t];
    const uint32_t j = sec - tb.sec0;
    if (j == 0) return;
    const BuildParams Pm = tp[t];
    if (Pm.status) return;
    const SplitCtx C = bseg_ctx(Pm, tb, t, lh, ckl, ckh, zero);
    const uint64_t k = (uint64_t)j * kBSeg;
    uint64_t a, b;
    crange(C, k, a, b);   // the answer c lies in [a, b]; P(b) holds
    while (a < b) {
        const uint64_t step = (b - a + 31) / 32;
        const uint64_t p = a + (uint64_t)lane * step;
        const uint32_t bal = __ballot_sync(0xffffffffu, p < b && pred_c(C, k, p));
        if (bal) {
            const uint32_t f = __ffs(bal) - 1;   // P false before a + f step, true there
            b = a + f * step;
            if (f) a = a + (f - 1) * step + 1;
        } else {
            const uint64_t last = min((uint64_t)31, (b - 1 - a) / step);
            a = a + last * step + 1;
        }
    }
    u128 Dbase, Ebase;
    if (a > 0) {
        Dbase = ck_D(C, a - 1);
        Ebase = ck_E(C, (k - 32 * a) >> 5);
    } else {
        Dbase = 0;
        Ebase = ck_E(C, k >> 5);
    }
    split_fine(C, Pm, k, a, Dbase, Ebase, recs + tb.rec0 + j, lane);
}

// Pack of every table's sections: one CTA of kBSeg / 8 threads per section,
// the single-table pack on the table's lists, parameters and splits; rows
// by table-local item index.
__global__ void __maxnreg__(48)
k_bseg_pack(const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ sec_tab,
            const BatchTab *__restrict__ tabs, BuildParams *__restrict__ tp,
            const Entry *__restrict__ lh, const SplitRec *__restrict__ recs,
            uint2 *__restrict__ rows, uint2 *const *__restrict__ row_ptrs) {
    pdl_trigger();
    pdl_wait();
    const uint32_t sec = blockIdx.x;
    if (sec >= ctr[1]) return;
    const uint32_t t = sec_tab[sec];
    const BatchTab tb = tabs[t];
    uint2 *rt = row_ptrs ? row_ptrs[t] : rows + tb.base;
    pack_section<8>(tp + t, lh + tb.base, recs + tb.rec0, rt, tp[t].n, kBSeg, sec - tb.sec0);
}

// A table whose split or pack found an inconsistency reports it.
__global__ void k_bseg_info(const BuildParams *__restrict__ tp, uint32_t ntab,
                            wrs_table_summary *__restrict__ info) {
    pdl_wait();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntab && (tp[t].status & ERR_INTERNAL)) info[t].status = WRS_EINVAL;
}

cudaError_t launch_bseg_split_pack(unsigned char *ws, const BatchSegLayout &L, uint32_t ntab,
                                   wrs_row *d_rows, wrs_row *const *d_row_ptrs,
                                   wrs_table_summary *d_info, cudaStream_t st) {
    const uint32_t smem = pack_smem_bytes(kBSeg);
    cudaError_t e = ensure_dynamic_smem<k_bseg_pack>(smem);
    if (e) return e;
    auto *ctr = reinterpret_cast<const uint32_t *>(ws + L.counters);
    auto *sec_tab = reinterpret_cast<const uint32_t *>(ws + L.sec_tab);
    auto *tabs = reinterpret_cast<const BatchTab *>(ws + L.tabs);
    auto *tp = reinterpret_cast<BuildParams *>(ws + L.tp);
    auto *lh = reinterpret_cast<const Entry *>(ws + L.lh);
    auto *ckl = reinterpret_cast<const CkRec *>(ws + L.ckl);
    auto *ckh = reinterpret_cast<const CkRec *>(ws + L.ckh);
    auto *zero = reinterpret_cast<const SegVal *>(ws + L.zero);
    auto *recs = reinterpret_cast<SplitRec *>(ws + L.recs);
    const uint64_t maxsec = L.cap / kBSeg + ntab;   // an upper bound of the sections
    if (maxsec >= (1ull << 31)) return cudaErrorInvalidValue;
    e = launch_pdl(k_bseg_split, dim3((unsigned)((maxsec + 7) / 8)), dim3(256), 0, st, ctr, sec_tab,
                   tabs, (const BuildParams *)tp, lh, ckl, ckh, zero, recs);
    if (!e)
        e = launch_pdl(k_bseg_pack, dim3((unsigned)maxsec), dim3(kBSeg / 8), smem, st, ctr, sec_tab,
                       tabs, tp, lh, (const SplitRec *)recs,
                       reinterpret_cast<uint2 *>(d_rows), reinterpret_cast<uint2 *const *>(d_row_ptrs));
    if (!e)
        e = launch_pdl(k_bseg_info, dim3((ntab + 255) / 256), dim3(256), 0, st,
                       (const BuildParams *)tp, ntab, d_info);
    return e;
}

// ===========================================================================
// build summary
// ===========================================================================
__global__ void k_info(const BuildParams *__restrict__ P, wrs_build_info *__restrict__ out) {
    pdl_wait();
    uint32_t st = P->status;
    wrs_build_info r;
    r.status = (st & ERR_NONFINITE) ? WRS_ENONFINITE
             : (st & (ERR_NEGATIVE | ERR_INTERNAL)) ? WRS_EINVAL
             : (st & ERR_ZEROSUM) ? WRS_EZEROSUM : WRS_OK;
    r.scale = P->scale;
    r.W = P->W;
    r.avg = P->avg;
    r.nl = P->nl;
    r.nh = P->nh;
    r.Q[0] = (uint32_t)P->Q;
    r.Q[1] = (uint32_t)(P->Q >> 32);
    r.Q[2] = r.Q[3] = 0;
    r.light_max = P->light_max;
    r.sections = P->sections;
    for (int k = 0; k < 4; ++k) r.reserved[k] = 0;
    *out = r;
}

// ===========================================================================
// host launchers
// ===========================================================================

// SM count of the current device (cached per device; any positive value
// gives valid grids, so a race only repeats the query).
int num_sms() {
    static std::atomic<int> sms[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = dev >= 0 && dev < kMaxDevices ? dev : 0;
    int v = sms[slot].load(std::memory_order_relaxed);
    if (v <= 0) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 152;
        sms[slot].store(v, std::memory_order_relaxed);
    }
    return v;
}

cudaError_t launch_total(const float *d_w, uint64_t n, unsigned char *ws, const Layout &L,
                         cudaStream_t st) {
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    cudaError_t err = cudaMemsetAsync(P, 0, sizeof(BuildParams), st);
    if (err) return err;
    // one wave of CTAs (six fit on an SM), at least 4096 items each
    const uint64_t cap = std::min<uint64_t>((uint64_t)num_sms() * 6, kSumMaxBlocks);
    uint64_t want = (n + 4095) / 4096;
    int blocks = (int)(want < cap ? (want ? want : 1) : cap);
    int aligned = ((uintptr_t)d_w % 16) == 0;
    k_sum<<<blocks, kSumThreads, 0, st>>>(d_w, n, reinterpret_cast<u128 *>(ws + L.sum_bins), P,
                                           aligned, (uint32_t)L.sections);
    return cudaGetLastError();
}

// One wave of partition CTAs (kSegPerSM resident per SM, one sub-segment per
// warp); tables of 2^28 items and more take two waves of half-size
// sub-segments, which evens out the CTAs that finish last.
uint32_t num_segments(uint64_t n) {
    const uint64_t C = (n + kChunk - 1) / kChunk;
    const uint64_t waves = n >= (1ull << 28) ? 2 : 1;
    uint64_t g = (uint64_t)num_sms() * kSegPerSM * (kPartThreads / 32) * waves;
    if (g > (uint64_t)kMaxSegs - 1) g = kMaxSegs - 1;
    if (g > C) g = C;
    return (uint32_t)(g ? g : 1);
}

// The light counts and the q sum of every sub-segment, then Q and the light
// offsets (the part of the partition that PSA+ shares).
cudaError_t launch_count(const float *d_w, uint64_t n, unsigned char *ws, const Layout &L,
                         cudaStream_t st) {
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    auto *cnt = reinterpret_cast<uint32_t *>(ws + L.seg_cnt);
    auto *segq = reinterpret_cast<uint64_t *>(ws + L.seg_q);
    auto *loff = reinterpret_cast<uint64_t *>(ws + L.seg_loff);
    const uint64_t C = (n + kChunk - 1) / kChunk;
    const uint32_t NS = num_segments(n);
    const unsigned blocks = (NS + kPartThreads / 32 - 1) / (kPartThreads / 32);
    const int aligned = ((uintptr_t)d_w % 16) == 0;
    // plain launches (see launch_partition)
    k_count<<<blocks, kPartThreads, 0, st>>>(d_w, n, P, cnt, segq, C, NS, aligned);
    k_qsum<<<1, 1024, 0, st>>>(P, cnt, segq, loff, NS, n);
    return cudaGetLastError();
}

cudaError_t launch_partition(const float *d_w, uint64_t n, unsigned char *ws, const Layout &L,
                             cudaStream_t st) {
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    auto *cnt = reinterpret_cast<uint32_t *>(ws + L.seg_cnt);
    auto *segq = reinterpret_cast<uint64_t *>(ws + L.seg_q);
    auto *loff = reinterpret_cast<uint64_t *>(ws + L.seg_loff);
    auto *sum = reinterpret_cast<SegVal *>(ws + L.seg_sum);
    auto *pre = reinterpret_cast<SegVal *>(ws + L.seg_pre);
    auto *lh = reinterpret_cast<Entry *>(ws + L.lh);
    auto *ckl = reinterpret_cast<CkRec *>(ws + L.ckl);
    auto *ckh = reinterpret_cast<CkRec *>(ws + L.ckh);
    const uint64_t C = (n + kChunk - 1) / kChunk;
    const uint32_t NS = num_segments(n);
    const unsigned blocks = (NS + kPartThreads / 32 - 1) / (kPartThreads / 32);
    const int aligned = ((uintptr_t)d_w % 16) == 0;
    // Plain launches: the count and scatter grids are sized in whole waves
    // of resident CTAs, and blocks launched early as programmatic
    // dependents land unevenly while the previous kernel drains (2^30
    // build: 10.77 ms plain, 11.47 ms with these four chained).  The split,
    // pack and summary that follow are chained.
    k_count<<<blocks, kPartThreads, 0, st>>>(d_w, n, P, cnt, segq, C, NS, aligned);
    k_qsum<<<1, 1024, 0, st>>>(P, cnt, segq, loff, NS, n);
    if (aligned)
        k_scatter<true><<<blocks, kPartThreads, 0, st>>>(d_w, n, P, loff, lh, ckl, ckh, sum, C, NS);
    else
        k_scatter<false><<<blocks, kPartThreads, 0, st>>>(d_w, n, P, loff, lh, ckl, ckh, sum, C,
                                                          NS);
    k_segscan<<<1, 1024, 0, st>>>(P, loff, sum, pre, ckl, ckh, n, NS);
    return cudaGetLastError();
}

cudaError_t launch_split(uint64_t n, unsigned char *ws, const Layout &L, uint32_t S,
                         uint32_t method, cudaStream_t st) {
    const BuildParams *P = reinterpret_cast<const BuildParams *>(ws + L.params);
    auto *lh = reinterpret_cast<const Entry *>(ws + L.lh);
    auto *ckl = reinterpret_cast<const CkRec *>(ws + L.ckl);
    auto *ckh = reinterpret_cast<const CkRec *>(ws + L.ckh);
    auto *pre = reinterpret_cast<const SegVal *>(ws + L.seg_pre);
    auto *sp = reinterpret_cast<SplitRec *>(ws + L.splits);
    uint32_t s = (uint32_t)L.sections;
    cudaError_t e = launch_pdl(k_split_ends, dim3(1), dim3(1), 0, st, P, sp, s);
    if (!e && s > 1) {
        unsigned blocks = (unsigned)((s - 1 + kSplitThreads - 1) / kSplitThreads);
        e = launch_pdl(method == WRS_SPLIT_BINARY ? k_split<false> : k_split<true>, dim3(blocks),
                       dim3(kSplitThreads), 0, st, P, lh, ckl, ckh, pre, sp, n, (uint64_t)S, s);
        const unsigned fblocks = (unsigned)((s - 1 + kSplitThreads / 32 - 1) / (kSplitThreads / 32));
        if (!e)
            e = launch_pdl(k_split_fine, dim3(fblocks), dim3(kSplitThreads), 0, st, P, lh, ckl, ckh,
                           pre, sp, n, (uint64_t)S, s);
    }
    return e;
}

template <int kPer>
static cudaError_t launch_pack_t(void (*kern)(const BuildParams *, const Entry *, const SplitRec *,
                                              uint2 *, uint64_t, uint32_t),
                                 uint64_t n, wrs_row *d_rows, unsigned char *ws, const Layout &L,
                                 uint32_t S, cudaStream_t st) {
    const BuildParams *P = reinterpret_cast<const BuildParams *>(ws + L.params);
    const uint32_t smem = pack_smem_bytes(S);
    cudaError_t e = kPer == 8 ? ensure_dynamic_smem<k_pack8>(smem) : ensure_dynamic_smem<k_pack16>(smem);
    if (e) return e;
    const uint32_t threads = (S + kPer - 1) / kPer;   // S is a multiple of 256: whole warps
    return launch_pdl(kern, dim3((unsigned)L.sections), dim3(threads), smem, st, P,
                      reinterpret_cast<const Entry *>(ws + L.lh),
                      reinterpret_cast<const SplitRec *>(ws + L.splits),
                      reinterpret_cast<uint2 *>(d_rows), n, S);
}

cudaError_t launch_pack(uint64_t n, wrs_row *d_rows, unsigned char *ws, const Layout &L,
                        uint32_t S, cudaStream_t st) {
    return pack_per(S) == 8 ? launch_pack_t<8>(k_pack8, n, d_rows, ws, L, S, st)
                            : launch_pack_t<16>(k_pack16, n, d_rows, ws, L, S, st);
}

cudaError_t launch_info(unsigned char *ws, const Layout &L, wrs_build_info *d_info,
                        cudaStream_t st) {
    return launch_pdl(k_info, dim3(1), dim3(1), 0, st,
                      reinterpret_cast<const BuildParams *>(ws + L.params), d_info);
}

}  // namespace wrs
