// wrs_build.cu - alias-table construction on GB300 (sm_103a).
//
// The PSA method (Sec. 2.2, Sec. 4 of "Weighted Random Sampling on GPUs")
// in four kernels, with integer fixed-point prefix sums:
//
//   k_sum / k_total      a1: W = sum w_i, exact (per-exponent-band integer
//                        sums), rounded once to FP64; avg = W/N; the scale S
//                        of the fixed point q_i = round(w_i 2^S).
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
// sum of the first j heavy e' (both < 2^94).  The sweep closes heavy h[j]
// (its remaining weight fits in one bucket) iff E'(j+1) <= D'(i), else light
// l[i]; a heavy row keeps 1 - (D'(i) - E'(j+1)) / Q of its bucket.  All of it
// is exact integer arithmetic: the splits and every section end agree
// exactly, and no FP64 unit is used per item.  The rounding of q costs at
// most N/(2Q) <= 2^-32 of a bucket per item, far below the FP32 rounding of
// the stored probabilities.
#include <stdio.h>

#include "wrs_device.cuh"

namespace wrs {

Layout make_layout(uint64_t n, uint32_t S) {
    Layout L;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    L.ntiles = (n + kTile - 1) / kTile;
    L.sections = (n + S - 1) / S;
    L.params = take(sizeof(BuildParams));
    L.sum_bins = take((uint64_t)kSumMaxBlocks * kBands * sizeof(u128));
    L.seg_cnt = take((uint64_t)kMaxSegs * 4);
    L.seg_q = take((uint64_t)kMaxSegs * 8);
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

// Each FP32 weight m * 2^(e'-150) (e' = max(biased exponent, 1)) goes into
// band e'/24 as m << (e' mod 24) < 2^47.  A thread sees at most 2^15 items,
// so its per-band sum stays below 2^62; blocks reduce to 128-bit sums.
__global__ void __launch_bounds__(kSumThreads)
k_sum(const float *__restrict__ w, uint64_t n, u128 *__restrict__ bins_out,
      BuildParams *__restrict__ P, int aligned) {
    __shared__ uint64_t bins[kBands][kSumThreads];
    const int tid = threadIdx.x;
#pragma unroll
    for (int b = 0; b < kBands; ++b) bins[b][tid] = 0;
    uint32_t bad = 0;
    auto add = [&](float x) {
        uint32_t band;
        uint64_t val;
        band_of(x, band, val, bad);
        bins[band][tid] += val;
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
    for (int b = warp; b < kBands; b += kSumThreads / 32) {
        u128 s = 0;
#pragma unroll
        for (int k = 0; k < kSumThreads / 32; ++k) s += bins[b][lane + 32 * k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)s, d);
            uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(s >> 64), d);
            s += ((u128)hi << 64) | lo;
        }
        if (lane == 0) bins_out[(uint64_t)blockIdx.x * kBands + b] = s;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicOr(&P->status, bad);
}

// kBands warps: warp b reduces band b over the blocks; thread 0 then
// assembles W exactly (units of 2^-150), rounds it to FP64 (ties to even)
// and derives avg, the light threshold and the fixed-point scale.
__global__ void __launch_bounds__(32 * kBands)
k_total(const u128 *__restrict__ bins_in, int nblocks, uint64_t n, uint32_t sections,
        BuildParams *__restrict__ P) {
    __shared__ u128 band[kBands];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        u128 s = 0;
        for (int b = lane; b < nblocks; b += 32) s += bins_in[(uint64_t)b * kBands + warp];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)s, d);
            uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(s >> 64), d);
            s += ((u128)hi << 64) | lo;
        }
        if (lane == 0) band[warp] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    P->n = n;
    P->sections = sections;
    double W;
    int top;
    if (!exact_total(band, W, top)) {
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
// a2 + a3: classify, stable partition, prefix sums (decoupled look-back)
// ===========================================================================


// Segment g of G covers tiles [g*T/G, (g+1)*T/G) of kTile items.
__device__ __forceinline__ void seg_tiles(uint32_t g, uint32_t G, uint64_t T, uint64_t &t0,
                                          uint64_t &t1) {
    t0 = (uint64_t)g * T / G;
    t1 = (uint64_t)(g + 1) * T / G;
}

// Block-wide sum of one uint32 per thread (blockDim.x a multiple of 32).
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0u;
        t = __reduce_add_sync(0xffffffffu, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    uint32_t r = red[0];
    __syncthreads();
    return r;
}

// Per segment (one CTA each, coalesced 16-byte loads): the number of light
// items and the sum of q over all items (light and heavy, unclamped).
__global__ void __launch_bounds__(kPartThreads)
k_count(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
        uint32_t *__restrict__ seg_cnt, uint64_t *__restrict__ seg_q, uint64_t T, uint32_t G,
        int aligned) {
    __shared__ uint32_t red[32];
    __shared__ uint64_t redq[32];
    if (P->status) return;
    const float lmax = P->light_max;
    const int qshift = P->qshift;
    uint64_t t0, t1;
    seg_tiles(blockIdx.x, G, T, t0, t1);
    const uint64_t a = t0 * kTile, b = min(t1 * kTile, n);
    uint32_t cnt = 0;
    uint64_t qs = 0;
    uint64_t tail = a;
    if (aligned) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        const uint64_t b4 = b / 4;
#pragma unroll 4
        for (uint64_t i = a / 4 + threadIdx.x; i < b4; i += kPartThreads) {
            float4 v = __ldg(w4 + i);
            cnt += (v.x <= lmax) + (v.y <= lmax) + (v.z <= lmax) + (v.w <= lmax);
            qs += fixed_q(v.x, qshift) + fixed_q(v.y, qshift) + fixed_q(v.z, qshift) +
                  fixed_q(v.w, qshift);
        }
        tail = b4 * 4 > a ? b4 * 4 : a;
    }
    for (uint64_t i = tail + threadIdx.x; i < b; i += kPartThreads) {
        float x = __ldg(w + i);
        cnt += (x <= lmax);
        qs += fixed_q(x, qshift);
    }
    // block sums (q: each thread's sum < 2^63, the segment's too)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, d);
    if (lane == 0) redq[warp] = qs;
    cnt = block_sum_u32(cnt, red);
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int k = 0; k < kPartThreads / 32; ++k) t += redq[k];
        seg_cnt[blockIdx.x] = cnt;
        seg_q[blockIdx.x] = t;
    }
}

// One CTA: Q = sum of all q (the bucket in fixed point) and its derived
// constants.
__global__ void __launch_bounds__(kMaxSegs)
k_qsum(BuildParams *__restrict__ P, const uint64_t *__restrict__ seg_q, uint32_t G, uint64_t n) {
    __shared__ uint64_t red[32];
    if (P->status) return;
    uint64_t v = threadIdx.x < G ? seg_q[threadIdx.x] : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x != 0) return;
    uint64_t Q = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) Q += red[k];
    P->Q = Q;
    P->Qn = Q / n;
    P->NQn = (u128)P->Qn * n;
    P->NQn1 = P->NQn + n;
    P->Qf = __ull2float_rn(Q);
    P->invQ = __frcp_rn(P->Qf);
    P->nseg = G;
}

struct ScatterShared {
    float wv[kTile + kTile / 32];       // staged weights (padded, conflict-free)
    Entry e[kTile + kTile / 16];        // staged entries in list order (padded)
    uint64_t wsum[kPartThreads / 32];   // per-warp q totals of the list-order pass
    uint32_t wnl[kPartThreads / 32];    // per-warp light counts
    uint64_t tile_l;                    // q sum of the tile's lights
    uint64_t run_sl, run_sh;            // segment-local q sums before the tile
    uint64_t run_l;                     // global light rank of the tile's first light
    uint32_t red[32];
};

__device__ __forceinline__ void put_ck(CkRec *ck, uint64_t idx, uint32_t seg, uint64_t v) {
    uint4 r = make_uint4(seg, 0u, (uint32_t)v, (uint32_t)(v >> 32));
    *reinterpret_cast<uint4 *>(ck + idx) = r;
}

// Place every item of the segment: lights at l[rank] (entry rank), heavies at
// h[rank] (entry n-1-rank); both stay in index order.  Every 32nd list entry
// gets a checkpoint of the q sum before it (segment-relative).
//
// Per tile: classify in input order (lane = 16 consecutive items), rank with
// a count scan, stage the entries in list order, then compute q once per
// entry in list order (thread = 16 consecutive slots, so light and heavy
// slots rarely share a thread) with one block scan; the checkpoint sums are
// snapshots of the running sum at the one slot per thread where a
// checkpoint can fall.
template <bool kAligned>
__global__ void __launch_bounds__(kPartThreads, 3)
k_scatter(const float *__restrict__ w, uint64_t n, const BuildParams *__restrict__ P,
          const uint32_t *__restrict__ seg_cnt, Entry *__restrict__ lh, CkRec *__restrict__ ckl,
          CkRec *__restrict__ ckh, SegVal *__restrict__ seg_sum, uint64_t T, uint32_t G) {
    __shared__ ScatterShared sm;
    if (P->status) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t g = blockIdx.x;
    uint64_t t0, t1;
    seg_tiles(g, G, T, t0, t1);
    const int qshift = P->qshift;
    const uint64_t Qn = P->Qn;
    const float lmax = P->light_max;

    uint32_t pre = 0;
    for (uint32_t k = tid; k < g; k += kPartThreads) pre += seg_cnt[k];
    pre = block_sum_u32(pre, sm.red);
    if (tid == 0) {
        sm.run_l = pre;
        sm.run_sl = 0;
        sm.run_sh = 0;
    }

    const int wbase = warp * 512;
    const int e0 = wbase + lane * kPartItems;   // this lane's first item of the tile
    const int s0 = tid * kPartItems;            // this thread's first list slot
    // coalesced 16-byte loads of one tile (the next tile is loaded while the
    // current one is processed)
    float4 pv[4];
    auto load_tile = [&](uint64_t tile) {
        const uint64_t base = tile * kTile;
        const uint64_t lim = n - base;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = wbase + r * 128 + lane * 4;
            if (kAligned && (uint64_t)e + 3 < lim) {
                pv[r] = __ldcs(reinterpret_cast<const float4 *>(w + base + e));
            } else {
                pv[r].x = (uint64_t)e + 0 < lim ? w[base + e + 0] : 0.f;
                pv[r].y = (uint64_t)e + 1 < lim ? w[base + e + 1] : 0.f;
                pv[r].z = (uint64_t)e + 2 < lim ? w[base + e + 2] : 0.f;
                pv[r].w = (uint64_t)e + 3 < lim ? w[base + e + 3] : 0.f;
            }
        }
    };
    if (t0 < t1) load_tile(t0);
    for (uint64_t tile = t0; tile < t1; ++tile) {
        const uint64_t base = tile * kTile;
        const uint64_t lim = n - base;   // items e of the tile are valid for e < lim
        __syncthreads();                 // previous tile fully consumed
        // ---- padded transpose to blocked, then start loading the next tile
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = wbase + r * 128 + lane * 4;
            sm.wv[pad32(e + 0)] = pv[r].x;
            sm.wv[pad32(e + 1)] = pv[r].y;
            sm.wv[pad32(e + 2)] = pv[r].z;
            sm.wv[pad32(e + 3)] = pv[r].w;
        }
        if (tile + 1 < t1) load_tile(tile + 1);
        __syncwarp();
        // ---- classify (input order) and count
        uint32_t lmask = 0, vmask = 0;
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            float x = sm.wv[pad32(e0 + k)];
            bool valid = (uint64_t)(e0 + k) < lim;
            vmask |= (uint32_t)valid << k;
            lmask |= (uint32_t)(valid && x <= lmax) << k;
        }
        const uint32_t cnt = __popc(lmask);
        uint32_t icnt = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t c2 = __shfl_up_sync(0xffffffffu, icnt, d);
            if (lane >= d) icnt += c2;
        }
        if (lane == 31) sm.wnl[warp] = icnt;
        __syncthreads();
        uint32_t wl = 0, tl = 0;
#pragma unroll
        for (int k = 0; k < kPartThreads / 32; ++k) {
            uint32_t c = sm.wnl[k];
            wl += (k < warp) ? c : 0u;
            tl += c;
        }
        const uint64_t run_l = sm.run_l;
        const uint64_t run_h = base - run_l;
        const uint32_t tv = lim < (uint64_t)kTile ? (uint32_t)lim : (uint32_t)kTile;
        const uint32_t tnh = tv - tl;
        // ---- stage entries in list order: lights at slot rank, heavies at
        // slot kTile-1-rank
        {
            uint32_t lrank = wl + icnt - cnt;
            uint32_t hrank = (uint32_t)e0 - lrank;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                if (!((vmask >> k) & 1u)) break;
                Entry en{(uint32_t)(base + e0 + k), sm.wv[pad32(e0 + k)]};
                if ((lmask >> k) & 1u) sm.e[pad16(lrank++)] = en;
                else sm.e[pad16(kTile - 1 - hrank++)] = en;
            }
        }
        __syncthreads();
        // ---- list-order q pass: slots [s0, s0+16) of this thread
        const uint32_t hstart = kTile - tnh;   // first heavy slot
        const int cl = (int)((32u - (uint32_t)(run_l & 31u)) & 31u);   // light ckpt slots = cl mod 32
        const int ch = (int)((uint32_t)(run_h + kTile - 1) & 31u);   // heavy ckpt slots = ch mod 32
        const int kl = (cl - s0) & 31;    // local index of this thread's light ckpt slot (if < 16)
        const int kh = (ch - s0) & 31;
        const int kb = (int)tl - s0;      // local index of the light/heavy boundary
        uint64_t acc = 0, snap_l = 0, snap_h = 0, snap_b = 0;
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            uint32_t slot = (uint32_t)(s0 + k);
            if (k == kl) snap_l = acc;
            if (k == kb) snap_b = acc;
            uint64_t v = 0;
            if (slot < tl) v = light_q(sm.e[pad16(slot)].w, qshift, Qn);
            else if (slot >= hstart) v = heavy_q(sm.e[pad16(slot)].w, qshift, Qn);
            acc += v;
            if (k == kh) snap_h = acc;    // inclusive of the heavy ckpt slot
        }
        // block exclusive scan of the thread totals
        uint64_t inc = acc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        if (lane == 31) sm.wsum[warp] = inc;
        __syncthreads();
        uint64_t X = inc - acc, Tall = 0;
#pragma unroll
        for (int k = 0; k < kPartThreads / 32; ++k) {
            uint64_t c = sm.wsum[k];
            X += (k < warp) ? c : 0ull;
            Tall += c;
        }
        if (kb >= 0 && kb < kPartItems) sm.tile_l = X + snap_b;
        if (tl == (uint32_t)kTile && tid == 0) sm.tile_l = Tall;
        const uint64_t run_sl = sm.run_sl, run_sh = sm.run_sh;
        if (kl < kPartItems && (uint32_t)(s0 + kl) < tl)
            put_ck(ckl, (run_l + s0 + kl) >> 5, g, run_sl + X + snap_l);
        if (kh < kPartItems && (uint32_t)(s0 + kh) >= hstart)
            put_ck(ckh, (run_h + kTile - 1 - (s0 + kh)) >> 5, g, run_sh + (Tall - X - snap_h));
        // ---- coalesced copy-out
        uint2 *lh2 = reinterpret_cast<uint2 *>(lh);
        const uint2 *e2 = reinterpret_cast<const uint2 *>(sm.e);
        for (uint32_t a = tid; a < tl; a += kPartThreads) lh2[run_l + a] = e2[pad16(a)];
        for (uint32_t b = tid; b < tnh; b += kPartThreads)
            lh2[n - 1 - (run_h + b)] = e2[pad16(kTile - 1 - b)];
        __syncthreads();   // tile_l written
        if (tid == 0) {
            uint64_t TL = sm.tile_l;
            sm.run_l = run_l + tl;
            sm.run_sl = run_sl + TL;
            sm.run_sh = run_sh + (Tall - TL);
        }
    }
    __syncthreads();
    if (tid == 0) {
        SegVal v;
        v.sl = sm.run_sl;
        v.sh = sm.run_sh;
        v.nl = 0;
        v.pad = 0;
        seg_sum[g] = v;
    }
}

// One CTA: exclusive scan over the segments of (light count, light q sum,
// heavy q sum); totals nl, nh, D'(nl), E'(nh); the checkpoints that fall on
// the very end of a list.
__global__ void __launch_bounds__(kMaxSegs)
k_segscan(BuildParams *__restrict__ P, const uint32_t *__restrict__ seg_cnt,
          const SegVal *__restrict__ seg_sum, SegVal *__restrict__ seg_pre,
          CkRec *__restrict__ ckl, CkRec *__restrict__ ckh, uint64_t n, uint32_t G) {
    __shared__ uint64_t wc[kMaxSegs / 32], wl[kMaxSegs / 32], wh[kMaxSegs / 32];
    if (P->status) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t c = 0, sl = 0, sh = 0;
    if ((uint32_t)tid < G) {
        c = seg_cnt[tid];
        sl = (uint64_t)seg_sum[tid].sl;
        sh = (uint64_t)seg_sum[tid].sh;
    }
    uint64_t ic = c, isl = sl, ish = sh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t c2 = __shfl_up_sync(0xffffffffu, ic, d);
        uint64_t a2 = __shfl_up_sync(0xffffffffu, isl, d);
        uint64_t b2 = __shfl_up_sync(0xffffffffu, ish, d);
        if (lane >= d) { ic += c2; isl += a2; ish += b2; }
    }
    if (lane == 31) {
        wc[warp] = ic;
        wl[warp] = isl;
        wh[warp] = ish;
    }
    __syncthreads();
    uint64_t pc = ic - c, psl = isl - sl, psh = ish - sh;
    for (int k = 0; k < warp; ++k) {
        pc += wc[k];
        psl += wl[k];
        psh += wh[k];
    }
    if ((uint32_t)tid <= G) {
        SegVal v;
        v.sl = psl;
        v.sh = psh;
        v.nl = pc;
        v.pad = 0;
        seg_pre[tid] = v;
    }
    if ((uint32_t)tid == G) {
        // thread G holds the totals (its own value is zero)
        const uint64_t Q = P->Q;
        const uint64_t nl = pc, nh = n - nl;
        P->nl = nl;
        P->nh = nh;
        P->Dtot = (u128)nl * Q - (u128)psl * n;
        P->Etot = (u128)psh * n - (u128)nh * Q;
        if ((nl & 31u) == 0) put_ck(ckl, nl >> 5, G, 0);
        if ((nh & 31u) == 0) put_ck(ckh, nh >> 5, G, 0);
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
    return ck_E(C, (k - i) >> 5) <= ck_D(C, c);
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
                           SplitRec *out, int lane) {
    uint64_t lo = k > C.nh ? k - C.nh : 0;
    uint64_t hi = k < C.nl ? k : C.nl;
    const uint32_t N = (uint32_t)C.n;
    uint64_t ans;
    u128 Dv, Ev;
    if (c == 0) {
        ans = 0;
        Dv = 0;
        Ev = ck_E(C, k >> 5);
    } else {
        uint64_t lb = 32 * (c - 1);  // light base
        uint64_t hb = k - 32 * c;    // heavy base, multiple of 32
        u128 d = 0, e = 0;
        if (lb + lane < C.nl) {
            Entry en = C.lh[lb + lane];
            d = (u128)(Pm.Q - N * light_q(en.w, Pm.qshift, Pm.Qn));   // <= Q
        }
        if (hb + lane < C.nh) {
            Entry en = C.lh[C.n - 1 - (hb + lane)];
            e = mul_nq(N, heavy_q(en.w, Pm.qshift, Pm.Qn)) - Pm.Q;
        }
        u128 dinc = d, einc = e;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            u128 a = shfl_up_u128(dinc, s), b = shfl_up_u128(einc, s);
            if (lane >= s) { dinc += a; einc += b; }
        }
        u128 eexc = einc - e;
        u128 Dbase = ck_D(C, c - 1);
        u128 Ebase = ck_E(C, hb >> 5);
        u128 Dl = Dbase + dinc;                                   // D'(lb + 1 + lane)
        u128 Eh = Ebase + shfl_u128(eexc, 31 - lane);             // E'(k - (lb + 1 + lane))
        uint64_t i = lb + 1 + lane;
        bool ok = i >= lo && i <= hi && (i == hi || Eh <= Dl);
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
    __shared__ uint64_t s_c[kSplitThreads];
    __shared__ unsigned long long s_a, s_b;
    __shared__ int s_go;
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
    }
    s_c[tid] = a;
    __syncthreads();
    // fine phase: each warp handles its 32 splits one after another
    const int warp = tid >> 5, lane = tid & 31;
    for (int q = 0; q < 32; ++q) {
        int st = warp * 32 + q;
        uint64_t tt = t0 + st;
        if (tt >= sections) break;
        split_fine(C, Pm, tt * S, s_c[st], splits + tt, lane);
    }
    (void)s_go;
}

// Splits 0 and s (the whole table's ends).
__global__ void k_split_ends(const BuildParams *__restrict__ P, SplitRec *__restrict__ splits,
                             uint32_t sections) {
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

// Shared memory of one pack CTA for a section of up to S buckets:
//   P[K+1] (u128 prefix of the section's d' (lights first) then e'
//   (heavies), one pad slot every 8 entries against bank conflicts),
//   item[K+1] (uint32), w[K+1 padded] (float).
__host__ __device__ inline uint32_t pack_p_slots(uint32_t S) { return S + 1 + (S + 1) / 8 + 1; }
__host__ __device__ inline uint32_t pack_smem_bytes(uint32_t S) {
    uint32_t K1 = S + 1;
    uint32_t b = 16 * pack_p_slots(S);          // P
    b += 4 * K1;                                // item
    b += 4 * (K1 + K1 / 32 + 1);                // w (padded)
    return (b + 15) & ~15u;
}

__device__ __forceinline__ uint32_t pp8(uint32_t e) { return e + (e >> 3); }

__global__ void __launch_bounds__(kPackThreads)
k_pack(const BuildParams *__restrict__ P, const Entry *__restrict__ lh,
       const SplitRec *__restrict__ splits, uint2 *__restrict__ rows, uint64_t n,
       uint32_t S) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (P->status) return;
    const uint32_t K1 = S + 1;
    u128 *sP = reinterpret_cast<u128 *>(smem);
    uint32_t *sItem = reinterpret_cast<uint32_t *>(smem + 16 * pack_p_slots(S));
    float *sW = reinterpret_cast<float *>(smem + 16 * pack_p_slots(S) + 4 * K1);

    const int tid = threadIdx.x;
    const uint32_t t = blockIdx.x;
    const uint64_t nh = P->nh;
    const uint64_t Q = P->Q, Qn = P->Qn;
    const uint32_t N = (uint32_t)n;
    const int qshift = P->qshift;
    const float inv_avg = P->inv_avg, invQ = P->invQ;
    const SplitRec R0 = splits[t], R1 = splits[t + 1];
    const uint32_t i0 = R0.i, j0 = R0.j;
    const uint32_t L = R1.i - R0.i, H = R1.j - R0.j, K = L + H;
    const uint32_t extra = (R1.j < nh) ? 1u : 0u;
    const u128 D0 = R0.D, E0 = R0.E;
    if (R1.i < R0.i || R1.j < R0.j || K > S || R1.i > P->nl || R1.j > nh) {
        if (tid == 0) atomicOr(const_cast<uint32_t *>(&P->status), ERR_INTERNAL);
        return;   // inconsistent splits: write nothing
    }

    // phase 1: coalesced load of the section's lights, heavies and the next
    // heavy item (the alias of the last rows)
    for (uint32_t e = tid; e < K + extra; e += kPackThreads) {
        Entry en = (e < L) ? lh[(uint64_t)i0 + e] : lh[n - 1 - ((uint64_t)j0 + (e - L))];
        sItem[e] = en.item;
        sW[pad32(e)] = en.w;
    }
    __syncthreads();

    // phase 2: blocked values (d' for lights, e' for heavies) written to
    // P[e+1], then a block exclusive scan in place: P[e] = sum of values < e
    const uint32_t per = (S + kPackThreads - 1) / kPackThreads;
    const uint32_t b0 = tid * per;
    u128 run = 0;
    for (uint32_t k = 0; k < per; ++k) {
        uint32_t e = b0 + k;
        if (e >= K) break;
        float wv = sW[pad32(e)];
        u128 val = (e < L) ? (u128)(Q - (uint64_t)N * light_q(wv, qshift, Qn))
                           : mul_nq(N, heavy_q(wv, qshift, Qn)) - Q;
        sP[pp8(e + 1)] = val;
        run += val;
    }
    __shared__ u128 s_wsum[kPackThreads / 32];
    const int warp = tid >> 5, lane = tid & 31;
    u128 inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u128 o = shfl_up_u128(inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    u128 pre = inc - run;
    for (int k = 0; k < warp; ++k) pre += s_wsum[k];
    if (tid == 0) sP[0] = 0;
    for (uint32_t k = 0; k < per; ++k) {
        uint32_t e = b0 + k;
        if (e >= K) break;
        pre += sP[pp8(e + 1)];
        sP[pp8(e + 1)] = pre;
    }
    __syncthreads();

    // phase 3: merge path.  A(x) = D'(i0+x) = D0 + P[x] (x <= L);
    // B(y) = E'(j0+y+1) = E0 + P[L+y+1] - P[L] (y < H).
    const u128 PL = sP[pp8(L)];
    auto Av = [&](uint32_t x) { return D0 + sP[pp8(x)]; };
    auto Bv = [&](uint32_t y) { return E0 + (sP[pp8(L + y + 1)] - PL); };
    const uint32_t d0 = b0;
    if (d0 >= K) return;
    uint32_t lo = d0 > H ? d0 - H : 0, hi = d0 < L ? d0 : L;
    while (lo < hi) {   // smallest x with (d0-x == 0) || x == L || B(d0-x-1) <= A(x)
        uint32_t m = (lo + hi) >> 1;
        bool p = (d0 - m == 0) || (m == L) || (Bv(d0 - m - 1) <= Av(m));
        if (p) hi = m;
        else lo = m + 1;
    }
    uint32_t x = lo, y = d0 - lo;
    u128 a = Av(x);                 // D'(i0 + x)
    u128 b = y < H ? Bv(y) : 0;     // E'(j0 + y + 1)
    const uint32_t dend = min(d0 + per, K);
    for (uint32_t d = d0; d < dend; ++d) {
        bool heavy = (y < H) && (x == L || b <= a);
        uint32_t item, alias;
        float prob;
        if (heavy) {
            item = sItem[L + y];
            if ((uint64_t)j0 + y + 1 < nh) {
                if (b > a) {
                    prob = 1.0f;      // rounding left more excess than deficit
                } else {
                    uint64_t delta = (uint64_t)(a - b);   // < Q < 2^63
                    prob = fminf(fmaxf(1.0f - __ull2float_rn(delta) * invQ, 0.0f), 1.0f);
                }
                alias = sItem[L + y + 1];
            } else {
                prob = 1.0f;          // last heavy item keeps its whole bucket
                alias = item;
            }
            ++y;
            if (y < H) b = Bv(y);
        } else {
            item = sItem[x];
            if ((uint64_t)j0 + y < nh) {
                prob = fminf(sW[pad32(x)] * inv_avg, 1.0f);
                alias = sItem[L + y];
            } else {
                prob = 1.0f;          // no heavy item left to fill the bucket
                alias = item;
            }
            ++x;
            a = Av(x);
        }
        rows[item] = make_uint2(__float_as_uint(prob), alias);
    }
}

// ===========================================================================
// build summary
// ===========================================================================
__global__ void k_info(const BuildParams *__restrict__ P, wrs_build_info *__restrict__ out) {
    uint32_t st = P->status;
    wrs_build_info r;
    r.status = (st & ERR_NONFINITE) ? WRS_ENONFINITE
             : (st & (ERR_NEGATIVE | ERR_INTERNAL)) ? WRS_EINVAL
             : (st & ERR_ZEROSUM) ? WRS_EZEROSUM
             : (st & ERR_TIMEOUT) ? WRS_ETIMEOUT : WRS_OK;
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

static int g_num_sms = 0;
int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 152;
    }
    return g_num_sms;
}

cudaError_t launch_total(const float *d_w, uint64_t n, unsigned char *ws, const Layout &L,
                         cudaStream_t st) {
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    cudaError_t err = cudaMemsetAsync(P, 0, sizeof(BuildParams), st);
    if (err) return err;
    uint64_t want = (n + 4095) / 4096;
    int blocks = (int)(want < (uint64_t)kSumMaxBlocks ? (want ? want : 1) : kSumMaxBlocks);
    int aligned = ((uintptr_t)d_w % 16) == 0;
    k_sum<<<blocks, kSumThreads, 0, st>>>(d_w, n, reinterpret_cast<u128 *>(ws + L.sum_bins), P,
                                           aligned);
    k_total<<<1, 32 * kBands, 0, st>>>(reinterpret_cast<const u128 *>(ws + L.sum_bins), blocks, n,
                              (uint32_t)L.sections, P);
    return cudaGetLastError();
}

uint32_t num_segments(const Layout &L) {
    uint64_t g = (uint64_t)num_sms() * kSegPerSM;
    if (g > (uint64_t)kMaxSegs - 1) g = kMaxSegs - 1;
    if (g > L.ntiles) g = L.ntiles;
    return (uint32_t)(g ? g : 1);
}

cudaError_t launch_partition(const float *d_w, uint64_t n, unsigned char *ws, const Layout &L,
                             cudaStream_t st) {
    BuildParams *P = reinterpret_cast<BuildParams *>(ws + L.params);
    auto *cnt = reinterpret_cast<uint32_t *>(ws + L.seg_cnt);
    auto *segq = reinterpret_cast<uint64_t *>(ws + L.seg_q);
    auto *sum = reinterpret_cast<SegVal *>(ws + L.seg_sum);
    auto *pre = reinterpret_cast<SegVal *>(ws + L.seg_pre);
    auto *lh = reinterpret_cast<Entry *>(ws + L.lh);
    auto *ckl = reinterpret_cast<CkRec *>(ws + L.ckl);
    auto *ckh = reinterpret_cast<CkRec *>(ws + L.ckh);
    const uint32_t G = num_segments(L);
    const int aligned = ((uintptr_t)d_w % 16) == 0;
    k_count<<<G, kPartThreads, 0, st>>>(d_w, n, P, cnt, segq, L.ntiles, G, aligned);
    k_qsum<<<1, kMaxSegs, 0, st>>>(P, segq, G, n);
    if (aligned)
        k_scatter<true><<<G, kPartThreads, 0, st>>>(d_w, n, P, cnt, lh, ckl, ckh, sum, L.ntiles, G);
    else
        k_scatter<false><<<G, kPartThreads, 0, st>>>(d_w, n, P, cnt, lh, ckl, ckh, sum, L.ntiles, G);
    k_segscan<<<1, kMaxSegs, 0, st>>>(P, cnt, sum, pre, ckl, ckh, n, G);
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
    k_split_ends<<<1, 1, 0, st>>>(P, sp, s);
    if (s > 1) {
        unsigned blocks = (unsigned)((s - 1 + kSplitThreads - 1) / kSplitThreads);
        if (method == WRS_SPLIT_BINARY)
            k_split<false><<<blocks, kSplitThreads, 0, st>>>(P, lh, ckl, ckh, pre, sp, n, S, s);
        else
            k_split<true><<<blocks, kSplitThreads, 0, st>>>(P, lh, ckl, ckh, pre, sp, n, S, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(uint64_t n, wrs_row *d_rows, unsigned char *ws, const Layout &L,
                        uint32_t S, cudaStream_t st) {
    const BuildParams *P = reinterpret_cast<const BuildParams *>(ws + L.params);
    uint32_t smem = pack_smem_bytes(S);
    static uint32_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_pack, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e) return e;
        configured = smem;
    }
    k_pack<<<(unsigned)L.sections, kPackThreads, smem, st>>>(
        P, reinterpret_cast<const Entry *>(ws + L.lh),
        reinterpret_cast<const SplitRec *>(ws + L.splits), reinterpret_cast<uint2 *>(d_rows), n,
        S);
    return cudaGetLastError();
}

cudaError_t launch_info(unsigned char *ws, const Layout &L, wrs_build_info *d_info,
                        cudaStream_t st) {
    k_info<<<1, 1, 0, st>>>(reinterpret_cast<const BuildParams *>(ws + L.params), d_info);
    return cudaGetLastError();
}

}  // namespace wrs
