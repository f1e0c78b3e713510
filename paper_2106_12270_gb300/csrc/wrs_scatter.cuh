// wrs_scatter.cuh - the warp-level stable partition (Sec. 2.2 classify and
// partition, with the prefix sums of Sec. 4 at every 32nd list entry), shared
// by the single-table partition (wrs_build.cu, one warp per sub-segment) and
// the batched build (wrs_batched.cu, one warp per table).
#pragma once

#include "wrs_device.cuh"

namespace wrs {

__device__ __forceinline__ void put_ck(CkRec *ck, uint64_t idx, uint32_t seg, uint64_t v) {
    uint4 r = make_uint4(seg, 0u, (uint32_t)v, (uint32_t)(v >> 32));
    *reinterpret_cast<uint4 *>(ck + idx) = r;
}

struct WarpStage {
    float wv[kChunk + kChunk / 32];     // staged weights (padded, conflict-free)
    Entry e[kChunk + kChunk / 16];      // staged entries in list order (padded)
};

// The interval [mid - half, mid + half] that holds every weight whose clamp
// of q can change: between the light threshold lm and wq (the least weight
// with q >= floor(Q/N) + 1, about (floor(Q/N) + 1/2) 2^-S), widened by a
// relative 2^-16 (far above the FP64 and FP32 rounding of its ends).
__device__ __forceinline__ void threshold_interval(double wq, double lm, float &mid,
                                                   float &half) {
    const double lo = fmin(wq, lm) * (1.0 - 0x1p-16);
    const double hi = fmax(wq, lm) * (1.0 + 0x1p-16);
    mid = (float)(0.5 * (lo + hi));
    half = (float)(0.5 * (hi - lo) * (1.0 + 0x1p-10));
    if (!(lm > 0.0) || !(half > 0.0f) || !(half < INFINITY)) {
        mid = 0.0f;
        half = INFINITY;   // no usable interval: every chunk takes the exact clamps
    }
}

// What a warp's placement reads: the weights and the lists of one table
// (lh, ckl, ckh already offset to the table), and its fixed-point constants.
struct ScatterCtx {
    const float *w;
    uint64_t n;          // items of the table (list positions run 0..n-1)
    Entry *lh;
    CkRec *ckl, *ckh;
    QScale qsc;
    uint64_t Qn;
    float lmax, tmid, thalf;
};

// Place the items [a, b) of a table: lights at l[rank] (entry rank), heavies
// at h[rank] (entry n-1-rank), both in index order; every 32nd list entry
// gets a checkpoint {seg, q sum before it}, the sum counted from item a (the
// caller adds the segment's prefix).  run_l: the global light rank of the
// first light of [a, b).  Returns the clamped q sums of the lights and of the
// heavies placed.
//
// One warp works alone, chunk by chunk (no CTA barrier): classify in input
// order (lane = 16 consecutive items), rank with a warp count scan, stage
// the chunk's entries in list order in the warp's shared memory, then
// compute q once per entry in list order (lane = 16 consecutive slots) with
// one warp scan; checkpoint sums are snapshots of the running sum at the one
// slot per lane where a checkpoint can fall.  The next chunk's weights are
// loaded while the current one is processed.  Full chunks (every chunk but
// the range's last) skip the per-item bounds tests, and those without a
// weight near the light threshold skip the clamps of q.
template <bool kAligned>
__device__ __forceinline__ void scatter_range(const ScatterCtx &X, WarpStage &sm, uint32_t s,
                                              uint64_t a, uint64_t b, uint64_t run_l,
                                              uint64_t &sum_l, uint64_t &sum_h) {
    const int lane = threadIdx.x & 31;
    const float *__restrict__ w = X.w;
    const uint64_t n = X.n;
    const QScale qsc = X.qsc;
    const uint64_t Qn = X.Qn;
    const float lmax = X.lmax, tmid = X.tmid, thalf = X.thalf;
    uint64_t run_h = a - run_l;         // global rank of the next heavy
    uint64_t run_sl = 0, run_sh = 0;    // q sums from item a on
    const int e0 = lane * kPartItems;   // this lane's first item of the chunk
    const int s0 = lane * kPartItems;   // this lane's first list slot
    float4 pv[4];
    auto load_chunk = [&](uint64_t base) {
        const uint64_t lim = n - base;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = r * 128 + lane * 4;
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
    if (a < b) load_chunk(a);
    for (uint64_t base = a; base < b; base += kChunk) {
        const uint64_t lim = b - base;   // items e of the chunk are valid for e < lim
        __syncwarp();                    // previous chunk fully consumed
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = r * 128 + lane * 4;
            sm.wv[pad32(e + 0)] = pv[r].x;
            sm.wv[pad32(e + 1)] = pv[r].y;
            sm.wv[pad32(e + 2)] = pv[r].z;
            sm.wv[pad32(e + 3)] = pv[r].w;
        }
        if (base + kChunk < b) load_chunk(base + kChunk);
        __syncwarp();
        // ---- classify (input order) and count
        const bool full = lim >= (uint64_t)kChunk;   // every chunk but the range's last
        uint32_t lmask = 0, vmask = 0;
        if (full) {
            vmask = (1u << kPartItems) - 1u;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k)
                lmask |= (uint32_t)(sm.wv[pad32(e0 + k)] <= lmax) << k;
        } else {
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                float x = sm.wv[pad32(e0 + k)];
                bool valid = (uint64_t)(e0 + k) < lim;
                vmask |= (uint32_t)valid << k;
                lmask |= (uint32_t)(valid && x <= lmax) << k;
            }
        }
        const uint32_t cnt = __popc(lmask);
        uint32_t icnt = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t c2 = __shfl_up_sync(0xffffffffu, icnt, d);
            if (lane >= d) icnt += c2;
        }
        const uint32_t tl = __shfl_sync(0xffffffffu, icnt, 31);       // lights of the chunk
        const uint32_t tv = lim < (uint64_t)kChunk ? (uint32_t)lim : (uint32_t)kChunk;
        const uint32_t tnh = tv - tl;
        // ---- stage entries in list order: lights at slot rank, heavies at
        // slot kChunk-1-rank
        {
            uint32_t lrank = icnt - cnt;
            uint32_t hslot = kChunk - 1 - ((uint32_t)e0 - lrank);
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const bool lt = (lmask >> k) & 1u;
                const uint32_t slot = lt ? lrank : hslot;
                if (full || ((vmask >> k) & 1u))
                    sm.e[pad16(slot)] = Entry{(uint32_t)(base + e0 + k), sm.wv[pad32(e0 + k)]};
                lrank += lt;
                hslot -= !lt;
            }
        }
        __syncwarp();
        // ---- list-order q pass: slots [s0, s0+16) of this lane
        const uint32_t hstart = kChunk - tnh;   // first heavy slot
        const int cl = (int)((32u - (uint32_t)(run_l & 31u)) & 31u);   // light ckpt slots = cl mod 32
        const int ch = (int)((uint32_t)(run_h + kChunk - 1) & 31u);  // heavy ckpt slots = ch mod 32
        const int kl = (cl - s0) & 31;
        const int kh = (ch - s0) & 31;
        const int kb = (int)tl - s0;
        const uint64_t Qn1 = Qn + 1;
        uint64_t acc = 0, snap_l = 0, snap_h = 0, snap_b = 0;
        // A full chunk with no weight near the light threshold needs no
        // clamp (its lights have q <= Qn, its heavies q > Qn): sum q as is.
        // Otherwise (a partial chunk, or a weight in the threshold
        // interval) the pass applies the clamps.
        bool exact = tv < (uint32_t)kChunk;
        if (!exact) {
            float dmin = INFINITY;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                if (k == kl) snap_l = acc;
                if (k == kb) snap_b = acc;
                const float x = sm.e[pad16(s0 + k)].w;
                dmin = fminf(dmin, fabsf(x - tmid));
                acc += fixed_q(x, qsc);
                if (k == kh) snap_h = acc;    // inclusive of the heavy ckpt slot
            }
            exact = __any_sync(0xffffffffu, dmin <= thalf);
        }
        if (exact) {
            acc = snap_l = snap_h = snap_b = 0;
#pragma unroll
            for (int k = 0; k < kPartItems; ++k) {
                const uint32_t slot = (uint32_t)(s0 + k);
                if (k == kl) snap_l = acc;
                if (k == kb) snap_b = acc;
                const uint64_t q = fixed_q(sm.e[pad16(slot)].w, qsc);
                const uint64_t v = slot < tl ? min(q, Qn) : (slot >= hstart ? max(q, Qn1) : 0ull);
                acc += v;
                if (k == kh) snap_h = acc;    // inclusive of the heavy ckpt slot
            }
        }
        uint64_t inc = acc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        const uint64_t X0 = inc - acc;
        const uint64_t Tall = __shfl_sync(0xffffffffu, inc, 31);
        // q sum of the chunk's lights: from the lane that holds slot tl
        const int owner = tl >= (uint32_t)kChunk ? 31 : (int)(tl / kPartItems);
        uint64_t TLcand = (kb >= 0 && kb < kPartItems) ? X0 + snap_b : Tall;
        const uint64_t TL = tl >= (uint32_t)kChunk ? Tall : __shfl_sync(0xffffffffu, TLcand, owner);
        if (kl < kPartItems && (uint32_t)(s0 + kl) < tl)
            put_ck(X.ckl, (run_l + s0 + kl) >> 5, s, run_sl + X0 + snap_l);
        if (kh < kPartItems && (uint32_t)(s0 + kh) >= hstart)
            put_ck(X.ckh, (run_h + kChunk - 1 - (s0 + kh)) >> 5, s, run_sh + (Tall - X0 - snap_h));
        // ---- coalesced copy-out
        uint2 *lh2 = reinterpret_cast<uint2 *>(X.lh);
        const uint2 *e2 = reinterpret_cast<const uint2 *>(sm.e);
        // two entries in flight per lane
        for (uint32_t q = lane; q < tl; q += 64) {
            const uint2 v0 = e2[pad16(q)];
            const bool two = q + 32 < tl;
            const uint2 v1 = two ? e2[pad16(q + 32)] : v0;
            lh2[run_l + q] = v0;
            if (two) lh2[run_l + q + 32] = v1;
        }
        for (uint32_t q = lane; q < tnh; q += 64) {
            const uint2 v0 = e2[pad16(kChunk - 1 - q)];
            const bool two = q + 32 < tnh;
            const uint2 v1 = two ? e2[pad16(kChunk - 1 - (q + 32))] : v0;
            lh2[n - 1 - (run_h + q)] = v0;
            if (two) lh2[n - 1 - (run_h + q + 32)] = v1;
        }
        run_l += tl;
        run_h += tnh;
        run_sl += TL;
        run_sh += Tall - TL;
    }
    sum_l = run_sl;
    sum_h = run_sh;
}

}  // namespace wrs
